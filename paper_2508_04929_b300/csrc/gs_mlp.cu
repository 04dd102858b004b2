// Point-MLP of the learned warm start: training and inference kernels (BF16 operands,
// FP32 accumulation).  Not part of the paper (arXiv 2508.04929), whose reconstructions start
// from a random initialization (Sec. 4.1).
//
// Network: Z1 = X W1^T + b1, H1 = relu(Z1), Z2 = H1 W2^T + b2, H2 = relu(Z2),
// Y = H2 W3^T + b3.  Every product rounds both operands to bfloat16 (nearest even) and
// accumulates in FP32; biases, pre-activations and gradients are FP32.  The layers are
// (n x <=128) x (<=128 x <=128) contractions, a few GFLOP per training step, so they run on
// the FP32 pipe: each operand is rounded once while it is staged into shared memory (kept
// as an FP32 whose low 16 bits are zero), and the inner loops are plain FMAs over
// register tiles.
#include <cuda_bf16.h>

#include "gs_internal.cuh"

namespace gs {
namespace {

constexpr int kMaxWidth = 128;
constexpr int kDenseThreads = 256;
constexpr int kRows = 8;  // samples per thread per tile in k_dense

__device__ __forceinline__ float bf(float x) { return __bfloat162float(__float2bfloat16_rn(x)); }

__host__ __device__ inline int round4(int x) { return (x + 3) & ~3; }
__host__ __device__ inline int round32(int x) { return (x + 31) & ~31; }

// out[s][o] = epilogue(sum_i bf(in[row(s)][i]) bf(M[o][i])) for o < n_out, where M is the
// weight matrix W[n_out][k_in] (transpose = 0) or the transpose of W[k_in][n_out]
// (transpose = 1, the data backward).  row(s) = idx[s] if idx is given.
//   mode 0 (forward):   z = acc + bias[o]; if (pre) pre[s][o] = z; out = relu ? max(z, 0) : z
//   mode 1 (backward):  g = acc; if (mask) g = mask[s][o] > 0 ? g : 0; out = g
// Persistent: each CTA stages M once and walks sample tiles.  Threads form groups of
// round32(n_out) (one output each) and every group owns kRows samples of the tile.
__global__ void __launch_bounds__(kDenseThreads) k_dense(const float* __restrict__ in, const int* __restrict__ idx,
                                                          int n, int k_in, const float* __restrict__ Wm, int transpose,
                                                          int n_out, const float* __restrict__ bias, int mode,
                                                          int relu, const float* __restrict__ mask,
                                                          float* __restrict__ pre, float* __restrict__ out) {
  extern __shared__ float4 smem4[];
  float* sm = reinterpret_cast<float*>(smem4);
  const int k4 = round4(k_in);
  const int ldw = k4 + 4;  // padded row stride: conflict-free 16-byte loads
  const int outw = round32(n_out);
  const int groups = kDenseThreads / outw;
  const int tile = groups * kRows;
  float* Ms = sm;                       // [outw][ldw]
  float* Xs = sm + (size_t)outw * ldw;  // [tile][k4]
  for (int e = threadIdx.x; e < outw * ldw; e += blockDim.x) {
    const int o = e / ldw, i = e - o * ldw;
    float v = 0.f;
    if (o < n_out && i < k_in) v = transpose ? Wm[(size_t)i * n_out + o] : Wm[(size_t)o * k_in + i];
    Ms[e] = bf(v);
  }
  const int o = threadIdx.x % outw, g = threadIdx.x / outw;
  const bool active = g < groups;
  const float b = (mode == 0 && o < n_out && bias) ? bias[o] : 0.f;
  const float4* mrow = reinterpret_cast<const float4*>(Ms + (size_t)o * ldw);
  for (int s0 = blockIdx.x * tile; s0 < n; s0 += gridDim.x * tile) {
    __syncthreads();
    for (int e = threadIdx.x; e < tile * k4; e += blockDim.x) {
      const int s = e / k4, i = e - s * k4;
      float v = 0.f;
      if (s0 + s < n && i < k_in) {
        const long long r = idx ? (long long)idx[s0 + s] : (long long)(s0 + s);
        v = in[r * k_in + i];
      }
      Xs[e] = bf(v);
    }
    __syncthreads();
    if (!active) continue;
    float acc[kRows];
#pragma unroll
    for (int r = 0; r < kRows; ++r) acc[r] = 0.f;
    const float4* xb = reinterpret_cast<const float4*>(Xs + (size_t)(g * kRows) * k4);
    const int q4 = k4 >> 2;
    for (int i = 0; i < q4; ++i) {
      const float4 w = mrow[i];
#pragma unroll
      for (int r = 0; r < kRows; ++r) {
        const float4 x = xb[r * q4 + i];
        acc[r] = fmaf(x.x, w.x, acc[r]);
        acc[r] = fmaf(x.y, w.y, acc[r]);
        acc[r] = fmaf(x.z, w.z, acc[r]);
        acc[r] = fmaf(x.w, w.w, acc[r]);
      }
    }
    if (o >= n_out) continue;
#pragma unroll
    for (int r = 0; r < kRows; ++r) {
      const int s = s0 + g * kRows + r;
      if (s >= n) break;
      const size_t oi = (size_t)s * n_out + o;
      if (mode == 0) {
        const float z = acc[r] + b;
        if (pre) pre[oi] = z;
        out[oi] = relu ? fmaxf(z, 0.f) : z;
      } else {
        float gr = acc[r];
        if (mask && !(mask[oi] > 0.f)) gr = 0.f;
        out[oi] = gr;
      }
    }
  }
}

size_t dense_smem(int k_in, int n_out) {
  const int outw = round32(n_out);
  const int tile = (kDenseThreads / outw) * kRows;
  return ((size_t)outw * (round4(k_in) + 4) + (size_t)tile * round4(k_in)) * sizeof(float);
}

// dW[o][i] += sum_s bf(dZ[s][o]) bf(in[row(s)][i]),  db[o] += sum_s dZ[s][o].
// Persistent CTAs walk chunks of kGradChunk samples; thread t owns the 8 x 8 output tile
// (to, ti) = (t / tiles_i, t % tiles_i) in registers and adds it to dW once at the end.
constexpr int kGradChunk = 32;
constexpr int kGradThreads = 256;

__global__ void __launch_bounds__(kGradThreads) k_weight_grad(const float* __restrict__ dZ, const float* __restrict__ in,
                                                               const int* __restrict__ idx, int n, int n_out, int k_in,
                                                               float* __restrict__ dW, float* __restrict__ db) {
  __shared__ __align__(16) float Gs[kGradChunk][kMaxWidth];  // bf16-rounded dZ
  __shared__ __align__(16) float Is[kGradChunk][kMaxWidth];  // bf16-rounded inputs
  __shared__ float Gu[kGradChunk][kMaxWidth];                // unrounded dZ (bias gradient)
  const int tiles_o = (n_out + 7) >> 3, tiles_i = (k_in + 7) >> 3;
  const int t = threadIdx.x;
  const bool own = t < tiles_o * tiles_i;
  const int to = own ? t / tiles_i : 0, ti = own ? t % tiles_i : 0;
  float acc[8][8];
#pragma unroll
  for (int a = 0; a < 8; ++a)
#pragma unroll
    for (int c = 0; c < 8; ++c) acc[a][c] = 0.f;
  float accb = 0.f;
  const int wo = tiles_o * 8, wi = tiles_i * 8;
  for (int s0 = blockIdx.x * kGradChunk; s0 < n; s0 += gridDim.x * kGradChunk) {
    __syncthreads();
    for (int e = t; e < kGradChunk * wo; e += blockDim.x) {
      const int s = e / wo, oo = e - s * wo;
      const float v = (s0 + s < n && oo < n_out) ? dZ[(size_t)(s0 + s) * n_out + oo] : 0.f;
      Gs[s][oo] = bf(v);
      Gu[s][oo] = v;
    }
    for (int e = t; e < kGradChunk * wi; e += blockDim.x) {
      const int s = e / wi, ii = e - s * wi;
      float v = 0.f;
      if (s0 + s < n && ii < k_in) {
        const long long r = idx ? (long long)idx[s0 + s] : (long long)(s0 + s);
        v = in[r * k_in + ii];
      }
      Is[s][ii] = bf(v);
    }
    __syncthreads();
    if (t < n_out) {
      const int sn = min(kGradChunk, n - s0);
      for (int s = 0; s < sn; ++s) accb += Gu[s][t];
    }
    if (!own) continue;
    for (int s = 0; s < kGradChunk; ++s) {
      const float4 g0 = *reinterpret_cast<const float4*>(&Gs[s][to * 8]);
      const float4 g1 = *reinterpret_cast<const float4*>(&Gs[s][to * 8 + 4]);
      const float4 x0 = *reinterpret_cast<const float4*>(&Is[s][ti * 8]);
      const float4 x1 = *reinterpret_cast<const float4*>(&Is[s][ti * 8 + 4]);
      const float gv[8] = {g0.x, g0.y, g0.z, g0.w, g1.x, g1.y, g1.z, g1.w};
      const float xv[8] = {x0.x, x0.y, x0.z, x0.w, x1.x, x1.y, x1.z, x1.w};
#pragma unroll
      for (int a = 0; a < 8; ++a)
#pragma unroll
        for (int c = 0; c < 8; ++c) acc[a][c] = fmaf(gv[a], xv[c], acc[a][c]);
    }
  }
  if (t < n_out && accb != 0.f) atomicAdd(&db[t], accb);
  if (!own) return;
#pragma unroll
  for (int a = 0; a < 8; ++a) {
    const int oo = to * 8 + a;
    if (oo >= n_out) break;
#pragma unroll
    for (int c = 0; c < 8; ++c) {
      const int ii = ti * 8 + c;
      if (ii < k_in) atomicAdd(&dW[(size_t)oo * k_in + ii], acc[a][c]);
    }
  }
}

// loss[0] += scale * sum (Y - T[row])^2, dY = 2 scale (Y - T[row]) (row = idx[s] if given).
__global__ void k_mse(const float* __restrict__ Y, const float* __restrict__ T, const int* __restrict__ idx, int n,
                      int width, float scale, float* __restrict__ loss, float* __restrict__ dY) {
  float acc = 0.f;
  const long long count = (long long)n * width;
  for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < count;
       k += (long long)gridDim.x * blockDim.x) {
    const long long s = k / width, c = k - s * width;
    const long long r = idx ? (long long)idx[s] : s;
    const float d = Y[k] - T[r * width + c];
    acc = fmaf(d, d, acc);
    if (dY) dY[k] = 2.f * scale * d;
  }
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  __shared__ float red[32];
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x < 32) {
    float v = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.f;
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (threadIdx.x == 0) atomicAdd(loss, v * scale);
  }
}

struct Offsets {
  size_t W1, b1, W2, b2, W3, b3, total;
};

Offsets offsets(int din, int hidden, int dout) {
  Offsets o;
  o.W1 = 0;
  o.b1 = o.W1 + (size_t)hidden * din;
  o.W2 = o.b1 + hidden;
  o.b2 = o.W2 + (size_t)hidden * hidden;
  o.W3 = o.b2 + hidden;
  o.b3 = o.W3 + (size_t)dout * hidden;
  o.total = o.b3 + dout;
  return o;
}

bool dims_ok(int din, int hidden, int dout) {
  return din >= 1 && din <= kMaxWidth && hidden >= 1 && hidden <= kMaxWidth && dout >= 1 && dout <= kMaxWidth;
}

int dense_grid(int n, int n_out, int ctas_per_sm) {
  const int tile = (kDenseThreads / round32(n_out)) * kRows;
  const int tiles = (n + tile - 1) / tile;
  const int cap = num_sms() * ctas_per_sm;
  return tiles < cap ? tiles : cap;
}

cudaError_t launch_dense(const float* in, const int* idx, int n, int k_in, const float* Wm, int transpose, int n_out,
                         const float* bias, int mode, int relu, const float* mask, float* pre, float* out,
                         cudaStream_t s) {
  static int cache[64];
  const size_t smem = dense_smem(k_in, n_out);
  cudaError_t e = ensure_smem((const void*)k_dense, smem, cache);
  if (e != cudaSuccess) return e;
  k_dense<<<dense_grid(n, n_out, 2), kDenseThreads, smem, s>>>(in, idx, n, k_in, Wm, transpose, n_out, bias, mode,
                                                               relu, mask, pre, out);
  return cudaGetLastError();
}

cudaError_t launch_wgrad(const float* dZ, const float* in, const int* idx, int n, int n_out, int k_in, float* dW,
                         float* db, cudaStream_t s) {
  int blocks = (n + kGradChunk - 1) / kGradChunk;
  const int cap = num_sms() * 2;
  if (blocks > cap) blocks = cap;
  k_weight_grad<<<blocks, kGradThreads, 0, s>>>(dZ, in, idx, n, n_out, k_in, dW, db);
  return cudaGetLastError();
}

int rc(cudaError_t e) { return e == cudaSuccess ? GS_OK : GS_ECUDA; }

}  // namespace
}  // namespace gs

using namespace gs;

extern "C" {

int gs_mlp_param_count(int din, int hidden, int dout, size_t* count) {
  if (!dims_ok(din, hidden, dout) || !count) return GS_EINVAL;
  *count = offsets(din, hidden, dout).total;
  return GS_OK;
}

int gs_mlp_forward(const float* params, int din, int hidden, int dout, const float* X, const int* idx, int n,
                   float* acts, float* Y, gs_stream_t stream) {
  if (!dims_ok(din, hidden, dout) || n < 0) return GS_EINVAL;
  if (n == 0) return GS_OK;
  if (!params || !X || !acts || !Y) return GS_EINVAL;
  const Offsets o = offsets(din, hidden, dout);
  cudaStream_t s = (cudaStream_t)stream;
  const size_t nh = (size_t)n * hidden;
  float *Z1 = acts, *H1 = acts + nh, *Z2 = acts + 2 * nh, *H2 = acts + 3 * nh;
  cudaError_t e = launch_dense(X, idx, n, din, params + o.W1, 0, hidden, params + o.b1, 0, 1, nullptr, Z1, H1, s);
  if (e == cudaSuccess)
    e = launch_dense(H1, nullptr, n, hidden, params + o.W2, 0, hidden, params + o.b2, 0, 1, nullptr, Z2, H2, s);
  if (e == cudaSuccess)
    e = launch_dense(H2, nullptr, n, hidden, params + o.W3, 0, dout, params + o.b3, 0, 0, nullptr, nullptr, Y, s);
  return rc(e);
}

int gs_mlp_backward(const float* params, int din, int hidden, int dout, const float* X, const int* idx, int n,
                    const float* acts, const float* dY, float* dparams, float* scratch, gs_stream_t stream) {
  if (!dims_ok(din, hidden, dout) || n < 0) return GS_EINVAL;
  if (n == 0) return GS_OK;
  if (!params || !X || !acts || !dY || !dparams || !scratch) return GS_EINVAL;
  const Offsets o = offsets(din, hidden, dout);
  cudaStream_t s = (cudaStream_t)stream;
  const size_t nh = (size_t)n * hidden;
  const float *Z1 = acts, *H1 = acts + nh, *Z2 = acts + 2 * nh, *H2 = acts + 3 * nh;
  float* dZ2 = scratch;
  float* dZ1 = scratch + nh;
  // data backward with the ReLU masks fused: dZ2 = (dY W3) . [Z2 > 0], dZ1 = (dZ2 W2) . [Z1 > 0]
  cudaError_t e = launch_dense(dY, nullptr, n, dout, params + o.W3, 1, hidden, nullptr, 1, 0, Z2, nullptr, dZ2, s);
  if (e == cudaSuccess)
    e = launch_dense(dZ2, nullptr, n, hidden, params + o.W2, 1, hidden, nullptr, 1, 0, Z1, nullptr, dZ1, s);
  if (e == cudaSuccess) e = launch_wgrad(dY, H2, nullptr, n, dout, hidden, dparams + o.W3, dparams + o.b3, s);
  if (e == cudaSuccess) e = launch_wgrad(dZ2, H1, nullptr, n, hidden, hidden, dparams + o.W2, dparams + o.b2, s);
  if (e == cudaSuccess) e = launch_wgrad(dZ1, X, idx, n, hidden, din, dparams + o.W1, dparams + o.b1, s);
  return rc(e);
}

int gs_mse(const float* Y, const float* T, const int* idx, int n, int width, float scale, float* loss, float* dY,
           gs_stream_t stream) {
  if (n < 0 || width < 1 || !loss) return GS_EINVAL;
  if (n == 0) return GS_OK;
  if (!Y || !T) return GS_EINVAL;
  const long long count = (long long)n * width;
  long long blocks = (count + 255) / 256;
  const long long cap = (long long)num_sms() * 8;
  if (blocks > cap) blocks = cap;
  k_mse<<<(int)blocks, 256, 0, (cudaStream_t)stream>>>(Y, T, idx, n, width, scale, loss, dY);
  return rc(cudaGetLastError());
}

}  // extern "C"
