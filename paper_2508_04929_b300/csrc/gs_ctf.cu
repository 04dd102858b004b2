// ApplyCTF (App. A.2 Eq. 14), the loss (Sec. 3.3.5) and Adam (Sec. 4.1).
//
// k_ctf_mul multiplies the R2C half spectrum of each image by H_hat / D^2.  H_hat depends
// on the integer n = fx^2 + fy^2 only: chi / pi = alpha n - beta n^2 with per-image
// constants alpha = lambda df / (D apix)^2 and beta = Cs lambda^3 / (2 (D apix)^4), formed
// once per CTA (a few CTAs per image) in FP64.  The phase is reduced modulo 2 exactly (the product alpha_hi * n is
// split into its rounded value and its exact FMA remainder), so sinpi / cospi see an
// argument accurate to ~1e-7 even where chi reaches hundreds of radians.
#include <cooperative_groups.h>

#include "gs_internal.cuh"

namespace cg = cooperative_groups;

namespace gs {
namespace {

// Per-image CTF constants, formed in FP64 by one thread: alpha split into hi + lo, beta,
// sqrt(1 - w^2), w.
__device__ __forceinline__ void ctf_constants(const float* __restrict__ ctf, int b, int D, float cst[5]) {
  const double df = ctf[b * 5 + 0], kv = ctf[b * 5 + 1], cs = ctf[b * 5 + 2] * 1e7, w = ctf[b * 5 + 3],
               apix = ctf[b * 5 + 4];
  const double V = kv * 1e3;
  const double lam = 12.2643 / sqrt(V * (1.0 + 0.978466e-6 * V));
  const double s2 = 1.0 / ((double)D * apix * (double)D * apix);
  const double alpha = lam * df * s2;
  const double beta = 0.5 * cs * lam * lam * lam * s2 * s2;
  const float ahi = (float)alpha;
  cst[0] = ahi;
  cst[1] = (float)(alpha - (double)ahi);
  cst[2] = (float)beta;
  cst[3] = (float)sqrt(1.0 - w * w);
  cst[4] = (float)w;
}

// H_hat at half-spectrum element idx = l (D / 2 + 1) + m (row l, column m) of a D x D image.
__device__ __forceinline__ float ctf_value(int idx, int D, int W2, const float cst[5]) {
  const int l = idx / W2, m = idx - l * W2;
  const int fy = l < (D + 1) / 2 ? l : l - D;
  const float n = (float)(fy * fy + m * m);  // exact (< 2^24)
  const float p = cst[0] * n;
  const float perr = fmaf(cst[0], n, -p);        // exact remainder of alpha_hi * n
  const float pred = p - 2.f * rintf(0.5f * p);  // exact: p mod 2 in [-1, 1]
  const float q = cst[2] * n * n;
  const float qred = q - 2.f * rintf(0.5f * q);
  const float tt = (pred + perr + cst[1] * n) - qred;
  float sp, cp;
  sincospif(tt, &sp, &cp);
  return -(cst[3] * sp + cst[4] * cp);
}

__global__ void k_ctf_mul(float2* __restrict__ spec, const float* __restrict__ ctf, int D) {
  const int b = blockIdx.y;
  const int W2 = D / 2 + 1;
  __shared__ float cst[6];
  if (threadIdx.x == 0) {
    ctf_constants(ctf, b, D, cst);
    cst[5] = (float)(1.0 / ((double)D * (double)D));
  }
  __syncthreads();
  const float c[5] = {cst[0], cst[1], cst[2], cst[3], cst[4]};
  const float sc = cst[5];
  float2* img = spec + (size_t)b * D * W2;
  for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < D * W2; idx += gridDim.x * blockDim.x) {
    const float H = ctf_value(idx, D, W2, c) * sc;
    float2 v = img[idx];
    v.x *= H;
    v.y *= H;
    img[idx] = v;
  }
}

// Loss of one image per cluster of kLossCtas CTAs: each CTA reduces a strided slice of the
// pixels, and CTA 0 adds the CTAs' sums, read from their shared memory, in rank order (the
// result does not depend on scheduling).
constexpr int kLossCtas = 8;

__global__ void __cluster_dims__(kLossCtas, 1, 1) k_loss(const float* __restrict__ X, const float* __restrict__ Y,
                                                         int P, float scale, float* __restrict__ loss,
                                                         float* __restrict__ dLdX) {
  cg::cluster_group cluster = cg::this_cluster();
  const int b = blockIdx.y, part = (int)cluster.block_rank();
  const float* x = X + (size_t)b * P;
  const float* y = Y + (size_t)b * P;
  float acc = 0.f;
  for (int p = part * blockDim.x + threadIdx.x; p < P; p += kLossCtas * blockDim.x) {
    const float r = x[p] - y[p];
    acc = fmaf(r, r, acc);
    if (dLdX) dLdX[(size_t)b * P + p] = 2.f * scale * r;
  }
  __shared__ float red[32];
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x < 32) {
    float v = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.f;
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (threadIdx.x == 0) red[0] = v;
  }
  cluster.sync();
  if (part == 0 && threadIdx.x == 0) {
    float v = 0.f;
    for (int r = 0; r < kLossCtas; ++r) v += *cluster.map_shared_rank(&red[0], r);
    loss[b] = v * scale;
  }
  cluster.sync();  // the other CTAs' shared memory stays alive until it has been read
}

// CTF, loss and adjoint CTF of one image in the Fourier domain, one cluster of kLossCtas CTAs
// per image.  With the unnormalized R2C spectra Q_hat, Y_hat and Z = H_hat Q_hat - Y_hat (the
// spectrum of X - Y, since H_hat is real and even), Parseval gives
// sum (X - Y)^2 = sum over the full spectrum |Z|^2 / D^2 (half-spectrum columns other than 0
// and D / 2 count twice), and the adjoint CTF of dL/dX = 2 s (X - Y) is
// C2R(2 s H_hat Z) / D^2, written over Q_hat.  The loss is reduced as in k_loss.
__global__ void __cluster_dims__(kLossCtas, 1, 1) k_ctf_loss(float2* __restrict__ specQ,
                                                             const float2* __restrict__ specY,
                                                             const float* __restrict__ ctf, int D, float scale,
                                                             float* __restrict__ loss) {
  cg::cluster_group cluster = cg::this_cluster();
  const int b = blockIdx.y, part = (int)cluster.block_rank();
  const int W2 = D / 2 + 1;
  __shared__ float cst[5];
  __shared__ float red[32];
  if (threadIdx.x == 0) ctf_constants(ctf, b, D, cst);
  __syncthreads();
  const float c[5] = {cst[0], cst[1], cst[2], cst[3], cst[4]};
  const float inv_d2 = 1.f / ((float)D * (float)D);
  const float gscale = 2.f * scale * inv_d2;
  float2* q = specQ + (size_t)b * D * W2;
  const float2* y = specY + (size_t)b * D * W2;
  float acc = 0.f;
  for (int idx = part * blockDim.x + threadIdx.x; idx < D * W2; idx += kLossCtas * blockDim.x) {
    const float H = ctf_value(idx, D, W2, c);
    const float2 qv = q[idx], yv = y[idx];
    const float zx = fmaf(H, qv.x, -yv.x), zy = fmaf(H, qv.y, -yv.y);
    const int m = idx % W2;
    const float wgt = (m == 0 || 2 * m == D) ? 1.f : 2.f;
    acc = fmaf(wgt, fmaf(zx, zx, zy * zy), acc);
    const float gH = gscale * H;
    q[idx] = make_float2(gH * zx, gH * zy);
  }
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x < 32) {
    float v = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.f;
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (threadIdx.x == 0) red[0] = v;
  }
  cluster.sync();
  if (part == 0 && threadIdx.x == 0) {
    float v = 0.f;
    for (int r = 0; r < kLossCtas; ++r) v += *cluster.map_shared_rank(&red[0], r);
    loss[b] = v * inv_d2 * scale;
  }
  cluster.sync();  // the other CTAs' shared memory stays alive until it has been read
}

// One Adam update (Sec. 4.1; bias corrections c1 = 1 / (1 - b1^t), c2 = 1 / (1 - b2^t)).
__device__ __forceinline__ void adam_one(float& th, float g, float& m, float& v, float lr, float b1, float b2,
                                         float eps, float c1, float c2) {
  m = b1 * m + (1.f - b1) * g;
  v = b2 * v + (1.f - b2) * g * g;
  th = th - lr * (m * c1) / (sqrtf(v * c2) + eps);
}

// Adam over n floats, four per thread and iteration when all buffers are 16-byte aligned
// (kVec), with a grid of two CTAs per SM.  kCounted: the step counter is on the device
// (t_dev = steps already taken) so that a captured graph can be replayed; the bias
// corrections are then formed in FP64 by one thread per CTA.
template <bool kCounted, bool kVec>
__global__ void k_adam(float* __restrict__ th, const float* __restrict__ g, float* __restrict__ m,
                       float* __restrict__ v, int n, const int* __restrict__ t_dev, float lr, float b1, float b2,
                       float eps, float c1, float c2) {
  if (kCounted) {
    __shared__ float cc[2];
    if (threadIdx.x == 0) {
      const double t = (double)(*t_dev + 1);
      cc[0] = (float)(1.0 / (1.0 - pow((double)b1, t)));
      cc[1] = (float)(1.0 / (1.0 - pow((double)b2, t)));
    }
    __syncthreads();
    c1 = cc[0];
    c2 = cc[1];
  }
  const int tid = blockIdx.x * blockDim.x + threadIdx.x, stride = gridDim.x * blockDim.x;
  int done = 0;
  if (kVec) {
    const int n4 = n / 4;
    float4* th4 = reinterpret_cast<float4*>(th);
    float4* m4 = reinterpret_cast<float4*>(m);
    float4* v4 = reinterpret_cast<float4*>(v);
    const float4* g4 = reinterpret_cast<const float4*>(g);
    for (int i = tid; i < n4; i += stride) {
      float4 T = th4[i], M = m4[i], V = v4[i];
      const float4 G = g4[i];
      adam_one(T.x, G.x, M.x, V.x, lr, b1, b2, eps, c1, c2);
      adam_one(T.y, G.y, M.y, V.y, lr, b1, b2, eps, c1, c2);
      adam_one(T.z, G.z, M.z, V.z, lr, b1, b2, eps, c1, c2);
      adam_one(T.w, G.w, M.w, V.w, lr, b1, b2, eps, c1, c2);
      th4[i] = T;
      m4[i] = M;
      v4[i] = V;
    }
    done = 4 * n4;
  }
  for (int i = done + tid; i < n; i += stride) {
    float T = th[i], M = m[i], V = v[i];
    adam_one(T, g[i], M, V, lr, b1, b2, eps, c1, c2);
    th[i] = T;
    m[i] = M;
    v[i] = V;
  }
}

__global__ void k_count_step(int* t_dev) { *t_dev += 1; }

}  // namespace

// Grid for the Adam kernels: two CTAs per SM at most (grid-stride loops).
static int adam_blocks(int n) {
  int blocks = (n / 4 + 255) / 256;
  const int cap = 2 * num_sms();
  if (blocks > cap) blocks = cap;
  return blocks < 1 ? 1 : blocks;
}

static bool all16(const void* a, const void* b, const void* c, const void* d) {
  return ((reinterpret_cast<uintptr_t>(a) | reinterpret_cast<uintptr_t>(b) | reinterpret_cast<uintptr_t>(c) |
           reinterpret_cast<uintptr_t>(d)) & 15) == 0;
}

cudaError_t launch_adam_counted(float* theta, const float* g, float* m, float* v, int n, int* t_dev, float lr,
                                float b1, float b2, float eps, cudaStream_t s) {
  if (n > 0) {
    const int blocks = adam_blocks(n);
    if (all16(theta, g, m, v))
      k_adam<true, true><<<blocks, 256, 0, s>>>(theta, g, m, v, n, t_dev, lr, b1, b2, eps, 0.f, 0.f);
    else
      k_adam<true, false><<<blocks, 256, 0, s>>>(theta, g, m, v, n, t_dev, lr, b1, b2, eps, 0.f, 0.f);
  }
  k_count_step<<<1, 1, 0, s>>>(t_dev);
  return cudaGetLastError();
}

cudaError_t launch_ctf_mul(const gs_config& cfg, float2* spec, const float* ctf, int B, cudaStream_t s) {
  if (B <= 0) return cudaSuccess;
  const int D = cfg.D, cnt = D * (D / 2 + 1);
  int per_image = (cnt + 255) / 256;
  if (per_image > 8) per_image = 8;  // a few CTAs per image: few FP64 prologues
  dim3 grid(per_image, B);
  k_ctf_mul<<<grid, 256, 0, s>>>(spec, ctf, D);
  return cudaGetLastError();
}

cudaError_t launch_ctf_loss(const gs_config& cfg, float2* specQ, const float2* specY, const float* ctf, int B,
                            float* loss, cudaStream_t s) {
  if (B <= 0) return cudaSuccess;
  const float scale = cfg.reduction == 1 ? 1.f / ((float)cfg.D * (float)cfg.D) : 1.f;
  k_ctf_loss<<<dim3(kLossCtas, B), 256, 0, s>>>(specQ, specY, ctf, cfg.D, scale, loss);
  return cudaGetLastError();
}

cudaError_t launch_loss(const gs_config& cfg, const float* X, const float* Y, int B, float* loss, float* dLdX,
                        cudaStream_t s) {
  if (B <= 0) return cudaSuccess;
  const int P = cfg.D * cfg.D;
  const float scale = cfg.reduction == 1 ? 1.f / (float)P : 1.f;
  k_loss<<<dim3(kLossCtas, B), 256, 0, s>>>(X, Y, P, scale, loss, dLdX);
  return cudaGetLastError();
}

cudaError_t launch_adam(float* theta, const float* g, float* m, float* v, int n, float lr, float b1, float b2,
                        float eps, float c1, float c2, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  const int blocks = adam_blocks(n);
  if (all16(theta, g, m, v))
    k_adam<false, true><<<blocks, 256, 0, s>>>(theta, g, m, v, n, nullptr, lr, b1, b2, eps, c1, c2);
  else
    k_adam<false, false><<<blocks, 256, 0, s>>>(theta, g, m, v, n, nullptr, lr, b1, b2, eps, c1, c2);
  return cudaGetLastError();
}

}  // namespace gs
