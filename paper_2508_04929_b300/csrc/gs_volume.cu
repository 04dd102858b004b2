// GMM voxelization and Fourier shell correlation: the evaluation side of a reconstruction.
// The paper (arXiv 2508.04929) judges its GMMs by FSC of the mixture evaluated on a voxel
// grid (Sec. 4) without giving formulas; the definitions here are the library's own and are
// restated in gs.h.
//
// k_voxelize: one CTA per Gaussian.  Thread 0 forms the Gaussian's k-sigma voxel box in FP32
// with a fixed sequence of correctly rounded operations (so that it is reproducible), the
// CTA then walks the box and adds A N(r; mu, Sigma) at every voxel centre with a global
// reduction.  The exponent uses Sigma^-1 = R S^-2 R^T through M = R diag(s):
// d^T Sigma^-1 d = sum_m ((M[:, m] . d) / s_m^2)^2.
// k_fsc_shells: the R2C half spectra of the two volumes (cuFFT), Hermitian-weighted (2 for
// the interior columns, 1 for kx = 0 and kx = D/2), summed per shell in FP64: the shell of
// (kx, ky, kz) is the integer nearest to |k|, decided by integer arithmetic.
#include <cufft.h>

#include "gs_internal.cuh"

namespace gs {
namespace {

constexpr float kInv2Pi15 = 0.063493635934240969f;  // (2 pi)^-3/2

__global__ void k_voxelize(const float* __restrict__ gauss, int N, int D, float inv_h, float h, float kcut,
                           float* __restrict__ vol) {
  __shared__ int box[6];
  __shared__ float P[16];  // mu[3], M[9], invS2[3], norm
  const int g = blockIdx.x;
  const float* G = gauss + (size_t)g * kGaussStride;
  if (threadIdx.x == 0) {
    bool ok = G[kBad] == 0.f;
    const float c0 = (float)(D / 2);
    for (int a = 0; a < 3 && ok; ++a) {
      const float v0 = G[kM + 3 * a], v1 = G[kM + 3 * a + 1], v2 = G[kM + 3 * a + 2];
      const float saa = __fadd_rn(__fadd_rn(__fmul_rn(v0, v0), __fmul_rn(v1, v1)), __fmul_rn(v2, v2));
      const float r = __fmul_rn(kcut, __fmul_rn(__fsqrt_rn(saa), inv_h));
      const float c = a == 1 ? __fsub_rn(c0, __fmul_rn(G[kMu + 1], inv_h)) : __fadd_rn(__fmul_rn(G[kMu + a], inv_h), c0);
      const float lo = fmaxf(ceilf(__fsub_rn(c, r)), 0.f), hi = fminf(floorf(__fadd_rn(c, r)), (float)(D - 1));
      ok = isfinite(lo) && isfinite(hi) && lo <= hi;
      box[2 * a] = ok ? (int)lo : 1;
      box[2 * a + 1] = ok ? (int)hi : 0;
    }
    if (!ok) box[0] = 1, box[1] = 0;
#pragma unroll
    for (int k = 0; k < 3; ++k) P[k] = G[kMu + k];
#pragma unroll
    for (int k = 0; k < 9; ++k) P[3 + k] = G[kM + k];
#pragma unroll
    for (int k = 0; k < 3; ++k) P[12 + k] = G[kInvS2 + k];
    P[15] = G[kA] * kInv2Pi15 / G[kSprod];
  }
  __syncthreads();
  const int j0 = box[0], j1 = box[1], i0 = box[2], i1 = box[3], k0 = box[4], k1 = box[5];
  if (j0 > j1 || i0 > i1 || k0 > k1) return;  // CTA-uniform
  const int nx = j1 - j0 + 1, ny = i1 - i0 + 1, nz = k1 - k0 + 1;
  const int total = nx * ny * nz;
  const float mx = P[0], my = P[1], mz = P[2];
  const float nrm = P[15];
  const float half_log2e = -0.5f * kLog2e;
  for (int e = threadIdx.x; e < total; e += blockDim.x) {
    const int j = j0 + e % nx, i = i0 + (e / nx) % ny, k = k0 + e / (nx * ny);
    const float dx = (float)(j - D / 2) * h - mx;
    const float dy = -(float)(i - D / 2) * h - my;
    const float dz = (float)(k - D / 2) * h - mz;
    float q = 0.f;
#pragma unroll
    for (int m = 0; m < 3; ++m) {
      const float p = (P[3 + m] * dx + P[6 + m] * dy + P[9 + m] * dz) * P[12 + m];
      q = fmaf(p, p, q);
    }
    const float v = nrm * ex2_approx(half_log2e * q);
    atomicAdd(vol + ((size_t)k * D + i) * D + j, v);
  }
}

// Shell sums of one R2C coefficient pair: acc[3 s + 0..2] += w (Re F1 conj F2, |F1|^2, |F2|^2).
__global__ void k_fsc_shells(const float2* __restrict__ F1, const float2* __restrict__ F2, int D,
                             double* __restrict__ acc) {
  extern __shared__ double sacc[];  // [3 * (D / 2 + 1)]
  const int ns = D / 2 + 1, W2 = D / 2 + 1;
  for (int t = threadIdx.x; t < 3 * ns; t += blockDim.x) sacc[t] = 0.0;
  __syncthreads();
  const long long count = (long long)D * D * W2;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < count;
       e += (long long)gridDim.x * blockDim.x) {
    const int kx = (int)(e % W2);
    const int i = (int)((e / W2) % D), k = (int)(e / ((long long)W2 * D));
    const int ky = i < (D + 1) / 2 ? i : i - D, kz = k < (D + 1) / 2 ? k : k - D;
    const int k2 = kx * kx + ky * ky + kz * kz;
    int r = (int)sqrtf((float)k2);
    while (r * r > k2) --r;
    while ((r + 1) * (r + 1) <= k2) ++r;
    if (k2 > r * r + r) ++r;  // nearest integer to sqrt(k2); never a tie
    if (r >= ns) continue;
    const double w = (kx == 0 || 2 * kx == D) ? 1.0 : 2.0;
    const float2 a = F1[e], b = F2[e];
    atomicAdd(&sacc[3 * r + 0], w * ((double)a.x * b.x + (double)a.y * b.y));
    atomicAdd(&sacc[3 * r + 1], w * ((double)a.x * a.x + (double)a.y * a.y));
    atomicAdd(&sacc[3 * r + 2], w * ((double)b.x * b.x + (double)b.y * b.y));
  }
  __syncthreads();
  for (int t = threadIdx.x; t < 3 * ns; t += blockDim.x)
    if (sacc[t] != 0.0) atomicAdd(&acc[t], sacc[t]);
}

__global__ void k_fsc_final(const double* __restrict__ acc, int ns, float* __restrict__ fsc) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= ns) return;
  const double d = sqrt(acc[3 * s + 1] * acc[3 * s + 2]);
  fsc[s] = d > 0.0 ? (float)(acc[3 * s] / d) : 0.f;
}

struct VoxLayout {
  size_t status, gauss, gacc, total;
};

VoxLayout vox_layout(int N) {
  VoxLayout L;
  size_t o = 0;
  L.status = o; o = align256(o + 256);
  L.gauss = o; o = align256(o + sizeof(float) * kGaussStride * (size_t)N);
  L.gacc = o; o = align256(o + sizeof(float) * kGradStride * (size_t)N);
  L.total = o;
  return L;
}

struct FscLayout {
  size_t spec1, spec2, acc, work, total;
};

FscLayout fsc_layout(int D, size_t work) {
  FscLayout L;
  const size_t spec = sizeof(float2) * (size_t)D * D * (D / 2 + 1);
  size_t o = 0;
  L.spec1 = o; o = align256(o + spec);
  L.spec2 = o; o = align256(o + spec);
  L.acc = o; o = align256(o + sizeof(double) * 3 * (D / 2 + 1));
  L.work = o; o = align256(o + work);
  L.total = o;
  return L;
}

int rc(cudaError_t e) { return e == cudaSuccess ? GS_OK : GS_ECUDA; }

}  // namespace
}  // namespace gs

using namespace gs;

extern "C" {

int gs_voxel_workspace_size(int N, size_t* bytes) {
  if (N < 0 || !bytes) return GS_EINVAL;
  *bytes = vox_layout(N).total;
  return GS_OK;
}

int gs_voxelize(const float* theta, int N, int Dv, float E, float cutoff_sigma, float* vol, void* ws, size_t ws_bytes,
                gs_stream_t stream) {
  if (N < 0 || Dv < 1 || Dv > 1024 || !(E > 0.f) || !(cutoff_sigma > 0.f) || !vol || !ws) return GS_EINVAL;
  if (N > 0 && !theta) return GS_EINVAL;
  const VoxLayout L = vox_layout(N);
  if (ws_bytes < L.total) return GS_ENOSPC;
  cudaStream_t s = (cudaStream_t)stream;
  cudaError_t e = cudaMemsetAsync(vol, 0, sizeof(float) * (size_t)Dv * Dv * Dv, s);
  if (e != cudaSuccess || N == 0) return rc(e);
  e = cudaMemsetAsync(ws_ptr<int>(ws, L.status), 0, sizeof(int), s);
  if (e != cudaSuccess) return rc(e);
  float* gauss = ws_ptr<float>(ws, L.gauss);
  e = launch_activate(theta, N, gauss, ws_ptr<float>(ws, L.gacc), ws_ptr<int>(ws, L.status), s);
  if (e != cudaSuccess) return rc(e);
  const float inv_h = (float)Dv / (2.f * E);  // host IEEE division: correctly rounded
  const float h = 2.f * E / (float)Dv;
  k_voxelize<<<N, 128, 0, s>>>(gauss, N, Dv, inv_h, h, cutoff_sigma, vol);
  return rc(cudaGetLastError());
}

int gs_fsc_create(int D, gs_fsc_plan* plan) {
  if (!plan || D < 2 || D > 1024) return GS_EINVAL;
  plan->r2c = 0;
  plan->D = D;
  plan->work_bytes = 0;
  cufftHandle a;
  if (cufftCreate(&a) != CUFFT_SUCCESS) return GS_ECUDA;
  cufftSetAutoAllocation(a, 0);
  size_t wa = 0;
  if (cufftMakePlan3d(a, D, D, D, CUFFT_R2C, &wa) != CUFFT_SUCCESS) {
    cufftDestroy(a);
    return GS_ECUDA;
  }
  plan->r2c = (int)a;
  plan->work_bytes = wa;
  return GS_OK;
}

int gs_fsc_destroy(gs_fsc_plan* plan) {
  if (!plan) return GS_EINVAL;
  if (plan->r2c) cufftDestroy((cufftHandle)plan->r2c);
  plan->r2c = 0;
  return GS_OK;
}

int gs_fsc_workspace_size(const gs_fsc_plan* plan, size_t* bytes) {
  if (!plan || !bytes) return GS_EINVAL;
  *bytes = fsc_layout(plan->D, plan->work_bytes).total;
  return GS_OK;
}

int gs_fsc(const gs_fsc_plan* plan, const float* vol1, const float* vol2, float* fsc, void* ws, size_t ws_bytes,
           gs_stream_t stream) {
  if (!plan || !plan->r2c || !vol1 || !vol2 || !fsc || !ws) return GS_EINVAL;
  const int D = plan->D;
  const FscLayout L = fsc_layout(D, plan->work_bytes);
  if (ws_bytes < L.total) return GS_ENOSPC;
  cudaStream_t s = (cudaStream_t)stream;
  cufftHandle a = (cufftHandle)plan->r2c;
  if (cufftSetStream(a, s) != CUFFT_SUCCESS) return GS_ECUDA;
  if (cufftSetWorkArea(a, ws_ptr<char>(ws, L.work)) != CUFFT_SUCCESS) return GS_ECUDA;
  float2* F1 = ws_ptr<float2>(ws, L.spec1);
  float2* F2 = ws_ptr<float2>(ws, L.spec2);
  if (cufftExecR2C(a, const_cast<float*>(vol1), reinterpret_cast<cufftComplex*>(F1)) != CUFFT_SUCCESS ||
      cufftExecR2C(a, const_cast<float*>(vol2), reinterpret_cast<cufftComplex*>(F2)) != CUFFT_SUCCESS)
    return GS_ECUDA;
  const int ns = D / 2 + 1;
  double* acc = ws_ptr<double>(ws, L.acc);
  cudaError_t e = cudaMemsetAsync(acc, 0, sizeof(double) * 3 * ns, s);
  if (e != cudaSuccess) return rc(e);
  const long long count = (long long)D * D * (D / 2 + 1);
  long long blocks = (count + 255) / 256;
  if (blocks > (long long)num_sms() * 8) blocks = (long long)num_sms() * 8;
  k_fsc_shells<<<(int)blocks, 256, sizeof(double) * 3 * ns, s>>>(F1, F2, D, acc);
  k_fsc_final<<<(ns + 127) / 128, 128, 0, s>>>(acc, ns, fsc);
  return rc(cudaGetLastError());
}

}  // extern "C"
