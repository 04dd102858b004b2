// Internal definitions shared by the CUDA translation units of libgs (not part of the ABI).
#pragma once

#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "../../include/gs.h"

namespace gs {

constexpr int kBinChunk = 2048;       // Gaussians per binning CTA (8 warps x 256, in order)
constexpr int kBinWarps = 8;
constexpr int kGaussStride = 24;      // floats per activated Gaussian in the workspace
constexpr int kGradStride = 12;       // floats per Gaussian in the gradient accumulator
constexpr float kLog2e = 1.4426950408889634f;
constexpr float kInv2Pi = 0.15915494309189535f;
// Ill-conditioned splats -- row curvature a (log2 units per px^2) above kAThr, a conditional
// standard deviation below 0.49 px, or a 2 x 2 covariance with (Sxx + Syy)^2 > kKappa det, a
// condition number above about kKappa -- are stored as a completed square and rendered by
// the exact path, which reads the low parts of the centre; gs_project writes those low parts
// for them only.
constexpr float kAThr = 3.f;
constexpr float kKappa = 100.f;

// Layout of the activated-Gaussian table (one row of kGaussStride floats per Gaussian).
enum GaussField {
  kMu = 0,     // mu[3]
  kM = 3,      // M = R diag(s), row-major [3][3]
  kS = 12,     // s[3] (FP32, rounded once from the FP64 softplus)
  kA = 15,     // A
  kSprod = 16, // s0 s1 s2
  kBad = 17,   // 1 if a parameter is not finite
  kInvS2 = 18, // 1 / s[m]^2
};

// Workspace carve-up; every part 256-byte aligned.
struct WsLayout {
  size_t status, gauss, hist, tstart, ttotal, itotal, ibase, gacc, spec, spec2, fftwork, red, total;
  int Tn, C, ntx;
};

inline size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

// Argument checks shared by the entry points (host side).
inline bool cfg_ok(const gs_config* c) {
  if (!c) return false;
  if (c->D < 1 || c->D > 4096) return false;
  if (!(c->tile == 8 || c->tile == 16 || c->tile == 32)) return false;
  if (c->chunk < 32 || c->chunk > 512 || (c->chunk % 32) != 0) return false;
  if (!(c->E > 0.f) || !isfinite(c->E)) return false;
  if (!(c->cutoff_sigma > 0.f) || !isfinite(c->cutoff_sigma)) return false;
  if (c->reduction != 0 && c->reduction != 1) return false;
  const int ntx = (c->D + c->tile - 1) / c->tile;
  if (ntx > 64) return false;
  return true;
}

inline bool sizes_ok(const gs_config* c, int B, int N) {
  if (B < 0 || N < 0 || B > 65535) return false;
  const int ntx = (c->D + c->tile - 1) / c->tile;
  if ((unsigned long long)N * (unsigned long long)(ntx * ntx) >= (1ull << 32)) return false;
  return true;
}

// CTAs per image of the D = 256 column kernel of gs_ctf_loss_grad (16 of the 129 columns
// each) and the bytes of its loss partial sums and per-image tickets.
constexpr int kColCtas = 9;
inline size_t ctf_cols_red_bytes(int B) {
  return align256(sizeof(float) * (size_t)B * kColCtas) + align256(sizeof(unsigned) * (size_t)B);
}

inline WsLayout ws_layout(const gs_config& cfg, int B, int N, size_t fft_work) {
  WsLayout L;
  L.ntx = (cfg.D + cfg.tile - 1) / cfg.tile;
  L.Tn = L.ntx * L.ntx;
  L.C = (N + kBinChunk - 1) / kBinChunk;
  if (L.C < 1) L.C = 1;
  size_t o = 0;
  L.status = o; o = align256(o + 256);
  L.gauss = o; o = align256(o + sizeof(float) * kGaussStride * (size_t)N);
  L.hist = o; o = align256(o + sizeof(uint32_t) * (size_t)B * L.C * L.Tn);
  L.tstart = o; o = align256(o + sizeof(uint32_t) * (size_t)B * L.Tn);
  L.ttotal = o; o = align256(o + sizeof(uint32_t) * (size_t)B * L.Tn);
  L.itotal = o; o = align256(o + sizeof(uint32_t) * ((size_t)B + 1));
  L.ibase = o; o = align256(o + sizeof(unsigned long long) * ((size_t)B + 1));
  L.gacc = o; o = align256(o + sizeof(float) * kGradStride * (size_t)N);
  L.spec = o; o = align256(o + 2 * sizeof(float) * (size_t)B * cfg.D * (cfg.D / 2 + 1));
  L.spec2 = o; o = align256(o + 2 * sizeof(float) * (size_t)B * cfg.D * (cfg.D / 2 + 1));
  L.fftwork = o; o = align256(o + fft_work);
  L.red = o; o += ctf_cols_red_bytes(B);
  L.total = o;
  return L;
}

template <class T>
inline T* ws_ptr(void* ws, size_t off) { return reinterpret_cast<T*>(static_cast<char*>(ws) + off); }

__device__ __forceinline__ float ex2_approx(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

__device__ __forceinline__ void red_add_v4(float* p, float a, float b, float c, float d) {
  asm volatile("red.global.add.v4.f32 [%0], {%1, %2, %3, %4};" ::"l"(p), "f"(a), "f"(b), "f"(c),
               "f"(d)
               : "memory");
}

__device__ __forceinline__ void red_add_v2(float* p, float a, float b) {
  asm volatile("red.global.add.v2.f32 [%0], {%1, %2};" ::"l"(p), "f"(a), "f"(b) : "memory");
}

__device__ __forceinline__ unsigned lanemask_lt() {
  unsigned m;
  asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
  return m;
}

// Raise a kernel's dynamic shared-memory limit once per device and size (the call is
// skipped when an earlier call already allowed at least `bytes`, e.g. during stream capture).
inline cudaError_t ensure_smem(const void* func, size_t bytes, int* cache /* [64] per call site */) {
  if (bytes <= 48 * 1024) return cudaSuccess;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev >= 0 && dev < 64 && cache[dev] >= (int)bytes) return cudaSuccess;
  e = cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  if (e == cudaSuccess && dev >= 0 && dev < 64) cache[dev] = (int)bytes;
  return e;
}

// Multiprocessor count of the current device (cached per device): grid sizes of the
// persistent kernels are multiples of it.
inline int num_sms() {
  static int cache[64] = {0};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 148;
  if (cache[dev] == 0) {
    int n = 0;
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0) n = 148;
    cache[dev] = n;
  }
  return cache[dev];
}

// Host-side launchers (one per translation unit).
cudaError_t launch_activate(const float* theta, int N, float* gauss, float* gacc, int* status, cudaStream_t s);
cudaError_t launch_project(const gs_config& cfg, const float* gauss, int N, const float* W, int B,
                           gs_record* proj, int* status, cudaStream_t s);
// inv_h = D / (2E) in FP32, correctly rounded (part of the support-box arithmetic)
inline float inv_pixel(const gs_config& cfg) {
  volatile float twoE = 2.0f * cfg.E;  // exact
  volatile float r = (float)cfg.D / twoE;
  return r;
}
cudaError_t launch_bin(const gs_config& cfg, const WsLayout& L, const gs_record* proj, int B, int N,
                       void* ws, uint32_t* pair_gauss, size_t cap, uint32_t* ranges,
                       uint32_t* n_pairs, cudaStream_t s);
cudaError_t launch_render_fwd(const gs_config& cfg, const gs_record* proj, int N,
                              const uint32_t* pair_gauss, const uint32_t* ranges, int B, float* Q,
                              cudaStream_t s);
cudaError_t launch_render_bwd(const gs_config& cfg, const gs_record* proj, int N,
                              const uint32_t* pair_gauss, const uint32_t* ranges, int B, const float* dLdQ,
                              const float* W, float* wacc, const float* gauss, float* dpose, cudaStream_t s);
cudaError_t launch_bwd_finalize(const float* theta, const float* gauss, int N, float* gacc, float* dtheta,
                                cudaStream_t s);
cudaError_t launch_ctf_mul(const gs_config& cfg, float2* spec, const float* ctf, int B, cudaStream_t s);
// Row transforms of the D = 256 training path: the 1-D R2C of Q and Y (one launch), and the 1-D C2R.
cudaError_t launch_rows_r2c2(const float* Q, const float* Y, float2* qr, float2* yr, int B, cudaStream_t s);
cudaError_t launch_rows_c2r(const float2* spec, float* out, int B, cudaStream_t s);
cudaError_t launch_ctf_cols(const gs_config& cfg, float2* qr, const float2* yr, const float* ctf, int B,
                            float* loss, void* red, cudaStream_t s);
cudaError_t launch_ctf_loss(const gs_config& cfg, float2* specQ, const float2* specY, const float* ctf, int B,
                            float* loss, cudaStream_t s);
cudaError_t launch_loss(const gs_config& cfg, const float* X, const float* Y, int B, float* loss,
                        float* dLdX, cudaStream_t s);
cudaError_t launch_adam(float* theta, const float* g, float* m, float* v, int n, float lr,
                        float b1, float b2, float eps, float c1, float c2, cudaStream_t s);
cudaError_t launch_adam_counted(float* theta, const float* g, float* m, float* v, int n, int* t_dev, float lr,
                                float b1, float b2, float eps, cudaStream_t s);

}  // namespace gs
