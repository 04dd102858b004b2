// BuildGaussians, ViewingTransform and Projection (Algorithm 2; Sec. 3.3.1-3.3.3, Eqs. 5, 6,
// 8; App. A.2 Eqs. 12-13).
//
// k_activate runs once per Gaussian (pose independent): softplus of the scales and the
// amplitude, quaternion normalization, R(q) and M = R diag(s).  k_project forms, per
// (particle, Gaussian), mu_dot = W mu, Sigma_tilde = (W M)_{2x3} (W M)_{2x3}^T, the k-sigma
// support box and the record consumed by the rasterizer; a thread serves one Gaussian for
// sixteen particles, so that the Gaussian's row of the activated table is read once for them.
//
// The support box is an integer decision.  It is computed with explicitly rounded FP32
// intrinsics (no FMA contraction) in a fixed order, so that any FP32 implementation of the
// same sequence reproduces it bit for bit (the order is spelled out in include/gs.h).  The
// three scale activations, which the box depends on, are evaluated in FP64 and rounded
// once, so that they are the correctly rounded FP32 values with overwhelming probability;
// the amplitude only scales values and is activated in FP32.
#include "gs_internal.cuh"

namespace gs {
namespace {

__device__ __forceinline__ double softplus_d(double x) {
  return fmax(x, 0.0) + log1p(exp(-fabs(x)));
}

__global__ void k_activate(const float* __restrict__ theta, int N, float* __restrict__ gauss,
                           float* __restrict__ gacc, int* __restrict__ status) {
  int g = blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= N) return;
  const float* t = theta + (size_t)g * 11;
  float th[11];
#pragma unroll
  for (int k = 0; k < 11; ++k) th[k] = t[k];
  bool bad = false;
#pragma unroll
  for (int k = 0; k < 11; ++k) bad |= !isfinite(th[k]);

  float s0 = (float)softplus_d((double)th[3]);
  float s1 = (float)softplus_d((double)th[4]);
  float s2 = (float)softplus_d((double)th[5]);
  const float A = fmaxf(th[10], 0.f) + log1pf(expf(-fabsf(th[10])));

  float qw = th[6], qx = th[7], qy = th[8], qz = th[9];
  float n2 = __fadd_rn(__fadd_rn(__fadd_rn(__fmul_rn(qw, qw), __fmul_rn(qx, qx)), __fmul_rn(qy, qy)),
                       __fmul_rn(qz, qz));
  float nr = __fsqrt_rn(n2);
  float w = __fdiv_rn(qw, nr), x = __fdiv_rn(qx, nr), y = __fdiv_rn(qy, nr), z = __fdiv_rn(qz, nr);
  float xx = __fmul_rn(x, x), yy = __fmul_rn(y, y), zz = __fmul_rn(z, z);
  float xy = __fmul_rn(x, y), xz = __fmul_rn(x, z), yz = __fmul_rn(y, z);
  float wx = __fmul_rn(w, x), wy = __fmul_rn(w, y), wz = __fmul_rn(w, z);
  float R[9];
  R[0] = __fsub_rn(1.f, __fmul_rn(2.f, __fadd_rn(yy, zz)));
  R[1] = __fmul_rn(2.f, __fsub_rn(xy, wz));
  R[2] = __fmul_rn(2.f, __fadd_rn(xz, wy));
  R[3] = __fmul_rn(2.f, __fadd_rn(xy, wz));
  R[4] = __fsub_rn(1.f, __fmul_rn(2.f, __fadd_rn(xx, zz)));
  R[5] = __fmul_rn(2.f, __fsub_rn(yz, wx));
  R[6] = __fmul_rn(2.f, __fsub_rn(xz, wy));
  R[7] = __fmul_rn(2.f, __fadd_rn(yz, wx));
  R[8] = __fsub_rn(1.f, __fmul_rn(2.f, __fadd_rn(xx, yy)));
  float s[3] = {s0, s1, s2};
  float* o = gauss + (size_t)g * kGaussStride;
  o[kMu + 0] = th[0];
  o[kMu + 1] = th[1];
  o[kMu + 2] = th[2];
#pragma unroll
  for (int k = 0; k < 3; ++k)
#pragma unroll
    for (int m = 0; m < 3; ++m) o[kM + 3 * k + m] = __fmul_rn(R[3 * k + m], s[m]);
  o[kS + 0] = s0;
  o[kS + 1] = s1;
  o[kS + 2] = s2;
  o[kA] = A;
  o[kSprod] = s0 * s1 * s2;
  bad |= !isfinite(nr) || nr == 0.f;
  o[kBad] = bad ? 1.f : 0.f;
  o[kInvS2 + 0] = 1.f / (s0 * s0);
  o[kInvS2 + 1] = 1.f / (s1 * s1);
  o[kInvS2 + 2] = 1.f / (s2 * s2);
  o[21] = 0.f;
  o[22] = 0.f;
  o[23] = 0.f;
  // reset this Gaussian's gradient accumulator for the next gs_render_bwd
  float4* ga = reinterpret_cast<float4*>(gacc + (size_t)g * kGradStride);
  ga[0] = make_float4(0.f, 0.f, 0.f, 0.f);
  ga[1] = make_float4(0.f, 0.f, 0.f, 0.f);
  ga[2] = make_float4(0.f, 0.f, 0.f, 0.f);
  if (bad) atomicOr(status, GS_STATUS_NONFINITE);
}

constexpr int kProjParticles = 16;  // particles per thread: one load of the Gaussian's row serves them all

// One 32-byte store: the record fills its sector in a single request (proj 32-byte aligned).
__device__ __forceinline__ void st_record32(gs_record* dst, const gs_record& r) {
  const float* f = reinterpret_cast<const float*>(&r);
  asm volatile("st.global.v8.f32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8};" ::"l"(dst), "f"(f[0]), "f"(f[1]),
               "f"(f[2]), "f"(f[3]), "f"(f[4]), "f"(f[5]), "f"(f[6]), "f"(f[7])
               : "memory");
}

template <bool kV8>
__global__ void k_project(const float* __restrict__ gauss, int N, const float* __restrict__ Wall, int B, int D,
                          float inv_h, float kcut, gs_record* __restrict__ proj, int2* __restrict__ boxes,
                          int* __restrict__ status) {
  const int b0 = blockIdx.y * kProjParticles;
  __shared__ float Wsh[kProjParticles * 9];
  if (threadIdx.x < kProjParticles * 9 && b0 + (int)threadIdx.x / 9 < B)
    Wsh[threadIdx.x] = Wall[(size_t)b0 * 9 + threadIdx.x];
  __syncthreads();
  int g = blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= N) return;
  float G[kGaussStride];
  {
    const float4* src = reinterpret_cast<const float4*>(gauss + (size_t)g * kGaussStride);
#pragma unroll
    for (int k = 0; k < kGaussStride / 4; ++k) {
      const float4 v = __ldg(src + k);
      G[4 * k] = v.x; G[4 * k + 1] = v.y; G[4 * k + 2] = v.z; G[4 * k + 3] = v.w;
    }
  }
  const float mux = G[kMu], muy = G[kMu + 1], muz = G[kMu + 2];
  float M[9];
#pragma unroll
  for (int k = 0; k < 9; ++k) M[k] = G[kM + k];
  const bool bad_g = G[kBad] != 0.f;
  bool any_bad = false;
  for (int p = 0; p < kProjParticles; ++p) {
    const int b = b0 + p;
    if (b >= B) break;
    const float* Ws = Wsh + 9 * p;
    bool bad = bad_g;
    // V = W_{2x3} M, Sigma_tilde = V V^T (Eqs. 5, 6, 12)
    float V[2][3];
#pragma unroll
    for (int a = 0; a < 2; ++a)
#pragma unroll
      for (int m = 0; m < 3; ++m)
        V[a][m] = __fadd_rn(__fadd_rn(__fmul_rn(Ws[3 * a + 0], M[0 + m]), __fmul_rn(Ws[3 * a + 1], M[3 + m])),
                            __fmul_rn(Ws[3 * a + 2], M[6 + m]));
    const float Sxx = __fadd_rn(__fadd_rn(__fmul_rn(V[0][0], V[0][0]), __fmul_rn(V[0][1], V[0][1])),
                                __fmul_rn(V[0][2], V[0][2]));
    const float Syy = __fadd_rn(__fadd_rn(__fmul_rn(V[1][0], V[1][0]), __fmul_rn(V[1][1], V[1][1])),
                                __fmul_rn(V[1][2], V[1][2]));
    const float mx = __fadd_rn(__fadd_rn(__fmul_rn(Ws[0], mux), __fmul_rn(Ws[1], muy)), __fmul_rn(Ws[2], muz));
    const float my = __fadd_rn(__fadd_rn(__fmul_rn(Ws[3], mux), __fmul_rn(Ws[4], muy)), __fmul_rn(Ws[5], muz));
    const float c0 = (float)(D / 2);
    const float cx = __fadd_rn(__fmul_rn(mx, inv_h), c0);
    const float cy = __fsub_rn(c0, __fmul_rn(my, inv_h));
    const float rx = __fmul_rn(kcut, __fmul_rn(__fsqrt_rn(Sxx), inv_h));
    const float ry = __fmul_rn(kcut, __fmul_rn(__fsqrt_rn(Syy), inv_h));
    bad |= !(isfinite(cx) && isfinite(cy) && isfinite(rx) && isfinite(ry));

    // Value path (free FP32).  det Sigma_tilde by the Schur-complement identity
    // det(Sigma_tilde) = det(Sigma) * (w_z^T Sigma^-1 w_z), w_z the third row of W:
    // sqrt(det) = s0 s1 s2 * || (w_z^T M)_m / s_m^2 ||, a sum of squares (no cancellation).
    const float Sxy = V[0][0] * V[1][0] + V[0][1] * V[1][1] + V[0][2] * V[1][2];
    const float t0 = (Ws[6] * M[0] + Ws[7] * M[3] + Ws[8] * M[6]) * G[kInvS2];
    const float t1 = (Ws[6] * M[1] + Ws[7] * M[4] + Ws[8] * M[7]) * G[kInvS2 + 1];
    const float t2 = (Ws[6] * M[2] + Ws[7] * M[5] + Ws[8] * M[8]) * G[kInvS2 + 2];
    const float sqrt_det = G[kSprod] * sqrtf(t0 * t0 + t1 * t1 + t2 * t2);
    const float det = sqrt_det * sqrt_det;
    const float wgt = __fdividef(G[kA] * kInv2Pi, sqrt_det);
    const float k2 = __fdividef(-0.5f * kLog2e, det * inv_h * inv_h);
    bad |= !(isfinite(wgt) && isfinite(k2) && sqrt_det > 0.f);

    gs_record r;
    r.cx = cx;
    r.cy = cy;
    r.ca = k2 * Syy;
    r.cb = 2.f * k2 * Sxy;
    r.cc = k2 * Sxx;
    r.w = wgt;
    r.x0 = 1; r.x1 = 0; r.y0 = 1; r.y1 = 0;
    if (!bad) {
      const float x0f = fmaxf(ceilf(__fsub_rn(cx, rx)), 0.f);
      const float x1f = fminf(floorf(__fadd_rn(cx, rx)), (float)(D - 1));
      const float y0f = fmaxf(ceilf(__fsub_rn(cy, ry)), 0.f);
      const float y1f = fminf(floorf(__fadd_rn(cy, ry)), (float)(D - 1));
      if (x0f <= x1f && y0f <= y1f) {
        r.x0 = (int16_t)x0f; r.x1 = (int16_t)x1f; r.y0 = (int16_t)y0f; r.y1 = (int16_t)y1f;
      }
    }
    any_bad |= bad;
    if (kV8) {
      st_record32(proj + (size_t)b * N + g, r);
    } else {
      float4* dst = reinterpret_cast<float4*>(proj + (size_t)b * N + g);
      const float4* srcp = reinterpret_cast<const float4*>(&r);
      dst[0] = srcp[0];
      dst[1] = srcp[1];
    }
    // the box again in the plane after the records, for the binning passes
    boxes[(size_t)b * N + g] = make_int2((int)(((unsigned)(uint16_t)r.x0) | ((unsigned)(uint16_t)r.x1 << 16)),
                                         (int)(((unsigned)(uint16_t)r.y0) | ((unsigned)(uint16_t)r.y1 << 16)));
  }
  if (any_bad) atomicOr(status, GS_STATUS_NONFINITE);
}

}  // namespace

cudaError_t launch_activate(const float* theta, int N, float* gauss, float* gacc, int* status, cudaStream_t s) {
  if (N <= 0) return cudaSuccess;
  k_activate<<<(N + 255) / 256, 256, 0, s>>>(theta, N, gauss, gacc, status);
  return cudaGetLastError();
}

cudaError_t launch_project(const gs_config& cfg, const float* gauss, int N, const float* W, int B,
                           gs_record* proj, int* status, cudaStream_t s) {
  if (N <= 0 || B <= 0) return cudaSuccess;
  dim3 grid((N + 255) / 256, (B + kProjParticles - 1) / kProjParticles);
  int2* boxes = reinterpret_cast<int2*>(proj + (size_t)B * N);  // box plane after the B * N records
  if ((reinterpret_cast<uintptr_t>(proj) & 31) == 0)
    k_project<true><<<grid, 256, 0, s>>>(gauss, N, W, B, cfg.D, inv_pixel(cfg), cfg.cutoff_sigma, proj, boxes, status);
  else
    k_project<false><<<grid, 256, 0, s>>>(gauss, N, W, B, cfg.D, inv_pixel(cfg), cfg.cutoff_sigma, proj, boxes, status);
  return cudaGetLastError();
}

}  // namespace gs
