// BuildGaussians, ViewingTransform and Projection (Algorithm 2; Sec. 3.3.1-3.3.3, Eqs. 5, 6,
// 8; App. A.2 Eqs. 12-13).
//
// k_activate runs once per Gaussian (pose independent, four lanes each): softplus of the
// scales and the amplitude, quaternion normalization, R(q) and M = R diag(s).  k_project forms, per
// (particle, Gaussian), mu_dot = W mu, Sigma_tilde = (W M)_{2x3} (W M)_{2x3}^T, the k-sigma
// support box and the record consumed by the rasterizer; a thread serves one Gaussian for
// sixteen particles, so that the Gaussian's row of the activated table is read once for them.
//
// The support box is an integer decision.  It is computed with explicitly rounded FP32
// intrinsics (no FMA contraction) in a fixed order, so that any FP32 implementation of the
// same sequence reproduces it bit for bit (the order is spelled out in include/gs.h).  The
// three scale activations, which the box depends on, are the FP64 softplus rounded once
// (softplus_rn: float-float arithmetic, with FP64 where that cannot decide the rounding), so
// that they are the correctly rounded FP32 values with overwhelming probability; the
// amplitude only scales values and is activated in FP32.
#include "gs_internal.cuh"

namespace gs {
namespace {

__device__ __forceinline__ double softplus_d(double x) {
  return fmax(x, 0.0) + log1p(exp(-fabs(x)));
}

// ---------------------------------------------------------------------------------------
// softplus(x) rounded once to FP32: the correctly rounded value of the FP64 evaluation above,
// mostly without FP64 arithmetic (scarce on this GPU).  Fast path in float-float arithmetic
// (a value is a pair hi + lo; Knuth's two-sum, Dekker's fast two-sum and the FMA two-product
// are exact), accurate to better than 2^-44 (relative) on [-60, 17]:
//   exp(y), y = -|x| <= 0: Cody-Waite reduction y = k ln2 + r with ln2 in three parts, then
//     the Taylor series of exp(r) to r^12 (|r| <= ln2 / 2);
//   log1p(e): m = 1 + e, c = 1 + i / 16 <= m (i < 16), log1p(e) = log(c) + log1p((m - c) / c)
//     with the Taylor series of log1p(t) to t^11 (t < 1/16);
//   softplus(x) = log1p(exp(x)) for x <= 0, x + log1p(exp(-x)) for x > 0.
// The pair's leading float is the rounded result unless the pair lies within 2^-37 (relative)
// of a rounding midpoint; then, and outside [-60, 17], the FP64 evaluation decides.
// ---------------------------------------------------------------------------------------
struct FF {
  float h, l;
};

__device__ __forceinline__ FF ff_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b), bb = __fsub_rn(s, a);
  return {s, __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb))};
}
__device__ __forceinline__ FF ff_fast(float a, float b) {  // |a| >= |b|
  const float s = __fadd_rn(a, b);
  return {s, __fsub_rn(b, __fsub_rn(s, a))};
}
__device__ __forceinline__ FF ff_prod(float a, float b) {
  const float p = __fmul_rn(a, b);
  return {p, fmaf(a, b, -p)};
}
__device__ __forceinline__ FF ff_add(FF a, FF b) {
  const FF s = ff_two_sum(a.h, b.h);
  return ff_fast(s.h, __fadd_rn(s.l, __fadd_rn(a.l, b.l)));
}
__device__ __forceinline__ FF ff_mul(FF a, FF b) {
  const FF p = ff_prod(a.h, b.h);
  return ff_fast(p.h, fmaf(a.h, b.l, fmaf(a.l, b.h, p.l)));
}

__constant__ float2 c_log_c[16] = {  // log(1 + i / 16) as (hi, lo)
    {0.0f, 0.0f},                        {0x1.f0a30cp-5f, 0x1.162a66p-37f},   {0x1.e27076p-4f, 0x1.c55e5cp-29f},
    {0x1.5ff308p-3f, -0x1.eb0d86p-28f},  {0x1.c8ff7cp-3f, 0x1.e6a688p-29f},   {0x1.1675cap-2f, 0x1.7574c2p-27f},
    {0x1.4618bcp-2f, 0x1.0e2f62p-29f},   {0x1.739d8p-2f, -0x1.2886p-27f},     {0x1.9f323ep-2f, 0x1.97f30ap-27f},
    {0x1.c8ff7cp-2f, 0x1.e6a688p-28f},   {0x1.f128f6p-2f, -0x1.43e44ep-32f},  {0x1.0be72ep-1f, 0x1.094aap-27f},
    {0x1.1e85f6p-1f, -0x1.8fbf3p-29f},   {0x1.307d74p-1f, -0x1.961de8p-26f},  {0x1.41d8fep-1f, 0x1.08ce56p-26f},
    {0x1.52a2d2p-1f, 0x1.96f16ap-27f}};

__device__ __forceinline__ FF exp_ff(float y) {  // y in [-60, 0]
  // 1 / n! as (hi, lo), n = 0 .. 12
  const FF inv_fact[13] = {{0x1p+0f, 0.0f},
                           {0x1p+0f, 0.0f},
                           {0x1p-1f, 0.0f},
                           {0x1.555556p-3f, -0x1.555556p-28f},
                           {0x1.555556p-5f, -0x1.555556p-30f},
                           {0x1.111112p-7f, -0x1.dddddep-32f},
                           {0x1.6c16c2p-10f, -0x1.27d27ep-35f},
                           {0x1.a01a02p-13f, -0x1.7f97fap-39f},
                           {0x1.a01a02p-16f, -0x1.7f97fap-42f},
                           {0x1.71de3ap-19f, 0x1.55b1ccp-45f},
                           {0x1.27e4fcp-22f, -0x1.10ec14p-47f},
                           {0x1.ae6456p-26f, 0x1.fd5138p-52f},
                           {0x1.1eed8ep-29f, 0x1.ff1b12p-54f}};
  const float ln2a = 0x1.62e4p-1f, ln2b = 0x1.7f7d1cp-20f, ln2c = 0x1.ef357ap-45f;  // ln2 = a + b + c
  const float k = rintf(__fmul_rn(y, 0x1.715476p+0f));
  const float r1 = __fsub_rn(y, __fmul_rn(k, ln2a));  // exact: k ln2a has at most 24 bits
  FF r = ff_add({r1, 0.0f}, ff_prod(-k, ln2b));
  r.l = __fsub_rn(r.l, __fmul_rn(k, ln2c));
  FF acc = inv_fact[12];
#pragma unroll
  for (int n = 11; n >= 0; --n) acc = ff_add(ff_mul(acc, r), inv_fact[n]);
  const int ki = (int)k;
  return {ldexpf(acc.h, ki), ldexpf(acc.l, ki)};
}

__device__ __forceinline__ FF log1p_ff(FF e) {  // e in (0, 1]
  // (-1)^(n + 1) / n as (hi, lo), n = 1 .. 11
  const FF coef[11] = {{0x1p+0f, 0.0f},
                       {-0x1p-1f, 0.0f},
                       {0x1.555556p-2f, -0x1.555556p-27f},
                       {-0x1p-2f, 0.0f},
                       {0x1.99999ap-3f, -0x1.99999ap-29f},
                       {-0x1.555556p-3f, 0x1.555556p-28f},
                       {0x1.24924ap-3f, -0x1.b6db6ep-28f},
                       {-0x1p-3f, 0.0f},
                       {0x1.c71c72p-4f, -0x1.c71c72p-31f},
                       {-0x1.99999ap-4f, 0x1.99999ap-30f},
                       {0x1.745d18p-4f, -0x1.745d18p-29f}};
  const FF m = ff_add({1.0f, 0.0f}, e);
  const int i = min(max((int)__fmul_rn(__fsub_rn(m.h, 1.0f), 16.0f), 0), 15);
  FF t = e;
  if (i > 0) {
    const float c = 1.0f + (float)i * 0.0625f;  // exact
    const FF d = ff_add(m, {-c, 0.0f});
    const float q = __fdiv_rn(d.h, c);
    const FF pq = ff_prod(q, c);
    const float rem = __fadd_rn(__fsub_rn(__fsub_rn(d.h, pq.h), pq.l), d.l);
    t = ff_fast(q, __fdiv_rn(rem, c));
  }
  FF acc = coef[10];
#pragma unroll
  for (int n = 9; n >= 0; --n) acc = ff_add(ff_mul(acc, t), coef[n]);
  FF res = ff_mul(acc, t);
  if (i > 0) res = ff_add({c_log_c[i].x, c_log_c[i].y}, res);
  return res;
}

__device__ __forceinline__ float softplus_rn(float x) {
  if (x > 17.0f) return x;  // e^-17 is below half an ulp of x
  if (!(x >= -60.0f)) return (float)softplus_d((double)x);
  const FF lp = log1p_ff(exp_ff(-fabsf(x)));
  const FF y = x > 0.0f ? ff_add({x, 0.0f}, lp) : lp;
  const float up = __fsub_rn(nextafterf(y.h, INFINITY), y.h), dn = __fsub_rn(y.h, nextafterf(y.h, -INFINITY));
  const float margin = fabsf(y.h) * 0x1p-37f;
  const bool decided = y.l >= 0.0f ? (0.5f * up - y.l > margin) : (0.5f * dn + y.l > margin);
  return decided ? y.h : (float)softplus_d((double)x);
}

// Four lanes per Gaussian: lanes 0-2 of a quad each activate one scale (the long float-float
// chains then run side by side), lane 3 the amplitude, the normalized quaternion and R; the quad
// exchanges them by shuffles and each lane writes six of the 24 table entries.
__global__ void k_activate(const float* __restrict__ theta, int N, float* __restrict__ gauss,
                           float* __restrict__ gacc, int* __restrict__ status) {
  const int tid = blockIdx.x * blockDim.x + threadIdx.x;
  const int g = tid >> 2, j = tid & 3;
  const int lane = threadIdx.x & 31, q0 = lane & ~3;
  const bool live = g < N;
  const float* t = theta + (size_t)(live ? g : 0) * 11;
  float th[11];
#pragma unroll
  for (int k = 0; k < 11; ++k) th[k] = live ? t[k] : 0.f;
  bool bad = false;
#pragma unroll
  for (int k = 0; k < 11; ++k) bad |= !isfinite(th[k]);
  // lanes 0-2: s_j;  lane 3: A, the quaternion's norm and R
  float mine = 0.f, nr = 1.f;
  float R[9] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
  if (j < 3) {
    mine = softplus_rn(th[3 + j]);
  } else {
    mine = fmaxf(th[10], 0.f) + log1pf(expf(-fabsf(th[10])));
    const float qw = th[6], qx = th[7], qy = th[8], qz = th[9];
    const float n2 = __fadd_rn(__fadd_rn(__fadd_rn(__fmul_rn(qw, qw), __fmul_rn(qx, qx)), __fmul_rn(qy, qy)),
                               __fmul_rn(qz, qz));
    nr = __fsqrt_rn(n2);
    const float w = __fdiv_rn(qw, nr), x = __fdiv_rn(qx, nr), y = __fdiv_rn(qy, nr), z = __fdiv_rn(qz, nr);
    const float xx = __fmul_rn(x, x), yy = __fmul_rn(y, y), zz = __fmul_rn(z, z);
    const float xy = __fmul_rn(x, y), xz = __fmul_rn(x, z), yz = __fmul_rn(y, z);
    const float wx = __fmul_rn(w, x), wy = __fmul_rn(w, y), wz = __fmul_rn(w, z);
    R[0] = __fsub_rn(1.f, __fmul_rn(2.f, __fadd_rn(yy, zz)));
    R[1] = __fmul_rn(2.f, __fsub_rn(xy, wz));
    R[2] = __fmul_rn(2.f, __fadd_rn(xz, wy));
    R[3] = __fmul_rn(2.f, __fadd_rn(xy, wz));
    R[4] = __fsub_rn(1.f, __fmul_rn(2.f, __fadd_rn(xx, zz)));
    R[5] = __fmul_rn(2.f, __fsub_rn(yz, wx));
    R[6] = __fmul_rn(2.f, __fsub_rn(xz, wy));
    R[7] = __fmul_rn(2.f, __fadd_rn(yz, wx));
    R[8] = __fsub_rn(1.f, __fmul_rn(2.f, __fadd_rn(xx, yy)));
  }
  const float s0 = __shfl_sync(0xffffffffu, mine, q0), s1 = __shfl_sync(0xffffffffu, mine, q0 + 1),
              s2 = __shfl_sync(0xffffffffu, mine, q0 + 2), A = __shfl_sync(0xffffffffu, mine, q0 + 3);
  nr = __shfl_sync(0xffffffffu, nr, q0 + 3);
#pragma unroll
  for (int k = 0; k < 9; ++k) R[k] = __shfl_sync(0xffffffffu, R[k], q0 + 3);
  if (!live) return;
  bad |= !isfinite(nr) || nr == 0.f;
  const float sv[3] = {s0, s1, s2};
  float o[24];
  o[kMu + 0] = th[0];
  o[kMu + 1] = th[1];
  o[kMu + 2] = th[2];
#pragma unroll
  for (int k = 0; k < 3; ++k)
#pragma unroll
    for (int m = 0; m < 3; ++m) o[kM + 3 * k + m] = __fmul_rn(R[3 * k + m], sv[m]);
  o[kS + 0] = s0;
  o[kS + 1] = s1;
  o[kS + 2] = s2;
  o[kA] = A;
  o[kSprod] = s0 * s1 * s2;
  o[kBad] = bad ? 1.f : 0.f;
  o[kInvS2 + 0] = 1.f / (s0 * s0);
  o[kInvS2 + 1] = 1.f / (s1 * s1);
  o[kInvS2 + 2] = 1.f / (s2 * s2);
  o[21] = 0.f;
  o[22] = 0.f;
  o[23] = 0.f;
  // lane j writes table entries 6 j .. 6 j + 5 and a third of the gradient accumulator
  float2* dst = reinterpret_cast<float2*>(gauss + (size_t)g * kGaussStride + 6 * j);
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    float a = 0.f, c = 0.f;
#pragma unroll
    for (int jj = 0; jj < 4; ++jj)
      if (jj == j) {
        a = o[6 * jj + 2 * k];
        c = o[6 * jj + 2 * k + 1];
      }
    dst[k] = make_float2(a, c);
  }
  // reset this Gaussian's gradient accumulator for the next gs_render_bwd
  if (j < 3) reinterpret_cast<float4*>(gacc + (size_t)g * kGradStride)[j] = make_float4(0.f, 0.f, 0.f, 0.f);
  if (bad && j == 0) atomicOr(status, GS_STATUS_NONFINITE);
}

constexpr float kHalfLog2eP = 0.72134752044448170f;  // log2(e) / 2
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
                          float2* __restrict__ lo, int* __restrict__ status) {
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
    const float wgt = G[kA] * kInv2Pi / sqrt_det;
    // A well-conditioned splat keeps the expanded form of Eq. 12's exponent (log2 units, pixel
    // offsets): ca dx^2 + cb dx dy + cc dy^2 with (ca, cb, cc) = k2 (Syy, 2 Sxy, Sxx),
    // k2 = -log2(e) / (2 det) (Sigma~ in px^2), and the linear weight w.  A thin or strongly
    // anisotropic one (a > kAThr, or (Sxx + Syy)^2 > kKappa det, i.e. a condition number above
    // about kKappa) is stored as the completed square -a (dx + r dy)^2 - q dy^2 with
    // a = log2(e)/2 Syy / det, r = Sxy / Syy, q = log2(e)/2 / Syy, and log2 w.
    const float ih2 = inv_h * inv_h;
    const float k2 = -kHalfLog2eP / (det * ih2);
    const float a = -k2 * Syy;
    const bool exact = a > kAThr || (Sxx + Syy) * (Sxx + Syy) > kKappa * det;
    float c1, c2, c3, c4;
    if (!exact) {
      c1 = k2 * Syy;
      c2 = 2.f * k2 * Sxy;
      c3 = k2 * Sxx;
      c4 = wgt;
    } else {
      c1 = a;
      c2 = Sxy / Syy;
      c3 = -kHalfLog2eP / (Syy * ih2);
      c4 = log2f(wgt);
    }
    bad |= !(isfinite(c1) && isfinite(c2) && isfinite(c3) && isfinite(c4) && isfinite(wgt) && sqrt_det > 0.f);

    gs_record r;
    r.cx = cx;
    r.cy = cy;
    r.c1 = c1;
    r.c2 = c2;
    r.c3 = c3;
    r.c4 = c4;
    r.x0 = 1; r.x1 = 0; r.y0 = 1; r.y1 = 0;
    if (!bad) {
      const float x0f = fmaxf(ceilf(__fsub_rn(cx, rx)), 0.f);
      const float x1f = fminf(floorf(__fadd_rn(cx, rx)), (float)(D - 1));
      const float y0f = fmaxf(ceilf(__fsub_rn(cy, ry)), 0.f);
      const float y1f = fminf(floorf(__fadd_rn(cy, ry)), (float)(D - 1));
      if (x0f <= x1f && y0f <= y1f) {
        r.x0 = (int16_t)x0f; r.x1 = (int16_t)x1f; r.y0 = (int16_t)y0f; r.y1 = (int16_t)y1f;
      }
      // Ill-conditioned splats are rendered with the centre as a float-float: the low parts
      // are the FP64 centre (exact products of the FP32 pose and mean) minus the FP32 one.
      // Other records never read them, and they are not written.
      if (exact) {
        const double mx64 = ((double)Ws[0] * mux + (double)Ws[1] * muy) + (double)Ws[2] * muz;
        const double my64 = ((double)Ws[3] * mux + (double)Ws[4] * muy) + (double)Ws[5] * muz;
        const double c064 = (double)(D / 2), ih64 = (double)inv_h;
        lo[(size_t)b * N + g] = make_float2((float)((mx64 * ih64 + c064) - (double)cx),
                                            (float)((c064 - my64 * ih64) - (double)cy));
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
  k_activate<<<(int)((4 * (long long)N + 255) / 256), 256, 0, s>>>(theta, N, gauss, gacc, status);
  return cudaGetLastError();
}

cudaError_t launch_project(const gs_config& cfg, const float* gauss, int N, const float* W, int B,
                           gs_record* proj, int* status, cudaStream_t s) {
  if (N <= 0 || B <= 0) return cudaSuccess;
  dim3 grid((N + 255) / 256, (B + kProjParticles - 1) / kProjParticles);
  int2* boxes = reinterpret_cast<int2*>(proj + (size_t)B * N);  // box plane after the B * N records
  float2* lo = reinterpret_cast<float2*>(boxes + (size_t)B * N);  // then the centres' low parts
  if ((reinterpret_cast<uintptr_t>(proj) & 31) == 0)
    k_project<true><<<grid, 256, 0, s>>>(gauss, N, W, B, cfg.D, inv_pixel(cfg), cfg.cutoff_sigma, proj, boxes, lo,
                                         status);
  else
    k_project<false><<<grid, 256, 0, s>>>(gauss, N, W, B, cfg.D, inv_pixel(cfg), cfg.cutoff_sigma, proj, boxes, lo,
                                          status);
  return cudaGetLastError();
}

}  // namespace gs
