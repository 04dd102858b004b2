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

// H_hat at squared frequency index n = fy^2 + m^2 (exact in FP32, < 2^24).
__device__ __forceinline__ float ctf_value_n(float n, const float cst[5]) {
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

// H_hat at half-spectrum element idx = l (D / 2 + 1) + m (row l, column m) of a D x D image.
__device__ __forceinline__ float ctf_value(int idx, int D, int W2, const float cst[5]) {
  const int l = idx / W2, m = idx - l * W2;
  const int fy = l < (D + 1) / 2 ? l : l - D;
  return ctf_value_n((float)(fy * fy + m * m), cst);
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

// ---------------------------------------------------------------------------------------
// CTF, loss and adjoint CTF for D = 256 on row-transformed spectra (the column half of the
// 2-D transforms, the pointwise step and the inverse column transforms in one pass).
// qr, yr [B][256][129]: the 1-D R2C transforms of the rows of Q and Y.  One CTA owns 16
// columns kx of one image: it runs the forward 256-point FFT along y of both (y = 16 a + b,
// k = c + 16 d: a 16-point DFT over a, twiddle w256^(b c), a 16-point DFT over b; each
// 16-point DFT is 4 x 4 in registers), forms Z = H Q_hat - Y_hat, the loss terms and
// G = 2 s H Z / D^2, and runs the inverse FFT of G along y, written over qr for the row C2R.
// Each CTA adds its loss terms in a fixed order; the image's last CTA (a ticket counter)
// adds the CTAs' sums in index order.
// ---------------------------------------------------------------------------------------
constexpr int kColD = 256, kColW2 = kColD / 2 + 1, kColNC = 16;
static_assert(kColNC == 16, "k_ctf_cols indexes its CTF table with e >> 4 and e & 15");
static_assert(kColCtas == (kColW2 + kColNC - 1) / kColNC, "CTAs per image of k_ctf_cols");

__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
__device__ __forceinline__ float2 conjf2(float2 a) { return make_float2(a.x, -a.y); }

// 4-point DFT in place, X_k = sum_m x_m w^(m k), w = exp(-2 pi i / 4) (kInv: the conjugate).
template <bool kInv>
__device__ __forceinline__ void dft4(float2& a, float2& b, float2& c, float2& d) {
  const float2 s0 = cadd(a, c), s1 = csub(a, c), s2 = cadd(b, d), bd = csub(b, d);
  const float2 s3 = kInv ? make_float2(-bd.y, bd.x) : make_float2(bd.y, -bd.x);  // w (b - d)
  a = cadd(s0, s2);
  c = csub(s0, s2);
  b = cadd(s1, s3);
  d = csub(s1, s3);
}

// 16-point DFT of x[0..15] (x[n] at position n): X[k1 + 4 k2] ends at position 4 k1 + k2.
template <bool kInv>
__device__ __forceinline__ void dft16(float2 (&x)[16]) {
#pragma unroll
  for (int l = 0; l < 4; ++l) dft4<kInv>(x[l], x[4 + l], x[8 + l], x[12 + l]);  // over m, x[4 m + l]
  // twiddles w16^(l k1) at position 4 k1 + l (cos, sin of 2 pi j / 16)
  const float c1 = 0.92387953251128674f, s1 = 0.38268343236508978f, h = 0.70710678118654752f;
  const float2 w1 = make_float2(c1, kInv ? s1 : -s1), w2 = make_float2(h, kInv ? h : -h),
               w3 = make_float2(s1, kInv ? c1 : -c1), w6 = make_float2(-h, kInv ? h : -h),
               w9 = make_float2(-c1, kInv ? -s1 : s1);
  x[5] = cmul(x[5], w1);    // l 1, k1 1
  x[6] = cmul(x[6], w2);    // l 2, k1 1
  x[7] = cmul(x[7], w3);    // l 3, k1 1
  x[9] = cmul(x[9], w2);    // l 1, k1 2
  x[10] = kInv ? make_float2(-x[10].y, x[10].x) : make_float2(x[10].y, -x[10].x);  // w16^4
  x[11] = cmul(x[11], w6);  // l 3, k1 2
  x[13] = cmul(x[13], w3);  // l 1, k1 3
  x[14] = cmul(x[14], w6);  // l 2, k1 3
  x[15] = cmul(x[15], w9);  // l 3, k1 3
#pragma unroll
  for (int k1 = 0; k1 < 4; ++k1) dft4<kInv>(x[4 * k1], x[4 * k1 + 1], x[4 * k1 + 2], x[4 * k1 + 3]);
}

// 256-point FFT down the 16 columns of a [256][16] shared array in two radix-16 steps
// (thread: column j = t & 15, index sub = t >> 4; tw[m] = w256^m, kInv uses the conjugates).
// Step 1 takes x[n] = element 16 n + sub of column j (the rows this thread loaded), DFTs over
// n, twiddles and stores to a.
template <bool kInv>
__device__ __forceinline__ void fft256_cols_step1(float2 (&x)[16], float2* __restrict__ a,
                                                  const float2* __restrict__ tw) {
  const int j = threadIdx.x & 15, sub = threadIdx.x >> 4;
  dft16<kInv>(x);
#pragma unroll
  for (int c = 0; c < 16; ++c) {
    float2 v = x[4 * (c & 3) + (c >> 2)];
    if (c != 0) v = cmul(v, kInv ? conjf2(tw[sub * c]) : tw[sub * c]);
    a[(16 * c + sub) * kColNC + j] = v;
  }
}

// Step 2 (after a barrier that follows step 1) DFTs over the fine index, the result kept in registers:
// X[sub + 16 d] of column j in x[4 (d & 3) + (d >> 2)], the rows sub + 16 d that this thread
// also loaded.
template <bool kInv>
__device__ __forceinline__ void fft256_cols_step2(float2 (&x)[16], const float2* __restrict__ a) {
  const int j = threadIdx.x & 15, sub = threadIdx.x >> 4;
#pragma unroll
  for (int n = 0; n < 16; ++n) x[n] = a[(16 * sub + n) * kColNC + j];
  dft16<kInv>(x);
}

__global__ void __launch_bounds__(256) k_ctf_cols(float2* __restrict__ qr, const float2* __restrict__ yr,
                                                  const float* __restrict__ ctf, float scale,
                                                  float* __restrict__ partial, unsigned* __restrict__ ticket,
                                                  float* __restrict__ loss) {
  extern __shared__ float2 csm[];
  float2* aq = csm;                      // [256][16]
  float2* ay = csm + kColD * kColNC;     // [256][16]
  float2* tw = csm + 2 * kColD * kColNC; // [256]
  __shared__ float cst[5];
  __shared__ float Hs[(kColD / 2 + 1) * kColNC];  // H at rows ky = 0..128 (row D - ky has the same |k|)
  __shared__ float red[8];
  __shared__ bool last;
  const int b = blockIdx.y, c0 = blockIdx.x * kColNC;
  const int j = threadIdx.x & 15, sub = threadIdx.x >> 4;
  const bool col = c0 + j < kColW2;
  // rows sub + 16 r of column j: exactly this thread's inputs to step 1 of both column FFTs
  const size_t img = (size_t)b * kColD * kColW2;
  float2 xq[16], xy[16];
#pragma unroll
  for (int r = 0; r < 16; ++r) {
    const size_t gi = img + (size_t)(sub + 16 * r) * kColW2 + c0 + j;
    xq[r] = col ? qr[gi] : make_float2(0.f, 0.f);
    xy[r] = col ? yr[gi] : make_float2(0.f, 0.f);
  }
  if (threadIdx.x == 0) ctf_constants(ctf, b, kColD, cst);
  {
    float sn, cs;
    sincospif((float)threadIdx.x / 128.f, &sn, &cs);  // w256^m = exp(-2 pi i m / 256)
    tw[threadIdx.x] = make_float2(cs, -sn);
  }
  __syncthreads();
  {
    const float c[5] = {cst[0], cst[1], cst[2], cst[3], cst[4]};
    for (int e = threadIdx.x; e < (kColD / 2 + 1) * kColNC; e += blockDim.x) {
      const int ky = e >> 4, kx = c0 + (e & 15);
      Hs[e] = ctf_value_n((float)(ky * ky + kx * kx), c);
    }
  }
  fft256_cols_step1<false>(xq, aq, tw);
  fft256_cols_step1<false>(xy, ay, tw);
  __syncthreads();
  // From here each thread works on rows sub + 16 r of column j in registers: the forward FFTs'
  // outputs, the pointwise step and the inverse FFT's inputs are the same rows.
  fft256_cols_step2<false>(xq, aq);
  fft256_cols_step2<false>(xy, ay);
  const float inv_d2 = 1.f / ((float)kColD * (float)kColD);
  const float gscale = 2.f * scale * inv_d2;
  const int kx = c0 + j;
  const float wgt = (kx == 0 || 2 * kx == kColD) ? 1.f : 2.f;
  float acc = 0.f;
  float2 xg[16];  // the adjoint G at row 16 n + sub, the inverse FFT's step-1 input
#pragma unroll
  for (int r = 0; r < 16; ++r) {
    const int ky = sub + 16 * r, p = 4 * (r & 3) + (r >> 2);
    const float H = Hs[(ky <= kColD / 2 ? ky : kColD - ky) * kColNC + j];
    const float2 qv = xq[p], yv = xy[p];
    const float zx = fmaf(H, qv.x, -yv.x), zy = fmaf(H, qv.y, -yv.y);
    if (col) acc = fmaf(wgt, fmaf(zx, zx, zy * zy), acc);
    const float gH = gscale * H;
    xg[r] = make_float2(gH * zx, gH * zy);
  }
  __syncthreads();  // every thread has read its step-2 inputs from aq before it is overwritten
  fft256_cols_step1<true>(xg, aq, tw);
  __syncthreads();
  fft256_cols_step2<true>(xg, aq);
#pragma unroll
  for (int d = 0; d < 16; ++d) {
    const int y = sub + 16 * d;
    if (col) qr[img + (size_t)y * kColW2 + c0 + j] = xg[4 * (d & 3) + (d >> 2)];
  }
  // loss: this CTA's sum, then the image's last CTA adds the CTAs' sums in order
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    float v = 0.f;
    for (int w = 0; w < 8; ++w) v += red[w];
    partial[b * kColCtas + blockIdx.x] = v;
    __threadfence();
    last = atomicAdd(&ticket[b], 1u) == (unsigned)(kColCtas - 1);
  }
  __syncthreads();
  if (last && threadIdx.x == 0) {
    __threadfence();
    float v = 0.f;
    for (int k = 0; k < kColCtas; ++k) v += __ldcg(&partial[b * kColCtas + k]);
    loss[b] = v * inv_d2 * scale;
    ticket[b] = 0u;
  }
}

// ---------------------------------------------------------------------------------------
// Row transforms of the D = 256 training path (the 1-D R2C of Q and Y along x, and the
// final 1-D C2R: the x half of the 2-D transforms of App. A.2 Eq. 14), unnormalized like
// cuFFT's.  A CTA holds 16 complex rows of 256 in shared
// memory, element n of row j at j * kRowP + n + n / 16 (the padding spreads the 16-strided
// accesses of the radix-16 steps over the banks), 16 threads per row.
//   k_rows_r2c2: one complex FFT of Z = Q + iY per row gives both half spectra:
//                Q^[k] = (Z[k] + conj Z[256 - k]) / 2,  Y^[k] = (Z[k] - conj Z[256 - k]) / 2i.
//   k_rows_c2r:  one complex FFT per pair of rows: Z = F1 + i F2, F the Hermitian extension of
//                the row's half spectrum (imaginary parts of the DC and Nyquist terms dropped,
//                as a C2R transform does), and the rows are Re z and Im z.
// ---------------------------------------------------------------------------------------
constexpr int kRowP = kColD + kColD / 16;  // padded row of 272 complex values
constexpr int kRowsPerCta = 16;

__device__ __forceinline__ int rpos(int n) { return n + (n >> 4); }

// 256-point FFT of the 16 rows of z (this thread: row j = t >> 4, index sub = t & 15), in two
// radix-16 steps.  Step 1 takes x[n] = element 16 n + sub of the row (from wherever the caller
// read it), DFTs over n, twiddles and stores to z; step 2 DFTs over the fine index and leaves
// X[sub + 16 d] in x[4 (d & 3) + (d >> 2)].
template <bool kInv>
__device__ __forceinline__ void fft256_rows_step1(float2 (&x)[16], float2* __restrict__ z,
                                                  const float2* __restrict__ tw) {
  const int j = threadIdx.x >> 4, sub = threadIdx.x & 15;
  float2* a = z + j * kRowP;
  dft16<kInv>(x);
#pragma unroll
  for (int c = 0; c < 16; ++c) {
    float2 v = x[4 * (c & 3) + (c >> 2)];
    if (c != 0) v = cmul(v, kInv ? conjf2(tw[sub * c]) : tw[sub * c]);
    a[rpos(16 * c + sub)] = v;
  }
}

template <bool kInv>
__device__ __forceinline__ void fft256_rows_step2(float2 (&x)[16], const float2* __restrict__ z) {
  const int j = threadIdx.x >> 4, sub = threadIdx.x & 15;
  const float2* a = z + j * kRowP;
#pragma unroll
  for (int n = 0; n < 16; ++n) x[n] = a[rpos(16 * sub + n)];
  dft16<kInv>(x);
}

__device__ __forceinline__ void row_twiddles(float2* tw) {
  float sn, cs;
  sincospif((float)threadIdx.x / 128.f, &sn, &cs);  // w256^m = exp(-2 pi i m / 256)
  tw[threadIdx.x] = make_float2(cs, -sn);
}

__global__ void __launch_bounds__(256) k_rows_r2c2(const float* __restrict__ Q, const float* __restrict__ Y,
                                                   float2* __restrict__ qr, float2* __restrict__ yr) {
  __shared__ float2 z[kRowsPerCta * kRowP];
  __shared__ float2 tw[kColD];
  const size_t r0 = (size_t)blockIdx.x * kRowsPerCta;  // first row of the CTA (rows of all images)
  const int j = threadIdx.x >> 4, sub = threadIdx.x & 15;
  const float* q = Q + (r0 + j) * kColD + sub;
  const float* y = Y + (r0 + j) * kColD + sub;
  float2 x[16];
#pragma unroll
  for (int n = 0; n < 16; ++n) x[n] = make_float2(__ldg(q + 16 * n), __ldg(y + 16 * n));  // 64-byte runs
  row_twiddles(tw);
  __syncthreads();
  fft256_rows_step1<false>(x, z, tw);
  __syncthreads();
  fft256_rows_step2<false>(x, z);
  // Z[k], k = sub + 16 d, is in this thread; Z[256 - k] is element 15 - d of lane 16 - sub of
  // the same half-warp (its own element (16 - d) mod 16 for sub = 0)
  float2* oq = qr + (r0 + j) * kColW2 + sub;
  float2* oy = yr + (r0 + j) * kColW2 + sub;
  const int partner = (16 - sub) & 15;
#pragma unroll
  for (int d = 0; d <= 8; ++d) {
    const float2 a = x[4 * (d & 3) + (d >> 2)];
    const float2 send = x[4 * ((15 - d) & 3) + ((15 - d) >> 2)];
    const int ds = (16 - d) & 15;
    const float2 self = x[4 * (ds & 3) + (ds >> 2)];
    float2 b = make_float2(__shfl_sync(0xffffffffu, send.x, partner, 16), __shfl_sync(0xffffffffu, send.y, partner, 16));
    if (sub == 0) b = self;
    b = conjf2(b);
    if (d < 8 || sub == 0) {  // k <= 128
      oq[16 * d] = make_float2(0.5f * (a.x + b.x), 0.5f * (a.y + b.y));
      oy[16 * d] = make_float2(0.5f * (a.y - b.y), -0.5f * (a.x - b.x));
    }
  }
}

__global__ void __launch_bounds__(256) k_rows_c2r(const float2* __restrict__ spec, float* __restrict__ out) {
  __shared__ float2 z[kRowsPerCta * kRowP];
  __shared__ float2 tw[kColD];
  const size_t r0 = (size_t)blockIdx.x * 2 * kRowsPerCta;  // 32 rows, paired into 16 complex rows
  const int j = threadIdx.x >> 4, sub = threadIdx.x & 15;
  // step-1 inputs straight from the half spectra of rows 2 j and 2 j + 1:
  // Z[k] = F1[k] + i F2[k] for k <= 128, and Z[k] = conj F1[256 - k] + i conj F2[256 - k] above
  const float2* g1 = spec + (r0 + 2 * j) * kColW2;
  const float2* g2 = g1 + kColW2;
  float2 x[16];
#pragma unroll
  for (int n = 0; n < 16; ++n) {
    const int k = 16 * n + sub;
    const bool lower = k <= kColD / 2;
    const int m = lower ? k : kColD - k;
    float2 v1 = g1[m], v2 = g2[m];
    if (k == 0 || k == kColD / 2) v1.y = v2.y = 0.f;
    x[n] = lower ? make_float2(v1.x - v2.y, v1.y + v2.x) : make_float2(v1.x + v2.y, v2.x - v1.y);
  }
  row_twiddles(tw);
  __syncthreads();
  fft256_rows_step1<true>(x, z, tw);
  __syncthreads();
  fft256_rows_step2<true>(x, z);
  // element sub + 16 d of complex row j: real part to row 2 j, imaginary part to row 2 j + 1
  float* o0 = out + (r0 + 2 * j) * kColD + sub;
  float* o1 = o0 + kColD;
#pragma unroll
  for (int d = 0; d < 16; ++d) {
    const float2 v = x[4 * (d & 3) + (d >> 2)];
    o0[16 * d] = v.x;
    o1[16 * d] = v.y;
  }
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
// (t_dev = steps already taken) so that a captured graph can be replayed; each CTA then forms
// the two bias corrections in FP64, one per warp of its first two.
template <bool kCounted, bool kVec>
__global__ void k_adam(float* __restrict__ th, const float* __restrict__ g, float* __restrict__ m,
                       float* __restrict__ v, int n, const int* __restrict__ t_dev, float lr, float b1, float b2,
                       float eps, float c1, float c2) {
  const int tid = blockIdx.x * blockDim.x + threadIdx.x, stride = gridDim.x * blockDim.x;
  const int n4 = kVec ? n / 4 : 0;
  float4* th4 = reinterpret_cast<float4*>(th);
  float4* m4 = reinterpret_cast<float4*>(m);
  float4* v4 = reinterpret_cast<float4*>(v);
  const float4* g4 = reinterpret_cast<const float4*>(g);
  // the thread's first four values are loaded before the bias corrections are known
  float4 T = make_float4(0.f, 0.f, 0.f, 0.f), M = T, V = T, G = T;
  if (kVec && tid < n4) {
    T = th4[tid];
    M = m4[tid];
    V = v4[tid];
    G = g4[tid];
  }
  if (kCounted) {
    // the two FP64 bias corrections on two warps at once (FP64 pow is slow on this part)
    __shared__ float cc[2];
    if ((threadIdx.x & 31) == 0 && threadIdx.x < 64) {
      const int k = threadIdx.x >> 5;
      const double t = (double)(*t_dev + 1);
      cc[k] = (float)(1.0 / (1.0 - pow((double)(k == 0 ? b1 : b2), t)));
    }
    __syncthreads();
    c1 = cc[0];
    c2 = cc[1];
  }
  if (kVec) {
    for (int i = tid; i < n4; i += stride) {
      if (i != tid) {
        T = th4[i];
        M = m4[i];
        V = v4[i];
        G = g4[i];
      }
      adam_one(T.x, G.x, M.x, V.x, lr, b1, b2, eps, c1, c2);
      adam_one(T.y, G.y, M.y, V.y, lr, b1, b2, eps, c1, c2);
      adam_one(T.z, G.z, M.z, V.z, lr, b1, b2, eps, c1, c2);
      adam_one(T.w, G.w, M.w, V.w, lr, b1, b2, eps, c1, c2);
      th4[i] = T;
      m4[i] = M;
      v4[i] = V;
    }
  }
  for (int i = 4 * n4 + tid; i < n; i += stride) {
    float Ts = th[i], Ms = m[i], Vs = v[i];
    adam_one(Ts, g[i], Ms, Vs, lr, b1, b2, eps, c1, c2);
    th[i] = Ts;
    m[i] = Ms;
    v[i] = Vs;
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

cudaError_t launch_ctf_cols(const gs_config& cfg, float2* qr, const float2* yr, const float* ctf, int B,
                            float* loss, void* red, cudaStream_t s) {
  if (B <= 0) return cudaSuccess;
  float* partial = static_cast<float*>(red);
  unsigned* ticket = reinterpret_cast<unsigned*>(static_cast<char*>(red) + align256(sizeof(float) * (size_t)B * kColCtas));
  cudaError_t e = cudaMemsetAsync(ticket, 0, sizeof(unsigned) * (size_t)B, s);
  if (e != cudaSuccess) return e;
  const size_t sm = sizeof(float2) * (2 * kColD * kColNC + kColD);
  static int cache[64] = {0};
  e = ensure_smem((const void*)k_ctf_cols, sm, cache);
  if (e != cudaSuccess) return e;
  const float scale = cfg.reduction == 1 ? 1.f / ((float)cfg.D * (float)cfg.D) : 1.f;
  k_ctf_cols<<<dim3(kColCtas, B), 256, sm, s>>>(qr, yr, ctf, scale, partial, ticket, loss);
  return cudaGetLastError();
}

cudaError_t launch_rows_r2c2(const float* Q, const float* Y, float2* qr, float2* yr, int B, cudaStream_t s) {
  if (B <= 0) return cudaSuccess;
  k_rows_r2c2<<<B * kColD / kRowsPerCta, 256, 0, s>>>(Q, Y, qr, yr);
  return cudaGetLastError();
}

cudaError_t launch_rows_c2r(const float2* spec, float* out, int B, cudaStream_t s) {
  if (B <= 0) return cudaSuccess;
  k_rows_c2r<<<B * kColD / (2 * kRowsPerCta), 256, 0, s>>>(spec, out);
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
