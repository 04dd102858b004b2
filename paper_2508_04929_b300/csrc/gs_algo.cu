// The two remaining steps of Algorithm 1 around the hot path: FourierShift of the observed
// images (center alignment with the published translations, Sec. 4.1) and SplitGaussian
// (the optional densification).  The paper gives no formula for either; the definitions are
// the library's own and are restated in gs.h.
//
// k_shift_mul multiplies the R2C half spectrum of each image by the separable phase
// exp(-2 pi i (m s_x + l s_y) / D) (s_x = t_x / h columns, s_y = -t_y / h rows; cos(pi s) at
// the Nyquist index of an axis for even D) and by 1 / D^2.  The D / 2 + 1 column and D row
// factors of an image are formed in FP64 (sincospi) in shared memory by each CTA, so the
// per-coefficient work is one complex multiply.
#include <cufft.h>

#include "gs_internal.cuh"

namespace gs {
namespace {

__global__ void k_shift_mul(float2* __restrict__ spec, const float* __restrict__ t, int D, double inv_h) {
  extern __shared__ float2 fac[];  // column factors [D / 2 + 1], then row factors [D]
  const int b = blockIdx.y, W2 = D / 2 + 1;
  float2* colf = fac;
  float2* rowf = fac + W2;
  const double sx = (double)t[2 * b] * inv_h, sy = -(double)t[2 * b + 1] * inv_h;
  const double scale = 1.0 / ((double)D * (double)D);
  for (int k = threadIdx.x; k < W2 + D; k += blockDim.x) {
    const bool col = k < W2;
    const int idx = col ? k : k - W2;
    const int f = col ? idx : (idx < (D + 1) / 2 ? idx : idx - D);  // signed frequency index
    const double s = col ? sx : sy;
    double re, im;
    if ((D & 1) == 0 && 2 * idx == D) {
      re = cospi(s);
      im = 0.0;
    } else {
      sincospi(-2.0 * (double)f * s / (double)D, &im, &re);
    }
    if (col) {
      re *= scale;
      im *= scale;
    }
    (col ? colf : rowf)[idx] = make_float2((float)re, (float)im);
  }
  __syncthreads();
  float2* img = spec + (size_t)b * D * W2;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < D * W2; e += gridDim.x * blockDim.x) {
    const int l = e / W2, m = e - l * W2;
    const float2 c = colf[m], r = rowf[l];
    const float2 h = make_float2(c.x * r.x - c.y * r.y, c.x * r.y + c.y * r.x);
    const float2 v = img[e];
    img[e] = make_float2(v.x * h.x - v.y * h.y, v.x * h.y + v.y * h.x);
  }
}

__device__ __forceinline__ double softplus_d(double x) { return log1p(exp(-fabs(x))) + fmax(x, 0.0); }
__device__ __forceinline__ double inv_softplus_d(double y) { return y > 30.0 ? y : log(expm1(y)); }

// Moment-preserving split: children at mu +- alpha s_max v (v the rotation's column of the
// largest scale, lower index on ties), amplitude A / 2, major scale s_max sqrt(1 - alpha^2).
// Rows g (first child) and N + g (second child) of out.
__global__ void k_split(const float* __restrict__ theta, int N, double alpha, float* __restrict__ out) {
  const int g = blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= N) return;
  const float* th = theta + (size_t)g * 11;
  double s[3];
  for (int a = 0; a < 3; ++a) s[a] = softplus_d(th[3 + a]);
  int m = 0;
  if (s[1] > s[m]) m = 1;
  if (s[2] > s[m]) m = 2;
  const double qn = sqrt((double)th[6] * th[6] + (double)th[7] * th[7] + (double)th[8] * th[8] + (double)th[9] * th[9]);
  const double w = th[6] / qn, x = th[7] / qn, y = th[8] / qn, z = th[9] / qn;
  double v[3];  // column m of R(q) (Sec. 3.3.1)
  if (m == 0) {
    v[0] = 1 - 2 * (y * y + z * z); v[1] = 2 * (x * y + w * z); v[2] = 2 * (x * z - w * y);
  } else if (m == 1) {
    v[0] = 2 * (x * y - w * z); v[1] = 1 - 2 * (x * x + z * z); v[2] = 2 * (y * z + w * x);
  } else {
    v[0] = 2 * (x * z + w * y); v[1] = 2 * (y * z - w * x); v[2] = 1 - 2 * (x * x + y * y);
  }
  const double d = alpha * s[m];
  const float sm = (float)inv_softplus_d(s[m] * sqrt(1.0 - alpha * alpha));
  const float an = (float)inv_softplus_d(softplus_d(th[10]) * 0.5);
  for (int c = 0; c < 2; ++c) {
    float* o = out + ((size_t)c * N + g) * 11;
    const double sign = c == 0 ? 1.0 : -1.0;
    for (int a = 0; a < 3; ++a) o[a] = (float)((double)th[a] + sign * d * v[a]);
    for (int a = 0; a < 3; ++a) o[3 + a] = a == m ? sm : th[3 + a];
    for (int a = 0; a < 4; ++a) o[6 + a] = th[6 + a];
    o[10] = an;
  }
}

int rc(cudaError_t e) { return e == cudaSuccess ? GS_OK : GS_ECUDA; }

bool shift_cfg_ok(const gs_config* c) { return c && c->D >= 1 && c->D <= 4096 && c->E > 0.f; }

}  // namespace
}  // namespace gs

using namespace gs;

extern "C" {

int gs_fourier_shift(const gs_config* cfg, const float* in, const float* t, int B, float* out, const gs_fft* fft,
                     void* ws, size_t ws_bytes, gs_stream_t stream) {
  if (!shift_cfg_ok(cfg) || B < 0 || B > 65535) return GS_EINVAL;
  if (B == 0) return GS_OK;
  if (!in || !t || !out || !fft || !ws || ((uintptr_t)ws & 255) || in == out) return GS_EINVAL;
  if (fft->D != cfg->D || fft->B != B) return GS_EINVAL;
  const int D = cfg->D;
  // half spectra and cuFFT work area at the tail of the workspace, as for gs_apply_ctf
  const size_t spec_bytes = align256(2 * sizeof(float) * (size_t)B * D * (D / 2 + 1));
  const size_t need = spec_bytes + align256(fft->work_bytes);
  if (ws_bytes < need) return GS_ENOSPC;
  const size_t spec_off = (ws_bytes - need) & ~size_t(255);
  float2* spec = ws_ptr<float2>(ws, spec_off);
  void* work = ws_ptr<void>(ws, spec_off + spec_bytes);
  cudaStream_t s = (cudaStream_t)stream;
  cufftHandle a = (cufftHandle)fft->r2c, c = (cufftHandle)fft->c2r;
  if (cufftSetStream(a, s) != CUFFT_SUCCESS || cufftSetStream(c, s) != CUFFT_SUCCESS) return GS_ECUDA;
  if (cufftSetWorkArea(a, work) != CUFFT_SUCCESS || cufftSetWorkArea(c, work) != CUFFT_SUCCESS) return GS_ECUDA;
  if (cufftExecR2C(a, const_cast<float*>(in), reinterpret_cast<cufftComplex*>(spec)) != CUFFT_SUCCESS)
    return GS_ECUDA;
  const size_t sm = sizeof(float2) * ((size_t)D / 2 + 1 + D);
  static int cache[64] = {0};
  cudaError_t e = ensure_smem((const void*)k_shift_mul, sm, cache);
  if (e != cudaSuccess) return rc(e);
  const int cnt = D * (D / 2 + 1);
  int per_image = (cnt + 255) / 256;
  if (per_image > 8) per_image = 8;
  const double inv_h = (double)D / (2.0 * (double)cfg->E);
  k_shift_mul<<<dim3(per_image, B), 256, sm, s>>>(spec, t, D, inv_h);
  e = cudaGetLastError();
  if (e != cudaSuccess) return rc(e);
  if (cufftExecC2R(c, reinterpret_cast<cufftComplex*>(spec), out) != CUFFT_SUCCESS) return GS_ECUDA;
  return GS_OK;
}

int gs_split_gaussians(const float* theta, int N, float alpha, float* out, gs_stream_t stream) {
  if (N < 0 || !(alpha >= 0.f && alpha < 1.f)) return GS_EINVAL;
  if (N == 0) return GS_OK;
  if (!theta || !out || theta == out) return GS_EINVAL;
  k_split<<<(N + 255) / 256, 256, 0, (cudaStream_t)stream>>>(theta, N, (double)alpha, out);
  return rc(cudaGetLastError());
}

}  // extern "C"
