// C-ABI entry points of libgs (declared and documented in include/gs.h): argument
// validation, workspace carve-up, cuFFT plans and kernel launches.
#include <cufft.h>
#include <math.h>

#include "gs_internal.cuh"

using namespace gs;

namespace {

bool aligned(const void* p, size_t a) { return (reinterpret_cast<uintptr_t>(p) % a) == 0; }

int cuda_rc(cudaError_t e) { return e == cudaSuccess ? GS_OK : GS_ECUDA; }

}  // namespace

extern "C" {

int gs_tiles_per_image(const gs_config* cfg, int* n) {
  if (!cfg_ok(cfg) || !n) return GS_EINVAL;
  const int ntx = (cfg->D + cfg->tile - 1) / cfg->tile;
  *n = ntx * ntx;
  return GS_OK;
}

int gs_proj_size(int B, int N, size_t* bytes) {
  if (B < 0 || N < 0 || !bytes) return GS_EINVAL;
  *bytes = (sizeof(gs_record) + sizeof(int2) + sizeof(float2)) * (size_t)B * (size_t)N;
  return GS_OK;
}

int gs_workspace_size(const gs_config* cfg, int B, int N, size_t fft_work_bytes, size_t* bytes) {
  if (!cfg_ok(cfg) || !bytes || !sizes_ok(cfg, B, N)) return GS_EINVAL;
  *bytes = ws_layout(*cfg, B, N, fft_work_bytes).total;
  return GS_OK;
}

int gs_fft_create(int D, int B, gs_fft* fft) {
  if (!fft || D < 1 || D > 4096 || B < 1) return GS_EINVAL;
  fft->r2c = fft->c2r = fft->r2c_rows = fft->c2r_rows = 0;
  fft->D = D;
  fft->B = B;
  fft->work_bytes = 0;
  cufftHandle a, c;
  if (cufftCreate(&a) != CUFFT_SUCCESS) return GS_ECUDA;
  if (cufftCreate(&c) != CUFFT_SUCCESS) { cufftDestroy(a); return GS_ECUDA; }
  cufftSetAutoAllocation(a, 0);
  cufftSetAutoAllocation(c, 0);
  int n[2] = {D, D};
  size_t wa = 0, wc = 0;
  if (cufftMakePlanMany(a, 2, n, nullptr, 1, D * D, nullptr, 1, D * (D / 2 + 1), CUFFT_R2C, B, &wa) !=
          CUFFT_SUCCESS ||
      cufftMakePlanMany(c, 2, n, nullptr, 1, D * (D / 2 + 1), nullptr, 1, D * D, CUFFT_C2R, B, &wc) !=
          CUFFT_SUCCESS) {
    cufftDestroy(a);
    cufftDestroy(c);
    return GS_ECUDA;
  }
  fft->r2c = (int)a;
  fft->c2r = (int)c;
  fft->work_bytes = wa > wc ? wa : wc;
  return GS_OK;
}

int gs_fft_destroy(gs_fft* fft) {
  if (!fft) return GS_EINVAL;
  if (fft->r2c) cufftDestroy((cufftHandle)fft->r2c);
  if (fft->c2r) cufftDestroy((cufftHandle)fft->c2r);
  if (fft->r2c_rows) cufftDestroy((cufftHandle)fft->r2c_rows);
  if (fft->c2r_rows) cufftDestroy((cufftHandle)fft->c2r_rows);
  fft->r2c = fft->c2r = fft->r2c_rows = fft->c2r_rows = 0;
  return GS_OK;
}

int gs_read_status(const void* ws, gs_stream_t stream, int clear, int* status) {
  if (!ws || !status) return GS_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  int* dev = (int*)const_cast<void*>(ws);
  if (cudaMemcpyAsync(status, dev, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess) return GS_ECUDA;
  if (cudaStreamSynchronize(s) != cudaSuccess) return GS_ECUDA;
  if (clear && cudaMemsetAsync(dev, 0, sizeof(int), s) != cudaSuccess) return GS_ECUDA;
  return GS_OK;
}

int gs_clear_status(void* ws, gs_stream_t stream) {
  if (!ws) return GS_EINVAL;
  return cuda_rc(cudaMemsetAsync(ws, 0, sizeof(int), (cudaStream_t)stream));
}

int gs_project(const gs_config* cfg, const float* theta, int N, const float* W, int B, gs_record* proj,
               void* ws, size_t ws_bytes, gs_stream_t stream) {
  if (!cfg_ok(cfg) || !sizes_ok(cfg, B, N)) return GS_EINVAL;
  if (N > 0 && (!theta || !ws)) return GS_EINVAL;
  if (N > 0 && B > 0 && (!W || !proj || !aligned(proj, 16))) return GS_EINVAL;
  if (!ws || !aligned(ws, 256)) return GS_EINVAL;
  const WsLayout L = ws_layout(*cfg, B, N, 0);
  if (ws_bytes < L.spec) return GS_ENOSPC;  // everything before the spectrum area
  cudaStream_t s = (cudaStream_t)stream;
  float* gauss = ws_ptr<float>(ws, L.gauss);
  int* status = ws_ptr<int>(ws, L.status);
  cudaError_t e = launch_activate(theta, N, gauss, ws_ptr<float>(ws, L.gacc), status, s);
  if (e == cudaSuccess) e = launch_project(*cfg, gauss, N, W, B, proj, status, s);
  return cuda_rc(e);
}

int gs_bin_sort(const gs_config* cfg, const gs_record* proj, int B, int N, void* ws, size_t ws_bytes,
                uint32_t* pair_gauss, size_t pair_capacity, uint32_t* tile_ranges, uint32_t* n_pairs,
                gs_stream_t stream) {
  if (!cfg_ok(cfg) || !sizes_ok(cfg, B, N)) return GS_EINVAL;
  if (!ws || !aligned(ws, 256) || !n_pairs) return GS_EINVAL;
  if (B > 0 && (!tile_ranges || (N > 0 && !proj))) return GS_EINVAL;
  if (pair_capacity > 0 && !pair_gauss) return GS_EINVAL;
  if (pair_capacity > 0xffffffffull) pair_capacity = 0xffffffffull;
  const WsLayout L = ws_layout(*cfg, B, N, 0);
  if (ws_bytes < L.spec) return GS_ENOSPC;
  cudaStream_t s = (cudaStream_t)stream;
  if (B == 0) return cuda_rc(cudaMemsetAsync(n_pairs, 0, sizeof(uint32_t), s));
  return cuda_rc(launch_bin(*cfg, L, proj, B, N, ws, pair_gauss, pair_capacity, tile_ranges, n_pairs, s));
}

int gs_render_fwd(const gs_config* cfg, const gs_record* proj, int N, const uint32_t* pair_gauss,
                  const uint32_t* tile_ranges, int B, float* Q, gs_stream_t stream) {
  if (!cfg_ok(cfg) || !sizes_ok(cfg, B, N)) return GS_EINVAL;
  if (B > 0 && (!tile_ranges || !Q)) return GS_EINVAL;
  if (proj && !aligned(proj, 16)) return GS_EINVAL;
  return cuda_rc(launch_render_fwd(*cfg, proj, N, pair_gauss, tile_ranges, B, Q, (cudaStream_t)stream));
}

int gs_apply_ctf(const gs_config* cfg, const float* in, const float* ctf, int B, float* out, const gs_fft* fft,
                 void* ws, size_t ws_bytes, gs_stream_t stream) {
  if (!cfg_ok(cfg) || B < 0 || B > 65535) return GS_EINVAL;
  if (B == 0) return GS_OK;
  if (!in || !ctf || !out || !fft || !ws || !aligned(ws, 256) || in == out) return GS_EINVAL;
  if (fft->D != cfg->D || fft->B != B) return GS_EINVAL;
  // The half spectra and the cuFFT work area occupy the tail of the workspace (the last
  // two parts of the layout of gs_workspace_size), so this call does not need N.
  cudaStream_t s = (cudaStream_t)stream;
  const size_t spec_bytes = align256(2 * sizeof(float) * (size_t)B * cfg->D * (cfg->D / 2 + 1));
  const size_t need = spec_bytes + align256(fft->work_bytes);
  if (ws_bytes < need) return GS_ENOSPC;
  const size_t spec_off = (ws_bytes - need) & ~size_t(255);
  float2* spec = ws_ptr<float2>(ws, spec_off);
  void* work = ws_ptr<void>(ws, spec_off + spec_bytes);
  cufftHandle a = (cufftHandle)fft->r2c, c = (cufftHandle)fft->c2r;
  if (cufftSetStream(a, s) != CUFFT_SUCCESS || cufftSetStream(c, s) != CUFFT_SUCCESS) return GS_ECUDA;
  if (cufftSetWorkArea(a, work) != CUFFT_SUCCESS || cufftSetWorkArea(c, work) != CUFFT_SUCCESS) return GS_ECUDA;
  if (cufftExecR2C(a, const_cast<float*>(in), reinterpret_cast<cufftComplex*>(spec)) != CUFFT_SUCCESS)
    return GS_ECUDA;
  cudaError_t e = launch_ctf_mul(*cfg, spec, ctf, B, s);
  if (e != cudaSuccess) return GS_ECUDA;
  if (cufftExecC2R(c, reinterpret_cast<cufftComplex*>(spec), out) != CUFFT_SUCCESS) return GS_ECUDA;
  return GS_OK;
}

int gs_ctf_loss_grad(const gs_config* cfg, const float* Q, const float* Y, const float* ctf, int B, float* loss,
                     float* dLdQ, const gs_fft* fft, void* ws, size_t ws_bytes, gs_stream_t stream) {
  if (!cfg_ok(cfg) || B < 0 || B > 65535) return GS_EINVAL;
  if (B == 0) return GS_OK;
  if (!Q || !Y || !ctf || !loss || !dLdQ || !fft || !ws || !aligned(ws, 256)) return GS_EINVAL;
  if (fft->D != cfg->D || fft->B != B) return GS_EINVAL;
  // two half spectra, the cuFFT work area and the loss partial sums at the tail of the workspace
  cudaStream_t s = (cudaStream_t)stream;
  const size_t spec_bytes = align256(2 * sizeof(float) * (size_t)B * cfg->D * (cfg->D / 2 + 1));
  const size_t work_bytes = align256(fft->work_bytes);
  const size_t need = 2 * spec_bytes + work_bytes + ctf_cols_red_bytes(B);
  if (ws_bytes < need) return GS_ENOSPC;
  const size_t off = (ws_bytes - need) & ~size_t(255);
  float2* specY = ws_ptr<float2>(ws, off);
  float2* specQ = ws_ptr<float2>(ws, off + spec_bytes);
  void* work = ws_ptr<void>(ws, off + 2 * spec_bytes);
  if (cfg->D == 256) {
    // the row transforms (Q and Y in one launch, then the C2R), and the column FFTs, the
    // pointwise step and the inverse column FFT in one kernel: no cuFFT on this path
    if (launch_rows_r2c2(Q, Y, specQ, specY, B, s) != cudaSuccess) return GS_ECUDA;
    if (launch_ctf_cols(*cfg, specQ, specY, ctf, B, loss, ws_ptr<void>(ws, off + 2 * spec_bytes + work_bytes), s) !=
        cudaSuccess)
      return GS_ECUDA;
    if (launch_rows_c2r(specQ, dLdQ, B, s) != cudaSuccess) return GS_ECUDA;
    return GS_OK;
  }
  cufftHandle a = (cufftHandle)fft->r2c, c = (cufftHandle)fft->c2r;
  if (cufftSetStream(a, s) != CUFFT_SUCCESS || cufftSetStream(c, s) != CUFFT_SUCCESS) return GS_ECUDA;
  if (cufftSetWorkArea(a, work) != CUFFT_SUCCESS || cufftSetWorkArea(c, work) != CUFFT_SUCCESS) return GS_ECUDA;
  if (cufftExecR2C(a, const_cast<float*>(Q), reinterpret_cast<cufftComplex*>(specQ)) != CUFFT_SUCCESS)
    return GS_ECUDA;
  if (cufftExecR2C(a, const_cast<float*>(Y), reinterpret_cast<cufftComplex*>(specY)) != CUFFT_SUCCESS)
    return GS_ECUDA;
  if (launch_ctf_loss(*cfg, specQ, specY, ctf, B, loss, s) != cudaSuccess) return GS_ECUDA;
  if (cufftExecC2R(c, reinterpret_cast<cufftComplex*>(specQ), dLdQ) != CUFFT_SUCCESS) return GS_ECUDA;
  return GS_OK;
}

int gs_loss(const gs_config* cfg, const float* X, const float* Y, int B, float* loss, float* dLdX,
            gs_stream_t stream) {
  if (!cfg_ok(cfg) || B < 0) return GS_EINVAL;
  if (B > 0 && (!X || !Y || !loss)) return GS_EINVAL;
  return cuda_rc(launch_loss(*cfg, X, Y, B, loss, dLdX, (cudaStream_t)stream));
}

static int render_bwd_impl(const gs_config* cfg, const float* theta, int N, const float* W, int B,
                           const gs_record* proj, const uint32_t* pair_gauss, const uint32_t* tile_ranges,
                           const float* dLdQ, float* dtheta, float* dpose, void* ws, size_t ws_bytes,
                           gs_stream_t stream) {
  if (!cfg_ok(cfg) || !sizes_ok(cfg, B, N)) return GS_EINVAL;
  if (!ws || !aligned(ws, 256)) return GS_EINVAL;
  if (N > 0 && (!theta || !dtheta)) return GS_EINVAL;
  if (N > 0 && B > 0 && (!W || !proj || !tile_ranges || !dLdQ || !aligned(proj, 16))) return GS_EINVAL;
  if (dpose && !aligned(dpose, 16)) return GS_EINVAL;
  const WsLayout L = ws_layout(*cfg, B, N, 0);
  if (ws_bytes < L.spec) return GS_ENOSPC;
  cudaStream_t s = (cudaStream_t)stream;
  float* gacc = ws_ptr<float>(ws, L.gacc);
  const float* gauss = ws_ptr<float>(ws, L.gauss);
  cudaError_t e = launch_render_bwd(*cfg, proj, N, pair_gauss, tile_ranges, B, dLdQ, W, gacc, gauss, dpose, s);
  if (e == cudaSuccess) e = launch_bwd_finalize(theta, gauss, N, gacc, dtheta, s);
  return cuda_rc(e);
}

int gs_render_bwd(const gs_config* cfg, const float* theta, int N, const float* W, int B, const gs_record* proj,
                  const uint32_t* pair_gauss, const uint32_t* tile_ranges, const float* dLdQ, float* dtheta,
                  void* ws, size_t ws_bytes, gs_stream_t stream) {
  return render_bwd_impl(cfg, theta, N, W, B, proj, pair_gauss, tile_ranges, dLdQ, dtheta, nullptr, ws, ws_bytes,
                         stream);
}

int gs_render_bwd_pose(const gs_config* cfg, const float* theta, int N, const float* W, int B, const gs_record* proj,
                       const uint32_t* pair_gauss, const uint32_t* tile_ranges, const float* dLdQ, float* dtheta,
                       float* dpose, void* ws, size_t ws_bytes, gs_stream_t stream) {
  if (B > 0 && !dpose) return GS_EINVAL;
  return render_bwd_impl(cfg, theta, N, W, B, proj, pair_gauss, tile_ranges, dLdQ, dtheta, dpose, ws, ws_bytes,
                         stream);
}

int gs_step(float* theta, const float* dtheta, float* m, float* v, int n, int t, float lr, float beta1,
            float beta2, float eps, gs_stream_t stream) {
  if (n < 0 || t < 1) return GS_EINVAL;
  if (n > 0 && (!theta || !dtheta || !m || !v)) return GS_EINVAL;
  const double c1 = 1.0 / (1.0 - pow((double)beta1, (double)t));
  const double c2 = 1.0 / (1.0 - pow((double)beta2, (double)t));
  return cuda_rc(launch_adam(theta, dtheta, m, v, n, lr, beta1, beta2, eps, (float)c1, (float)c2,
                             (cudaStream_t)stream));
}

int gs_step_counted(float* theta, const float* dtheta, float* m, float* v, int n, int* t_dev, float lr,
                    float beta1, float beta2, float eps, gs_stream_t stream) {
  if (n < 0 || !t_dev) return GS_EINVAL;
  if (n > 0 && (!theta || !dtheta || !m || !v)) return GS_EINVAL;
  return cuda_rc(launch_adam_counted(theta, dtheta, m, v, n, t_dev, lr, beta1, beta2, eps, (cudaStream_t)stream));
}

}  // extern "C"
