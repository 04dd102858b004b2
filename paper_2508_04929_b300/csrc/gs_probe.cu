// gs_probe_ex2: throughput probe of ex2.approx, the one special-function operation that every
// evaluated splat pixel takes (Algorithm 2 SumSplats and its backward).  The roofline that the
// render kernels are judged against is this unit's rate on the GPU at hand, so it is measured
// rather than taken from a data sheet: each thread runs kChains independent chains
// x <- ex2(x) * s - 1 (one ex2 and one FMA per step; the FMA pipe has four times the ex2
// rate, so the chains are bound by ex2), and the caller times the launch.
#include "gs_internal.cuh"

namespace gs {
namespace {

constexpr int kChains = 8;
constexpr int kProbeThreads = 256;

__global__ void __launch_bounds__(kProbeThreads) k_probe_ex2(int iters, float s, float* __restrict__ sink) {
  float x[kChains];
#pragma unroll
  for (int k = 0; k < kChains; ++k) x[k] = -1e-3f * (float)(threadIdx.x + k);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < kChains; ++k) x[k] = fmaf(ex2_approx(x[k]), s, -1.f);
  }
  float t = 0.f;
#pragma unroll
  for (int k = 0; k < kChains; ++k) t += x[k];
  if (t == 1.2345e30f) sink[0] = t;  // never true: keeps the chains alive
}

}  // namespace
}  // namespace gs

extern "C" int gs_probe_ex2(int blocks, int iters, float* sink, gs_stream_t stream, double* ex2_count) {
  if (blocks < 1 || blocks > (1 << 20) || iters < 1 || iters > (1 << 24) || !sink) return GS_EINVAL;
  gs::k_probe_ex2<<<blocks, gs::kProbeThreads, 0, (cudaStream_t)stream>>>(iters, 1.0001f, sink);
  if (ex2_count) *ex2_count = (double)blocks * gs::kProbeThreads * gs::kChains * (double)iters;
  return cudaGetLastError() == cudaSuccess ? GS_OK : GS_ECUDA;
}
