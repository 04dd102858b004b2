// gs_bin_sort_noalloc: the tile binning and sort of gs_bin_sort for callers that cannot
// hand the library a workspace.
//
// Some callers of this library cannot call cudaMalloc (or any allocating routine) at the
// point where they bin a batch: a host application that owns every byte of device memory
// through its own pool and forbids allocations from plug-ins, or a pipeline that must not
// allocate once it is running because an allocation can synchronize the device and stall
// the other streams.  For them this entry point keeps its scratch in one file-scope device
// array, kGsNoallocScratchBytes (8 MiB) large, that exists on every GPU that loads the
// library until the process exits.  The caller still provides the records (input) and the
// pair list, tile ranges and pair count (outputs).
//
// The array's host-side name is not a device address, so the first call on each device
// looks the address up with cudaGetSymbolAddress (with that device current) and caches it.
// That look-up may load the library's device code, which a stream capture must not see, so
// a first call on a capturing stream is refused with GS_ECAPTURE before any other CUDA
// call; make the first call before capturing.  Every call on a device shares the
// array and leaves its contents behind; everything the kernels need to start at zero is
// cleared by this call, but two calls whose work overlaps on the GPU (e.g. on two streams
// without ordering between them) race on the array and give wrong results.
#include <mutex>

#include "gs_internal.cuh"

namespace {

constexpr size_t kGsNoallocScratchBytes = size_t(8) << 20;
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_bin_scratch[kGsNoallocScratchBytes];

std::mutex g_mutex;
void* g_scratch_addr[kMaxDevices] = {};

// Device address of g_bin_scratch on the current device, looked up once per device.  A look-up
// on a capturing stream is refused (GS_ECAPTURE) without touching the capture.
int scratch_address(cudaStream_t s, void** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return GS_ECUDA;
  if (dev < 0 || dev >= kMaxDevices) return GS_ECUDA;
  std::lock_guard<std::mutex> lock(g_mutex);
  if (!g_scratch_addr[dev]) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone) return GS_ECAPTURE;
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_bin_scratch) != cudaSuccess) return GS_ECUDA;
    g_scratch_addr[dev] = p;
  }
  *out = g_scratch_addr[dev];
  return GS_OK;
}

}  // namespace

extern "C" int gs_bin_sort_noalloc(const gs_config* cfg, const gs_record* proj, int B, int N,
                                   uint32_t* pair_gauss, size_t pair_capacity, uint32_t* tile_ranges,
                                   uint32_t* n_pairs, gs_stream_t stream, size_t* scratch_needed) {
  using namespace gs;
  if (!cfg_ok(cfg) || !sizes_ok(cfg, B, N)) return GS_EINVAL;
  if (!n_pairs || (B > 0 && (!tile_ranges || (N > 0 && !proj)))) return GS_EINVAL;
  if (pair_capacity > 0 && !pair_gauss) return GS_EINVAL;
  if (pair_capacity > 0xffffffffull) pair_capacity = 0xffffffffull;

  // Only the binning parts of the workspace layout, packed from offset 0 of the array.
  const WsLayout full = ws_layout(*cfg, B, N, 0);
  WsLayout L = full;
  size_t o = 0;
  L.status = o; o = align256(o + 256);
  L.hist = o; o = align256(o + sizeof(uint32_t) * (size_t)B * full.C * full.Tn);
  L.tstart = o; o = align256(o + sizeof(uint32_t) * (size_t)B * full.Tn);
  L.ttotal = o; o = align256(o + sizeof(uint32_t) * (size_t)B * full.Tn);
  L.itotal = o; o = align256(o + sizeof(uint32_t) * ((size_t)B + 1));
  L.ibase = o; o = align256(o + sizeof(unsigned long long) * ((size_t)B + 1));
  L.gauss = L.gacc = L.spec = L.spec2 = L.fftwork = L.total = o;
  if (scratch_needed) *scratch_needed = o;
  if (o > kGsNoallocScratchBytes) return GS_ENOSPC;

  cudaStream_t s = (cudaStream_t)stream;
  if (B == 0) return cudaMemsetAsync(n_pairs, 0, sizeof(uint32_t), s) == cudaSuccess ? GS_OK : GS_ECUDA;
  void* scratch = nullptr;
  const int rc = scratch_address(s, &scratch);
  if (rc != GS_OK) return rc;
  if (cudaMemsetAsync(scratch, 0, 256, s) != cudaSuccess) return GS_ECUDA;  // status word
  cudaError_t e = launch_bin(*cfg, L, proj, B, N, scratch, pair_gauss, pair_capacity, tile_ranges, n_pairs, s);
  return e == cudaSuccess ? GS_OK : GS_ECUDA;
}
