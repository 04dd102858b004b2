// CreateTiles, DuplicateWithKeys, SortByKeys and IdentifyTileRanges (Algorithm 2).
//
// Every (particle b, Gaussian g) with a non-empty support box is instantiated once per
// tile its box touches.  The instances are ordered by the key (b, tile, g).  Because the
// Gaussians are visited in index order, a single stable counting-sort pass on the tile
// digit produces that order (it is the last pass of an LSD radix sort keyed on
// (tile, Gaussian), the Gaussian digits being sorted already), and the scan of the tile
// histogram gives the tile ranges directly.
//
//   k_bin_count   (chunk, b): per-chunk tile histogram (chunk = kBinChunk Gaussians)
//   k_bin_scan    (b):        per tile, exclusive scan over chunks; exclusive scan over tiles
//   k_bin_base    (1 CTA):    exclusive scan over particles (64-bit), total instance count
//   k_bin_scatter (chunk, b): stable ranks inside the chunk (8 warps in order, 32 lanes in
//                             order), scatter of the Gaussian indices, tile ranges
//
// Inside a warp the rank of lane l's instance in tile (tx, ty) is the number of lower lanes
// whose box covers that tile: popc(colmask[tx] & rowmask[ty] & lanemask_lt), where
// colmask[tx] / rowmask[ty] are the lanes whose tile-column / tile-row range holds tx / ty,
// obtained for all tx at once by a 32 x 32 bit transpose of the lanes' range masks.
#include "gs_internal.cuh"

namespace gs {
namespace {

struct TileRect {
  int tx0, tx1, ty0, ty1;
};

__device__ __forceinline__ bool load_rect(const gs_record* proj, size_t idx, int T, TileRect& r) {
  const int2 bx = *reinterpret_cast<const int2*>(reinterpret_cast<const char*>(proj + idx) + 24);
  int x0 = (int)(int16_t)(bx.x & 0xffff), x1 = (int)(int16_t)((unsigned)bx.x >> 16);
  int y0 = (int)(int16_t)(bx.y & 0xffff), y1 = (int)(int16_t)((unsigned)bx.y >> 16);
  if (x0 > x1 || y0 > y1) return false;
  r.tx0 = x0 / T; r.tx1 = x1 / T; r.ty0 = y0 / T; r.ty1 = y1 / T;
  return true;
}

// Bits [lo, hi] of the 32-bit word that holds positions [base, base + 32) (0 if disjoint).
__device__ __forceinline__ unsigned range_bits(int lo, int hi, int base) {
  lo -= base;
  hi -= base;
  if (hi < 0 || lo > 31 || lo > hi) return 0u;
  lo = max(lo, 0);
  hi = min(hi, 31);
  const unsigned up = hi >= 31 ? 0xffffffffu : ((2u << hi) - 1u);
  return up & ~((1u << lo) - 1u);
}

// Transpose of the 32 x 32 bit matrix whose row l is lane l's word: on return lane x
// holds column x (bit l = bit x of lane l's input).
__device__ __forceinline__ unsigned transpose32(unsigned x) {
  const int lane = threadIdx.x & 31;
  const unsigned masks[5] = {0x0000ffffu, 0x00ff00ffu, 0x0f0f0f0fu, 0x33333333u, 0x55555555u};
#pragma unroll
  for (int s = 0; s < 5; ++s) {
    const int j = 16 >> s;
    const unsigned m = masks[s];
    const unsigned o = __shfl_xor_sync(0xffffffffu, x, j);
    x = (lane & j) ? ((x & ~m) | ((o & ~m) >> j)) : ((x & m) | ((o & m) << j));
  }
  return x;
}

__global__ void k_bin_count(const gs_record* __restrict__ proj, int N, int T, int ntx, int Tn, int C,
                            uint32_t* __restrict__ hist) {
  extern __shared__ uint32_t h[];
  const int c = blockIdx.x, b = blockIdx.y;
  for (int t = threadIdx.x; t < Tn; t += blockDim.x) h[t] = 0;
  __syncthreads();
  const int g0 = c * kBinChunk, g1 = min(N, g0 + kBinChunk);
  for (int g = g0 + threadIdx.x; g < g1; g += blockDim.x) {
    TileRect r;
    if (!load_rect(proj, (size_t)b * N + g, T, r)) continue;
    for (int ty = r.ty0; ty <= r.ty1; ++ty)
      for (int tx = r.tx0; tx <= r.tx1; ++tx) atomicAdd(&h[ty * ntx + tx], 1u);
  }
  __syncthreads();
  uint32_t* out = hist + ((size_t)b * C + c) * Tn;
  for (int t = threadIdx.x; t < Tn; t += blockDim.x) out[t] = h[t];
}

// Block-wide exclusive scan of up to 4096 values held in shared memory (1024 threads).
__device__ uint32_t block_exclusive_scan(uint32_t* v, int n) {
  __shared__ uint32_t wsum[32];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int per = (n + blockDim.x - 1) / blockDim.x;  // <= 4
  uint32_t loc[4];
  uint32_t s = 0;
  for (int k = 0; k < per; ++k) {
    int i = tid * per + k;
    loc[k] = (i < n) ? v[i] : 0u;
    s += loc[k];
  }
  uint32_t incl = s;
  for (int o = 1; o < 32; o <<= 1) {
    uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += y;
  }
  if (lane == 31) wsum[warp] = incl;
  __syncthreads();
  if (warp == 0) {
    uint32_t x = (lane < (int)(blockDim.x >> 5)) ? wsum[lane] : 0u;
    uint32_t xi = x;
    for (int o = 1; o < 32; o <<= 1) {
      uint32_t y = __shfl_up_sync(0xffffffffu, xi, o);
      if (lane >= o) xi += y;
    }
    wsum[lane] = xi - x;
  }
  __syncthreads();
  uint32_t run = wsum[warp] + incl - s;
  uint32_t total = 0;
  __syncthreads();
  for (int k = 0; k < per; ++k) {
    int i = tid * per + k;
    if (i < n) v[i] = run;
    run += loc[k];
  }
  if (tid == blockDim.x - 1) wsum[0] = run;
  __syncthreads();
  total = wsum[0];
  __syncthreads();
  return total;
}

__global__ void __launch_bounds__(1024) k_bin_scan(uint32_t* __restrict__ hist, int Tn, int C, uint32_t* __restrict__ tstart,
                           uint32_t* __restrict__ ttotal, uint32_t* __restrict__ itotal) {
  extern __shared__ uint32_t sh[];  // Tn
  const int b = blockIdx.x;
  uint32_t* H = hist + (size_t)b * C * Tn;
  constexpr int kBatch = 8;  // independent loads in flight per thread
  for (int t = threadIdx.x; t < Tn; t += blockDim.x) {
    uint32_t run = 0;
    for (int c0 = 0; c0 < C; c0 += kBatch) {
      uint32_t v[kBatch];
#pragma unroll
      for (int j = 0; j < kBatch; ++j) v[j] = (c0 + j < C) ? H[(size_t)(c0 + j) * Tn + t] : 0u;
#pragma unroll
      for (int j = 0; j < kBatch; ++j) {
        if (c0 + j < C) H[(size_t)(c0 + j) * Tn + t] = run;
        run += v[j];
      }
    }
    sh[t] = run;
    ttotal[(size_t)b * Tn + t] = run;
  }
  __syncthreads();
  uint32_t total = block_exclusive_scan(sh, Tn);
  for (int t = threadIdx.x; t < Tn; t += blockDim.x) {
    const uint32_t st = sh[t];
    tstart[(size_t)b * Tn + t] = st;
    for (int c0 = 0; c0 < C; c0 += kBatch) {
      uint32_t v[kBatch];
#pragma unroll
      for (int j = 0; j < kBatch; ++j) v[j] = (c0 + j < C) ? H[(size_t)(c0 + j) * Tn + t] : 0u;
#pragma unroll
      for (int j = 0; j < kBatch; ++j)
        if (c0 + j < C) H[(size_t)(c0 + j) * Tn + t] = v[j] + st;
    }
  }
  if (threadIdx.x == 0) itotal[b] = total;
}

__global__ void k_bin_base(const uint32_t* __restrict__ itotal, int B, unsigned long long* __restrict__ ibase,
                           uint32_t* __restrict__ n_pairs, unsigned long long cap, int* __restrict__ status) {
  if (threadIdx.x != 0) return;
  unsigned long long run = 0;
  for (int b = 0; b < B; ++b) {
    ibase[b] = run;
    run += itotal[b];
  }
  ibase[B] = run;
  *n_pairs = run > 0xffffffffull ? 0xffffffffu : (uint32_t)run;
  if (run > cap) atomicOr(status, GS_STATUS_OVERFLOW);
}

__global__ void k_bin_scatter(const gs_record* __restrict__ proj, int N, int T, int ntx, int Tn, int C,
                              const uint32_t* __restrict__ hist, const uint32_t* __restrict__ tstart,
                              const uint32_t* __restrict__ ttotal,
                              const unsigned long long* __restrict__ ibase, uint32_t* __restrict__ pair_gauss,
                              unsigned long long cap, uint32_t* __restrict__ ranges) {
  extern __shared__ uint32_t cur[];  // [kBinWarps][Tn]
  const int c = blockIdx.x, b = blockIdx.y;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const unsigned long long base = ibase[b];
  for (int i = threadIdx.x; i < kBinWarps * Tn; i += blockDim.x) cur[i] = 0;
  __syncthreads();
  const int per_warp = kBinChunk / kBinWarps;
  const int g0 = c * kBinChunk + warp * per_warp;
  const int g1 = min(N, g0 + per_warp);
  uint32_t* mycur = cur + warp * Tn;
  // 1. per-warp tile histogram
  for (int g = g0 + lane; g < g1; g += 32) {
    TileRect r;
    if (!load_rect(proj, (size_t)b * N + g, T, r)) continue;
    for (int ty = r.ty0; ty <= r.ty1; ++ty)
      for (int tx = r.tx0; tx <= r.tx1; ++tx) atomicAdd(&mycur[ty * ntx + tx], 1u);
  }
  __syncthreads();
  // 2. exclusive scan over warps, offset by this chunk's start within the image
  const uint32_t* Hc = hist + ((size_t)b * C + c) * Tn;
  for (int t = threadIdx.x; t < Tn; t += blockDim.x) {
    uint32_t run = Hc[t];
    for (int w = 0; w < kBinWarps; ++w) {
      uint32_t v = cur[w * Tn + t];
      cur[w * Tn + t] = run;
      run += v;
    }
  }
  __syncthreads();
  // 3. stable scatter, 32 Gaussians per round in lane order
  const unsigned ltmask = lanemask_lt();
  const bool wide = ntx > 32;
  for (int gr = g0; gr < g1; gr += 32) {
    const int g = gr + lane;
    TileRect r;
    bool valid = (g < g1) && load_rect(proj, (size_t)b * N + g, T, r);
    if (!valid) { r.tx0 = 1; r.tx1 = 0; r.ty0 = 1; r.ty1 = 0; }
    // colmask[x] (in lane x) = lanes whose tile-column range holds x; rowmask likewise
    const unsigned colm0 = transpose32(range_bits(r.tx0, r.tx1, 0));
    const unsigned rowm0 = transpose32(range_bits(r.ty0, r.ty1, 0));
    unsigned colm1 = 0, rowm1 = 0;
    if (wide) {
      colm1 = transpose32(range_bits(r.tx0, r.tx1, 32));
      rowm1 = transpose32(range_bits(r.ty0, r.ty1, 32));
    }
    const int cnt = valid ? (r.tx1 - r.tx0 + 1) * (r.ty1 - r.ty0 + 1) : 0;
    const int kmax = (int)__reduce_max_sync(0xffffffffu, (unsigned)cnt);
    for (int pass = 0; pass < 2; ++pass) {
      int cx = r.tx0, cy = r.ty0;
      for (int k = 0; k < kmax; ++k) {
        const bool act = k < cnt;
        const int tx = act ? cx : 0, ty = act ? cy : 0;
        unsigned cm = __shfl_sync(0xffffffffu, colm0, tx & 31);
        unsigned rm = __shfl_sync(0xffffffffu, rowm0, ty & 31);
        if (wide) {
          const unsigned c1 = __shfl_sync(0xffffffffu, colm1, tx & 31);
          const unsigned r1 = __shfl_sync(0xffffffffu, rowm1, ty & 31);
          if (tx >= 32) cm = c1;
          if (ty >= 32) rm = r1;
        }
        const unsigned both = cm & rm;
        if (act) {
          const int t = ty * ntx + tx;
          if (pass == 0) {
            const unsigned long long pos = base + mycur[t] + __popc(both & ltmask);
            if (pos < cap) pair_gauss[pos] = (uint32_t)g;
          } else if ((both >> lane) == 1u) {
            mycur[t] += __popc(both);  // the highest covering lane moves the cursor
          }
        }
        if (++cx > r.tx1) { cx = r.tx0; ++cy; }
      }
      __syncwarp();
    }
  }
  // 4. tile ranges (absolute, clipped to the pair capacity)
  if (c == 0) {
    for (int t = threadIdx.x; t < Tn; t += blockDim.x) {
      unsigned long long s = base + tstart[(size_t)b * Tn + t];
      unsigned long long e = s + ttotal[(size_t)b * Tn + t];
      s = s < cap ? s : cap;
      e = e < cap ? e : cap;
      ranges[((size_t)b * Tn + t) * 2 + 0] = (uint32_t)s;
      ranges[((size_t)b * Tn + t) * 2 + 1] = (uint32_t)e;
    }
  }
}

}  // namespace

cudaError_t launch_bin(const gs_config& cfg, const WsLayout& L, const gs_record* proj, int B, int N,
                       void* ws, uint32_t* pair_gauss, size_t cap, uint32_t* ranges, uint32_t* n_pairs,
                       cudaStream_t s) {
  if (B <= 0) return cudaSuccess;
  uint32_t* hist = ws_ptr<uint32_t>(ws, L.hist);
  uint32_t* tstart = ws_ptr<uint32_t>(ws, L.tstart);
  uint32_t* ttotal = ws_ptr<uint32_t>(ws, L.ttotal);
  uint32_t* itotal = ws_ptr<uint32_t>(ws, L.itotal);
  unsigned long long* ibase = ws_ptr<unsigned long long>(ws, L.ibase);
  int* status = ws_ptr<int>(ws, L.status);
  const int T = cfg.tile, ntx = L.ntx, Tn = L.Tn, C = L.C;
  dim3 g2(C, B);
  size_t sm_count = sizeof(uint32_t) * Tn;
  cudaError_t e;
  {
    static int cache[64] = {0};
    e = ensure_smem((const void*)k_bin_count, sm_count, cache);
    if (e != cudaSuccess) return e;
  }
  k_bin_count<<<g2, 256, sm_count, s>>>(proj, N, T, ntx, Tn, C, hist);
  {
    static int cache[64] = {0};
    e = ensure_smem((const void*)k_bin_scan, sm_count, cache);
    if (e != cudaSuccess) return e;
  }
  k_bin_scan<<<B, 1024, sm_count, s>>>(hist, Tn, C, tstart, ttotal, itotal);
  k_bin_base<<<1, 32, 0, s>>>(itotal, B, ibase, n_pairs, (unsigned long long)cap, status);
  size_t sm_scatter = sizeof(uint32_t) * kBinWarps * Tn;
  {
    static int cache[64] = {0};
    e = ensure_smem((const void*)k_bin_scatter, sm_scatter, cache);
    if (e != cudaSuccess) return e;
  }
  k_bin_scatter<<<g2, 32 * kBinWarps, sm_scatter, s>>>(proj, N, T, ntx, Tn, C, hist, tstart, ttotal, ibase,
                                                      pair_gauss, (unsigned long long)cap, ranges);
  return cudaGetLastError();
}

}  // namespace gs
