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
//   k_bin_scan    (tiles, b): per tile, exclusive scan over chunks
//   k_bin_tiles   (b):        exclusive scan over tiles
//   k_bin_base    (1 warp):   exclusive scan over particles (64-bit), total instance count
//   k_bin_scatter (chunk, b): stable ranks inside the chunk (8 warps in order, 32 lanes in
//                             order), scatter of the Gaussian indices, tile ranges
//
// The boxes are read from the 8-byte box plane that gs_project writes after the records,
// so each pass reads a quarter of the bytes of the full records.
//
// k_bin_count adds each box as the four corners of a 2-D difference array (+1 at
// (tx0, ty0) and (tx1 + 1, ty1 + 1), -1 at (tx1 + 1, ty0) and (tx0, ty1 + 1); corners past
// the grid are dropped) and takes the 2-D inclusive prefix sum once per chunk: four shared
// atomics per Gaussian whatever the size of its box.
//
// The scatter walks the instances of 32 consecutive Gaussians (lane-major, row-major inside
// a box) in windows of 32, one instance per lane, so a warp's cost follows the total number
// of instances rather than the largest box among its lanes.  The rank of lane l's instance
// in tile (tx, ty) is the number of lower lanes whose box covers that tile:
// popc(colmask[tx] & rowmask[ty] & lanemask_lt(l)), where colmask[tx] / rowmask[ty] are the
// lanes whose tile-column / tile-row range holds tx / ty, obtained for all tx at once by a
// 32 x 32 bit transpose of the lanes' range masks; the highest covering lane moves the
// tile's cursor.
#include "gs_internal.cuh"

namespace gs {
namespace {

struct TileRect {
  int tx0, tx1, ty0, ty1;
};

// Tile rectangle of a box of the plane ({x0 | x1 << 16, y0 | y1 << 16}); false if empty.
// Boxes are clipped to the image, so the pixel bounds are non-negative and tile = pixel >> sh.
__device__ __forceinline__ bool unpack_rect(const int2 bx, int sh, TileRect& r) {
  int x0 = (int)(int16_t)(bx.x & 0xffff), x1 = (int)(int16_t)((unsigned)bx.x >> 16);
  int y0 = (int)(int16_t)(bx.y & 0xffff), y1 = (int)(int16_t)((unsigned)bx.y >> 16);
  if (x0 > x1 || y0 > y1) return false;
  r.tx0 = x0 >> sh; r.tx1 = x1 >> sh; r.ty0 = y0 >> sh; r.ty1 = y1 >> sh;
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

// In-place 2-D inclusive prefix sum of the n x n array h (row-major) by the whole CTA:
// along rows one warp per row (shuffle scans of 32 columns), then down columns one thread
// per column.  Unsigned wrap-around is exact: every result is a count.
__device__ void prefix2d(uint32_t* h, int n) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int y = warp; y < n; y += nw) {
    uint32_t carry = 0;
    for (int x0 = 0; x0 < n; x0 += 32) {
      const int x = x0 + lane;
      uint32_t v = x < n ? h[y * n + x] : 0u;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const uint32_t u = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += u;
      }
      if (x < n) h[y * n + x] = v + carry;
      carry += __shfl_sync(0xffffffffu, v, 31);
    }
  }
  __syncthreads();
  for (int x = threadIdx.x; x < n; x += blockDim.x) {
    uint32_t run = 0;
    for (int y = 0; y < n; ++y) {
      run += h[y * n + x];
      h[y * n + x] = run;
    }
  }
  __syncthreads();
}

__global__ void k_bin_count(const int2* __restrict__ boxes, int N, int sh, int ntx, int Tn, int C,
                            uint32_t* __restrict__ hist) {
  extern __shared__ uint32_t h[];
  const int c = blockIdx.x, b = blockIdx.y;
  for (int t = threadIdx.x; t < Tn; t += blockDim.x) h[t] = 0;
  __syncthreads();
  const int g0 = c * kBinChunk, g1 = min(N, g0 + kBinChunk);
  constexpr int kPer = kBinChunk / 256;  // boxes per thread (blockDim 256), loaded up front
  int2 bxs[kPer];
  const int2* bb = boxes + (size_t)b * N;
#pragma unroll
  for (int j = 0; j < kPer; ++j) {
    const int g = g0 + (int)threadIdx.x + 256 * j;
    bxs[j] = g < g1 ? __ldg(bb + g) : make_int2(1, 0);  // x0 = 1 > x1 = 0: empty
  }
#pragma unroll
  for (int j = 0; j < kPer; ++j) {
    TileRect r;
    if (!unpack_rect(bxs[j], sh, r)) continue;
    const bool xe = r.tx1 + 1 < ntx, ye = r.ty1 + 1 < ntx;
    atomicAdd(&h[r.ty0 * ntx + r.tx0], 1u);
    if (xe) atomicAdd(&h[r.ty0 * ntx + r.tx1 + 1], 0xffffffffu);
    if (ye) atomicAdd(&h[(r.ty1 + 1) * ntx + r.tx0], 0xffffffffu);
    if (xe && ye) atomicAdd(&h[(r.ty1 + 1) * ntx + r.tx1 + 1], 1u);
  }
  __syncthreads();
  prefix2d(h, ntx);
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

// Per tile, the exclusive scan of its counts over the chunks, in place (each chunk's offset
// inside the tile's run), and the tile's total; 256 tiles of one particle image per CTA.  The
// loads of the next 8 chunks are issued before the stores of the current 8.
__global__ void __launch_bounds__(256) k_bin_scan(uint32_t* __restrict__ hist, int Tn, int C,
                                                  uint32_t* __restrict__ ttotal) {
  const int b = blockIdx.y, t = blockIdx.x * 256 + (int)threadIdx.x;
  if (t >= Tn) return;
  uint32_t* H = hist + (size_t)b * C * Tn + t;
  constexpr int kBatch = 8;
  uint32_t nxt[kBatch];
#pragma unroll
  for (int j = 0; j < kBatch; ++j) nxt[j] = j < C ? H[(size_t)j * Tn] : 0u;
  uint32_t run = 0;
  for (int c0 = 0; c0 < C; c0 += kBatch) {
    uint32_t v[kBatch];
#pragma unroll
    for (int j = 0; j < kBatch; ++j) v[j] = nxt[j];
#pragma unroll
    for (int j = 0; j < kBatch; ++j) nxt[j] = c0 + kBatch + j < C ? H[(size_t)(c0 + kBatch + j) * Tn] : 0u;
#pragma unroll
    for (int j = 0; j < kBatch; ++j) {
      if (c0 + j < C) H[(size_t)(c0 + j) * Tn] = run;
      run += v[j];
    }
  }
  ttotal[(size_t)b * Tn + t] = run;
}

// Per particle image, the exclusive scan of the tile totals (each tile's start inside the
// image's instances) and the image's total.
__global__ void __launch_bounds__(1024) k_bin_tiles(const uint32_t* __restrict__ ttotal, int Tn,
                                                    uint32_t* __restrict__ tstart, uint32_t* __restrict__ itotal) {
  extern __shared__ uint32_t sh[];  // Tn
  const int b = blockIdx.x;
  for (int t = threadIdx.x; t < Tn; t += blockDim.x) sh[t] = ttotal[(size_t)b * Tn + t];
  __syncthreads();
  const uint32_t total = block_exclusive_scan(sh, Tn);
  // the chunk offsets stay relative to the tile's start; k_bin_scatter adds tstart
  for (int t = threadIdx.x; t < Tn; t += blockDim.x) tstart[(size_t)b * Tn + t] = sh[t];
  if (threadIdx.x == 0) itotal[b] = total;
}

// Exclusive scan over the particles' instance counts (64-bit) by one warp: each lane sums a
// contiguous run of particles, the lanes' sums are scanned by shuffles, and each lane writes
// its run's bases.
__global__ void k_bin_base(const uint32_t* __restrict__ itotal, int B, unsigned long long* __restrict__ ibase,
                           uint32_t* __restrict__ n_pairs, unsigned long long cap, int* __restrict__ status) {
  const int lane = threadIdx.x;
  const int per = (B + 31) / 32, b0 = min(B, lane * per), b1 = min(B, b0 + per);
  unsigned long long mine = 0;
  for (int b = b0; b < b1; ++b) mine += itotal[b];
  unsigned long long incl = mine;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const unsigned long long u = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += u;
  }
  unsigned long long run = incl - mine;
  for (int b = b0; b < b1; ++b) {
    ibase[b] = run;
    run += itotal[b];
  }
  const unsigned long long total = __shfl_sync(0xffffffffu, incl, 31);
  if (lane == 0) {
    ibase[B] = total;
    *n_pairs = total > 0xffffffffull ? 0xffffffffu : (uint32_t)total;
    if (total > cap) atomicOr(status, GS_STATUS_OVERFLOW);
  }
}

__global__ void k_bin_scatter(const int2* __restrict__ boxes, int N, int sh, int ntx, int Tn, int sp, int C,
                              const uint32_t* __restrict__ hist, const uint32_t* __restrict__ tstart,
                              const uint32_t* __restrict__ ttotal,
                              const unsigned long long* __restrict__ ibase, uint32_t* __restrict__ pair_gauss,
                              unsigned long long cap, uint32_t* __restrict__ ranges) {
  // shared: [kBinWarps][ntx rows of sp] cursors, [kBinWarps][32] window owners, [65] k / w multipliers.
  // The cursor rows are sp = 3 (mod 32) words apart, so the tiles of a small box, which a window
  // touches together, fall in distinct banks (tx + 3 ty differs for boxes up to 3 tiles wide)
  extern __shared__ uint32_t cur[];
  const int Tp = ntx * sp;
  const int c = blockIdx.x, b = blockIdx.y;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const unsigned long long base = ibase[b];
  for (int i = threadIdx.x; i < kBinWarps * Tp; i += blockDim.x) cur[i] = 0;
  __syncthreads();
  const int per_warp = kBinChunk / kBinWarps;
  const int g0 = c * kBinChunk + warp * per_warp;
  const int g1 = min(N, g0 + per_warp);
  uint32_t* mycur = cur + warp * Tp;
  int* slot = reinterpret_cast<int*>(cur + kBinWarps * Tp) + warp * 32;
  const int2* bx = boxes + (size_t)b * N;
  // floor(2^20 / w) + 1 for box widths w = 1..64: (k * m) >> 20 = k / w exactly for k < 4096
  unsigned* divmul = reinterpret_cast<unsigned*>(slot + (kBinWarps - warp) * 32);
  if (threadIdx.x >= 1 && threadIdx.x <= 64) divmul[threadIdx.x] = (1u << 20) / (unsigned)threadIdx.x + 1u;
  // 1. per-warp tile histogram (the lane's boxes loaded up front)
  constexpr int kRounds = kBinChunk / kBinWarps / 32;
  int2 bxs[kRounds];
#pragma unroll
  for (int j = 0; j < kRounds; ++j) {
    const int g = g0 + lane + 32 * j;
    bxs[j] = g < g1 ? __ldg(bx + g) : make_int2(1, 0);  // empty
  }
#pragma unroll
  for (int j = 0; j < kRounds; ++j) {
    TileRect r;
    if (!unpack_rect(bxs[j], sh, r)) continue;
    for (int ty = r.ty0; ty <= r.ty1; ++ty)
      for (int tx = r.tx0; tx <= r.tx1; ++tx) atomicAdd(&mycur[ty * sp + tx], 1u);
  }
  __syncthreads();
  // 2. exclusive scan over warps, offset by this chunk's start within the image (the tile's
  // start plus the chunk's offset inside the tile)
  const uint32_t* Hc = hist + ((size_t)b * C + c) * Tn;
  for (int t = threadIdx.x; t < Tn; t += blockDim.x) {
    uint32_t run = Hc[t] + tstart[(size_t)b * Tn + t];
    const int ty = t / ntx, tp = ty * sp + (t - ty * ntx);
    for (int w = 0; w < kBinWarps; ++w) {
      uint32_t v = cur[w * Tp + tp];
      cur[w * Tp + tp] = run;
      run += v;
    }
  }
  __syncthreads();
  // 3. stable scatter of the instances of 32 Gaussians per round, 32 instances per window
  const bool wide = ntx > 32;
  int2 nxt = g0 + lane < g1 ? __ldg(bx + g0 + lane) : make_int2(1, 0);
  for (int gr = g0; gr < g1; gr += 32) {
    const int g = gr + lane;
    TileRect r;
    const int2 cb = nxt;
    nxt = g + 32 < g1 ? __ldg(bx + g + 32) : make_int2(1, 0);  // next round's box, in flight meanwhile
    const bool valid = unpack_rect(cb, sh, r);
    if (!valid) { r.tx0 = 1; r.tx1 = 0; r.ty0 = 1; r.ty1 = 0; }
    // colmask[x] (in lane x) = lanes whose tile-column range holds x; rowmask likewise
    const unsigned colm0 = transpose32(range_bits(r.tx0, r.tx1, 0));
    const unsigned rowm0 = transpose32(range_bits(r.ty0, r.ty1, 0));
    unsigned colm1 = 0, rowm1 = 0;
    if (wide) {
      colm1 = transpose32(range_bits(r.tx0, r.tx1, 32));
      rowm1 = transpose32(range_bits(r.ty0, r.ty1, 32));
    }
    const int wdt = valid ? r.tx1 - r.tx0 + 1 : 1;
    const int cnt = valid ? wdt * (r.ty1 - r.ty0 + 1) : 0;  // <= 64 x 64
    int incl = cnt;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int u = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += u;
    }
    const int pre = incl - cnt;  // first instance of this lane (lane-major order)
    const int total = __shfl_sync(0xffffffffu, incl, 31);
    // what a window lane needs from the instance's owner: its first instance and box origin,
    // and the box width with the multiplier of k / width
    const unsigned own0 = (unsigned)pre | ((unsigned)(valid ? r.tx0 : 0) << 18) | ((unsigned)(valid ? r.ty0 : 0) << 25);
    const unsigned own1 = (unsigned)wdt | (divmul[wdt] << 7);
    for (int w0 = 0; w0 < total; w0 += 32) {
      // lanes with instances in [w0, w0 + 32) mark where in the window their instances start
      const bool meets = cnt > 0 && pre < w0 + 32 && pre + cnt > w0;
      const int sb = max(pre - w0, 0);
      if (meets) slot[sb] = lane;
      const unsigned starts = __reduce_or_sync(0xffffffffu, meets ? (1u << sb) : 0u);
      __syncwarp();
      // the owner of window position `lane` is the lane whose start is the last one at or
      // before it (bit 0 is always set: the window's first instance has an owner)
      const int q = 31 - __clz(starts & (0xffffffffu >> (31 - lane)));
      const int owner = slot[q];
      __syncwarp();
      const unsigned o0 = __shfl_sync(0xffffffffu, own0, owner);
      const unsigned o1 = __shfl_sync(0xffffffffu, own1, owner);
      const int i = w0 + lane;
      const bool act = i < total;
      const unsigned k = act ? (unsigned)(i - (int)(o0 & 0x3ffffu)) : 0u;
      const unsigned ky = (k * (o1 >> 7)) >> 20;
      const int tx = (int)((o0 >> 18) & 0x7fu) + (int)(k - ky * (o1 & 0x7fu));
      const int ty = (int)((o0 >> 25) & 0x7fu) + (int)ky;
      unsigned cm = __shfl_sync(0xffffffffu, colm0, tx & 31);
      unsigned rm = __shfl_sync(0xffffffffu, rowm0, ty & 31);
      if (wide) {
        const unsigned c1 = __shfl_sync(0xffffffffu, colm1, tx & 31);
        const unsigned r1 = __shfl_sync(0xffffffffu, rowm1, ty & 31);
        if (tx >= 32) cm = c1;
        if (ty >= 32) rm = r1;
      }
      const unsigned both = cm & rm;  // lanes of this round whose box covers (tx, ty)
      const int t = ty * sp + tx;
      if (act) {
        const unsigned long long pos = base + mycur[t] + __popc(both & ((1u << owner) - 1u));
        if (pos < cap) pair_gauss[pos] = (uint32_t)(gr + owner);
      }
      __syncwarp();
      // the highest covering lane's instance comes after every other instance of this tile
      // in the round (lane-major order), so the cursor moves once all of them have read it
      if (act && (both >> owner) == 1u) mycur[t] += __popc(both);
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
  const int ntx = L.ntx, Tn = L.Tn, C = L.C;
  const int sh = cfg.tile == 8 ? 3 : cfg.tile == 16 ? 4 : 5;
  const int2* boxes = reinterpret_cast<const int2*>(proj + (size_t)B * N);  // the box plane
  dim3 g2(C, B);
  size_t sm_count = sizeof(uint32_t) * Tn;
  cudaError_t e;
  {
    static int cache[64] = {0};
    e = ensure_smem((const void*)k_bin_count, sm_count, cache);
    if (e != cudaSuccess) return e;
  }
  k_bin_count<<<g2, 256, sm_count, s>>>(boxes, N, sh, ntx, Tn, C, hist);
  {
    static int cache[64] = {0};
    e = ensure_smem((const void*)k_bin_tiles, sm_count, cache);
    if (e != cudaSuccess) return e;
  }
  k_bin_scan<<<dim3((Tn + 255) / 256, B), 256, 0, s>>>(hist, Tn, C, ttotal);
  k_bin_tiles<<<B, 1024, sm_count, s>>>(ttotal, Tn, tstart, itotal);
  k_bin_base<<<1, 32, 0, s>>>(itotal, B, ibase, n_pairs, (unsigned long long)cap, status);
  const int sp = ntx + ((35 - ntx) & 31);  // cursor row stride, 3 (mod 32)
  size_t sm_scatter = sizeof(uint32_t) * (kBinWarps * (ntx * sp + 32) + 65);
  {
    static int cache[64] = {0};
    e = ensure_smem((const void*)k_bin_scatter, sm_scatter, cache);
    if (e != cudaSuccess) return e;
  }
  k_bin_scatter<<<g2, 32 * kBinWarps, sm_scatter, s>>>(boxes, N, sh, ntx, Tn, sp, C, hist, tstart, ttotal, ibase,
                                                      pair_gauss, (unsigned long long)cap, ranges);
  return cudaGetLastError();
}

}  // namespace gs
