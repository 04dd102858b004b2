// SumSplats (Algorithm 2; App. A.2 Eq. 15) and its backward (App. A.2 Eqs. 16-21).
//
// Work decomposition.  A CTA covers a region of one particle's tile (the whole tile for
// tiles of 8 or 16 pixels, a 16 x 16 quadrant of a 32-pixel tile) and stages the tile's
// Gaussian records through shared memory in chunks.  Each warp owns one 4 x 4 pixel block
// of the region.  For every chunk a warp compacts, with ballots, the records whose support
// box touches its block into a per-warp list (the forward tests a block mask formed once per
// record while staging); the lanes then take different list entries ("items" = one Gaussian
// on one block) and each lane evaluates its Gaussian on the block's 16 pixels.  The work executed is therefore that of 4 x 4 blocks (1.76x the algorithmic
// Gaussian-pixel count on the bench workload, against 3.1x for 8 x 8 warp regions).
//
// Per item a lane forms the row start values of the exponent E(u, v) = ca (dx0+u)^2 +
// cb (dx0+u)(dy0+v) + cc (dy0+v)^2 and runs the multiplicative recurrence described at
// for_block_values (two rows per f32x2 instruction), masking the pixels outside the support
// box (box columns as predicates, box rows as zero start values).
//
// Forward: each lane accumulates its items' contributions to the 16 pixels in registers; at
// the end the 32 partial sums of each pixel are added by a transposing butterfly (16
// shuffles for 16 pixels), in a fixed order.  Entry i of a block's list always goes to lane
// i mod 32, so Q does not depend on the tile size or chunk depth.
//
// Backward: per item the lane forms the six moment sums of Gc = dL/dQ(p) * contribution(p)
// about the Gaussian centre (S0, Sx, Sy, Sxx, Sxy, Syy, weights 1, dx, dy, dx^2, dx dy, dy^2
// in pixel units) and stores them in a per-warp slot.  After the chunk one thread per
// record adds its slots over the warps, converts them to world-space gradients of mu and
// Sigma for this particle's pose (grad_mu_tilde = h P (Sx, -Sy), grad_Sigma_tilde =
// (h^2 P M P - S0 P) / 2 with P = Sigma_tilde^-1 taken from the record's exponent and
// M = [[Sxx, -Sxy], [-Sxy, Syy]]; grad_mu = W^T [grad_mu_tilde; 0],
// grad_Sigma = W_{2x3}^T grad_Sigma_tilde W_{2x3}) and adds them, with S0, into a
// per-Gaussian accumulator of 12 floats (three vector atomics; 4.8 MB at N = 100k, resident
// in L2).  A per-Gaussian finalize kernel applies dL/dA = sum S0 / A, the chain through
// Sigma = (R S)(R S)^T to s and q, and the softplus derivatives.
#include "gs_internal.cuh"

namespace gs {
namespace {

constexpr int kBlk = 4;  // pixel block side owned by one warp

struct Rec {
  float cx, cy, ca, cb, cc, w;
  int x0, x1, y0, y1;
};

__device__ __forceinline__ void unpack_box(const gs_record* r, int& x0, int& x1, int& y0, int& y1) {
  const int2 bx = *reinterpret_cast<const int2*>(reinterpret_cast<const char*>(r) + 24);
  x0 = (int)(int16_t)(bx.x & 0xffff);
  x1 = bx.x >> 16;
  y0 = (int)(int16_t)(bx.y & 0xffff);
  y1 = bx.y >> 16;
}

__device__ __forceinline__ Rec load_rec(const gs_record* r) {
  const float4 a = reinterpret_cast<const float4*>(r)[0];
  const float4 b = reinterpret_cast<const float4*>(r)[1];
  Rec o;
  o.cx = a.x; o.cy = a.y; o.ca = a.z; o.cb = a.w; o.cc = b.x; o.w = b.y;
  const int bx = __float_as_int(b.z), by = __float_as_int(b.w);
  o.x0 = (int)(int16_t)(bx & 0xffff);
  o.x1 = bx >> 16;
  o.y0 = (int)(int16_t)(by & 0xffff);
  o.y1 = by >> 16;
  return o;
}

// Geometry of a CTA: region origin and this warp's 4 x 4 block.
struct Geo {
  int X, Y;        // block origin (pixels)
  int regions;     // CTAs per tile (4 for 32-pixel tiles, else 1)
};

__device__ __forceinline__ Geo geometry(int T, int ntx, int tile, int sub) {
  const int side = T == 32 ? 16 : T;       // region side
  const int bpr = side / kBlk;             // blocks per region row
  const int warp = threadIdx.x >> 5;
  Geo g;
  g.regions = T == 32 ? 4 : 1;
  const int RX = (tile % ntx) * T + (sub & 1) * 16;
  const int RY = (tile / ntx) * T + (sub >> 1) * 16;
  g.X = RX + (warp % bpr) * kBlk;
  g.Y = RY + (warp / bpr) * kBlk;
  return g;
}

__device__ __forceinline__ void stage_chunk(gs_record* rec, const gs_record* __restrict__ proj, size_t pbase,
                                            const uint32_t* __restrict__ pair_gauss, uint32_t start, int n) {
  for (int k = threadIdx.x; k < n; k += blockDim.x) {
    const uint32_t g = pair_gauss[start + k];
    const float4* src = reinterpret_cast<const float4*>(proj + pbase + g);
    float4* dst = reinterpret_cast<float4*>(rec + k);
    dst[0] = __ldg(src);
    dst[1] = __ldg(src + 1);
  }
}

// Ballot compaction of the chunk's records whose box touches the block [X, X+3] x [Y, Y+3].
// Writes the record indices to list[0..cnt) in index order; with inv != nullptr also the
// inverse map inv[k] = position in list or 0xffff.  Returns cnt (warp-uniform).
__device__ __forceinline__ int compact(const gs_record* rec, int n, int X, int Y, uint16_t* list, uint16_t* inv) {
  const int lane = threadIdx.x & 31;
  const unsigned lt = lanemask_lt();
  int cnt = 0;
  for (int base = 0; base < n; base += 32) {
    const int k = base + lane;
    bool hit = false;
    if (k < n) {
      int x0, x1, y0, y1;
      unpack_box(rec + k, x0, x1, y0, y1);
      hit = x1 >= X && x0 <= X + kBlk - 1 && y1 >= Y && y0 <= Y + kBlk - 1;
    }
    const unsigned m = __ballot_sync(0xffffffffu, hit);
    const int pos = cnt + __popc(m & lt);
    if (hit) list[pos] = (uint16_t)k;
    if (inv && k < n) inv[k] = hit ? (uint16_t)pos : (uint16_t)0xffff;
    cnt += __popc(m);
  }
  __syncwarp();
  return cnt;
}

// Column predicates and row weights of an item on the block at (X, Y).
struct Mask {
  bool col[kBlk];
  float roww[kBlk];
};

__device__ __forceinline__ Mask make_mask(const Rec& r, int X, int Y, float w) {
  Mask m;
  const int a = r.x0 - X, b = r.x1 - X, c = r.y0 - Y, d = r.y1 - Y;
#pragma unroll
  for (int u = 0; u < kBlk; ++u) m.col[u] = u >= a && u <= b;
#pragma unroll
  for (int v = 0; v < kBlk; ++v) m.roww[v] = (v >= c && v <= d) ? w : 0.f;
  return m;
}

// Region of a CTA: origin, side (8 or 16 pixels) and blocks per side.
struct Region {
  int RX, RY, S, bs;
};

__device__ __forceinline__ Region region_of(int T, int ntx, int tile, int sub) {
  Region r;
  r.S = T == 32 ? 16 : T;
  r.bs = r.S / kBlk;
  r.RX = (tile % ntx) * T + (sub & 1) * 16;
  r.RY = (tile / ntx) * T + (sub >> 1) * 16;
  return r;
}

// Bit j = by * bs + bx set iff the box touches block (bx, by) of the region.
__device__ __forceinline__ unsigned block_mask(int x0, int x1, int y0, int y1, const Region& g) {
  const int lx = max(x0 - g.RX, 0), hx = min(x1 - g.RX, g.S - 1);
  const int ly = max(y0 - g.RY, 0), hy = min(y1 - g.RY, g.S - 1);
  if (lx > hx || ly > hy) return 0u;
  const int bx0 = lx >> 2, bx1 = hx >> 2, by0 = ly >> 2, by1 = hy >> 2;
  const unsigned cols = ((2u << bx1) - 1u) & ~((1u << bx0) - 1u);
  unsigned m = 0u;
  for (int by = by0; by <= by1; ++by) m |= cols << (by * g.bs);
  return m;
}

// Stage records [start, start + n) of the tile list and their block masks.
__device__ __forceinline__ void stage_chunk_masked(gs_record* rec, uint16_t* msk, const gs_record* __restrict__ proj,
                                                   size_t pbase, const uint32_t* __restrict__ pair_gauss,
                                                   uint32_t start, int n, const Region& reg) {
  for (int k = threadIdx.x; k < n; k += blockDim.x) {
    const uint32_t g = pair_gauss[start + k];
    const float4* src = reinterpret_cast<const float4*>(proj + pbase + g);
    float4* dst = reinterpret_cast<float4*>(rec + k);
    const float4 a = __ldg(src), b = __ldg(src + 1);
    dst[0] = a;
    dst[1] = b;
    const int bx = __float_as_int(b.z), by = __float_as_int(b.w);
    msk[k] = (uint16_t)block_mask((int)(int16_t)(bx & 0xffff), bx >> 16, (int)(int16_t)(by & 0xffff), by >> 16, reg);
  }
}

// Ballot compaction of the chunk's records whose mask has bit `blk`: writes their indices
// to list[0..cnt) in index order and returns cnt (warp-uniform).
__device__ __forceinline__ int compact_mask(const uint16_t* msk, int n, int blk, uint16_t* list) {
  const int lane = threadIdx.x & 31;
  const unsigned lt = lanemask_lt();
  int cnt = 0;
  for (int base = 0; base < n; base += 32) {
    const int k = base + lane;
    const bool hit = k < n && ((msk[k] >> blk) & 1u);
    const unsigned m = __ballot_sync(0xffffffffu, hit);
    if (hit) list[cnt + __popc(m & lt)] = (uint16_t)k;
    cnt += __popc(m);
  }
  __syncwarp();
  return cnt;
}

// ---------------------------------------------------------------------------------------
// Item evaluation.  Rows v = 0..3 of the block are handled in packed pairs (0,1) and (2,3)
// with the f32x2 instructions of sm_100+ (two lanes of work per instruction).
//
// Along a row the exponent is quadratic in u, so the value follows the recurrence
//   V(u+1) = V(u) R(u),  R(u+1) = R(u) 2^(2 ca),   V(0) = 2^E(0,v), R(0) = 2^D(0,v),
// with E(0,v) the exponent at the block's first column and D(0,v) = E(1,v) - E(0,v): nine
// ex2 per item instead of sixteen, and two multiplies per packed pixel pair.  The recurrence
// is used when V(0) cannot underflow and R(0) cannot overflow (E(0,v) > -100, D(0,v) < 100,
// which holds for every Gaussian wider than ~0.35 px); otherwise the item takes the exact
// path (one ex2 per pixel of the exponent formed by forward differences).  Rows outside the
// support box start at V(0) = 0 (and stay 0); columns outside it are skipped by predicates.
// ---------------------------------------------------------------------------------------
typedef unsigned long long u64;

__device__ __forceinline__ u64 pk(float a, float b) {
  u64 r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b));
  return r;
}
__device__ __forceinline__ void upk(u64 r, float& a, float& b) {
  asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(r));
}
__device__ __forceinline__ u64 mul2(u64 a, u64 b) {
  u64 r;
  asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
  return r;
}
__device__ __forceinline__ u64 add2(u64 a, u64 b) {
  u64 r;
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
  return r;
}
__device__ __forceinline__ u64 fma2(u64 a, u64 b, u64 c) {
  u64 r;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r) : "l"(a), "l"(b), "l"(c));
  return r;
}

// Start exponents E(0,v) and first differences D(0,v) of the 4 rows of a block whose
// corner is (dx0, dy0) pixels from the Gaussian centre.
struct RowStart {
  float E[kBlk], D[kBlk];
};

__device__ __forceinline__ RowStart row_start(const Rec& r, float dx0, float dy0) {
  RowStart s;
  float G = fmaf(r.cb, dx0, r.cc * (2.f * dy0 + 1.f));
  s.E[0] = fmaf(dx0, fmaf(r.ca, dx0, r.cb * dy0), r.cc * dy0 * dy0);
  s.D[0] = fmaf(r.ca, 2.f * dx0 + 1.f, r.cb * dy0);
#pragma unroll
  for (int v = 1; v < kBlk; ++v) {
    s.E[v] = s.E[v - 1] + G;
    G = fmaf(2.f, r.cc, G);
    s.D[v] = s.D[v - 1] + r.cb;
  }
  return s;
}

__device__ __forceinline__ bool recurrence_safe(const RowStart& s) {
  const float emin = fminf(fminf(s.E[0], s.E[1]), fminf(s.E[2], s.E[3]));
  const float dmax = fmaxf(fmaxf(s.D[0], s.D[1]), fmaxf(s.D[2], s.D[3]));
  return emin > -100.f && dmax < 100.f;
}

// Values of the 4 rows (as two packed pairs) at every column u of the block, handed to
// body(u, v01, v23).  rowscale[v] multiplies row v (0 for rows outside the box).
template <class Body>
__device__ __forceinline__ void for_block_values(const Rec& r, const RowStart& s, const float rowscale[kBlk],
                                                 Body body) {
  if (recurrence_safe(s)) {
    u64 V01 = pk(rowscale[0] * ex2_approx(s.E[0]), rowscale[1] * ex2_approx(s.E[1]));
    u64 V23 = pk(rowscale[2] * ex2_approx(s.E[2]), rowscale[3] * ex2_approx(s.E[3]));
    u64 R01 = pk(ex2_approx(s.D[0]), ex2_approx(s.D[1]));
    u64 R23 = pk(ex2_approx(s.D[2]), ex2_approx(s.D[3]));
    const float st = ex2_approx(2.f * r.ca);
    const u64 S = pk(st, st);
#pragma unroll
    for (int u = 0; u < kBlk; ++u) {
      body(u, V01, V23);
      if (u + 1 < kBlk) {
        V01 = mul2(V01, R01);
        V23 = mul2(V23, R23);
        if (u + 2 < kBlk) {
          R01 = mul2(R01, S);
          R23 = mul2(R23, S);
        }
      }
    }
  } else {
    float e[kBlk], d[kBlk];
#pragma unroll
    for (int v = 0; v < kBlk; ++v) { e[v] = s.E[v]; d[v] = s.D[v]; }
    const float two_a = 2.f * r.ca;
#pragma unroll
    for (int u = 0; u < kBlk; ++u) {
      const u64 V01 = pk(rowscale[0] * ex2_approx(e[0]), rowscale[1] * ex2_approx(e[1]));
      const u64 V23 = pk(rowscale[2] * ex2_approx(e[2]), rowscale[3] * ex2_approx(e[3]));
      body(u, V01, V23);
#pragma unroll
      for (int v = 0; v < kBlk; ++v) { e[v] += d[v]; d[v] += two_a; }
    }
  }
}

__global__ void k_render_fwd(const gs_record* __restrict__ proj, int N, const uint32_t* __restrict__ pair_gauss,
                             const uint32_t* __restrict__ ranges, int D, int T, int ntx, int chunk,
                             float* __restrict__ Q) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  gs_record* rec = reinterpret_cast<gs_record*>(smem_raw);
  uint16_t* msk = reinterpret_cast<uint16_t*>(smem_raw + sizeof(gs_record) * chunk);
  uint16_t* list = msk + chunk + warp * chunk;
  const int regions = T == 32 ? 4 : 1;
  const int tile = blockIdx.x / regions, sub = blockIdx.x % regions, b = blockIdx.y, Tn = ntx * ntx;
  const Geo geo = geometry(T, ntx, tile, sub);
  const Region reg = region_of(T, ntx, tile, sub);
  const uint32_t start = ranges[((size_t)b * Tn + tile) * 2], end = ranges[((size_t)b * Tn + tile) * 2 + 1];
  const size_t pbase = (size_t)b * N;
  const float fX = (float)geo.X, fY = (float)geo.Y;
  u64 acc01[kBlk], acc23[kBlk];  // (row 0, row 1) and (row 2, row 3) of column u
#pragma unroll
  for (int u = 0; u < kBlk; ++u) acc01[u] = acc23[u] = pk(0.f, 0.f);
  int running = 0;
  for (uint32_t base = start; base < end; base += chunk) {
    const int n = (int)min((uint32_t)chunk, end - base);
    __syncthreads();
    stage_chunk_masked(rec, msk, proj, pbase, pair_gauss, base, n, reg);
    __syncthreads();
    const int cnt = compact_mask(msk, n, warp, list);
    for (int i = (lane - running) & 31; i < cnt; i += 32) {
      const Rec r = load_rec(rec + list[i]);
      const Mask mk = make_mask(r, geo.X, geo.Y, r.w);
      const RowStart rs = row_start(r, fX - r.cx, fY - r.cy);
      for_block_values(r, rs, mk.roww, [&](int u, u64 v01, u64 v23) {
        if (mk.col[u]) {
          acc01[u] = add2(acc01[u], v01);
          acc23[u] = add2(acc23[u], v23);
        }
      });
    }
    running = (running + cnt) & 31;
  }
  float sv[16];
#pragma unroll
  for (int u = 0; u < kBlk; ++u) {
    upk(acc01[u], sv[0 * kBlk + u], sv[1 * kBlk + u]);
    upk(acc23[u], sv[2 * kBlk + u], sv[3 * kBlk + u]);
  }
  // transposing butterfly: 16 values over 32 lanes
#pragma unroll
  for (int half = 8, off = 16; half >= 1; half >>= 1, off >>= 1) {
    const bool up = lane & off;
#pragma unroll
    for (int k = 0; k < half; ++k) {
      const float send = up ? sv[k] : sv[k + half];
      const float keep = up ? sv[k + half] : sv[k];
      sv[k] = keep + __shfl_xor_sync(0xffffffffu, send, off);
    }
  }
  sv[0] += __shfl_xor_sync(0xffffffffu, sv[0], 1);
  // lane holds pixel p = (bit4 << 3) | (bit3 << 2) | (bit2 << 1) | bit1 of its lane index
  if ((lane & 1) == 0) {
    const int p = ((lane >> 4) & 1) * 8 + ((lane >> 3) & 1) * 4 + ((lane >> 2) & 1) * 2 + ((lane >> 1) & 1);
    const int i = geo.Y + p / kBlk, j = geo.X + p % kBlk;
    if (i < D && j < D) Q[((size_t)b * D + i) * D + j] = sv[0];
  }
}

__global__ void k_render_bwd(const gs_record* __restrict__ proj, int N, const uint32_t* __restrict__ pair_gauss,
                             const uint32_t* __restrict__ ranges, int D, int T, int ntx, int chunk,
                             const float* __restrict__ dLdQ, const float* __restrict__ Wall, float h,
                             float* __restrict__ wacc) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int nwarps = blockDim.x >> 5, warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  gs_record* rec = reinterpret_cast<gs_record*>(smem_raw);
  float* res = reinterpret_cast<float*>(smem_raw + sizeof(gs_record) * chunk);  // [nwarps][chunk][6]
  uint16_t* lists = reinterpret_cast<uint16_t*>(res + (size_t)nwarps * chunk * 6);
  uint16_t* list = lists + warp * chunk;
  uint16_t* invs = lists + (size_t)nwarps * chunk;  // [nwarps][chunk]
  __shared__ float Ws[9];
  const int regions = T == 32 ? 4 : 1;
  const int tile = blockIdx.x / regions, sub = blockIdx.x % regions, b = blockIdx.y, Tn = ntx * ntx;
  if (threadIdx.x < 9) Ws[threadIdx.x] = Wall[(size_t)b * 9 + threadIdx.x];
  const Geo geo = geometry(T, ntx, tile, sub);
  const uint32_t start = ranges[((size_t)b * Tn + tile) * 2], end = ranges[((size_t)b * Tn + tile) * 2 + 1];
  const size_t pbase = (size_t)b * N;
  const float fX = (float)geo.X, fY = (float)geo.Y;
  float g[kBlk][kBlk];
#pragma unroll
  for (int v = 0; v < kBlk; ++v)
#pragma unroll
    for (int u = 0; u < kBlk; ++u) {
      const int i = geo.Y + v, j = geo.X + u;
      g[v][u] = (i < D && j < D) ? dLdQ[((size_t)b * D + i) * D + j] : 0.f;
    }
  u64 g01[kBlk], g23[kBlk];  // dL/dQ of the block as packed row pairs per column
#pragma unroll
  for (int u = 0; u < kBlk; ++u) {
    g01[u] = pk(g[0][u], g[1][u]);
    g23[u] = pk(g[2][u], g[3][u]);
  }
  const float kap = -2.f / (kLog2e * h * h);  // P = kap * [[ca, -cb/2], [-cb/2, cc]]
  const float h2 = h * h;
  float* myres = res + (size_t)warp * chunk * 6;
  for (uint32_t base = start; base < end; base += chunk) {
    const int n = (int)min((uint32_t)chunk, end - base);
    __syncthreads();
    stage_chunk(rec, proj, pbase, pair_gauss, base, n);
    __syncthreads();
    const int cnt = compact(rec, n, geo.X, geo.Y, list, invs + warp * chunk);
    for (int i = lane; i < cnt; i += 32) {
      const Rec r = load_rec(rec + list[i]);
      const Mask mk = make_mask(r, geo.X, geo.Y, 1.f);
      const float dx0 = fX - r.cx, dy0 = fY - r.cy;
      // per row pair: sums over u of t, u t, u^2 t with t = dL/dQ * 2^E (masked)
      u64 A01 = pk(0.f, 0.f), B01 = A01, C01 = A01, A23 = A01, B23 = A01, C23 = A01;
      const RowStart rs = row_start(r, dx0, dy0);
      for_block_values(r, rs, mk.roww, [&](int u, u64 v01, u64 v23) {
        if (mk.col[u]) {
          const u64 t01 = mul2(g01[u], v01), t23 = mul2(g23[u], v23);
          A01 = add2(A01, t01);
          A23 = add2(A23, t23);
          if (u > 0) {
            const u64 fu = pk((float)u, (float)u), fu2 = pk((float)(u * u), (float)(u * u));
            B01 = fma2(fu, t01, B01);
            B23 = fma2(fu, t23, B23);
            C01 = fma2(fu2, t01, C01);
            C23 = fma2(fu2, t23, C23);
          }
        }
      });
      float R0[kBlk], R1[kBlk], R2[kBlk];
      upk(A01, R0[0], R0[1]); upk(A23, R0[2], R0[3]);
      upk(B01, R1[0], R1[1]); upk(B23, R1[2], R1[3]);
      upk(C01, R2[0], R2[1]); upk(C23, R2[2], R2[3]);
      // moments about the block origin: M0 = sum t, Mu = sum u t, Mv, Muu, Muv, Mvv
      const float M0 = (R0[0] + R0[1]) + (R0[2] + R0[3]);
      const float Mu = (R1[0] + R1[1]) + (R1[2] + R1[3]);
      const float Muu = (R2[0] + R2[1]) + (R2[2] + R2[3]);
      const float Mv = fmaf(3.f, R0[3], fmaf(2.f, R0[2], R0[1]));
      const float Muv = fmaf(3.f, R1[3], fmaf(2.f, R1[2], R1[1]));
      const float Mvv = fmaf(9.f, R0[3], fmaf(4.f, R0[2], R0[1]));
      // shift to moments about the Gaussian centre (dx = dx0 + u, dy = dy0 + v), times w
      const float w = r.w;
      float* o = myres + (size_t)i * 6;
      o[0] = w * M0;
      o[1] = w * fmaf(dx0, M0, Mu);
      o[2] = w * fmaf(dy0, M0, Mv);
      o[3] = w * fmaf(dx0, fmaf(dx0, M0, 2.f * Mu), Muu);
      o[4] = w * (fmaf(dx0, fmaf(dy0, M0, Mv), dy0 * Mu) + Muv);
      o[5] = w * fmaf(dy0, fmaf(dy0, M0, 2.f * Mv), Mvv);
    }
    __syncthreads();
    // per record: add the warps' slots, convert to world space, one set of atomics
    for (int k = threadIdx.x; k < n; k += blockDim.x) {
      float S[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
      bool any = false;
      for (int wv = 0; wv < nwarps; ++wv) {
        const uint16_t pos = invs[wv * chunk + k];
        if (pos == 0xffff) continue;
        const float* q = res + ((size_t)wv * chunk + pos) * 6;
#pragma unroll
        for (int e = 0; e < 6; ++e) S[e] += q[e];
        any = true;
      }
      if (!any) continue;
      const float4 ra = reinterpret_cast<const float4*>(rec + k)[0];
      const float rc = reinterpret_cast<const float*>(rec + k)[4];
      const float pxx = kap * ra.z, pyy = kap * rc, pxy = -0.5f * kap * ra.w;
      // App. A.2 Eq. 18: grad_mu_tilde = sum Gc P d, d = (h dx, -h dy)
      const float gmx = h * (pxx * S[1] - pxy * S[2]);
      const float gmy = h * (pxy * S[1] - pyy * S[2]);
      // Eq. 20: grad_Sigma_tilde = -P (S0 Sigma_tilde - h^2 M) P / 2 = (h^2 P M P - S0 P) / 2
      const float a00 = pxx * S[3] - pxy * S[4], a01 = -pxx * S[4] + pxy * S[5];
      const float a10 = pxy * S[3] - pyy * S[4], a11 = -pxy * S[4] + pyy * S[5];
      const float b00 = a00 * pxx + a01 * pxy, b01 = a00 * pxy + a01 * pyy, b11 = a10 * pxy + a11 * pyy;
      const float gxx = 0.5f * (h2 * b00 - S[0] * pxx);
      const float gxy = 0.5f * (h2 * b01 - S[0] * pxy);
      const float gyy = 0.5f * (h2 * b11 - S[0] * pyy);
      // mu_dot = W mu, Sigma_dot = W Sigma W^T, Eq. 21 embedding
      float o[12];
#pragma unroll
      for (int c = 0; c < 3; ++c) o[c] = Ws[c] * gmx + Ws[3 + c] * gmy;
      const int kk[6] = {0, 0, 0, 1, 1, 2}, ll[6] = {0, 1, 2, 1, 2, 2};
#pragma unroll
      for (int e = 0; e < 6; ++e) {
        const float ak = Ws[kk[e]], bk = Ws[3 + kk[e]], al = Ws[ll[e]], bl = Ws[3 + ll[e]];
        o[3 + e] = ak * gxx * al + ak * gxy * bl + bk * gxy * al + bk * gyy * bl;
      }
      o[9] = S[0];
      o[10] = 0.f;
      o[11] = 0.f;
      const uint32_t gi = pair_gauss[base + k];
      float* dst = wacc + (size_t)gi * 12;
      red_add_v4(dst, o[0], o[1], o[2], o[3]);
      red_add_v4(dst + 4, o[4], o[5], o[6], o[7]);
      red_add_v2(dst + 8, o[8], o[9]);
    }
  }
}

// Per Gaussian: dL/dA = sum S0 / A and the chain from (grad_mu, grad_Sigma) to theta.
// Re-zeroes the accumulator it consumed.
__global__ void k_bwd_finalize(const float* __restrict__ theta, const float* __restrict__ gauss, int N,
                               float* __restrict__ wacc, float* __restrict__ dtheta) {
  const int g = blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= N) return;
  const float* G = gauss + (size_t)g * kGaussStride;
  if (G[kBad] != 0.f) return;
  float* acc = wacc + (size_t)g * 12;
  const float4 a0 = reinterpret_cast<const float4*>(acc)[0];
  const float4 a1 = reinterpret_cast<const float4*>(acc)[1];
  const float4 a2 = reinterpret_cast<const float4*>(acc)[2];
  reinterpret_cast<float4*>(acc)[0] = make_float4(0.f, 0.f, 0.f, 0.f);
  reinterpret_cast<float4*>(acc)[1] = make_float4(0.f, 0.f, 0.f, 0.f);
  reinterpret_cast<float4*>(acc)[2] = make_float4(0.f, 0.f, 0.f, 0.f);
  float M[9], s[3];
#pragma unroll
  for (int k = 0; k < 9; ++k) M[k] = G[kM + k];
  s[0] = G[kS]; s[1] = G[kS + 1]; s[2] = G[kS + 2];
  const float A = G[kA];
  const float gmu[3] = {a0.x, a0.y, a0.z};
  const float gS[6] = {a0.w, a1.x, a1.y, a1.z, a1.w, a2.x};  // 00 01 02 11 12 22
  const float gA = a2.y / A;  // Eq. 17 summed: sum dL/dQ G_tilde = S0 / A
  // Sigma = M M^T: grad_M = (G + G^T) M = 2 G M (G symmetric)
  const float Gm[9] = {gS[0], gS[1], gS[2], gS[1], gS[3], gS[4], gS[2], gS[4], gS[5]};
  float dM[9];
#pragma unroll
  for (int k = 0; k < 3; ++k)
#pragma unroll
    for (int m = 0; m < 3; ++m)
      dM[3 * k + m] = 2.f * (Gm[3 * k] * M[m] + Gm[3 * k + 1] * M[3 + m] + Gm[3 * k + 2] * M[6 + m]);
  // M = R diag(s): grad_s[m] = sum_k dM[k][m] R[k][m]; grad_R[k][m] = dM[k][m] s[m]
  float ds[3], dR[9];
#pragma unroll
  for (int m = 0; m < 3; ++m) {
    ds[m] = 0.f;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      const float R = M[3 * k + m] / s[m];
      ds[m] += dM[3 * k + m] * R;
      dR[3 * k + m] = dM[3 * k + m] * s[m];
    }
  }
  const float* th = theta + (size_t)g * 11;
  const float qw = th[6], qx = th[7], qy = th[8], qz = th[9];
  const float qn = sqrtf(qw * qw + qx * qx + qy * qy + qz * qz);
  const float w = qw / qn, x = qx / qn, y = qy / qn, zq = qz / qn;
  // dR / dq_hat for R(w, x, y, z) of Sec. 3.3.1
  const float dw = dR[1] * (-2.f * zq) + dR[2] * (2.f * y) + dR[3] * (2.f * zq) + dR[5] * (-2.f * x) +
                   dR[6] * (-2.f * y) + dR[7] * (2.f * x);
  const float dx = dR[1] * (2.f * y) + dR[2] * (2.f * zq) + dR[3] * (2.f * y) + dR[4] * (-4.f * x) +
                   dR[5] * (-2.f * w) + dR[6] * (2.f * zq) + dR[7] * (2.f * w) + dR[8] * (-4.f * x);
  const float dy = dR[0] * (-4.f * y) + dR[1] * (2.f * x) + dR[2] * (2.f * w) + dR[3] * (2.f * x) +
                   dR[5] * (2.f * zq) + dR[6] * (-2.f * w) + dR[7] * (2.f * zq) + dR[8] * (-4.f * y);
  const float dz = dR[0] * (-4.f * zq) + dR[1] * (-2.f * w) + dR[2] * (2.f * x) + dR[3] * (2.f * w) +
                   dR[4] * (-4.f * zq) + dR[5] * (2.f * y) + dR[6] * (2.f * x) + dR[7] * (2.f * y);
  const float dot = w * dw + x * dx + y * dy + zq * dz;
  float* out = dtheta + (size_t)g * 11;
  out[0] += gmu[0];
  out[1] += gmu[1];
  out[2] += gmu[2];
#pragma unroll
  for (int m = 0; m < 3; ++m) out[3 + m] += ds[m] / (1.f + expf(-th[3 + m]));
  out[6] += (dw - w * dot) / qn;
  out[7] += (dx - x * dot) / qn;
  out[8] += (dy - y * dot) / qn;
  out[9] += (dz - zq * dot) / qn;
  out[10] += gA / (1.f + expf(-th[10]));
}

}  // namespace

static int render_warps(int T) {
  const int side = T == 32 ? 16 : T;
  return (side / kBlk) * (side / kBlk);
}

static dim3 render_grid(const gs_config& cfg, int B) {
  const int ntx = (cfg.D + cfg.tile - 1) / cfg.tile;
  return dim3(ntx * ntx * (cfg.tile == 32 ? 4 : 1), B);
}

static size_t render_fwd_smem(const gs_config& cfg) {
  return sizeof(gs_record) * cfg.chunk + sizeof(uint16_t) * (1 + render_warps(cfg.tile)) * cfg.chunk;
}

static size_t render_bwd_smem(int tile, int chunk) {
  const int nw = render_warps(tile);
  return sizeof(gs_record) * chunk + sizeof(float) * 6 * nw * chunk + 2 * sizeof(uint16_t) * nw * chunk;
}

// The backward keeps a result slot per (warp, record) of the chunk; its chunk is the
// configured one, reduced (by multiples of 32) until the slots fit in 200 KB of shared memory.
static int render_bwd_chunk(const gs_config& cfg) {
  int c = cfg.chunk;
  while (c > 32 && render_bwd_smem(cfg.tile, c) > 200 * 1024) c -= 32;
  return c;
}

cudaError_t launch_render_fwd(const gs_config& cfg, const gs_record* proj, int N, const uint32_t* pair_gauss,
                              const uint32_t* ranges, int B, float* Q, cudaStream_t s) {
  if (B <= 0) return cudaSuccess;
  const int ntx = (cfg.D + cfg.tile - 1) / cfg.tile;
  const size_t sm = render_fwd_smem(cfg);
  {
    static int cache[64] = {0};
    cudaError_t e = ensure_smem((const void*)k_render_fwd, sm, cache);
    if (e != cudaSuccess) return e;
  }
  k_render_fwd<<<render_grid(cfg, B), render_warps(cfg.tile) * 32, sm, s>>>(proj, N, pair_gauss, ranges, cfg.D,
                                                                          cfg.tile, ntx, cfg.chunk, Q);
  return cudaGetLastError();
}

cudaError_t launch_render_bwd(const gs_config& cfg, const gs_record* proj, int N, const uint32_t* pair_gauss,
                              const uint32_t* ranges, int B, const float* dLdQ, const float* W, float* wacc,
                              cudaStream_t s) {
  if (B <= 0) return cudaSuccess;
  const int ntx = (cfg.D + cfg.tile - 1) / cfg.tile;
  const int chunk = render_bwd_chunk(cfg);
  const size_t sm = render_bwd_smem(cfg.tile, chunk);
  {
    static int cache[64] = {0};
    cudaError_t e = ensure_smem((const void*)k_render_bwd, sm, cache);
    if (e != cudaSuccess) return e;
  }
  const float h = 2.f * cfg.E / (float)cfg.D;
  k_render_bwd<<<render_grid(cfg, B), render_warps(cfg.tile) * 32, sm, s>>>(proj, N, pair_gauss, ranges, cfg.D,
                                                                          cfg.tile, ntx, chunk, dLdQ, W, h, wacc);
  return cudaGetLastError();
}

cudaError_t launch_bwd_finalize(const float* theta, const float* gauss, int N, float* wacc, float* dtheta,
                                cudaStream_t s) {
  if (N <= 0) return cudaSuccess;
  k_bwd_finalize<<<(N + 255) / 256, 256, 0, s>>>(theta, gauss, N, wacc, dtheta);
  return cudaGetLastError();
}

}  // namespace gs
