// SumSplats (Algorithm 2; App. A.2 Eq. 15) and its backward (App. A.2 Eqs. 16-21).
//
// Work decomposition.  Every 8 x 8 pixel block of a particle image is owned by one warp,
// and the block's list of Gaussians (those whose support box touches it, in Gaussian
// order) is dealt to the lanes: entry j goes to lane j mod 32.  A lane evaluates its
// Gaussian on all 64 pixels of the block (an "item"), so the per-Gaussian set-up is paid
// once per block and the box's row and column ranges are the only per-pixel test.
//   - Tiles of 8 pixels: each warp of a CTA owns one tile of a 2 x 2 quad (Gaussians shared by
//     neighbouring tiles then meet in the same L1); its lanes read their records straight
//     from global memory (the tile's list is the block's list), one record and two pair
//     indices ahead; the forward also prefetches the record two items ahead into L1.
//   - Tiles of 16 or 32 pixels: a CTA of four warps covers a 16 x 16 region (the tile, or
//     a quadrant of a 32-pixel tile), stages the tile's records through shared memory in
//     chunks, and each warp compacts, by ballots, the records whose box touches its block.
// In both cases a block's list and its lane assignment are the same, and the item's
// arithmetic is one function of (record, block), so Q does not depend on the tile size or the
// chunk depth (bitwise).
//
// Exponent.  With dx = j - cx, dy = i - cy the pixel's offsets from the splat centre (pixel
// units), the record stores the completed square of App. A.2 Eq. 12's quadratic form along
// the row:  2^E = w exp(-1/2 d^T Sigma~^-1 d)  with  E = lw - a (dx + r dy)^2 - q dy^2,
// a = log2(e)/2 Syy/det, r = Sxy/Syy, q = log2(e)/2 / Syy (Sigma~ in pixel units, lw = log2 w).
// Every term is a square, so nothing cancels for thin splats (the expanded form
// ca dx^2 + cb dx dy + cc dy^2 loses a factor of the covariance's condition number).  The row
// constants lw - q dy^2 and t = dx + r dy at the block's first column are formed directly for
// every row, two rows per packed f32x2 instruction.  Along a row:
//   - Fast path (a <= kAThr, a conditional standard deviation of at least 0.49 px): E is
//     advanced by forward differences, E += D, D += -2a.  Its rounding error grows with a
//     times the squared distance travelled, which is small at this curvature.
//   - Exact path (a > kAThr): t is advanced by exact unit steps and E = fma(-a t, t, lw - q dy^2)
//     is formed at every pixel, with the centre read as a float-float (record centre + the
//     low parts of the projection buffer).
// Every pixel takes one ex2.  Rows outside the box start at E = -inf; a column's contributions
// are added with a 0/1 factor (1 inside the box), which costs a few integer operations per
// column instead of a predicate per packed accumulation.
//
// Forward: each lane accumulates its items' contributions to the block's 64 pixels in
// registers; a transposing butterfly over the 32 lanes (62 shuffles, fixed order) leaves two
// pixel sums per lane, which it stores.
//
// Backward: per item the lane forms, from T = dL/dQ(p) * contribution(p), the moment sums of
// each row in the column offset uc = u - 3.5, then moments in t = dx + r dy and dy:
// M0 = sum T, Mt = sum T t, Md = sum T dy, Mtt = sum T t^2, Mtd = sum T t dy, Mdd = sum T dy^2.
// Working in (t, dy) keeps a thin splat's narrow direction apart from its long one.  It turns
// them into the gradient of this particle's (mu~, Sigma~) by the chain through (a, r, q, lw,
// cx, cy), maps that to world space with the pose (App. A.2 Eqs. 18, 21 with
// grad_mu = W^T [grad_mu~; 0]) and adds it, with M0, into a per-Gaussian accumulator of 12
// floats (three vector reductions).  A per-Gaussian finalize kernel applies
// dL/dA = sum M0 / A, the chain through Sigma = (R S)(R S)^T to s and q, and the softplus
// derivatives.
#include "gs_internal.cuh"

namespace gs {
namespace {

constexpr int kB = 8;            // side of the pixel block owned by one warp
constexpr int kRegionWarps = 4;  // warps of a CTA covering a 16 x 16 region
constexpr int kTileWarps = 4;    // tiles of 8 pixels per CTA (one warp each)
constexpr int kFwd8MinBlocks = 4;  // caps k_render_fwd8 at 128 registers: 16 warps per SM
constexpr int kBwd8MinBlocks = 5;  // caps k_render_bwd8 at 96 registers: 20 warps per SM
constexpr float kHalfLog2e = 0.72134752044448170f;
constexpr float kLn2 = 0.69314718055994531f;

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
__device__ __forceinline__ u64 ex2x2(u64 e) {
  float e0, e1;
  upk(e, e0, e1);
  return pk(ex2_approx(e0), ex2_approx(e1));
}

// Tile of warp w in CTA q: CTAs tile the image in 2 x 2 quads of tiles, (-1 past the image).
__device__ __forceinline__ int quad_tile(int q, int w, int ntx) {
  const int nqx = (ntx + 1) >> 1;
  const int tx = 2 * (q % nqx) + (w & 1), ty = 2 * (q / nqx) + (w >> 1);
  return (tx < ntx && ty < ntx) ? ty * ntx + tx : -1;
}

// An ill-conditioned record: the completed square (a > 0, r, -q) and log2 w.
struct Rec {
  float cx, cy, na, r, nq, lw;  // centre; -a, r, -q, log2 w of the completed square
  int x0, x1, y0, y1;
};

__device__ __forceinline__ Rec rec_from(const float4 a, const float4 b) {
  Rec o;
  o.cx = a.x; o.cy = a.y; o.na = -a.z; o.r = a.w; o.nq = b.x; o.lw = b.y;
  const int bx = __float_as_int(b.z), by = __float_as_int(b.w);
  o.x0 = (int)(int16_t)(bx & 0xffff);
  o.x1 = bx >> 16;
  o.y0 = (int)(int16_t)(by & 0xffff);
  o.y1 = by >> 16;
  return o;
}

// The record's form: the third float is ca < 0 in a well-conditioned record, a > 0 in an
// ill-conditioned one.
__device__ __forceinline__ bool exact_record(const float4 a) { return a.z > 0.f; }

// A well-conditioned record: the expanded quadratic form (ca < 0) and the linear weight w.
struct FastRec {
  float cx, cy, ca, cb, cc, w;
  int x0, x1, y0, y1;
};

__device__ __forceinline__ FastRec fast_rec(const float4 a, const float4 b) {
  FastRec o;
  o.cx = a.x; o.cy = a.y; o.ca = a.z; o.cb = a.w; o.cc = b.x; o.w = b.y;
  const int bx = __float_as_int(b.z), by = __float_as_int(b.w);
  o.x0 = (int)(int16_t)(bx & 0xffff);
  o.x1 = bx >> 16;
  o.y0 = (int)(int16_t)(by & 0xffff);
  o.y1 = by >> 16;
  return o;
}

__device__ __forceinline__ float lg2_approx(float x) {
  float y;
  asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}


__device__ __forceinline__ unsigned range_bits(int lo, int hi) {
  return lo > hi ? 0u : (((2u << hi) - 1u) & ~((1u << lo) - 1u));
}

// 1.0f if bit u of cm is set, else 0.0f, in both halves: the column's mask as a factor.
__device__ __forceinline__ u64 col_factor(unsigned cm, int u) {
  const float m = __uint_as_float((0u - ((cm >> u) & 1u)) & 0x3f800000u);
  return pk(m, m);
}

// ---------------------------------------------------------------------------------------
// Fast path: one well-conditioned Gaussian on one 8 x 8 block with origin (X, Y), the
// expanded form advanced by forward differences in both directions.
// ---------------------------------------------------------------------------------------
struct FastItem {
  u64 E[4];     // exponent (+ log2 w) at the current column, rows (0,1) (2,3) (4,5) (6,7)
  u64 Dd[4];    // its first difference along the row
  u64 S2;       // second difference 2 ca, both halves
  unsigned cm;  // bit u set iff column u is inside the support box
};

__device__ __forceinline__ FastItem make_fast_item(const FastRec& r, int X, int Y) {
  FastItem it;
  const float dx0 = (float)X - r.cx, dy0 = (float)Y - r.cy;
  float E = fmaf(dx0, fmaf(r.ca, dx0, r.cb * dy0), r.cc * dy0 * dy0) + lg2_approx(r.w);
  float Dv = fmaf(r.ca, 2.f * dx0 + 1.f, r.cb * dy0);
  float G = fmaf(r.cb, dx0, r.cc * (2.f * dy0 + 1.f));  // E(0, v + 1) - E(0, v)
  const float two_cc = 2.f * r.cc;
  const unsigned rspan = (unsigned)(r.y1 - r.y0);
  const int r0 = r.y0 - Y;
  float Ev[kB], Dvv[kB];
#pragma unroll
  for (int v = 0; v < kB; ++v) {
    Ev[v] = ((unsigned)(v - r0) <= rspan) ? E : -INFINITY;
    Dvv[v] = Dv;
    E += G;
    G += two_cc;
    Dv += r.cb;
  }
#pragma unroll
  for (int rp = 0; rp < 4; ++rp) {
    it.E[rp] = pk(Ev[2 * rp], Ev[2 * rp + 1]);
    it.Dd[rp] = pk(Dvv[2 * rp], Dvv[2 * rp + 1]);
  }
  const float s2 = 2.f * r.ca;
  it.S2 = pk(s2, s2);
  const int c0 = max(r.x0 - X, 0), c1 = min(r.x1 - X, kB - 1);
  it.cm = c0 > c1 ? 0u : (((2u << c1) - 1u) & ~((1u << c0) - 1u));
  return it;
}

// Contributions of the item to acc[u][rp] (column u, rows 2 rp and 2 rp + 1).
__device__ __forceinline__ void fwd_fast_item(FastItem& it, u64 (&acc)[kB][4]) {
#pragma unroll
  for (int u = 0; u < kB; ++u) {
    const u64 M = col_factor(it.cm, u);
#pragma unroll
    for (int rp = 0; rp < 4; ++rp) {
      float e0, e1;
      upk(it.E[rp], e0, e1);
      const u64 V = pk(ex2_approx(e0), ex2_approx(e1));
      acc[u][rp] = fma2(V, M, acc[u][rp]);
      if (u + 1 < kB) {
        it.E[rp] = add2(it.E[rp], it.Dd[rp]);
        if (u + 2 < kB) it.Dd[rp] = add2(it.Dd[rp], it.S2);
      }
    }
  }
}

// ---------------------------------------------------------------------------------------
// Exact path: one Gaussian on one 8 x 8 block with origin (X, Y), rows (2 rp, 2 rp + 1) per
// packed pair.
// ---------------------------------------------------------------------------------------
template <bool kExact>
struct Item {
  u64 E[4];    // fast: exponent at the current column;  exact: t at the current column
  u64 D[4];    // fast: its first difference along the row;  exact: lw - q dy^2
  u64 S2;      // fast: -2a (both halves);  exact: -a
  unsigned cm; // bit u set iff column u is inside the support box
};

// dx0, dyY: offsets of the block origin from the centre (float-float centre on the exact path).
template <bool kExact>
__device__ __forceinline__ Item<kExact> make_item(const Rec& r, float dx0, float dyY, int X, int Y) {
  Item<kExact> it;
  const u64 DX = pk(dx0, dx0), DY = pk(dyY, dyY), R2 = pk(r.r, r.r), NQ = pk(r.nq, r.nq), LW = pk(r.lw, r.lw);
  const u64 NA = pk(r.na, r.na), NA2 = pk(2.f * r.na, 2.f * r.na);
  const unsigned rm = range_bits(max(r.y0 - Y, 0), min(r.y1 - Y, kB - 1));
#pragma unroll
  for (int rp = 0; rp < 4; ++rp) {
    const u64 dy = add2(DY, pk((float)(2 * rp), (float)(2 * rp + 1)));
    const u64 t = fma2(R2, dy, DX);
    float c0, c1;
    upk(fma2(mul2(NQ, dy), dy, LW), c0, c1);
    const u64 c = pk((rm >> (2 * rp)) & 1u ? c0 : -INFINITY, (rm >> (2 * rp + 1)) & 1u ? c1 : -INFINITY);
    if (kExact) {
      it.E[rp] = t;
      it.D[rp] = c;
    } else {
      it.E[rp] = fma2(mul2(NA, t), t, c);
      it.D[rp] = fma2(NA2, t, NA);
    }
  }
  it.S2 = kExact ? NA : NA2;
  it.cm = range_bits(max(r.x0 - X, 0), min(r.x1 - X, kB - 1));
  return it;
}

// Exponents of column u (four row pairs), then the step to column u + 1.
template <bool kExact>
__device__ __forceinline__ void item_exp(Item<kExact>& it, int u, u64 (&V)[4]) {
#pragma unroll
  for (int rp = 0; rp < 4; ++rp) {
    if (kExact) {
      V[rp] = ex2x2(fma2(mul2(it.S2, it.E[rp]), it.E[rp], it.D[rp]));
      if (u + 1 < kB) it.E[rp] = add2(it.E[rp], pk(1.f, 1.f));
    } else {
      V[rp] = ex2x2(it.E[rp]);
      if (u + 1 < kB) {
        it.E[rp] = add2(it.E[rp], it.D[rp]);
        if (u + 2 < kB) it.D[rp] = add2(it.D[rp], it.S2);
      }
    }
  }
}

// Contributions of the item to acc[u][rp] (column u, rows 2 rp and 2 rp + 1).
template <bool kExact>
__device__ __forceinline__ void fwd_item(Item<kExact>& it, u64 (&acc)[kB][4]) {
#pragma unroll
  for (int u = 0; u < kB; ++u) {
    u64 V[4];
    item_exp<kExact>(it, u, V);
    const u64 M = col_factor(it.cm, u);  // a factor, not a branch: no per-pair predicate work
#pragma unroll
    for (int rp = 0; rp < 4; ++rp) acc[u][rp] = fma2(V[rp], M, acc[u][rp]);
  }
}

// The item of a well-conditioned record (a, b) on block (X, Y).
__device__ __forceinline__ void fwd_fast_record(const float4 a, const float4 b, int X, int Y, u64 (&acc)[kB][4]) {
  FastItem it = make_fast_item(fast_rec(a, b), X, Y);
  fwd_fast_item(it, acc);
}

// The item of an ill-conditioned record (a, b) on block (X, Y).  lo_g: its centre's low parts.
__device__ __forceinline__ void fwd_exact_record(const float4 a, const float4 b, const float2* __restrict__ lo_g,
                                                 int X, int Y, u64 (&acc)[kB][4]) {
  const Rec r = rec_from(a, b);
  const float2 lo = __ldg(lo_g);
  Item<true> it = make_item<true>(r, ((float)X - r.cx) - lo.x, ((float)Y - r.cy) - lo.y, X, Y);
  fwd_item<true>(it, acc);
}

// Sums of the 32 lanes' accumulators; lane L stores pixels (row L / 4, columns 2 (L % 4)
// and 2 (L % 4) + 1) of the block.
__device__ __forceinline__ void store_block(const u64 (&acc)[kB][4], float* __restrict__ Q, int b, int D, int X,
                                            int Y) {
  const int lane = threadIdx.x & 31;
  float sv[64];  // sv[8 v + u]
#pragma unroll
  for (int u = 0; u < kB; ++u)
#pragma unroll
    for (int rp = 0; rp < 4; ++rp) upk(acc[u][rp], sv[(2 * rp) * kB + u], sv[(2 * rp + 1) * kB + u]);
#pragma unroll
  for (int half = 32, off = 16; off >= 1; half >>= 1, off >>= 1) {
    const bool up = lane & off;
#pragma unroll
    for (int k = 0; k < half; ++k) {
      const float send = up ? sv[k] : sv[k + half];
      const float keep = up ? sv[k + half] : sv[k];
      sv[k] = keep + __shfl_xor_sync(0xffffffffu, send, off);
    }
  }
  const int i = Y + (lane >> 2), j = X + 2 * (lane & 3);
  if (i < D) {
    float* row = Q + ((size_t)b * D + i) * D;
    if (j < D) row[j] = sv[0];
    if (j + 1 < D) row[j + 1] = sv[1];
  }
}

// The block of a tile whose list is empty: zeros, in the layout store_block writes.
__device__ __forceinline__ void store_zero_block(float* __restrict__ Q, int b, int D, int X, int Y) {
  const int lane = threadIdx.x & 31;
  const int i = Y + (lane >> 2), j = X + 2 * (lane & 3);
  if (i < D) {
    float* row = Q + ((size_t)b * D + i) * D;
    if (j < D) row[j] = 0.f;
    if (j + 1 < D) row[j + 1] = 0.f;
  }
}

// ---------------------------------------------------------------------------------------
// Backward of one item: the six moment sums in (t, dy).
// g2[u][rp] holds dL/dQ at (column u, rows 2 rp, 2 rp + 1).
// ---------------------------------------------------------------------------------------
template <bool kExact>
__device__ __forceinline__ void bwd_item(Item<kExact>& it, const u64 (*g2)[4], const Rec& r, float dx0, float dyY,
                                         float m[6]) {
  u64 A[4], Bm[4], C[4];
#pragma unroll
  for (int rp = 0; rp < 4; ++rp) A[rp] = Bm[rp] = C[rp] = 0ull;  // +0.0 in both halves
#pragma unroll
  for (int u = 0; u < kB; ++u) {
    const float uc = (float)u - 3.5f;
    const u64 U = pk(uc, uc), U2 = pk(uc * uc, uc * uc);
    const ulonglong2 ga = reinterpret_cast<const ulonglong2*>(g2[u])[0];
    const ulonglong2 gb = reinterpret_cast<const ulonglong2*>(g2[u])[1];
    u64 V[4];
    item_exp<kExact>(it, u, V);
    // the column mask as a factor on the three weights: (A, B, C) += (1, uc, uc^2) m T
    const u64 M = col_factor(it.cm, u), UM = mul2(U, M), U2M = mul2(U2, M);
    const u64 gg[4] = {ga.x, ga.y, gb.x, gb.y};
#pragma unroll
    for (int rp = 0; rp < 4; ++rp) {
      const u64 T = mul2(gg[rp], V[rp]);
      A[rp] = fma2(T, M, A[rp]);
      Bm[rp] = fma2(UM, T, Bm[rp]);
      C[rp] = fma2(U2M, T, C[rp]);
    }
  }
  // per row: sum T t = tc R0 + R1, sum T t^2 = tc (tc R0 + R1) + (tc R1 + R2), with tc = t at
  // uc = 0 (column 3.5); then weights dy, dy^2 for the rows
  const u64 DXc = pk(dx0 + 3.5f, dx0 + 3.5f), DY = pk(dyY, dyY), R2 = pk(r.r, r.r);
  u64 s0 = 0ull, s1 = 0ull, s2 = 0ull, s3 = 0ull, s4 = 0ull, s5 = 0ull;
#pragma unroll
  for (int rp = 0; rp < 4; ++rp) {
    const u64 dy = add2(DY, pk((float)(2 * rp), (float)(2 * rp + 1)));
    const u64 tc = fma2(R2, dy, DXc);
    const u64 X1 = fma2(tc, A[rp], Bm[rp]);
    const u64 X2 = fma2(tc, X1, fma2(tc, Bm[rp], C[rp]));
    s0 = add2(s0, A[rp]);
    s1 = add2(s1, X1);
    s2 = fma2(dy, A[rp], s2);
    s3 = add2(s3, X2);
    s4 = fma2(dy, X1, s4);
    s5 = fma2(mul2(dy, dy), A[rp], s5);
  }
  float p, q;
  upk(s0, p, q); m[0] = p + q;
  upk(s1, p, q); m[1] = p + q;
  upk(s2, p, q); m[2] = p + q;
  upk(s3, p, q); m[3] = p + q;
  upk(s4, p, q); m[4] = p + q;
  upk(s5, p, q); m[5] = p + q;
}

// Moment sums of the exact-path item of record r on block (X, Y).
__device__ __forceinline__ void bwd_exact_record(const Rec& r, const float2* __restrict__ lo_g, int X, int Y,
                                                 const u64 (*g2)[4], float m[6]) {
  const float2 lo = __ldg(lo_g);
  const float dx0 = ((float)X - r.cx) - lo.x, dyY = ((float)Y - r.cy) - lo.y;
  Item<true> it = make_item<true>(r, dx0, dyY, X, Y);
  bwd_item<true>(it, g2, r, dx0, dyY, m);
}

// Gradient of one (particle, Gaussian) pair: mu~ and Sigma~ (full-matrix, symmetric).
struct Grad2 {
  float gmx, gmy, gxx, gxy, gyy;
};

// From the moment sums (M0, Mt, Md, Mtt, Mtd, Mdd) of the pair's pixels:
// dL/dlw = ln2 M0, dL/da = -ln2 Mtt, dL/dr = -2 a ln2 Mtd, dL/dq = -ln2 Mdd,
// dL/dcx = 2 a ln2 Mt, dL/dcy = 2 ln2 (a r Mt + q Md); then the chain to Sigma~ through
// a = c Syy/det, r = Sxy/Syy, q = c/Syy (c = log2(e)/2, pixel units) and the
// normalization lw = log2(A / (2 pi sqrt(det))), whose Sigma~ gradient is -M0 P / 2.
// ih = 1/h and ih2 = 1/h^2 (h the pixel size in model units).
__device__ __forceinline__ Grad2 pair_grad(const Rec& r, const float* m, float ih, float ih2) {
  const float a = -r.na, rr = r.r, q = -r.nq;
  const float M0 = m[0], Mt = m[1], Md = m[2], Mtt = m[3], Mtd = m[4], Mdd = m[5];
  const float lp = kLn2 / kHalfLog2e, hc = 0.5f / kHalfLog2e;
  const float ar = a * rr;
  Grad2 o;
  o.gmx = 2.f * kLn2 * a * Mt * ih;
  o.gmy = -2.f * kLn2 * fmaf(ar, Mt, q * Md) * ih;
  o.gxx = (lp * a * a * Mtt - hc * a * M0) * ih2;
  o.gyy = (lp * fmaf(ar * ar, Mtt, fmaf(2.f * ar * q, Mtd, q * q * Mdd)) - hc * fmaf(ar, rr, q) * M0) * ih2;
  o.gxy = (hc * ar * M0 - lp * a * fmaf(ar, Mtt, q * Mtd)) * ih2;
  return o;
}

// Fast path backward: the six centred moment sums of t = g * contribution in (dx, dy), then
// grad_mu~ = h P (Sx, -Sy), grad_Sigma~ = (h^2 P M P - S0 P) / 2 with P from the expanded form.
__device__ __forceinline__ void bwd_fast_item(FastItem& it, const u64 (*g2)[4], const FastRec& r, int X, int Y, float S[6]) {
  u64 A[4], Bm[4], C[4];
#pragma unroll
  for (int rp = 0; rp < 4; ++rp) A[rp] = Bm[rp] = C[rp] = pk(0.f, 0.f);
#pragma unroll
  for (int u = 0; u < kB; ++u) {
    const bool on = (it.cm >> u) & 1u;
    const float uc = (float)u - 3.5f;
    const u64 U = pk(uc, uc), U2 = pk(uc * uc, uc * uc);
    const ulonglong2 ga = reinterpret_cast<const ulonglong2*>(g2[u])[0];
    const ulonglong2 gb = reinterpret_cast<const ulonglong2*>(g2[u])[1];
    const u64 gg[4] = {ga.x, ga.y, gb.x, gb.y};
#pragma unroll
    for (int rp = 0; rp < 4; ++rp) {
      float e0, e1;
      upk(it.E[rp], e0, e1);
      const u64 V = pk(ex2_approx(e0), ex2_approx(e1));
      const u64 t = on ? mul2(gg[rp], V) : 0ull;  // +0.0 in both halves
      A[rp] = add2(A[rp], t);
      Bm[rp] = fma2(U, t, Bm[rp]);
      C[rp] = fma2(U2, t, C[rp]);
      if (u + 1 < kB) {
        it.E[rp] = add2(it.E[rp], it.Dd[rp]);
        if (u + 2 < kB) it.Dd[rp] = add2(it.Dd[rp], it.S2);
      }
    }
  }
  float R0[kB], R1[kB], R2[kB];
#pragma unroll
  for (int rp = 0; rp < 4; ++rp) {
    upk(A[rp], R0[2 * rp], R0[2 * rp + 1]);
    upk(Bm[rp], R1[2 * rp], R1[2 * rp + 1]);
    upk(C[rp], R2[2 * rp], R2[2 * rp + 1]);
  }
  // moments about the block centre (uc, vc = u - 3.5, v - 3.5)
  float M0 = 0.f, Mu = 0.f, Muu = 0.f, Mv = 0.f, Muv = 0.f, Mvv = 0.f;
#pragma unroll
  for (int v = 0; v < kB; ++v) {
    const float vc = (float)v - 3.5f;
    M0 += R0[v];
    Mu += R1[v];
    Muu += R2[v];
    Mv = fmaf(vc, R0[v], Mv);
    Muv = fmaf(vc, R1[v], Muv);
    Mvv = fmaf(vc * vc, R0[v], Mvv);
  }
  // shift to the Gaussian centre: dx = dxc + uc, dy = dyc + vc
  const float dxc = (float)X + 3.5f - r.cx, dyc = (float)Y + 3.5f - r.cy;
  S[0] = M0;
  S[1] = fmaf(dxc, M0, Mu);
  S[2] = fmaf(dyc, M0, Mv);
  S[3] = fmaf(dxc, fmaf(dxc, M0, 2.f * Mu), Muu);
  S[4] = fmaf(dxc, fmaf(dyc, M0, Mv), fmaf(dyc, Mu, Muv));
  S[5] = fmaf(dyc, fmaf(dyc, M0, 2.f * Mv), Mvv);
}

__device__ __forceinline__ Grad2 fast_grad(const FastRec& r, const float S[6], float kap, float h) {
  const float pxx = kap * r.ca, pyy = kap * r.cc, pxy = -0.5f * kap * r.cb;
  // App. A.2 Eq. 18: grad_mu_tilde = sum Gc P d, d = (h dx, -h dy)
  const float gmx = h * (pxx * S[1] - pxy * S[2]);
  const float gmy = h * (pxy * S[1] - pyy * S[2]);
  // Eq. 20: grad_Sigma_tilde = -P (S0 Sigma_tilde - h^2 M) P / 2 = (h^2 P M P - S0 P) / 2
  const float h2 = h * h;
  const float a00 = pxx * S[3] - pxy * S[4], a01 = -pxx * S[4] + pxy * S[5];
  const float a10 = pxy * S[3] - pyy * S[4], a11 = -pxy * S[4] + pyy * S[5];
  const float b00 = a00 * pxx + a01 * pxy, b01 = a00 * pxy + a01 * pyy, b11 = a10 * pxy + a11 * pyy;
  const float gxx = 0.5f * (h2 * b00 - S[0] * pxx);
  const float gxy = 0.5f * (h2 * b01 - S[0] * pxy);
  const float gyy = 0.5f * (h2 * b11 - S[0] * pyy);
  return Grad2{gmx, gmy, gxx, gxy, gyy};
}

// World-space gradient of the pair, added into the Gaussian's accumulator: mu_dot = W mu,
// Sigma_dot = W Sigma W^T, Eq. 21 embedding.  W holds the first two rows of the pose.
__device__ __forceinline__ void flush_grad(const Grad2& q, float M0, const float W[6], float* __restrict__ dst) {
  float o[10];
#pragma unroll
  for (int c = 0; c < 3; ++c) o[c] = W[c] * q.gmx + W[3 + c] * q.gmy;
  const int kk[6] = {0, 0, 0, 1, 1, 2}, ll[6] = {0, 1, 2, 1, 2, 2};
#pragma unroll
  for (int e = 0; e < 6; ++e) {
    const float ak = W[kk[e]], bk = W[3 + kk[e]], al = W[ll[e]], bl = W[3 + ll[e]];
    o[3 + e] = ak * q.gxx * al + ak * q.gxy * bl + bk * q.gxy * al + bk * q.gyy * bl;
  }
  o[9] = M0;
  red_add_v4(dst, o[0], o[1], o[2], o[3]);
  red_add_v4(dst + 4, o[4], o[5], o[6], o[7]);
  red_add_v2(dst + 8, o[8], o[9]);
}

// Pose gradients of one (particle, Gaussian) pair: mu_dot = W mu and Sigma_dot = W Sigma W^T
// give dL/dW = grad_mu_dot mu^T + 2 G W Sigma (G the embedded grad_Sigma_tilde, symmetric;
// rows 0 and 1 only), and a model translation t gives dL/dt = grad_mu_tilde.  acc: dW rows
// 0 and 1 (6 values), dt (2 values).  G row of the activated table: mu, M = R diag(s).
__device__ __forceinline__ void pose_accum(float acc[8], const float* __restrict__ Grow, const float W[6],
                                           const Grad2& q) {
  const float4 a0 = __ldg(reinterpret_cast<const float4*>(Grow));      // mu[3], M00
  const float4 a1 = __ldg(reinterpret_cast<const float4*>(Grow) + 1);  // M01 M02 M10 M11
  const float4 a2 = __ldg(reinterpret_cast<const float4*>(Grow) + 2);  // M12 M20 M21 M22
  const float mu[3] = {a0.x, a0.y, a0.z};
  const float M[9] = {a0.w, a1.x, a1.y, a1.z, a1.w, a2.x, a2.y, a2.z, a2.w};
  float V[2][3], WS[2][3];
#pragma unroll
  for (int a = 0; a < 2; ++a)
#pragma unroll
    for (int m = 0; m < 3; ++m) V[a][m] = W[3 * a] * M[m] + W[3 * a + 1] * M[3 + m] + W[3 * a + 2] * M[6 + m];
#pragma unroll
  for (int a = 0; a < 2; ++a)
#pragma unroll
    for (int i = 0; i < 3; ++i) WS[a][i] = V[a][0] * M[3 * i] + V[a][1] * M[3 * i + 1] + V[a][2] * M[3 * i + 2];
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    acc[i] += q.gmx * mu[i] + 2.f * (q.gxx * WS[0][i] + q.gxy * WS[1][i]);
    acc[3 + i] += q.gmy * mu[i] + 2.f * (q.gxy * WS[0][i] + q.gyy * WS[1][i]);
  }
  acc[6] += q.gmx;
  acc[7] += q.gmy;
}

// Warp sum of the lanes' pose accumulators, added by lane 0 into dpose[12] (dW row-major,
// rows 0 and 1 at 0..5; dt at 10 and 11, 8-byte aligned for the vector reduction).
__device__ __forceinline__ void pose_flush(float acc[8], float* __restrict__ dpose) {
#pragma unroll
  for (int k = 0; k < 8; ++k)
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc[k] += __shfl_xor_sync(0xffffffffu, acc[k], o);
  if ((threadIdx.x & 31) == 0) {
    red_add_v4(dpose, acc[0], acc[1], acc[2], acc[3]);
    red_add_v2(dpose + 4, acc[4], acc[5]);
    red_add_v2(dpose + 10, acc[6], acc[7]);
  }
}

// dL/dQ of the block into g2 (shared, [u][rp] packed row pairs); called by one warp.
__device__ __forceinline__ void load_block_grad(float* __restrict__ g2f, const float* __restrict__ dLdQ, int b, int D,
                                                int X, int Y) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int k = 0; k < 2; ++k) {
    const int p = 2 * lane + k;  // p = 8 v + u
    const int v = p >> 3, u = p & 7;
    const int i = Y + v, j = X + u;
    const float g = (i < D && j < D) ? dLdQ[((size_t)b * D + i) * D + j] : 0.f;
    g2f[(u * 4 + (v >> 1)) * 2 + (v & 1)] = g;
  }
}

// Backward of one (particle, Gaussian, block) item: moments, gradient, reductions.
// kap = -2 / (log2(e) h^2) turns a fast record's coefficients into P = Sigma~^-1.
template <bool kPose>
__device__ __forceinline__ void bwd_fast_pair(const float4 a, const float4 b, uint32_t g, int X, int Y,
                                              const u64 (*g2)[4], const float W[6], float h, float kap,
                                              float* __restrict__ wacc, const float* __restrict__ gauss,
                                              float* pacc) {
  const FastRec r = fast_rec(a, b);
  FastItem it = make_fast_item(r, X, Y);
  float S[6];
  bwd_fast_item(it, g2, r, X, Y, S);
  const Grad2 q = fast_grad(r, S, kap, h);
  flush_grad(q, S[0], W, wacc + (size_t)g * kGradStride);
  if (kPose) pose_accum(pacc, gauss + (size_t)g * kGaussStride, W, q);
}

template <bool kPose>
__device__ __forceinline__ void bwd_exact_pair(const float4 a, const float4 b, uint32_t g,
                                               const float2* __restrict__ lo, int X, int Y, const u64 (*g2)[4],
                                               const float W[6], float ih, float ih2, float* __restrict__ wacc,
                                               const float* __restrict__ gauss, float* pacc) {
  const Rec r = rec_from(a, b);
  float m[6];
  bwd_exact_record(r, lo + g, X, Y, g2, m);
  const Grad2 q = pair_grad(r, m, ih, ih2);
  flush_grad(q, m[0], W, wacc + (size_t)g * kGradStride);
  if (kPose) pose_accum(pacc, gauss + (size_t)g * kGaussStride, W, q);
}

// ---------------------------------------------------------------------------------------
// Tiles of 8 pixels: one warp per (particle, tile).
// ---------------------------------------------------------------------------------------
__global__ void __launch_bounds__(kTileWarps * 32, kFwd8MinBlocks) k_render_fwd8(
    const gs_record* __restrict__ proj, const float2* __restrict__ lo_all, int N,
    const uint32_t* __restrict__ pair_gauss, const uint32_t* __restrict__ ranges, int D, int ntx,
    float* __restrict__ Q) {
  const int lane = threadIdx.x & 31, b = blockIdx.y;
  const int tile = quad_tile(blockIdx.x, threadIdx.x >> 5, ntx);
  if (tile < 0) return;  // warp-uniform
  const int X = (tile % ntx) * kB, Y = (tile / ntx) * kB;
  const size_t rr = ((size_t)b * ntx * ntx + tile) * 2;
  const uint32_t start = ranges[rr], end = ranges[rr + 1];
  if (start >= end) {  // warp-uniform: no Gaussian touches the block
    store_zero_block(Q, b, D, X, Y);
    return;
  }
  const float4* pr = reinterpret_cast<const float4*>(proj + (size_t)b * N);
  const float2* lo = lo_all + (size_t)b * N;
  const uint32_t gmax = (uint32_t)N - 1u;  // pair entries are clamped: a bad list cannot leave proj
  u64 acc[kB][4];
#pragma unroll
  for (int u = 0; u < kB; ++u)
#pragma unroll
    for (int rp = 0; rp < 4; ++rp) acc[u][rp] = 0ull;
  // record of the current item in (na, nb); list entries (Gaussian indices) of the next three
  // in g1, g2, g3, kept as loaded and clamped only where used, so that nothing waits on a list
  // load before its use three items later (a clamp next to the load would stall the warp for
  // the load's full latency every item); the record two items ahead is prefetched into L1 so
  // that its load one item ahead hits there
  uint32_t i = start + lane;
  float4 na = make_float4(0.f, 0.f, 0.f, 0.f), nb = na;
  uint32_t g1 = 0, g2 = 0, g3 = 0;
  bool any_exact = false;
  if (i < end) {
    const uint32_t g0 = min(pair_gauss[i], gmax);
    na = __ldg(pr + 2 * (size_t)g0);
    nb = __ldg(pr + 2 * (size_t)g0 + 1);
  }
  if (i + 32 < end) g1 = pair_gauss[i + 32];
  if (i + 64 < end) g2 = pair_gauss[i + 64];
  if (i + 64 < end) asm volatile("prefetch.global.L1 [%0];" ::"l"(pr + 2 * (size_t)min(g2, gmax)));
  if (i + 96 < end) g3 = pair_gauss[i + 96];
  while (i < end) {
    const float4 ca = na, cb = nb;
    i += 32;
    if (i < end) {
      const uint32_t gc = min(g1, gmax);
      na = __ldg(pr + 2 * (size_t)gc);
      nb = __ldg(pr + 2 * (size_t)gc + 1);
      if (i + 64 < end) asm volatile("prefetch.global.L1 [%0];" ::"l"(pr + 2 * (size_t)min(g3, gmax)));
      g1 = g2;
      g2 = g3;
      if (i + 96 < end) g3 = pair_gauss[i + 96];
    }
    if (!exact_record(ca))
      fwd_fast_record(ca, cb, X, Y, acc);
    else
      any_exact = true;
  }
  // ill-conditioned records, in a second pass over the same lane's entries (rare)
  if (__any_sync(0xffffffffu, any_exact)) {
    for (uint32_t j = start + lane; j < end; j += 32) {
      const uint32_t g = min(pair_gauss[j], gmax);
      const float4 a = __ldg(pr + 2 * (size_t)g);
      if (exact_record(a)) fwd_exact_record(a, __ldg(pr + 2 * (size_t)g + 1), lo + g, X, Y, acc);
    }
  }
  store_block(acc, Q, b, D, X, Y);
}

template <bool kPose>
__global__ void __launch_bounds__(kTileWarps * 32, kBwd8MinBlocks) k_render_bwd8(const gs_record* __restrict__ proj,
                                                                 const float2* __restrict__ lo_all, int N,
                                                                 const uint32_t* __restrict__ pair_gauss,
                                                                 const uint32_t* __restrict__ ranges, int D, int ntx,
                                                                 const float* __restrict__ dLdQ,
                                                                 const float* __restrict__ Wall, float h,
                                                                 float ih, float ih2, float* __restrict__ wacc,
                                                                 const float* __restrict__ gauss,
                                                                 float* __restrict__ dpose) {
  __shared__ __align__(16) u64 g2all[kTileWarps][kB][4];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, b = blockIdx.y;
  const int tile = quad_tile(blockIdx.x, warp, ntx);
  if (tile < 0) return;  // warp-uniform
  const int X = (tile % ntx) * kB, Y = (tile / ntx) * kB;
  const size_t rr = ((size_t)b * ntx * ntx + tile) * 2;
  const uint32_t start = ranges[rr], end = ranges[rr + 1];
  if (start >= end) return;  // warp-uniform
  const u64(*g2)[4] = g2all[warp];
  load_block_grad(reinterpret_cast<float*>(g2all[warp]), dLdQ, b, D, X, Y);
  float W[6];
#pragma unroll
  for (int c = 0; c < 6; ++c) W[c] = Wall[(size_t)b * 9 + c];
  const float kap = -2.f * ih2 / kLog2e;  // P = kap * [[ca, -cb/2], [-cb/2, cc]] (fast records)
  __syncwarp();
  const float4* pr = reinterpret_cast<const float4*>(proj + (size_t)b * N);
  const float2* lo = lo_all + (size_t)b * N;
  const uint32_t gmax = (uint32_t)N - 1u;  // pair entries are clamped: a bad list cannot leave proj / wacc
  float pacc[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
  // list entries are kept as loaded and clamped where used (see k_render_fwd8)
  uint32_t i = start + lane;
  float4 na = make_float4(0.f, 0.f, 0.f, 0.f), nb = na;
  uint32_t g0 = 0, g1 = 0;
  bool any_exact = false;
  if (i < end) {
    g0 = min(pair_gauss[i], gmax);
    na = __ldg(pr + 2 * (size_t)g0);
    nb = __ldg(pr + 2 * (size_t)g0 + 1);
  }
  if (i + 32 < end) g1 = pair_gauss[i + 32];
  while (i < end) {
    const float4 ca = na, cb = nb;
    const uint32_t g = g0;
    i += 32;
    if (i < end) {
      g0 = min(g1, gmax);
      na = __ldg(pr + 2 * (size_t)g0);
      nb = __ldg(pr + 2 * (size_t)g0 + 1);
      if (i + 32 < end) g1 = pair_gauss[i + 32];
    }
    if (!exact_record(ca))
      bwd_fast_pair<kPose>(ca, cb, g, X, Y, g2, W, h, kap, wacc, gauss, pacc);
    else
      any_exact = true;
  }
  // ill-conditioned records, in a second pass over the same lane's entries (rare)
  if (__any_sync(0xffffffffu, any_exact)) {
    for (uint32_t j = start + lane; j < end; j += 32) {
      const uint32_t g = min(pair_gauss[j], gmax);
      const float4 a = __ldg(pr + 2 * (size_t)g);
      if (exact_record(a))
        bwd_exact_pair<kPose>(a, __ldg(pr + 2 * (size_t)g + 1), g, lo, X, Y, g2, W, ih, ih2, wacc, gauss, pacc);
    }
  }
  if (kPose) pose_flush(pacc, dpose + (size_t)b * 12);
}

// ---------------------------------------------------------------------------------------
// Tiles of 16 or 32 pixels: four warps per 16 x 16 region, records staged in chunks.
// ---------------------------------------------------------------------------------------
struct Region {
  int RX, RY;
};

__device__ __forceinline__ Region region_of(int T, int ntx, int tile, int sub) {
  Region g;
  g.RX = (tile % ntx) * T + (sub & 1) * 16;
  g.RY = (tile / ntx) * T + (sub >> 1) * 16;
  return g;
}

// Bit by * 2 + bx set iff the box touches 8 x 8 block (bx, by) of the region.
__device__ __forceinline__ unsigned block_mask(int x0, int x1, int y0, int y1, const Region& g) {
  const int lx = max(x0 - g.RX, 0), hx = min(x1 - g.RX, 15);
  const int ly = max(y0 - g.RY, 0), hy = min(y1 - g.RY, 15);
  if (lx > hx || ly > hy) return 0u;
  const int bx0 = lx >> 3, bx1 = hx >> 3, by0 = ly >> 3, by1 = hy >> 3;
  const unsigned cols = ((2u << bx1) - 1u) & ~((1u << bx0) - 1u);
  unsigned m = 0u;
  for (int by = by0; by <= by1; ++by) m |= cols << (by * 2);
  return m;
}

// Stage records [start, start + n) of the tile list, their Gaussian indices and block masks.
__device__ __forceinline__ void stage_chunk(gs_record* rec, uint32_t* gid, uint8_t* msk,
                                            const gs_record* __restrict__ proj, size_t pbase,
                                            const uint32_t* __restrict__ pair_gauss, uint32_t start, int n,
                                            const Region& reg, uint32_t gmax) {
  for (int k = threadIdx.x; k < n; k += blockDim.x) {
    const uint32_t g = min(pair_gauss[start + k], gmax);  // a bad list cannot leave proj
    const float4* src = reinterpret_cast<const float4*>(proj + pbase + g);
    float4* dst = reinterpret_cast<float4*>(rec + k);
    const float4 a = __ldg(src), b = __ldg(src + 1);
    dst[0] = a;
    dst[1] = b;
    gid[k] = g;
    const int bx = __float_as_int(b.z), by = __float_as_int(b.w);
    msk[k] = (uint8_t)block_mask((int)(int16_t)(bx & 0xffff), bx >> 16, (int)(int16_t)(by & 0xffff), by >> 16, reg);
  }
}

// Ballot compaction of the chunk's records whose mask has bit `blk`: their indices go to
// list[0..cnt) in index order; returns cnt (warp-uniform).
__device__ __forceinline__ int compact_mask(const uint8_t* msk, int n, int blk, uint16_t* list) {
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

__global__ void __launch_bounds__(kRegionWarps * 32) k_render_fwd16(const gs_record* __restrict__ proj,
                                                                    const float2* __restrict__ lo_all, int N,
                                                                    const uint32_t* __restrict__ pair_gauss,
                                                                    const uint32_t* __restrict__ ranges, int D, int T,
                                                                    int ntx, int chunk, float* __restrict__ Q) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  gs_record* rec = reinterpret_cast<gs_record*>(smem_raw);
  uint32_t* gid = reinterpret_cast<uint32_t*>(smem_raw + sizeof(gs_record) * chunk);
  uint8_t* msk = reinterpret_cast<uint8_t*>(gid + chunk);
  uint16_t* list = reinterpret_cast<uint16_t*>(msk + ((chunk + 15) & ~15)) + warp * chunk;
  const int regions = T == 32 ? 4 : 1;
  const int tile = blockIdx.x / regions, sub = blockIdx.x % regions, b = blockIdx.y;
  const Region reg = region_of(T, ntx, tile, sub);
  const int X = reg.RX + (warp & 1) * kB, Y = reg.RY + (warp >> 1) * kB;
  const size_t rr = ((size_t)b * ntx * ntx + tile) * 2;
  const uint32_t start = ranges[rr], end = ranges[rr + 1];
  if (start >= end) {  // uniform over the CTA: no Gaussian touches the region
    store_zero_block(Q, b, D, X, Y);
    return;
  }
  const size_t pbase = (size_t)b * N;
  const float2* lo = lo_all + pbase;
  u64 acc[kB][4];
#pragma unroll
  for (int u = 0; u < kB; ++u)
#pragma unroll
    for (int rp = 0; rp < 4; ++rp) acc[u][rp] = 0ull;
  // pass 0: well-conditioned records; pass 1 (only if any): ill-conditioned ones, dealt to the
  // same lanes, so every lane adds its items in the same order as the tile-8 kernel
  bool any_exact = false;
  for (int pass = 0; pass < 2; ++pass) {
    if (pass == 1 && !__syncthreads_or(any_exact)) break;
    int running = 0;
    for (uint32_t base = start; base < end; base += chunk) {
      const int n = (int)min((uint32_t)chunk, end - base);
      __syncthreads();
      stage_chunk(rec, gid, msk, proj, pbase, pair_gauss, base, n, reg, (uint32_t)N - 1u);
      __syncthreads();
      const int cnt = compact_mask(msk, n, warp, list);
      for (int j = (lane - running) & 31; j < cnt; j += 32) {
        const int k = list[j];
        const float4* src = reinterpret_cast<const float4*>(rec + k);
        const float4 a = src[0];
        if (!exact_record(a)) {
          if (pass == 0) fwd_fast_record(a, src[1], X, Y, acc);
        } else {
          any_exact = true;
          if (pass == 1) fwd_exact_record(a, src[1], lo + gid[k], X, Y, acc);
        }
      }
      running = (running + cnt) & 31;
    }
  }
  store_block(acc, Q, b, D, X, Y);
}

template <bool kPose>
__global__ void __launch_bounds__(kRegionWarps * 32) k_render_bwd16(const gs_record* __restrict__ proj,
                                                                    const float2* __restrict__ lo_all, int N,
                                                                    const uint32_t* __restrict__ pair_gauss,
                                                                    const uint32_t* __restrict__ ranges, int D, int T,
                                                                    int ntx, int chunk, const float* __restrict__ dLdQ,
                                                                    const float* __restrict__ Wall, float h,
                                                                    float ih, float ih2, float* __restrict__ wacc,
                                                                    const float* __restrict__ gauss,
                                                                    float* __restrict__ dpose) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ __align__(16) u64 g2all[kRegionWarps][kB][4];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  gs_record* rec = reinterpret_cast<gs_record*>(smem_raw);
  uint32_t* gid = reinterpret_cast<uint32_t*>(smem_raw + sizeof(gs_record) * chunk);
  uint8_t* msk = reinterpret_cast<uint8_t*>(gid + chunk);
  uint16_t* list = reinterpret_cast<uint16_t*>(msk + ((chunk + 15) & ~15)) + warp * chunk;
  const int regions = T == 32 ? 4 : 1;
  const int tile = blockIdx.x / regions, sub = blockIdx.x % regions, b = blockIdx.y;
  const Region reg = region_of(T, ntx, tile, sub);
  const int X = reg.RX + (warp & 1) * kB, Y = reg.RY + (warp >> 1) * kB;
  const size_t rr = ((size_t)b * ntx * ntx + tile) * 2;
  const uint32_t start = ranges[rr], end = ranges[rr + 1];
  if (start >= end) return;  // CTA-uniform
  load_block_grad(reinterpret_cast<float*>(g2all[warp]), dLdQ, b, D, X, Y);
  float W[6];
#pragma unroll
  for (int c = 0; c < 6; ++c) W[c] = Wall[(size_t)b * 9 + c];
  const float kap = -2.f * ih2 / kLog2e;
  const size_t pbase = (size_t)b * N;
  const float2* lo = lo_all + pbase;
  float pacc[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
  bool any_exact = false;
  for (int pass = 0; pass < 2; ++pass) {
    if (pass == 1 && !__syncthreads_or(any_exact)) break;
    for (uint32_t base = start; base < end; base += chunk) {
      const int n = (int)min((uint32_t)chunk, end - base);
      __syncthreads();
      stage_chunk(rec, gid, msk, proj, pbase, pair_gauss, base, n, reg, (uint32_t)N - 1u);
      __syncthreads();
      const int cnt = compact_mask(msk, n, warp, list);
      for (int j = lane; j < cnt; j += 32) {
        const int k = list[j];
        const float4* src = reinterpret_cast<const float4*>(rec + k);
        const float4 a = src[0];
        if (!exact_record(a)) {
          if (pass == 0) bwd_fast_pair<kPose>(a, src[1], gid[k], X, Y, g2all[warp], W, h, kap, wacc, gauss, pacc);
        } else {
          any_exact = true;
          if (pass == 1)
            bwd_exact_pair<kPose>(a, src[1], gid[k], lo, X, Y, g2all[warp], W, ih, ih2, wacc, gauss, pacc);
        }
      }
    }
  }
  if (kPose) pose_flush(pacc, dpose + (size_t)b * 12);
}

// dL/dTheta of one Gaussian from its accumulated sums: dL/dA = sum S0 / A, and the chain from
// (grad_mu, grad_Sigma) to theta through the activations.  Adds to out[11] and re-zeroes the
// accumulator it consumed.
__device__ __forceinline__ void finalize_one(const float* G, const float* th, float* acc, float* out) {
  if (G[kBad] != 0.f) return;
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

constexpr int kFinG = 128;     // Gaussians per finalize CTA, one per thread
constexpr int kFinGRow = kGaussStride + 1;  // padded table row in shared memory (no bank conflicts)

// The per-Gaussian rows (activated table, Theta, dL/dTheta) are staged through shared memory
// with coalesced loads; each thread then works on its own Gaussian's row.
__global__ void __launch_bounds__(kFinG) k_bwd_finalize(const float* __restrict__ theta,
                                                       const float* __restrict__ gauss, int N,
                                                       float* __restrict__ wacc, float* __restrict__ dtheta) {
  __shared__ float sG[kFinG * kFinGRow];
  __shared__ float sT[kFinG * 11];
  __shared__ float sD[kFinG * 11];
  const int g0 = blockIdx.x * kFinG;
  const int n = min(kFinG, N - g0);
  const float* gsrc = gauss + (size_t)g0 * kGaussStride;
  for (int i = threadIdx.x; i < n * kGaussStride; i += kFinG) {
    const int r = i / kGaussStride;
    sG[r * kFinGRow + (i - r * kGaussStride)] = __ldg(gsrc + i);
  }
  const float* tsrc = theta + (size_t)g0 * 11;
  float* dsrc = dtheta + (size_t)g0 * 11;
  for (int i = threadIdx.x; i < n * 11; i += kFinG) {
    sT[i] = __ldg(tsrc + i);
    sD[i] = dsrc[i];
  }
  __syncthreads();
  if ((int)threadIdx.x < n) finalize_one(sG + threadIdx.x * kFinGRow, sT + threadIdx.x * 11,
                                         wacc + (size_t)(g0 + threadIdx.x) * kGradStride,
                                         sD + threadIdx.x * 11);
  __syncthreads();
  for (int i = threadIdx.x; i < n * 11; i += kFinG) dsrc[i] = sD[i];
}

}  // namespace

static dim3 render_grid(const gs_config& cfg, int B) {
  const int ntx = (cfg.D + cfg.tile - 1) / cfg.tile;
  return dim3(ntx * ntx * (cfg.tile == 32 ? 4 : 1), B);
}

static size_t region_smem(int chunk) {
  return sizeof(gs_record) * chunk + sizeof(uint32_t) * chunk + ((chunk + 15) & ~15) +
         sizeof(uint16_t) * kRegionWarps * chunk;
}

// The low parts of the centres follow the records and the box plane in the projection buffer.
static const float2* lo_plane(const gs_record* proj, int B, int N) {
  return reinterpret_cast<const float2*>(reinterpret_cast<const char*>(proj) +
                                         (sizeof(gs_record) + sizeof(int2)) * (size_t)B * (size_t)N);
}

cudaError_t launch_render_fwd(const gs_config& cfg, const gs_record* proj, int N, const uint32_t* pair_gauss,
                              const uint32_t* ranges, int B, float* Q, cudaStream_t s) {
  if (B <= 0) return cudaSuccess;
  const int ntx = (cfg.D + cfg.tile - 1) / cfg.tile;
  const float2* lo = lo_plane(proj, B, N);
  if (cfg.tile == 8) {
    const dim3 grid(((ntx + 1) / 2) * ((ntx + 1) / 2), B);
    k_render_fwd8<<<grid, kTileWarps * 32, 0, s>>>(proj, lo, N, pair_gauss, ranges, cfg.D, ntx, Q);
    return cudaGetLastError();
  }
  const size_t sm = region_smem(cfg.chunk);
  {
    static int cache[64] = {0};
    cudaError_t e = ensure_smem((const void*)k_render_fwd16, sm, cache);
    if (e != cudaSuccess) return e;
  }
  k_render_fwd16<<<render_grid(cfg, B), kRegionWarps * 32, sm, s>>>(proj, lo, N, pair_gauss, ranges, cfg.D,
                                                                    cfg.tile, ntx, cfg.chunk, Q);
  return cudaGetLastError();
}

cudaError_t launch_render_bwd(const gs_config& cfg, const gs_record* proj, int N, const uint32_t* pair_gauss,
                              const uint32_t* ranges, int B, const float* dLdQ, const float* W, float* wacc,
                              const float* gauss, float* dpose, cudaStream_t s) {
  if (B <= 0) return cudaSuccess;
  const int ntx = (cfg.D + cfg.tile - 1) / cfg.tile;
  const float h = 2.f * cfg.E / (float)cfg.D, ih = 1.f / h, ih2 = 1.f / (h * h);
  const float2* lo = lo_plane(proj, B, N);
  if (cfg.tile == 8) {
    const dim3 grid(((ntx + 1) / 2) * ((ntx + 1) / 2), B);
    if (dpose)
      k_render_bwd8<true><<<grid, kTileWarps * 32, 0, s>>>(proj, lo, N, pair_gauss, ranges, cfg.D, ntx, dLdQ, W, h,
                                                            ih, ih2, wacc, gauss, dpose);
    else
      k_render_bwd8<false><<<grid, kTileWarps * 32, 0, s>>>(proj, lo, N, pair_gauss, ranges, cfg.D, ntx, dLdQ, W, h,
                                                             ih, ih2, wacc, gauss, dpose);
    return cudaGetLastError();
  }
  const size_t sm = region_smem(cfg.chunk);
  {
    static int cache[2][64] = {{0}};
    cudaError_t e = dpose ? ensure_smem((const void*)k_render_bwd16<true>, sm, cache[1])
                          : ensure_smem((const void*)k_render_bwd16<false>, sm, cache[0]);
    if (e != cudaSuccess) return e;
  }
  if (dpose)
    k_render_bwd16<true><<<render_grid(cfg, B), kRegionWarps * 32, sm, s>>>(
        proj, lo, N, pair_gauss, ranges, cfg.D, cfg.tile, ntx, cfg.chunk, dLdQ, W, h, ih, ih2, wacc, gauss, dpose);
  else
    k_render_bwd16<false><<<render_grid(cfg, B), kRegionWarps * 32, sm, s>>>(
        proj, lo, N, pair_gauss, ranges, cfg.D, cfg.tile, ntx, cfg.chunk, dLdQ, W, h, ih, ih2, wacc, gauss, dpose);
  return cudaGetLastError();
}

cudaError_t launch_bwd_finalize(const float* theta, const float* gauss, int N, float* wacc, float* dtheta,
                                cudaStream_t s) {
  if (N <= 0) return cudaSuccess;
  k_bwd_finalize<<<(N + kFinG - 1) / kFinG, kFinG, 0, s>>>(theta, gauss, N, wacc, dtheta);
  return cudaGetLastError();
}

}  // namespace gs
