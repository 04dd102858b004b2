// SumSplats (Algorithm 2; App. A.2 Eq. 15) and its backward (App. A.2 Eqs. 16-21).
//
// One CTA per (tile, particle).  The tile (T x T pixels) is split into 8 x 8 regions, one
// per warp; lane l owns the two horizontally adjacent pixels (row l / 4, columns
// 2 (l % 4) and 2 (l % 4) + 1) of its warp's region and keeps them in registers.  The
// tile's Gaussian records are staged through shared memory in chunks; each warp skips the
// records whose support box misses its region (a warp-uniform test), so that the executed
// work is that of 8 x 8 tiles whatever the binning tile size.
//
// Forward: Q(p) = sum_g w_g 2^(ca dx^2 + cb dx dy + cc dy^2) over the g whose box holds p
// (one ex2.approx per Gaussian-pixel).
// Backward: per (particle, Gaussian) the six sums of Gc = dL/dQ(p) * contribution(p):
// S0, Sx, Sy, Sxx, Sxy, Syy (weights 1, dx, dy, dx^2, dx dy, dy^2), reduced across the
// warp by a transposing butterfly (9 shuffles for 8 slots), across the CTA's warps in
// shared memory, and written with one vector atomic pair per (tile, Gaussian).  The
// per-Gaussian finalize kernel turns them into dL/dtheta, summing over particles.
#include "gs_internal.cuh"

namespace gs {
namespace {

struct RegionCtx {
  int i, j0;        // pixel row, first of the lane's two columns
  int X0, Y0;       // warp region origin
};

__device__ __forceinline__ RegionCtx region_ctx(int T, int tile_x, int tile_y) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int rpt = T >> 3;  // regions per tile side
  RegionCtx c;
  c.X0 = tile_x * T + (warp % rpt) * 8;
  c.Y0 = tile_y * T + (warp / rpt) * 8;
  c.i = c.Y0 + (lane >> 2);
  c.j0 = c.X0 + (lane & 3) * 2;
  return c;
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

__global__ void k_render_fwd(const gs_record* __restrict__ proj, int N, const uint32_t* __restrict__ pair_gauss,
                             const uint32_t* __restrict__ ranges, int D, int T, int ntx, int chunk,
                             float* __restrict__ Q) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  gs_record* rec = reinterpret_cast<gs_record*>(smem_raw);
  const int t = blockIdx.x, b = blockIdx.y, Tn = ntx * ntx;
  const RegionCtx c = region_ctx(T, t % ntx, t / ntx);
  const uint32_t start = ranges[((size_t)b * Tn + t) * 2], end = ranges[((size_t)b * Tn + t) * 2 + 1];
  const size_t pbase = (size_t)b * N;
  const float fi = (float)c.i, fj0 = (float)c.j0;
  float acc0 = 0.f, acc1 = 0.f;
  for (uint32_t base = start; base < end; base += chunk) {
    const int n = (int)min((uint32_t)chunk, end - base);
    __syncthreads();
    stage_chunk(rec, proj, pbase, pair_gauss, base, n);
    __syncthreads();
    for (int k = 0; k < n; ++k) {
      const float4 r0 = reinterpret_cast<const float4*>(rec + k)[0];
      const float4 r1 = reinterpret_cast<const float4*>(rec + k)[1];
      const int bx = __float_as_int(r1.z), by = __float_as_int(r1.w);
      const int x0 = (int)(int16_t)(bx & 0xffff), x1 = bx >> 16;
      const int y0 = (int)(int16_t)(by & 0xffff), y1 = by >> 16;
      if (x1 < c.X0 || x0 > c.X0 + 7 || y1 < c.Y0 || y0 > c.Y0 + 7) continue;  // warp-uniform
      const float cx = r0.x, cy = r0.y, ca = r0.z, cb = r0.w, cc = r1.x, w = r1.y;
      const float dy = fi - cy;
      const float dx0 = fj0 - cx, dx1 = dx0 + 1.f;
      const bool rowin = c.i >= y0 && c.i <= y1;
      const bool in0 = rowin && c.j0 >= x0 && c.j0 <= x1;
      const bool in1 = rowin && c.j0 + 1 >= x0 && c.j0 + 1 <= x1;
      const float cbdy = cb * dy, ccdy2 = cc * dy * dy;
      const float e0 = ex2_approx(fmaf(fmaf(ca, dx0, cbdy), dx0, ccdy2));
      const float e1 = ex2_approx(fmaf(fmaf(ca, dx1, cbdy), dx1, ccdy2));
      acc0 = fmaf(in0 ? w : 0.f, e0, acc0);
      acc1 = fmaf(in1 ? w : 0.f, e1, acc1);
    }
  }
  if (c.i < D) {
    float* row = Q + ((size_t)b * D + c.i) * D;
    if (c.j0 < D) row[c.j0] = acc0;
    if (c.j0 + 1 < D) row[c.j0 + 1] = acc1;
  }
}

// Transposing butterfly: on entry each lane holds v[0..7]; on exit lane l holds, in v[0],
// the warp sum of slot ((l >> 4) & 1) * 4 + ((l >> 3) & 1) * 2 + ((l >> 2) & 1).
__device__ __forceinline__ float warp_transpose_reduce8(float v[8]) {
  const int lane = threadIdx.x & 31;
  const bool u16 = lane & 16, u8 = lane & 8, u4 = lane & 4;
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    float send = u16 ? v[k] : v[k + 4];
    float keep = u16 ? v[k + 4] : v[k];
    v[k] = keep + __shfl_xor_sync(0xffffffffu, send, 16);
  }
#pragma unroll
  for (int k = 0; k < 2; ++k) {
    float send = u8 ? v[k] : v[k + 2];
    float keep = u8 ? v[k + 2] : v[k];
    v[k] = keep + __shfl_xor_sync(0xffffffffu, send, 8);
  }
  {
    float send = u4 ? v[0] : v[1];
    float keep = u4 ? v[1] : v[0];
    v[0] = keep + __shfl_xor_sync(0xffffffffu, send, 4);
  }
  v[0] += __shfl_xor_sync(0xffffffffu, v[0], 2);
  v[0] += __shfl_xor_sync(0xffffffffu, v[0], 1);
  return v[0];
}

__global__ void k_render_bwd(const gs_record* __restrict__ proj, int N, const uint32_t* __restrict__ pair_gauss,
                             const uint32_t* __restrict__ ranges, int D, int T, int ntx, int chunk,
                             const float* __restrict__ dLdQ, float* __restrict__ gacc) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  gs_record* rec = reinterpret_cast<gs_record*>(smem_raw);
  float* gsum = reinterpret_cast<float*>(smem_raw + sizeof(gs_record) * chunk);  // [chunk][6]
  const int t = blockIdx.x, b = blockIdx.y, Tn = ntx * ntx;
  const int lane = threadIdx.x & 31;
  const RegionCtx c = region_ctx(T, t % ntx, t / ntx);
  const uint32_t start = ranges[((size_t)b * Tn + t) * 2], end = ranges[((size_t)b * Tn + t) * 2 + 1];
  const size_t pbase = (size_t)b * N;
  const float fi = (float)c.i, fj0 = (float)c.j0;
  float g0 = 0.f, g1 = 0.f;
  if (c.i < D) {
    const float* row = dLdQ + ((size_t)b * D + c.i) * D;
    if (c.j0 < D) g0 = row[c.j0];
    if (c.j0 + 1 < D) g1 = row[c.j0 + 1];
  }
  const int slot = ((lane >> 4) & 1) * 4 + ((lane >> 3) & 1) * 2 + ((lane >> 2) & 1);
  for (uint32_t base = start; base < end; base += chunk) {
    const int n = (int)min((uint32_t)chunk, end - base);
    __syncthreads();
    stage_chunk(rec, proj, pbase, pair_gauss, base, n);
    for (int k = threadIdx.x; k < n * 6; k += blockDim.x) gsum[k] = 0.f;
    __syncthreads();
    for (int k = 0; k < n; ++k) {
      const float4 r0 = reinterpret_cast<const float4*>(rec + k)[0];
      const float4 r1 = reinterpret_cast<const float4*>(rec + k)[1];
      const int bx = __float_as_int(r1.z), by = __float_as_int(r1.w);
      const int x0 = (int)(int16_t)(bx & 0xffff), x1 = bx >> 16;
      const int y0 = (int)(int16_t)(by & 0xffff), y1 = by >> 16;
      if (x1 < c.X0 || x0 > c.X0 + 7 || y1 < c.Y0 || y0 > c.Y0 + 7) continue;  // warp-uniform
      const float cx = r0.x, cy = r0.y, ca = r0.z, cb = r0.w, cc = r1.x, w = r1.y;
      const float dy = fi - cy;
      const float dx0 = fj0 - cx, dx1 = dx0 + 1.f;
      const bool rowin = c.i >= y0 && c.i <= y1;
      const bool in0 = rowin && c.j0 >= x0 && c.j0 <= x1;
      const bool in1 = rowin && c.j0 + 1 >= x0 && c.j0 + 1 <= x1;
      const float cbdy = cb * dy, ccdy2 = cc * dy * dy;
      const float e0 = ex2_approx(fmaf(fmaf(ca, dx0, cbdy), dx0, ccdy2));
      const float e1 = ex2_approx(fmaf(fmaf(ca, dx1, cbdy), dx1, ccdy2));
      const float G0 = in0 ? g0 * w * e0 : 0.f;
      const float G1 = in1 ? g1 * w * e1 : 0.f;
      float v[8];
      v[0] = G0 + G1;                       // S0
      v[1] = fmaf(G0, dx0, G1 * dx1);       // Sx
      v[2] = v[0] * dy;                     // Sy
      v[3] = fmaf(G0 * dx0, dx0, G1 * dx1 * dx1);  // Sxx
      v[4] = v[1] * dy;                     // Sxy
      v[5] = v[2] * dy;                     // Syy
      v[6] = 0.f;
      v[7] = 0.f;
      const float s = warp_transpose_reduce8(v);
      if ((lane & 3) == 0 && slot < 6) atomicAdd(&gsum[k * 6 + slot], s);
    }
    __syncthreads();
    for (int k = threadIdx.x; k < n; k += blockDim.x) {
      const float* q = gsum + k * 6;
      if (q[0] == 0.f && q[1] == 0.f && q[2] == 0.f && q[3] == 0.f && q[4] == 0.f && q[5] == 0.f) continue;
      const uint32_t g = pair_gauss[base + k];
      float* dst = gacc + (pbase + g) * kGradStride;
      red_add_v4(dst, q[0], q[1], q[2], q[3]);
      red_add_v2(dst + 4, q[4], q[5]);
    }
  }
}

// Per Gaussian: sum over particles of the per-(particle, Gaussian) gradients, then the
// chain to theta.  Re-zeroes the partials it consumed.
__global__ void k_bwd_finalize(const float* __restrict__ theta, const float* __restrict__ gauss, int N,
                               const float* __restrict__ Wall, int B, int D, float E,
                               float* __restrict__ gacc, float* __restrict__ dtheta) {
  __shared__ float Ws[256 * 9];
  const int g = blockIdx.x * blockDim.x + threadIdx.x;
  const bool live = g < N;
  const float* G = gauss + (size_t)(live ? g : 0) * kGaussStride;
  float M[9], s[3];
#pragma unroll
  for (int k = 0; k < 9; ++k) M[k] = G[kM + k];
  s[0] = G[kS]; s[1] = G[kS + 1]; s[2] = G[kS + 2];
  const float A = G[kA], sprod = G[kSprod];
  const bool bad = G[kBad] != 0.f;
  const float h = 2.f * E / (float)D;
  float gA = 0.f, gmu[3] = {0.f, 0.f, 0.f}, gS[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};  // 00 01 02 11 12 22
  for (int b0 = 0; b0 < B; b0 += 256) {
    const int nb = min(256, B - b0);
    __syncthreads();
    for (int k = threadIdx.x; k < nb * 9; k += blockDim.x) Ws[k] = Wall[(size_t)b0 * 9 + k];
    __syncthreads();
    if (!live || bad) continue;
    for (int bb = 0; bb < nb; ++bb) {
      float* acc = gacc + ((size_t)(b0 + bb) * N + g) * kGradStride;
      const float4 a = *reinterpret_cast<const float4*>(acc);
      const float2 a2 = *reinterpret_cast<const float2*>(acc + 4);
      if (a.x == 0.f && a.y == 0.f && a.z == 0.f && a.w == 0.f && a2.x == 0.f && a2.y == 0.f) continue;
      *reinterpret_cast<float4*>(acc) = make_float4(0.f, 0.f, 0.f, 0.f);
      *reinterpret_cast<float2*>(acc + 4) = make_float2(0.f, 0.f);
      const float* W = Ws + bb * 9;
      float V[2][3];
#pragma unroll
      for (int r = 0; r < 2; ++r)
#pragma unroll
        for (int m = 0; m < 3; ++m) V[r][m] = W[3 * r] * M[m] + W[3 * r + 1] * M[3 + m] + W[3 * r + 2] * M[6 + m];
      const float sxx = V[0][0] * V[0][0] + V[0][1] * V[0][1] + V[0][2] * V[0][2];
      const float syy = V[1][0] * V[1][0] + V[1][1] * V[1][1] + V[1][2] * V[1][2];
      const float sxy = V[0][0] * V[1][0] + V[0][1] * V[1][1] + V[0][2] * V[1][2];
      const float t0 = (W[6] * M[0] + W[7] * M[3] + W[8] * M[6]) / (s[0] * s[0]);
      const float t1 = (W[6] * M[1] + W[7] * M[4] + W[8] * M[7]) / (s[1] * s[1]);
      const float t2 = (W[6] * M[2] + W[7] * M[5] + W[8] * M[8]) / (s[2] * s[2]);
      const float sd = sprod * sqrtf(t0 * t0 + t1 * t1 + t2 * t2);
      const float idet = 1.f / (sd * sd);
      const float pxx = syy * idet, pxy = -sxy * idet, pyy = sxx * idet;  // P = Sigma_tilde^-1
      const float S0 = a.x, Sx = a.y, Sy = a.z, Sxx = a.w, Sxy = a2.x, Syy = a2.y;
      // Eq. 17: dL/dA = sum dL/dQ G_tilde = S0 / A
      gA += S0 / A;
      // Eq. 18: grad_mu_tilde = sum Gc P d, d = (h dx, -h dy)
      const float gmx = h * (pxx * Sx - pxy * Sy);
      const float gmy = h * (pxy * Sx - pyy * Sy);
      // Eq. 20: grad_P = 1/2 sum Gc (Sigma_tilde - d d^T), then grad_Sigma_tilde = -P grad_P P
      const float h2 = h * h;
      const float u = 0.5f * (S0 * sxx - h2 * Sxx);
      const float vv = 0.5f * (S0 * sxy + h2 * Sxy);
      const float z = 0.5f * (S0 * syy - h2 * Syy);
      const float m00 = u * pxx + vv * pxy, m01 = u * pxy + vv * pyy;
      const float m10 = vv * pxx + z * pxy, m11 = vv * pxy + z * pyy;
      const float gxx = -(pxx * m00 + pxy * m10);
      const float gxy = -(pxx * m01 + pxy * m11);
      const float gyy = -(pxy * m01 + pyy * m11);
      // mu_dot = W mu: grad_mu = W^T [grad_mu_tilde; 0]; Sigma_dot = W Sigma W^T with the
      // Eq. 21 embedding: grad_Sigma = W_{2x3}^T grad_Sigma_tilde W_{2x3}
#pragma unroll
      for (int k = 0; k < 3; ++k) gmu[k] += W[k] * gmx + W[3 + k] * gmy;
      const int kk[6] = {0, 0, 0, 1, 1, 2}, ll[6] = {0, 1, 2, 1, 2, 2};
#pragma unroll
      for (int e = 0; e < 6; ++e) {
        const float ak = W[kk[e]], bk = W[3 + kk[e]], al = W[ll[e]], bl = W[3 + ll[e]];
        gS[e] += ak * gxx * al + ak * gxy * bl + bk * gxy * al + bk * gyy * bl;
      }
    }
  }
  if (!live || bad) return;
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

static int render_threads(int T) { return (T / 8) * (T / 8) * 32; }

cudaError_t launch_render_fwd(const gs_config& cfg, const gs_record* proj, int N, const uint32_t* pair_gauss,
                              const uint32_t* ranges, int B, float* Q, cudaStream_t s) {
  if (B <= 0) return cudaSuccess;
  const int ntx = (cfg.D + cfg.tile - 1) / cfg.tile;
  dim3 grid(ntx * ntx, B);
  size_t sm = sizeof(gs_record) * cfg.chunk;
  if (sm > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(k_render_fwd, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
  }
  k_render_fwd<<<grid, render_threads(cfg.tile), sm, s>>>(proj, N, pair_gauss, ranges, cfg.D, cfg.tile, ntx,
                                                         cfg.chunk, Q);
  return cudaGetLastError();
}

cudaError_t launch_render_bwd(const gs_config& cfg, const gs_record* proj, int N, const uint32_t* pair_gauss,
                              const uint32_t* ranges, int B, const float* dLdQ, float* gacc, cudaStream_t s) {
  if (B <= 0) return cudaSuccess;
  const int ntx = (cfg.D + cfg.tile - 1) / cfg.tile;
  dim3 grid(ntx * ntx, B);
  size_t sm = (sizeof(gs_record) + 6 * sizeof(float)) * cfg.chunk;
  if (sm > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(k_render_bwd, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
  }
  k_render_bwd<<<grid, render_threads(cfg.tile), sm, s>>>(proj, N, pair_gauss, ranges, cfg.D, cfg.tile, ntx,
                                                         cfg.chunk, dLdQ, gacc);
  return cudaGetLastError();
}

cudaError_t launch_bwd_finalize(const gs_config& cfg, const float* theta, const float* gauss, int N,
                                const float* W, int B, float* gacc, float* dtheta, cudaStream_t s) {
  if (N <= 0) return cudaSuccess;
  k_bwd_finalize<<<(N + 255) / 256, 256, 0, s>>>(theta, gauss, N, W, B, cfg.D, cfg.E, gacc, dtheta);
  return cudaGetLastError();
}

}  // namespace gs
