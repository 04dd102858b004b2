// Learned warm start, data side: coarse backprojection, mass estimate, seed sampling, seed
// features, labels from a fitted GMM, and decoding of network outputs into raw Theta.
// None of this is in the paper (arXiv 2508.04929), which starts from random Gaussians
// (Sec. 4.1); the definitions below are the library's own and are restated in gs.h.
#include "gs_internal.cuh"

namespace gs {
namespace {

// ---------------------------------------------------------------- backprojection
// Bilinear sample of img[D][D] at (column x, row y) of the zero-extended image.
__device__ __forceinline__ float bilinear(const float* __restrict__ img, int D, float x, float y) {
  const float fx = floorf(x), fy = floorf(y);
  const int j = (int)fx, i = (int)fy;
  const float ax = x - fx, ay = y - fy;
  const bool i0 = i >= 0 && i < D, i1 = i + 1 >= 0 && i + 1 < D;
  const bool j0 = j >= 0 && j < D, j1 = j + 1 >= 0 && j + 1 < D;
  const float v00 = (i0 && j0) ? __ldg(img + (size_t)i * D + j) : 0.f;
  const float v01 = (i0 && j1) ? __ldg(img + (size_t)i * D + j + 1) : 0.f;
  const float v10 = (i1 && j0) ? __ldg(img + (size_t)(i + 1) * D + j) : 0.f;
  const float v11 = (i1 && j1) ? __ldg(img + (size_t)(i + 1) * D + j + 1) : 0.f;
  return (1.f - ay) * ((1.f - ax) * v00 + ax * v01) + ay * ((1.f - ax) * v10 + ax * v11);
}

// vol[z][y][x] = (1/B) sum_b (1/f^2) sum_{a,c<f} img_b(col + a - (f-1)/2, row + c - (f-1)/2),
// (col, row) = (p_x / h + floor(D/2), floor(D/2) - p_y / h), p = W_b r, r the voxel centre.
// One thread per voxel; the poses are read through shared memory.
__global__ void k_backproject(const float* __restrict__ images, const float* __restrict__ Wall, int B, int D,
                              float E, int Dv, int f, float* __restrict__ vol) {
  const int nv = Dv * Dv * Dv;
  const int v = blockIdx.x * blockDim.x + threadIdx.x;
  const int x = v % Dv, y = (v / Dv) % Dv, z = v / (Dv * Dv);
  const float dv = 2.f * E / (float)Dv;
  const float rx = -E + (x + 0.5f) * dv, ry = -E + (y + 0.5f) * dv, rz = -E + (z + 0.5f) * dv;
  const float inv_h = (float)D / (2.f * E), c = (float)(D / 2);
  const float half = 0.5f * (float)(f - 1);
  __shared__ float Ws[64 * 6];
  float acc = 0.f;
  for (int b0 = 0; b0 < B; b0 += 64) {
    const int nb = min(64, B - b0);
    __syncthreads();
    for (int e = threadIdx.x; e < nb * 6; e += blockDim.x) Ws[e] = Wall[(size_t)(b0 + e / 6) * 9 + e % 6];
    __syncthreads();
    if (v < nv) {
      for (int bb = 0; bb < nb; ++bb) {
        const float* W = Ws + bb * 6;
        const float px = W[0] * rx + W[1] * ry + W[2] * rz;
        const float py = W[3] * rx + W[4] * ry + W[5] * rz;
        const float col = px * inv_h + c - half, row = c - py * inv_h - half;
        const float* img = images + (size_t)(b0 + bb) * D * D;
        float s = 0.f;
        for (int a = 0; a < f; ++a)
          for (int cc = 0; cc < f; ++cc) s += bilinear(img, D, col + (float)cc, row + (float)a);
        acc += s;
      }
    }
  }
  if (v < nv) vol[v] = acc / ((float)(f * f) * (float)(B > 0 ? B : 1));
}

// ---------------------------------------------------------------- mass estimate
// acc[0] += -w_b S_b, acc[1] += w_b^2 with S_b = sum_p Y_b(p); one CTA per image.
__global__ void k_mass_sum(const float* __restrict__ images, const float* __restrict__ ctf, int D,
                           double* __restrict__ acc) {
  const int b = blockIdx.x;
  const float* img = images + (size_t)b * D * D;
  float s = 0.f;
  for (int p = threadIdx.x; p < D * D; p += blockDim.x) s += img[p];
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  __shared__ float red[32];
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int k = 0; k < (int)(blockDim.x >> 5); ++k) t += (double)red[k];
    const double w = (double)ctf[b * 5 + 3];
    atomicAdd(acc, -w * t);
    atomicAdd(acc + 1, w * w);
  }
}

__global__ void k_zero2(double* acc) {
  acc[0] = 0.0;
  acc[1] = 0.0;
}

__global__ void k_mass_final(const double* __restrict__ acc, double h2, float* __restrict__ mass) {
  *mass = acc[1] > 0.0 ? (float)(h2 * acc[0] / acc[1]) : 0.f;
}

// ---------------------------------------------------------------- seeds
// One CTA: vmax, integer weights q_v = floor(fl32(max(vol, 0) / vmax) 2^20) (all ones if
// vmax <= 0) and their running sums cdf[v] = q_0 + ... + q_v.
constexpr int kScanThreads = 1024;

__global__ void __launch_bounds__(kScanThreads) k_seed_cdf(const float* __restrict__ vol, int nv,
                                                          unsigned long long* __restrict__ cdf,
                                                          float* __restrict__ vmax_out) {
  __shared__ float rmax[32];
  __shared__ unsigned long long wsum[32];
  const int t = threadIdx.x, lane = t & 31, wid = t >> 5;
  float m = -INFINITY;
  for (int v = t; v < nv; v += blockDim.x) m = fmaxf(m, vol[v]);
  for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
  if (lane == 0) rmax[wid] = m;
  __syncthreads();
  if (t < 32) {
    float mm = rmax[t];
    for (int o = 16; o > 0; o >>= 1) mm = fmaxf(mm, __shfl_xor_sync(0xffffffffu, mm, o));
    if (t == 0) rmax[0] = mm;
  }
  __syncthreads();
  const float vmax = rmax[0];
  const bool pos = vmax > 0.f;
  const int per = (nv + kScanThreads - 1) / kScanThreads;
  const int v0 = min(nv, t * per), v1 = min(nv, v0 + per);
  unsigned long long local = 0;
  for (int v = v0; v < v1; ++v)
    local += pos ? (unsigned long long)floorf(__fdiv_rn(fmaxf(vol[v], 0.f), vmax) * 1048576.f) : 1ull;
  // exclusive scan of the per-thread sums
  unsigned long long inc = local;
  for (int o = 1; o < 32; o <<= 1) {
    const unsigned long long y = __shfl_up_sync(0xffffffffu, inc, o);
    if (lane >= o) inc += y;
  }
  if (lane == 31) wsum[wid] = inc;
  __syncthreads();
  if (t < 32) {
    unsigned long long w = wsum[t];
    for (int o = 1; o < 32; o <<= 1) {
      const unsigned long long y = __shfl_up_sync(0xffffffffu, w, o);
      if (t >= o) w += y;
    }
    wsum[t] = w;
  }
  __syncthreads();
  unsigned long long run = inc - local + (wid > 0 ? wsum[wid - 1] : 0ull);
  for (int v = v0; v < v1; ++v) {
    run += pos ? (unsigned long long)floorf(__fdiv_rn(fmaxf(vol[v], 0.f), vmax) * 1048576.f) : 1ull;
    cdf[v] = run;
  }
  if (t == 0) *vmax_out = vmax;
}

// Seed k: t = min(floor(u0 T), T - 1) in FP64, voxel = first v with cdf[v] > t, position =
// voxel centre + (u_{1,2,3} - 1/2) dv, every FP32 operation rounded in the stated order.
__global__ void k_seed_draw(const unsigned long long* __restrict__ cdf, int Dv, float E, const float* __restrict__ u,
                            int K, int* __restrict__ vox, float* __restrict__ pos) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= K) return;
  const int nv = Dv * Dv * Dv;
  const unsigned long long T = cdf[nv - 1];
  unsigned long long t = (unsigned long long)floor((double)u[k * 4] * (double)T);
  if (t > T - 1) t = T - 1;
  int lo = 0, hi = nv - 1;  // first index with cdf > t (cdf[nv - 1] = T > t)
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    if (cdf[mid] > t)
      hi = mid;
    else
      lo = mid + 1;
  }
  const int v = lo;
  if (vox) vox[k] = v;
  const int ix[3] = {v % Dv, (v / Dv) % Dv, v / (Dv * Dv)};
  const float dv = __fdiv_rn(2.f * E, (float)Dv);
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const float centre = __fadd_rn(__fmul_rn((float)ix[a] + 0.5f, dv), -E);
    const float jit = __fmul_rn(__fadd_rn(u[k * 4 + 1 + a], -0.5f), dv);
    pos[k * 3 + a] = __fadd_rn(centre, jit);
  }
}

// Trilinear sample of vol at continuous voxel coordinates (voxel centres at integers).
__device__ __forceinline__ float trilinear(const float* __restrict__ vol, int Dv, float x, float y, float z) {
  const float fx = floorf(x), fy = floorf(y), fz = floorf(z);
  const int i = (int)fx, j = (int)fy, k = (int)fz;
  const float ax = x - fx, ay = y - fy, az = z - fz;
  float v = 0.f;
#pragma unroll
  for (int dz = 0; dz < 2; ++dz)
#pragma unroll
    for (int dy = 0; dy < 2; ++dy)
#pragma unroll
      for (int dx = 0; dx < 2; ++dx) {
        const int X = i + dx, Y = j + dy, Z = k + dz;
        if (X < 0 || X >= Dv || Y < 0 || Y >= Dv || Z < 0 || Z >= Dv) continue;
        const float w = (dx ? ax : 1.f - ax) * (dy ? ay : 1.f - ay) * (dz ? az : 1.f - az);
        v = fmaf(w, __ldg(vol + ((size_t)Z * Dv + Y) * Dv + X), v);
      }
  return v;
}

// feats[K][32]: the volume at seed + {-1, 0, 1}^3 voxels over vmax (27), pos / E (3), 0, 0.
__global__ void k_seed_features(const float* __restrict__ vol, int Dv, float E, const float* __restrict__ vmax_p,
                                const float* __restrict__ pos, int K, float* __restrict__ feats) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= K) return;
  const float inv = 1.f / *vmax_p;
  const float dv = 2.f * E / (float)Dv;
  const float px = pos[k * 3], py = pos[k * 3 + 1], pz = pos[k * 3 + 2];
  const float cx = (px + E) / dv - 0.5f, cy = (py + E) / dv - 0.5f, cz = (pz + E) / dv - 0.5f;
  float* f = feats + (size_t)k * 32;
  int t = 0;
  for (int dz = -1; dz <= 1; ++dz)
    for (int dy = -1; dy <= 1; ++dy)
      for (int dx = -1; dx <= 1; ++dx) f[t++] = trilinear(vol, Dv, cx + dx, cy + dy, cz + dz) * inv;
  f[27] = px / E;
  f[28] = py / E;
  f[29] = pz / E;
  f[30] = 0.f;
  f[31] = 0.f;
}

// ---------------------------------------------------------------- labels
__device__ __forceinline__ double softplus_d(double x) { return log1p(exp(-fabs(x))) + fmax(x, 0.0); }
__device__ __forceinline__ double inv_softplus_d(double y) { return y > 30.0 ? y : log(expm1(y)); }
__device__ __forceinline__ double clampd(double x, double lo, double hi) { return fmin(fmax(x, lo), hi); }

// Rotation of the unit quaternion (w, x, y, z) (Sec. 3.3.1), row-major.
__device__ void quat_rot(double w, double x, double y, double z, double R[9]) {
  R[0] = 1 - 2 * (y * y + z * z);
  R[1] = 2 * (x * y - w * z);
  R[2] = 2 * (x * z + w * y);
  R[3] = 2 * (x * y + w * z);
  R[4] = 1 - 2 * (x * x + z * z);
  R[5] = 2 * (y * z - w * x);
  R[6] = 2 * (x * z - w * y);
  R[7] = 2 * (y * z + w * x);
  R[8] = 1 - 2 * (x * x + y * y);
}

constexpr int kAssignSeeds = 1024;

// k(g): the seed nearest to fitted centre g (FP32 squared distance ((dx dx + dy dy) + dz dz),
// each step rounded; ties to the lower seed index).  One thread per fitted Gaussian, the
// seeds staged through shared memory.
__global__ void k_assign(const float* __restrict__ theta, int N, const float* __restrict__ pos, int K,
                         int* __restrict__ assign) {
  __shared__ float sx[kAssignSeeds], sy[kAssignSeeds], sz[kAssignSeeds];
  const int g = blockIdx.x * blockDim.x + threadIdx.x;
  const bool live = g < N;
  const float mx = live ? theta[(size_t)g * 11] : 0.f, my = live ? theta[(size_t)g * 11 + 1] : 0.f,
              mz = live ? theta[(size_t)g * 11 + 2] : 0.f;
  float best = INFINITY;
  int bi = 0;
  for (int k0 = 0; k0 < K; k0 += kAssignSeeds) {
    const int nk = min(kAssignSeeds, K - k0);
    __syncthreads();
    for (int e = threadIdx.x; e < nk; e += blockDim.x) {
      sx[e] = pos[(size_t)(k0 + e) * 3];
      sy[e] = pos[(size_t)(k0 + e) * 3 + 1];
      sz[e] = pos[(size_t)(k0 + e) * 3 + 2];
    }
    __syncthreads();
    for (int e = 0; e < nk; ++e) {
      const float dx = __fsub_rn(mx, sx[e]), dy = __fsub_rn(my, sy[e]), dz = __fsub_rn(mz, sz[e]);
      const float d2 = __fadd_rn(__fadd_rn(__fmul_rn(dx, dx), __fmul_rn(dy, dy)), __fmul_rn(dz, dz));
      if (d2 < best) {
        best = d2;
        bi = k0 + e;
      }
    }
  }
  if (live) assign[g] = bi;
}

__global__ void k_zero_d(double* __restrict__ p, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    p[i] = 0.0;
}

// acc[k][0..9] += A_g (1, d, Sigma_g + d d^T upper triangle xx xy xz yy yz zz), d = mu_g - p_k,
// for k = assign[g]; FP64.
__global__ void k_merge_moments(const float* __restrict__ theta, int N, const float* __restrict__ pos,
                                const int* __restrict__ assign, double* __restrict__ acc) {
  const int g = blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= N) return;
  const float* th = theta + (size_t)g * 11;
  const int k = assign[g];
  const double A = softplus_d(th[10]);
  const double d[3] = {(double)th[0] - (double)pos[k * 3], (double)th[1] - (double)pos[k * 3 + 1],
                       (double)th[2] - (double)pos[k * 3 + 2]};
  const double qn = sqrt((double)th[6] * th[6] + (double)th[7] * th[7] + (double)th[8] * th[8] + (double)th[9] * th[9]);
  double R[9];
  quat_rot(th[6] / qn, th[7] / qn, th[8] / qn, th[9] / qn, R);
  double s2[3];
  for (int a = 0; a < 3; ++a) {
    const double sa = softplus_d(th[3 + a]);
    s2[a] = sa * sa;
  }
  double* o = acc + (size_t)k * 10;
  atomicAdd(o, A);
  for (int a = 0; a < 3; ++a) atomicAdd(o + 1 + a, A * d[a]);
  int t = 4;
  for (int i = 0; i < 3; ++i)
    for (int j = i; j < 3; ++j) {
      const double S = R[i * 3] * s2[0] * R[j * 3] + R[i * 3 + 1] * s2[1] * R[j * 3 + 1] +
                       R[i * 3 + 2] * s2[2] * R[j * 3 + 2];
      atomicAdd(o + t++, A * (S + d[i] * d[j]));
    }
}

// Labels from the merged moments: delta / dv, log-Cholesky of C / dv^2 (clamped
// log-diagonal), relative mass A_k K / M (clamped to [0, 100]); empty seeds get
// (0, 0, 0, log 1/2 x 3, 0, 0, 0, 0).
__global__ void k_merge_label(const double* __restrict__ acc, int K, int Dv, float E, const float* __restrict__ mass_p,
                              float* __restrict__ labels) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= K) return;
  const double* a = acc + (size_t)k * 10;
  float* lab = labels + (size_t)k * 10;
  const double m = a[0];
  if (!(m > 0.0)) {
    const float lh = (float)log(0.5);
    const float empty[10] = {0.f, 0.f, 0.f, lh, lh, lh, 0.f, 0.f, 0.f, 0.f};
    for (int i = 0; i < 10; ++i) lab[i] = empty[i];
    return;
  }
  const double dv = 2.0 * (double)E / (double)Dv, id2 = 1.0 / (dv * dv);
  const double d0 = a[1] / m, d1 = a[2] / m, d2 = a[3] / m;
  const double Cxx = (a[4] / m - d0 * d0) * id2, Cxy = (a[5] / m - d0 * d1) * id2, Cxz = (a[6] / m - d0 * d2) * id2;
  const double Cyy = (a[7] / m - d1 * d1) * id2, Cyz = (a[8] / m - d1 * d2) * id2, Czz = (a[9] / m - d2 * d2) * id2;
  const double L00 = sqrt(Cxx);
  const double L10 = Cxy / L00, L20 = Cxz / L00;
  const double L11 = sqrt(Cyy - L10 * L10);
  const double L21 = (Cyz - L20 * L10) / L11;
  const double L22 = sqrt(Czz - L20 * L20 - L21 * L21);
  lab[0] = (float)(d0 / dv);
  lab[1] = (float)(d1 / dv);
  lab[2] = (float)(d2 / dv);
  lab[3] = (float)clampd(log(L00), -6.0, 3.0);
  lab[4] = (float)clampd(log(L11), -6.0, 3.0);
  lab[5] = (float)clampd(log(L22), -6.0, 3.0);
  lab[6] = (float)L10;
  lab[7] = (float)L20;
  lab[8] = (float)L21;
  lab[9] = (float)clampd(m * (double)K / (double)*mass_p, 0.0, 100.0);
}

// Eigen-decomposition of a symmetric 3 x 3 matrix by cyclic Jacobi rotations (each
// rotation zeroes one off-diagonal pair exactly in exact arithmetic; a few sweeps reach
// FP64 round-off).  On return A is diagonal (eigenvalues) and V holds the eigenvectors as
// columns.
__device__ void jacobi3(double A[3][3], double V[3][3]) {
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) V[i][j] = i == j ? 1.0 : 0.0;
  for (int sweep = 0; sweep < 12; ++sweep) {
    const double off = A[0][1] * A[0][1] + A[0][2] * A[0][2] + A[1][2] * A[1][2];
    const double dia = A[0][0] * A[0][0] + A[1][1] * A[1][1] + A[2][2] * A[2][2];
    if (off <= 1e-34 * dia || off == 0.0) break;
    for (int p = 0; p < 2; ++p)
      for (int q = p + 1; q < 3; ++q) {
        const double apq = A[p][q];
        if (apq == 0.0) continue;
        const double tau = (A[q][q] - A[p][p]) / (2.0 * apq);
        const double t = (tau >= 0.0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
        const double c = 1.0 / sqrt(1.0 + t * t), s = t * c;
        // A <- J^T A J with J = I except J_pp = J_qq = c, J_pq = s, J_qp = -s
        for (int k = 0; k < 3; ++k) {
          const double akp = A[k][p], akq = A[k][q];
          A[k][p] = c * akp - s * akq;
          A[k][q] = s * akp + c * akq;
        }
        for (int k = 0; k < 3; ++k) {
          const double apk = A[p][k], aqk = A[q][k];
          A[p][k] = c * apk - s * aqk;
          A[q][k] = s * apk + c * aqk;
        }
        A[p][q] = A[q][p] = 0.0;
        for (int k = 0; k < 3; ++k) {
          const double vkp = V[k][p], vkq = V[k][q];
          V[k][p] = c * vkp - s * vkq;
          V[k][q] = s * vkp + c * vkq;
        }
      }
  }
}

// Unit quaternion (w, x, y, z) of a proper rotation R (the inverse of quat_rot): the
// largest of 4w^2, 4x^2, 4y^2, 4z^2 (from the trace and the diagonal) is taken by square
// root and the other three follow from sums and differences of off-diagonal pairs.
__device__ void rot_quat(const double R[3][3], double q[4]) {
  const double tr = R[0][0] + R[1][1] + R[2][2];
  if (tr >= R[0][0] && tr >= R[1][1] && tr >= R[2][2]) {
    const double w = 0.5 * sqrt(fmax(1.0 + tr, 0.0));
    const double f = 0.25 / w;
    q[0] = w;
    q[1] = (R[2][1] - R[1][2]) * f;
    q[2] = (R[0][2] - R[2][0]) * f;
    q[3] = (R[1][0] - R[0][1]) * f;
  } else if (R[0][0] >= R[1][1] && R[0][0] >= R[2][2]) {
    const double x = 0.5 * sqrt(fmax(1.0 + R[0][0] - R[1][1] - R[2][2], 0.0));
    const double f = 0.25 / x;
    q[0] = (R[2][1] - R[1][2]) * f;
    q[1] = x;
    q[2] = (R[0][1] + R[1][0]) * f;
    q[3] = (R[0][2] + R[2][0]) * f;
  } else if (R[1][1] >= R[2][2]) {
    const double y = 0.5 * sqrt(fmax(1.0 - R[0][0] + R[1][1] - R[2][2], 0.0));
    const double f = 0.25 / y;
    q[0] = (R[0][2] - R[2][0]) * f;
    q[1] = (R[0][1] + R[1][0]) * f;
    q[2] = y;
    q[3] = (R[1][2] + R[2][1]) * f;
  } else {
    const double z = 0.5 * sqrt(fmax(1.0 - R[0][0] - R[1][1] + R[2][2], 0.0));
    const double f = 0.25 / z;
    q[0] = (R[1][0] - R[0][1]) * f;
    q[1] = (R[0][2] + R[2][0]) * f;
    q[2] = (R[1][2] + R[2][1]) * f;
    q[3] = z;
  }
}

// theta[k] from seed k and its 10 predicted numbers (the inverse of k_merge_label's encoding).
__global__ void k_decode(const float* __restrict__ pos, const float* __restrict__ pred, int K, int Dv, float E,
                         const float* __restrict__ mass_p, float* __restrict__ theta) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= K) return;
  const float* P = pred + (size_t)k * 10;
  float* th = theta + (size_t)k * 11;
  const double dv = 2.0 * (double)E / (double)Dv;
  for (int a = 0; a < 3; ++a) th[a] = (float)((double)pos[k * 3 + a] + dv * (double)P[a]);
  const double L00 = exp(clampd(P[3], -6.0, 3.0)), L11 = exp(clampd(P[4], -6.0, 3.0)),
               L22 = exp(clampd(P[5], -6.0, 3.0));
  const double L10 = P[6], L20 = P[7], L21 = P[8];
  const double d2 = dv * dv;
  double A[3][3];
  A[0][0] = d2 * (L00 * L00);
  A[1][0] = A[0][1] = d2 * (L10 * L00);
  A[2][0] = A[0][2] = d2 * (L20 * L00);
  A[1][1] = d2 * (L10 * L10 + L11 * L11);
  A[2][1] = A[1][2] = d2 * (L20 * L10 + L21 * L11);
  A[2][2] = d2 * (L20 * L20 + L21 * L21 + L22 * L22);
  double V[3][3];
  jacobi3(A, V);
  const double det = V[0][0] * (V[1][1] * V[2][2] - V[1][2] * V[2][1]) -
                     V[0][1] * (V[1][0] * V[2][2] - V[1][2] * V[2][0]) +
                     V[0][2] * (V[1][0] * V[2][1] - V[1][1] * V[2][0]);
  if (det < 0.0)
    for (int i = 0; i < 3; ++i) V[i][2] = -V[i][2];
  for (int a = 0; a < 3; ++a) th[3 + a] = (float)inv_softplus_d(sqrt(fmax(A[a][a], 0.0)));
  double q[4];
  rot_quat(V, q);
  for (int a = 0; a < 4; ++a) th[6 + a] = (float)q[a];
  th[10] = (float)inv_softplus_d((double)*mass_p / (double)K * fmax((double)P[9], 1e-3));
}

int rc(cudaError_t e) { return e == cudaSuccess ? GS_OK : GS_ECUDA; }

}  // namespace
}  // namespace gs

using namespace gs;

extern "C" {

int gs_backproject(const float* images, const float* W, int B, int D, float E, int Dv, float* vol,
                   gs_stream_t stream) {
  if (B < 0 || D < 1 || D > 4096 || Dv < 1 || Dv > 256 || !(E > 0.f) || !vol) return GS_EINVAL;
  if (B > 0 && (!images || !W)) return GS_EINVAL;
  const int nv = Dv * Dv * Dv;
  const int f = D / Dv > 1 ? D / Dv : 1;
  k_backproject<<<(nv + 255) / 256, 256, 0, (cudaStream_t)stream>>>(images, W, B, D, E, Dv, f, vol);
  return rc(cudaGetLastError());
}

int gs_mass_estimate(const float* images, const float* ctf, int B, int D, float E, double* scratch, float* mass,
                     gs_stream_t stream) {
  if (B < 1 || D < 1 || !(E > 0.f) || !images || !ctf || !scratch || !mass) return GS_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  const double h = 2.0 * (double)E / (double)D;
  k_zero2<<<1, 1, 0, s>>>(scratch);
  k_mass_sum<<<B, 256, 0, s>>>(images, ctf, D, scratch);
  k_mass_final<<<1, 1, 0, s>>>(scratch, h * h, mass);
  return rc(cudaGetLastError());
}

int gs_seed_sample(const float* vol, int Dv, float E, const float* u, int K, unsigned long long* cdf, float* vmax,
                   int* voxel, float* pos, gs_stream_t stream) {
  if (Dv < 1 || Dv > 256 || K < 0 || !(E > 0.f) || !vol || !cdf || !vmax) return GS_EINVAL;
  if (K > 0 && (!u || !pos)) return GS_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  const int nv = Dv * Dv * Dv;
  k_seed_cdf<<<1, kScanThreads, 0, s>>>(vol, nv, cdf, vmax);
  if (K > 0) k_seed_draw<<<(K + 127) / 128, 128, 0, s>>>(cdf, Dv, E, u, K, voxel, pos);
  return rc(cudaGetLastError());
}

int gs_seed_features(const float* vol, int Dv, float E, const float* vmax, const float* pos, int K, float* feats,
                     gs_stream_t stream) {
  if (Dv < 1 || K < 0 || !(E > 0.f)) return GS_EINVAL;
  if (K == 0) return GS_OK;
  if (!vol || !vmax || !pos || !feats) return GS_EINVAL;
  k_seed_features<<<(K + 127) / 128, 128, 0, (cudaStream_t)stream>>>(vol, Dv, E, vmax, pos, K, feats);
  return rc(cudaGetLastError());
}

int gs_merge_labels(const float* pos, int K, const float* theta_fit, int N, int Dv, float E, const float* mass,
                    int* assign, double* moments, float* labels, gs_stream_t stream) {
  if (K < 1 || N < 0 || Dv < 1 || !(E > 0.f)) return GS_EINVAL;
  if (!pos || !mass || !assign || !moments || !labels || (N > 0 && !theta_fit)) return GS_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  const long long nm = (long long)K * 10;
  long long zb = (nm + 255) / 256;
  if (zb > num_sms() * 8) zb = num_sms() * 8;
  k_zero_d<<<(int)zb, 256, 0, s>>>(moments, nm);
  if (N > 0) {
    k_assign<<<(N + 127) / 128, 128, 0, s>>>(theta_fit, N, pos, K, assign);
    k_merge_moments<<<(N + 127) / 128, 128, 0, s>>>(theta_fit, N, pos, assign, moments);
  }
  k_merge_label<<<(K + 127) / 128, 128, 0, s>>>(moments, K, Dv, E, mass, labels);
  return rc(cudaGetLastError());
}

int gs_decode_seeds(const float* pos, const float* pred, int K, int Dv, float E, const float* mass, float* theta,
                    gs_stream_t stream) {
  if (K < 0 || Dv < 1 || !(E > 0.f)) return GS_EINVAL;
  if (K == 0) return GS_OK;
  if (!pos || !pred || !mass || !theta) return GS_EINVAL;
  k_decode<<<(K + 127) / 128, 128, 0, (cudaStream_t)stream>>>(pos, pred, K, Dv, E, mass, theta);
  return rc(cudaGetLastError());
}

}  // extern "C"
