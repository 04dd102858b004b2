/*
 * gs.h -- C-ABI of the B300 (sm_103a) cryoSplat orthographic splatting path.
 *
 * The operations follow arXiv 2508.04929 ("CryoSplat: Gaussian Splatting for Cryo-EM
 * Homogeneous Reconstruction"): Algorithm 2 (Rasterize), App. A.2 Eqs. 12-21 (projection,
 * FFT-aligned pixel grid, CTF, gradients), Sec. 3.3.5 (loss) and Sec. 4.1 (Adam).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * - All array pointers are DEVICE pointers owned by the caller, except where a comment
 *   says "host".  The library never allocates device memory: scratch space is the
 *   caller's workspace (gs_workspace_size).  cuFFT plans are created by gs_fft_create.
 * - Every call is asynchronous and stream-ordered on `stream` (cudaStream_t; NULL is the
 *   legacy default stream).  Launch failures are reported as GS_ECUDA.  Conditions found
 *   on the device (non-finite parameters, pair-buffer overflow) are recorded as bits of a
 *   status word kept at the start of the workspace; read it with gs_read_status.
 * - Layouts are row-major and dense.  Floating point is FP32.  Model units: the box spans
 *   [-E, E] (E = 0.5), so one pixel is h = 2E / D.
 * - theta[N * 11] per Gaussian = [mu_x, mu_y, mu_z, s_x, s_y, s_z, q_w, q_x, q_y, q_z, A]
 *   in raw form: A = softplus(theta[10]), s = softplus(theta[3..5]), q normalized
 *   (Sec. 3.3.1).  W[B * 9] is the row-major pose of each particle, mu_dot = W mu
 *   (Sec. 3.3.2 Eq. 6; no in-plane translation on this path, Sec. 4.1).
 * - Pixel (i, j) of a D x D image samples the continuous image at
 *   ((j - floor(D/2)) h, -(i - floor(D/2)) h): App. A.2 Eq. 13 (FFT-aligned origin, y flip).
 * - Support: Gaussian g contributes to the pixels of its clipped k-sigma box
 *   [ceil(cx - rx), floor(cx + rx)] x [ceil(cy - ry), floor(cy + ry)] with
 *   rx = k sqrt(Sigma~xx) / h, ry = k sqrt(Sigma~yy) / h (k = cutoff_sigma).  The box is
 *   computed in FP32 with a fixed sequence of correctly rounded operations (documented in
 *   gs_project) so that it is reproducible; it does not depend on the tile size.
 *
 * Return codes: GS_OK on success; GS_EINVAL for a bad argument (null pointer with a
 * non-zero size, misaligned pointer, size out of range, unsupported tile); GS_ENOSPC when
 * a caller-provided buffer is too small (the needed size is reported where an argument
 * allows it); GS_ECUDA when a CUDA or cuFFT call fails.
 */
#ifndef GS_H_
#define GS_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st* gs_stream_t; /* = cudaStream_t */

enum {
  GS_OK = 0,
  GS_EINVAL = 1,
  GS_ENOSPC = 2,
  GS_ECUDA = 3,
  GS_ECAPTURE = 4, /* gs_bin_sort_noalloc: first call on a device made on a capturing stream */
};

/* Bits of the device status word (gs_read_status). */
enum {
  GS_STATUS_NONFINITE = 1, /* a Gaussian had a non-finite parameter or box; it was skipped */
  GS_STATUS_OVERFLOW = 2,  /* more tile pairs than pair_capacity; extra pairs were dropped */
};

typedef struct gs_config {
  int D;              /* image side in pixels, 1..4096 */
  float E;            /* half extent of the box in model units (the paper uses 0.5) */
  int tile;           /* tile side in pixels: 8, 16 or 32 (App. C.2 uses 16) */
  int chunk;          /* Gaussian records staged per shared-memory chunk: 32..512, multiple of 32 */
  float cutoff_sigma; /* k of the k-sigma support box (3) */
  int reduction;      /* loss per image: 0 = sum of squares (Sec. 3.3.5), 1 = mean over pixels */
} gs_config;

/* Projected record of one (particle, Gaussian) pair: 32 bytes, 16-byte aligned.  With
 * dx = j - cx, dy = i - cy the offsets of pixel (i, j) from the splat centre (pixel units) and
 * Sigma~ the 2 x 2 covariance in pixel units (Sxy its world off-diagonal entry), the splat
 * value there is App. A.2 Eq. 12's normalized 2-D Gaussian w exp(-1/2 d^T Sigma~^-1 d),
 * w = A / (2 pi sqrt(det Sigma~)) in model units, stored in one of two forms:
 *   c1 < 0 (well-conditioned): w 2^(c1 dx^2 + c2 dx dy + c3 dy^2), the expanded form with
 *     (c1, c2, c3) = -log2(e) / (2 det) (Syy, 2 Sxy, Sxx), and c4 = w;
 *   c1 > 0 (ill-conditioned: c1 > 3, a conditional standard deviation below 0.49 px, or
 *     (Sxx + Syy)^2 > 100 det, a condition number above about 100):
 *     2^(c4 - c1 (dx + c2 dy)^2 + c3 dy^2), the completed square with c1 = log2(e)/2 Syy/det,
 *     c2 = Sxy/Syy, c3 = -log2(e)/2 / Syy, and c4 = log2 w; its centre is refined by the low
 *     parts that follow the box plane (gs_proj_size).
 * [x0, x1] x [y0, y1] is the clipped support box (empty when x0 > x1). */
typedef struct gs_record {
  float cx, cy;
  float c1, c2, c3, c4;
  int16_t x0, x1, y0, y1;
} gs_record;

/* Opaque pair of batched cuFFT plans (R2C and C2R over B images of D x D). */
typedef struct gs_fft {
  int r2c;           /* cufftHandle: 2-D R2C over B images */
  int c2r;           /* cufftHandle: 2-D C2R over B images */
  int D;
  int B;
  size_t work_bytes; /* cuFFT work area needed (placed inside the gs workspace) */
  int r2c_rows;      /* reserved, 0 (the D = 256 row transforms are the library's own kernels) */
  int c2r_rows;      /* reserved, 0 */
} gs_fft;

/* ---------------------------------------------------------------------------------------
 * Sizes and set-up
 * ------------------------------------------------------------------------------------- */

/* Number of tiles per image, ceil(D / tile)^2, into *n.  GS_EINVAL on a bad config. */
int gs_tiles_per_image(const gs_config* cfg, int* n);

/* Bytes of the projection buffer that gs_project fills for B particles and N Gaussians:
 * the B*N records (gs_record, particle-major), then, at byte offset 32*B*N, the B*N
 * support boxes again as int32 pairs {x0 | x1 << 16, y0 | y1 << 16} (8 bytes each,
 * particle-major, the same values as the records' boxes), then, at byte offset 40*B*N, B*N
 * float pairs (cx_lo, cy_lo): for an ill-conditioned record (c1 > 0, see gs_record), the
 * centre's low parts -- the centre computed in FP64 from the FP32 pose and mean, minus
 * (cx, cy) -- which the render calls add to the record's centre; for other records that
 * pair is not written.  The binning
 * calls read the boxes from the box plane, a quarter of the bytes of the records.
 * GS_EINVAL if B or N is negative. */
int gs_proj_size(int B, int N, size_t* bytes);

/* Workspace bytes for batches of up to B particles and N Gaussians with the given cuFFT
 * work area (gs_fft.work_bytes, 0 if gs_apply_ctf is not used).  The workspace holds the
 * status word, the activated Gaussians, the binning histograms, the per-Gaussian
 * gradient accumulator, two batches of half spectra and the cuFFT work area.  It must be
 * 256-byte aligned; its contents need no initialization. */
int gs_workspace_size(const gs_config* cfg, int B, int N, size_t fft_work_bytes, size_t* bytes);

/* Create batched cuFFT plans for B images of D x D (automatic work-area allocation off;
 * the work area lives in the gs workspace).  Host-side call; cuFFT allocates its own plan
 * state.  Release with gs_fft_destroy. */
int gs_fft_create(int D, int B, gs_fft* fft);
int gs_fft_destroy(gs_fft* fft);

/* Copy the device status word to *status (host) and wait for `stream`.  If `clear` is
 * non-zero the word is reset to 0 afterwards (stream-ordered). */
int gs_read_status(const void* ws, gs_stream_t stream, int clear, int* status);

/* Reset the status word to 0 (stream-ordered, asynchronous). */
int gs_clear_status(void* ws, gs_stream_t stream);

/* ---------------------------------------------------------------------------------------
 * The path (Algorithm 1 body: Rasterize -> ApplyCTF -> Loss -> backprop -> Adam)
 * ------------------------------------------------------------------------------------- */

/* BuildGaussians + ViewingTransform + Projection (Algorithm 2; Sec. 3.3.1-3.3.3, Eqs. 5, 6,
 * 8; App. A.2 Eqs. 12-13).
 * theta[N*11] raw parameters, W[B*9] poses -> proj: the B*N records (gs_record,
 * particle-major: proj[b*N + g]) followed by the box plane (gs_proj_size(B, N) bytes in
 * all).  Also fills the activated-Gaussian table in `ws` used by gs_render_bwd.
 * The support box is computed in FP32 in this order, every operation correctly rounded:
 *   s = fp32(softplus(s_raw) in FP64);  n = sqrt(((qw*qw + qx*qx) + qy*qy) + qz*qz);
 *   (w,x,y,z) = q / n;  R from (w,x,y,z) with the pairwise products formed first,
 *   e.g. R00 = 1 - 2*(y*y + z*z), R01 = 2*(x*y - w*z), R02 = 2*(x*z + w*y), ...;
 *   M[k][m] = R[k][m] * s[m];  V[a][m] = (W[a][0]*M[0][m] + W[a][1]*M[1][m]) + W[a][2]*M[2][m];
 *   Sxx = (V00^2 + V01^2) + V02^2;  Syy = (V10^2 + V11^2) + V12^2;
 *   mx = (W00 mu_x + W01 mu_y) + W02 mu_z;  my = (W10 mu_x + W11 mu_y) + W12 mu_z;
 *   inv_h = D / (2E);  cx = mx * inv_h + floor(D/2);  cy = floor(D/2) - my * inv_h;
 *   rx = k * (sqrt(Sxx) * inv_h);  ry = k * (sqrt(Syy) * inv_h).
 * Gaussians with a non-finite parameter or box get an empty box and set
 * GS_STATUS_NONFINITE.  Pointers: theta, W 4-byte aligned; proj 16-byte aligned. */
int gs_project(const gs_config* cfg, const float* theta, int N, const float* W, int B,
               gs_record* proj, void* ws, size_t ws_bytes, gs_stream_t stream);

/* CreateTiles + DuplicateWithKeys + SortByKeys + IdentifyTileRanges (Algorithm 2).
 * Instantiates every Gaussian in every tile its support box touches and orders the
 * instances by the key (particle, tile, Gaussian): a stable counting sort on the tile
 * digit of Gaussians emitted in index order, i.e. the last pass of an LSD radix sort
 * keyed on (tile, Gaussian).
 * Outputs: pair_gauss[pair_capacity] Gaussian index of every instance;
 * tile_ranges[B * T * 2] absolute [start, end) of each (particle, tile) in pair_gauss
 * (T = gs_tiles_per_image); *n_pairs (device uint32) the number of instances needed.
 * If that exceeds pair_capacity the extra instances are dropped, the ranges are clipped
 * to pair_capacity and GS_STATUS_OVERFLOW is set.  Requires ceil(D/tile) <= 64 and
 * N * T < 2^32 (GS_EINVAL otherwise).  proj is gs_project's whole output for the same B
 * and N: the supports are read from its box plane. */
int gs_bin_sort(const gs_config* cfg, const gs_record* proj, int B, int N, void* ws,
                size_t ws_bytes, uint32_t* pair_gauss, size_t pair_capacity,
                uint32_t* tile_ranges, uint32_t* n_pairs, gs_stream_t stream);

/* SumSplats (Algorithm 2; App. A.2 Eq. 15 at the Eq. 13 pixel centres): additive
 * accumulation, no alpha compositing (Sec. 3.3.4).
 * Q[B * D * D] = sum over each pixel's tile list of w * 2^(quadratic) inside the support
 * box.  Every pixel is written (zero where nothing contributes). */
int gs_render_fwd(const gs_config* cfg, const gs_record* proj, int N, const uint32_t* pair_gauss,
                  const uint32_t* tile_ranges, int B, float* Q, gs_stream_t stream);

/* ApplyCTF (App. A.2 Eq. 14): out = F^-1(H_hat . F(in)) per image, with
 * H_hat(k) = -(sqrt(1 - w^2) sin chi + w cos chi), chi = pi lambda df |k|^2 -
 * (pi/2) Cs lambda^3 |k|^4 and the relativistic electron wavelength lambda.
 * ctf[B * 5] per image = (defocus_A, kV, Cs_mm, amplitude_contrast, pixel_size_A).
 * H_hat is real and even, so the operator is self-adjoint: the same call applies the
 * adjoint for the backward pass.  in and out may not alias.  Uses cuFFT (fft must have
 * been created for this D and B) and the spectrum / work area inside ws. */
int gs_apply_ctf(const gs_config* cfg, const float* in, const float* ctf, int B, float* out,
                 const gs_fft* fft, void* ws, size_t ws_bytes, gs_stream_t stream);

/* Loss (Sec. 3.3.5): loss[b] = sum_p (X - Y)^2 (reduction 0) or its mean over pixels
 * (reduction 1); dLdX = dloss[b]/dX (= 2 (X - Y) times the reduction scale).
 * dLdX may be NULL (loss only). */
int gs_loss(const gs_config* cfg, const float* X, const float* Y, int B, float* loss,
            float* dLdX, gs_stream_t stream);

/* ApplyCTF, Loss and the adjoint ApplyCTF of a training step in one call (App. A.2 Eq. 14;
 * Sec. 3.3.5), for callers that need loss[b] and dL/dQ but not X.  With the unnormalized
 * R2C spectra Q_hat, Y_hat and Z = H_hat Q_hat - Y_hat (the spectrum of X - Y, H_hat being
 * real and even), Parseval's identity gives loss[b] = s * sum over the full spectrum
 * |Z|^2 / D^2 (s = 1 for reduction 0, 1 / D^2 for reduction 1), and
 * dLdQ = C2R(2 s H_hat Z) / D^2 is the adjoint CTF of dL/dX = 2 s (X - Y): the values of
 * gs_apply_ctf + gs_loss + gs_apply_ctf up to FP32 rounding, with three FFTs instead of
 * four.  For D = 256 the library's own kernels do all of it: one launch transforms the rows
 * of Q and Y (one complex FFT of Q + iY per row, split by Hermitian symmetry), one kernel
 * runs the column FFTs of both, the pointwise step and the inverse column FFT, and one
 * launch transforms the rows back (two real rows per complex FFT); other sizes use cuFFT's
 * 2-D transforms (fft created for this D and B).  Q, Y, dLdQ [B * D * D]; ctf as for
 * gs_apply_ctf; dLdQ may alias Q.  Two half spectra and the work area sit at the tail of ws
 * (gs_workspace_size includes them). */
int gs_ctf_loss_grad(const gs_config* cfg, const float* Q, const float* Y, const float* ctf, int B,
                     float* loss, float* dLdQ, const gs_fft* fft, void* ws, size_t ws_bytes,
                     gs_stream_t stream);

/* Backward of Rasterize (App. A.2 Eqs. 16-21; grad_mu = W^T [grad_mu_tilde; 0]; the s, q
 * chain through Sigma = (R S)(R S)^T; softplus derivatives).  Accumulates (+=) dL/dtheta
 * into dtheta[N * 11] summed over the B particles; the caller zeroes it first.  proj,
 * pair_gauss and tile_ranges are the outputs of gs_project / gs_bin_sort for the same
 * theta and W, and ws must still hold what gs_project wrote. */
int gs_render_bwd(const gs_config* cfg, const float* theta, int N, const float* W, int B,
                  const gs_record* proj, const uint32_t* pair_gauss, const uint32_t* tile_ranges,
                  const float* dLdQ, float* dtheta, void* ws, size_t ws_bytes, gs_stream_t stream);

/* gs_render_bwd_pose: gs_render_bwd plus the gradients with respect to each particle's pose
 * and in-plane translation.  The paper keeps poses fixed (Sec. 4.1) and names their joint
 * optimization as future work (Sec. 5); these follow from the same chain one step earlier:
 * mu_dot = W mu and Sigma_dot = W Sigma W^T (Eq. 6) give, summed over the particle's
 * (Gaussian, tile) pairs, dL/dW = grad_mu_dot mu^T + G W Sigma^T + G^T W Sigma with
 * G = [[grad_Sigma_tilde, 0], [0, 0]] (Eq. 21), and a translation t of the model image
 * (mu_tilde -> mu_tilde + t, at t = 0) gives dL/dt = sum grad_mu_tilde.
 * dpose[B * 12] (device, 16-byte aligned) is ACCUMULATED (the caller zeroes it):
 * dL/dW row-major at 0..8 (row 2 stays 0: depth does not enter the image), 9 unused,
 * dL/dt at 10..11 (model units).  The summation order of dpose varies between runs. */
int gs_render_bwd_pose(const gs_config* cfg, const float* theta, int N, const float* W, int B, const gs_record* proj,
                       const uint32_t* pair_gauss, const uint32_t* tile_ranges, const float* dLdQ, float* dtheta,
                       float* dpose, void* ws, size_t ws_bytes, gs_stream_t stream);

/* Adam step with one learning rate for all parameters (Sec. 4.1):
 * m = b1 m + (1-b1) g; v = b2 v + (1-b2) g^2; theta -= lr (m / (1-b1^t)) / (sqrt(v / (1-b2^t)) + eps).
 * t >= 1 counts steps.  n = 11 N. */
int gs_step(float* theta, const float* dtheta, float* m, float* v, int n, int t, float lr,
            float beta1, float beta2, float eps, gs_stream_t stream);

/* Adam step as gs_step with the step counter kept on the device: *t_dev (device int) holds
 * the number of steps already taken; the call uses t = *t_dev + 1 and then increments
 * *t_dev (stream-ordered).  Nothing depends on host values that change between steps, so
 * the call can be recorded once in a CUDA graph and replayed (Sec. 4.1 Adam). */
int gs_step_counted(float* theta, const float* dtheta, float* m, float* v, int n, int* t_dev,
                    float lr, float beta1, float beta2, float eps, gs_stream_t stream);

/* ---------------------------------------------------------------------------------------
 * Binning without a caller workspace
 * ------------------------------------------------------------------------------------- */

/* gs_bin_sort_noalloc: the same binning and sort as gs_bin_sort, with the same outputs,
 * for callers that cannot allocate device memory -- e.g. a plug-in inside a host
 * application that manages every byte of device memory through its own pool and forbids
 * other allocations, or a pipeline that must not allocate while running because
 * cudaMalloc can synchronize the device.  The paper has no counterpart to this entry
 * point; it exists only for such callers.
 * The scratch space is a file-scope device array of 8 MiB that every GPU loading the
 * library holds until the process exits; this call allocates nothing (no cudaMalloc,
 * cudaFree or allocating library routine).  The scratch needed for (cfg, B, N) is written
 * to *scratch_needed (host, may be NULL); if it exceeds 8 MiB the call returns GS_ENOSPC
 * and does nothing else.  The first call on a device looks up the array's device address
 * (cudaGetSymbolAddress, with that device current) and caches it; that look-up must not
 * happen inside a stream capture, so a first call on a capturing stream returns GS_ECAPTURE
 * before any other CUDA call (the capture is left untouched): make that first call before
 * capturing any stream.  All calls on a device share the array and leave their
 * contents in it (the call clears what must start at zero); calls whose GPU work
 * overlaps -- on different streams without ordering -- race on the array.  Overflow of
 * pair_capacity is visible as *n_pairs > pair_capacity (the status word is internal).
 * proj is gs_project's whole output for the same B and N, box plane included. */
int gs_bin_sort_noalloc(const gs_config* cfg, const gs_record* proj, int B, int N,
                        uint32_t* pair_gauss, size_t pair_capacity, uint32_t* tile_ranges,
                        uint32_t* n_pairs, gs_stream_t stream, size_t* scratch_needed);

/* -------------------------------------------------------------------------------------
 * Learned warm start (not in the paper)
 *
 * The paper starts every reconstruction from random Gaussians (Sec. 4.1).  These calls
 * build a learned initializer on top of the method: a coarse backprojection of the
 * particle images, seeds drawn from it, a point-MLP that maps each seed's neighbourhood to
 * one Gaussian, and the labels it is trained on (nearest Gaussian of a GMM fitted by the
 * plain method).  Device pointers, caller-owned, stream-ordered like the rest of the ABI.
 * ------------------------------------------------------------------------------------- */

/* gs_backproject: vol[Dv][Dv][Dv] ([z][y][x]; voxel centres -E + (idx + 1/2) 2E/Dv) =
 * mean over the B particles of images[B][D][D] averaged over an f x f stencil of
 * bilinear samples (one pixel apart, f = max(1, D / Dv)) centred where the voxel centre r
 * projects: (column, row) = ((W r)_x / h + floor(D/2), floor(D/2) - (W r)_y / h), the
 * inverse of the pixel centres of App. A.2 Eq. 13.  Outside the image reads zero.  W is
 * [B][9] row-major (Sec. 3.3.2 Eq. 6).  Passing CTF-multiplied images (gs_apply_ctf) makes
 * this the adjoint of the coarse image formation model.  1 <= Dv <= 256. */
int gs_backproject(const float* images, const float* W, int B, int D, float E, int Dv, float* vol,
                   gs_stream_t stream);

/* gs_mass_estimate: *mass (device float) = h^2 sum_b (-w_b S_b) / sum_b w_b^2, S_b the pixel
 * sum of image b and w_b = ctf[b][3]: the least-squares total amplitude sum_i A_i, since
 * the CTF's DC term is -w (App. A.2 Eq. 14) and a splat inside the box integrates to its
 * amplitude (Eq. 12).  scratch: device double[2].  B >= 1. */
int gs_mass_estimate(const float* images, const float* ctf, int B, int D, float E, double* scratch, float* mass,
                     gs_stream_t stream);

/* gs_seed_sample: K seeds drawn from vol[Dv^3] with probability proportional to the integer
 * weights q_v = floor(fl32(max(vol_v, 0) / vmax) * 2^20) (all 1 if vmax <= 0).  Seed k with
 * uniforms u[k][0..3] in [0, 1) takes the first voxel whose running weight sum exceeds
 * t = min(floor(u0 T), T - 1) (T the total, product in FP64) and the point
 * (-E + (idx + 1/2) dv) + (u_{1,2,3} - 1/2) dv of it, dv = fl32(2E / Dv), each FP32
 * operation rounded in that order.  Outputs: cdf[Dv^3] (running sums, scratch),
 * *vmax (device float), voxel[K] (may be NULL), pos[K][3].  The volume must be finite. */
int gs_seed_sample(const float* vol, int Dv, float E, const float* u, int K, unsigned long long* cdf, float* vmax,
                   int* voxel, float* pos, gs_stream_t stream);

/* gs_seed_features: feats[K][32] = the volume (trilinear, voxel centres at integer
 * coordinates, zero outside) at pos + {-1, 0, 1}^3 voxels divided by *vmax (27 values,
 * z slowest, x fastest), then pos / E (3), then 0, 0. */
int gs_seed_features(const float* vol, int Dv, float E, const float* vmax, const float* pos, int K, float* feats,
                     gs_stream_t stream);

/* gs_merge_labels: labels[K][10] of the seeds pos[K][3] against a fitted GMM theta_fit[N][11]:
 * a mass-preserving coarse-graining of the fitted mixture onto the seeds.  Each fitted
 * Gaussian g goes to its nearest seed (squared distance ((dx dx + dy dy) + dz dz) in FP32,
 * each step rounded, ties to the lower seed index) -> assign[N] (int32).  Seed k is the
 * moment-matched merge of its Gaussians (FP64 sums in moments[K][10], caller scratch):
 * mass A_k, offset delta_k from the seed, covariance C_k (Sigma = R S S^T R^T, Sec. 3.3.1
 * Eq. 5, plus the spread of the centres).  Label: delta_k / dv (3); log L00, log L11,
 * log L22 (clamped to [-6, 3]), L10, L20, L21 of the Cholesky factor of C_k / dv^2 (6);
 * A_k K / M clamped to [0, 100] (1), M = *mass.  A seed with no Gaussian is labelled
 * (0, 0, 0, log 1/2 x 3, 0, 0, 0, 0).  dv = 2E / Dv.  K >= 1. */
int gs_merge_labels(const float* pos, int K, const float* theta_fit, int N, int Dv, float E, const float* mass,
                    int* assign, double* moments, float* labels, gs_stream_t stream);

/* gs_decode_seeds: raw theta[K][11] from seeds pos[K][3] and pred[K][10] in the label
 * encoding of gs_merge_labels: mu = pos + dv pred[0..2]; Sigma = dv^2 L L^T; its
 * eigen-decomposition (cyclic Jacobi, FP64) gives s = softplus^-1(sqrt(lambda)) and q, the
 * quaternion (w, x, y, z) of the eigenvector matrix with det +1; A = softplus^-1(M / K
 * max(pred[9], 1e-3)). */
int gs_decode_seeds(const float* pos, const float* pred, int K, int Dv, float E, const float* mass, float* theta,
                    gs_stream_t stream);

/* Point-MLP: Z1 = X W1^T + b1, H1 = relu(Z1), Z2 = H1 W2^T + b2, H2 = relu(Z2),
 * Y = H2 W3^T + b3, widths din, hidden, dout in [1, 128].  Every product rounds both
 * operands to bfloat16 (nearest even) and accumulates in FP32; biases, activations and
 * gradients are FP32.  params (FP32, flat): W1[hidden][din], b1[hidden],
 * W2[hidden][hidden], b2[hidden], W3[dout][hidden], b3[dout]; gs_mlp_param_count gives the
 * length (host size_t).  Rows of X are X[idx[s]] when idx (int32[n]) is given, else X[s]. */
int gs_mlp_param_count(int din, int hidden, int dout, size_t* count);

/* acts: n * 4 * hidden floats (Z1, H1, Z2, H2, each [n][hidden]), kept for the backward.
 * Y: [n][dout]. */
int gs_mlp_forward(const float* params, int din, int hidden, int dout, const float* X, const int* idx, int n,
                   float* acts, float* Y, gs_stream_t stream);

/* dparams += dL/dparams for upstream dY[n][dout] (the caller zeroes dparams); the
 * bfloat16 rounding is passed straight through.  scratch: n * 2 * hidden floats. */
int gs_mlp_backward(const float* params, int din, int hidden, int dout, const float* X, const int* idx, int n,
                    const float* acts, const float* dY, float* dparams, float* scratch, gs_stream_t stream);

/* loss[0] += scale * sum (Y[s][c] - T[row(s)][c])^2 and dY = 2 scale (Y - T[row]) (dY may
 * be NULL); row(s) = idx[s] if idx is given.  scale = 1 / (n width) gives the mean. */
int gs_mse(const float* Y, const float* T, const int* idx, int n, int width, float scale, float* loss, float* dY,
           gs_stream_t stream);

/* -------------------------------------------------------------------------------------
 * Evaluation: GMM voxelization and Fourier shell correlation (the paper judges its GMMs by
 * FSC of the mixture on a voxel grid, Sec. 4, without giving formulas; these are the
 * library's own definitions)
 * ------------------------------------------------------------------------------------- */

/* gs_voxelize: vol[Dv][Dv][Dv] (index [k][i][j]) = sum_g A_g N(r; mu_g, Sigma_g), the
 * normalized 3-D Gaussian density (Sec. 3.3.1 Eqs. 4-5), at r = ((j - floor(Dv/2)) h,
 * -(i - floor(Dv/2)) h, (k - floor(Dv/2)) h), h = 2E / Dv: the pixel grid of App. A.2 Eq. 13
 * extended along z, so that sum_k vol[k] h is the image rendered at W = I.  Gaussian g adds
 * only inside its per-axis k-sigma box [ceil(c - r), floor(c + r)] (c its centre in voxel
 * units, r = cutoff_sigma sqrt(Sigma_aa) / h, clipped to the grid), decided in FP32 with
 * correctly rounded operations in a fixed order: Sigma_aa = ((M_a0^2 + M_a1^2) + M_a2^2) with
 * M = R diag(s) as in gs_project, r = k (sqrt(Sigma_aa) (1/h)), c_x = mu_x (1/h) + floor(Dv/2),
 * c_y = floor(Dv/2) - mu_y (1/h), c_z = mu_z (1/h) + floor(Dv/2), 1/h = fl32(Dv / 2E).
 * Contributions are added with atomics, so the summation order (and the last bits) can vary
 * between runs.  Gaussians with non-finite parameters are skipped.  ws: workspace of
 * gs_voxel_workspace_size(N) bytes.  1 <= Dv <= 1024. */
int gs_voxel_workspace_size(int N, size_t* bytes);
int gs_voxelize(const float* theta, int N, int Dv, float E, float cutoff_sigma, float* vol, void* ws, size_t ws_bytes,
                gs_stream_t stream);

/* Fourier shell correlation of two D^3 volumes.  FSC(s) = Re sum F1 conj(F2) /
 * sqrt(sum |F1|^2 sum |F2|^2) over the coefficients of shell s = 0 .. D/2, the shell of
 * frequency index (kx, ky, kz) (signed, DFT order) being the integer nearest to |k|.  The
 * sums run over the R2C half spectrum with Hermitian weights (1 for kx = 0 and kx = D/2,
 * 2 otherwise) in FP64.  gs_fsc_create makes the cuFFT plan (host call, not stream-ordered);
 * gs_fsc writes fsc[D/2 + 1] (device) using a workspace of gs_fsc_workspace_size bytes. */
typedef struct gs_fsc_plan {
  int r2c;           /* cuFFT handle */
  int D;
  size_t work_bytes; /* cuFFT work area (inside the gs_fsc workspace) */
} gs_fsc_plan;

int gs_fsc_create(int D, gs_fsc_plan* plan);
int gs_fsc_destroy(gs_fsc_plan* plan);
int gs_fsc_workspace_size(const gs_fsc_plan* plan, size_t* bytes);
int gs_fsc(const gs_fsc_plan* plan, const float* vol1, const float* vol2, float* fsc, void* ws, size_t ws_bytes,
           gs_stream_t stream);

/* -------------------------------------------------------------------------------------
 * The remaining steps of Algorithm 1 (FourierShift, SplitGaussian).  The paper gives no
 * formula for either; these are the library's definitions.
 * ------------------------------------------------------------------------------------- */

/* gs_fourier_shift: out[b] = in[b] moved by t[b] = (t_x, t_y) (model units) on the periodic
 * pixel grid ("center alignment" with the published translations, Algorithm 1, Sec. 4.1):
 * the R2C spectrum is multiplied by exp(-2 pi i (m s_x + l s_y) / D) with s_x = t_x / h
 * (columns) and s_y = -t_y / h (rows grow downward, App. A.2 Eq. 13), the factor of each
 * axis replaced by cos(pi s) at its Nyquist index for even D (so the result stays real and an
 * integer shift is a circular roll).  fft and ws as for gs_apply_ctf; in != out. */
int gs_fourier_shift(const gs_config* cfg, const float* in, const float* t, int B, float* out, const gs_fft* fft,
                     void* ws, size_t ws_bytes, gs_stream_t stream);

/* gs_split_gaussians: SplitGaussian of Algorithm 1 for every Gaussian (the optional
 * densification that doubles N): out[2N * 11] holds, at rows g and N + g, the children of
 * Gaussian g, placed at mu +- alpha s_max v along its major axis (v the column of R(q) of the
 * largest softplus scale s_max, the lower index on ties), each with amplitude A / 2 and the
 * major scale s_max sqrt(1 - alpha^2); the other scales and the rotation are kept.  The pair
 * keeps the parent's mass, mean and covariance.  Raw parameters (softplus inverted in FP64).
 * 0 <= alpha < 1; out != theta. */
int gs_split_gaussians(const float* theta, int N, float alpha, float* out, gs_stream_t stream);

/* -------------------------------------------------------------------------------------
 * Diagnostics
 * ------------------------------------------------------------------------------------- */

/* gs_probe_ex2: launches a throughput probe of ex2.approx.ftz.f32, the special-function
 * operation that each evaluated splat pixel takes in SumSplats (Algorithm 2) and its
 * backward; the paper has no counterpart -- it measures the unit whose rate is the roofline
 * of the render kernels on the GPU at hand.  blocks CTAs of 256 threads each run 8
 * independent chains of `iters` steps x <- ex2(x) * s - 1 (bound by ex2, not by the FMA).
 * The caller times the launch on `stream` (e.g. with CUDA events); *ex2_count (host, may be
 * NULL) receives the number of ex2 the launch executes.  sink: one device float that is never
 * written in practice (it keeps the chains from being optimized away).  GS_EINVAL for
 * blocks outside [1, 2^20], iters outside [1, 2^24] or a NULL sink. */
int gs_probe_ex2(int blocks, int iters, float* sink, gs_stream_t stream, double* ex2_count);

#ifdef __cplusplus
}
#endif
#endif /* GS_H_ */
