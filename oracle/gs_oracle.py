"""FP64 oracle of the cryoSplat splatting path (test infrastructure; see package docstring).

Notation follows the paper (arXiv 2508.04929):

* Theta[N, 11] = [mu_x, mu_y, mu_z, s_x, s_y, s_z, q_w, q_x, q_y, q_z, A] in the raw
  (pre-activation) form, Sec. 3.3.1 and the parameter vector of Sec. 4.1.
* W in SO(3) is the particle pose, mu_dot = W mu, Sigma_dot = W Sigma W^T (Sec. 3.3.2,
  Eq. 6).  The in-plane translation t is zero on this path: Sec. 4.1 applies the
  published translations to the observed images instead.
* The splat is the 2-D normalized Gaussian with mean mu_tilde = mu_dot[:2] and covariance
  Sigma_tilde = Sigma_dot[:2, :2] (Sec. 3.3.3 Eq. 8, App. A.2 Eq. 12).
* Pixels follow the FFT-aligned convention of App. A.2 Eq. 13: pixel (i, j) samples the
  continuous image at ((j - floor(D/2)) 2E/D, -(i - floor(D/2)) 2E/D).
* Q = sum_i A_i G_tilde_i (App. A.2 Eq. 15), X = F^-1(H_hat . F(Q)) (Eq. 14), and the loss
  is L = ||X - Y||^2 (Sec. 3.3.5).
* Gradients follow App. A.2 Eqs. 16-21 with two readings: grad_mu = W^T [grad_mu_tilde; 0]
  (the paper prints W; mu_dot = W mu forces the transpose), and the s / q chain of 3DGS
  written out explicitly (the paper defers it to 3DGS).

Readings the paper leaves open:

* Support: a Gaussian contributes to the pixels of the axis-aligned bounding box of its
  k-sigma ellipse, k = 3 by default (the paper inherits 3-sigma culling from the 3DGS
  rasterizer it adopts, Sec. 3.3.4 and App. C.2, without stating it).  The box is an
  integer decision; it is taken in FP32 (``support_fp32``) by the exact sequence of
  correctly rounded operations that the CUDA kernel performs, so both sides take it in
  the same precision.
* CTF: H_hat(k) = -(sqrt(1 - w^2) sin chi + w cos chi), chi = pi lambda df |k|^2 -
  (pi / 2) Cs lambda^3 |k|^4, relativistic lambda; no envelope (the paper gives no formula,
  App. A.2 Eq. 14 only names the rasterized CTF).
* Loss: the literal sum of squares per image (reduction 0) or its mean over pixels
  (reduction 1).
* Adam with the PyTorch defaults beta1 = 0.9, beta2 = 0.999, eps = 1e-8 and one learning
  rate for all eleven parameters (Sec. 4.1).
"""
from __future__ import annotations

import math

import numpy as np

__all__ = [
    "softplus", "sigmoid", "quat_to_rot", "quat_to_rot_jacobian",
    "build_gaussians", "viewing_transform", "projection", "splat",
    "pixel_centres", "support_fp32", "render", "render_one",
    "tile_pairs", "tile_counts", "electron_wavelength", "ctf_radial", "ctf_image", "dft2", "idft2",
    "apply_ctf", "apply_ctf_adjoint", "loss", "backward", "adam_step",
    "forward_backward",
]

F64 = np.float64
F32 = np.float32


# ----------------------------------------------------------------------------------------
# Parameterization (Sec. 3.3.1, Eqs. 4-5)
# ----------------------------------------------------------------------------------------
def softplus(x):
    """softplus(x) = log(1 + e^x), written in the overflow-free form max(x,0) + log1p(e^-|x|).

    Sec. 3.3.1: softplus makes A and s positive."""
    x = np.asarray(x, dtype=F64)
    return np.maximum(x, 0.0) + np.log1p(np.exp(-np.abs(x)))


def sigmoid(x):
    """Derivative of softplus."""
    x = np.asarray(x, dtype=F64)
    return 0.5 * (1.0 + np.tanh(0.5 * x))


def quat_to_rot(qhat):
    """Rotation matrix of the unit quaternion [q_w, q_x, q_y, q_z] (Sec. 3.3.1).

    qhat: [..., 4] -> [..., 3, 3]."""
    w, x, y, z = (qhat[..., 0], qhat[..., 1], qhat[..., 2], qhat[..., 3])
    R = np.empty(qhat.shape[:-1] + (3, 3), dtype=F64)
    R[..., 0, 0] = 1 - 2 * (y * y + z * z)
    R[..., 0, 1] = 2 * (x * y - w * z)
    R[..., 0, 2] = 2 * (x * z + w * y)
    R[..., 1, 0] = 2 * (x * y + w * z)
    R[..., 1, 1] = 1 - 2 * (x * x + z * z)
    R[..., 1, 2] = 2 * (y * z - w * x)
    R[..., 2, 0] = 2 * (x * z - w * y)
    R[..., 2, 1] = 2 * (y * z + w * x)
    R[..., 2, 2] = 1 - 2 * (x * x + y * y)
    return R


def quat_to_rot_jacobian(qhat):
    """dR[k, m] / d qhat[c] for the rotation of ``quat_to_rot``: [..., 3, 3, 4]."""
    w, x, y, z = (qhat[..., 0], qhat[..., 1], qhat[..., 2], qhat[..., 3])
    J = np.zeros(qhat.shape[:-1] + (3, 3, 4), dtype=F64)
    # columns: d/dw, d/dx, d/dy, d/dz
    J[..., 0, 0, :] = np.stack([0 * w, 0 * w, -4 * y, -4 * z], -1)
    J[..., 0, 1, :] = np.stack([-2 * z, 2 * y, 2 * x, -2 * w], -1)
    J[..., 0, 2, :] = np.stack([2 * y, 2 * z, 2 * w, 2 * x], -1)
    J[..., 1, 0, :] = np.stack([2 * z, 2 * y, 2 * x, 2 * w], -1)
    J[..., 1, 1, :] = np.stack([0 * w, -4 * x, 0 * w, -4 * z], -1)
    J[..., 1, 2, :] = np.stack([-2 * x, -2 * w, 2 * z, 2 * y], -1)
    J[..., 2, 0, :] = np.stack([-2 * y, 2 * z, -2 * w, 2 * x], -1)
    J[..., 2, 1, :] = np.stack([2 * x, 2 * w, 2 * z, 2 * y], -1)
    J[..., 2, 2, :] = np.stack([0 * w, -4 * x, -4 * y, 0 * w], -1)
    return J


def build_gaussians(theta):
    """BuildGaussians of Algorithm 2: raw Theta -> (mu, Sigma, A) and the intermediates.

    Sec. 3.3.1: A = softplus(A_raw), s = softplus(s_raw), q normalized, R = R(q),
    Sigma = R S S^T R^T with S = diag(s) (Eq. 5)."""
    theta = np.asarray(theta, dtype=F64).reshape(-1, 11)
    mu = theta[:, 0:3].copy()
    s = softplus(theta[:, 3:6])
    q = theta[:, 6:10]
    qnorm = np.sqrt(np.sum(q * q, axis=1))
    qhat = q / qnorm[:, None]
    R = quat_to_rot(qhat)
    S = np.zeros((theta.shape[0], 3, 3), dtype=F64)
    S[:, 0, 0], S[:, 1, 1], S[:, 2, 2] = s[:, 0], s[:, 1], s[:, 2]
    M = R @ S
    Sigma = M @ np.transpose(M, (0, 2, 1))
    A = softplus(theta[:, 10])
    return dict(mu=mu, s=s, q=q, qnorm=qnorm, qhat=qhat, R=R, S=S, M=M, Sigma=Sigma, A=A)


def viewing_transform(mu, Sigma, W):
    """ViewingTransform of Algorithm 2 (Sec. 3.3.2, Eq. 6 with t = 0).

    mu_dot = W mu, Sigma_dot = W Sigma W^T."""
    W = np.asarray(W, dtype=F64).reshape(3, 3)
    mu_dot = mu @ W.T
    Sigma_dot = W[None] @ Sigma @ W.T[None]
    return mu_dot, Sigma_dot


def projection(mu_dot, Sigma_dot):
    """Projection of Algorithm 2 (App. A.2, Eq. 12): drop the z components."""
    return mu_dot[..., 0:2], Sigma_dot[..., 0:2, 0:2]


def splat(r, mu_t, Sigma_t):
    """Normalized 2-D splat G_tilde(r | mu_tilde, Sigma_tilde) of Sec. 3.3.3, Eq. 8.

    r: [..., 2] points; mu_t: [2]; Sigma_t: [2, 2].  Keeps the view-dependent normalization
    1 / (2 pi |Sigma_tilde|^(1/2)) that the paper insists on (Sec. 3.3.3)."""
    P = np.linalg.inv(Sigma_t)
    d = r - mu_t
    quad = np.einsum("...a,ab,...b->...", d, P, d)
    return np.exp(-0.5 * quad) / (2.0 * math.pi * math.sqrt(np.linalg.det(Sigma_t)))


def pixel_centres(D, E=0.5):
    """Continuous coordinates of the pixel centres (App. A.2, Eq. 13).

    Returns (rx[D, D], ry[D, D]): pixel (i, j) sits at ((j - floor(D/2)) h, -(i - floor(D/2)) h)
    with h = 2E / D; the row index is y (flipped), the column index is x."""
    h = 2.0 * E / D
    c = D // 2
    i = np.arange(D, dtype=F64)[:, None]
    j = np.arange(D, dtype=F64)[None, :]
    rx = (j - c) * h + 0.0 * i
    ry = -(i - c) * h + 0.0 * j
    return rx, ry


# ----------------------------------------------------------------------------------------
# Support: the k-sigma pixel box, an integer decision taken in FP32
# ----------------------------------------------------------------------------------------
def _sp32(x32):
    """FP32 value of softplus, computed in FP64 and rounded once to FP32."""
    return softplus(np.asarray(x32, dtype=F64)).astype(F32)


def support_fp32(theta, W, D, E=0.5, cutoff=3.0, centres=False):
    """Clipped k-sigma pixel box of every Gaussian for one pose, in FP32.

    Reading of the support rule (the paper inherits 3-sigma culling from 3DGS, Sec. 3.3.4,
    App. C.2): Gaussian g contributes to pixel (i, j) iff
    ceil(c_x - r_x) <= j <= floor(c_x + r_x) and ceil(c_y - r_y) <= i <= floor(c_y + r_y),
    clipped to [0, D-1], where c = the splat centre in pixel units (Eq. 13 inverted) and
    r_x = k sqrt(Sigma_tilde_xx) / h, r_y = k sqrt(Sigma_tilde_yy) / h.

    The box is an integer decision on floating-point values, so it is taken in the kernel's
    precision: FP32, with every operation correctly rounded, in this order:
      s = fp32(softplus_fp64(s_raw));  n = sqrt(((qw*qw + qx*qx) + qy*qy) + qz*qz);
      (w,x,y,z) = q / n;  R from the unit quaternion (Sec. 3.3.1) with products formed first;
      M[k,m] = R[k,m] * s[m];  V[a,m] = (W[a,0]*M[0,m] + W[a,1]*M[1,m]) + W[a,2]*M[2,m];
      Sxx = (V00^2 + V01^2) + V02^2;  Syy = (V10^2 + V11^2) + V12^2;
      mx = (W00 mu_x + W01 mu_y) + W02 mu_z;  my likewise with row 1;
      inv_h = D / (2E);  c_x = mx * inv_h + floor(D/2);  c_y = floor(D/2) - my * inv_h;
      r_x = k * (sqrt(Sxx) * inv_h);  r_y = k * (sqrt(Syy) * inv_h).
    (Sigma_tilde = V V^T, i.e. the top-left block of W R S S^T R^T W^T, Eqs. 5, 6, 12.)
    A Gaussian whose parameters or box coordinates are not finite is excluded.

    theta: [N, 11] (FP32 values), W: [3, 3] (FP32 values).
    Returns int64 arrays x0, x1, y0, y1 (inclusive; empty when x0 > x1 or y0 > y1) and a
    bool array ``bad`` marking excluded non-finite Gaussians; with ``centres`` also the
    FP32 centre (c_x, c_y) in pixel units."""
    th = np.asarray(theta, dtype=F32).reshape(-1, 11)
    Wf = np.asarray(W, dtype=F32).reshape(3, 3)
    n = th.shape[0]
    with np.errstate(all="ignore"):
        mux, muy, muz = th[:, 0], th[:, 1], th[:, 2]
        s = [_sp32(th[:, 3]), _sp32(th[:, 4]), _sp32(th[:, 5])]
        qw, qx, qy, qz = th[:, 6], th[:, 7], th[:, 8], th[:, 9]
        n2 = ((qw * qw + qx * qx) + qy * qy) + qz * qz
        nr = np.sqrt(n2)
        w, x, y, z = qw / nr, qx / nr, qy / nr, qz / nr
        xx, yy, zz = x * x, y * y, z * z
        xy, xz, yz = x * y, x * z, y * z
        wx, wy, wz = w * x, w * y, w * z
        one, two = F32(1.0), F32(2.0)
        R = [[one - two * (yy + zz), two * (xy - wz), two * (xz + wy)],
             [two * (xy + wz), one - two * (xx + zz), two * (yz - wx)],
             [two * (xz - wy), two * (yz + wx), one - two * (xx + yy)]]
        M = [[R[k][m] * s[m] for m in range(3)] for k in range(3)]
        V = [[(Wf[a, 0] * M[0][m] + Wf[a, 1] * M[1][m]) + Wf[a, 2] * M[2][m] for m in range(3)]
             for a in range(2)]
        Sxx = (V[0][0] * V[0][0] + V[0][1] * V[0][1]) + V[0][2] * V[0][2]
        Syy = (V[1][0] * V[1][0] + V[1][1] * V[1][1]) + V[1][2] * V[1][2]
        mx = (Wf[0, 0] * mux + Wf[0, 1] * muy) + Wf[0, 2] * muz
        my = (Wf[1, 0] * mux + Wf[1, 1] * muy) + Wf[1, 2] * muz
        inv_h = F32(D) / (two * F32(E))
        c0 = F32(D // 2)
        k = F32(cutoff)
        cx = mx * inv_h + c0
        cy = c0 - my * inv_h
        rx = k * (np.sqrt(Sxx) * inv_h)
        ry = k * (np.sqrt(Syy) * inv_h)
        bad = ~(np.isfinite(th).all(axis=1) & np.isfinite(cx) & np.isfinite(cy)
                & np.isfinite(rx) & np.isfinite(ry))
        x0f = np.ceil(cx - rx)
        x1f = np.floor(cx + rx)
        y0f = np.ceil(cy - ry)
        y1f = np.floor(cy + ry)
        lo, hi = F32(0.0), F32(D - 1)
        x0f, y0f = np.maximum(x0f, lo), np.maximum(y0f, lo)
        x1f, y1f = np.minimum(x1f, hi), np.minimum(y1f, hi)
    x0 = np.where(bad, 1, np.nan_to_num(x0f, nan=1)).astype(np.int64)
    x1 = np.where(bad, 0, np.nan_to_num(x1f, nan=0)).astype(np.int64)
    y0 = np.where(bad, 1, np.nan_to_num(y0f, nan=1)).astype(np.int64)
    y1 = np.where(bad, 0, np.nan_to_num(y1f, nan=0)).astype(np.int64)
    assert x0.shape == (n,)
    if centres:
        return x0, x1, y0, y1, bad, cx, cy
    return x0, x1, y0, y1, bad


# ----------------------------------------------------------------------------------------
# Rasterize (Algorithm 2) in FP64
# ----------------------------------------------------------------------------------------
def render_one(theta, W, D, E=0.5, cutoff=3.0, box=None):
    """Q for one pose (Algorithm 2; App. A.2 Eq. 15 sampled at the Eq. 13 pixel centres).

    For every Gaussian: BuildGaussians -> ViewingTransform -> Projection, then add
    A G_tilde at the pixels of its support box.  ``box`` overrides the support (x0, x1,
    y0, y1 arrays); by default it is ``support_fp32``.  Returns Q[D, D] in FP64."""
    g = build_gaussians(theta)
    mu_dot, Sigma_dot = viewing_transform(g["mu"], g["Sigma"], W)
    mu_t, Sigma_t = projection(mu_dot, Sigma_dot)
    if box is None:
        box = support_fp32(theta, W, D, E, cutoff)[:4]
    x0, x1, y0, y1 = box
    rx, ry = pixel_centres(D, E)
    Q = np.zeros((D, D), dtype=F64)
    for n in range(g["mu"].shape[0]):
        if x0[n] > x1[n] or y0[n] > y1[n]:
            continue
        sl = (slice(y0[n], y1[n] + 1), slice(x0[n], x1[n] + 1))
        r = np.stack([rx[sl], ry[sl]], axis=-1)
        Q[sl] += g["A"][n] * splat(r, mu_t[n], Sigma_t[n])
    return Q


def render(theta, Ws, D, E=0.5, cutoff=3.0):
    """Q[B, D, D] for a batch of poses Ws[B, 3, 3]."""
    Ws = np.asarray(Ws).reshape(-1, 3, 3)
    return np.stack([render_one(theta, Ws[b], D, E, cutoff) for b in range(Ws.shape[0])])


def tile_pairs(theta, Ws, D, tile, E=0.5, cutoff=3.0):
    """CreateTiles / DuplicateWithKeys / SortByKeys / IdentifyTileRanges of Algorithm 2.

    Every Gaussian is instantiated in every tile (tile x tile pixels, row-major tile index
    ty * ceil(D/tile) + tx) that its support box touches; the instances are ordered by the
    key (particle, tile, Gaussian).  Returns (pair_gauss[P] uint32, ranges[B, T, 2] uint32
    with absolute [start, end) offsets)."""
    Ws = np.asarray(Ws).reshape(-1, 3, 3)
    nt = -(-D // tile)
    keys = []
    for b in range(Ws.shape[0]):
        x0, x1, y0, y1, _ = support_fp32(theta, Ws[b], D, E, cutoff)
        for n in range(x0.shape[0]):
            if x0[n] > x1[n] or y0[n] > y1[n]:
                continue
            for ty in range(y0[n] // tile, y1[n] // tile + 1):
                for tx in range(x0[n] // tile, x1[n] // tile + 1):
                    keys.append((b, ty * nt + tx, n))
    keys.sort()
    B = Ws.shape[0]
    ranges = np.zeros((B, nt * nt, 2), dtype=np.uint32)
    pair_gauss = np.array([k[2] for k in keys], dtype=np.uint32)
    counts = np.zeros((B, nt * nt), dtype=np.int64)
    for b, t, _ in keys:
        counts[b, t] += 1
    start = np.concatenate([[0], np.cumsum(counts.reshape(-1))])[:-1].reshape(B, nt * nt)
    ranges[:, :, 0] = start
    ranges[:, :, 1] = start + counts
    return pair_gauss, ranges


def tile_counts(theta, Ws, D, tile, E=0.5, cutoff=3.0):
    """Instances per (particle, tile) of ``tile_pairs`` (counts[B, T]), without listing them:
    every Gaussian adds one to each tile of its support box's tile rectangle."""
    Ws = np.asarray(Ws).reshape(-1, 3, 3)
    nt = -(-D // tile)
    counts = np.zeros((Ws.shape[0], nt * nt), dtype=np.int64)
    for b in range(Ws.shape[0]):
        x0, x1, y0, y1, _ = support_fp32(theta, Ws[b], D, E, cutoff)
        ok = (x0 <= x1) & (y0 <= y1)
        tx0, tx1, ty0, ty1 = x0[ok] // tile, x1[ok] // tile, y0[ok] // tile, y1[ok] // tile
        for oy in range(int((ty1 - ty0).max(initial=-1)) + 1):
            for ox in range(int((tx1 - tx0).max(initial=-1)) + 1):
                m = (ty0 + oy <= ty1) & (tx0 + ox <= tx1)
                np.add.at(counts[b], (ty0[m] + oy) * nt + tx0[m] + ox, 1)
    return counts


# ----------------------------------------------------------------------------------------
# CTF (App. A.2 Eq. 14) with a direct FP64 DFT
# ----------------------------------------------------------------------------------------
def electron_wavelength(kv):
    """Relativistic electron wavelength in Angstrom for an accelerating voltage in kV."""
    V = kv * 1e3
    return 12.2643 / math.sqrt(V * (1.0 + 0.978466e-6 * V))


def _freqs(D):
    """Signed DFT frequency of every index, in cycles per pixel (index l -> l or l - D)."""
    l = np.arange(D, dtype=F64)
    return np.where(l < (D + 1) // 2, l, l - D) / D


def ctf_radial(k2, defocus_A, kv=300.0, cs_mm=2.7, w=0.1):
    """CTF at squared spatial frequency k2 (1/Angstrom^2), reading of App. A.2 Eq. 14:
    H_hat(k) = -(sqrt(1 - w^2) sin chi + w cos chi),
    chi = pi lambda df |k|^2 - (pi/2) Cs lambda^3 |k|^4 (relativistic lambda, Cs in A)."""
    lam = electron_wavelength(kv)
    cs = cs_mm * 1e7
    k2 = np.asarray(k2, dtype=F64)
    chi = math.pi * lam * defocus_A * k2 - 0.5 * math.pi * cs * lam ** 3 * k2 ** 2
    return -(math.sqrt(1.0 - w * w) * np.sin(chi) + w * np.cos(chi))


def ctf_image(D, defocus_A, kv=300.0, cs_mm=2.7, w=0.1, apix=1.5):
    """Rasterized CTF H_hat[D, D] on the unshifted DFT grid: index l of either axis is the
    signed frequency (l or l - D) / (D apix) in 1/Angstrom (App. A.2 Eq. 14)."""
    f = _freqs(D) / apix
    k2 = f[:, None] ** 2 + f[None, :] ** 2
    return ctf_radial(k2, defocus_A, kv, cs_mm, w)


def _dft_matrix(D):
    n = np.arange(D, dtype=F64)
    return np.exp(-2j * math.pi * np.outer(n, n) / D)


def dft2(x):
    """Direct 2-D DFT, F[k, n] = exp(-2 pi i k n / D) on both axes (no normalization)."""
    D = x.shape[-1]
    F = _dft_matrix(D)
    return F @ x @ F.T


def idft2(z):
    """Inverse of ``dft2`` (normalized by 1 / D^2)."""
    D = z.shape[-1]
    Fc = np.conj(_dft_matrix(D))
    return Fc @ z @ Fc.T / (D * D)


def apply_ctf(Q, H):
    """X = F^-1(H_hat . F(Q)) (App. A.2 Eq. 14).  Returns the real part; the imaginary part
    vanishes because H_hat is real and even."""
    Z = idft2(H * dft2(Q))
    return Z.real


def apply_ctf_adjoint(G, H):
    """Adjoint of ``apply_ctf`` as a real linear map: Q_bar = Re(F^H (conj(H) . (F^-1)^H G)),
    where (F^-1)^H = F / D^2 and F^H = conj(F) applied on both axes."""
    D = G.shape[-1]
    F = _dft_matrix(D)
    Fc = np.conj(F)
    inner = (F @ G @ F.T) / (D * D)
    return (Fc @ (np.conj(H) * inner) @ Fc.T).real


def loss(X, Y, reduction=0):
    """L = ||X - Y||_2^2 per image (Sec. 3.3.5); reduction 1 divides by the pixel count.

    Returns (L[B], dL/dX[B, D, D])."""
    R = X - Y
    scale = 1.0 if reduction == 0 else 1.0 / (X.shape[-1] * X.shape[-2])
    return scale * np.sum(R * R, axis=(-2, -1)), 2.0 * scale * R


# ----------------------------------------------------------------------------------------
# Backward (App. A.2 Eqs. 16-21, then the s / q chain of 3DGS)
# ----------------------------------------------------------------------------------------
def backward(theta, Ws, D, dLdQ, E=0.5, cutoff=3.0, boxes=None):
    """dL/dTheta[N, 11] given dL/dQ[B, D, D] (App. A.2 Eqs. 16-21).

    Per particle b and Gaussian, over the pixels r of the support:
      dL/dA            += sum dL/dQ(r) G_tilde(r)                                  (Eq. 17)
      grad_mu_tilde    += sum dL/dQ(r) A G_tilde(r) Sigma_tilde^-1 (r - mu_tilde)   (Eq. 18)
      grad_(Sigma~^-1) += sum dL/dQ(r) 1/2 A G_tilde(r) (Sigma_tilde - d d^T)       (Eq. 20)
      grad_Sigma_tilde  = -Sigma_tilde^-T grad_(Sigma~^-1) Sigma_tilde^-T           (Eq. 20)
      grad_Sigma_dot    = [[grad_Sigma_tilde, 0], [0, 0]]                           (Eq. 21)
      grad_Sigma       += W^T grad_Sigma_dot W    (Sigma_dot = W Sigma W^T, Eq. 6)
      grad_mu          += W^T [grad_mu_tilde; 0]  (mu_dot = W mu; the paper prints W)
    then per Gaussian, with Sigma = M M^T, M = R S:
      grad_M = (grad_Sigma + grad_Sigma^T) M,  grad_s[m] = sum_k grad_M[k,m] R[k,m],
      grad_R[k,m] = grad_M[k,m] s[m],  grad_qhat = sum grad_R dR/dqhat,
      grad_q = (grad_qhat - qhat (qhat . grad_qhat)) / |q|,
    and the softplus derivatives for s and A.  No symmetrization shortcut is taken: the
    matrices are differentiated as full matrices."""
    theta = np.asarray(theta, dtype=F64).reshape(-1, 11)
    Ws = np.asarray(Ws, dtype=F64).reshape(-1, 3, 3)
    g = build_gaussians(theta)
    N = theta.shape[0]
    rx, ry = pixel_centres(D, E)
    gA = np.zeros(N)
    gmu = np.zeros((N, 3))
    gSigma = np.zeros((N, 3, 3))
    for b in range(Ws.shape[0]):
        W = Ws[b]
        mu_dot, Sigma_dot = viewing_transform(g["mu"], g["Sigma"], W)
        mu_t, Sigma_t = projection(mu_dot, Sigma_dot)
        if boxes is None:
            x0, x1, y0, y1 = support_fp32(theta.astype(F32), W.astype(F32), D, E, cutoff)[:4]
        else:
            x0, x1, y0, y1 = boxes[b]
        for n in range(N):
            if x0[n] > x1[n] or y0[n] > y1[n]:
                continue
            sl = (slice(y0[n], y1[n] + 1), slice(x0[n], x1[n] + 1))
            r = np.stack([rx[sl], ry[sl]], axis=-1)
            Gt = splat(r, mu_t[n], Sigma_t[n])
            gq = dLdQ[b][sl]
            A = g["A"][n]
            P = np.linalg.inv(Sigma_t[n])
            d = r - mu_t[n]
            gA[n] += np.sum(gq * Gt)
            wgt = gq * A * Gt
            gmu_t = P @ np.einsum("ij,ija->a", wgt, d)
            gPinv = 0.5 * (np.sum(wgt) * Sigma_t[n] - np.einsum("ij,ija,ijb->ab", wgt, d, d))
            gSig_t = -P.T @ gPinv @ P.T
            gSig_dot = np.zeros((3, 3))
            gSig_dot[0:2, 0:2] = gSig_t
            gSigma[n] += W.T @ gSig_dot @ W
            gmu[n] += W.T @ np.array([gmu_t[0], gmu_t[1], 0.0])
    out = np.zeros((N, 11))
    out[:, 0:3] = gmu
    gM = (gSigma + np.transpose(gSigma, (0, 2, 1))) @ g["M"]
    s = g["s"]
    gs = np.einsum("nkm,nkm->nm", gM, g["R"])
    gR = gM * s[:, None, :]
    J = quat_to_rot_jacobian(g["qhat"])
    gqhat = np.einsum("nkm,nkmc->nc", gR, J)
    qhat = g["qhat"]
    gq = (gqhat - qhat * np.sum(qhat * gqhat, axis=1, keepdims=True)) / g["qnorm"][:, None]
    out[:, 3:6] = gs * sigmoid(theta[:, 3:6])
    out[:, 6:10] = gq
    out[:, 10] = gA * sigmoid(theta[:, 10])
    return out


def forward_backward(theta, Ws, D, Y, ctf_params, E=0.5, cutoff=3.0, reduction=0):
    """One pass of Algorithm 1's loop body for a batch (t = 0): Rasterize -> ApplyCTF ->
    Loss -> backprop.  ctf_params[B, 5] = (defocus_A, kV, Cs_mm, amp_contrast, apix_A).

    Returns dict(Q, X, L, dLdX, dLdQ, dtheta)."""
    Ws = np.asarray(Ws, dtype=F64).reshape(-1, 3, 3)
    B = Ws.shape[0]
    Q = render(theta, Ws, D, E, cutoff)
    X = np.empty_like(Q)
    Hs = []
    for b in range(B):
        df, kv, cs, w, apix = [float(v) for v in ctf_params[b]]
        H = ctf_image(D, df, kv, cs, w, apix)
        Hs.append(H)
        X[b] = apply_ctf(Q[b], H)
    L, dLdX = loss(X, np.asarray(Y, dtype=F64), reduction)
    dLdQ = np.stack([apply_ctf_adjoint(dLdX[b], Hs[b]) for b in range(B)])
    dtheta = backward(theta, Ws, D, dLdQ, E, cutoff)
    return dict(Q=Q, X=X, L=L, dLdX=dLdX, dLdQ=dLdQ, dtheta=dtheta)


# ----------------------------------------------------------------------------------------
# Adam with one learning rate for all parameters (Sec. 4.1)
# ----------------------------------------------------------------------------------------
def adam_step(theta, grad, m, v, t, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam step (t counts from 1).  Returns (theta, m, v) as new FP64 arrays."""
    theta = np.asarray(theta, dtype=F64)
    grad = np.asarray(grad, dtype=F64)
    m = beta1 * np.asarray(m, dtype=F64) + (1 - beta1) * grad
    v = beta2 * np.asarray(v, dtype=F64) + (1 - beta2) * grad * grad
    mhat = m / (1 - beta1 ** t)
    vhat = v / (1 - beta2 ** t)
    return theta - lr * mhat / (np.sqrt(vhat) + eps), m, v
