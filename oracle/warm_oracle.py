"""FP64 oracle of the learned warm start (test infrastructure; see package docstring).

The paper (arXiv 2508.04929) initializes every reconstruction at random (Sec. 4.1: means
N(0, 0.075^2), scales 0.0075, amplitudes 1/(2N)) and has no learned initializer and no
backprojection.  This module is the plain definition of the warm start that the library
adds on top of the paper's method.  Every quantity is defined here in words and code, and
``tests/test_warm_oracle_pins.py`` pins each function against something other than itself.

Pieces, in the order the pipeline uses them:

* ``backproject``: a coarse Dv^3 volume from particle images and their poses.  Voxel
  centres r = -E + (idx + 1/2) dv, dv = 2E/Dv, index order [z][y][x].  A voxel projects to
  p = W r (Sec. 3.3.2 Eq. 6) and so to pixel coordinates (column, row) =
  (p_x / h + floor(D/2), floor(D/2) - p_y / h), the inverse of the FFT-aligned pixel centres
  of App. A.2 Eq. 13.  The voxel value is the mean over particles of the image averaged
  over an f x f stencil of bilinear samples spaced one pixel apart and centred on that
  point, f = max(1, D // Dv), i.e. a box filter of the voxel's footprint.  Images outside
  [0, D) read as zero.  Fed with CTF-multiplied images (the CTF being self-adjoint) it is
  the adjoint of the coarse image formation model.
* ``mass_estimate``: the total amplitude sum_i A_i.  The DC term of the CTF is
  H_hat(0) = -w, so sum_p X_b(p) = -w_b sum_p Q_b(p), and sum_p Q_b(p) h^2 = sum_i A_i for
  Gaussians inside the box (mass conservation of the normalized splat, Eq. 12).  The
  least-squares estimate over the batch is M = h^2 sum_b (-w_b S_b) / sum_b w_b^2 with
  S_b = sum_p Y_b(p).
* ``seed_sample``: K seed positions drawn from the volume.  Voxel weights are the integers
  q_v = floor(fl32(max(vol_v, 0) / vmax) * 2^20) (all ones if vmax <= 0); with the running
  sums C_v = q_0 + ... + q_v and T = C_last, seed k picks the first voxel with C_v > t,
  t = min(floor(u0 * T), T - 1) formed in FP64, and a uniform point of that voxel,
  pos = (-E + (idx + 1/2) dv) + (u_{1,2,3} - 1/2) dv, each operation rounded to FP32 in
  that order.  The uniforms u[K, 4] are inputs.
* ``seed_features``: 32 inputs per seed: the volume at the 27 points seed + {-1, 0, 1}^3
  voxels (trilinear interpolation of the voxel-centre samples, zero outside) divided by
  vmax, then pos / E, then two zeros.
* ``merge_labels``: the label of each seed, from a fitted GMM Theta_fit: a mass-preserving
  coarse-graining of the fitted mixture onto the seeds.  Every fitted Gaussian g goes to
  its nearest seed k(g) (squared distance in FP32, ((dx dx + dy dy) + dz dz) with
  dx = mu_x - p_x, each step rounded; ties to the lower seed index).  Seed k then stands
  for the moment-matched merge of its Gaussians: mass A_k = sum A_g, offset
  delta_k = sum A_g (mu_g - p_k) / A_k and covariance
  C_k = sum A_g (Sigma_g + (mu_g - p_k)(mu_g - p_k)^T) / A_k - delta_k delta_k^T
  (Sigma = R S S^T R^T, Sec. 3.3.1 Eq. 5), all in FP64.  Its 10 numbers are delta_k / dv
  (3); the log-Cholesky factor of C_k / dv^2: log L00, log L11, log L22 clamped to
  [-6, 3], then L10, L20, L21 (6); the relative mass a_k = A_k K / M clamped to
  [0, 100] (1).  A seed that receives no Gaussian is labelled (0, 0, 0, log 1/2 x 3,
  0, 0, 0, 0): no offset, isotropic scale dv / 2, no mass.
* ``decode``: the inverse map from 10 predicted numbers to raw Theta[K, 11]: mu = pos +
  dv P[0:3]; Sigma = dv^2 L L^T; its eigen-decomposition Sigma = V diag(lambda) V^T with
  det V = +1 gives s = softplus^-1(sqrt(lambda)) and q = quaternion of V (the inverse of
  Sec. 3.3.1's R(q)); A = softplus^-1(M / K max(P[9], 1e-3)).
* The point-MLP: three layers, ReLU after the first two, params flat as
  W1[H][din], b1[H], W2[H][H], b2[H], W3[dout][H], b3[dout].  With ``bf16`` every product
  takes both operands rounded to bfloat16 (round to nearest even of the FP32 value) and
  accumulates exactly (FP64 here); biases and gradients stay unrounded.  The backward
  passes the rounding straight through.  The loss is the mean squared error over all
  outputs.
"""
from __future__ import annotations

import numpy as np
from scipy.spatial.transform import Rotation

F64 = np.float64
F32 = np.float32


# ----------------------------------------------------------------------------- bfloat16
def bf16_round(x):
    """Round to the nearest bfloat16 (ties to even) of the FP32 value of x; returns FP64."""
    u = np.ascontiguousarray(np.asarray(x, dtype=F32)).view(np.uint32).astype(np.uint64)
    lsb = (u >> np.uint64(16)) & np.uint64(1)
    r = ((u + np.uint64(0x7FFF) + lsb) & np.uint64(0xFFFF0000)).astype(np.uint32)
    return r.view(F32).astype(F64)


# ----------------------------------------------------------------------------- MLP
def mlp_slices(din, hidden, dout):
    """Offsets of W1, b1, W2, b2, W3, b3 in the flat parameter vector."""
    shapes = [(hidden, din), (hidden,), (hidden, hidden), (hidden,), (dout, hidden), (dout,)]
    out, off = [], 0
    for s in shapes:
        n = int(np.prod(s))
        out.append((off, s))
        off += n
    return out, off


def mlp_unpack(params, din, hidden, dout):
    sl, _ = mlp_slices(din, hidden, dout)
    p = np.asarray(params, dtype=F64)
    return [p[o:o + int(np.prod(s))].reshape(s) for o, s in sl]


def mlp_forward(params, X, din, hidden, dout, bf16=True):
    """Y[n, dout] and the cache (inputs and pre-activations of every layer)."""
    W1, b1, W2, b2, W3, b3 = mlp_unpack(params, din, hidden, dout)
    r = bf16_round if bf16 else (lambda a: np.asarray(a, dtype=F64))
    X = np.asarray(X, dtype=F64)
    Z1 = r(X) @ r(W1).T + b1
    H1 = np.maximum(Z1, 0.0)
    Z2 = r(H1) @ r(W2).T + b2
    H2 = np.maximum(Z2, 0.0)
    Y = r(H2) @ r(W3).T + b3
    return Y, (X, Z1, H1, Z2, H2)


def mlp_backward(params, cache, dY, din, hidden, dout, bf16=True):
    """Flat dL/dparams for upstream dY[n, dout] (rounding passed straight through)."""
    W1, b1, W2, b2, W3, b3 = mlp_unpack(params, din, hidden, dout)
    r = bf16_round if bf16 else (lambda a: np.asarray(a, dtype=F64))
    X, Z1, H1, Z2, H2 = cache
    dZ3 = np.asarray(dY, dtype=F64)
    dW3 = r(dZ3).T @ r(H2)
    db3 = dZ3.sum(0)
    dH2 = r(dZ3) @ r(W3)
    dZ2 = dH2 * (Z2 > 0)
    dW2 = r(dZ2).T @ r(H1)
    db2 = dZ2.sum(0)
    dH1 = r(dZ2) @ r(W2)
    dZ1 = dH1 * (Z1 > 0)
    dW1 = r(dZ1).T @ r(X)
    db1 = dZ1.sum(0)
    return np.concatenate([a.ravel() for a in (dW1, db1, dW2, db2, dW3, db3)])


def mse(Y, T):
    """Mean squared error over all elements and its gradient dL/dY."""
    R = np.asarray(Y, dtype=F64) - np.asarray(T, dtype=F64)
    return float(np.mean(R * R)), 2.0 * R / R.size


# ----------------------------------------------------------------------------- volume
def voxel_size(Dv, E=0.5):
    return F32(F32(2.0 * E) / F32(Dv))


def voxel_centres(Dv, E=0.5):
    """[Dv^3, 3] FP64 voxel centres (x, y, z) in [z][y][x] order."""
    dv = 2.0 * E / Dv
    c = -E + (np.arange(Dv) + 0.5) * dv
    z, y, x = np.meshgrid(c, c, c, indexing="ij")
    return np.stack([x.ravel(), y.ravel(), z.ravel()], -1)


def _bilinear(img, col, row):
    """Bilinear samples of img[D, D] at (column, row) arrays; zero outside the image."""
    D = img.shape[0]
    j0 = np.floor(col).astype(np.int64)
    i0 = np.floor(row).astype(np.int64)
    ax, ay = col - j0, row - i0
    out = np.zeros(np.shape(col), dtype=F64)
    for di, wy in ((0, 1.0 - ay), (1, ay)):
        for dj, wx in ((0, 1.0 - ax), (1, ax)):
            i, j = i0 + di, j0 + dj
            ok = (i >= 0) & (i < D) & (j >= 0) & (j < D)
            val = np.zeros(np.shape(col), dtype=F64)
            val[ok] = img[i[ok], j[ok]]
            out += wy * wx * val
    return out


def backproject(images, W, D, Dv, E=0.5):
    """vol[Dv, Dv, Dv] ([z][y][x]) = mean over particles of the box-filtered image at each
    voxel centre's projection (module docstring)."""
    images = np.asarray(images, dtype=F64)
    W = np.asarray(W, dtype=F64).reshape(-1, 3, 3)
    B = images.shape[0]
    h = 2.0 * E / D
    c = float(D // 2)
    f = max(1, D // Dv)
    offs = np.arange(f) - (f - 1) / 2.0
    r = voxel_centres(Dv, E)
    vol = np.zeros(r.shape[0], dtype=F64)
    for b in range(B):
        p = r @ W[b].T
        col = p[:, 0] / h + c
        row = c - p[:, 1] / h
        acc = np.zeros_like(vol)
        for oy in offs:
            for ox in offs:
                acc += _bilinear(images[b], col + ox, row + oy)
        vol += acc / (f * f)
    return (vol / max(B, 1)).reshape(Dv, Dv, Dv)


def mass_estimate(images, ctf, D, E=0.5):
    """Least-squares total amplitude from the images' DC terms (module docstring)."""
    images = np.asarray(images, dtype=F64)
    w = np.asarray(ctf, dtype=F64)[:, 3]
    S = images.reshape(images.shape[0], -1).sum(1)
    h = 2.0 * E / D
    return h * h * float(np.sum(-w * S)) / float(np.sum(w * w))


# ----------------------------------------------------------------------------- seeds
def seed_weights(vol):
    """Integer voxel weights q_v and vmax (module docstring)."""
    v = np.asarray(vol, dtype=F32).ravel()
    vmax = F32(v.max())
    if not vmax > 0:
        return np.ones(v.size, dtype=np.uint64), vmax
    ratio = (np.maximum(v, F32(0)) / vmax).astype(F32)  # correctly rounded FP32 division
    q = np.floor(ratio.astype(F64) * 2.0 ** 20).astype(np.uint64)
    return q, vmax


def seed_sample(vol, u, E=0.5):
    """(voxel index[K], pos[K, 3] float32, vmax) for uniforms u[K, 4] (module docstring)."""
    vol = np.asarray(vol, dtype=F32)
    Dv = vol.shape[0]
    u = np.asarray(u, dtype=F32)
    q, vmax = seed_weights(vol)
    C = np.cumsum(q)
    T = int(C[-1])
    K = u.shape[0]
    idx = np.empty(K, dtype=np.int64)
    for k in range(K):
        t = min(int(np.floor(F64(u[k, 0]) * F64(T))), T - 1)
        idx[k] = int(np.count_nonzero(C <= t))  # first voxel whose running sum exceeds t
    dv = voxel_size(Dv, E)
    xyz = np.stack([idx % Dv, (idx // Dv) % Dv, idx // (Dv * Dv)], -1).astype(F32)
    centre = ((xyz + F32(0.5)) * dv).astype(F32) + F32(-E)
    jitter = ((u[:, 1:4] + F32(-0.5)).astype(F32) * dv).astype(F32)
    pos = (centre.astype(F32) + jitter).astype(F32)
    return idx, pos, vmax


def trilinear(vol, x, y, z):
    """Trilinear interpolation of vol[z][y][x] at continuous voxel coordinates (voxel
    centres at integers); zero outside."""
    Dv = vol.shape[0]
    x, y, z = (np.asarray(a, dtype=F64) for a in (x, y, z))
    i0, j0, k0 = (np.floor(a).astype(np.int64) for a in (x, y, z))
    ax, ay, az = x - i0, y - j0, z - k0
    out = np.zeros(x.shape, dtype=F64)
    for dz in (0, 1):
        for dy in (0, 1):
            for dx in (0, 1):
                X, Y, Z = i0 + dx, j0 + dy, k0 + dz
                w = (ax if dx else 1 - ax) * (ay if dy else 1 - ay) * (az if dz else 1 - az)
                ok = (X >= 0) & (X < Dv) & (Y >= 0) & (Y < Dv) & (Z >= 0) & (Z < Dv)
                val = np.zeros(x.shape, dtype=F64)
                val[ok] = vol[Z[ok], Y[ok], X[ok]]
                out += w * val
    return out


def seed_features(vol, pos, vmax, E=0.5):
    """feats[K, 32] (module docstring)."""
    vol = np.asarray(vol, dtype=F64)
    Dv = vol.shape[0]
    pos = np.asarray(pos, dtype=F64)
    dv = 2.0 * E / Dv
    c = (pos + E) / dv - 0.5
    K = pos.shape[0]
    f = np.zeros((K, 32), dtype=F64)
    t = 0
    for dz in (-1, 0, 1):
        for dy in (-1, 0, 1):
            for dx in (-1, 0, 1):
                f[:, t] = trilinear(vol, c[:, 0] + dx, c[:, 1] + dy, c[:, 2] + dz) / float(vmax)
                t += 1
    f[:, 27:30] = pos / E
    return f


# ----------------------------------------------------------------------------- labels
def softplus(x):
    x = np.asarray(x, dtype=F64)
    return np.log1p(np.exp(-np.abs(x))) + np.maximum(x, 0.0)


def inv_softplus(y):
    y = np.asarray(y, dtype=F64)
    return np.where(y > 30.0, y, np.log(np.expm1(np.minimum(y, 30.0))))


def gaussian_covariance(theta):
    """Sigma = R S S^T R^T (Sec. 3.3.1 Eq. 5) of raw theta rows, FP64 [N, 3, 3]."""
    theta = np.asarray(theta, dtype=F64)
    q = theta[:, 6:10] / np.linalg.norm(theta[:, 6:10], axis=1, keepdims=True)
    w, x, y, z = q.T
    R = np.stack([
        np.stack([1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)], -1),
        np.stack([2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)], -1),
        np.stack([2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)], -1),
    ], -2)
    s = softplus(theta[:, 3:6])
    return np.einsum("nij,nj,nkj->nik", R, s * s, R)


def nearest(pos, mu):
    """Index of the nearest centre, distances in FP32 in the fixed order (module docstring)."""
    pos = np.asarray(pos, dtype=F32)
    mu = np.asarray(mu, dtype=F32)
    out = np.empty(pos.shape[0], dtype=np.int64)
    for k in range(pos.shape[0]):
        d = (mu - pos[k]).astype(F32)
        d2 = ((d[:, 0] * d[:, 0]).astype(F32) + (d[:, 1] * d[:, 1]).astype(F32)).astype(F32)
        d2 = (d2 + (d[:, 2] * d[:, 2]).astype(F32)).astype(F32)
        out[k] = int(np.argmin(d2))  # first minimum: ties go to the lower index
    return out


def cholesky3(S):
    """Lower Cholesky factors of SPD [n, 3, 3], written out entry by entry."""
    L = np.zeros_like(S)
    L[:, 0, 0] = np.sqrt(S[:, 0, 0])
    L[:, 1, 0] = S[:, 1, 0] / L[:, 0, 0]
    L[:, 2, 0] = S[:, 2, 0] / L[:, 0, 0]
    L[:, 1, 1] = np.sqrt(S[:, 1, 1] - L[:, 1, 0] ** 2)
    L[:, 2, 1] = (S[:, 2, 1] - L[:, 2, 0] * L[:, 1, 0]) / L[:, 1, 1]
    L[:, 2, 2] = np.sqrt(S[:, 2, 2] - L[:, 2, 0] ** 2 - L[:, 2, 1] ** 2)
    return L


EMPTY_LABEL = (0.0, 0.0, 0.0, float(np.log(0.5)), float(np.log(0.5)), float(np.log(0.5)), 0.0, 0.0, 0.0, 0.0)


def merge_moments(pos, theta_fit):
    """(assignment k(g) [N], mass [K], offset [K, 3], covariance [K, 3, 3]) of the
    coarse-graining onto the seeds (FP64; empty seeds have mass 0 and zero moments)."""
    pos = np.asarray(pos, dtype=F32)
    theta_fit = np.asarray(theta_fit, dtype=F32)
    K = pos.shape[0]
    k_of = nearest(theta_fit[:, 0:3], pos)
    A = softplus(theta_fit[:, 10].astype(F64))
    d = theta_fit[:, 0:3].astype(F64) - pos[k_of].astype(F64)
    Sig = gaussian_covariance(theta_fit)
    mass = np.zeros(K)
    first = np.zeros((K, 3))
    second = np.zeros((K, 3, 3))
    for g in range(theta_fit.shape[0]):
        k = k_of[g]
        mass[k] += A[g]
        first[k] += A[g] * d[g]
        second[k] += A[g] * (Sig[g] + np.outer(d[g], d[g]))
    offset = np.zeros((K, 3))
    cov = np.zeros((K, 3, 3))
    ok = mass > 0
    offset[ok] = first[ok] / mass[ok, None]
    cov[ok] = second[ok] / mass[ok, None, None] - np.einsum("ki,kj->kij", offset[ok], offset[ok])
    return k_of, mass, offset, cov


def merge_labels(pos, theta_fit, Dv, mass_total, E=0.5):
    """Labels[K, 10] of seeds ``pos`` against the fitted GMM ``theta_fit`` (module docstring)."""
    dv = 2.0 * E / Dv
    K = np.asarray(pos).shape[0]
    _, m, off, C = merge_moments(pos, theta_fit)
    lab = np.tile(np.asarray(EMPTY_LABEL), (K, 1))
    ok = m > 0
    if ok.any():
        L = cholesky3(C[ok] / (dv * dv))
        t = np.zeros((int(ok.sum()), 10))
        t[:, 0:3] = off[ok] / dv
        t[:, 3] = np.clip(np.log(L[:, 0, 0]), -6.0, 3.0)
        t[:, 4] = np.clip(np.log(L[:, 1, 1]), -6.0, 3.0)
        t[:, 5] = np.clip(np.log(L[:, 2, 2]), -6.0, 3.0)
        t[:, 6] = L[:, 1, 0]
        t[:, 7] = L[:, 2, 0]
        t[:, 8] = L[:, 2, 1]
        t[:, 9] = np.clip(m[ok] * K / mass_total, 0.0, 100.0)
        lab[ok] = t
    return lab


def decode(pos, pred, Dv, mass, E=0.5):
    """Raw Theta[K, 11] (FP64) from seeds and 10 predicted numbers each (module docstring)."""
    pos = np.asarray(pos, dtype=F64)
    P = np.asarray(pred, dtype=F64)
    K = pos.shape[0]
    dv = 2.0 * E / Dv
    th = np.zeros((K, 11), dtype=F64)
    th[:, 0:3] = pos + dv * P[:, 0:3]
    L = np.zeros((K, 3, 3), dtype=F64)
    L[:, 0, 0] = np.exp(np.clip(P[:, 3], -6.0, 3.0))
    L[:, 1, 1] = np.exp(np.clip(P[:, 4], -6.0, 3.0))
    L[:, 2, 2] = np.exp(np.clip(P[:, 5], -6.0, 3.0))
    L[:, 1, 0] = P[:, 6]
    L[:, 2, 0] = P[:, 7]
    L[:, 2, 1] = P[:, 8]
    S = dv * dv * np.einsum("nij,nkj->nik", L, L)
    lam, V = np.linalg.eigh(S)
    flip = np.linalg.det(V) < 0
    V[flip, :, 2] *= -1.0
    th[:, 3:6] = inv_softplus(np.sqrt(np.maximum(lam, 0.0)))
    xyzw = Rotation.from_matrix(V).as_quat()  # scalar last
    th[:, 6] = xyzw[:, 3]
    th[:, 7:10] = xyzw[:, 0:3]
    th[:, 10] = inv_softplus(mass / K * np.maximum(P[:, 9], 1e-3))
    return th


# ----------------------------------------------------------------------------- judging
def steps_to_reach(steps, losses, target):
    """First recorded step whose loss is at most ``target`` (None if never)."""
    for s, l in zip(steps, losses):
        if l <= target:
            return int(s)
    return None
