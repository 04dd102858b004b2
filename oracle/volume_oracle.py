"""FP64 oracle of GMM voxelization and Fourier shell correlation (test infrastructure; see
package docstring).

The paper (arXiv 2508.04929) judges its reconstructions by half-map FSC of the GMM evaluated
on a voxel grid (Sec. 4, "Evaluation"); it gives no formula for either step.  The definitions
below are the library's own:

* ``voxelize``: V[k][i][j] (k slowest) = sum_g A_g N(r; mu_g, Sigma_g), the normalized 3-D
  Gaussian density of Eq. 4 with Sigma = R S S^T R^T (Sec. 3.3.1 Eq. 5), at the voxel centres
  r = ((j - floor(D/2)) h, -(i - floor(D/2)) h, (k - floor(D/2)) h), h = 2E/D: the grid of
  App. A.2 Eq. 13 extended along z, so that sum_k V[k] h is the image rendered with W = I.
  A Gaussian contributes only inside its k-sigma box
  [ceil(c - r), floor(c + r)] per axis (c the centre in voxel units, r = k sqrt(Sigma_aa) / h),
  clipped to the grid; the box is decided in FP32 by the sequence of correctly rounded
  operations of ``support3_fp32`` (the kernel's).
* ``fsc``: FSC(s) = Re sum F1 conj(F2) / sqrt(sum |F1|^2 sum |F2|^2) over the Fourier
  coefficients of shell s, the shell of frequency index (kx, ky, kz) (signed, DFT order) being
  the integer nearest to |k| (never a tie: |k|^2 is an integer), for s = 0 .. D/2.
"""
from __future__ import annotations

import numpy as np

F64 = np.float64
F32 = np.float32


def _activate(theta):
    th = np.asarray(theta, dtype=F64)
    A = np.log1p(np.exp(-np.abs(th[:, 10]))) + np.maximum(th[:, 10], 0.0)
    s = np.log1p(np.exp(-np.abs(th[:, 3:6]))) + np.maximum(th[:, 3:6], 0.0)
    q = th[:, 6:10] / np.linalg.norm(th[:, 6:10], axis=1, keepdims=True)
    w, x, y, z = q.T
    R = np.stack([
        np.stack([1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)], -1),
        np.stack([2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)], -1),
        np.stack([2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)], -1),
    ], -2)
    return th[:, 0:3], R, s, A


def _sp32(x32):
    """Correctly rounded FP32 softplus (computed in FP64, rounded once)."""
    x = np.asarray(x32, dtype=F64)
    return (np.log1p(np.exp(-np.abs(x))) + np.maximum(x, 0.0)).astype(F32)


def support3_fp32(theta, D, E=0.5, cutoff=3.0):
    """Per-axis k-sigma voxel boxes [N, 3, 2] (lo, hi; lo > hi = empty), decided in FP32.

    Sequence (every step rounded to FP32): s = fl32(softplus), q normalized by its FP32 norm
    ((w w + x x) + y y) + z z, the diagonal of Sigma as sum_m (R_am s_m)^2 accumulated in the
    order m = 0, 1, 2 with R_am from the FP32 quaternion formulas, c_x = mu_x / h + floor(D/2),
    c_y = floor(D/2) - mu_y / h, c_z = mu_z / h + floor(D/2) (each a multiply by 1/h = fl32(D /
    2E) then an add), r_a = k * (sqrt(Sigma_aa) * (1/h)), lo = max(ceil(c - r), 0),
    hi = min(floor(c + r), D - 1)."""
    th = np.asarray(theta, dtype=F32)
    inv_h = F32(F32(D) / F32(2.0 * E))
    k = F32(cutoff)
    s = _sp32(th[:, 3:6])
    qw, qx, qy, qz = (th[:, 6 + i] for i in range(4))
    n2 = (((qw * qw).astype(F32) + (qx * qx).astype(F32)).astype(F32) + (qy * qy).astype(F32)).astype(F32)
    n2 = (n2 + (qz * qz).astype(F32)).astype(F32)
    nr = np.sqrt(n2).astype(F32)
    w, x, y, z = ((a / nr).astype(F32) for a in (qw, qx, qy, qz))
    m = lambda a, b: (a * b).astype(F32)  # noqa: E731
    ad = lambda a, b: (a + b).astype(F32)  # noqa: E731
    sb = lambda a, b: (a - b).astype(F32)  # noqa: E731
    two = F32(2.0)
    one = F32(1.0)
    R = [[sb(one, m(two, ad(m(y, y), m(z, z)))), m(two, sb(m(x, y), m(w, z))), m(two, ad(m(x, z), m(w, y)))],
         [m(two, ad(m(x, y), m(w, z))), sb(one, m(two, ad(m(x, x), m(z, z)))), m(two, sb(m(y, z), m(w, x)))],
         [m(two, sb(m(x, z), m(w, y))), m(two, ad(m(y, z), m(w, x))), sb(one, m(two, ad(m(x, x), m(y, y))))]]
    c0 = F32(D // 2)
    out = np.empty((th.shape[0], 3, 2), dtype=np.int64)
    for a in range(3):
        v0 = m(R[a][0], s[:, 0])
        v1 = m(R[a][1], s[:, 1])
        v2 = m(R[a][2], s[:, 2])
        saa = ad(ad(m(v0, v0), m(v1, v1)), m(v2, v2))
        r = m(k, m(np.sqrt(saa).astype(F32), inv_h))
        if a == 1:
            c = sb(c0, m(th[:, 1], inv_h))
        else:
            c = ad(m(th[:, a], inv_h), c0)
        lo = np.maximum(np.ceil(sb(c, r)), F32(0)).astype(np.int64)
        hi = np.minimum(np.floor(ad(c, r)), F32(D - 1)).astype(np.int64)
        out[:, a, 0] = lo
        out[:, a, 1] = hi
    return out  # axis 0: x (columns j), 1: y (rows i), 2: z (slices k)


def voxel_centres(D, E=0.5):
    """(x[j], y[i], z[k]) coordinate vectors of the voxel grid."""
    h = 2.0 * E / D
    idx = np.arange(D) - D // 2
    return idx * h, -idx * h, idx * h


def voxelize(theta, D, E=0.5, cutoff=3.0):
    """V[D, D, D] (k, i, j) in FP64 (module docstring)."""
    mu, R, s, A = _activate(theta)
    box = support3_fp32(theta, D, E, cutoff)
    xs, ys, zs = voxel_centres(D, E)
    V = np.zeros((D, D, D), dtype=F64)
    norm = A / ((2 * np.pi) ** 1.5 * s[:, 0] * s[:, 1] * s[:, 2])
    for g in range(mu.shape[0]):
        (j0, j1), (i0, i1), (k0, k1) = box[g]
        if j0 > j1 or i0 > i1 or k0 > k1:
            continue
        zz, yy, xx = np.meshgrid(zs[k0:k1 + 1], ys[i0:i1 + 1], xs[j0:j1 + 1], indexing="ij")
        d = np.stack([xx - mu[g, 0], yy - mu[g, 1], zz - mu[g, 2]], -1)
        u = d @ R[g] / s[g]  # coordinates in the Gaussian's frame, in units of its scales
        V[k0:k1 + 1, i0:i1 + 1, j0:j1 + 1] += norm[g] * np.exp(-0.5 * np.sum(u * u, -1))
    return V


def shell_index(D):
    """Shell of every coefficient of the full DFT grid (k, i, j), as in the module docstring;
    D // 2 + 1 marks coefficients beyond the last shell."""
    f = np.fft.fftfreq(D, 1.0 / D).astype(np.int64)
    kz, ky, kx = np.meshgrid(f, f, f, indexing="ij")
    k2 = kx * kx + ky * ky + kz * kz
    r = np.floor(np.sqrt(k2.astype(F64))).astype(np.int64)
    r = np.where(r * r > k2, r - 1, r)
    r = np.where((r + 1) * (r + 1) <= k2, r + 1, r)  # r = floor(sqrt(k2)) exactly
    r = np.where(k2 > r * r + r, r + 1, r)  # nearest integer to sqrt(k2)
    return np.minimum(r, D // 2 + 1)


def fsc(V1, V2):
    """FSC[D // 2 + 1] of two D^3 volumes (module docstring), from the full FP64 DFT."""
    V1 = np.asarray(V1, dtype=F64)
    V2 = np.asarray(V2, dtype=F64)
    D = V1.shape[0]
    F1 = np.fft.fftn(V1)
    F2 = np.fft.fftn(V2)
    sh = shell_index(D)
    n = D // 2 + 1
    num = np.bincount(sh.ravel(), weights=np.real(F1 * np.conj(F2)).ravel(), minlength=n + 1)[:n]
    d1 = np.bincount(sh.ravel(), weights=(np.abs(F1) ** 2).ravel(), minlength=n + 1)[:n]
    d2 = np.bincount(sh.ravel(), weights=(np.abs(F2) ** 2).ravel(), minlength=n + 1)[:n]
    with np.errstate(invalid="ignore", divide="ignore"):
        return num / np.sqrt(d1 * d2)
