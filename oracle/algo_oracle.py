"""FP64 oracle of the two remaining steps of the paper's Algorithm 1 (test infrastructure;
see package docstring): FourierShift of the observed images and SplitGaussian.

* ``fourier_shift``: Y_t(r) = Y(r - t), the image moved by t (model units) on the periodic
  pixel grid, by multiplying its DFT with exp(-2 pi i (m s_x + l s_y) / D), where (l, m) is the
  frequency index (row, column; signed, DFT order) and the shift in pixels is s_x = t_x / h
  along columns and s_y = -t_y / h along rows (rows grow downward, App. A.2 Eq. 13).  The
  phase factorizes into a column factor exp(-2 pi i m s_x / D) and a row factor; for even D
  the Nyquist index of each axis takes the Hermitian-symmetrized factor cos(pi s) (the mean
  of the +D/2 and -D/2 phases), so that the shift of a real image stays real and an integer
  shift is exactly a circular roll.  Algorithm 1 applies it with the published translations
  before Rasterize ("center alignment", Sec. 4.1).
* ``split_gaussians``: the paper's SplitGaussian (Algorithm 1, optional densification) gives
  no formula.  The reading here splits every Gaussian into two children placed at
  mu +- alpha s_max v along its major axis (v the column of R(q) of the largest scale s_max,
  the lower axis index on ties), each with amplitude A/2, the major scale reduced to
  s_max sqrt(1 - alpha^2) and the other scales and the rotation unchanged.  The pair keeps
  the parent's mass, mean and covariance exactly (a moment-preserving split).  Output order:
  the first children of all Gaussians, then the second children.
"""
from __future__ import annotations

import numpy as np

F64 = np.float64


def _axis_factor(D, shift):
    """exp(-2 pi i f shift / D) over the signed DFT indices f, cos(pi shift) at Nyquist."""
    f = np.fft.fftfreq(D, 1.0 / D)
    h = np.exp(-2j * np.pi * f * shift / D)
    if D % 2 == 0:
        h[D // 2] = np.cos(np.pi * shift)
    return h


def fourier_shift(images, t, E=0.5):
    """images[B, D, D], t[B, 2] (model units) -> shifted images[B, D, D] (FP64)."""
    Y = np.asarray(images, dtype=F64)
    t = np.asarray(t, dtype=F64).reshape(-1, 2)
    B, D, _ = Y.shape
    h = 2.0 * E / D
    out = np.empty_like(Y)
    for b in range(B):
        H = np.outer(_axis_factor(D, -t[b, 1] / h), _axis_factor(D, t[b, 0] / h))  # [row, column]
        out[b] = np.fft.ifft2(np.fft.fft2(Y[b]) * H).real
    return out


def _softplus(x):
    x = np.asarray(x, dtype=F64)
    return np.log1p(np.exp(-np.abs(x))) + np.maximum(x, 0.0)


def _inv_softplus(y):
    y = np.asarray(y, dtype=F64)
    return np.where(y > 30.0, y, np.log(np.expm1(np.minimum(y, 30.0))))


def split_gaussians(theta, alpha=0.5):
    """theta[N, 11] raw -> children[2N, 11] raw (FP64), module docstring."""
    th = np.asarray(theta, dtype=F64)
    N = th.shape[0]
    s = _softplus(th[:, 3:6])
    A = _softplus(th[:, 10])
    q = th[:, 6:10] / np.linalg.norm(th[:, 6:10], axis=1, keepdims=True)
    w, x, y, z = q.T
    R = np.stack([
        np.stack([1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)], -1),
        np.stack([2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)], -1),
        np.stack([2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)], -1),
    ], -2)
    m = np.argmax(s, axis=1)  # first maximum: the lower axis index on ties
    smax = s[np.arange(N), m]
    v = R[np.arange(N), :, m]
    out = np.repeat(th[None], 2, axis=0).copy()  # [2, N, 11]
    for c, sign in enumerate((1.0, -1.0)):
        out[c, :, 0:3] = th[:, 0:3] + sign * alpha * smax[:, None] * v
        out[c, np.arange(N), 3 + m] = _inv_softplus(smax * np.sqrt(1.0 - alpha * alpha))
        out[c, :, 10] = _inv_softplus(A / 2.0)
    return out.reshape(2 * N, 11)
