"""Seeded synthetic inputs shaped like the paper's workloads.

This module draws random inputs only: Gaussian parameters in the raw (pre-activation)
form, particle poses, CTF parameters and noise.  It holds none of the splatting method's
arithmetic and imports neither the CUDA path nor the oracle, so both can be fed the same
arrays.  Everything is NumPy with an explicit ``numpy.random.Generator`` (PCG64).

Recipe (the paper's EMPIAR and synthetic-80S data are not available; these stand in):

* centres uniform in a ball of radius 0.35 D pixels around the box centre;
* per-axis standard deviations log-uniform on [0.5, 3] pixels;
* rotations uniform unit quaternions (normalized 4-D normal draws);
* amplitudes log-normal(0, 0.5), taken as post-activation values;
* poses uniform on SO(3) (Haar measure, from the QR factorization of a normal matrix);
* CTF: defocus uniform on 1-3 um, 300 kV, Cs 2.7 mm, amplitude contrast 0.1, 1.5 A pixels;
* chain molecules (protein-backbone stand-in): random walks with 3.8 A steps that reflect
  at the 0.35 D ball, 500 steps per chain;
* the paper's initialization (Sec. 4.1): means N(0, 0.075^2), scale 0.0075, A = 1/(2N).

Raw parameters are the inverse of the activation the model applies (softplus for scales
and amplitudes), i.e. raw = v + log(-expm1(-v)) for a positive value v.
"""
from __future__ import annotations

import numpy as np

F32 = np.float32


def rng_for(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def inv_softplus(v):
    """Raw value whose softplus is v (v > 0)."""
    v = np.asarray(v, dtype=np.float64)
    return v + np.log(-np.expm1(-v))


def _unit_quaternions(n, rng):
    q = rng.standard_normal((n, 4))
    return q / np.linalg.norm(q, axis=1, keepdims=True)


def _ball(n, radius, rng):
    d = rng.standard_normal((n, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    r = radius * rng.random(n) ** (1.0 / 3.0)
    return d * r[:, None]


def random_gaussians(N, D, rng, E=0.5, centre_radius=0.35, scale_px=(0.5, 3.0),
                     amp_sigma=0.5):
    """Raw Theta[N, 11] (float32): [mu(3), s_raw(3), q(4), A_raw] in model units.

    Model units: the box spans [-E, E], so one pixel is h = 2E / D."""
    h = 2.0 * E / D
    mu = _ball(N, centre_radius * D * h, rng)
    lo, hi = np.log(scale_px[0]), np.log(scale_px[1])
    s_px = np.exp(rng.uniform(lo, hi, size=(N, 3)))
    q = _unit_quaternions(N, rng)
    A = np.exp(amp_sigma * rng.standard_normal(N))
    th = np.empty((N, 11), dtype=np.float64)
    th[:, 0:3] = mu
    th[:, 3:6] = inv_softplus(s_px * h)
    th[:, 6:10] = q
    th[:, 10] = inv_softplus(A)
    return th.astype(F32)


def chain_gaussians(N, D, rng, E=0.5, step_A=3.8, apix=1.5, chain_len=500,
                    centre_radius=0.35, scale_px=(0.5, 3.0), amp_sigma=0.5):
    """Raw Theta[N, 11] with centres on random-walk chains (3.8 A steps), reflected at the
    0.35 D ball: a protein-backbone-like clustering of the Gaussians."""
    h = 2.0 * E / D
    R = centre_radius * D * h
    step = step_A / apix * h
    mu = np.empty((N, 3))
    i = 0
    while i < N:
        p = _ball(1, R, rng)[0]
        for _ in range(min(chain_len, N - i)):
            mu[i] = p
            i += 1
            d = rng.standard_normal(3)
            p = p + step * d / np.linalg.norm(d)
            r = np.linalg.norm(p)
            if r > R:  # reflect back into the ball
                p = p * (2.0 * R - r) / r
    th = random_gaussians(N, D, rng, E, centre_radius, scale_px, amp_sigma).astype(np.float64)
    th[:, 0:3] = mu
    return th.astype(F32)


def paper_init(N, rng, E=0.5, spread=None, scale=None):
    """The paper's initialization (Sec. 4.1): means ~ N(0, (0.9 E / 6)^2) per axis, every
    scale 0.1 x that spread, amplitude 1 / (2N); rotations uniform."""
    spread = 0.9 * E / 6.0 if spread is None else spread
    scale = 0.1 * spread if scale is None else scale
    th = np.empty((N, 11), dtype=np.float64)
    th[:, 0:3] = spread * rng.standard_normal((N, 3))
    th[:, 3:6] = inv_softplus(np.full((N, 3), scale))
    th[:, 6:10] = _unit_quaternions(N, rng)
    th[:, 10] = inv_softplus(np.full(N, 1.0 / (2.0 * N)))
    return th.astype(F32)


def random_poses(B, rng):
    """W[B, 3, 3] (float32) uniform on SO(3): QR of a normal matrix with the sign fix."""
    out = np.empty((B, 3, 3))
    for b in range(B):
        Z = rng.standard_normal((3, 3))
        Qm, Rm = np.linalg.qr(Z)
        Qm = Qm * np.sign(np.diag(Rm))[None, :]
        if np.linalg.det(Qm) < 0:
            Qm[:, 0] = -Qm[:, 0]
        out[b] = Qm
    return out.astype(F32)


def random_ctf(B, rng, defocus_um=(1.0, 3.0), kv=300.0, cs_mm=2.7, w=0.1, apix=1.5):
    """ctf[B, 5] (float32) = (defocus_A, kV, Cs_mm, amplitude contrast, pixel size A)."""
    out = np.empty((B, 5))
    out[:, 0] = rng.uniform(defocus_um[0], defocus_um[1], size=B) * 1e4
    out[:, 1] = kv
    out[:, 2] = cs_mm
    out[:, 3] = w
    out[:, 4] = apix
    return out.astype(F32)


def add_noise(clean, snr, rng):
    """Observed images: clean + white Gaussian noise with variance var(clean) / snr, the
    variance taken over the whole batch."""
    clean = np.asarray(clean, dtype=np.float64)
    sigma = np.sqrt(np.var(clean) / snr)
    return (clean + sigma * rng.standard_normal(clean.shape)).astype(F32)


def smooth_field(B, D, rng, scale=1.0):
    """Arbitrary smooth real images[B, D, D] (float32), used as observed images or upstream
    gradients where only linearity matters."""
    x = rng.standard_normal((B, D, D))
    k = np.exp(-0.5 * (np.arange(-3, 4) / 1.5) ** 2)
    k /= k.sum()
    for ax in (1, 2):
        x = np.apply_along_axis(lambda v: np.convolve(np.concatenate([v[-3:], v, v[:3]]), k,
                                                      mode="valid"), ax, x)
    return (scale * x).astype(F32)
