"""Pins of the voxelization / FSC oracle (CPU only).

The voxelized GMM is tied to the splatting oracle by the projection identity (sum over z of
the volume = the image rendered at W = I, the line integral of Sec. 3.3.3), to the total
amplitude by mass conservation, its boxes to an independent FP64 bound, and the FSC to the
identities any correlation coefficient obeys and to white-noise statistics.
"""
import numpy as np
from scipy.spatial.transform import Rotation

import oracle as O
from oracle import volume_oracle as VO
from paper_2508_04929_b300 import synth

F64 = np.float64


def _wide(n, D, rng, lo=1.5, hi=2.5, radius=0.12):
    return synth.random_gaussians(n, D, rng, centre_radius=radius, scale_px=(lo, hi))


def test_projection_along_z_is_the_rendered_image():
    rng = synth.rng_for(31)
    D, E = 32, 0.5
    th = _wide(4, D, rng).astype(F64)
    V = VO.voxelize(th, D, E, cutoff=6.0)
    Q = O.render_one(th, np.eye(3), D, E, cutoff=6.0)
    proj = V.sum(0) * (2 * E / D)
    assert np.max(np.abs(proj - Q)) <= 1e-7 * np.max(np.abs(Q))


def test_mass_is_total_amplitude():
    rng = synth.rng_for(32)
    D, E = 32, 0.5
    th = _wide(5, D, rng).astype(F64)
    V = VO.voxelize(th, D, E, cutoff=6.0)
    h = 2 * E / D
    total = float(np.sum(np.log1p(np.exp(th[:, 10]))))
    assert abs(V.sum() * h ** 3 - total) <= 1e-7 * total


def test_boxes_match_fp64_bounds_away_from_ties():
    rng = synth.rng_for(33)
    D, E, k = 48, 0.5, 3.0
    th = synth.random_gaussians(300, D, rng)
    box = VO.support3_fp32(th, D, E, k)
    t = th.astype(F64)
    s = np.log1p(np.exp(t[:, 3:6]))
    q = t[:, 6:10] / np.linalg.norm(t[:, 6:10], axis=1, keepdims=True)
    R = Rotation.from_quat(q[:, [1, 2, 3, 0]]).as_matrix()
    diag = np.einsum("nam,nm->na", R * R, s * s)
    h = 2 * E / D
    c = np.stack([t[:, 0] / h + D // 2, D // 2 - t[:, 1] / h, t[:, 2] / h + D // 2], -1)
    r = k * np.sqrt(diag) / h
    lo, hi = c - r, c + r
    clear = (np.abs(lo - np.round(lo)) > 1e-4) & (np.abs(hi - np.round(hi)) > 1e-4)
    ok = clear.all(1)
    assert ok.sum() > 250
    exp_lo = np.maximum(np.ceil(lo), 0).astype(np.int64)
    exp_hi = np.minimum(np.floor(hi), D - 1).astype(np.int64)
    assert np.array_equal(box[ok, :, 0], exp_lo[ok]) and np.array_equal(box[ok, :, 1], exp_hi[ok])


def test_fsc_identities():
    rng = np.random.default_rng(34)
    D = 16
    V = rng.standard_normal((D, D, D))
    assert np.allclose(VO.fsc(V, V), 1.0, atol=1e-12)
    assert np.allclose(VO.fsc(V, -V), -1.0, atol=1e-12)
    assert np.allclose(VO.fsc(V, 3.5 * V), 1.0, atol=1e-12)
    W = rng.standard_normal((D, D, D))
    f = VO.fsc(V, W)
    sh = VO.shell_index(D)
    counts = np.bincount(sh.ravel(), minlength=D // 2 + 2)[: D // 2 + 1]
    # independent white noise: |FSC| within ~4 standard errors (1/sqrt(shell size))
    assert np.all(np.abs(f[1:]) <= 4.0 / np.sqrt(counts[1:]))


def test_shell_index_is_nearest_integer_radius():
    D = 12
    sh = VO.shell_index(D)
    f = np.fft.fftfreq(D, 1.0 / D)
    kz, ky, kx = np.meshgrid(f, f, f, indexing="ij")
    ref = np.minimum(np.rint(np.sqrt(kx ** 2 + ky ** 2 + kz ** 2)).astype(np.int64), D // 2 + 1)
    assert np.array_equal(sh, ref)
    assert sh[0, 0, 0] == 0 and sh[0, 0, 1] == 1 and sh[1, 1, 1] == 2  # sqrt(3) rounds to 2
