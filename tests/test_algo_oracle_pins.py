"""Pins of FourierShift and SplitGaussian (Algorithm 1) in the oracle (CPU only)."""
import numpy as np

import oracle as O
from oracle import algo_oracle as AO
from paper_2508_04929_b300 import synth

F64 = np.float64


def test_integer_shift_is_a_circular_roll():
    rng = np.random.default_rng(61)
    D = 16
    Y = rng.standard_normal((2, D, D))
    h = 1.0 / D
    t = np.array([[3 * h, -2 * h], [-5 * h, 4 * h]])
    out = AO.fourier_shift(Y, t)
    # +3 columns; t_y = -2 h moves the content 2 rows down (rows grow downward)
    assert np.allclose(out[0], np.roll(np.roll(Y[0], 3, axis=1), 2, axis=0), atol=1e-12)
    assert np.allclose(out[1], np.roll(np.roll(Y[1], -5, axis=1), -4, axis=0), atol=1e-12)


def test_shift_composes_and_inverts():
    rng = np.random.default_rng(62)
    D = 15
    Y = rng.standard_normal((1, D, D))
    a = np.array([[0.013, -0.021]])
    b = np.array([[-0.004, 0.017]])
    ab = AO.fourier_shift(AO.fourier_shift(Y, a), b)
    assert np.allclose(ab, AO.fourier_shift(Y, a + b), atol=1e-12)
    assert np.allclose(AO.fourier_shift(AO.fourier_shift(Y, a), -a), Y, atol=1e-12)


def test_subpixel_shift_moves_a_rendered_gaussian():
    """A well-sampled Gaussian image shifted by t equals the render of the Gaussian moved by
    t in the image plane (band-limited content, periodic grid far from the border)."""
    rng = synth.rng_for(63)
    D = 48
    th = synth.random_gaussians(1, D, rng, centre_radius=0.02, scale_px=(2.5, 3.0)).astype(F64)
    W = np.eye(3)
    t = np.array([[0.0137, -0.0093]])
    Q = O.render_one(th, W, D, cutoff=10.0)[None]
    moved = th.copy()
    moved[0, 0:2] += t[0]
    ref = O.render_one(moved, W, D, cutoff=10.0)
    assert np.max(np.abs(AO.fourier_shift(Q, t)[0] - ref)) <= 1e-6 * np.max(ref)


def test_split_preserves_mass_mean_and_covariance():
    rng = synth.rng_for(64)
    th = synth.random_gaussians(20, 64, rng).astype(F64)
    kids = AO.split_gaussians(th)
    p, c = O.build_gaussians(th), O.build_gaussians(kids)
    N = th.shape[0]
    A0, A1, A2 = p["A"], c["A"][:N], c["A"][N:]
    assert np.allclose(A1 + A2, A0, rtol=1e-12)
    m = (A1[:, None] * c["mu"][:N] + A2[:, None] * c["mu"][N:]) / A0[:, None]
    assert np.allclose(m, p["mu"], atol=1e-14)
    S = (A1[:, None, None] * (c["Sigma"][:N] + np.einsum("ni,nj->nij", c["mu"][:N] - m, c["mu"][:N] - m))
         + A2[:, None, None] * (c["Sigma"][N:] + np.einsum("ni,nj->nij", c["mu"][N:] - m, c["mu"][N:] - m))) / A0[:, None, None]
    assert np.allclose(S, p["Sigma"], rtol=1e-10, atol=1e-18)


def test_split_moves_along_the_major_axis():
    th = np.array([[0.1, 0.0, 0.0, np.log(np.expm1(0.01)), np.log(np.expm1(0.03)), np.log(np.expm1(0.02)),
                    1.0, 0.0, 0.0, 0.0, 0.0]])
    kids = AO.split_gaussians(th, alpha=0.5)
    assert np.allclose(kids[0, 0:3], [0.1, 0.015, 0.0]) and np.allclose(kids[1, 0:3], [0.1, -0.015, 0.0])
    s = np.log1p(np.exp(kids[:, 3:6]))
    assert np.allclose(s[:, 1], 0.03 * np.sqrt(0.75)) and np.allclose(s[:, [0, 2]], [0.01, 0.02])
