"""Pins of the pose-gradient oracle: central finite differences of the FP64 render (CPU).

The loss is the linear functional L = sum dL/dQ . Q, whose gradient is exactly the chain the
oracle forms.  Support boxes are frozen at the base point (a box edge moving under the
perturbation would add a jump that finite differences cannot see past).
"""
import numpy as np
from scipy.spatial.transform import Rotation

import oracle as O
from oracle import pose_oracle as PO
from paper_2508_04929_b300 import synth

F64 = np.float64
F32 = np.float32


def _setup(seed, N=12, D=24, B=2):
    rng = synth.rng_for(seed)
    th = synth.random_gaussians(N, D, rng, centre_radius=0.25, scale_px=(1.0, 2.5)).astype(F64)
    Ws = Rotation.random(B, random_state=seed).as_matrix()
    G = rng.standard_normal((B, D, D))
    boxes = [O.support_fp32(th.astype(F32), Ws[b].astype(F32), D)[:4] for b in range(B)]
    return th, Ws, G, boxes, D


def _L(th, Ws, G, boxes, D):
    return sum(float(np.sum(G[b] * O.render_one(th, Ws[b], D, box=boxes[b]))) for b in range(len(Ws)))


def test_dW_matches_central_differences():
    th, Ws, G, boxes, D = _setup(41)
    dW, _ = PO.pose_backward(th, Ws, D, G, boxes=boxes)
    eps = 1e-6
    fd = np.zeros_like(dW)
    for b in range(Ws.shape[0]):
        for i in range(3):
            for j in range(3):
                Wp, Wm = Ws.copy(), Ws.copy()
                Wp[b, i, j] += eps
                Wm[b, i, j] -= eps
                fd[b, i, j] = (_L(th, Wp, G, boxes, D) - _L(th, Wm, G, boxes, D)) / (2 * eps)
    assert np.linalg.norm(dW - fd) <= 1e-6 * np.linalg.norm(fd)
    assert np.allclose(dW[:, 2, :], fd[:, 2, :], atol=1e-9)  # the depth row contributes nothing


def test_dt_matches_central_differences():
    """A shift t of the model image is mu -> mu + W^T [t; 0] for every Gaussian."""
    th, Ws, G, boxes, D = _setup(42, B=1)
    _, dt = PO.pose_backward(th, Ws, D, G, boxes=boxes)
    eps = 1e-6
    for a in range(2):
        e = np.zeros(3)
        e[a] = eps
        shift = Ws[0].T @ e
        tp, tm = th.copy(), th.copy()
        tp[:, 0:3] += shift
        tm[:, 0:3] -= shift
        fd = (_L(tp, Ws, G, boxes, D) - _L(tm, Ws, G, boxes, D)) / (2 * eps)
        assert abs(dt[0, a] - fd) <= 1e-6 * max(abs(fd), 1e-12)


def test_dt_of_a_column_ramp_is_the_mass_over_h_cubed():
    """With dL/dQ = column index j, L = sum_g A_g (mu_tilde_x / h + floor(D/2)) / h^2 (the
    normalized splat's mean column, Eq. 12, for Gaussians inside the image), so
    dL/dt_x = sum A / h^3 and dL/dt_y = 0 exactly (Poisson error ~1e-19 at these widths)."""
    rng = synth.rng_for(43)
    D, E = 48, 0.5
    h = 2 * E / D
    th = synth.random_gaussians(6, D, rng, centre_radius=0.05, scale_px=(1.5, 2.0)).astype(F64)
    W = Rotation.random(1, random_state=7).as_matrix()
    G = np.tile(np.arange(D, dtype=F64), (D, 1))[None]
    _, dt = PO.pose_backward(th, W, D, G, cutoff=8.0)
    total = float(np.sum(np.log1p(np.exp(th[:, 10]))))
    assert abs(dt[0, 0] - total / h ** 3) <= 1e-9 * total / h ** 3
    assert abs(dt[0, 1]) <= 1e-9 * total / h ** 3
