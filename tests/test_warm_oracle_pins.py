"""Pins of the warm-start oracle (CPU only).

Each function of ``oracle.warm_oracle`` is checked against something other than itself:
torch's own bfloat16 conversion and linear layers, central finite differences, exact
integer arithmetic, closed forms of bilinear and trilinear interpolation on linear fields,
mass conservation of rendered splats, library routines (numpy searchsorted and Cholesky,
SciPy's k-d tree), statistics of the sampler, closed forms and invariants of moment
matching, and the label / decode round trip read back through the splatting oracle's own
Gaussian builder.
"""
import numpy as np
import pytest
import torch
from scipy.spatial import cKDTree
from scipy.spatial.transform import Rotation

import oracle as O
from oracle import warm_oracle as WO
from paper_2508_04929_b300 import synth

F64 = np.float64
F32 = np.float32


def _params(rng, din, hidden, dout, scale=0.5):
    _, n = WO.mlp_slices(din, hidden, dout)
    return rng.standard_normal(n) * scale


# ------------------------------------------------------------------------------ bf16 / MLP
def test_bf16_round_matches_torch():
    rng = np.random.default_rng(0)
    x = np.concatenate([rng.standard_normal(5000) * 10.0 ** rng.integers(-8, 8, 5000),
                        [0.0, -0.0, 1.0, 1.00390625, 1.005859375, 65504.0, 3.0e38]]).astype(F32)
    ref = torch.from_numpy(x).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(WO.bf16_round(x), ref)


def test_mlp_forward_matches_torch_linear():
    """bf16 off: the three layers are torch's linear / relu chain (W[out, in] layout)."""
    rng = np.random.default_rng(1)
    din, hid, dout, n = 6, 9, 4, 11
    p = _params(rng, din, hid, dout)
    X = rng.standard_normal((n, din))
    W1, b1, W2, b2, W3, b3 = (torch.from_numpy(a) for a in WO.mlp_unpack(p, din, hid, dout))
    F = torch.nn.functional
    ref = F.linear(F.relu(F.linear(F.relu(F.linear(torch.from_numpy(X), W1, b1)), W2, b2)), W3, b3).numpy()
    Y, _ = WO.mlp_forward(p, X, din, hid, dout, bf16=False)
    assert np.allclose(Y, ref, rtol=1e-13, atol=1e-13)


def test_mlp_backward_matches_finite_differences():
    rng = np.random.default_rng(2)
    din, hid, dout, n = 5, 7, 3, 6
    p = _params(rng, din, hid, dout)
    X = rng.standard_normal((n, din))
    T = rng.standard_normal((n, dout))

    def f(pp):
        Y, _ = WO.mlp_forward(pp, X, din, hid, dout, bf16=False)
        return WO.mse(Y, T)[0]

    Y, cache = WO.mlp_forward(p, X, din, hid, dout, bf16=False)
    _, dY = WO.mse(Y, T)
    g = WO.mlp_backward(p, cache, dY, din, hid, dout, bf16=False)
    eps = 1e-6
    fd = np.empty_like(p)
    for i in range(p.size):
        e = np.zeros_like(p)
        e[i] = eps
        fd[i] = (f(p + e) - f(p - e)) / (2 * eps)
    assert np.linalg.norm(g - fd) <= 1e-7 * np.linalg.norm(fd)
    # no ReLU sits on a kink at this seed (FD would be meaningless there)
    assert np.min(np.abs(cache[1])) > 1e-4 and np.min(np.abs(cache[3])) > 1e-4


def test_mlp_bf16_path_exact_on_representable_values():
    """With small integers everywhere every operand is a bfloat16, so the rounded path must
    equal the unrounded one exactly (forward and backward): the rounding is wired to
    operands only, never to accumulators or biases."""
    rng = np.random.default_rng(3)
    din, hid, dout, n = 3, 4, 2, 5
    _, npar = WO.mlp_slices(din, hid, dout)
    p = rng.integers(-1, 2, npar).astype(F64)
    X = rng.integers(0, 4, (n, din)).astype(F64)
    dY = rng.integers(-2, 3, (n, dout)).astype(F64)
    Ya, ca = WO.mlp_forward(p, X, din, hid, dout, bf16=True)
    Yb, cb = WO.mlp_forward(p, X, din, hid, dout, bf16=False)
    assert np.array_equal(Ya, Yb)
    assert np.array_equal(WO.mlp_backward(p, ca, dY, din, hid, dout, True),
                          WO.mlp_backward(p, cb, dY, din, hid, dout, False))


def test_mlp_bf16_rounding_is_applied():
    """A weight that is not a bfloat16 changes the output by exactly its rounding error."""
    din, hid, dout = 1, 1, 1
    p = np.array([1.0, 0.0, 1.0, 0.0, 1.0 + 2.0 ** -10, 0.0])  # W3 = 1 + 2^-10 rounds to 1
    X = np.array([[3.0]])
    Y, _ = WO.mlp_forward(p, X, din, hid, dout, bf16=True)
    Y0, _ = WO.mlp_forward(p, X, din, hid, dout, bf16=False)
    assert Y[0, 0] == 3.0 and Y0[0, 0] == 3.0 * (1.0 + 2.0 ** -10)


# ------------------------------------------------------------------------------ volume
def test_backprojection_of_linear_images_is_closed_form():
    """Bilinear sampling and the box stencil reproduce a linear image exactly, so a voxel
    whose stencil stays inside the image reads a (col + b row + c averaged over poses, with
    (col, row) = (p_x / h + D/2, D/2 - p_y / h), p = W r."""
    rng = np.random.default_rng(4)
    D, Dv, E = 40, 10, 0.5
    B = 3
    W = Rotation.random(B, random_state=5).as_matrix()
    coef = rng.standard_normal((B, 3))
    i, j = np.meshgrid(np.arange(D), np.arange(D), indexing="ij")
    imgs = np.stack([coef[b, 0] * j + coef[b, 1] * i + coef[b, 2] for b in range(B)])
    vol = WO.backproject(imgs, W, D, Dv, E).ravel()
    r = WO.voxel_centres(Dv, E)
    h = 2 * E / D
    expect = np.zeros(r.shape[0])
    inside = np.ones(r.shape[0], dtype=bool)
    f = D // Dv
    for b in range(B):
        p = r @ W[b].T
        col, row = p[:, 0] / h + D // 2, D // 2 - p[:, 1] / h
        expect += coef[b, 0] * col + coef[b, 1] * row + coef[b, 2]
        m = (f - 1) / 2 + 1e-9
        inside &= (col - m >= 0) & (col + m <= D - 1) & (row - m >= 0) & (row + m <= D - 1)
    expect /= B
    assert inside.sum() > 100
    assert np.allclose(vol[inside], expect[inside], rtol=0, atol=1e-11)
    # a voxel far outside every projection reads zero
    assert np.all(np.isfinite(vol))


def test_mass_estimate_recovers_total_amplitude():
    """DC of the CTF is -w (App. A.2 Eq. 14) and the splat conserves mass (Eq. 12): the
    estimate from CTF images of rendered Gaussians equals sum A."""
    rng = synth.rng_for(6)
    D, E = 48, 0.5
    th = synth.random_gaussians(5, D, rng, centre_radius=0.1, scale_px=(1.5, 2.5)).astype(F64)
    Ws = synth.random_poses(3, rng)
    ctf = synth.random_ctf(3, rng)
    Q = O.render(th, Ws, D, E, cutoff=6.0)
    X = np.stack([O.apply_ctf(Q[b], O.ctf_image(D, float(ctf[b, 0]), apix=float(ctf[b, 4]), w=float(ctf[b, 3])))
                  for b in range(3)])
    mass = WO.mass_estimate(X, ctf, D, E)
    total = float(np.sum(np.log1p(np.exp(th[:, 10]))))
    assert abs(mass - total) <= 1e-7 * total


# ------------------------------------------------------------------------------ seeds
def test_seed_sample_single_voxel():
    Dv, E = 8, 0.5
    vol = np.zeros((Dv, Dv, Dv), dtype=F32)
    vol[5, 2, 6] = 3.0
    vol[1, 1, 1] = -7.0  # negative density never draws
    u = np.random.default_rng(7).random((200, 4)).astype(F32)
    idx, pos, vmax = WO.seed_sample(vol, u, E)
    assert vmax == F32(3.0)
    assert np.all(idx == (5 * Dv + 2) * Dv + 6)
    dv = 2 * E / Dv
    lo = -E + np.array([6, 2, 5]) * dv
    assert np.all(pos >= lo - 1e-7) and np.all(pos <= lo + dv + 1e-7)


def test_seed_sample_matches_searchsorted_and_frequencies():
    rng = np.random.default_rng(8)
    Dv = 6
    vol = (rng.random((Dv, Dv, Dv)) - 0.3).astype(F32)
    u = rng.random((4000, 4)).astype(F32)
    idx, pos, vmax = WO.seed_sample(vol, u)
    q, _ = WO.seed_weights(vol)
    C = np.cumsum(q)
    t = np.minimum(np.floor(u[:, 0].astype(F64) * F64(C[-1])), C[-1] - 1)
    assert np.array_equal(idx, np.searchsorted(C, t, side="right"))
    # frequencies follow max(vol, 0) (binomial 5-sigma band)
    p = np.maximum(vol.ravel().astype(F64), 0) / np.maximum(vol.ravel().astype(F64), 0).sum()
    cnt = np.bincount(idx, minlength=Dv ** 3)
    sd = np.sqrt(4000 * p * (1 - p)) + 1e-9
    assert np.all(np.abs(cnt - 4000 * p) <= 5 * sd + 1)
    # each seed lies in its voxel
    dv = 1.0 / Dv
    xyz = np.stack([idx % Dv, (idx // Dv) % Dv, idx // Dv ** 2], -1)
    assert np.all(np.abs(pos - (-0.5 + (xyz + 0.5) * dv)) <= dv / 2 + 1e-6)


def test_seed_features_on_linear_volume():
    """Trilinear interpolation reproduces a linear field; the features are that field at
    the 27 stencil points over vmax, then pos / E."""
    Dv, E = 12, 0.5
    a = np.array([0.3, -0.2, 0.5])
    z, y, x = np.meshgrid(np.arange(Dv), np.arange(Dv), np.arange(Dv), indexing="ij")
    vol = (a[0] * x + a[1] * y + a[2] * z + 2.0).astype(F64)
    vmax = vol.max()
    rng = np.random.default_rng(9)
    pos = (rng.random((50, 3)) - 0.5) * 0.5  # stencil stays inside
    f = WO.seed_features(vol, pos, vmax, E)
    dv = 2 * E / Dv
    c = (pos + E) / dv - 0.5
    t = 0
    for dz in (-1, 0, 1):
        for dy in (-1, 0, 1):
            for dx in (-1, 0, 1):
                ref = (a[0] * (c[:, 0] + dx) + a[1] * (c[:, 1] + dy) + a[2] * (c[:, 2] + dz) + 2.0) / vmax
                assert np.allclose(f[:, t], ref, atol=1e-12)
                t += 1
    assert np.allclose(f[:, 27:30], pos / E) and np.all(f[:, 30:] == 0)


# ------------------------------------------------------------------------------ labels
def test_nearest_matches_kdtree():
    rng = np.random.default_rng(10)
    mu = (rng.random((300, 3)) - 0.5).astype(F32)
    pos = (rng.random((200, 3)) - 0.5).astype(F32)
    g = WO.nearest(pos, mu)
    d, ref = cKDTree(mu.astype(F64)).query(pos.astype(F64), k=2)
    clear = (d[:, 1] - d[:, 0]) > 1e-5  # no near tie that FP32 could break either way
    assert clear.sum() > 190
    assert np.array_equal(g[clear], ref[clear, 0])


def test_cholesky3_matches_numpy():
    rng = np.random.default_rng(11)
    A = rng.standard_normal((20, 3, 3))
    S = A @ A.transpose(0, 2, 1) + 0.1 * np.eye(3)
    assert np.allclose(WO.cholesky3(S), np.linalg.cholesky(S), atol=1e-13)


def _separated_gmm(rng, K, D=128):
    """K Gaussians whose centres are at least 0.05 apart, and seeds within 1e-3 of them
    (so every Gaussian's nearest seed is its own)."""
    th = synth.random_gaussians(4 * K, D, rng).astype(F64)
    keep = []
    for i in range(th.shape[0]):
        if all(np.linalg.norm(th[i, 0:3] - th[j, 0:3]) > 0.05 for j in keep):
            keep.append(i)
        if len(keep) == K:
            break
    th = th[keep]
    pos = (th[:, 0:3] + rng.uniform(-1e-3, 1e-3, (len(keep), 3))).astype(F32)
    return th, pos


def test_merge_of_one_gaussian_per_seed_round_trips():
    """With one Gaussian per seed the merge is that Gaussian, and decode(label) rebuilds
    it: centres, covariances (read back by the splatting oracle's BuildGaussians,
    Sec. 3.3.1) and amplitudes."""
    rng = synth.rng_for(12)
    Dv, E = 32, 0.5
    th, pos = _separated_gmm(rng, 40)
    K = pos.shape[0]
    mass = 3.7
    lab = WO.merge_labels(pos, th, Dv, mass, E)
    back = WO.decode(pos, lab, Dv, mass, E)
    g0, g1 = O.build_gaussians(th), O.build_gaussians(back)
    assert np.allclose(g1["mu"], g0["mu"], atol=1e-14)
    assert np.allclose(g1["Sigma"], g0["Sigma"], rtol=1e-9, atol=1e-16)
    assert np.allclose(g1["A"], g0["A"], rtol=1e-12)
    assert np.allclose(lab[:, 9], g0["A"] * K / mass, rtol=1e-12)
    Rm = O.quat_to_rot(back[:, 6:10] / np.linalg.norm(back[:, 6:10], axis=1, keepdims=True))
    assert np.allclose(np.linalg.det(Rm), 1.0)


def test_merge_of_two_gaussians_is_closed_form():
    """Two equal isotropic Gaussians at p +- a e_x merged onto a seed at p: no offset,
    covariance sigma^2 I + diag(a^2, 0, 0), mass 2A; a far seed receives nothing and gets
    the empty label."""
    Dv, E, a, sig = 16, 0.5, 0.01, 0.004
    dv = 2 * E / Dv
    sp_raw = float(synth.inv_softplus(np.array(sig)))
    A_raw = float(synth.inv_softplus(np.array(0.2)))
    th = np.array([[a, 0, 0, sp_raw, sp_raw, sp_raw, 1, 0, 0, 0, A_raw],
                   [-a, 0, 0, sp_raw, sp_raw, sp_raw, 0.6, 0.8, 0, 0, A_raw]])
    pos = np.array([[0.0, 0.0, 0.0], [0.3, 0.3, 0.3]], dtype=F32)
    lab = WO.merge_labels(pos, th.astype(F32), Dv, 1.0, E)
    C = (np.diag([a * a, 0, 0]) + sig * sig * np.eye(3)) / dv ** 2
    Lc = np.linalg.cholesky(C)
    assert np.allclose(lab[0, 0:3], 0.0, atol=1e-6)
    assert np.allclose(lab[0, 3:6], np.log(np.diag(Lc)), atol=1e-5)
    assert np.allclose(lab[0, 6:9], [Lc[1, 0], Lc[2, 0], Lc[2, 1]], atol=1e-6)
    assert np.isclose(lab[0, 9], 2 * 0.2 * 2 / 1.0, rtol=1e-6)
    assert np.array_equal(lab[1], np.asarray(WO.EMPTY_LABEL))


def test_merge_preserves_mass_and_first_two_moments():
    """Moment matching keeps the mixture's total mass, mass-weighted mean and second
    moment (every fitted Gaussian lands on exactly one seed)."""
    rng = synth.rng_for(14)
    th = synth.random_gaussians(300, 64, rng)
    pos = (rng.uniform(-0.3, 0.3, (50, 3))).astype(F32)
    k_of, m, off, C = WO.merge_moments(pos, th)
    A = np.log1p(np.exp(th[:, 10].astype(F64)))
    mu = th[:, 0:3].astype(F64)
    Sig = np.stack([_indep_cov(r) for r in th])
    centre = pos.astype(F64) + off
    assert np.isclose(m.sum(), A.sum(), rtol=1e-13)
    assert np.allclose((m[:, None] * centre).sum(0), (A[:, None] * mu).sum(0), atol=1e-13)
    lhs = np.einsum("k,kij->ij", m, C + np.einsum("ki,kj->kij", centre, centre))
    rhs = np.einsum("g,gij->ij", A, Sig + np.einsum("gi,gj->gij", mu, mu))
    assert np.allclose(lhs, rhs, rtol=1e-11, atol=1e-15)
    assert (m == 0).sum() > 0  # some seeds are empty in this draw


def _indep_cov(row):
    th = np.asarray(row, dtype=F64)
    s = np.log1p(np.exp(th[3:6]))
    q = th[6:10] / np.linalg.norm(th[6:10])
    R = Rotation.from_quat([q[1], q[2], q[3], q[0]]).as_matrix()
    return R @ np.diag(s * s) @ R.T


def test_steps_to_reach():
    assert WO.steps_to_reach([0, 10, 20, 30], [5.0, 3.0, 1.0, 0.5], 1.0) == 20
    assert WO.steps_to_reach([0, 10], [5.0, 3.0], 1.0) is None
