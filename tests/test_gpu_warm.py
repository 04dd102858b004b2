"""GPU parity of the learned warm start (point-MLP, backprojection, seeds, labels, decode)
against the FP64 oracle, and a test that the trained network beats the random start.

Tolerances.  The MLP rounds operands to bfloat16 on both sides; the GPU accumulates in
FP32 and rounds hidden activations from FP32 values, so a rounding can occasionally land
one bfloat16 step away from the oracle's (relative 2^-8 on one of 128 terms): outputs are
compared at relative L2 1e-4 and gradients at 1e-3 per parameter block.  Against central
finite differences of the unrounded FP64 network the bfloat16 operands themselves set the
gap (~2^-9 per operand): 3e-2.  Integer decisions (seed voxels, nearest Gaussian) are
taken in the same FP32/FP64 arithmetic on both sides and compared exactly.
"""
import numpy as np
import pytest
import torch

from oracle import warm_oracle as WO

pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("needs a GPU", allow_module_level=True)

from paper_2508_04929_b300 import _lib as L  # noqa: E402
from paper_2508_04929_b300 import synth  # noqa: E402
from paper_2508_04929_b300 import warmstart as WS  # noqa: E402

DEV = "cuda"


def rel(a, b):
    a, b = np.asarray(a, np.float64), np.asarray(b, np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def _t(x, dtype=torch.float32):
    return torch.from_numpy(np.ascontiguousarray(x)).to(DEV, dtype)


def _mlp_case(din, hid, dout, n, seed, with_idx):
    rng = np.random.default_rng(seed)
    _, npar = WO.mlp_slices(din, hid, dout)
    p = (rng.standard_normal(npar) * 0.3).astype(np.float32)
    rows = n + 17 if with_idx else n
    X = rng.standard_normal((rows, din)).astype(np.float32)
    T = rng.standard_normal((rows, dout)).astype(np.float32)
    idx = rng.permutation(rows)[:n].astype(np.int32) if with_idx else None
    return p, X, T, idx


@pytest.mark.parametrize("dims,n,with_idx", [((32, 128, 10), 300, True), ((5, 7, 3), 37, False),
                                             ((128, 128, 128), 130, True), ((32, 96, 10), 1, False)])
def test_mlp_forward_backward_matches_oracle(dims, n, with_idx):
    din, hid, dout = dims
    p, X, T, idx = _mlp_case(din, hid, dout, n, 1, with_idx)
    Xr = X[idx] if with_idx else X
    Tr = T[idx] if with_idx else T
    Y_o, cache = WO.mlp_forward(p, Xr, din, hid, dout, bf16=True)
    loss_o, dY_o = WO.mse(Y_o, Tr)
    g_o = WO.mlp_backward(p, cache, dY_o, din, hid, dout, bf16=True)

    params = _t(p)
    Xd, Td = _t(X), _t(T)
    idd = _t(idx, torch.int32) if with_idx else None
    acts = torch.empty(n * 4 * hid, device=DEV)
    Y = torch.empty((n, dout), device=DEV)
    L.gs_mlp_forward(params, dims, Xd, acts, Y, idx=idd)
    loss = torch.zeros(1, device=DEV)
    dY = torch.empty_like(Y)
    L.gs_mse(Y, Td, loss, dY, idx=idd)
    grad = torch.zeros_like(params)
    L.gs_mlp_backward(params, dims, Xd, acts, dY, grad, torch.empty(n * 2 * hid, device=DEV), idx=idd)
    torch.cuda.synchronize()
    assert rel(Y.cpu().numpy(), Y_o) <= 1e-4
    assert abs(float(loss) - loss_o) <= 1e-4 * loss_o
    g = grad.cpu().numpy()
    sl, _ = WO.mlp_slices(din, hid, dout)
    for off, shape in sl:
        k = int(np.prod(shape))
        assert rel(g[off:off + k], g_o[off:off + k]) <= 1e-3, (off, shape)


def test_mlp_gradient_against_fp64_finite_differences():
    """The kernels' gradient against central finite differences of the unrounded FP64
    network, every parameter.  The bfloat16 operands (8 significant bits) move the
    gradient by a few percent per block through the two ReLU layers (4-6% in L2 for this
    size, from the oracle with and without rounding), so the bound is 0.1 per block and a
    cosine of at least 0.995: the kernels descend the true loss."""
    din, hid, dout, n = 8, 16, 4, 48
    p, X, T, _ = _mlp_case(din, hid, dout, n, 2, False)
    params = _t(p)
    acts = torch.empty(n * 4 * hid, device=DEV)
    Y = torch.empty((n, dout), device=DEV)
    L.gs_mlp_forward(params, (din, hid, dout), _t(X), acts, Y)
    dY = torch.empty_like(Y)
    L.gs_mse(Y, _t(T), torch.zeros(1, device=DEV), dY)
    grad = torch.zeros_like(params)
    L.gs_mlp_backward(params, (din, hid, dout), _t(X), acts, dY, grad, torch.empty(n * 2 * hid, device=DEV))
    g = grad.cpu().numpy().astype(np.float64)

    def f(pp):
        return WO.mse(WO.mlp_forward(pp, X, din, hid, dout, bf16=False)[0], T)[0]

    p64 = p.astype(np.float64)
    eps = 1e-6
    fd = np.empty_like(p64)
    for i in range(p64.size):
        e = np.zeros_like(p64)
        e[i] = eps
        fd[i] = (f(p64 + e) - f(p64 - e)) / (2 * eps)
    sl, _ = WO.mlp_slices(din, hid, dout)
    for off, shape in sl:
        k = int(np.prod(shape))
        a, b = g[off:off + k], fd[off:off + k]
        assert rel(a, b) <= 0.1, (shape, rel(a, b))
        assert a @ b >= 0.995 * np.linalg.norm(a) * np.linalg.norm(b), shape


def test_mlp_training_fits_a_teacher():
    """Adam through the library's kernels drives a student network to a teacher's outputs."""
    din, hid, dout, n = 32, 128, 10, 4096
    rng = np.random.default_rng(4)
    teacher = (rng.standard_normal(WO.mlp_slices(din, hid, dout)[1]) * 0.2)
    X = rng.standard_normal((n, din)).astype(np.float32)
    T = WO.mlp_forward(teacher, X, din, hid, dout, bf16=False)[0].astype(np.float32)
    net = WS.PointMLP(hid, din, dout, seed=5, device=DEV)
    Xd, Td = _t(X), _t(T)
    first = float(net.evaluate(Xd, Td))
    gen = torch.Generator(device=DEV)
    gen.manual_seed(0)
    for _ in range(400):
        idx = torch.randint(0, n, (512,), generator=gen, device=DEV, dtype=torch.int32)
        net.train_step(Xd, Td, idx, 2e-3)
    last = float(net.evaluate(Xd, Td))
    assert last < 0.1 * first, (first, last)


def test_backprojection_and_mass_match_oracle():
    rng = np.random.default_rng(6)
    D, Dv, B = 64, 16, 6
    imgs = synth.smooth_field(B, D, rng) + np.float32(0.5)
    W = synth.random_poses(B, rng)
    ctf = synth.random_ctf(B, rng)
    vol_o = WO.backproject(imgs, W, D, Dv)
    vol = torch.empty((Dv, Dv, Dv), device=DEV)
    L.gs_backproject(_t(imgs), _t(W.reshape(B, 9)), Dv, vol)
    mass = torch.empty(1, device=DEV)
    L.gs_mass_estimate(_t(imgs), _t(ctf), torch.empty(2, dtype=torch.float64, device=DEV), mass)
    torch.cuda.synchronize()
    assert rel(vol.cpu().numpy(), vol_o) <= 1e-5
    m_o = WO.mass_estimate(imgs, ctf, D)
    assert abs(float(mass) - m_o) <= 1e-5 * abs(m_o)
    # ragged: Dv that does not divide D, a single particle
    vol_o = WO.backproject(imgs[:1], W[:1], D, 10)
    vol = torch.empty((10, 10, 10), device=DEV)
    L.gs_backproject(_t(imgs[:1]), _t(W[:1].reshape(1, 9)), 10, vol)
    torch.cuda.synchronize()
    assert rel(vol.cpu().numpy(), vol_o) <= 1e-5


@pytest.mark.parametrize("Dv,K", [(32, 5000), (7, 333), (16, 1)])
def test_seed_sampling_is_bit_exact(Dv, K):
    rng = np.random.default_rng(7 + Dv)
    vol = (rng.standard_normal((Dv, Dv, Dv)) + 0.5).astype(np.float32)
    u = rng.random((K, 4), dtype=np.float32)
    idx_o, pos_o, vmax_o = WO.seed_sample(vol, u)
    vd = _t(vol)
    cdf = torch.empty(Dv ** 3, dtype=torch.int64, device=DEV)
    vmax = torch.empty(1, device=DEV)
    pos = torch.empty((K, 3), device=DEV)
    vox = torch.empty(K, dtype=torch.int32, device=DEV)
    L.gs_seed_sample(vd, _t(u), cdf, vmax, pos, voxel=vox)
    feats = torch.empty((K, 32), device=DEV)
    L.gs_seed_features(vd, vmax, pos, feats)
    torch.cuda.synchronize()
    q, _ = WO.seed_weights(vol)
    assert np.array_equal(cdf.cpu().numpy().astype(np.uint64), np.cumsum(q))
    assert float(vmax) == float(vmax_o)
    assert np.array_equal(vox.cpu().numpy(), idx_o)
    assert np.array_equal(pos.cpu().numpy(), pos_o)
    f_o = WO.seed_features(vol, pos_o, vmax_o)
    assert rel(feats.cpu().numpy(), f_o) <= 1e-5


def test_seed_sampling_of_an_empty_volume_is_uniform():
    Dv, K = 8, 64
    vol = np.zeros((Dv, Dv, Dv), dtype=np.float32)
    u = np.random.default_rng(8).random((K, 4), dtype=np.float32)
    idx_o, pos_o, _ = WO.seed_sample(vol, u)
    cdf = torch.empty(Dv ** 3, dtype=torch.int64, device=DEV)
    vmax = torch.empty(1, device=DEV)
    pos = torch.empty((K, 3), device=DEV)
    L.gs_seed_sample(_t(vol), _t(u), cdf, vmax, pos)
    torch.cuda.synchronize()
    assert np.array_equal(pos.cpu().numpy(), pos_o)


def test_merge_labels_and_decode_match_oracle():
    rng = synth.rng_for(9)
    N, K, Dv = 3000, 1500, 32
    th = WS.unit_mass(synth.random_gaussians(N, 128, rng))
    pos = (th[rng.integers(0, N, K), 0:3] + rng.normal(0, 0.01, (K, 3))).astype(np.float32)
    mass_v = np.float32(1.3)
    k_o, m_o, _, _ = WO.merge_moments(pos, th)
    lab_o = WO.merge_labels(pos, th, Dv, float(mass_v))
    pd, md = _t(pos), _t(np.array([mass_v]))
    assign = torch.empty(N, dtype=torch.int32, device=DEV)
    lab = torch.empty((K, 10), device=DEV)
    L.gs_merge_labels(pd, _t(th), Dv, md, lab, assign=assign)
    torch.cuda.synchronize()
    assert np.array_equal(assign.cpu().numpy(), k_o)
    assert (m_o == 0).sum() > 10  # empty seeds are exercised
    assert rel(lab.cpu().numpy(), lab_o) <= 1e-6
    # decode labels perturbed like a network's output (covers every Jacobi / quaternion branch)
    pred = (lab_o + rng.normal(0, 0.3, lab_o.shape)).astype(np.float32)
    th_o = WO.decode(pos, pred, Dv, float(mass_v))
    out = torch.empty((K, 11), device=DEV)
    L.gs_decode_seeds(pd, _t(pred), Dv, md, out)
    torch.cuda.synchronize()
    got = out.cpu().numpy().astype(np.float64)
    assert rel(got[:, 0:3], th_o[:, 0:3]) <= 3e-7
    S_g, S_o = WO.gaussian_covariance(got), WO.gaussian_covariance(th_o)
    err = np.linalg.norm(S_g - S_o, axis=(1, 2)) / np.linalg.norm(S_o, axis=(1, 2))
    assert err.max() <= 1e-5
    assert rel(WO.softplus(got[:, 10]), WO.softplus(th_o[:, 10])) <= 2e-6
    assert np.allclose(np.linalg.norm(got[:, 6:10], axis=1), 1.0, atol=1e-6)


def test_merge_labels_without_fitted_gaussians():
    K = 5
    pos = torch.zeros((K, 3), device=DEV)
    lab = torch.empty((K, 10), device=DEV)
    L.gs_merge_labels(pos, torch.empty((0, 11), device=DEV), 32, torch.ones(1, device=DEV), lab)
    torch.cuda.synchronize()
    assert np.allclose(lab.cpu().numpy(), np.tile(np.asarray(WO.EMPTY_LABEL), (K, 1)), atol=1e-7)


@pytest.mark.slow
def test_learned_start_reaches_target_sooner_than_random():
    """Small version of the warm-start experiment: a network trained on plain fits of a
    few molecules must bring a held-out molecule's fit within 1% of the random-init
    converged loss in fewer Adam steps than the random init needs."""
    data = WS.build_dataset(10, D=64, N_range=(1000, 3000), P=128, batch=32, fit_steps=400, seed=11, device=DEV)
    net = WS.PointMLP(seed=0, device=DEV)
    WS.train(net, data, epochs=15, batch=2048, lr=2e-3)
    rng = np.random.default_rng(12)
    sp = WS.Splatter(64, 3000, 32, tile=8, chunk=128, device=DEV)
    mol = WS.simulate(sp, 2000, 192, rng, seed=99)
    res = WS.compare_starts(sp, mol, net, rng, steps=600, eval_every=20)
    r, w = res["random"]["steps_to_target"], res["learned"]["steps_to_target"]
    assert w is not None and (r is None or w < r), (r, w, res["target"])
