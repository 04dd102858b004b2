"""Parity of the CUDA path (through the C-ABI) with the FP64 oracle.

Tolerances: images (Q, X) relative L2 <= 1e-5 per image; gradients relative L2 <= 1e-3
per parameter group (mu, s, q, A) over all Gaussians; integer work (support boxes, tile
pairs, ranges) bit-exact.  Inputs are seeded synthetic batches shaped like the paper's
workloads (paper_2508_04929_b300.synth).
"""
import numpy as np
import pytest

import oracle as O
from paper_2508_04929_b300 import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2508_04929_b300 import build  # noqa: E402

build.build()
from paper_2508_04929_b300 import _lib as L  # noqa: E402
from paper_2508_04929_b300.splat import Splatter  # noqa: E402

DEV = "cuda"
GROUPS = (("mu", slice(0, 3)), ("s", slice(3, 6)), ("q", slice(6, 10)), ("A", slice(10, 11)))


def rel_l2(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def make_batch(seed, D, N, B, snr=0.1, chains=False):
    rng = synth.rng_for(seed)
    th = (synth.chain_gaussians if chains else synth.random_gaussians)(N, D, rng)
    Ws = synth.random_poses(B, rng)
    ctf = synth.random_ctf(B, rng)
    ref = synth.random_gaussians(N, D, rng)
    clean = []
    for b in range(B):
        H = O.ctf_image(D, *[float(v) for v in ctf[b, 0:4]], apix=float(ctf[b, 4]))
        clean.append(O.apply_ctf(O.render_one(ref, Ws[b], D), H))
    Y = synth.add_noise(np.stack(clean), snr, rng)
    return th, Ws, ctf, Y


def to_dev(*arrs):
    return [torch.from_numpy(np.ascontiguousarray(a)).to(DEV) for a in arrs]


def records(sp):
    raw = sp.proj[: sp.B * sp.N * 32].view(torch.float32).view(sp.B, sp.N, 8).cpu()
    f = raw.numpy()
    box = raw.view(torch.int16).view(sp.B, sp.N, 16)[:, :, 12:16].numpy().astype(np.int64)
    return f, box


def cuda_step(th, Ws, ctf, Y, D, tile=16, chunk=128, reduction=0):
    N, B = th.shape[0], Ws.shape[0]
    sp = Splatter(D, N, B, tile=tile, chunk=chunk, reduction=reduction)
    t, W, c, y = to_dev(th, Ws.reshape(B, 9), ctf, Y)
    dth = torch.zeros_like(t)
    loss = sp.forward_backward(t, W, c, y, dth)
    torch.cuda.synchronize()
    out = dict(Q=sp.Q.cpu().numpy(), X=sp.X.cpu().numpy(), L=loss.cpu().numpy(), dX=sp.dX.cpu().numpy(),
               dQ=sp.dQ.cpu().numpy(), dtheta=dth.cpu().numpy(), status=sp.status(),
               n_pairs=int(sp.n_pairs.item()) & 0xFFFFFFFF,
               pairs=sp.pairs.cpu().numpy().view(np.uint32), ranges=sp.ranges.cpu().numpy().view(np.uint32))
    out["rec"], out["box"] = records(sp)
    sp.close()
    return out


@pytest.fixture(scope="module")
def c1():
    """Config 1: D = 64, N = 2000, B = 8, SNR 0.1, seed 0."""
    th, Ws, ctf, Y = make_batch(0, 64, 2000, 8)
    ref = O.forward_backward(th, Ws, 64, Y, ctf)
    return th, Ws, ctf, Y, ref


def test_support_boxes_and_centres_bit_exact(c1):
    th, Ws, ctf, Y, _ = c1
    out = cuda_step(th, Ws, ctf, Y, 64)
    for b in range(Ws.shape[0]):
        x0, x1, y0, y1, bad, cx, cy = O.support_fp32(th, Ws[b], 64, centres=True)
        empty = (x0 > x1) | (y0 > y1)
        box = out["box"][b]
        gpu_empty = box[:, 0] > box[:, 1]
        assert np.array_equal(empty, gpu_empty)
        ok = ~empty
        assert np.array_equal(box[ok], np.stack([x0, x1, y0, y1], 1)[ok])
        assert np.array_equal(out["rec"][b, :, 0], cx) and np.array_equal(out["rec"][b, :, 1], cy)
    assert out["status"] == 0


@pytest.mark.parametrize("tile", [8, 16, 32])
def test_tile_pairs_bit_exact(c1, tile):
    th, Ws, ctf, Y, _ = c1
    out = cuda_step(th, Ws, ctf, Y, 64, tile=tile)
    pg, ranges = O.tile_pairs(th, Ws, 64, tile)
    assert out["n_pairs"] == len(pg)
    assert np.array_equal(out["pairs"][: len(pg)], pg)
    assert np.array_equal(out["ranges"].reshape(ranges.shape), ranges)


def test_forward_images_match_oracle(c1):
    th, Ws, ctf, Y, ref = c1
    out = cuda_step(th, Ws, ctf, Y, 64)
    for b in range(Ws.shape[0]):
        assert rel_l2(out["Q"][b], ref["Q"][b]) < 1e-5
        assert rel_l2(out["X"][b], ref["X"][b]) < 1e-5
    assert np.allclose(out["L"], ref["L"], rtol=1e-5)
    assert rel_l2(out["dX"], ref["dLdX"]) < 1e-5
    assert rel_l2(out["dQ"], ref["dLdQ"]) < 1e-5


def test_gradients_match_oracle(c1):
    th, Ws, ctf, Y, ref = c1
    out = cuda_step(th, Ws, ctf, Y, 64)
    for name, sl in GROUPS:
        assert rel_l2(out["dtheta"][:, sl], ref["dtheta"][:, sl]) < 1e-3, name


def test_results_do_not_depend_on_tile_or_chunk(c1):
    """The support rule is tile independent and every pixel sums its Gaussians in index
    order, so Q is bitwise identical for every tile size and chunk depth."""
    th, Ws, ctf, Y, _ = c1
    base = cuda_step(th, Ws, ctf, Y, 64, tile=16, chunk=128)
    for tile, chunk in ((8, 32), (8, 512), (16, 32), (32, 64), (32, 512)):
        o = cuda_step(th, Ws, ctf, Y, 64, tile=tile, chunk=chunk)
        assert np.array_equal(o["Q"], base["Q"]), (tile, chunk)
        for name, sl in GROUPS:
            assert rel_l2(o["dtheta"][:, sl], base["dtheta"][:, sl]) < 1e-5


def test_tile_independence_with_ill_conditioned_splats():
    """A batch mixing well- and ill-conditioned splats (both record forms, the exact path's
    second pass): Q is still bitwise identical for every tile size and chunk depth."""
    rng = synth.rng_for(5)
    D, N, B = 64, 400, 3
    th = synth.random_gaussians(N, D, rng)
    sc = np.where(np.arange(N)[:, None] % 3 == 0, np.array([0.1, 8.0, 0.1]), np.exp(rng.uniform(-0.7, 1.1, (N, 3))))
    th[:, 3:6] = synth.inv_softplus(sc / D)
    Ws = synth.random_poses(B, rng)
    ctf = synth.random_ctf(B, rng)
    Y = synth.smooth_field(B, D, rng)
    base = cuda_step(th, Ws, ctf, Y, D, tile=8)
    assert 0 < int((base["rec"][:, :, 2] > 0).sum()) < B * N  # both forms present
    for tile, chunk in ((16, 32), (16, 128), (32, 64)):
        o = cuda_step(th, Ws, ctf, Y, D, tile=tile, chunk=chunk)
        assert np.array_equal(o["Q"], base["Q"]), (tile, chunk)


@pytest.mark.parametrize("D,tile", [(40, 16), (33, 8), (50, 32)])
def test_ragged_and_odd_boxes(D, tile):
    th, Ws, ctf, Y = make_batch(3, D, 300, 3)
    ref = O.forward_backward(th, Ws, D, Y, ctf)
    out = cuda_step(th, Ws, ctf, Y, D, tile=tile)
    pg, ranges = O.tile_pairs(th, Ws, D, tile)
    assert np.array_equal(out["pairs"][: len(pg)], pg)
    assert np.array_equal(out["ranges"].reshape(ranges.shape), ranges)
    for b in range(3):
        assert rel_l2(out["Q"][b], ref["Q"][b]) < 1e-5
        assert rel_l2(out["X"][b], ref["X"][b]) < 1e-5
    for name, sl in GROUPS:
        assert rel_l2(out["dtheta"][:, sl], ref["dtheta"][:, sl]) < 1e-3, name


def test_mean_reduction(c1):
    th, Ws, ctf, Y, _ = c1
    ref = O.forward_backward(th, Ws, 64, Y, ctf, reduction=1)
    out = cuda_step(th, Ws, ctf, Y, 64, reduction=1)
    assert np.allclose(out["L"], ref["L"], rtol=1e-5)
    for name, sl in GROUPS:
        assert rel_l2(out["dtheta"][:, sl], ref["dtheta"][:, sl]) < 1e-3, name


@pytest.mark.parametrize("D,reduction", [(64, 0), (33, 0), (40, 1), (256, 0), (256, 1)])
def test_fused_ctf_loss_grad_matches_oracle(D, reduction):
    """gs_ctf_loss_grad (CTF, loss and adjoint CTF by Parseval in the Fourier domain) gives
    the oracle's loss and dL/dQ, and the unfused calls' values; dLdQ may alias Q.  D = 256
    takes the row-transform + column-kernel path, the other sizes the 2-D transforms."""
    th, Ws, ctf, Y = make_batch(80 + D, D, 600, 5)
    ref = O.forward_backward(th, Ws, D, Y, ctf, reduction=reduction)
    N, B = th.shape[0], Ws.shape[0]
    sp = Splatter(D, N, B, tile=8, chunk=64, reduction=reduction)
    t, W, c, y = to_dev(th, Ws.reshape(B, 9), ctf, Y)
    dth = torch.zeros_like(t)
    loss = sp.forward_backward(t, W, c, y, dth, fused=True).cpu().numpy()
    dQ = sp.dQ.cpu().numpy()
    assert np.allclose(loss, ref["L"], rtol=1e-5, atol=0)
    for b in range(B):
        assert rel_l2(dQ[b], ref["dLdQ"][b]) < 1e-5
    g = dth.cpu().numpy()
    for name, sl in GROUPS:
        assert rel_l2(g[:, sl], ref["dtheta"][:, sl]) < 1e-3, name
    # the unfused calls on the same Q
    sp.apply_ctf(sp.Q, c, sp.X)
    l2, _ = sp.loss_grad(sp.X, y)
    sp.apply_ctf(sp.dX, c, sp.X)
    assert np.allclose(loss, l2.cpu().numpy(), rtol=2e-6)
    assert rel_l2(dQ, sp.X.cpu().numpy()) < 2e-6
    # in place: dLdQ written over Q
    Qc = sp.Q.clone()
    l3 = torch.empty(B, device=DEV)
    L.gs_ctf_loss_grad(sp.cfg, Qc, y, c, l3, Qc, sp.fft, sp.ws)
    torch.cuda.synchronize()
    assert torch.equal(Qc, sp.dQ) and np.array_equal(l3.cpu().numpy(), loss)
    sp.close()


def test_scale_activation_is_the_rounded_fp64_softplus():
    """The scales of the activated table are fp32(softplus in FP64) bit for bit (the support
    box depends on them): inside the range of the float-float evaluation, beyond it, and at
    its ends.  The table is the first array of the workspace after the 256-byte status block,
    24 floats per Gaussian with the scales at 12..14."""
    rng = np.random.default_rng(9)
    raw = np.concatenate([rng.uniform(-60, 17, 200_000), rng.uniform(-90, 40, 50_000), rng.normal(-4.9, 1.0, 50_000),
                          [-60.0, -59.999, 17.0, 17.0001, 0.0, -0.0, 1e-30, -1e-30, 30.0]]).astype(np.float32)
    n = (len(raw) + 2) // 3
    flat = np.zeros(3 * n, np.float32)
    flat[:len(raw)] = raw
    th = np.zeros((n, 11), np.float32)
    th[:, 6] = 1.0
    th[:, 3:6] = flat.reshape(n, 3)
    sp = Splatter(64, n, 1, tile=8, with_ctf=False)
    sp.project(torch.from_numpy(th).to(DEV), torch.eye(3, device=DEV).reshape(1, 9))
    torch.cuda.synchronize()
    table = sp.ws[256:256 + n * 96].view(torch.float32).view(n, 24).cpu().numpy()
    got = np.ascontiguousarray(table[:, 12:15]).reshape(-1)
    x = flat.astype(np.float64)
    ref = (np.maximum(x, 0.0) + np.log1p(np.exp(-np.abs(x)))).astype(np.float32)
    assert np.array_equal(got.view(np.uint32), ref.view(np.uint32)), int(np.sum(got != ref))
    sp.close()


def test_adam_step_matches_oracle():
    rng = synth.rng_for(5)
    th = rng.standard_normal(11 * 500).astype(np.float32)
    t, = to_dev(th)
    m = torch.zeros_like(t)
    v = torch.zeros_like(t)
    x, mo, vo = th.astype(np.float64), np.zeros(th.size), np.zeros(th.size)
    for step in range(1, 6):
        g = rng.standard_normal(th.size).astype(np.float32)
        gd, = to_dev(g)
        L.gs_step(t, gd, m, v, step)
        x, mo, vo = O.adam_step(x, g, mo, vo, step)
    assert np.max(np.abs(t.cpu().numpy() - x)) < 1e-6


# ---------------------------------------------------------------------------------------
# Edge cases
# ---------------------------------------------------------------------------------------
def test_no_gaussians_gives_zero_image():
    _, Ws, ctf, Y = make_batch(6, 32, 10, 2)
    th = np.zeros((0, 11), np.float32)
    out = cuda_step(th, Ws, ctf, Y, 32)
    assert np.all(out["Q"] == 0) and out["n_pairs"] == 0
    assert np.allclose(out["L"], np.sum(Y.astype(np.float64) ** 2, axis=(1, 2)), rtol=1e-5)


def test_gaussians_outside_the_box_are_culled():
    th, Ws, ctf, Y = make_batch(7, 32, 50, 2)
    th[:, 0:3] = 5.0  # ten box widths away
    out = cuda_step(th, Ws, ctf, Y, 32)
    assert np.all(out["Q"] == 0) and out["n_pairs"] == 0
    assert np.all(out["dtheta"] == 0)


def test_nonfinite_gaussian_is_flagged_and_skipped():
    th, Ws, ctf, Y = make_batch(8, 48, 200, 2)
    bad = th.copy()
    bad[17, 4] = np.nan
    bad[99, 7] = np.inf
    out = cuda_step(bad, Ws, ctf, Y, 48)
    assert out["status"] & L.GS_STATUS_NONFINITE
    keep = np.ones(200, bool)
    keep[[17, 99]] = False
    ref = O.forward_backward(th[keep], Ws, 48, Y, ctf)
    for b in range(2):
        assert rel_l2(out["Q"][b], ref["Q"][b]) < 1e-5
    assert np.all(out["dtheta"][~keep] == 0)
    for name, sl in GROUPS:
        assert rel_l2(out["dtheta"][keep][:, sl], ref["dtheta"][:, sl]) < 1e-3


def test_large_gaussian_covering_many_tiles():
    th, Ws, ctf, Y = make_batch(9, 64, 40, 2)
    th[0, 3:6] = synth.inv_softplus(np.array([12.0, 9.0, 15.0]) / 64)
    th[0, 0:3] = 0.0
    ref = O.forward_backward(th, Ws, 64, Y, ctf)
    out = cuda_step(th, Ws, ctf, Y, 64, tile=8)
    for b in range(2):
        assert rel_l2(out["Q"][b], ref["Q"][b]) < 1e-5
    for name, sl in GROUPS:
        assert rel_l2(out["dtheta"][:, sl], ref["dtheta"][:, sl]) < 1e-3, name


@pytest.mark.parametrize("D,tile,mode", [(384, 8, "full"), (512, 8, "pairs"), (1024, 16, "pairs"),
                                         (2048, 32, "image")])
def test_wide_tile_grids(D, tile, mode):
    """More than 32 tiles per side (up to the 64 the binning allows), where the scatter takes
    the second word of its transposed lane masks.  A few large Gaussians near the centre make
    boxes cross tile 32; at D = 2048 (the largest image) they cover most of the 64 x 64 tiles.
    Pair lists and ranges bit-exact; at D = 384 also the images and gradients, at D = 2048 the
    rendered images.  FP32 pixel coordinates carry an absolute error that grows with D (the
    unit in the last place of D / 2), and a splat's value moves with its centre, so the image
    bar is 1e-5 scaled by D / 256 (the largest box of the paper's workloads)."""
    full = mode == "full"
    rng = synth.rng_for(40 + D)
    th = synth.random_gaussians(300, D, rng)
    th[:6, 0:3] = rng.uniform(-0.05, 0.05, size=(6, 3))
    th[:6, 3:6] = synth.inv_softplus(np.array([40.0, 25.0, 60.0]) * max(1.0, D / 1024.0) / D)
    Ws = synth.random_poses(2, rng)
    ctf = synth.random_ctf(2, rng)
    pg, ranges = O.tile_pairs(th, Ws, D, tile)
    tx1 = []
    for b in range(2):
        x0, x1, y0, y1 = O.support_fp32(th, Ws[b], D)[:4]
        tx1.append((np.asarray(x1) // tile >= 32) & (np.asarray(x0) // tile < 32))
    assert np.concatenate(tx1).any()  # some boxes straddle tile column 32
    if full:
        Y = synth.add_noise(np.stack([O.apply_ctf(O.render_one(th, Ws[b], D), O.ctf_image(
            D, *[float(v) for v in ctf[b, 0:4]], apix=float(ctf[b, 4]))) for b in range(2)]), 0.1, rng)
        ref = O.forward_backward(th, Ws, D, Y, ctf)
        out = cuda_step(th, Ws, ctf, Y, D, tile=tile)
        for b in range(2):
            assert rel_l2(out["Q"][b], ref["Q"][b]) < 1e-5
        for name, sl in GROUPS:
            assert rel_l2(out["dtheta"][:, sl], ref["dtheta"][:, sl]) < 1e-3, name
        pairs, rng_out, n = out["pairs"], out["ranges"], out["n_pairs"]
    else:
        sp = Splatter(D, th.shape[0], 2, tile=tile, with_ctf=False)
        t, W = to_dev(th, Ws.reshape(2, 9))
        sp.project(t, W)
        sp.bin_sort(grow=True)
        if mode == "image":
            sp.render()
            Q = sp.Q.cpu().numpy()
            for b in range(2):
                assert rel_l2(Q[b], O.render_one(th, Ws[b], D)) < 1e-5 * max(1.0, D / 256)
        torch.cuda.synchronize()
        n = int(sp.n_pairs.item()) & 0xFFFFFFFF
        pairs = sp.pairs.cpu().numpy().view(np.uint32)
        rng_out = sp.ranges.cpu().numpy().view(np.uint32)
        assert sp.status() == 0
        sp.close()
    assert n == len(pg)
    assert np.array_equal(pairs[: len(pg)], pg)
    assert np.array_equal(rng_out.reshape(ranges.shape), ranges)



@pytest.mark.parametrize("ratio", [10, 40, 160])
@pytest.mark.parametrize("tile", [8, 16])
def test_needles_and_pancakes(ratio, tile):
    """Strong anisotropy: needles (one axis of 8 px, two of 8 / ratio px; at ratio 160 the thin
    axes are 0.05 px) and pancakes (one thin axis) in random orientations.  Boxes bit-exact;
    images within 1e-5 and gradients within 1e-3 per parameter group, the bars of every other
    test.  Such splats are stored as a completed square with the centre as a float-float (their
    expanded quadratic form would lose a factor of the 2 x 2 condition number, ratio^2)."""
    rng = synth.rng_for(77)
    D, N, B = 64, 60, 4
    th = synth.random_gaussians(N, D, rng)
    thin = 8.0 / ratio
    sc = np.where(np.arange(N)[:, None] % 2 == 0, np.array([thin, 8.0, thin]), np.array([8.0, 6.0, thin]))
    th[:, 3:6] = synth.inv_softplus(sc / D)
    Ws = synth.random_poses(B, rng)
    ctf = synth.random_ctf(B, rng)
    Y = synth.add_noise(np.stack([O.apply_ctf(O.render_one(synth.random_gaussians(N, D, rng), Ws[b], D),
                                              O.ctf_image(D, *[float(v) for v in ctf[b, 0:4]],
                                                          apix=float(ctf[b, 4]))) for b in range(B)]), 0.1, rng)
    ref = O.forward_backward(th, Ws, D, Y, ctf)
    out = cuda_step(th, Ws, ctf, Y, D, tile=tile)
    if ratio >= 40:  # most of these splats take the completed-square form (third float > 0)
        assert int((out["rec"][:, :, 2] > 0).sum()) > B * N // 3
    for b in range(B):
        x0, x1, y0, y1 = O.support_fp32(th, Ws[b], D)[:4]
        empty = (np.asarray(x0) > np.asarray(x1)) | (np.asarray(y0) > np.asarray(y1))
        box = out["box"][b]
        assert np.array_equal(empty, box[:, 0] > box[:, 1])
        ok = ~empty
        assert np.array_equal(box[ok], np.stack([x0, x1, y0, y1], 1)[ok])
        assert rel_l2(out["Q"][b], ref["Q"][b]) < 1e-5
        assert rel_l2(out["X"][b], ref["X"][b]) < 1e-5
    for name, sl in GROUPS:
        assert rel_l2(out["dtheta"][:, sl], ref["dtheta"][:, sl]) < 1e-3, name


def test_pair_overflow_is_reported_and_recovered(c1):
    th, Ws, ctf, Y, ref = c1
    sp = Splatter(64, th.shape[0], Ws.shape[0], tile=16, pair_capacity=100)
    t, W, c = to_dev(th, Ws.reshape(-1, 9), ctf)
    sp.project(t, W)
    sp.bin_sort(grow=False)
    need = int(sp.n_pairs.item())
    assert need > 100
    assert sp.status() & L.GS_STATUS_OVERFLOW
    r = sp.ranges.cpu().numpy().view(np.uint32)
    assert r.max() <= 100
    sp.bin_sort(grow=True)
    sp.render()
    assert sp.status() == 0
    Q = sp.Q.cpu().numpy()
    for b in range(Ws.shape[0]):
        assert rel_l2(Q[b], ref["Q"][b]) < 1e-5
    sp.close()


def test_binding_validates_tensors():
    """The binding checks dtype, device and contiguity before handing pointers to the
    kernels: a float64 theta, a CPU theta and a transposed (strided) W each raise ValueError."""
    cfg = L.config(64)
    N, B = 10, 3
    W = torch.zeros(B, 9, device=DEV)
    proj = torch.empty(L.gs_proj_size(B, N), dtype=torch.uint8, device=DEV)
    ws = torch.empty(L.gs_workspace_size(cfg, B, N), dtype=torch.uint8, device=DEV)
    with pytest.raises(ValueError, match="float32"):
        L.gs_project(cfg, torch.zeros(N, 11, dtype=torch.float64, device=DEV), W, proj, ws)
    with pytest.raises(ValueError, match="CUDA device memory"):
        L.gs_project(cfg, torch.zeros(N, 11), W, proj, ws)
    with pytest.raises(ValueError, match="contiguous"):
        L.gs_project(cfg, torch.zeros(N, 11, device=DEV), torch.zeros(9, B, device=DEV).t(), proj, ws)
    with pytest.raises(ValueError, match="int32"):
        L.gs_render_fwd(cfg, proj, N, torch.zeros(5, dtype=torch.int64, device=DEV),
                        torch.zeros(16 * B * 2, dtype=torch.int32, device=DEV), B,
                        torch.zeros(B, 64, 64, device=DEV))


def test_invalid_arguments_raise():
    cfg = L.config(64)
    t = torch.zeros(10, 11, device=DEV)
    W = torch.zeros(2, 9, device=DEV)
    proj = torch.empty(L.gs_proj_size(2, 10), dtype=torch.uint8, device=DEV)
    assert proj.numel() == 2 * 10 * (32 + 8 + 8)  # records, the box plane, the centres' low parts
    with pytest.raises(L.GsError):
        L.gs_project(L.config(64, tile=12), t, W, proj, torch.empty(1 << 20, dtype=torch.uint8, device=DEV))
    small_ws = torch.empty(256, dtype=torch.uint8, device=DEV)
    with pytest.raises(L.GsError) as e:
        L.gs_project(cfg, t, W, proj, small_ws)
    assert e.value.rc == L.GS_ENOSPC
    with pytest.raises(ValueError):  # records only, without room for the planes that follow
        L.gs_project(cfg, t, W, torch.empty(2 * 10 * 32, dtype=torch.uint8, device=DEV),
                     torch.empty(1 << 20, dtype=torch.uint8, device=DEV))


# ---------------------------------------------------------------------------------------
# Full size, as the bench launches it: sampled images and gradients, all tile counts
# ---------------------------------------------------------------------------------------
@pytest.mark.slow
def test_full_size_sampled_against_oracle():
    D, N, B, tile = 256, 100_000, 128, 16
    rng = synth.rng_for(0)
    th = synth.random_gaussians(N, D, rng)
    Ws = synth.random_poses(B, rng)
    ctf = synth.random_ctf(B, rng)
    sp = Splatter(D, N, B, tile=tile)
    t, W, c = to_dev(th, Ws.reshape(B, 9), ctf)
    sp.forward(t, W, c)
    torch.cuda.synchronize()
    counts = O.tile_counts(th, Ws, D, tile)
    r = sp.ranges.cpu().numpy().view(np.uint32).reshape(B, -1, 2).astype(np.int64)
    assert np.array_equal(r[:, :, 1] - r[:, :, 0], counts)
    assert int(sp.n_pairs.item()) == counts.sum()
    pairs = sp.pairs.cpu().numpy().view(np.uint32)
    Q = sp.Q.cpu().numpy()
    for b in (0, 127):
        x0, x1, y0, y1, _ = O.support_fp32(th, Ws[b], D)
        for tt in (0, 100, 137, 255):
            ty, tx = divmod(tt, D // tile)
            hit = (x0 <= x1) & (y0 <= y1) & (x0 // tile <= tx) & (x1 // tile >= tx) & (y0 // tile <= ty) & (y1 // tile >= ty)
            assert np.array_equal(pairs[r[b, tt, 0]:r[b, tt, 1]], np.nonzero(hit)[0])
        assert rel_l2(Q[b], O.render_one(th, Ws[b], D)) < 1e-5
    # gradient of one image inside the full batch launch
    dQ = np.zeros((B, D, D), np.float32)
    dQ[5] = synth.smooth_field(1, D, rng, scale=1e-3)[0]
    dq, = to_dev(dQ)
    dth = torch.zeros_like(t)
    sp.backward(t, W, dq, dth)
    g = dth.cpu().numpy()
    ref = O.backward(th, Ws[5:6], D, dQ[5:6])
    for name, sl in GROUPS:
        assert rel_l2(g[:, sl], ref[:, sl]) < 1e-3, name
    assert sp.status() == 0
    sp.close()
