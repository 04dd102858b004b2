"""Parity at the full sizes of the workloads, in the launch configurations that are timed: the
bench's graph-captured step (D = 256, N = 100k, B = 128, tile 8, the fused CTF-loss path), the
batched fused step at D = 128, N = 20k, B = 64 (autotuned), the autograd step at scale
(D = 256, N = 200k Gaussians on random-walk chains, B = 256, lists recomputed per 64-particle
chunk) and the mixed batch of four volumes (D = 96-256, N = 10k-100k, 128 particles each).  The FP64 oracle computes sampled images' losses and dL/dQ and one image's gradient,
taken from inside the full batch launch; the tile counts are compared in full (bit-exact)."""
import numpy as np
import pytest

import oracle as O
from paper_2508_04929_b300 import synth

pytestmark = [pytest.mark.gpu, pytest.mark.slow]
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2508_04929_b300 import build  # noqa: E402

build.build()
from paper_2508_04929_b300 import autograd as AG  # noqa: E402
from paper_2508_04929_b300.batched import GraphStep, Problem  # noqa: E402

GROUPS = (("mu", slice(0, 3)), ("s", slice(3, 6)), ("q", slice(6, 10)), ("A", slice(10, 11)))
DEV = "cuda"


def rel_l2(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def oracle_image(th, W, ctf_row, Y, D):
    """FP64 loss and dL/dQ of one image (App. A.2 Eq. 14, Sec. 3.3.5)."""
    H = O.ctf_image(D, *[float(v) for v in ctf_row[0:4]], apix=float(ctf_row[4]))
    R = O.apply_ctf(O.render_one(th, W, D), H) - Y
    return float(np.sum(R * R)), O.apply_ctf_adjoint(2.0 * R, H)


def batched_step_checks(D, N, B, tile, chunk, seed, samples, grad_image):
    rng = synth.rng_for(seed)
    th = synth.random_gaussians(N, D, rng)
    Ws = synth.random_poses(B, rng)
    ctf = synth.random_ctf(B, rng)
    Y = synth.smooth_field(B, D, rng, scale=1.0)
    dev = torch.device(DEV)
    p = Problem(D=D, theta=torch.from_numpy(th).to(dev), W=torch.from_numpy(Ws.reshape(B, 9)).to(dev),
                ctf=torch.from_numpy(ctf).to(dev), Y=torch.from_numpy(Y).to(dev), tile=tile, chunk=chunk)
    gs = GraphStep([p], adam=False)
    losses = gs.replay()[0].cpu().numpy()
    torch.cuda.synchronize()
    assert gs.check() == 0
    dQ = p.sp.dQ.cpu().numpy()
    T = p.sp.cfg.tile
    counts = O.tile_counts(th, Ws, D, T)
    r = p.sp.ranges.cpu().numpy().view(np.uint32).reshape(B, -1, 2).astype(np.int64)
    assert np.array_equal(r[:, :, 1] - r[:, :, 0], counts)
    for b in samples:
        L_ref, dQ_ref = oracle_image(th, Ws[b], ctf[b], Y[b], D)
        assert abs(losses[b] - L_ref) <= 1e-5 * L_ref, (b, losses[b], L_ref)
        assert rel_l2(dQ[b], dQ_ref) < 1e-5, b
    # one image's gradient through the same lists (the projection is re-run: it resets the
    # gradient accumulator that the step's own backward consumed)
    g_img = np.zeros((B, D, D), np.float32)
    g_img[grad_image] = dQ[grad_image]
    p.sp.project(p.theta, p.W)
    dth = torch.zeros_like(p.theta)
    p.sp.backward(p.theta, p.W, torch.from_numpy(g_img).to(dev), dth)
    g = dth.cpu().numpy()
    ref = O.backward(th, Ws[grad_image:grad_image + 1], D, g_img[grad_image:grad_image + 1].astype(np.float64))
    for name, sl in GROUPS:
        assert rel_l2(g[:, sl], ref[:, sl]) < 1e-3, name
    assert p.sp.status() == 0
    gs.close()


def test_bench_step_full_size():
    """D = 256, N = 100k, B = 128, tile 8: the graph-captured step bench.py times."""
    batched_step_checks(256, 100_000, 128, 8, 64, seed=0, samples=(0, 127), grad_image=5)


def test_batched_fused_step_d128():
    """D = 128, N = 20k, B = 64: one graph-captured step, launch shape chosen by the autotuner."""
    batched_step_checks(128, 20_000, 64, 0, 0, seed=1, samples=(0, 63), grad_image=7)


def test_autograd_step_at_scale():
    """D = 256, N = 200k chain Gaussians, B = 256 through the autograd path (64-particle chunks,
    lists recomputed in the backward): sampled losses and one image's gradient (one-hot
    backward of the per-image losses)."""
    D, N, B = 256, 200_000, 256
    rng = synth.rng_for(3)
    th = synth.chain_gaussians(N, D, rng)
    Ws = synth.random_poses(B, rng)
    ctf = synth.random_ctf(B, rng)
    Y = synth.smooth_field(B, D, rng, scale=1.0)
    eng = AG.RenderEngine(D, N, particles_per_chunk=64, tile=8)
    t = torch.from_numpy(th).cuda().requires_grad_(True)
    W = torch.from_numpy(Ws.reshape(B, 9)).cuda()
    C = torch.from_numpy(ctf).cuda()
    Yd = torch.from_numpy(Y).cuda()
    losses = AG.ctf_loss(AG.render(t, W, eng), C, Yd, eng)
    b_sel = 200
    onehot = torch.zeros(B, device=DEV)
    onehot[b_sel] = 1.0
    losses.backward(onehot)
    lo = losses.detach().cpu().numpy()
    g = t.grad.cpu().numpy()
    for b in (0, b_sel):
        L_ref, dQ_ref = oracle_image(th, Ws[b], ctf[b], Y[b], D)
        assert abs(lo[b] - L_ref) <= 1e-5 * L_ref, (b, lo[b], L_ref)
        if b == b_sel:
            ref = O.backward(th, Ws[b:b + 1], D, dQ_ref[None])
            for name, sl in GROUPS:
                assert rel_l2(g[:, sl], ref[:, sl]) < 1e-3, name
    eng.close()


def test_mixed_batch_full_size():
    """Four volumes in one graph: N = 10k/30k/60k/100k at D = 96/128/192/256, 128 particles each,
    launch shapes autotuned per volume; one sampled image's loss and dL/dQ per volume and one
    image's gradient for the smallest volume."""
    dev = torch.device(DEV)
    specs = [(96, 10_000), (128, 30_000), (192, 60_000), (256, 100_000)]
    made = []
    for k, (D, N) in enumerate(specs):
        rng = synth.rng_for(20 + k)
        th = synth.random_gaussians(N, D, rng)
        Ws = synth.random_poses(128, rng)
        ctf = synth.random_ctf(128, rng)
        Y = synth.smooth_field(128, D, rng, scale=1.0)
        p = Problem(D=D, theta=torch.from_numpy(th).to(dev), W=torch.from_numpy(Ws.reshape(128, 9)).to(dev),
                    ctf=torch.from_numpy(ctf).to(dev), Y=torch.from_numpy(Y).to(dev))
        made.append((p, th, Ws, ctf, Y))
    gs = GraphStep([m[0] for m in made], adam=False, autotune_chunks=(64, 128))
    losses = [x.cpu().numpy() for x in gs.replay()]
    torch.cuda.synchronize()
    assert gs.check() == 0
    for (p, th, Ws, ctf, Y), lo, (D, N) in zip(made, losses, specs):
        b = 31
        L_ref, dQ_ref = oracle_image(th, Ws[b], ctf[b], Y[b], D)
        assert abs(lo[b] - L_ref) <= 1e-5 * L_ref, (D, lo[b], L_ref)
        assert rel_l2(p.sp.dQ[b].cpu().numpy(), dQ_ref) < 1e-5, D
    p, th, Ws, ctf, Y = made[0]
    D = specs[0][0]
    g_img = np.zeros((128, D, D), np.float32)
    g_img[3] = p.sp.dQ[3].cpu().numpy()
    p.sp.project(p.theta, p.W)
    dth = torch.zeros_like(p.theta)
    p.sp.backward(p.theta, p.W, torch.from_numpy(g_img).to(dev), dth)
    ref = O.backward(th, Ws[3:4], D, g_img[3:4].astype(np.float64))
    g = dth.cpu().numpy()
    for name, sl in GROUPS:
        assert rel_l2(g[:, sl], ref[:, sl]) < 1e-3, name
    gs.close()
