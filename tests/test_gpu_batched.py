"""CUDA-graph-captured batched steps: one graph over a mixed batch of volumes (different
box sizes and Gaussian counts) must give the per-problem losses and gradients of the eager
calls, equal the FP64 oracle, take new inputs between replays, recover from a pair-buffer
overflow, and its device-counted Adam must equal the host-counted one bit for bit."""
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
from paper_2508_04929_b300.batched import GraphStep, HostFeeder, Problem, SlotFeeder  # noqa: E402
from paper_2508_04929_b300.splat import Splatter  # noqa: E402

GROUPS = (slice(0, 3), slice(3, 6), slice(6, 10), slice(10, 11))


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a, np.float64) - b) / np.linalg.norm(b))


def _problem(seed, D, N, B, tile=16, chunk=64):
    rng = synth.rng_for(seed)
    th = synth.random_gaussians(N, D, rng)
    Ws = synth.random_poses(B, rng)
    ctf = synth.random_ctf(B, rng)
    Y = synth.smooth_field(B, D, rng, scale=100.0)
    dev = torch.device("cuda")
    p = Problem(D=D, theta=torch.from_numpy(th).to(dev), W=torch.from_numpy(Ws.reshape(B, 9)).to(dev),
                ctf=torch.from_numpy(ctf).to(dev), Y=torch.from_numpy(Y).to(dev), tile=tile, chunk=chunk)
    return p, (th, Ws, ctf, Y)


def _eager(D, host, tile=16, chunk=64):
    th, Ws, ctf, Y = host
    B = Ws.shape[0]
    sp = Splatter(D, th.shape[0], B, tile=tile, chunk=chunk)
    t = torch.from_numpy(th).cuda()
    g = torch.zeros_like(t)
    loss = sp.forward_backward(t, torch.from_numpy(Ws.reshape(B, 9)).cuda(), torch.from_numpy(ctf).cuda(),
                               torch.from_numpy(Y).cuda(), g, fused=True)
    out = loss.cpu().numpy(), g.cpu().numpy()
    sp.close()
    return out


def test_mixed_batch_graph_matches_eager_and_oracle():
    specs = [(50, 32, 300, 3, 8), (51, 40, 500, 4, 16), (52, 48, 700, 5, 16), (53, 64, 900, 3, 32)]
    made = [_problem(s, D, N, B, tile=T) for s, D, N, B, T in specs]
    gs = GraphStep([m[0] for m in made], adam=False)
    losses = [x.cpu().numpy() for x in gs.replay()]
    torch.cuda.synchronize()
    assert gs.check() == 0
    for (p, host), (s, D, N, B, T), lo in zip(made, specs, losses):
        le, ge = _eager(D, host, tile=T)
        assert np.allclose(lo, le, rtol=1e-6)
        g = p.dtheta.cpu().numpy()
        for sl in GROUPS:
            assert rel(g[:, sl], ge[:, sl]) < 1e-5
    th, Ws, ctf, Y = made[1][1]
    ref = O.forward_backward(th, Ws, 40, Y, ctf)
    assert np.allclose(losses[1], ref["L"], rtol=1e-5)
    g = made[1][0].dtheta.cpu().numpy()
    for sl in GROUPS:
        assert rel(g[:, sl], ref["dtheta"][:, sl]) < 1e-3
    gs.close()


def test_replay_with_new_inputs_and_counted_adam():
    p, host = _problem(60, 40, 400, 4)
    th0 = p.theta.clone()
    gs = GraphStep([p], adam=True)
    # step 1 on the original batch
    l1 = gs.replay()[0].cpu().numpy()
    # step 2 on a new batch copied into the static buffers
    rng = synth.rng_for(61)
    W2 = torch.from_numpy(synth.random_poses(4, rng).reshape(4, 9)).cuda()
    C2 = torch.from_numpy(synth.random_ctf(4, rng)).cuda()
    Y2 = torch.from_numpy(synth.smooth_field(4, 40, rng, scale=100.0)).cuda()
    gs.load(0, W=W2, ctf=C2, Y=Y2)
    l2 = gs.replay()[0].cpu().numpy()
    torch.cuda.synchronize()
    assert int(p.t.item()) == 2
    # the same two steps eagerly, with the host-counted Adam
    sp = Splatter(40, 400, 4, tile=16, chunk=64)
    t = th0.clone()
    m, v, g = torch.zeros_like(t), torch.zeros_like(t), torch.zeros_like(t)
    W1, C1, Y1 = (torch.from_numpy(x).cuda() for x in (host[1].reshape(4, 9), host[2], host[3]))
    e1 = sp.forward_backward(t, W1, C1, Y1, g, fused=True).cpu().numpy()
    L.gs_step(t, g, m, v, 1)
    g.zero_()
    e2 = sp.forward_backward(t, W2, C2, Y2, g, fused=True).cpu().numpy()
    L.gs_step(t, g, m, v, 2)
    torch.cuda.synchronize()
    assert np.allclose(l1, e1, rtol=1e-6) and np.allclose(l2, e2, rtol=1e-5)
    d = (p.theta - t).abs().cpu().numpy()
    assert np.mean(d > 1e-5) < 0.01 and d.max() <= 4.1e-3  # Adam may flip the sign of ~0 gradients
    sp.close()
    gs.close()


def test_split_replay_equals_whole_step():
    """replay_front() + replay_back() is the step that replay() runs: the same first loss bit for
    bit, and then the same losses and Theta up to the order of the backward's float atomics."""
    p, _ = _problem(63, 40, 400, 4)
    th0 = p.theta.clone()
    gs = GraphStep([p], adam=True)
    la = [gs.replay()[0].cpu().numpy() for _ in range(3)]
    tha = p.theta.clone()
    p.theta.copy_(th0)
    p.m.zero_()
    p.v.zero_()
    p.t.zero_()
    gs.record_split()
    lb = []
    for _ in range(3):
        gs.replay_front()
        lb.append(gs.replay_back()[0].cpu().numpy())
    torch.cuda.synchronize()
    assert np.array_equal(la[0], lb[0])
    for x, y in zip(la[1:], lb[1:]):
        assert np.allclose(x, y, rtol=1e-5)
    d = (p.theta - tha).abs().cpu().numpy()
    assert np.mean(d > 1e-5) < 0.01 and d.max() <= 4.1e-3  # Adam may flip the sign of ~0 gradients
    assert int(p.t.item()) == 3
    gs.close()


def test_host_feeder_halves_match_whole_loads():
    """Feeding a step in two parts (poses and CTF before the front half, images before the
    back half) gives the losses of feeding it whole, step after step."""
    p, _ = _problem(64, 40, 400, 4)
    gs = GraphStep([p], adam=False)
    rng = synth.rng_for(65)
    batches = [(torch.from_numpy(synth.random_poses(4, rng).reshape(4, 9)).pin_memory(),
                torch.from_numpy(synth.random_ctf(4, rng)).pin_memory(),
                torch.from_numpy(synth.smooth_field(4, 40, rng, scale=100.0)).pin_memory()) for _ in range(3)]
    whole, halves = [], []
    fa = HostFeeder(gs)
    fa.prefetch(*batches[0])
    for i in range(3):
        fa.load()
        if i + 1 < 3:
            fa.prefetch(*batches[i + 1])
        whole.append(gs.replay()[0].clone())
    fb = HostFeeder(gs)
    fb.prefetch(*batches[0])
    for i in range(3):
        fb.load_front()
        if i + 1 < 3:
            fb.prefetch(*batches[i + 1])
        gs.replay_front()
        fb.load_back()
        halves.append(gs.replay_back()[0].clone())
    torch.cuda.synchronize()
    for x, y in zip(whole, halves):
        assert torch.equal(x, y)
    assert not torch.equal(whole[0], whole[1])  # the steps did take new inputs
    gs.close()


def test_slot_feeder_matches_host_feeder():
    """Steps fed through the graph's input slots (host copies straight into the buffers the
    slot's graphs read) give the losses of steps fed through the static buffers, step after
    step, and the slot graphs are re-recorded when an overflow re-sizes the pair buffer."""
    p, _ = _problem(66, 40, 400, 4)
    gs = GraphStep([p], adam=False)
    rng = synth.rng_for(67)
    batches = [(torch.from_numpy(synth.random_poses(4, rng).reshape(4, 9)).pin_memory(),
                torch.from_numpy(synth.random_ctf(4, rng)).pin_memory(),
                torch.from_numpy(synth.smooth_field(4, 40, rng, scale=100.0)).pin_memory()) for _ in range(4)]
    ref = []
    fa = HostFeeder(gs)
    for i in range(4):
        fa.prefetch(*batches[i])
        fa.load()
        ref.append(gs.replay()[0].clone())
    sf = SlotFeeder(gs)
    got = []
    sf.prefetch(*batches[0])
    for i in range(4):
        if i + 1 < 4:
            sf.prefetch(*batches[i + 1])
        got.append(sf.step()[0].clone())
    torch.cuda.synchronize()
    for x, y in zip(ref, got):
        assert torch.equal(x, y)
    with pytest.raises(RuntimeError):
        sf.step()  # nothing prefetched
    gs.close()


def test_counted_adam_equals_host_counted_adam():
    rng = synth.rng_for(62)
    a = torch.from_numpy(rng.standard_normal(5000).astype(np.float32)).cuda()
    b = a.clone()
    ma, va, mb, vb = (torch.zeros_like(a) for _ in range(4))
    t = torch.zeros(1, dtype=torch.int32, device="cuda")
    for step in range(1, 5):
        g = torch.from_numpy(rng.standard_normal(5000).astype(np.float32)).cuda()
        L.gs_step(a, g, ma, va, step)
        L.gs_step_counted(b, g, mb, vb, t)
    torch.cuda.synchronize()
    assert torch.equal(a, b) and int(t.item()) == 4


def test_overflow_is_detected_and_rerecorded():
    p, host = _problem(70, 48, 600, 4)
    gs = GraphStep([p], adam=False, margin=0.5, min_pairs=16)  # deliberately too small a pair buffer
    gs.replay()
    st = gs.check()
    assert st & L.GS_STATUS_OVERFLOW
    gs.replay()
    torch.cuda.synchronize()
    assert gs.check() == 0
    le, ge = _eager(48, host)
    assert np.allclose(gs.problems[0].sp.loss[:4].cpu().numpy(), le, rtol=1e-6)
    gs.close()


def test_autotuner_candidates_and_choice():
    """The tuner times tile 8 once (its kernels take no chunk depth), every admissible
    (16 or 32, chunk) pair otherwise, returns the fastest, and a GraphStep built with
    tile = chunk = 0 takes that choice and reproduces the images of another launch shape."""
    from paper_2508_04929_b300.autotune import tune
    p, host = _problem(60, 48, 600, 3)
    out = tune(48, 600, 3, p.theta, p.W, p.ctf, p.Y, tiles=(8, 16, 32), chunks=(64, 128))
    shapes = [(r["tile"], r["chunk"]) for r in out["table"]]
    assert shapes == [(8, 64), (16, 64), (16, 128), (32, 64), (32, 128)]
    assert all(r["ms"] > 0 for r in out["table"])
    best = min(out["table"], key=lambda r: r["ms"])
    assert (out["tile"], out["chunk"]) == (best["tile"], best["chunk"])
    q, _ = _problem(60, 48, 600, 3, tile=0, chunk=0)
    gs = GraphStep([q], adam=False, autotune_chunks=(64, 128))
    assert (q.tile, q.chunk) in shapes
    gs.replay()
    torch.cuda.synchronize()
    Q_tuned = q.sp.Q[:3].clone()
    ref = Splatter(48, 600, 3, tile=32 if q.tile != 32 else 8, chunk=64)
    ref.forward(p.theta, p.W, p.ctf, grow=True)
    torch.cuda.synchronize()
    assert torch.equal(Q_tuned, ref.Q[:3])  # the support rule does not depend on the tile
    ref.close()
