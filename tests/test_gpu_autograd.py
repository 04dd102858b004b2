"""torch.autograd wrappers: gradients through render -> CTF -> loss against the FP64 oracle,
a directional central difference of the CUDA forward itself, and chunked rendering with
recomputed tile lists equal to the one-shot batch."""
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
from paper_2508_04929_b300 import autograd as AG  # noqa: E402
from paper_2508_04929_b300.splat import Splatter  # noqa: E402

GROUPS = (("mu", slice(0, 3)), ("s", slice(3, 6)), ("q", slice(6, 10)), ("A", slice(10, 11)))


def _inputs(seed=40, D=48, N=400, B=7):
    rng = synth.rng_for(seed)
    th = synth.random_gaussians(N, D, rng)
    Ws = synth.random_poses(B, rng)
    ctf = synth.random_ctf(B, rng)
    Y = synth.smooth_field(B, D, rng, scale=200.0)
    return th, Ws, ctf, Y


def _loss_fn(engine, W, C, Yd, D):
    def f(t):
        Q = AG.render(t, W, engine)
        X = AG.apply_ctf(Q, C, engine)
        return AG.loss(X, Yd, D).sum()
    return f


def test_autograd_gradient_matches_oracle_with_recomputed_lists():
    th, Ws, ctf, Y = _inputs()
    D, B = 48, Ws.shape[0]
    ref = O.forward_backward(th, Ws, D, Y, ctf)
    eng = AG.RenderEngine(D, th.shape[0], particles_per_chunk=3, tile=16, chunk=64)
    t = torch.from_numpy(th).cuda().requires_grad_(True)
    W = torch.from_numpy(Ws.reshape(B, 9)).cuda()
    C = torch.from_numpy(ctf).cuda()
    Yd = torch.from_numpy(Y).cuda()
    L = _loss_fn(eng, W, C, Yd, D)(t)
    L.backward()
    g = t.grad.cpu().numpy()
    assert abs(float(L.detach()) - ref["L"].sum()) < 1e-5 * ref["L"].sum()
    for name, sl in GROUPS:
        rel = np.linalg.norm(g[:, sl] - ref["dtheta"][:, sl]) / np.linalg.norm(ref["dtheta"][:, sl])
        assert rel < 1e-3, (name, rel)
    eng.close()


@pytest.mark.parametrize("D", [48, 256])
def test_fused_ctf_loss_matches_composed_and_oracle(D):
    """ctf_loss(render(theta)) gives the loss and gradient of loss(apply_ctf(render(theta))),
    and the oracle's (D = 256: the row-transform + column-kernel path)."""
    th, Ws, ctf, Y = _inputs(seed=44, D=D, N=300, B=5)
    B = Ws.shape[0]
    ref = O.forward_backward(th, Ws, D, Y, ctf)
    eng = AG.RenderEngine(D, th.shape[0], particles_per_chunk=2, tile=8, chunk=64)
    W = torch.from_numpy(Ws.reshape(B, 9)).cuda()
    C = torch.from_numpy(ctf).cuda()
    Yd = torch.from_numpy(Y).cuda()
    t1 = torch.from_numpy(th).cuda().requires_grad_(True)
    L1 = AG.ctf_loss(AG.render(t1, W, eng), C, Yd, eng)
    L1.sum().backward()
    t2 = torch.from_numpy(th).cuda().requires_grad_(True)
    L2 = _loss_fn(eng, W, C, Yd, D)(t2)
    L2.backward()
    assert np.allclose(L1.detach().cpu().numpy(), ref["L"], rtol=1e-5)
    assert abs(float(L1.sum().detach()) - float(L2.detach())) < 2e-6 * float(L2.detach())
    g1, g2 = t1.grad.cpu().numpy(), t2.grad.cpu().numpy()
    for name, sl in GROUPS:
        assert np.linalg.norm(g1[:, sl] - g2[:, sl]) < 1e-5 * np.linalg.norm(g2[:, sl]), name
        assert np.linalg.norm(g1[:, sl] - ref["dtheta"][:, sl]) < 1e-3 * np.linalg.norm(ref["dtheta"][:, sl]), name
    eng.close()


def test_directional_difference_of_cuda_forward():
    """<grad L, v> against (L(theta + e v) - L(theta - e v)) / 2e computed by the CUDA forward
    itself.  The support boxes are integer decisions, so v is restricted to the Gaussians
    whose boxes stay the same at theta +- e v in every image (the loss is smooth there);
    per-image losses are summed in FP64.  1 % (the strict check is the FP64 oracle)."""
    th, Ws, ctf, Y = _inputs(seed=41, N=300, B=4)
    D, B, N = 48, Ws.shape[0], th.shape[0]
    eng = AG.RenderEngine(D, N, particles_per_chunk=4, tile=16, chunk=64)
    W = torch.from_numpy(Ws.reshape(B, 9)).cuda()
    C = torch.from_numpy(ctf).cuda()
    Yd = torch.from_numpy(Y).cuda()

    def losses(t):
        Q = AG.render(t, W, eng)
        return AG.loss(AG.apply_ctf(Q, C, eng), Yd, D)

    probe = Splatter(D, N, B, tile=16, chunk=64, with_ctf=False)

    def boxes(t):
        probe.project(t, W)
        raw = probe.proj[: B * N * 32].view(torch.int16).view(B, N, 16)[:, :, 12:16]
        return raw.cpu().numpy()

    t = torch.from_numpy(th).cuda().requires_grad_(True)
    losses(t).sum().backward()
    rng = synth.rng_for(7)
    for sl, eps in ((slice(0, 3), 2e-4), (slice(3, 6), 1e-3), (slice(6, 10), 1e-3), (slice(10, 11), 1e-3)):
        v = np.zeros_like(th)
        v[:, sl] = rng.standard_normal(v[:, sl].shape).astype(np.float32)
        b0 = boxes(t.detach())
        for _ in range(3):
            vd = torch.from_numpy(v).cuda()
            moved = ((boxes(t.detach() + eps * vd) != b0) | (boxes(t.detach() - eps * vd) != b0)).any(axis=(0, 2))
            if not moved.any():
                break
            v[moved] = 0.0
        assert not moved.any() and np.count_nonzero(v[:, sl].any(axis=1)) > N // 2
        vd = torch.from_numpy(v).cuda()
        with torch.no_grad():
            Lp = losses(t.detach() + eps * vd).double().sum().item()
            Lm = losses(t.detach() - eps * vd).double().sum().item()
        fd = (Lp - Lm) / (2 * eps)
        an = float((t.grad.double() * vd.double()).sum())
        assert abs(fd - an) < 1e-2 * abs(an), (sl, fd, an)
    probe.close()
    eng.close()


def test_chunked_render_equals_batch_render():
    th, Ws, ctf, Y = _inputs(seed=42, N=500, B=9)
    D, B = 48, Ws.shape[0]
    t = torch.from_numpy(th).cuda()
    W = torch.from_numpy(Ws.reshape(B, 9)).cuda()
    eng = AG.RenderEngine(D, th.shape[0], particles_per_chunk=4, tile=16, chunk=64)
    Qc = eng.render(t, W)
    sp = Splatter(D, th.shape[0], B, tile=16, chunk=64, with_ctf=False)
    Qb, _ = sp.forward(t, W)
    assert torch.equal(Qc, Qb)
    eng.close()
    sp.close()
