"""torch.autograd wrappers of the splatting path (render, CTF, loss).

``render(theta, W, engine)`` returns Q[B, D, D] and differentiates to theta through the
hand-written backward (gs_render_bwd).  The engine processes the particles in chunks and,
in the backward pass, recomputes each chunk's projection and per-tile Gaussian lists
(gs_project + gs_bin_sort) instead of keeping them alive between forward and backward, so
the memory held across the two passes is theta, W and Q only, whatever the batch size.
``apply_ctf`` (self-adjoint, so its backward is itself) and ``loss`` complete the image
formation model X = F^-1(H F Q), L = ||X - Y||^2 (App. A.2 Eq. 14, Sec. 3.3.5).
``ctf_loss`` is the two in one call (gs_ctf_loss_grad): it returns the loss and keeps dL/dQ
from its forward pass, without forming X.
"""
from __future__ import annotations

import torch

from . import _lib as L
from .splat import Splatter


class RenderEngine:
    """Chunked render / backward with recomputed tile lists."""

    def __init__(self, D, N, particles_per_chunk=64, tile=16, chunk=128, E=0.5, cutoff_sigma=3.0,
                 reduction=0, device="cuda"):
        self.D, self.N, self.P = int(D), int(N), int(particles_per_chunk)
        self.kw = dict(tile=tile, chunk=chunk, E=E, cutoff_sigma=cutoff_sigma, reduction=reduction, device=device)
        self._sp = {}

    def _splatter(self, B):
        if B not in self._sp:
            self._sp[B] = Splatter(self.D, self.N, B, **self.kw)
        return self._sp[B]

    def _chunks(self, B):
        for b0 in range(0, B, self.P):
            yield b0, min(B, b0 + self.P)

    def render(self, theta, W):
        B = W.shape[0]
        Q = torch.empty((B, self.D, self.D), dtype=torch.float32, device=theta.device)
        for b0, b1 in self._chunks(B):
            sp = self._splatter(b1 - b0)
            sp.project(theta, W[b0:b1])
            sp.bin_sort(grow=True)
            sp.render(out=Q[b0:b1])
        return Q

    def render_backward(self, theta, W, dQ):
        dtheta = torch.zeros_like(theta)
        for b0, b1 in self._chunks(W.shape[0]):
            sp = self._splatter(b1 - b0)
            sp.project(theta, W[b0:b1])  # recompute the lists of this chunk
            sp.bin_sort(grow=True)
            sp.backward(theta, W[b0:b1], dQ[b0:b1].contiguous(), dtheta)
        return dtheta

    def apply_ctf(self, inp, ctf):
        out = torch.empty_like(inp)
        for b0, b1 in self._chunks(inp.shape[0]):
            sp = self._splatter(b1 - b0)
            sp.apply_ctf(inp[b0:b1].contiguous(), ctf[b0:b1].contiguous(), out[b0:b1])
        return out

    def ctf_loss(self, Q, ctf, Y):
        """Per-image loss of X = CTF(Q) against Y and dL/dQ, by chunks (gs_ctf_loss_grad)."""
        B = Q.shape[0]
        loss = torch.empty(B, dtype=torch.float32, device=Q.device)
        dQ = torch.empty_like(Q)
        for b0, b1 in self._chunks(B):
            sp = self._splatter(b1 - b0)
            lo, g = sp.ctf_loss_grad(Q[b0:b1].contiguous(), ctf[b0:b1].contiguous(), Y[b0:b1].contiguous())
            loss[b0:b1] = lo
            dQ[b0:b1] = g
        return loss, dQ

    def close(self):
        for sp in self._sp.values():
            sp.close()
        self._sp.clear()


class _Render(torch.autograd.Function):
    @staticmethod
    def forward(ctx, theta, W, engine):
        ctx.engine = engine
        ctx.save_for_backward(theta, W)
        return engine.render(theta.contiguous(), W.contiguous())

    @staticmethod
    def backward(ctx, dQ):
        theta, W = ctx.saved_tensors
        return ctx.engine.render_backward(theta.contiguous(), W.contiguous(), dQ.contiguous()), None, None


class _CTF(torch.autograd.Function):
    @staticmethod
    def forward(ctx, Q, ctf, engine):
        ctx.engine = engine
        ctx.save_for_backward(ctf)
        return engine.apply_ctf(Q.contiguous(), ctf)

    @staticmethod
    def backward(ctx, dX):
        (ctf,) = ctx.saved_tensors
        return ctx.engine.apply_ctf(dX.contiguous(), ctf), None, None  # H_hat real and even


class _Loss(torch.autograd.Function):
    @staticmethod
    def forward(ctx, X, Y, cfg):
        B = X.shape[0]
        loss = torch.empty(B, dtype=torch.float32, device=X.device)
        dX = torch.empty_like(X)
        L.gs_loss(cfg, X.contiguous(), Y.contiguous(), loss, dX)
        ctx.save_for_backward(dX)
        return loss

    @staticmethod
    def backward(ctx, dloss):
        (dX,) = ctx.saved_tensors
        return dX * dloss.view(-1, 1, 1), None, None


class _CTFLoss(torch.autograd.Function):
    @staticmethod
    def forward(ctx, Q, ctf, Y, engine):
        loss, dQ = engine.ctf_loss(Q.contiguous(), ctf, Y)
        ctx.save_for_backward(dQ)
        return loss

    @staticmethod
    def backward(ctx, dloss):
        (dQ,) = ctx.saved_tensors
        return dQ * dloss.view(-1, 1, 1), None, None, None


def render(theta, W, engine: RenderEngine):
    """Q[B, D, D] = Rasterize(theta, W) (Algorithm 2), differentiable in theta."""
    return _Render.apply(theta, W, engine)


def apply_ctf(Q, ctf, engine: RenderEngine):
    """X = F^-1(H_hat . F(Q)) per image (App. A.2 Eq. 14), differentiable in Q."""
    return _CTF.apply(Q, ctf, engine)


def loss(X, Y, D, reduction=0):
    """Per-image L = ||X - Y||^2 (Sec. 3.3.5), differentiable in X."""
    return _Loss.apply(X, Y, L.config(D, reduction=reduction))


def ctf_loss(Q, ctf, Y, engine: RenderEngine):
    """Per-image L = ||CTF(Q) - Y||^2 (App. A.2 Eq. 14, Sec. 3.3.5), differentiable in Q: the
    value of loss(apply_ctf(Q, ctf), Y) in one call that does not form X."""
    return _CTFLoss.apply(Q, ctf, Y, engine)


def main(argv=None):
    """Training steps through the autograd path at scale, the lists recomputed in the
    backward: one step = render -> CTF + loss -> backward -> Adam over the whole batch.
    Prints one JSON line (images/s, ms per step, peak device memory)."""
    import argparse
    import json
    import math

    from . import synth

    ap = argparse.ArgumentParser(description="autograd training steps with recomputed tile lists")
    ap.add_argument("--D", type=int, default=256)
    ap.add_argument("--N", type=int, default=200_000)
    ap.add_argument("--B", type=int, default=256)
    ap.add_argument("--chunk-particles", type=int, default=64)
    ap.add_argument("--tile", type=int, default=8)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=2)
    ap.add_argument("--chains", type=int, default=1, help="Gaussians on random-walk chains (1) or uniform (0)")
    a = ap.parse_args(argv)
    dev = torch.device("cuda")
    rng = synth.rng_for(0)
    make = synth.chain_gaussians if a.chains else synth.random_gaussians
    theta = torch.from_numpy(make(a.N, a.D, rng)).to(dev).requires_grad_(True)
    W = torch.from_numpy(synth.random_poses(a.B, rng).reshape(a.B, 9)).to(dev)
    C = torch.from_numpy(synth.random_ctf(a.B, rng)).to(dev)
    eng = RenderEngine(a.D, a.N, particles_per_chunk=a.chunk_particles, tile=a.tile, device=dev)
    with torch.no_grad():
        gt = torch.from_numpy(make(a.N, a.D, rng)).to(dev)
        X = apply_ctf(render(gt, W, eng), C, eng)
        Y = X + math.sqrt(float(X.double().var()) / 0.1) * torch.randn_like(X)
    m = torch.zeros_like(theta)
    v = torch.zeros_like(theta)
    t_dev = torch.zeros(1, dtype=torch.int32, device=dev)

    def step():
        theta.grad = None
        Ls = ctf_loss(render(theta, W, eng), C, Y, eng).sum()
        Ls.backward()
        with torch.no_grad():
            L.gs_step_counted(theta.data, theta.grad, m, v, t_dev, lr=1e-3)
        return Ls

    for _ in range(a.warmup):
        step()
    torch.cuda.synchronize()
    torch.cuda.reset_peak_memory_stats(dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(a.steps):
        last = step()
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / a.steps
    out = {"workload": f"autograd training step, D={a.D}, N={a.N} ({'chains' if a.chains else 'uniform'}), "
                       f"B={a.B}, lists recomputed per {a.chunk_particles}-particle chunk in the backward",
           "images_per_s": a.B / (ms * 1e-3), "ms_per_step": ms, "loss": float(last.detach()),
           "peak_device_bytes": torch.cuda.max_memory_allocated(dev)}
    print(json.dumps(out))
    eng.close()
    return out


if __name__ == "__main__":
    main()
