"""Device buffers and call sequence for one batch of particles (Algorithm 1 loop body).

``Splatter`` owns the torch-allocated buffers that the C-ABI calls need for a fixed
(D, N, B) and runs the path: gs_project -> gs_bin_sort -> gs_render_fwd -> gs_apply_ctf ->
gs_loss -> gs_apply_ctf (adjoint) -> gs_render_bwd -> gs_step, or with the three middle steps
fused into gs_ctf_loss_grad.  Every step runs in libgs;
this module only allocates and sequences.
"""
from __future__ import annotations

import torch

from . import _lib as L


def default_pair_capacity(B: int, N: int, tile: int) -> int:
    per = {8: 6, 16: 4, 32: 3}[tile]
    return max(1024, B * N * per)


class Splatter:
    """Buffers and calls for batches of B particles, N Gaussians, D x D images."""

    def __init__(self, D, N, B, tile=16, chunk=128, E=0.5, cutoff_sigma=3.0, reduction=0,
                 pair_capacity=None, device="cuda", with_ctf=True):
        self.D, self.N, self.B = int(D), int(N), int(B)
        self.N_cap = self.N  # buffers hold up to N_cap Gaussians; project() sets the active N
        self.cfg = L.config(D, E, tile, chunk, cutoff_sigma, reduction)
        self.device = torch.device(device)
        self.Tn = L.gs_tiles_per_image(self.cfg)
        self.fft = L.gs_fft_create(self.D, max(self.B, 1)) if (with_ctf and self.B > 0) else None
        fw = self.fft.work_bytes if self.fft is not None else 0
        ws_bytes = L.gs_workspace_size(self.cfg, self.B, self.N, fw)
        dev = self.device
        self.ws = torch.empty(ws_bytes, dtype=torch.uint8, device=dev)
        self.proj = torch.empty(max(L.gs_proj_size(self.B, self.N), 1), dtype=torch.uint8, device=dev)
        self.ranges = torch.empty(max(self.B * self.Tn * 2, 2), dtype=torch.int32, device=dev)
        self.n_pairs = torch.zeros(1, dtype=torch.int32, device=dev)
        cap = default_pair_capacity(self.B, self.N, tile) if pair_capacity is None else int(pair_capacity)
        self.pairs = torch.empty(max(cap, 1), dtype=torch.int32, device=dev)
        shape = (self.B, self.D, self.D)
        self.Q = torch.empty(shape, dtype=torch.float32, device=dev)
        self.X = torch.empty(shape, dtype=torch.float32, device=dev)
        self.dX = torch.empty(shape, dtype=torch.float32, device=dev)
        self.dQ = torch.empty(shape, dtype=torch.float32, device=dev)
        self.loss = torch.empty(max(self.B, 1), dtype=torch.float32, device=dev)
        L.gs_clear_status(self.ws)

    def close(self):
        if self.fft is not None:
            L.gs_fft_destroy(self.fft)
            self.fft = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- individual steps ------------------------------------------------------------------
    def project(self, theta, W):
        n = theta.shape[0]
        if n > self.N_cap or W.shape[0] != self.B:
            raise ValueError(f"Splatter holds N <= {self.N_cap}, B = {self.B}; got N = {n}, B = {W.shape[0]}")
        self.N = n
        L.gs_project(self.cfg, theta, W, self.proj, self.ws)

    def bin_sort(self, grow=True):
        """Bin and sort.  With ``grow`` the needed pair count is read back (a host sync) and
        the pair buffer is enlarged and the call repeated if it was too small."""
        L.gs_bin_sort(self.cfg, self.proj, self.B, self.N, self.ws, self.pairs, self.ranges, self.n_pairs)
        if grow:
            need = int(self.n_pairs.item()) & 0xFFFFFFFF
            if need > self.pairs.numel():
                self.pairs = torch.empty(int(need * 1.25) + 1024, dtype=torch.int32, device=self.device)
                L.gs_clear_status(self.ws)
                L.gs_bin_sort(self.cfg, self.proj, self.B, self.N, self.ws, self.pairs, self.ranges,
                              self.n_pairs)
        return self

    def render(self, out=None):
        out = self.Q if out is None else out
        L.gs_render_fwd(self.cfg, self.proj, self.N, self.pairs, self.ranges, self.B, out)
        return out

    def apply_ctf(self, inp, ctf, out):
        L.gs_apply_ctf(self.cfg, inp, ctf, out, self.fft, self.ws)
        return out

    def fourier_shift(self, inp, t, out):
        """out = inp moved by t[B, 2] (model units), FourierShift of Algorithm 1."""
        L.gs_fourier_shift(self.cfg, inp, t, out, self.fft, self.ws)
        return out

    def loss_grad(self, X, Y):
        L.gs_loss(self.cfg, X, Y, self.loss, self.dX)
        return self.loss[: self.B], self.dX

    def ctf_loss_grad(self, Q, ctf, Y):
        """Loss and dL/dQ (into self.dQ) through CTF, loss and adjoint CTF in one call
        (Parseval in the Fourier domain); X is not formed."""
        L.gs_ctf_loss_grad(self.cfg, Q, Y, ctf, self.loss, self.dQ, self.fft, self.ws)
        return self.loss[: self.B], self.dQ

    def backward(self, theta, W, dQ, dtheta, dpose=None):
        """Accumulates dL/dtheta into dtheta; with ``dpose`` ([B, 12], zeroed by the caller)
        also dL/dW (dpose[:, 0:9], row-major) and dL/dt (dpose[:, 10:12])."""
        if dpose is None:
            L.gs_render_bwd(self.cfg, theta, W, self.proj, self.pairs, self.ranges, dQ, dtheta, self.ws)
        else:
            L.gs_render_bwd_pose(self.cfg, theta, W, self.proj, self.pairs, self.ranges, dQ, dtheta, dpose, self.ws)
        return dtheta

    def status(self, clear=True) -> int:
        return L.gs_read_status(self.ws, clear)

    # -- composed passes -------------------------------------------------------------------
    def forward(self, theta, W, ctf=None, grow=True):
        """Q (and X if ctf is given) for the batch."""
        self.project(theta, W)
        self.bin_sort(grow)
        self.render()
        if ctf is not None:
            self.apply_ctf(self.Q, ctf, self.X)
            return self.Q, self.X
        return self.Q, None

    def forward_backward(self, theta, W, ctf, Y, dtheta, grow=True, fused=False):
        """One fwd+CTF+loss+bwd pass; accumulates dL/dtheta into dtheta (caller zeroes it).
        Returns the per-image losses (device tensor).  fused: CTF, loss and adjoint CTF in
        one call that does not form X (as a training step runs them); otherwise X and dL/dX
        are left in self.X and self.dX."""
        if fused:
            self.forward(theta, W, None, grow)
            self.ctf_loss_grad(self.Q, ctf, Y)
        else:
            self.forward(theta, W, ctf, grow)
            self.loss_grad(self.X, Y)
            self.apply_ctf(self.dX, ctf, self.dQ)
        self.backward(theta, W, self.dQ, dtheta)
        return self.loss[: self.B]
