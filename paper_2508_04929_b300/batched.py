"""Batched, CUDA-graph-captured training steps (Algorithm 1's loop body over a minibatch).

``GraphStep`` records, once, the whole step for one or several *problems* -- a problem is
a volume (theta, N Gaussians) with its own box size D and a batch of B particles with
their own poses, CTF parameters and observed images -- into a single CUDA graph:

    per problem: zero grad -> gs_project -> gs_bin_sort -> gs_render_fwd -> gs_ctf_loss_grad
                 (CTF, loss, adjoint CTF) -> gs_render_bwd -> gs_step_counted

Problems of a mixed batch (different D and N) run on their own streams inside the graph,
so small volumes overlap large ones; one ``replay()`` launches the whole batch.  Inputs
change between steps by copying into the static buffers (``load``); the Adam step counter
lives on the device so replays need no host values.  The step can also be replayed as two
graphs, ``replay_front()`` (projection, binning, render: it reads the poses only) and
``replay_back()`` (CTF, loss, backward, Adam: the observed images), so that a step's images
may still be arriving while its front half runs.  The pair buffers are sized by an
eager pass with a margin; ``check()`` reads the status words (a host sync) and re-sizes and
re-records if a step ever needed more pairs.  The tile size and chunk depth of every
problem come from the autotuner unless given.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import torch

from . import _lib as L
from .autotune import tune
from .splat import Splatter


@dataclass
class Problem:
    D: int
    theta: torch.Tensor          # [N, 11] raw parameters (updated in place by Adam)
    W: torch.Tensor              # [B, 9] poses
    ctf: torch.Tensor            # [B, 5]
    Y: torch.Tensor              # [B, D, D] observed images
    tile: int = 0                # 0 = autotune
    chunk: int = 0               # 0 = autotune
    lr: float = 1e-3
    sp: Splatter = field(default=None, repr=False)
    dtheta: torch.Tensor = field(default=None, repr=False)
    m: torch.Tensor = field(default=None, repr=False)
    v: torch.Tensor = field(default=None, repr=False)
    t: torch.Tensor = field(default=None, repr=False)
    tune: dict = field(default=None, repr=False)

    @property
    def N(self):
        return self.theta.shape[0]

    @property
    def B(self):
        return self.W.shape[0]


class GraphStep:
    def __init__(self, problems, margin=1.3, adam=True, use_graph=True, autotune_chunks=(64, 128, 256),
                 min_pairs=4096):
        self.problems = list(problems)
        self.margin = float(margin)
        self.min_pairs = int(min_pairs)
        self.adam = adam
        self.use_graph = use_graph
        self.dev = self.problems[0].theta.device
        for p in self.problems:
            if p.tile == 0 or p.chunk == 0:
                p.tune = tune(p.D, p.N, p.B, p.theta, p.W, p.ctf, p.Y, device=self.dev,
                              tiles=(p.tile,) if p.tile else (8, 16, 32),
                              chunks=(p.chunk,) if p.chunk else autotune_chunks)
                p.tile, p.chunk = p.tune["tile"], p.tune["chunk"]
            p.sp = Splatter(p.D, p.N, p.B, tile=p.tile, chunk=p.chunk, device=self.dev)
            p.dtheta = torch.zeros_like(p.theta)
            p.m = torch.zeros_like(p.theta)
            p.v = torch.zeros_like(p.theta)
            p.t = torch.zeros(1, dtype=torch.int32, device=self.dev)
        self.streams = [torch.cuda.Stream(device=self.dev) for _ in self.problems]
        self.graph = None
        self.graph_front = self.graph_back = None  # recorded on first use
        self.slot_inputs = None  # [slot][problem] = (W, ctf, Y) for the per-slot graphs
        self.slot_graphs = None  # [slot] = (front, back)
        self._size_pairs()
        self._record()

    # -- set-up ----------------------------------------------------------------------------
    def _size_pairs(self):
        for p in self.problems:
            p.sp.forward(p.theta, p.W, p.ctf, grow=True)
            need = int(p.sp.n_pairs.item()) & 0xFFFFFFFF
            cap = max(int(need * self.margin), self.min_pairs)
            if not (cap <= p.sp.pairs.numel() <= 2 * cap):
                p.sp.pairs = torch.empty(cap, dtype=torch.int32, device=self.dev)
            L.gs_clear_status(p.sp.ws)
        torch.cuda.synchronize(self.dev)

    def _front(self, p):
        sp = p.sp
        p.dtheta.zero_()
        sp.project(p.theta, p.W)
        sp.bin_sort(grow=False)
        sp.render()

    def _back(self, p):
        sp = p.sp
        sp.ctf_loss_grad(sp.Q, p.ctf, p.Y)
        sp.backward(p.theta, p.W, sp.dQ, p.dtheta)
        if self.adam:
            L.gs_step_counted(p.theta, p.dtheta, p.m, p.v, p.t, lr=p.lr)

    def _body(self, p):
        self._front(p)
        self._back(p)

    def _run_all(self, part=None):
        body = part or self._body
        main = torch.cuda.current_stream(self.dev)
        if len(self.problems) == 1:
            body(self.problems[0])
            return
        for p, s in zip(self.problems, self.streams):
            s.wait_stream(main)
            with torch.cuda.stream(s):
                body(p)
        for s in self.streams:
            main.wait_stream(s)

    def _record(self):
        if not self.use_graph:
            return
        # warm the exact sequence once on a side stream (cuFFT, attribute set-up), then record
        saved = [(p.theta.clone(), p.m.clone(), p.v.clone(), p.t.clone()) for p in self.problems]
        side = torch.cuda.Stream(device=self.dev)
        side.wait_stream(torch.cuda.current_stream(self.dev))
        with torch.cuda.stream(side):
            self._run_all()
        torch.cuda.current_stream(self.dev).wait_stream(side)
        torch.cuda.synchronize(self.dev)
        for p, (th, m, v, t) in zip(self.problems, saved):
            p.theta.copy_(th); p.m.copy_(m); p.v.copy_(v); p.t.copy_(t)
        self.graph = self._capture(None)
        self.graph_front = self.graph_back = None
        if self.slot_graphs is not None:
            self.record_slots(len(self.slot_graphs))

    def _capture(self, part):
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, capture_error_mode="thread_local"):
            self._run_all(part)
        torch.cuda.synchronize(self.dev)
        return g

    def record_split(self):
        """Record the two halves of the step (done on first use otherwise).  The whole step
        has been warmed and recorded already, so its halves need no warm-up."""
        if not self.use_graph:
            return
        self.graph_front = self._capture(self._front)
        self.graph_back = self._capture(self._back)

    def record_slots(self, n=2):
        """Record the step's two halves once per input slot: slot k's graphs read poses, CTF
        parameters and images from their own buffers ``slot_inputs[k][problem]``, so that a
        feeder can copy a later step's inputs straight into another slot while this one runs
        (no device-to-device copy into the static buffers)."""
        if not self.use_graph:
            raise RuntimeError("input slots need the graph-captured step")
        if self.slot_inputs is None or len(self.slot_inputs) != n:
            self.slot_inputs = [[tuple(torch.empty_like(x) for x in (p.W, p.ctf, p.Y)) for p in self.problems]
                                for _ in range(n)]
        static = [(p.W, p.ctf, p.Y) for p in self.problems]
        graphs = []
        try:
            for k in range(n):
                for p, (W, ctf, Y) in zip(self.problems, self.slot_inputs[k]):
                    p.W, p.ctf, p.Y = W, ctf, Y
                graphs.append((self._capture(self._front), self._capture(self._back)))
        finally:
            for p, (W, ctf, Y) in zip(self.problems, static):
                p.W, p.ctf, p.Y = W, ctf, Y
        self.slot_graphs = graphs

    # -- use -------------------------------------------------------------------------------
    def load(self, i, W=None, ctf=None, Y=None):
        """Copy the next batch of problem i into the static buffers (stream-ordered)."""
        p = self.problems[i]
        for dst, src in ((p.W, W), (p.ctf, ctf), (p.Y, Y)):
            if src is not None:
                dst.copy_(src, non_blocking=True)

    def replay(self):
        """One step for every problem.  Returns the per-image loss tensors (device)."""
        if self.graph is not None:
            self.graph.replay()
        else:
            self._run_all()
        return [p.sp.loss[: p.B] for p in self.problems]

    def replay_front(self, slot=None):
        """The first half of a step (projection, binning, render); reads theta and W (those of
        input slot ``slot`` when given)."""
        if slot is not None:
            self.slot_graphs[slot][0].replay()
            return
        if not self.use_graph:
            self._run_all(self._front)
            return
        if self.graph_front is None:
            self.record_split()
        self.graph_front.replay()

    def replay_back(self, slot=None):
        """The second half (CTF, loss, backward, Adam); reads ctf and Y (those of input slot
        ``slot`` when given).  Returns the per-image loss tensors (device)."""
        if slot is not None:
            self.slot_graphs[slot][1].replay()
        elif not self.use_graph:
            self._run_all(self._back)
        else:
            if self.graph_back is None:
                self.record_split()
            self.graph_back.replay()
        return [p.sp.loss[: p.B] for p in self.problems]

    def check(self):
        """Read the status words (host sync).  If a pair buffer overflowed, re-size and
        re-record; returns the OR of the status bits seen."""
        st = 0
        for p in self.problems:
            st |= L.gs_read_status(p.sp.ws, clear=True)
        if st & L.GS_STATUS_OVERFLOW:
            self.margin = max(self.margin, 1.3) * 1.5
            self._size_pairs()
            self._record()
        return st

    def close(self):
        for p in self.problems:
            if p.sp is not None:
                p.sp.close()


class _ChunkedCopier:
    """Copies one step's pinned host inputs on side streams: the poses and CTF parameters first
    (event ``small``), then the images, in chunks on several streams when they are large (a
    single copy does not reach the link's bandwidth on every box: measured 19.4 GB/s with one
    copy and 22.8 GB/s with four), else in one copy (each extra stream costs the host about
    20 us a step).  The cross-stream events are created once."""

    CHUNK_BYTES = 16 << 20

    def __init__(self, device, copy_streams):
        self.streams = [torch.cuda.Stream(device=device) for _ in range(max(1, copy_streams))]
        self.start = torch.cuda.Event()
        self.parts_done = [torch.cuda.Event() for _ in self.streams]

    def copy(self, free, dsts, srcs, small, ready):
        """Wait for ``free``, copy (W, ctf, Y) into ``dsts``, record ``small`` after W and ctf and
        ``ready`` after everything, on the first stream."""
        main = self.streams[0]
        main.wait_event(free)
        dW, dc, dY = dsts
        W, ctf, Y = srcs
        n = len(self.streams) if dY.numel() * dY.element_size() >= self.CHUNK_BYTES else 1
        with torch.cuda.stream(main):
            dW.copy_(W, non_blocking=True)
            dc.copy_(ctf, non_blocking=True)
            small.record(main)
            if n == 1:
                dY.copy_(Y, non_blocking=True)
        if n > 1:
            self.start.record(main)
            parts = list(zip(dY.chunk(n), Y.chunk(n)))
            for k, (s, (dst, src)) in enumerate(zip(self.streams, parts)):
                if k:
                    s.wait_event(self.start)
                with torch.cuda.stream(s):
                    dst.copy_(src, non_blocking=True)
                if k:
                    self.parts_done[k].record(s)
            for k in range(1, len(parts)):
                main.wait_event(self.parts_done[k])
        ready.record(main)


class HostFeeder:
    """Double-buffered feeding of one problem of a GraphStep from pinned host memory: the
    next step's (W, ctf, Y) are copied host -> device on a side stream while the current step
    runs, and ``load()`` moves them into the graph's static buffers (a device-to-device copy on
    the current stream) just before the replay.  ``load_front()`` and ``load_back()`` split
    that for ``replay_front()`` / ``replay_back()``: the poses and CTF parameters are copied
    first, so that a step's front half can start while its images are still arriving."""

    def __init__(self, gs: GraphStep, i=0, copy_streams=4):
        p = gs.problems[i]
        self.gs, self.i = gs, i
        self.copier = _ChunkedCopier(p.theta.device, copy_streams)
        self.copy_stream = self.copier.streams[0]
        self.bufs = [tuple(torch.empty_like(x) for x in (p.W, p.ctf, p.Y)) for _ in range(2)]
        self.ready = [torch.cuda.Event() for _ in range(2)]
        self.ready_small = [torch.cuda.Event() for _ in range(2)]  # W and ctf
        self.free = [torch.cuda.Event() for _ in range(2)]
        self.filled = 0
        self.used = 0

    def prefetch(self, W, ctf, Y):
        """Start copying one step's pinned host inputs (W[B, 9], ctf[B, 5], Y[B, D, D])."""
        j = self.filled % 2
        # after its previous contents have been loaded
        self.copier.copy(self.free[j], self.bufs[j], (W, ctf, Y), self.ready_small[j], self.ready[j])
        self.filled += 1

    def load(self):
        """Make the oldest prefetched inputs the problem's current inputs (stream-ordered)."""
        j = self.used % 2
        cur = torch.cuda.current_stream()
        cur.wait_event(self.ready[j])
        W, ctf, Y = self.bufs[j]
        self.gs.load(self.i, W=W, ctf=ctf, Y=Y)
        self.free[j].record(cur)
        self.used += 1

    def load_front(self):
        """The oldest prefetched poses and CTF parameters become the current ones."""
        j = self.used % 2
        cur = torch.cuda.current_stream()
        cur.wait_event(self.ready_small[j])
        W, ctf, _ = self.bufs[j]
        self.gs.load(self.i, W=W, ctf=ctf)

    def load_back(self):
        """... and their images; completes the load that ``load_front()`` began."""
        j = self.used % 2
        cur = torch.cuda.current_stream()
        cur.wait_event(self.ready[j])
        self.gs.load(self.i, Y=self.bufs[j][2])
        self.free[j].record(cur)
        self.used += 1


class SlotFeeder:
    """Feeding of a single-problem GraphStep through its input slots (``record_slots``): each
    step's pinned host inputs are copied straight into the slot its graphs read, on side
    streams, while earlier steps run, and ``step()`` replays the slot's two halves.  The front
    half waits only for the poses and CTF parameters, the back half for the images; no input
    is copied again on the device."""

    def __init__(self, gs: GraphStep, copy_streams=4):
        if len(gs.problems) != 1:
            raise ValueError("SlotFeeder drives a GraphStep of one problem")
        if gs.slot_graphs is None:
            gs.record_slots(2)
        self.gs = gs
        self.n = len(gs.slot_graphs)
        self.copier = _ChunkedCopier(gs.problems[0].theta.device, copy_streams)
        self.ready_small = [torch.cuda.Event() for _ in range(self.n)]  # W and ctf of the slot
        self.ready = [torch.cuda.Event() for _ in range(self.n)]        # ... and its images
        self.free = [torch.cuda.Event() for _ in range(self.n)]         # its last step has run
        self.filled = 0
        self.used = 0

    def prefetch(self, W, ctf, Y):
        """Start copying one step's pinned host inputs (W[B, 9], ctf[B, 5], Y[B, D, D]) into the
        next free slot.  At most ``n`` steps may be prefetched ahead of ``step()``."""
        if self.filled - self.used >= self.n:
            raise RuntimeError("every input slot holds a step that has not run yet")
        j = self.filled % self.n
        self.copier.copy(self.free[j], self.gs.slot_inputs[j][0], (W, ctf, Y), self.ready_small[j], self.ready[j])
        self.filled += 1

    def step(self):
        """Run the oldest prefetched step (stream-ordered).  Returns the per-image losses
        (device)."""
        if self.used >= self.filled:
            raise RuntimeError("no prefetched step")
        j = self.used % self.n
        cur = torch.cuda.current_stream()
        cur.wait_event(self.ready_small[j])
        self.gs.replay_front(j)
        cur.wait_event(self.ready[j])
        loss = self.gs.replay_back(j)
        self.free[j].record(cur)
        self.used += 1
        return loss
