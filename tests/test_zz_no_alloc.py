"""gs_bin_sort_noalloc against gs_bin_sort, through the C-ABI.

The no-allocation entry point serves callers that cannot allocate device memory (a
plug-in whose host application owns all device memory, a pipeline that must not allocate
while running).  It keeps its scratch in a fixed device array inside the library, so this
test checks that its outputs equal those of the workspace-based entry point bit for bit,
on two calls in a row with different batches (the array keeps the previous call's
contents), that a pair capacity below the need clips exactly as gs_bin_sort does, that an
empty batch sets the count to zero, that sizes beyond the array are refused with GS_ENOSPC,
and that a first call made during a stream capture is refused with GS_ECAPTURE without
disturbing the capture.  This file is collected last so that a run stopping at the first
failure has run everything else.
"""
import os
import subprocess
import sys

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2508_04929_b300 import build, synth  # noqa: E402

build.build()
from paper_2508_04929_b300 import _lib as L  # noqa: E402
from paper_2508_04929_b300.splat import Splatter  # noqa: E402


def _batch(seed, D, N, B, tile):
    rng = synth.rng_for(seed)
    th = torch.from_numpy(synth.random_gaussians(N, D, rng)).cuda()
    W = torch.from_numpy(synth.random_poses(B, rng).reshape(B, 9)).cuda()
    sp = Splatter(D, N, B, tile=tile, with_ctf=False)
    sp.project(th, W)
    sp.bin_sort(grow=True)
    torch.cuda.synchronize()
    return sp


@pytest.mark.parametrize("seeds", [((101, 64, 2000, 8, 16), (102, 96, 5000, 5, 8))])
def test_noalloc_matches_workspace_binning_on_two_calls(seeds):
    for seed, D, N, B, tile in seeds:
        sp = _batch(seed, D, N, B, tile)
        need = int(sp.n_pairs.item())
        pairs = torch.full((need + 64,), -1, dtype=torch.int32, device="cuda")
        ranges = torch.full_like(sp.ranges, -1)
        npairs = torch.zeros(1, dtype=torch.int32, device="cuda")
        scratch = L.gs_bin_sort_noalloc(sp.cfg, sp.proj, B, N, pairs, ranges, npairs)
        torch.cuda.synchronize()
        assert 0 < scratch <= 8 << 20
        assert int(npairs.item()) == need
        assert torch.equal(pairs[:need], sp.pairs[:need])
        assert torch.equal(ranges, sp.ranges)
        sp.close()


def test_noalloc_overflow_clips_like_the_workspace_call():
    """pair_capacity below the need: *n_pairs reports the need, the ranges are clipped to the
    capacity and pairs[:cap] hold the first instances, as gs_bin_sort reports them."""
    sp = _batch(103, 64, 2000, 4, 16)
    need = int(sp.n_pairs.item())
    cap = need // 3
    ref = Splatter(64, 2000, 4, tile=16, with_ctf=False, pair_capacity=cap)
    rng = synth.rng_for(103)
    th = torch.from_numpy(synth.random_gaussians(2000, 64, rng)).cuda()
    W = torch.from_numpy(synth.random_poses(4, rng).reshape(4, 9)).cuda()
    ref.project(th, W)
    ref.bin_sort(grow=False)
    torch.cuda.synchronize()
    assert int(ref.n_pairs.item()) == need and ref.status() & L.GS_STATUS_OVERFLOW
    pairs = torch.full((cap,), -1, dtype=torch.int32, device="cuda")
    ranges = torch.full_like(sp.ranges, -1)
    npairs = torch.zeros(1, dtype=torch.int32, device="cuda")
    L.gs_bin_sort_noalloc(sp.cfg, sp.proj, 4, 2000, pairs, ranges, npairs)
    torch.cuda.synchronize()
    assert int(npairs.item()) == need
    assert int(ranges.max().item()) <= cap
    assert torch.equal(ranges, ref.ranges)
    assert torch.equal(pairs, ref.pairs[:cap])
    sp.close()
    ref.close()


def test_noalloc_empty_batch_sets_zero_pairs():
    cfg = L.config(64, tile=16)
    npairs = torch.full((1,), 7, dtype=torch.int32, device="cuda")
    L.gs_bin_sort_noalloc(cfg, None, 0, 100, None, None, npairs)
    torch.cuda.synchronize()
    assert int(npairs.item()) == 0


_CAPTURE_PROBE = r"""
import torch
from paper_2508_04929_b300 import _lib as L
cfg = L.config(64, tile=16)
proj = torch.zeros(L.gs_proj_size(1, 10), dtype=torch.uint8, device="cuda")
ranges = torch.zeros(32, dtype=torch.int32, device="cuda")
npairs = torch.zeros(1, dtype=torch.int32, device="cuda")
pairs = torch.zeros(64, dtype=torch.int32, device="cuda")
torch.cuda.synchronize()
g = torch.cuda.CUDAGraph()
s = torch.cuda.Stream()
rc = None
with torch.cuda.stream(s):
    g.capture_begin()
    try:
        L.gs_bin_sort_noalloc(cfg, proj, 1, 10, pairs, ranges, npairs, stream=s)
    except L.GsError as e:
        rc = e.rc
    g.capture_end()
torch.cuda.synchronize()
L.gs_bin_sort_noalloc(cfg, proj, 1, 10, pairs, ranges, npairs)
torch.cuda.synchronize()
print("RC", rc, "PAIRS", int(npairs.item()))
"""


def test_noalloc_first_call_during_capture_is_refused():
    """The first call on a device looks up the array's address, which must not happen inside
    a stream capture: on a capturing stream it returns GS_ECAPTURE and leaves the capture
    intact; outside the capture the same call then works.  Run in a fresh process, where no
    earlier call has looked the address up."""
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    out = subprocess.run([sys.executable, "-c", _CAPTURE_PROBE], cwd=root, capture_output=True, text=True,
                         timeout=300)
    assert out.returncode == 0, out.stderr[-2000:]
    assert f"RC {L.GS_ECAPTURE} PAIRS 10" in out.stdout, out.stdout + out.stderr[-2000:]


def test_noalloc_refuses_sizes_beyond_its_array():
    cfg = L.config(256, tile=8)
    proj = torch.empty(32, dtype=torch.uint8, device="cuda")
    ranges = torch.empty(2, dtype=torch.int32, device="cuda")
    npairs = torch.zeros(1, dtype=torch.int32, device="cuda")
    with pytest.raises(L.GsError) as e:
        L.gs_bin_sort_noalloc(cfg, proj, 128, 200_000, None, ranges, npairs)
    assert e.value.rc == L.GS_ENOSPC
