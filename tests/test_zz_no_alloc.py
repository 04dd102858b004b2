"""gs_bin_sort_noalloc against gs_bin_sort, through the C-ABI.

The no-allocation entry point serves callers that cannot allocate device memory (a
plug-in whose host application owns all device memory, a pipeline that must not allocate
while running).  It keeps its scratch in a fixed device array inside the library, so this
test checks that its outputs equal those of the workspace-based entry point bit for bit,
on two calls in a row with different batches (the array keeps the previous call's
contents), and that sizes beyond the array are refused with GS_ENOSPC.  This file is
collected last so that a run stopping at the first failure has run everything else.
"""
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


def test_noalloc_refuses_sizes_beyond_its_array():
    cfg = L.config(256, tile=8)
    proj = torch.empty(32, dtype=torch.uint8, device="cuda")
    ranges = torch.empty(2, dtype=torch.int32, device="cuda")
    npairs = torch.zeros(1, dtype=torch.int32, device="cuda")
    with pytest.raises(L.GsError) as e:
        L.gs_bin_sort_noalloc(cfg, proj, 128, 200_000, None, ranges, npairs)
    assert e.value.rc == L.GS_ENOSPC
