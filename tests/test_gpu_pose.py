"""GPU parity of the pose and translation gradients (gs_render_bwd_pose) with the FP64
oracle.  Tolerance: 1e-3 relative L2 per particle, as for the Gaussian gradients (FP32 sums of
FP32 per-pixel terms over thousands of pixels)."""
import numpy as np
import pytest
import torch

from oracle import pose_oracle as PO

pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("needs a GPU", allow_module_level=True)

from paper_2508_04929_b300 import _lib as L  # noqa: E402
from paper_2508_04929_b300 import synth  # noqa: E402
from paper_2508_04929_b300.splat import Splatter  # noqa: E402

DEV = "cuda"


def rel(a, b):
    a, b = np.asarray(a, np.float64), np.asarray(b, np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


@pytest.mark.parametrize("tile", [8, 16])
def test_pose_gradients_match_oracle(tile):
    rng = synth.rng_for(51)
    D, N, B = 40, 80, 3
    th = synth.random_gaussians(N, D, rng)
    Ws = synth.random_poses(B, rng)
    G = synth.smooth_field(B, D, rng)
    dW_o, dt_o = PO.pose_backward(th, Ws, D, G)
    sp = Splatter(D, N, B, tile=tile, device=DEV, with_ctf=False)
    t = torch.from_numpy(th).to(DEV)
    W = torch.from_numpy(Ws.reshape(B, 9)).to(DEV)
    sp.forward(t, W)
    dth = torch.zeros_like(t)
    dpose = torch.zeros((B, 12), device=DEV)
    sp.backward(t, W, torch.from_numpy(G).to(DEV), dth, dpose=dpose)
    dth_plain = torch.zeros_like(t)
    sp.backward(t, W, torch.from_numpy(G).to(DEV), dth_plain)
    torch.cuda.synchronize()
    p = dpose.cpu().numpy().astype(np.float64)
    for b in range(B):
        assert rel(p[b, 0:6], dW_o[b, 0:2].ravel()) <= 1e-3, b
        assert rel(p[b, 10:12], dt_o[b]) <= 1e-3, b
    assert np.all(p[:, 6:10] == 0)  # depth row and the unused slot
    assert rel(dth.cpu().numpy(), dth_plain.cpu().numpy()) <= 1e-5


def test_pose_entry_rejects_missing_output():
    sp = Splatter(16, 4, 1, tile=8, device=DEV, with_ctf=False)
    t = torch.from_numpy(synth.random_gaussians(4, 16, synth.rng_for(1))).to(DEV)
    W = torch.eye(3, device=DEV).reshape(1, 9)
    sp.forward(t, W)
    with pytest.raises(L.GsError):
        L.gs_render_bwd_pose(sp.cfg, t, W, sp.proj, sp.pairs, sp.ranges, torch.zeros(1, 16, 16, device=DEV),
                             torch.zeros_like(t), None, sp.ws)
