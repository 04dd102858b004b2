"""GPU parity of FourierShift and SplitGaussian (Algorithm 1) with the FP64 oracle.

FourierShift: FP32 FFTs and FP32 coefficient products against FP64, 1e-5 relative L2 per
image (integer shifts: circular rolls, within 1e-5 of the maximum).  SplitGaussian: FP64
arithmetic rounded once to FP32 on the GPU, so the children agree to FP32 rounding.
"""
import numpy as np
import pytest
import torch

from oracle import algo_oracle as AO
import oracle as O

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


@pytest.mark.parametrize("D", [32, 33])
def test_fourier_shift_matches_oracle(D):
    rng = np.random.default_rng(71 + D)
    B = 4
    Y = synth.smooth_field(B, D, rng)
    h = 1.0 / D
    t = np.array([[0.37 * h, -1.6 * h], [-4.2 * h, 2.5 * h], [3 * h, -2 * h], [0.0, 0.0]], dtype=np.float32)
    ref = AO.fourier_shift(Y, t)
    sp = Splatter(D, 1, B, device=DEV)
    out = torch.empty((B, D, D), device=DEV)
    sp.fourier_shift(torch.from_numpy(Y).to(DEV), torch.from_numpy(t).to(DEV), out)
    got = out.cpu().numpy()
    for b in range(B):
        assert rel(got[b], ref[b]) <= 1e-5, b
    roll = np.roll(np.roll(Y[2], 3, axis=1), 2, axis=0)
    assert np.max(np.abs(got[2] - roll)) <= 1e-5 * np.max(np.abs(Y[2]))
    assert np.max(np.abs(got[3] - Y[3])) <= 1e-5 * np.max(np.abs(Y[3]))


def test_split_matches_oracle():
    rng = synth.rng_for(72)
    N = 500
    th = synth.random_gaussians(N, 128, rng)
    th[0, 3:6] = th[0, 3]  # a tie between scales: the lower axis wins on both sides
    ref = AO.split_gaussians(th, alpha=0.5)
    t = torch.from_numpy(th).to(DEV)
    out = torch.empty((2 * N, 11), device=DEV)
    L.gs_split_gaussians(t, out, alpha=0.5)
    got = out.cpu().numpy().astype(np.float64)
    assert np.allclose(got[:, 0:3], ref[:, 0:3], rtol=0, atol=2e-7)
    assert np.allclose(got[:, 3:6], ref[:, 3:6], rtol=2e-6, atol=1e-6)
    assert np.array_equal(got[:, 6:10], np.repeat(th[None, :, 6:10], 2, axis=0).reshape(2 * N, 4).astype(np.float64))
    assert np.allclose(got[:, 10], ref[:, 10], rtol=2e-6, atol=1e-6)
    # the children of every Gaussian keep its mass (through the splatting oracle's builder)
    p, c = O.build_gaussians(th.astype(np.float64)), O.build_gaussians(got)
    assert np.allclose(c["A"][:N] + c["A"][N:], p["A"], rtol=1e-5)
