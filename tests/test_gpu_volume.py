"""GPU parity of voxelization and FSC against the FP64 oracle.

Tolerances: the voxel values are FP32 sums of FP32 exponentials (ex2.approx, relative error
~2^-22) over a handful of Gaussians, so 1e-5 relative L2 and 1e-5 of the maximum per voxel;
the support boxes are integer decisions taken in the same FP32 sequence on both sides and
compared exactly (through the zero pattern).  FSC: FP32 FFTs against FP64, 1e-5 absolute.
"""
import numpy as np
import pytest
import torch

from oracle import volume_oracle as VO

pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("needs a GPU", allow_module_level=True)

from paper_2508_04929_b300 import synth  # noqa: E402
from paper_2508_04929_b300 import volume as V  # noqa: E402
from paper_2508_04929_b300.splat import Splatter  # noqa: E402

DEV = "cuda"


def rel(a, b):
    a, b = np.asarray(a, np.float64), np.asarray(b, np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


@pytest.mark.parametrize("D,N,seed", [(32, 40, 1), (33, 25, 2), (48, 200, 3)])
def test_voxelize_matches_oracle(D, N, seed):
    rng = synth.rng_for(seed)
    th = synth.random_gaussians(N, D, rng, centre_radius=0.45)  # some boxes clip at the faces
    ref = VO.voxelize(th, D)
    got = V.voxelize(torch.from_numpy(th).to(DEV), D).cpu().numpy()
    assert rel(got, ref) <= 1e-5
    assert np.max(np.abs(got - ref)) <= 1e-5 * np.max(np.abs(ref))
    # identical supports: nothing outside the oracle's boxes, and every value FP32 can hold
    # inside them (exponents far below -126 underflow in FP32 only)
    assert np.all(got[ref == 0] == 0)
    assert np.all(got[ref > 1e-25 * np.max(ref)] != 0)


def test_voxelize_edge_cases():
    D = 16
    empty = torch.zeros((0, 11), device=DEV)
    assert float(V.voxelize(empty, D).abs().sum()) == 0.0
    rng = synth.rng_for(4)
    th = synth.random_gaussians(5, D, rng)
    th[2, 4] = np.nan  # skipped, the others unaffected
    ref = VO.voxelize(np.delete(th, 2, axis=0), D)
    got = V.voxelize(torch.from_numpy(th).to(DEV), D).cpu().numpy()
    assert rel(got, ref) <= 1e-5


def test_projection_of_the_volume_is_the_rendered_image():
    """sum_k vol h on the GPU = the GPU render at W = I (the line integral of Sec. 3.3.3)."""
    rng = synth.rng_for(5)
    D, N = 48, 30
    th = synth.random_gaussians(N, D, rng, centre_radius=0.15, scale_px=(1.5, 2.5))
    t = torch.from_numpy(th).to(DEV)
    vol = V.voxelize(t, D, cutoff_sigma=6.0)
    sp = Splatter(D, N, 1, tile=8, cutoff_sigma=6.0, device=DEV, with_ctf=False)
    Q, _ = sp.forward(t, torch.eye(3, device=DEV).reshape(1, 9))
    proj = (vol.sum(0) * (1.0 / D)).cpu().numpy()
    q = Q[0].cpu().numpy()
    assert np.max(np.abs(proj - q)) <= 1e-5 * np.max(np.abs(q))


@pytest.mark.parametrize("D", [16, 15])
def test_fsc_matches_oracle(D):
    rng = np.random.default_rng(6 + D)
    a = rng.standard_normal((D, D, D)).astype(np.float32)
    b = (0.6 * a + rng.standard_normal((D, D, D))).astype(np.float32)
    ref = VO.fsc(a, b)
    got = V.fsc(torch.from_numpy(a).to(DEV), torch.from_numpy(b).to(DEV)).cpu().numpy()
    assert np.allclose(got, ref, atol=1e-5)
    same = V.fsc(torch.from_numpy(a).to(DEV), torch.from_numpy(a).to(DEV)).cpu().numpy()
    assert np.allclose(same, 1.0, atol=1e-6)


def test_resolution_reads_the_threshold_crossing():
    curve = [1.0, 0.9, 0.6, 0.4, 0.1]  # D = 8
    # 0.5 is crossed between shells 2 and 3, at 2.5: frequency 2.5 / (8 * 1.5 A)
    assert abs(V.resolution(curve, 1.5, 0.5) - 8 * 1.5 / 2.5) < 1e-9
    assert V.resolution([1.0, 0.9, 0.9], 2.0, 0.143) == 4.0  # never crosses: Nyquist
