"""GMM voxelization and Fourier shell correlation (the evaluation of a reconstruction).

``voxelize(theta, D)`` evaluates the mixture on a D^3 grid (gs_voxelize) and ``fsc(v1, v2)``
returns the Fourier shell correlation per integer shell (gs_fsc).  ``resolution(curve,
apix)`` reads the resolution at a threshold (0.5 or 0.143) off an FSC curve.  Every step runs
in libgs; this module only allocates.
"""
from __future__ import annotations

import torch

from . import _lib as L

_plans = {}


def voxelize(theta, D, E=0.5, cutoff_sigma=3.0):
    """vol[D, D, D] (index [k][i][j]) of raw Gaussians theta[N, 11] (device)."""
    dev = theta.device
    vol = torch.empty((D, D, D), dtype=torch.float32, device=dev)
    ws = torch.empty(L.gs_voxel_workspace_size(theta.shape[0]), dtype=torch.uint8, device=dev)
    L.gs_voxelize(theta.contiguous(), D, vol, ws, E=E, cutoff_sigma=cutoff_sigma)
    return vol


def fsc(v1, v2):
    """FSC[D // 2 + 1] of two D^3 volumes (device tensors)."""
    D = v1.shape[-1]
    key = (D, v1.device.index)
    if key not in _plans:
        _plans[key] = L.gs_fsc_create(D)
    plan = _plans[key]
    ws = torch.empty(L.gs_fsc_workspace_size(plan), dtype=torch.uint8, device=v1.device)
    out = torch.empty(D // 2 + 1, dtype=torch.float32, device=v1.device)
    L.gs_fsc(plan, v1.contiguous(), v2.contiguous(), out, ws)
    return out


def resolution(curve, apix, threshold=0.143):
    """Resolution in Angstrom where the FSC curve first falls below ``threshold`` (linear
    interpolation between shells; shell s is the spatial frequency s / (D apix)).  Returns
    the Nyquist resolution 2 apix if it never does."""
    c = [float(x) for x in curve]
    D = 2 * (len(c) - 1)
    for s in range(1, len(c)):
        if c[s] < threshold:
            f0, f1 = c[s - 1], c[s]
            t = (f0 - threshold) / (f0 - f1) if f0 != f1 else 0.0
            freq = (s - 1 + t) / (D * apix)
            return 1.0 / freq if freq > 0 else float("inf")
    return 2.0 * apix
