"""Autotuner for the rasterizer's launch shape: binning tile size and Gaussian chunk depth.

The support rule does not depend on the tile, so every candidate computes the same images
(bitwise) and the same gradients up to FP32 summation order; the tuner only times them.
Each candidate runs the batched fwd+CTF+loss+bwd pass on the caller's own inputs and is
timed with CUDA events on the current stream; the fastest is returned with the table.
The chunk depth only shapes the 16- and 32-pixel kernels, which stage records through
shared memory; the 8-pixel kernels read records directly, so tile 8 is timed once, at the
first chunk depth.
"""
from __future__ import annotations

import torch

from .splat import Splatter


def tune(D, N, B, theta, W, ctf, Y, device="cuda", tiles=(8, 16, 32), chunks=(64, 128, 256), iters=2):
    results = []
    for tile in tiles:
        for chunk in (chunks[:1] if tile == 8 else chunks):
            sp = Splatter(D, N, B, tile=tile, chunk=chunk, device=device)
            dth = torch.zeros_like(theta)
            sp.forward_backward(theta, W, ctf, Y, dth, grow=True, fused=True)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            for _ in range(iters):
                dth.zero_()
                sp.forward_backward(theta, W, ctf, Y, dth, grow=False, fused=True)
            e1.record()
            torch.cuda.synchronize()
            results.append({"tile": tile, "chunk": chunk, "ms": e0.elapsed_time(e1) / iters})
            sp.close()
            del sp
    best = min(results, key=lambda r: r["ms"])
    return {"tile": best["tile"], "chunk": best["chunk"], "ms": best["ms"], "table": results}
