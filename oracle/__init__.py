"""Plain FP64 CPU oracle of the cryoSplat orthographic splatting path.

This package is TEST INFRASTRUCTURE.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import it.  The product
path (``paper_2508_04929_b300``) never imports, calls or links anything here, and this
package imports nothing from the product path: the two share no code.  The only module
both sides use is the seeded input generator ``paper_2508_04929_b300.synth``, which holds
none of the method's arithmetic and which the oracle itself does not import either (the
tests hand the same arrays to both sides).

Every function follows the passage of the paper (arXiv 2508.04929, "CryoSplat: Gaussian
Splatting for Cryo-EM Homogeneous Reconstruction") that it cites, in the paper's order and
notation.  Floating point is FP64 throughout, except the integer support decision
(``support_fp32``), which is taken in FP32 like the kernel takes it.

Parity pins: every function here is pinned by a ``-m "not gpu"`` test in
``tests/test_oracle_pins.py`` against something other than itself (closed forms,
quadrature, brute force, library routines for special cases, invariants).
"""
from .gs_oracle import *  # noqa: F401,F403
from . import warm_oracle  # noqa: F401,E402  (learned warm start; not in the paper)
from . import volume_oracle  # noqa: F401,E402  (voxelization and FSC)
from . import pose_oracle  # noqa: F401,E402  (pose and translation gradients)
from . import algo_oracle  # noqa: F401,E402  (FourierShift and SplitGaussian of Algorithm 1)
