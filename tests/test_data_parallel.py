"""Data-parallel step on CPU with two gloo ranks: Theta stays identical on every rank and the
update equals the single-process update on the concatenated batch (the loss is a sum over
particles, Sec. 3.3.5).  The second test uses the method itself: each rank's gradient is the
FP64 oracle's dL/dTheta of its half of the particles, and the all-reduced gradient equals the
oracle's gradient of the whole batch."""
import json
import os
import socket
import subprocess
import sys
import textwrap

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = textwrap.dedent("""
    import json, sys
    sys.path.insert(0, {root!r})
    import torch
    from paper_2508_04929_b300 import distributed as DP
    rank, world = DP.init_from_env("gloo")
    torch.manual_seed(100 + rank)
    theta = torch.randn(7, 11, dtype=torch.float64)  # differs per rank until broadcast
    # each rank's batch: a quadratic loss sum_p |theta - y_p|^2 over its own targets
    g = torch.Generator().manual_seed(7)
    targets = torch.randn(4, 7, 11, generator=g, dtype=torch.float64)  # the whole batch
    mine = targets[2 * rank: 2 * rank + 2]

    def local_grad(th, d):
        d += 2.0 * (th[None] - mine).sum(0)

    def adam_like(th, d):  # plain gradient step: linear in the gradient
        th -= 0.01 * d

    step = DP.DataParallelStep(theta, local_grad, adam_like)
    for _ in range(3):
        step()
    print(json.dumps({{"rank": rank, "theta": theta.flatten().tolist()}}))
""")


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_two_rank_data_parallel_step_matches_single_process():
    port = _free_port()
    procs = []
    for r in range(2):
        env = dict(os.environ, RANK=str(r), WORLD_SIZE="2", MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port),
                   CUDA_VISIBLE_DEVICES="")
        procs.append(subprocess.Popen([sys.executable, "-c", CHILD.format(root=ROOT)], env=env,
                                      stdout=subprocess.PIPE, stderr=subprocess.PIPE, text=True))
    outs = []
    for p in procs:
        o, e = p.communicate(timeout=240)
        assert p.returncode == 0, e[-2000:]
        outs.append(json.loads(o.strip().splitlines()[-1]))
    import torch
    t0 = torch.tensor(outs[0]["theta"], dtype=torch.float64)
    t1 = torch.tensor(outs[1]["theta"], dtype=torch.float64)
    assert torch.equal(t0, t1)  # replicated
    # single process on the whole batch, from rank 0's initial Theta
    torch.manual_seed(100)
    theta = torch.randn(7, 11, dtype=torch.float64)
    g = torch.Generator().manual_seed(7)
    targets = torch.randn(4, 7, 11, generator=g, dtype=torch.float64)
    for _ in range(3):
        theta -= 0.01 * 2.0 * (theta[None] - targets).sum(0)
    assert torch.allclose(t0, theta.flatten(), rtol=0, atol=1e-12)


ORACLE_CHILD = textwrap.dedent("""
    import json, sys
    sys.path.insert(0, {root!r})
    import numpy as np
    import torch
    import oracle as O
    from paper_2508_04929_b300 import distributed as DP, synth
    rank, world = DP.init_from_env("gloo")
    rng = synth.rng_for(31)
    D, N, B = 24, 40, 4
    th = synth.random_gaussians(N, D, rng)
    Ws = synth.random_poses(B, rng)
    ctf = synth.random_ctf(B, rng)
    Y = synth.smooth_field(B, D, rng)
    mine = slice(rank * (B // world), (rank + 1) * (B // world))
    theta = torch.from_numpy(th.astype(np.float64))

    def local_grad(t, d):  # this rank's particles only: the splat loss and gradient of the oracle
        d += torch.from_numpy(O.forward_backward(th, Ws[mine], D, Y[mine], ctf[mine])["dtheta"])

    seen = []
    step = DP.DataParallelStep(theta, local_grad, lambda t, d: seen.append(d.clone()))
    step()
    print(json.dumps({{"rank": rank, "grad": seen[0].flatten().tolist()}}))
""")


def test_all_reduced_oracle_gradient_equals_the_whole_batch():
    """Two gloo ranks, two particles each: the all-reduce of the ranks' oracle gradients equals
    the oracle gradient of all four particles (to 1e-12), the additivity that the data-parallel
    training step relies on."""
    port = _free_port()
    procs = []
    for r in range(2):
        env = dict(os.environ, RANK=str(r), WORLD_SIZE="2", MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port),
                   CUDA_VISIBLE_DEVICES="")
        procs.append(subprocess.Popen([sys.executable, "-c", ORACLE_CHILD.format(root=ROOT)], env=env,
                                      stdout=subprocess.PIPE, stderr=subprocess.PIPE, text=True))
    outs = []
    for p in procs:
        o, e = p.communicate(timeout=240)
        assert p.returncode == 0, e[-2000:]
        outs.append(json.loads(o.strip().splitlines()[-1]))
    import numpy as np
    sys.path.insert(0, ROOT)
    import oracle as O
    from paper_2508_04929_b300 import synth
    rng = synth.rng_for(31)
    D, N, B = 24, 40, 4
    th = synth.random_gaussians(N, D, rng)
    Ws = synth.random_poses(B, rng)
    ctf = synth.random_ctf(B, rng)
    Y = synth.smooth_field(B, D, rng)
    full = O.forward_backward(th, Ws, D, Y, ctf)["dtheta"].flatten()
    g0, g1 = np.array(outs[0]["grad"]), np.array(outs[1]["grad"])
    assert np.array_equal(g0, g1)
    assert np.abs(full).max() > 0
    assert np.max(np.abs(g0 - full)) <= 1e-12 * np.abs(full).max()

