"""Host logic of the multi-GPU bench on CPU with two gloo ranks (no GPU).

The path shards by particles: every rank renders its own batch (weak scaling) and the job's
time is the maximum over ranks.  These tests run that host logic as two processes.
"""
import os
import socket
import subprocess
import sys
import textwrap

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = textwrap.dedent("""
    import json, os, sys, types
    sys.path.insert(0, {root!r})
    import torch.distributed as dist
    dist.init_process_group("gloo")
    rank, world = dist.get_rank(), dist.get_world_size()
    import importlib.util
    spec = importlib.util.spec_from_file_location("bench", os.path.join({root!r}, "bench.py"))
    bench = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(bench)
    args = types.SimpleNamespace(D=32, N=50, B=3)
    th, Ws, ctf, th_gt, _ = bench.make_inputs(args, seed=rank)
    out = {{"rank": rank, "world": world,
            "max": bench.max_over_ranks(1.5 + rank, dist),
            "w0": float(Ws[0, 0]), "theta0": float(th[0, 0])}}
    print(json.dumps(out), flush=True)
    dist.destroy_process_group()
""")


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _run_ranks(code, world=2, extra_env=None, timeout=240):
    port = _free_port()
    procs = []
    for r in range(world):
        env = dict(os.environ, RANK=str(r), WORLD_SIZE=str(world), LOCAL_RANK=str(r),
                   MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), CUDA_VISIBLE_DEVICES="")
        env.update(extra_env or {})
        procs.append(subprocess.Popen([sys.executable, "-c", code], env=env, stdout=subprocess.PIPE,
                                      stderr=subprocess.PIPE, text=True))
    outs = []
    for p in procs:
        o, e = p.communicate(timeout=timeout)
        assert p.returncode == 0, e[-2000:]
        outs.append(o)
    return outs


def test_two_rank_timing_is_max_and_batches_differ():
    import json
    outs = [json.loads(o.strip().splitlines()[-1]) for o in _run_ranks(CHILD.format(root=ROOT))]
    assert sorted(o["rank"] for o in outs) == [0, 1]
    assert all(o["world"] == 2 for o in outs)
    assert all(o["max"] == 2.5 for o in outs)          # the slowest rank's time
    assert outs[0]["w0"] != outs[1]["w0"]              # each rank draws its own particles
    assert outs[0]["theta0"] != outs[1]["theta0"]


def test_reference_arm_runs_on_rank_zero_only():
    """Under torchrun the reference arm prints from rank 0 and the other ranks exit without
    work."""
    code = textwrap.dedent(f"""
        import os, sys, types
        sys.path.insert(0, {ROOT!r})
        import importlib.util
        spec = importlib.util.spec_from_file_location("bench", os.path.join({ROOT!r}, "bench.py"))
        bench = importlib.util.module_from_spec(spec)
        spec.loader.exec_module(bench)
        calls = []
        bench.make_inputs = lambda *a, **k: calls.append(1) or (_ for _ in ()).throw(SystemExit(3))
        bench.run_reference(types.SimpleNamespace(), int(os.environ["RANK"]))
        print("done", len(calls))
    """)
    port = _free_port()
    env1 = dict(os.environ, RANK="1", WORLD_SIZE="2", MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    p = subprocess.run([sys.executable, "-c", code], env=env1, capture_output=True, text=True, timeout=120)
    assert p.returncode == 0 and p.stdout.strip().endswith("done 0"), p.stderr[-1000:]
    env0 = dict(env1, RANK="0")
    p = subprocess.run([sys.executable, "-c", code], env=env0, capture_output=True, text=True, timeout=120)
    assert p.returncode == 3  # rank 0 starts the work (stopped here by the stub)


def test_bench_starts_its_own_ranks_and_defaults_to_data_parallel():
    """bench.py --gpus 2 without a launcher starts two ranks itself (torch.distributed.run on
    127.0.0.1) and, with several ranks, times the data-parallel training step by default.  The
    dry run exercises that launch and the collective on the host (gloo) and prints the JSON line
    without a measurement."""
    import json
    env = dict(os.environ, CUDA_VISIBLE_DEVICES="")
    env.pop("WORLD_SIZE", None)
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--gpus", "2", "--dry-run", "--D", "32",
                          "--N", "200", "--B", "4"], cwd=ROOT, env=env, capture_output=True, text=True, timeout=300)
    assert out.returncode == 0, out.stderr[-3000:]
    lines = [json.loads(x) for x in out.stdout.splitlines() if x.startswith("{")]
    assert len(lines) == 1  # rank 0 alone prints
    line = lines[0]
    assert line["n_gpus"] == 2 and line["config"]["parallelism"] == "dp"
    assert line["dry_run"]["allreduce_ok"] and line["value"] is None



def test_plain_baseline_is_the_faster_variant():
    """The speedups divide by the faster of the plain form's two measured variants, so that the
    baseline is the best the per-image form achieved; a variant without a number is ignored."""
    import importlib.util
    spec = importlib.util.spec_from_file_location("bench", os.path.join(ROOT, "bench.py"))
    bench = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(bench)
    assert bench.best_plain({"presized": 2480.0, "grow_sync": 2774.0}) == 2774.0
    assert bench.best_plain({"presized": 7354.0, "grow_sync": 5828.0}) == 7354.0
    assert bench.best_plain({"presized": None, "grow_sync": 5828.0}) == 5828.0
    assert bench.best_plain({"presized": None, "grow_sync": None}) is None
    assert bench.best_plain(None) is None
