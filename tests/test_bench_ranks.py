"""Host logic of the benchmark's multi-rank (replica) mode, on CPU with gloo."""
import json
import os
import socket
import subprocess
import sys

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    mine = 10.0 * (rank + 1)  # rank 1 is the slow one
    slowest = bench.max_over_ranks(mine, dist, "cpu")
    out[rank] = (slowest, bench.whole_job_value(world, 20, 900, slowest))
    dist.barrier()
    dist.destroy_process_group()


def test_max_over_ranks_and_whole_job_value_gloo_world_2():
    port = _free_port()
    with mp.Manager() as man:
        out = man.dict()
        mp.spawn(_worker, args=(2, port, out), nprocs=2, join=True)
        res = dict(out)
    assert res[0] == res[1]
    slowest, value = res[0]
    assert slowest == 20.0
    assert value == pytest.approx(2 * 20 * 900 / 0.020)


def test_single_rank_needs_no_process_group():
    assert bench.max_over_ranks(3.5, None, "cpu") == 3.5
    assert bench.whole_job_value(1, 10, 900, 5.0) == pytest.approx(10 * 900 / 0.005)


def test_reference_arm_runs_on_rank_0_only():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--gpus", "2",
                        "--steps", "3", "--warmup", "3"], env=env, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0
    assert r.stdout.strip() == ""


def test_reference_arm_times_the_oracle_on_every_core():
    """Rank 0 of the reference arm prints one line: the FP64 oracle run by one
    process per host core, its value the line's cpu_baseline and e2e."""
    env = dict(os.environ, RANK="0", WORLD_SIZE="1", LOCAL_RANK="0")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--workload", "tiny",
                        "--steps", "2", "--warmup", "3"], env=env, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr
    line = json.loads(r.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["value"] > 0
    assert line["cpu_baseline"]["cores"] == bench.host_cores()
    assert line["cpu_baseline"]["value"] == line["value"] == line["e2e"]["value"]
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["e2e"]["d2h_bytes_per_step"] == 0


def test_bench_nrmse_is_the_oracle_definition():
    """The bench's quality figure (its own code: the bench runs no oracle on
    the GPU side) equals the oracle's NRMSE over the illuminated mask, and is
    blind to a global phase."""
    import numpy as np

    from oracle import magpie_oracle as O
    from paper_2504_10118_gb300 import synth

    w = synth.WORKLOADS["tiny"]
    z_true, Q, pos = synth.make_problem(w)
    rng = np.random.default_rng(5)
    z = z_true + 0.05 * (rng.normal(size=z_true.shape) + 1j * rng.normal(size=z_true.shape))
    q2 = np.abs(Q) ** 2
    ref = O.nrmse(z, z_true, O.illuminated_mask(Q, pos, z_true.shape))
    assert bench.nrmse_lit(z, z_true, q2, pos) == pytest.approx(ref, rel=1e-12)
    assert bench.nrmse_lit(np.exp(0.7j) * z, z_true, q2, pos) == pytest.approx(ref, rel=1e-9)
