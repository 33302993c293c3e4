"""Multi-rank logic of bench.py on CPU (gloo, two ranks) and the reference arm's output line."""
import json
import os
import socket
import subprocess
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import torch
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    import bgk_inputs as bi
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    p = bench.rank_config(bi.config(bench.WORKLOAD), rank, world)
    m = bench.reduce_max(float(10 + rank), dist, "cpu")
    dist.barrier()
    out[rank] = (p["kn"], m, p["n"])
    dist.destroy_process_group()


def test_two_ranks_take_independent_cavities_and_the_max_time():
    world, port = 2, _free_port()
    out = mp.get_context("spawn").Manager().dict()
    mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
    assert out[0][1] == out[1][1] == 11.0          # max over ranks
    assert out[0][0] != out[1][0]                  # Kn sweep by rank (weak scaling)
    assert out[0][2] == out[1][2] == 201           # same cavity size on every rank


def _plan_worker(rank, world, port, out):
    import torch
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    import bgk_inputs as bi
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    p = bi.config(bench.WORKLOAD)
    plan = bench.sharded_plan(p, rank, world)
    # the allreduce the sharded step makes, on buffers of the planned size
    xm = torch.full((plan["exchange_bytes"] // 8,), float(rank + 1), dtype=torch.float64)
    dist.all_reduce(xm)
    out[rank] = (plan["lo"], plan["hi"], plan["exchange_bytes"], float(xm[0]), float(xm[-1]))
    dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_velocity_sharded_plan_splits_the_grid_and_sums_over_ranks(world):
    # the multi-GPU line of bench.py (velocity slabs, strong scaling): the slabs of the
    # ranks tile the 32^2 velocity grid without overlap, every rank exchanges the same
    # (dim + 2) n + (2 dim + 6) n_wall doubles, and the allreduce sums over the ranks
    port = _free_port()
    out = mp.get_context("spawn").Manager().dict()
    mp.spawn(_plan_worker, args=(world, port, out), nprocs=world, join=True)
    spans = sorted((out[r][0], out[r][1]) for r in range(world))
    assert spans[0][0] == 0 and spans[-1][1] == 32 * 32
    assert all(spans[k][1] == spans[k + 1][0] for k in range(world - 1))
    n, n_wall = 201 ** 2, 4 * 200
    assert all(out[r][2] == 8 * (4 * n + 10 * n_wall) for r in range(world))
    total = world * (world + 1) / 2
    assert all(out[r][3] == total and out[r][4] == total for r in range(world))


def test_reference_arm_prints_its_line():
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "2",
                        "--warmup", "1"], capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr
    line = json.loads([ln for ln in r.stdout.splitlines() if ln.startswith("{")][-1])
    assert line["impl"] == "reference" and line["unit"] == "updates/s" and line["value"] > 0
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["cpu_baseline"]["kind"] == "oracle"
    # the oracle's OpenMP build on the bench workload itself, all host cores
    assert line["config"]["same_workload"] and line["config"]["points"] == 201 ** 2
    assert line["cpu_baseline"]["cores"] == line["cpu_baseline"]["host"]["logical_cores"] or \
        line["cpu_baseline"]["cores"] >= 1


def test_cpu_baseline_compares_the_library_with_the_oracle():
    # the cpu_baseline leg on a small cavity, with a stand-in library whose solver is the
    # oracle itself: the comparison runs end to end and finds no difference, and the
    # seeded start is the FP32-rounded perturbed Maxwellian
    sys.path.insert(0, ROOT)
    import numpy as np
    import bench
    import bgk_inputs as bi
    import oracle

    class _Solver:
        def __init__(self, ps, cls):
            self.p, self.cl = ps[0], cls[0]

        def set_f(self, f):
            self.sim = oracle.Simulation(self.p, self.cl, f0=f)

        def step(self, k):
            self.sim.run(k)

        def sync(self):
            pass

        def moments(self):
            return self.sim.rho, self.sim.U, self.sim.T

        def get_f(self):
            return self.sim.f

        def close(self):
            pass

    class _Lib:
        Solver = _Solver

    p = bi.config("cavity2d_ale_n201_v32_f32", n=13, nv=8)
    out = bench.cpu_baseline(p, 1, _Lib())
    e = out["oracle_errors"]
    assert e["steps"] == 3 and max(e["rho"], e["u"], e["T"], e["f"]) == 0.0, e
    f0 = bench.noisy_state(p, len(bi.cloud_for(p)["kind"]), 2408105)
    M = oracle.maxwellian(p, 1.0, (0.0, 0.0, 0.0), 1.0)
    assert f0.dtype == np.float32 and np.all(np.abs(f0 / M[None] - 1.0) <= 0.1 + 1e-6)
