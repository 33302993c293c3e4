"""Benchmark of the per-time-step hot path (point-velocity updates per second).

Default workload: the 2D driven cavity with ALE motion, 201^2 points, 32^2
velocities in [-6, 6]^2, Kn = 0.1, lid 0.1, f stored in FP32 (the
configuration the headline metric is quoted on).  One step = one full time
step: cell lists, neighbour lists and WLS stencils (rebuilt every step under
ALE), upwind transport + moments + BGK relaxation, diffuse-reflection walls,
point motion.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun each rank runs its own independent cavity (Kn from the sweep
0.01 / 0.1 / 1 by rank): weak scaling, no data-path collective; the time is
the max over ranks.  Rank 0 prints one JSON line.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import bgk_inputs as bi  # noqa: E402

METRIC = "point·velocity updates/s, FP32/batched vs plain FP64 GPU at 1e-4 moments"
UNIT = "updates/s"
WORKLOAD = "cavity2d_ale_n201_v32_f32"
PEAKS_FALLBACK = {"hbm_gbs": 6800.0, "sm_max_mhz": 2070.0, "source": "fallback"}
N_SM = 152
FP32_LANES_PER_SM = 128
# Algorithmic FP32 lane-instructions per (point, neighbour, velocity) of the upwind
# transport, the smallest count the scheme admits: d projections abar_d (c.e_d), one FMA
# each from a base shared along a row of the velocity grid; c.coef, one FMA; d FMAs
# with |.| operand modifiers for the dissipation sum_d |abar_d c.e_d|; then per component
# (2D: g and h) one difference f_j - f_i and one accumulation.  2D: 2+1+2+2+2 = 9,
# 3D: 3+1+3+1+1 = 9.
OPS_PER_PAIR = {2: 9, 3: 9}


def _peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        d = json.load(open(path))
        d["source"] = "measured"
        return d
    return dict(PEAKS_FALLBACK)


def _dist_env():
    return int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("LOCAL_RANK", "0"))


def rank_config(p: dict, rank: int, world: int) -> dict:
    """The workload of one rank: every rank runs its own independent cavity of the same size
    (weak scaling); with ALE the ranks take the Kn sweep 0.01 / 0.1 / 1 in turn."""
    q = dict(p)
    if world > 1 and q.get("ale"):
        q["kn"] = bi.KN_SWEEP_ALE[rank % len(bi.KN_SWEEP_ALE)]
    return q


def reduce_max(value: float, dist, device) -> float:
    """Maximum of a per-rank value over all ranks (identity without a process group)."""
    if dist is None:
        return value
    import torch
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.FIELDS,
                                          "--format=csv,noheader,nounits", "-lms", "25"],
                                         stdout=self.fh, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None
            return
        # the first sample comes some 100 ms after the start: wait for it (3 s at most), so
        # that the samples that follow fall inside the timed region
        t0 = time.perf_counter()
        while time.perf_counter() - t0 < 3.0 and self.proc.poll() is None:
            if os.path.getsize(self.path) > 0:
                break
            time.sleep(0.01)
        with open(self.path) as fh:
            self.before = sum(1 for line in fh if line.endswith("\n"))

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.fh.close()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as fh:
            lines = fh.readlines()
        # the samples taken inside the timed region; when it was shorter than the sampling
        # interval, the ones just before it (the warm-up steps) stand in
        inside = lines[getattr(self, "before", 0):]
        for line in (inside if any(x.strip() for x in inside) else lines):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, val in zip(names, parts[5:9]):
                if val.lower() == "active":
                    reasons.add(nm)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def transport_source_sha() -> str:
    """Hash of the sources that define the transport kernel (step.cu and its headers)."""
    d = os.path.join(ROOT, "paper_2408_02350_gb300", "csrc")
    hs = hashlib.sha256()
    for f in ("step.cu", "transport_wp.cuh", "device_common.cuh", "bgk_internal.cuh"):
        hs.update(open(os.path.join(d, f), "rb").read())
    return hs.hexdigest()[:16]


def _traffic_record(kernel: str, workload: str):
    """DRAM bytes per launch from the committed ncu summary, if it matches the current kernel source."""
    path = os.path.join(ROOT, "profiles", "ncu_traffic.json")
    if not os.path.exists(path):
        return None
    try:
        rec = json.load(open(path))
    except ValueError:
        return None
    h = transport_source_sha()
    r = rec.get(kernel + ":" + workload)
    if not r or r.get("source_sha") != h:
        return None
    return r.get("dram_bytes_per_launch")


def noisy_state(p: dict, n: int, seed: int):
    """f = M(v; 1, 0, 1) (1 + 0.1 u), u uniform in [-1, 1] per (point, component, velocity)
    from SplitMix64, rounded to FP32 (the FP32 library and the FP64 oracle start from the
    same values)."""
    import oracle
    M = oracle.maxwellian(p, 1.0, (0.0, 0.0, 0.0), 1.0)
    u = bi.uniform01(seed, n * M.size).reshape((n,) + M.shape)
    return (M[None] * (1.0 + 0.1 * (2.0 * u - 1.0))).astype(np.float32)


def oracle_errors(g, p: dict, cl: dict, f0, sim, nsteps: int) -> dict:
    """The library's steps against the oracle's from the same state f0: relative max errors
    of rho and T, the velocity normwise (max |du| / max |u|) and f (max |df| / max |f|)."""
    s = g.Solver([p], [cl])
    try:
        s.set_f(np.ascontiguousarray(f0))
        s.step(nsteps)
        s.sync()
        rho, u, T = s.moments()
        f = s.get_f()
    finally:
        s.close()
    rel = lambda a, b: float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))
    return {"steps": nsteps, "start": "seeded non-uniform state f = M (1 + 0.1 u), FP32-rounded",
            "rho": rel(rho, sim.rho), "u": rel(u, sim.U), "T": rel(T, sim.T), "f": rel(f, sim.f)}


def cpu_baseline(p: dict, nsteps: int = 1, g=None) -> dict:
    """The FP64 CPU oracle on a bounded sample of the workload: single-threaded, and its
    OpenMP build (loops over points split among all host cores) beside it.  The OpenMP
    run starts from a seeded non-uniform state; with the library g given, the same three
    steps on the GPU are compared with it (`oracle_errors`)."""
    import oracle
    cl = bi.cloud_for(p)
    sim = oracle.Simulation(p, cl)
    t0 = time.perf_counter()
    sim.run(nsteps)
    dt = time.perf_counter() - t0
    n = cl["x"].shape[0]
    upd = n * p["nv"] ** p["dim"] * nsteps
    out = {"value": upd / dt, "unit": UNIT, "cores": 1, "kind": "oracle",
           "sample": "%d full time step(s) of the %d^%d x %d^%d cavity (%d points), FP64, one thread, %.1f s"
                     % (nsteps, p["n"], p["dim"], p["nv"], p["dim"], n, dt),
           "host": _host_cpu()}
    try:
        f0 = noisy_state(p, n, 2408105) if g is not None else None
        somp = oracle.Simulation(p, cl, omp=True, f0=f0)
        somp.run(1)  # warm-up: thread pool start
        k = max(2, nsteps)
        t0 = time.perf_counter()
        somp.run(k)
        dto = time.perf_counter() - t0
        thr = oracle.threads(True)
        out["omp"] = {"value": n * p["nv"] ** p["dim"] * k / dto, "unit": UNIT, "cores": thr,
                      "kind": "oracle_omp",
                      "sample": "%d full time steps of the same cavity after one warm-up step, FP64, OpenMP "
                                "over points on %d threads, %.1f s" % (k, thr, dto)}
    except (OSError, subprocess.CalledProcessError) as e:
        out["omp"] = {"unavailable": "OpenMP build of the oracle failed: %s" % e}
        return out
    if g is not None:
        try:
            out["oracle_errors"] = oracle_errors(g, p, cl, f0, somp, 1 + k)
        except Exception as e:  # noqa: BLE001 - a failed comparison must not cost the bench line
            out["oracle_errors"] = {"unavailable": "%s: %s" % (type(e).__name__, e)}
    return out


def _host_cpu() -> dict:
    """The host's CPU model and logical core count (the oracle uses one of them)."""
    import platform
    model = platform.processor() or platform.machine()
    try:
        for line in open("/proc/cpuinfo"):
            key = line.split(":")[0].strip().lower()
            if key in ("model name", "cpu part", "hardware"):
                model = line.split(":", 1)[1].strip()
                if key == "model name":
                    break
    except OSError:
        pass
    arm_parts = {"0xd4f": "Arm Neoverse V2", "0xd40": "Arm Neoverse V1", "0xd0c": "Arm Neoverse N1"}
    model = arm_parts.get(model.lower(), model)
    return {"model": model, "machine": platform.machine(), "logical_cores": os.cpu_count()}


def adjoint_cost(g, torch, stream) -> dict:
    """Forward step and adjoint step times on the adjoint workload, event-timed per kernel."""
    p = bi.config("adjoint2d_n101_v24_f32")
    cl = bi.cloud_for(p)
    s = g.Solver([p], [cl])
    s.set_maxwellian(stream=stream)
    s.step(3, stream=stream)
    s.sync(stream)
    n, NV = len(cl["kind"]), p["nv"] ** 2
    nvp = s.stats()["nv_pad"]
    lam = torch.randn((n, 2, nvp), dtype=torch.float32, device="cuda") * 1e-3
    lam2 = torch.zeros_like(lam)
    dth = torch.zeros(4, dtype=torch.float64, device="cuda")
    g.bgk_adjoint_step(s.ctx, 0, lam, lam2, dth, stream)  # allocates work buffers
    K = 50
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    s.step(K, stream=stream)
    e1.record(stream)
    torch.cuda.synchronize()
    fwd = e0.elapsed_time(e1) / K
    e0.record(stream)
    for _ in range(K):
        g.bgk_adjoint_step(s.ctx, 0, lam, lam2, dth, stream)
        lam, lam2 = lam2, lam
    e1.record(stream)
    torch.cuda.synchronize()
    adj = e0.elapsed_time(e1) / K
    s.sync(stream)
    s.close()
    return {"workload": "adjoint2d_n101_v24_f32", "points": n, "velocities": NV, "ms_forward_step": fwd,
            "ms_adjoint_step": adj, "ratio": adj / fwd}


def manage_cost(g, torch, stream, p: dict, name: str, steps: int = 200) -> dict:
    """One point-management pass (merge pairs closer than 0.25 dx, fill holes next to
    points with fewer than 14 neighbours) on the bench workload after `steps` ALE steps,
    wall-clock (the call is synchronous), against the mean step time."""
    cl = bi.cloud_for(p)
    n = len(cl["kind"])
    q = dict(p, spare_points=n // 16)
    s = g.Solver([q], [cl])
    s.set_maxwellian(stream=stream)
    s.step(steps, stream=stream)
    s.sync(stream)
    dx = 1.0 / (p["n"] - 1)
    s.manage(0.25 * dx, 14, stream=stream)  # allocates the scratch, removes what accumulated
    s.step(10, stream=stream)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    npts, removed, added = s.manage(0.25 * dx, 14, stream=stream)
    ms = (time.perf_counter() - t0) * 1e3
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    s.step(20, stream=stream)
    e1.record(stream)
    torch.cuda.synchronize()
    step_ms = e0.elapsed_time(e1) / 20
    s.sync(stream)
    s.close()
    return {"workload": name, "after_steps": steps + 10, "ms_per_pass": ms,
            "ms_per_step": step_ms, "points": npts, "removed": removed, "added": added}


def _rate(g, torch, stream, p: dict, steps: int) -> dict:
    """Device-resident updates/s of `steps` steps of workload p (after 3 warm-up steps)."""
    cl = bi.cloud_for(p)
    s = g.Solver([p], [cl])
    s.set_maxwellian(stream=stream)
    s.step(3, stream=stream)
    s.sync(stream)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    s.step(steps, stream=stream)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / steps
    s.sync(stream)
    s.close()
    upd = len(cl["kind"]) * p["nv"] ** p["dim"]
    return {"value": upd / (ms * 1e-3), "unit": UNIT, "ms_per_step": ms, "steps": steps}


def body_managed(g, torch, stream, steps: int = 400, every: int = 100) -> dict:
    """The moving-disc ALE workload with a point-management pass every `every` steps;
    time per step includes the passes."""
    p = bi.config("body2d_ale_n201_v32_f32", spare_points=4000)
    cl = bi.cloud_for(p)
    s = g.Solver([p], [cl])
    s.set_maxwellian(stream=stream)
    s.step(3, stream=stream)
    s.sync(stream)
    rmin, mn = 0.3 * p["dx"], 14
    merges = adds = 0
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps // every):
        s.step(every, stream=stream)
        _, r, a = s.manage(rmin, mn, stream=stream)
        merges, adds = merges + r, adds + a
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / steps
    s.sync(stream)
    n = s.n[0]
    s.close()
    return {"ms_per_step": ms, "value": n * p["nv"] ** 2 / (ms * 1e-3), "unit": UNIT, "steps": steps,
            "manage_every": every, "merges": merges, "adds": adds, "points_end": n}


def sharded_rate(torch, stream, p: dict, parts: int, steps: int) -> dict:
    """Workload p as `parts` velocity slabs on this GPU (a context each, their sums added
    by bgk_shard_allreduce): device time per step of all slabs after 3 warm-up steps, and
    the bytes of the two exchanges per step (what an allreduce over `parts` GPUs carries)."""
    from paper_2408_02350_gb300.sharded import ShardedSolver
    cl = bi.cloud_for(p)
    s = ShardedSolver.on_one_device(p, cl, parts)
    s.set_maxwellian(stream=stream)
    s.step(3, stream=stream)
    s.sync(stream)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    s.step(steps, stream=stream)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / steps
    s.sync(stream)
    xbytes = 8 * (s.slabs[0].xm.numel() + s.slabs[0].xw.numel())
    s.close()
    upd = len(cl["kind"]) * p["nv"] ** p["dim"]
    return {"value": upd / (ms * 1e-3), "unit": UNIT, "ms_per_step": ms, "steps": steps, "slabs": parts,
            "exchange_bytes_per_step": xbytes}


def extra_configs(g, torch, stream, workload: str) -> dict:
    """The ALE workload over its Kn sweep and with the second-order WLS stencils, the same
    cavity with a moving disc (plain and with point management), the plain FP64 41^2 x
    16^2 cavity, the 3D 41^3 x 16^3 cavity (FP32), the workload with fixed points (first- and
    second-order steps) and the workload in velocity slabs."""
    out = {}
    p = bi.config(workload)
    if p.get("ale"):
        out["kn_sweep"] = {str(kn): _rate(g, torch, stream, bi.config(workload, kn=kn), 200)
                           for kn in bi.KN_SWEEP_ALE}
    out["body2d_ale_n201_v32_f32"] = _rate(g, torch, stream, bi.config("body2d_ale_n201_v32_f32"), 200)
    if p.get("ale"):
        # the same ALE workload with the second-order (quadratic) WLS stencils
        out[workload + "_quadratic_wls"] = _rate(g, torch, stream, bi.config(workload, wls_order=2), 50)
    out["body2d_ale_n201_v32_f32_managed"] = body_managed(g, torch, stream)
    out["cavity2d_n41_v16_f64"] = _rate(g, torch, stream, bi.config("cavity2d_n41_v16_f64"), 100)
    out["cavity3d_n41_v16_f32"] = _rate(g, torch, stream, bi.config("cavity3d_n41_v16_f32"), 10)
    # BF16 storage (FP32 arithmetic) on the 3D cavity and on the workload, beside FP32
    out["cavity3d_n41_v16_bf16"] = _rate(g, torch, stream, bi.config("cavity3d_n41_v16_f32", storage="bf16"), 10)
    out[workload + "_bf16"] = _rate(g, torch, stream, bi.config(workload, storage="bf16"), 100)
    # the same cavity with fixed points, with the paper's first-order step and with the
    # second-order time discretisation (time_order = 2)
    out[workload + "_fixed"] = _rate(g, torch, stream, bi.config(workload, ale=0), 100)
    out[workload + "_fixed_time_order2"] = _rate(g, torch, stream, bi.config(workload, ale=0, time_order=2), 50)
    # the workload through the velocity-sharded step: one slab (the split's own cost
    # against the fused step) and 4 slabs sharing this GPU
    out[workload + "_sharded"] = {str(k): sharded_rate(torch, stream, p, k, 100) for k in (1, 4)}
    return out


def batched_cost(g, torch, stream, steps: int = 20, cases: int = 64) -> dict:
    """64 independent 2D cavities (sides 41..121, 16..32 velocity nodes, FP32): batched + graph vs per case
    (`cases` < 64 takes the first ones, for profiling runs)."""
    ps = bi.batched_cases(cases)
    cls = [bi.cloud_for(p) for p in ps]
    s = g.Solver(ps, cls)
    s.set_maxwellian(stream=stream)
    upd = sum(len(c["kind"]) * p["nv"] ** 2 for p, c in zip(ps, cls))
    out = {"workload": "batched2d_%d" % len(ps), "cases": len(ps), "updates_per_step": upd}
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    for mode, key in ((0, "per_case"), (2, "batched_graph")):
        g.bgk_set_batching(s.ctx, mode)
        if mode == 2:
            g.bgk_autotune(s.ctx, stream)
        s.step(3, stream=stream)
        torch.cuda.synchronize()
        e0.record(stream)
        s.step(steps, stream=stream)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / steps
        out[key] = {"ms_per_step": ms, "value": upd / (ms * 1e-3), "unit": UNIT}
    st = s.stats()
    out["tuned"] = {"warps": st["batch_warps"], "grid": st["batch_grid"]}
    s.sync(stream)
    s.close()
    return out


def run_reference(args, p: dict, over: dict | None = None) -> None:
    """Reference arm: the FP64 CPU oracle (its OpenMP build, all host cores) on the bench
    workload itself, W warm-up and K timed full steps; when those would take longer than
    about four minutes, each step is instead one full step of a smaller cavity with the
    same velocity grid and parameters, sized to fit, and the line says so."""
    rank, world, _ = _dist_env()
    if rank != 0:
        return
    import oracle
    budget_s = 240.0
    cl = bi.cloud_for(p)
    sim = oracle.Simulation(p, cl, omp=True)
    t0 = time.perf_counter()
    sim.run(1)  # first warm-up step, also the estimate of one step
    t1 = time.perf_counter() - t0
    q, sample_n = p, p["n"]
    if (args.warmup + args.steps) * t1 > budget_s:
        # a smaller cavity: the step cost is about linear in the point count
        scale = budget_s / ((args.warmup + args.steps) * t1)
        sample_n = max(11, int((p["n"] - 1) * scale ** (1.0 / p["dim"])) + 1)
        q = bi.config(args.workload, **dict(over or {}, n=sample_n))
        q["storage"] = p["storage"]
        cl = bi.cloud_for(q)
        sim = oracle.Simulation(q, cl, omp=True)
        sim.run(1)
    sim.run(max(0, args.warmup - 1))
    t0 = time.perf_counter()
    sim.run(args.steps)
    dt = time.perf_counter() - t0
    n = cl["x"].shape[0]
    value = n * q["nv"] ** q["dim"] * args.steps / dt
    thr = oracle.threads(True)
    same = sample_n == p["n"]
    mode = "ALE" if p.get("ale") else "fixed points"
    what = ("one full FP64 time step of the bench workload itself (%d^%d points, %d^%d velocities, %s, Kn %.2g)"
            % (p["n"], p["dim"], p["nv"], p["dim"], mode, p["kn"]) if same else
            "one full FP64 time step of a %d^%d-point cavity with the bench's %d^%d velocity grid, %s, Kn %.2g "
            "(%d points; the full workload would not fit the time budget)"
            % (sample_n, q["dim"], q["nv"], q["dim"], mode, q["kn"], n))
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
            "config": {"workload": args.workload, "points": n, "velocities": q["nv"] ** q["dim"], "kn": q["kn"],
                       "ale": bool(p.get("ale")), "l2": "n/a (CPU)", "same_workload": same},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": thr, "kind": "oracle",
                             "sample": "each step: " + what + ", OpenMP over points on %d threads" % thr,
                             "host": _host_cpu()},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def sharded_plan(p: dict, rank: int, world: int) -> dict:
    """The slab of one rank in the velocity-sharded step and the bytes of its two
    exchanges per step (the allreduce buffers: (dim + 2) n and (2 dim + 6) n_wall doubles)."""
    from paper_2408_02350_gb300.sharded import velocity_slabs
    cl = bi.cloud_for(p)
    n = cl["x"].shape[0]
    dim = p["dim"]
    n_wall = int((cl["kind"] != 0).sum())
    lo, hi = velocity_slabs(p["nv"] ** dim, world)[rank]
    return {"lo": lo, "hi": hi, "points": n, "exchange_bytes": 8 * ((dim + 2) * n + (2 * dim + 6) * n_wall)}


def measure_sharded(args, p: dict, dist, stream) -> dict:
    """One cavity split over the ranks by velocity slabs, the sums exchanged by an allreduce
    of the process group twice a step (strong scaling: the same cavity for every rank
    count).  Device time of K steps (max over ranks) and the end-to-end rate with this
    rank's slab of f uploaded from pinned host memory every step."""
    import torch
    import paper_2408_02350_gb300 as g
    from paper_2408_02350_gb300.sharded import ShardedSolver

    world = dist.get_world_size()
    cl = bi.cloud_for(p)
    n = cl["x"].shape[0]
    dim, NV = p["dim"], p["nv"] ** p["dim"]
    s = ShardedSolver.distributed(p, cl)
    sl = s.slabs[0]
    s.set_maxwellian(stream=stream)
    s.step(args.warmup, stream=stream)
    s.sync(stream)

    def barrier():
        dist.barrier()
        torch.cuda.synchronize()

    launches0 = g.bgk_get_stats(sl.ctx)["launches"]
    clocks = ClockSampler(torch.cuda.current_device())
    clocks.start()
    barrier()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    s.step(args.steps, stream=stream)
    e1.record(stream)
    barrier()
    clk = clocks.stop()
    ms = reduce_max(e0.elapsed_time(e1), dist, "cuda")
    s.sync(stream)
    launches = g.bgk_get_stats(sl.ctx)["launches"] - launches0
    value = n * NV * args.steps / (ms * 1e-3)

    # end to end: this rank's slab of f from pinned host memory, the moments refreshed
    # (partial sums, allreduce), one step, the moments read back
    ncomp = 2 if dim == 2 else 1
    tdt = {"f64": torch.float64, "f32": torch.float32, "bf16": torch.bfloat16}[p["storage"]]
    code = {"f64": 0, "f32": 1, "bf16": 2}[p["storage"]]
    f_host = torch.empty((n, ncomp, sl.hi - sl.lo), dtype=tdt, pin_memory=True)
    g.bgk_get_f(sl.ctx, 0, f_host, code, stream)
    mom = [torch.empty(n, dtype=torch.float64, pin_memory=True),
           torch.empty((n, dim), dtype=torch.float64, pin_memory=True),
           torch.empty(n, dtype=torch.float64, pin_memory=True)]
    barrier()
    t0 = time.perf_counter()
    for _ in range(args.e2e_steps):
        g.bgk_set_f(sl.ctx, 0, f_host, code, stream)
        s.refresh_moments(stream)
        s.step(1, stream=stream)
        g.bgk_moments(sl.ctx, 0, *mom, stream)
    barrier()
    e2e_s = reduce_max(time.perf_counter() - t0, dist, "cuda")
    s.sync(stream)
    xbytes = 8 * (sl.xm.numel() + sl.xw.numel())
    out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
           "scaling": "strong", "vs_baseline": None, "dtype": p["storage"], "data": "synthetic",
           "config": {"workload": args.workload, "points": n, "velocities": NV, "dim": dim,
                      "kn": p["kn"], "ale": bool(p["ale"]), "storage": p["storage"],
                      "stencil_solve": "f64", "moment_combine": "f64",
                      "parallelism": "velocity slabs, one per rank; allreduce of %d bytes twice a step" % xbytes,
                      "l2": "inputs larger than L2 (f %.0f MB per buffer over all ranks)"
                            % (f_host.numel() * f_host.element_size() * world / 1e6)},
           "clocks": clk, "gpu_launches": launches,
           "e2e": {"value": n * NV * args.e2e_steps / e2e_s, "unit": UNIT,
                   "h2d_bytes_per_step": f_host.numel() * f_host.element_size(),
                   "d2h_bytes_per_step": n * (dim + 2) * 8, "steps": args.e2e_steps}}
    s.close()
    return out


def run_sharded(args, p: dict, rank: int, world: int, local_rank: int) -> None:
    """bench.py --sharded: the velocity-sharded strong-scaling line as the headline."""
    import torch
    import torch.distributed as dist

    torch.cuda.set_device(local_rank)
    os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
    os.environ.setdefault("MASTER_PORT", "29517")
    dist.init_process_group("nccl", rank=rank, world_size=world)
    line = measure_sharded(args, p, dist, torch.cuda.current_stream())
    if rank == 0:
        print(json.dumps(line), flush=True)
    dist.destroy_process_group()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    # (the ALE workload runs about 2300 steps without point management before the lid
    # corners empty; a run takes about 2 K + 80 steps in all)
    ap.add_argument("--steps", type=int, default=500)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default=WORKLOAD)
    ap.add_argument("--config-file", default=None,
                    help="a workload file (workloads/<name>.json, or an edited copy): its workload and "
                         "parameters replace --workload")
    ap.add_argument("--storage", default=None, choices=[None, "f64", "f32", "bf16"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--e2e-steps", type=int, default=20)
    ap.add_argument("--no-fp64", action="store_true", help="skip the plain FP64 GPU comparison")
    ap.add_argument("--n", type=int, default=None, help="override points per axis (profiling runs)")
    ap.add_argument("--no-adjoint", action="store_true", help="skip the adjoint-step cost measurement")
    ap.add_argument("--no-batched", action="store_true", help="skip the 64-cavity batched measurement")
    ap.add_argument("--no-manage", action="store_true", help="skip the point-management measurement")
    ap.add_argument("--no-extra", action="store_true", help="skip the Kn sweep and the FP64 41^2 cavity")
    ap.add_argument("--sharded", action="store_true",
                    help="one cavity split over the ranks by velocity slabs (strong scaling)")
    ap.add_argument("--batch-cases", type=int, default=64,
                    help="cavities of the batched measurement (fewer than 64 for profiling runs)")
    ap.add_argument("--manage-steps", type=int, default=200,
                    help="ALE steps before the point-management measurement")
    ap.add_argument("--no-sharded", action="store_true",
                    help="under torchrun, skip the velocity-sharded line beside the replica line")
    ap.add_argument("--time-order", type=int, default=None,
                    help="2: the workload with fixed points and the second-order time step (profiling runs)")
    args = ap.parse_args()
    rank, world, local_rank = _dist_env()
    over = {}
    if args.config_file:
        args.workload, over = bi.workload_from_file(args.config_file)
    if args.n:
        over["n"] = args.n
    if args.time_order:
        over.update(ale=0, time_order=args.time_order)
    if args.sharded and args.impl == "ours":
        q = bi.config(args.workload, **over)
        if args.storage:
            q["storage"] = args.storage
        run_sharded(args, q, rank, world, local_rank)
        return
    p = rank_config(bi.config(args.workload, **over), rank, world)
    if args.storage:
        p["storage"] = args.storage
    if args.impl == "reference":
        run_reference(args, p, over)
        return

    import torch
    import paper_2408_02350_gb300 as g

    torch.cuda.set_device(local_rank)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    stream = torch.cuda.current_stream()
    cl = bi.cloud_for(p)
    n = cl["x"].shape[0]
    dim, nv = p["dim"], p["nv"]
    NV = nv ** dim
    ncomp = 2 if dim == 2 else 1
    upd_per_step = n * NV

    s = g.Solver([p], [cl])
    s.set_maxwellian(stream=stream)
    s.step(args.warmup, stream=stream)
    s.sync(stream)

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    # ---- device-resident timed region (no per-kernel events: an event pair around each
    # transport launch costs the step 12-15 us, so the transport's own time is taken in an
    # identical run of K steps right after) ----
    launches0 = s.stats()["launches"]
    clocks = ClockSampler(torch.cuda.current_device())
    clocks.start()
    barrier()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    s.step(args.steps, stream=stream)
    e1.record(stream)
    barrier()
    clk = clocks.stop()
    ms = e0.elapsed_time(e1)
    s.sync(stream)
    launches = s.stats()["launches"] - launches0
    # the same K steps again with an event pair around every transport launch
    g.bgk_set_timing(s.ctx, 1 << g.K_TRANSPORT)
    s.step(args.steps, stream=stream)
    s.sync(stream)
    kt_ms, kt_n = g.bgk_get_timing(s.ctx, g.K_TRANSPORT)
    g.bgk_set_timing(s.ctx, False)
    ms = reduce_max(ms, dist, "cuda")
    # per-kernel breakdown from a short separate run with every group timed
    g.bgk_set_timing(s.ctx, True)
    s.step(min(args.steps, 50), stream=stream)
    s.sync(stream)
    per_kernel = {name: g.bgk_get_timing(s.ctx, k) for name, k in
                  (("transport", g.K_TRANSPORT), ("walls", g.K_WALLS), ("neighbours", g.K_NBR),
                   ("stencils", g.K_STENCIL), ("move", g.K_MOVE))}
    if per_kernel["move"][1] == 0 and p.get("ale"):
        # the cooperative side-chain kernel runs motion, lists and interior stencils in one
        # launch (timed under the neighbour group); "stencils" is then the wall weights only
        per_kernel["motion_lists_stencils"] = per_kernel.pop("neighbours")
        per_kernel.pop("move")
    g.bgk_set_timing(s.ctx, False)
    value = upd_per_step * args.steps * world / (ms * 1e-3)

    # ---- end to end through the C ABI with host buffers ----
    elem = {"f64": 8, "f32": 4, "bf16": 2}[p["storage"]]
    tdt = {"f64": torch.float64, "f32": torch.float32, "bf16": torch.bfloat16}[p["storage"]]
    f_host = torch.empty((n, ncomp, NV), dtype=tdt, pin_memory=True)
    g.bgk_get_f(s.ctx, 0, f_host, {"f64": 0, "f32": 1, "bf16": 2}[p["storage"]], stream)
    mom_host = [torch.empty(n, dtype=torch.float64, pin_memory=True),
                torch.empty((n, dim), dtype=torch.float64, pin_memory=True),
                torch.empty(n, dtype=torch.float64, pin_memory=True)]
    h2d = f_host.numel() * elem
    d2h = n * (dim + 2) * 8
    # each step's input is uploaded with bgk_stage_f, which overlaps the copy with the
    # step before; the step takes it, and its moments come back to the host
    code = {"f64": 0, "f32": 1, "bf16": 2}[p["storage"]]
    barrier()
    t0 = time.perf_counter()
    g.bgk_stage_f(s.ctx, 0, f_host, code)
    for k in range(args.e2e_steps):
        g.bgk_step(s.ctx, 1, stream)
        if k + 1 < args.e2e_steps:
            g.bgk_stage_f(s.ctx, 0, f_host, code)
        g.bgk_moments(s.ctx, 0, *mom_host, stream)
    barrier()
    e2e_s = time.perf_counter() - t0
    e2e_s = reduce_max(e2e_s, dist, "cuda")
    s.sync(stream)
    e2e_value = upd_per_step * args.e2e_steps * world / e2e_s
    # host-to-device rate of the upload alone: an upload followed by the step that takes it
    # (nothing else runs meanwhile), less the device time of a step
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(3):
        g.bgk_stage_f(s.ctx, 0, f_host, code)
        g.bgk_step(s.ctx, 1, stream)
    e1.record(stream)
    torch.cuda.synchronize()
    up_ms = max(e0.elapsed_time(e1) / 3 - ms / args.steps, 1e-6)
    h2d_gbs = h2d / (up_ms * 1e-3) / 1e9
    s.sync(stream)

    # ---- plain FP64 GPU step on the same workload (the comparison the metric names) ----
    fp64 = None
    if p["storage"] != "f64" and not args.no_fp64:
        q = dict(p, storage="f64")
        s64 = g.Solver([q], [cl])
        s64.set_maxwellian(stream=stream)
        s64.step(2, stream=stream)
        s64.sync(stream)
        k64 = 5
        e0.record(stream)
        s64.step(k64, stream=stream)
        e1.record(stream)
        torch.cuda.synchronize()
        ms64 = e0.elapsed_time(e1)
        s64.sync(stream)
        fp64 = {"value": upd_per_step * k64 / (ms64 * 1e-3), "unit": UNIT, "steps": k64,
                "ms_per_step": ms64 / k64}
        s64.close()

    # ---- discrete adjoint cost on the adjoint workload (101^2 x 24^2, FP32, fixed points) ----
    adj = None
    manage = None
    if not args.no_manage and world == 1 and p.get("ale"):
        manage = manage_cost(g, torch, stream, p, args.workload, steps=args.manage_steps)
    if not args.no_adjoint and world == 1:
        adj = adjoint_cost(g, torch, stream)

    batched = None
    if not args.no_batched and world == 1:
        batched = batched_cost(g, torch, stream, cases=args.batch_cases)
    extra = None
    if not args.no_extra and world == 1:
        extra = extra_configs(g, torch, stream, args.workload)

    # ---- roofline of the dominant kernel (transport + moments + relaxation) ----
    peaks = _peaks()
    rowptr, _ = s.get_neighbours()
    nnz_interior = int(sum(rowptr[i + 1] - rowptr[i] for i in np.where(cl["kind"] == 0)[0]))
    kt_avg_s = kt_ms / max(kt_n, 1) * 1e-3
    instr_per_launch = nnz_interior * NV * OPS_PER_PAIR[dim]
    sm_max = peaks.get("sm_max_mhz", 2070.0)
    alu_peak = N_SM * FP32_LANES_PER_SM * sm_max * 1e6 / 1e12  # Tinstr/s
    achieved = instr_per_launch / kt_avg_s / 1e12
    bytes_per_update = 2 * ncomp * elem  # read f once, write f^{n+1} once
    hbm_achieved = bytes_per_update * upd_per_step / kt_avg_s / 1e9
    # (the captured traffic is that of the named workload as it stands: none for variants)
    traffic = _traffic_record("k_transport", args.workload) if not over and not args.storage else None
    roofline = {"bound": "alu", "achieved": achieved, "peak": alu_peak, "unit": "Tinstr/s",
                "frac": achieved / alu_peak, "traffic": traffic,
                "peak_source": "152 SMs x 128 FP32 lanes x %.0f MHz (max SM clock, %s)" % (sm_max, peaks["source"]),
                "kernel": "k_transport", "avg_launch_ms": kt_avg_s * 1e3,
                "avg_launch_from": "CUDA event pairs around every transport launch of a run of the same K "
                                   "steps right after the timed region (on the launching stream)",
                "instr_per_launch": instr_per_launch,
                "hbm": {"achieved": hbm_achieved, "peak": peaks.get("hbm_gbs"), "unit": "GB/s",
                        "frac": hbm_achieved / peaks.get("hbm_gbs", 6800.0),
                        "bytes_per_update": bytes_per_update}}
    # the FP32 FMA rate measured on this device by the project's microbenchmark
    try:
        pk = g.bgk_peak_fp32(stream)
        roofline["peak_measured"] = {"fma_tflops_scalar": pk["fma_per_s"] / 1e12,
                                     "fma_tflops_packed_pairs": pk["fma2_per_s"] / 1e12, "n_sm": pk["n_sm"],
                                     "frac_of_scalar_fma": achieved / (pk["fma_per_s"] / 1e12),
                                     "fp64_fma_tflops": g.bgk_peak_fp64(stream) / 1e12}
    except g.BGKError as e:
        roofline["peak_measured"] = {"error": str(e)}
    kernels = {k: {"ms_total": v[0], "launches": v[1]} for k, v in per_kernel.items()}

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": p["storage"], "data": "synthetic",
                "config": {"workload": args.workload, "points": n, "velocities": NV, "dim": dim,
                           "kn": p["kn"], "ale": bool(p["ale"]), "storage": p["storage"],
                           "stencil_solve": "f64", "moment_combine": "f64",
                           "l2": "inputs larger than L2 (f %.0f MB per buffer, two buffers)"
                                 % (n * ncomp * NV * elem / 1e6)},
                "clocks": clk, "gpu_launches": launches,
                "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                        "steps": args.e2e_steps, "h2d_gbs": h2d_gbs,
                        "how": "bgk_stage_f of every step's f from pinned host memory (four copies on "
                               "four streams; the upload overlaps the step before), bgk_step, bgk_moments "
                               "to pinned host memory; h2d_gbs: the upload alone"},
                "roofline": roofline, "kernels": kernels, "fp64_gpu": fp64, "adjoint": adj, "batched": batched,
                "manage": manage, "extra": extra}
        if world == 1 and not args.no_cpu_baseline:
            line["cpu_baseline"] = cpu_baseline(p, 1, g)
    if dist is not None and not args.no_sharded:
        # the multi-GPU design for one cavity: the same workload split over the ranks by
        # velocity slabs (strong scaling), beside the weak-scaled replicas above
        sh = measure_sharded(args, dict(bi.config(args.workload, **over), **({"storage": args.storage}
                                                                            if args.storage else {})), dist, stream)
        if rank == 0:
            line["sharded"] = sh
    if rank == 0:
        print(json.dumps(line), flush=True)
    s.close()
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
