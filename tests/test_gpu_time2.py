"""GPU parity of the second-order time discretisation (time_order = 2: Strang splitting
with the exact relaxation solve around a two-stage transport) against the oracle: small
cavities in 2D and 3D (FP64 to 1e-10, FP32 to 1e-4), the uniform-relaxation closed form
on the GPU, and one step of the 201^2 x 32^2 cavity (fixed points) at full size.
"""
import math

import numpy as np
import pytest

import bgk_inputs as bi
import oracle

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def g():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2408_02350_gb300 import _build
    _build.build()
    import paper_2408_02350_gb300 as g
    return g


def _rel(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


@pytest.mark.parametrize("dim,n,nv,storage,steps,tol", [
    (2, 13, 8, "f64", 10, 1e-10), (2, 15, 6, "f64", 6, 1e-10), (3, 6, 4, "f64", 4, 1e-10),
    (2, 13, 8, "f32", 10, 1e-4), (2, 15, 6, "f32", 6, 1e-4), (3, 6, 4, "f32", 4, 1e-4), (3, 5, 6, "f32", 3, 1e-4)])
def test_second_order_steps_match_oracle(g, dim, n, nv, storage, steps, tol):
    name = "cavity2d_n41_v16_f64" if dim == 2 else "cavity3d_n41_v16_f32"
    p = bi.config(name, n=n, nv=nv, vmax=3.0, storage=storage, time_order=2)
    cl = bi.cloud_for(p)
    sim = oracle.Simulation(p, cl)
    sim.run(steps)
    s = g.Solver([p], [cl])
    s.set_maxwellian()
    s.step(steps)
    s.sync()
    rho, u, T = s.moments()
    f = s.get_f(0, np.float64)
    s.close()
    assert _rel(rho, sim.rho) < tol and _rel(T, sim.T) < tol and _rel(u, sim.U) < max(tol, 1e-12)
    assert np.abs(f - sim.f).max() < 10 * tol * np.abs(sim.f).max()


def test_gpu_uniform_relaxation_is_exponential(g):
    # a uniform non-equilibrium state in a periodic box: f_N = M + (f0 - M) exp(-N dt / tau)
    n, nv, vmax, kn, dt, N = 8, 32, 9.0, 0.3, 0.05, 12
    p = {"dim": 2, "nv": nv, "vmax": vmax, "kn": kn, "tau_mode": 1, "dt": dt, "h": 2.5 / n, "alpha": 6.25,
         "max_nbrs": 48, "periodic": 1, "ale": 0, "time_order": 2, "storage": "f64"}
    cl = bi.periodic_box(2, n)
    f0row = 0.5 * (oracle.maxwellian(p, 1.0, (0.3, -0.1), 1.0) + oracle.maxwellian(p, 0.6, (-0.4, 0.2), 1.3))
    f0 = np.ascontiguousarray(np.broadcast_to(f0row, (n * n,) + f0row.shape))
    rho, U, T = oracle.moments_point(p, f0row)
    M = oracle.maxwellian(p, rho, U, T)
    s = g.Solver([p], [cl])
    s.set_f(f0)
    s.step(N)
    s.sync()
    f = s.get_f(0, np.float64)
    s.close()
    tau = math.sqrt(2.0 / math.pi) * kn
    want = M + (f0row - M) * math.exp(-N * dt / tau)
    assert np.abs(f - want[None]).max() < 1e-11 * np.abs(f0row).max()


def test_second_order_step_at_workload_size(g):
    # the 201^2 x 32^2 cavity with fixed points, one second-order step in FP32 against the
    # FP64 oracle's step at every point
    p = bi.config("cavity2d_ale_n201_v32_f32", ale=0, time_order=2)
    cl = bi.cloud_for(p)
    sim = oracle.Simulation(p, cl)
    sim.run(1)
    s = g.Solver([p], [cl])
    s.set_maxwellian()
    s.step(1)
    s.sync()
    rho, u, T = s.moments()
    s.close()
    assert _rel(rho, sim.rho) < 1e-5 and _rel(T, sim.T) < 1e-5 and np.abs(u - sim.U).max() < 1e-5


def test_second_order_refusals(g):
    p = bi.config("cavity2d_n41_v16_f64", n=9, nv=4, vmax=3.0, time_order=2)
    cl = bi.cloud_for(p)
    s = g.Solver([p], [cl])
    s.set_maxwellian()
    import torch
    lam = torch.zeros((len(cl["kind"]), 2, 16), dtype=torch.float64, device="cuda")
    th = torch.zeros(4, dtype=torch.float64, device="cuda")
    with pytest.raises(g.BGKError) as e:
        g.bgk_adjoint_step(s.ctx, 0, lam, lam.clone(), th)
    assert e.value.code == g.BGK_E_STATE
    xm = torch.zeros(len(cl["kind"]) * 4, dtype=torch.float64, device="cuda")
    with pytest.raises(g.BGKError) as e:
        g.bgk_shard_transport(s.ctx, 0, xm)
    assert e.value.code == g.BGK_E_STATE
    s.close()


def test_second_order_bf16_tracks_fp32(g):
    # BF16 storage through the same second-order step, which rounds f to 8 mantissa bits
    # three times a step (opening relaxation, first stage, result): a regression bound
    # with margin over the measured 8.6e-3 in rho after 10 steps, as for the first-order
    # BF16 path, not the FP32 bar
    p = bi.config("cavity2d_n41_v16_f64", n=21, nv=8, vmax=3.0, time_order=2)
    cl = bi.cloud_for(p)
    out = {}
    for st in ("f32", "bf16"):
        s = g.Solver([dict(p, storage=st)], [cl])
        s.set_maxwellian()
        s.step(10)
        s.sync()
        out[st] = s.moments()
        s.close()
    (r1, u1, t1), (r2, u2, t2) = out["f32"], out["bf16"]
    assert _rel(r2, r1) < 3e-2 and _rel(t2, t1) < 3e-2 and np.abs(u2 - u1).max() < 5e-2
