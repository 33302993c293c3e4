"""GPU parity: the CUDA library (through the C ABI) against the FP64 CPU oracle on the same seeded inputs.

Bars: neighbour lists bit-exact; FP64 path within 1e-10 relative on rho, u, T
(1e-12 on one step and on stencils); FP32 path within 1e-4 relative L-inf on
rho and T and normwise on u (||du||_inf / ||u||_inf) after 100 steps.  The
wall classification v.n > 0 is taken in FP64 without fused multiply-add on
both sides, so it is identical.
"""
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


def _gpu_run(g, p, cl, nsteps, storage=None, rho0=1.0, u0=(0.0, 0.0, 0.0), T0=1.0, f0=None):
    q = dict(p)
    if storage:
        q["storage"] = storage
    s = g.Solver([q], [cl])
    if f0 is None:
        s.set_maxwellian(rho0, u0, T0)
    else:
        s.set_f(np.ascontiguousarray(f0))
    s.step(nsteps)
    s.sync()
    return s


def _cmp_moments(sim, s, tol, what=""):
    rho, u, T = s.moments()
    er = np.abs(rho - sim.rho).max() / np.abs(sim.rho).max()
    eT = np.abs(T - sim.T).max() / np.abs(sim.T).max()
    eu = np.abs(u - sim.U).max() / max(np.abs(sim.U).max(), 1e-300)
    assert er < tol and eT < tol and eu < tol, (what, er, eu, eT)
    return er, eu, eT


def _cmp_lists(g, s, x, h, periodic, cap):
    rowptr, col = s.get_neighbours()
    cnt, ocol = oracle.neighbours(x, h, periodic, cap)
    orp, oc = oracle.to_csr(cnt, ocol)
    assert np.array_equal(rowptr, orp)
    assert np.array_equal(col, oc)
    return rowptr, col, cnt, ocol


@pytest.mark.parametrize("dim,n", [(2, 41), (2, 201), (3, 17), (3, 41)])
def test_neighbour_lists_bit_exact(g, dim, n):
    name = "cavity2d_n41_v16_f64" if dim == 2 else "cavity3d_n41_v16_f32"
    p = bi.config(name, n=n, nv=4)
    cl = bi.cloud_for(p)
    s = g.Solver([p], [cl])
    s.neighbours()
    s.sync()
    _cmp_lists(g, s, cl["x"], p["h"], False, p["max_nbrs"])


def test_neighbour_lists_periodic_random_cloud(g):
    x = bi.uniform01(99, 3000 * 2).reshape(-1, 2)
    cl = {"x": x, "kind": np.zeros(len(x), np.int32), "normal": np.zeros_like(x)}
    p = {"dim": 2, "nv": 4, "vmax": 1.0, "kn": 1.0, "tau_mode": 2, "dt": 1e-3, "h": 0.04, "alpha": 6.25,
         "max_nbrs": 64, "periodic": 1, "storage": "f64"}
    s = g.Solver([p], [cl])
    s.neighbours()
    s.sync()
    _cmp_lists(g, s, x, p["h"], True, 64)


# FP32 path: separations (from the FP32 hi/lo split of x) and Gaussian weights are FP32,
# the normal matrix is accumulated and solved in FP64, the coefficients are stored in FP32.
# Interior stencils: measured 4e-7 to 5.5e-7 of the largest entry on these clouds, bar
# 2e-6.  Wall reconstruction weights (FP64 solve of one-sided fits whose condition numbers
# are ~30 in 2D to ~100 in 3D, from FP32 separations): measured up to 1.15e-5, bar 3e-5.
@pytest.mark.parametrize("dim,n,storage,tol,tol_r", [(2, 21, "f64", 1e-12, 1e-12), (3, 9, "f64", 1e-12, 1e-12),
                                                     (2, 21, "f32", 2e-6, 3e-5), (3, 9, "f32", 2e-6, 3e-5)])
def test_stencils_match(g, dim, n, storage, tol, tol_r):
    name = "cavity2d_n41_v16_f64" if dim == 2 else "cavity3d_n41_v16_f32"
    p = bi.config(name, n=n, nv=4, storage=storage)
    cl = bi.cloud_for(p)
    s = g.Solver([p], [cl])
    s.neighbours()
    s.sync()
    P, R = s.get_stencils()
    cnt, col = oracle.neighbours(cl["x"], p["h"], False, p["max_nbrs"])
    st = oracle.stencils(p, cl["x"], cl["kind"], cnt, col)
    k = 0
    for i in range(len(cnt)):
        m = cnt[i]
        if cl["kind"][i] == 0:
            Po = st["abar"][i, :m, :, None] * st["frame"][i, :m]
            scale = np.abs(Po).max()
            assert np.abs(P[k:k + m] - Po).max() <= tol * scale, i
        else:
            assert np.abs(R[k:k + m] - st["recon"][i, :m]).max() <= tol_r * max(1.0, np.abs(st["recon"][i]).max()), i
        k += m


@pytest.mark.parametrize("dim,n,nv", [(2, 21, 8), (2, 13, 5), (3, 9, 6), (3, 7, 5)])
def test_one_fp64_step(g, dim, n, nv):
    name = "cavity2d_n41_v16_f64" if dim == 2 else "cavity3d_n41_v16_f32"
    p = bi.config(name, n=n, nv=nv, storage="f64")
    cl = bi.cloud_for(p)
    sim = oracle.Simulation(p, cl)
    sim.run(1)
    s = _gpu_run(g, p, cl, 1)
    f = s.get_f()
    assert np.abs(f - sim.f).max() < 1e-12 * np.abs(sim.f).max()
    _cmp_moments(sim, s, 1e-12)


def test_cavity2d_fp64_100_steps(g):
    # 41^2 points, 16^2 velocities, Kn 0.1, lid 0.1, 100 steps, FP64
    p = bi.config("cavity2d_n41_v16_f64")
    cl = bi.cloud_for(p)
    sim = oracle.Simulation(p, cl)
    sim.run(100)
    s = _gpu_run(g, p, cl, 100)
    _cmp_moments(sim, s, 1e-10, "fp64 100 steps")


def test_cavity2d_fp32_100_steps(g):
    p = bi.config("cavity2d_n41_v16_f64")
    cl = bi.cloud_for(p)
    sim = oracle.Simulation(p, cl)
    sim.run(100)
    s = _gpu_run(g, p, cl, 100, storage="f32")
    _cmp_moments(sim, s, 1e-4, "fp32 100 steps")


# BF16 storage with FP32 arithmetic does not meet the 1e-4 bar: every stored value is
# rounded to an 8-bit mantissa each step, and round-to-nearest of a smooth Maxwellian is
# not random across velocities, so the moment errors add up step after step; the low-Mach
# velocity, a small difference of O(1) terms, carries the largest relative error.  The
# bounds are twice the measured errors (41^2 x 16^2 after 100 steps: rho 4.76e-2, u 0.438,
# T 4.89e-3; ALE 31^2 x 12^2 after 30 steps: 2.23e-2, 0.255, 1.63e-3; 3D 9^3 x 8^3 after
# 10 steps: 5.50e-3, 5.50e-2, 2.32e-3), a regression guard on the measured floor.
@pytest.mark.parametrize("name,over,steps,bounds", [
    ("cavity2d_n41_v16_f64", {}, 100, (0.095, 0.88, 9.8e-3)),
    ("cavity2d_ale_n201_v32_f32", {"n": 31, "nv": 12}, 30, (4.5e-2, 0.51, 3.3e-3)),
    ("cavity3d_n41_v16_f32", {"n": 9, "nv": 8}, 10, (1.1e-2, 0.11, 4.7e-3))])
def test_bf16_error_is_at_its_measured_floor(g, name, over, steps, bounds):
    p = bi.config(name, **over)
    cl = bi.cloud_for(p)
    sim = oracle.Simulation(p, cl)
    sim.run(steps)
    s = _gpu_run(g, p, cl, steps, storage="bf16")
    rho, u, T = s.moments()
    er = np.abs(rho - sim.rho).max() / np.abs(sim.rho).max()
    eT = np.abs(T - sim.T).max() / np.abs(sim.T).max()
    eu = np.abs(u - sim.U).max() / np.abs(sim.U).max()
    assert er < bounds[0] and eu < bounds[1] and eT < bounds[2], (er, eu, eT)


@pytest.mark.parametrize("storage,tol", [("f64", 1e-10), ("f32", 1e-4)])
@pytest.mark.parametrize("kn", [0.01, 0.1, 1.0])
def test_ale_cavity(g, storage, tol, kn):
    # ALE: points move with U, neighbour lists and stencils rebuilt every step
    p = bi.config("cavity2d_ale_n201_v32_f32", n=31, nv=12, kn=kn)
    cl = bi.cloud_for(p)
    sim = oracle.Simulation(p, cl)
    sim.run(30)
    s = _gpu_run(g, p, cl, 30, storage=storage)
    x = s.positions()
    # positions integrate U: |dx| <= steps * dt * (tolerance of u) * ||u||_inf
    xtol = 1e-14 if storage == "f64" else 30 * p["dt"] * tol * np.abs(sim.U).max()
    assert np.abs(x - sim.x).max() < xtol
    _cmp_moments(sim, s, tol, "ale")
    assert s.stats()["clamps"] == sim.clamps


@pytest.mark.parametrize("storage,tol", [("f64", 1e-10), ("f32", 1e-4)])
def test_cavity3d_steps(g, storage, tol):
    p = bi.config("cavity3d_n41_v16_f32", n=9, nv=8)
    cl = bi.cloud_for(p)
    sim = oracle.Simulation(p, cl)
    sim.run(10)
    s = _gpu_run(g, p, cl, 10, storage=storage)
    _cmp_moments(sim, s, tol, "3d")


def test_periodic_free_transport(g):
    n, nv, vmax = 24, 4, 1.0
    cl = bi.periodic_box(2, n)
    p = {"dim": 2, "nv": nv, "vmax": vmax, "kn": 1.0, "tau_mode": 2, "dt": 0.5 / n / (vmax * 2 ** 0.5),
         "h": 2.5 / n, "alpha": 6.25, "max_nbrs": 48, "periodic": 1, "ale": 0, "storage": "f64"}
    M = oracle.maxwellian(p, 1.0, (0.0, 0.0), 1.0)
    f0 = (1 + 0.1 * np.sin(2 * np.pi * cl["x"][:, 0]))[:, None, None] * M[None]
    sim = oracle.Simulation(p, cl, f0=f0)
    sim.run(20)
    s = _gpu_run(g, p, cl, 20, f0=f0)
    assert np.abs(s.get_f() - sim.f).max() < 1e-12 * np.abs(f0).max()


def test_state_round_trip_reproduces_steps(g):
    p = bi.config("cavity2d_n41_v16_f64", n=21, nv=8, storage="f32")
    cl = bi.cloud_for(p)
    s = _gpu_run(g, p, cl, 3)
    blob = g.bgk_get_state(s.ctx)
    s.step(4)
    s.sync()
    f1 = s.get_f()
    g.bgk_set_state(s.ctx, blob)
    s.step(4)
    s.sync()
    assert np.array_equal(s.get_f(), f1)


def test_neighbour_overflow_is_reported(g):
    p = bi.config("cavity2d_n41_v16_f64", n=21, nv=4, max_nbrs=6)
    cl = bi.cloud_for(p)
    s = g.Solver([p], [cl])
    s.set_maxwellian()
    s.step(1)
    with pytest.raises(g.BGKError) as e:
        s.sync()
    assert e.value.code == g.BGK_E_NBR_OVERFLOW
    s.sync()  # cleared


def test_wall_point_without_interior_neighbours_is_singular(g):
    x = np.array([[0.0, 0.0], [1.0, 0.0], [0.0, 1.0], [1.0, 1.0]])
    cl = {"x": x, "kind": np.array([5, 5, 5, 5], np.int32), "normal": np.array([[1, 1], [-1, 1], [1, -1], [-1, -1]]) / 2 ** 0.5}
    p = bi.config("cavity2d_n41_v16_f64", n=5, nv=4)
    s = g.Solver([p], [cl])
    s.set_maxwellian()
    s.step(1)
    with pytest.raises(g.BGKError) as e:
        s.sync()
    assert e.value.code == g.BGK_E_SINGULAR


def _noisy_state(p, n, seed):
    """f = M(v; 1, 0, 1) (1 + 0.1 u), u uniform in [-1, 1] per (point, component, velocity),
    rounded to FP32 so that the FP32 library and the FP64 oracle start from the same values."""
    d = p["dim"]
    M = oracle.maxwellian(p, 1.0, (0.0, 0.0, 0.0), 1.0)
    u = bi.uniform01(seed, n * M.size).reshape((n,) + M.shape)
    return (M[None] * (1.0 + 0.1 * (2.0 * u - 1.0))).astype(np.float32)


def _sample_points(cl, p, cnt, col, nsamp, seed):
    """nsamp random interior points plus interior points next to the lid and next to
    corner or edge points (where the wall rows enter the transport)."""
    kind = cl["kind"]
    interior = np.where(kind == 0)[0]
    rng = np.random.default_rng(seed)
    pick = set(rng.choice(interior, size=nsamp, replace=False).tolist())
    lid = [i for i in interior if (kind[col[i, :cnt[i]]] == p["lid_wall"]).any()]
    corner = [i for i in interior if (kind[col[i, :cnt[i]]] == 2 * p["dim"] + 1).any()]
    pick.update(rng.choice(lid, size=min(32, len(lid)), replace=False).tolist())
    pick.update(rng.choice(corner, size=min(32, len(corner)), replace=False).tolist())
    return np.array(sorted(pick), dtype=np.int64)


def _sampled_step_check(s, p, x, f_host, U, nsamp, tol_f, seed=7):
    """The step the solver s has just taken, from positions x, state f_host (FP64 copy of
    the FP32 state) and transport velocities U: the lists it used bit-exact against the
    oracle's lists of x, then f^{n+1} and the moments at sampled interior points against
    the oracle's transport and relaxation of the same state, element by element."""
    cl = {"x": x, "kind": s.clouds[0]["kind"]}
    rowptr, col = s.get_neighbours()
    cnt, ocol = oracle.neighbours(x, p["h"], False, p["max_nbrs"])
    orp, oc = oracle.to_csr(cnt, ocol)
    assert np.array_equal(rowptr, orp) and np.array_equal(col, oc)
    st = oracle.stencils(p, x, cl["kind"], cnt, ocol)
    idx = _sample_points(cl, p, cnt, ocol, nsamp, seed)
    out, rho, u, T = oracle.transport_relax_points(p, idx, cnt, ocol, st, U, f_host)
    fg = s.get_f()[idx]
    # the transport is not trivial at these points: f~ differs from f by far more than the bar
    assert np.abs(out - f_host[idx]).max() > 100 * tol_f * np.abs(out).max()
    assert np.abs(fg - out).max() < tol_f * np.abs(out).max()
    rg, ug, Tg = s.moments()
    assert np.abs(rg[idx] - rho).max() < 1e-5 and np.abs(Tg[idx] - T).max() < 1e-5
    assert np.abs(ug[idx] - u).max() < 1e-5 * max(1.0, np.abs(u).max())
    return idx


def test_full_size_ale_cavity_sampled(g):
    # 201^2 points, 32^2 velocities, ALE, FP32: the benchmark's workload and launch
    # configuration, from a seeded non-uniform state.  Step 1 uses lists built from scratch;
    # step 4 filters the Verlet-skin candidate lists of the first build (skin 0.2: after
    # three steps every point has moved about dt |U| 3 = 1e-4, far less than h skin / 2).
    p = bi.config("cavity2d_ale_n201_v32_f32")
    cl = bi.cloud_for(p)
    n, d = len(cl["kind"]), p["dim"]
    f0 = _noisy_state(p, n, 2408102)
    s = g.Solver([p], [cl])
    s.set_f(f0)
    f0d = f0.astype(np.float64)
    _, U0, _ = oracle.moments(p, f0d)
    s.step(1)
    s.sync()
    idx = _sampled_step_check(s, p, cl["x"], f0d, U0, 256, 1e-5)
    assert len(idx) >= 256
    # positions after the move: x + dt U^{n+1} with the library's own U (FP64 arithmetic)
    x = s.positions()
    _, ug, _ = s.moments()
    inner = cl["kind"] == 0
    expect = np.clip(cl["x"][inner] + p["dt"] * ug[inner], p["guard"], 1 - p["guard"])
    assert np.abs(x[inner] - expect).max() < 1e-15
    assert np.array_equal(x[~inner], cl["x"][~inner])
    s.step(2)
    s.sync()
    x3, f3 = s.positions(), s.get_f()
    _, U3, _ = s.moments()
    s.step(1)
    s.sync()
    _sampled_step_check(s, p, x3, f3, U3, 256, 1e-5, seed=8)
    s.close()


def test_full_size_cavity3d_sampled(g):
    # 41^3 points, 16^3 velocities, FP32, fixed points (the mirror-paired transport), from a
    # seeded non-uniform state
    p = bi.config("cavity3d_n41_v16_f32")
    cl = bi.cloud_for(p)
    n, d = len(cl["kind"]), p["dim"]
    f0 = _noisy_state(p, n, 2408103)
    s = g.Solver([p], [cl])
    s.set_f(f0)
    s.step(1)
    s.sync()
    _sampled_step_check(s, p, cl["x"], f0.astype(np.float64), np.zeros((n, d)), 256, 1e-5)
    s.close()
