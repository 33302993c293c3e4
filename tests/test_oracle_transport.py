"""Pins of the oracle's positive upwind transport, walls and point motion.

Transport: constants are preserved bitwise; on a centrally symmetric
neighbourhood the upwind flux equals c.grad(p) for linear p; the operator is
positive (off-diagonal entries >= 0, rows sum to one); free transport in a
periodic box converges at first order to f0(x - v t).  A 1D-like check fixes
the upwind direction.  Walls: zero net normal mass flux at every wall point;
diffuse reflection leaves the wall Maxwellian's shape on leaving velocities; a
global Maxwellian with walls at rest is stationary.  Point motion: U = 0 leaves
points in place bitwise; a uniform drift moves every point by dt U.
"""
import math

import numpy as np
import pytest

import bgk_inputs as bi
import oracle


def _case(dim, n, nv, vmax, seed=21, jitter=0.1, **kw):
    name = "cavity2d_n41_v16_f64" if dim == 2 else "cavity3d_n41_v16_f32"
    p = bi.config(name, n=n, nv=nv, vmax=vmax)
    p.update(kw)
    c = bi.cavity(dim, n, seed, jitter)
    cnt, col = oracle.neighbours(c["x"], p["h"], False, p["max_nbrs"])
    st = oracle.stencils(p, c["x"], c["kind"], cnt, col)
    return p, c, cnt, col, st


@pytest.mark.parametrize("dim,ale", [(2, 0), (2, 1), (3, 0), (3, 1)])
def test_constants_are_preserved_bitwise(dim, ale):
    p, c, cnt, col, st = _case(dim, 9 if dim == 2 else 5, 6, 2.0, ale=ale)
    n = c["x"].shape[0]
    rng = np.random.default_rng(3)
    fv = rng.uniform(0.5, 2.0, size=(oracle.ncomp(dim), 6 ** dim))
    f = np.broadcast_to(fv, (n,) + fv.shape).copy()
    U = rng.normal(size=(n, dim)) * 0.3
    ft = oracle.transport(p, c["kind"], cnt, col, st, U, f)
    assert np.array_equal(ft, f)


@pytest.mark.parametrize("dim", [2, 3])
def test_symmetric_neighbourhood_gives_exact_linear_flux(dim):
    # Sec. 3.4.2: on a centrally symmetric stencil the dissipative parts of pairs j, -j cancel
    # for linear f, leaving Q = c.grad f; so f~ = f - dt c.b for f = a + b.x.
    n = 11 if dim == 2 else 9
    p, c, cnt, col, st = _case(dim, n, 4, 1.5, jitter=0.0)
    b = np.array([0.8, -0.5, 0.3])[:dim]
    fval = 2.0 + c["x"] @ b
    NV = 4 ** dim
    f = np.repeat(fval[:, None, None], oracle.ncomp(dim) * NV, axis=2).reshape(-1, oracle.ncomp(dim), NV)
    ft = oracle.transport(p, c["kind"], cnt, col, st, np.zeros((len(fval), dim)), f)
    vel = oracle.velocity_grid(dim, 4, 1.5)
    idx = np.indices((n,) * dim).reshape(dim, -1)[::-1].T
    far = np.where(np.all((idx >= 3) & (idx <= n - 4), axis=1))[0]
    expect = fval[far][:, None] - p["dt"] * (vel @ b)[None, :]
    for q in range(oracle.ncomp(dim)):
        assert np.allclose(ft[far, q, :], expect, atol=1e-12)


def test_upwind_direction_on_a_line():
    # Three points on a line (1D reduction of Sec. 3.4.2): with c > 0 only the upstream
    # neighbour contributes, f~_i = f_i - dt c (f_i - f_{i-1}) / dx.
    dx = 0.1
    x = np.array([[0.4, 0.5], [0.5, 0.5], [0.6, 0.5], [0.5, 0.6], [0.5, 0.4]])
    kind = np.array([1, 0, 1, 1, 1], dtype=np.int32)
    p = {"dim": 2, "nv": 2, "vmax": 1.0, "kn": 1.0, "dt": 0.01, "h": 0.11, "alpha": 6.25, "max_nbrs": 8,
         "tau_mode": 2}
    cnt, col = oracle.neighbours(x, p["h"], False, 8)
    st = oracle.stencils(p, x, kind, cnt, col)
    vel = oracle.velocity_grid(2, 2, 1.0)  # (+-1, +-1)
    rng = np.random.default_rng(5)
    f = rng.uniform(1, 2, size=(5, 2, 4))
    ft = oracle.transport(p, kind, cnt, col, st, np.zeros((5, 2)), f)
    for k in range(4):
        vx, vy = vel[k]
        up_x = 0 if vx > 0 else 2
        up_y = 4 if vy > 0 else 3
        expect = f[1, :, k] - p["dt"] * (abs(vx) * (f[1, :, k] - f[up_x, :, k]) + abs(vy) * (f[1, :, k] - f[up_y, :, k])) / dx
        assert np.allclose(ft[1, :, k], expect, rtol=1e-13)


def _dense_transport(p, c, cnt, col, st, U):
    """Transport matrix per velocity, by applying the oracle to unit vectors."""
    n = c["x"].shape[0]
    NV = p["nv"] ** p["dim"]
    nc = oracle.ncomp(p["dim"])
    L = np.zeros((NV, n, n))
    for j in range(n):
        f = np.zeros((n, nc, NV))
        f[j] = 1.0
        ft = oracle.transport(p, c["kind"], cnt, col, st, U, f)
        L[:, :, j] = ft[:, 0, :].T
        assert np.array_equal(ft[:, 0, :], ft[:, -1, :])  # same operator for g and h
    return L


@pytest.mark.parametrize("dim,ale", [(2, 0), (2, 1), (3, 0)])
def test_transport_is_positive_and_conservative_of_constants(dim, ale):
    # Positivity (Sec. 3.4.2): every off-diagonal coefficient -dt K_ij >= 0, rows sum to one,
    # and under dt sum_j |K_ij| <= 1 all entries are >= 0.
    n = 7 if dim == 2 else 4
    p, c, cnt, col, st = _case(dim, n, 4, 1.0, ale=ale)
    U = np.random.default_rng(2).normal(size=(c["x"].shape[0], dim)) * 0.2
    L = _dense_transport(p, c, cnt, col, st, U)
    interior = np.where(c["kind"] == 0)[0]
    for k in range(L.shape[0]):
        Li = L[k][interior]
        off = Li.copy()
        off[np.arange(len(interior)), interior] = 0.0
        assert off.min() >= 0.0
        assert np.allclose(Li.sum(1), 1.0, atol=1e-13)
        assert np.all(Li[np.arange(len(interior)), interior] >= -1e-15)


@pytest.mark.parametrize("dim,n,seed,ale", [(2, 11, 5, 0), (2, 11, 5, 1), (3, 5, 7, 0)])
def test_quadratic_fit_with_negative_normal_coefficient_stays_positive(dim, n, seed, ale):
    # Sec. 3.4.2 with the second-order fit of Sec. 3.4.1 on a strongly jittered cloud
    # (0.45 dx): some projected normal coefficients abar_n are negative, which the linear
    # fit never gives.  Every term abar_d c_d - |abar_d||c_d| is <= 0 whatever the sign of
    # abar_d, so the assembled operator keeps off-diagonal entries >= 0 and unit row sums.
    # The printed normal term abar_n (c_n - |c_n|) would make some entries negative here.
    p, c, cnt, col, st = _case(dim, n, 4, 1.0, seed=seed, jitter=0.45, ale=ale, wls_order=2)
    interior = np.where(c["kind"] == 0)[0]
    neg = [(i, s) for i in interior for s in range(cnt[i]) if st["abar"][i, s, 0] < 0.0]
    assert len(neg) > 0
    U = np.random.default_rng(4).normal(size=(c["x"].shape[0], dim)) * 0.2 if ale else np.zeros((len(c["x"]), dim))
    vel = oracle.velocity_grid(dim, 4, 1.0)
    # the printed form gives a positive K (a negative off-diagonal entry) for some of
    # these slots and velocities; the reading must not
    printed_positive = 0
    for i, s in neg:
        ab, fr = st["abar"][i, s], st["frame"][i, s]
        for v in vel:
            cd = fr @ (v - U[i])
            k = ab[0] * (cd[0] - abs(cd[0])) + sum(ab[d] * cd[d] - abs(ab[d]) * abs(cd[d]) for d in range(1, dim))
            printed_positive += k > 1e-12
    assert printed_positive > 0
    L = _dense_transport(p, c, cnt, col, st, U)
    for k in range(L.shape[0]):
        Li = L[k][interior]
        off = Li.copy()
        off[np.arange(len(interior)), interior] = 0.0
        assert off.min() >= 0.0
        assert np.allclose(Li.sum(1), 1.0, atol=1e-13)


@pytest.mark.parametrize("order,jitter", [(1, 0.0), (2, 0.1)])
def test_free_transport_converges_at_first_order(order, jitter):
    # Free transport: periodic box, no collisions, f0 = (1 + 0.1 sin 2 pi x) M(v);
    # the exact solution is f0(x - v t).  Fixed CFL, dx in {1/20, 1/40, 1/80}.  The
    # second-order WLS fit (on a jittered box) keeps first order: the upwind dissipation
    # and the explicit time step are O(h).
    nv, vmax, tfin, errs = 4, 1.0, 0.25, []
    for n in (20, 40, 80):
        cl = bi.periodic_box(2, n, seed=7, jitter=jitter) if jitter else bi.periodic_box(2, n)
        dx = 1.0 / n
        dt0 = 0.5 * dx / (vmax * math.sqrt(2))
        nsteps = int(math.ceil(tfin / dt0))
        p = {"dim": 2, "nv": nv, "vmax": vmax, "kn": 1.0, "tau_mode": 2, "dt": tfin / nsteps, "h": 2.5 * dx,
             "alpha": 6.25, "max_nbrs": 48, "periodic": 1, "ale": 0, "wls_order": order}
        vel = oracle.velocity_grid(2, nv, vmax)
        M = oracle.maxwellian(p, 1.0, (0.0, 0.0), 1.0)
        f0 = (1 + 0.1 * np.sin(2 * np.pi * cl["x"][:, 0]))[:, None, None] * M[None]
        sim = oracle.Simulation(p, cl, f0=f0)
        sim.run(nsteps)
        xs = cl["x"][:, 0][:, None] - vel[None, :, 0] * tfin
        exact = (1 + 0.1 * np.sin(2 * np.pi * xs))[:, None, :] * M[None]
        errs.append(np.sqrt(((sim.f - exact) ** 2).mean()))
    orders = [math.log2(errs[i] / errs[i + 1]) for i in range(2)]
    assert all(0.8 <= o <= 1.2 for o in orders), (errs, orders)


def _run_cavity(dim, n, nv, vmax, steps, lid, seed=9):
    name = "cavity2d_n41_v16_f64" if dim == 2 else "cavity3d_n41_v16_f32"
    p = bi.config(name, n=n, nv=nv, vmax=vmax)
    p["lid_u"] = [lid, 0.0, 0.0]
    cl = bi.cavity(dim, n, seed)
    sim = oracle.Simulation(p, cl)
    return p, cl, sim


@pytest.mark.parametrize("dim", [2, 3])
def test_walls_have_zero_net_mass_flux(dim):
    p, cl, sim = _run_cavity(dim, 13 if dim == 2 else 6, 12 if dim == 2 else 8, 4.0, 0, 0.3)
    sim.run(3)
    vel = oracle.velocity_grid(dim, p["nv"], p["vmax"])
    for b in np.where(cl["kind"] != 0)[0]:
        vn = vel @ cl["normal"][b]
        g = sim.f[b, 0]
        flux = (vn * g).sum()
        scale = (np.abs(vn) * g).sum()
        assert abs(flux) < 1e-13 * scale


def test_diffuse_reflection_has_wall_maxwellian_shape():
    p, cl, sim = _run_cavity(2, 13, 12, 4.0, 0, 0.3)
    sim.run(2)
    vel = oracle.velocity_grid(2, p["nv"], p["vmax"])
    for b in np.where(cl["kind"] != 0)[0]:
        uw = p["lid_u"][:2] if cl["kind"][b] == p["lid_wall"] else [0.0, 0.0]
        Mw = oracle.maxwellian(p, 1.0, uw, p["wall_T"])
        nb = cl["normal"][b]
        out = (vel[:, 0] * nb[0] + vel[:, 1] * nb[1]) > 0  # same rounding as the oracle (no FMA)
        ratio = sim.f[b, 0, out] / Mw[0, out]
        assert np.allclose(ratio, ratio[0], rtol=1e-13)
        assert np.allclose(sim.f[b, 1, out], p["wall_T"] * sim.f[b, 0, out], rtol=1e-15)


@pytest.mark.parametrize("dim,n,nv,vmax,steps", [(2, 9, 40, 9.0, 100), (3, 5, 24, 8.5, 6)])
def test_global_maxwellian_with_walls_at_rest_is_stationary(dim, n, nv, vmax, steps):
    # A global Maxwellian with walls at rest stays put, on a velocity grid whose discrete
    # moments of a unit Maxwellian are exact to rounding.
    p, cl, sim = _run_cavity(dim, n, nv, vmax, steps, 0.0)
    f0 = sim.f.copy()
    sim.run(steps)
    assert np.abs(sim.f - f0).max() < 1e-12 * f0.max()
    assert np.abs(sim.rho - 1).max() < 1e-12 and np.abs(sim.T - 1).max() < 1e-12


def test_ale_points_at_rest_do_not_move():
    # U = 0 exactly leaves positions bitwise unchanged; a global Maxwellian at rest (fine
    # velocity grid, so U = O(1e-15)) moves no point by more than rounding.
    p, cl, sim = _run_cavity(2, 9, 40, 9.0, 0, 0.0)
    x = cl["x"].copy()
    assert oracle.move(dict(p, ale=1), cl["kind"], np.zeros_like(x), x) == 0
    assert np.array_equal(x, cl["x"])
    sim.p["ale"] = 1
    sim.q = oracle.params(sim.p)
    sim.run(5)
    assert np.abs(sim.U).max() < 1e-13
    assert np.abs(sim.x - cl["x"]).max() < 1e-16


def test_ale_uniform_drift_translates_every_point():
    # Eq. (ALE1): x^{n+1} = x^n + dt U^{n+1}; a drifting global Maxwellian in a periodic box
    # keeps U uniform, so every point moves by the same dt U each step.
    n, nv, vmax = 8, 40, 9.0
    cl = bi.periodic_box(2, n)
    p = {"dim": 2, "nv": nv, "vmax": vmax, "kn": 0.1, "tau_mode": 0, "dt": 0.01, "h": 2.5 / n,
         "alpha": 6.25, "max_nbrs": 48, "periodic": 1, "ale": 1}
    u0 = np.array([0.37, -0.21])
    sim = oracle.Simulation(p, cl, U0=(u0[0], u0[1], 0.0))
    x = cl["x"].copy()
    f0 = sim.f.copy()
    for _ in range(4):
        sim.run(1)
        assert np.allclose(sim.U, sim.U[0], atol=1e-14)
        x = np.mod(x + p["dt"] * sim.U, 1.0)
        assert np.allclose(sim.x, x, atol=1e-15)
    assert np.allclose(sim.U[0], u0, atol=1e-12)
    assert np.abs(sim.f - f0).max() < 1e-12 * f0.max()


def test_ale_wall_guard_clamps():
    p = {"dim": 2, "nv": 4, "vmax": 1.0, "kn": 0.1, "dt": 0.1, "h": 0.1, "alpha": 6.25, "guard": 0.05,
         "max_nbrs": 8, "ale": 1}
    x = np.array([[0.5, 0.06], [0.5, 0.5], [0.0, 0.5]])
    kind = np.array([0, 0, 1], dtype=np.int32)
    U = np.array([[0.0, -0.5], [0.2, 0.0], [5.0, 5.0]])
    nclamp = oracle.move(p, kind, U, x)
    assert nclamp == 1
    assert np.array_equal(x, [[0.5, 0.05], [0.52, 0.5], [0.0, 0.5]])
