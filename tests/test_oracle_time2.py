"""Pins of the oracle's second-order time discretisation (time_order = 2; the paper's is
first order, Sec. 3.2, and it names higher order as future work): Strang splitting
R(dt/2) T(dt) R(dt/2) with the exact relaxation solve and a two-stage explicit (Heun,
SSP-RK2) transport.

- Relaxation alone (a uniform state in a periodic box, where the transport is the
  identity): after N steps f = M + (f0 - M) exp(-N dt / tau) for time_order 2, and
  M + (f0 - M) (tau / (tau + dt))^N for the paper's implicit step (time_order 1).
- Transport alone (no collisions, periodic lattice): against the exact solution
  expm(t A) f0 of the semi-discrete system df/dt = A f, where A is the oracle's
  first-order transport operator assembled column by column, the time error falls as
  dt^2 for time_order 2 and as dt for time_order 1.  One step of time_order 2 equals
  (I + dt A + dt^2 A^2 / 2) f.
- Both together (a non-uniform, non-equilibrium start with collisions): the difference
  between runs at dt and dt/2 to a fixed time falls by 4 per halving (by 2 for the
  first-order scheme).
"""
import math

import numpy as np
import pytest
import scipy.linalg

import bgk_inputs as bi
import oracle


def _box_params(n, nv, vmax, tau_mode, kn, dt, order, dim=2):
    dx = 1.0 / n
    return {"dim": dim, "nv": nv, "vmax": vmax, "kn": kn, "tau_mode": tau_mode, "dt": dt, "h": 2.5 * dx,
            "alpha": 6.25, "max_nbrs": 48 if dim == 2 else 160, "periodic": 1, "ale": 0, "time_order": order}


@pytest.mark.parametrize("dim", [2, 3])
def test_uniform_relaxation_follows_the_closed_forms(dim):
    # grids on which the discrete moments of these Maxwellians are exact to about 1e-12
    # (the relaxation keeps the moments only as far as the discrete M reproduces them)
    nv, vmax = (32, 9.0) if dim == 2 else (22, 8.0)
    n = 4
    cl = bi.periodic_box(dim, n)
    kn, dt, N = 0.3, 0.05, 12
    tau = math.sqrt(2.0 / math.pi) * kn  # tau_mode 1
    p1 = _box_params(n, nv, vmax, 1, kn, dt, 1, dim)
    u_a, u_b = [0.3, -0.1, 0.2][:dim], [-0.4, 0.2, 0.1][:dim]
    f0row = 0.5 * (oracle.maxwellian(p1, 1.0, u_a, 1.0) + oracle.maxwellian(p1, 0.6, u_b, 1.3))
    f0 = np.broadcast_to(f0row, (n ** dim,) + f0row.shape).copy()
    rho, U, T = oracle.moments_point(p1, f0row)
    M = oracle.maxwellian(p1, rho, U, T)
    for order, factor in ((2, math.exp(-N * dt / tau)), (1, (tau / (tau + dt)) ** N)):
        p = dict(p1, time_order=order)
        sim = oracle.Simulation(p, cl, f0=f0)
        sim.run(N)
        want = M + (f0row - M) * factor
        assert np.abs(sim.f - want[None]).max() < 1e-11 * np.abs(f0row).max(), order


def _transport_operator(p, cl):
    """A with T1 f = f + dt A f (T1 the first-order transport), per (component, velocity):
    A[c, k] is n x n; column j from the transport of the unit vector of point j."""
    n = len(cl["kind"])
    nc, NV = oracle.ncomp(p["dim"]), oracle.nvel(p["dim"], p["nv"])
    cnt, col = oracle.neighbours(cl["x"], p["h"], True, p["max_nbrs"])
    st = oracle.stencils(p, cl["x"], cl["kind"], cnt, col)
    A = np.zeros((nc, NV, n, n))
    U = np.zeros((n, p["dim"]))
    for j in range(n):
        e = np.zeros((n, nc, NV))
        e[j] = 1.0
        ft = oracle.transport(p, cl["kind"], cnt, col, st, U, e)
        A[:, :, :, j] = ((ft - e) / p["dt"]).transpose(1, 2, 0)
    return A


def test_heun_step_is_the_second_order_taylor_polynomial():
    n, nv, vmax = 6, 4, 1.0
    cl = bi.periodic_box(2, n, seed=3, jitter=0.1)
    p = _box_params(n, nv, vmax, 2, 1.0, 0.02, 2)
    A = _transport_operator(dict(p, time_order=1), cl)
    rng = np.random.default_rng(11)
    f0 = rng.uniform(0.5, 1.5, (n * n, 2, nv * nv))
    sim = oracle.Simulation(p, cl, f0=f0)
    sim.run(1)
    dt = p["dt"]
    for c in range(2):
        for k in range(nv * nv):
            g = f0[:, c, k]
            Ag = A[c, k] @ g
            want = g + dt * Ag + 0.5 * dt * dt * (A[c, k] @ Ag)
            assert np.abs(sim.f[:, c, k] - want).max() < 1e-13


def test_free_transport_time_error_orders():
    n, nv, vmax, tfin = 8, 4, 1.0, 0.2
    cl = bi.periodic_box(2, n, seed=5, jitter=0.1)
    dt0 = 0.5 * (1.0 / n) / (vmax * math.sqrt(2))
    base = _box_params(n, nv, vmax, 2, 1.0, dt0, 1)
    A = _transport_operator(base, cl)
    vel = oracle.velocity_grid(2, nv, vmax)
    M = oracle.maxwellian(base, 1.0, (0.0, 0.0), 1.0)
    x = cl["x"]
    f0 = (1 + 0.2 * np.sin(2 * np.pi * x[:, 0]) * np.cos(2 * np.pi * x[:, 1]))[:, None, None] * M[None]
    exact = np.zeros_like(f0)
    for c in range(2):
        for k in range(nv * nv):
            exact[:, c, k] = scipy.linalg.expm(tfin * A[c, k]) @ f0[:, c, k]
    for order, lo, hi in ((1, 0.85, 1.15), (2, 1.85, 2.15)):
        errs = []
        for m in (8, 16, 32):
            p = dict(base, dt=tfin / m, time_order=order)
            sim = oracle.Simulation(p, cl, f0=f0)
            sim.run(m)
            errs.append(np.abs(sim.f - exact).max())
        orders = [math.log2(errs[i] / errs[i + 1]) for i in range(2)]
        assert all(lo <= o <= hi for o in orders), (order, errs, orders)


def test_full_scheme_self_convergence_orders():
    # a smooth density and velocity perturbation out of equilibrium, Kn such that tau is
    # a few steps: the splitting and both sub-steps contribute to the error
    n, nv, vmax, tfin = 8, 8, 4.0, 0.16
    cl = bi.periodic_box(2, n, seed=9, jitter=0.1)
    x = cl["x"]
    base = _box_params(n, nv, vmax, 0, 0.05, tfin / 8, 1)
    f0 = np.empty((n * n, 2, nv * nv))
    for i in range(n * n):
        r = 1.0 + 0.1 * np.sin(2 * np.pi * x[i, 0])
        u = (0.1 * np.cos(2 * np.pi * x[i, 1]), 0.05)
        f0[i] = 0.7 * oracle.maxwellian(base, r, u, 1.0) + 0.3 * oracle.maxwellian(base, r, (0.0, -0.2), 0.7)
    for order, lo, hi in ((1, 0.8, 1.25), (2, 1.8, 2.25)):
        sols = []
        for m in (8, 16, 32, 64):
            p = dict(base, dt=tfin / m, time_order=order)
            sim = oracle.Simulation(p, cl, f0=f0)
            sim.run(m)
            sols.append(sim.f.copy())
        d = [np.abs(sols[i] - sols[i + 1]).max() for i in range(3)]
        orders = [math.log2(d[i] / d[i + 1]) for i in range(2)]
        assert all(lo <= o <= hi for o in orders), (order, d, orders)


def test_second_order_needs_fixed_points():
    p = bi.config("cavity2d_ale_n201_v32_f32", n=9, nv=4, storage="f64", time_order=2)
    sim = oracle.Simulation(p, bi.cloud_for(p))
    with pytest.raises(RuntimeError):
        sim.run(1)


@pytest.mark.parametrize("dim,n,nv,vmax,steps", [(2, 9, 40, 9.0, 40), (3, 5, 24, 8.5, 4)])
def test_global_maxwellian_with_walls_at_rest_stays_stationary(dim, n, nv, vmax, steps):
    # walls applied to the first stage and to the result: a global Maxwellian with every
    # wall at rest (lid speed 0) is a fixed point of the second-order step too, on a grid
    # whose discrete moments of a unit Maxwellian are exact to rounding
    name = "cavity2d_n41_v16_f64" if dim == 2 else "cavity3d_n41_v16_f32"
    p = bi.config(name, n=n, nv=nv, vmax=vmax, storage="f64", time_order=2)
    p["lid_u"] = [0.0, 0.0, 0.0]
    sim = oracle.Simulation(p, bi.cavity(dim, n, 9))
    f0 = sim.f.copy()
    sim.run(steps)
    assert np.abs(sim.f - f0).max() < 1e-12 * f0.max()
    assert np.abs(sim.rho - 1).max() < 1e-12 and np.abs(sim.T - 1).max() < 1e-12
