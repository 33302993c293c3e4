"""Pins of the oracle's kinetic model: velocity grid, Maxwellian, moments, tau, relaxation.

Each check compares the oracle with something other than itself: closed-form
moments of a Gaussian, the paper's printed relaxation times, the Chu marginals
of the 3D Maxwellian, and the closed-form solution of homogeneous relaxation.
"""
import math
import os

import numpy as np
import pytest

import bgk_inputs as bi
import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _p(dim, nv, vmax, **kw):
    p = {"dim": dim, "nv": nv, "vmax": vmax, "kn": 0.1, "tau_mode": 0, "dt": 1e-3, "h": 0.1,
         "alpha": 6.25, "max_nbrs": 48 if dim == 2 else 160}
    p.update(kw)
    return p


def test_velocity_nodes_follow_paper_grid():
    # Sec. 3.3: nodes -vmax + (j-1) dv, j = 1..N_v+1, dv = 2 vmax / N_v; here nv = N_v + 1 nodes.
    for nv, vmax in [(16, 5.0), (32, 6.0), (17, 5.0), (2, 1.0)]:
        v = oracle.velocity_nodes(nv, vmax)
        assert len(v) == nv
        assert abs(v[0] + vmax) < 1e-14 * vmax
        assert abs(v[-1] - vmax) < 1e-14 * vmax
        assert np.allclose(np.diff(v), 2 * vmax / (nv - 1), rtol=0, atol=1e-14)
        assert abs(oracle.dv(nv, vmax) - 2 * vmax / (nv - 1)) < 1e-15
        # exactly symmetric about zero
        assert np.array_equal(v, -v[::-1])


def test_velocity_grid_order_kx_fastest():
    g = oracle.velocity_grid(3, 4, 1.5)
    nodes = oracle.velocity_nodes(4, 1.5)
    k = 1 + 4 * (2 + 4 * 3)
    assert np.array_equal(g[k], [nodes[1], nodes[2], nodes[3]])
    g2 = oracle.velocity_grid(2, 5, 2.0)
    assert np.array_equal(g2[7], [oracle.velocity_nodes(5, 2.0)[2], oracle.velocity_nodes(5, 2.0)[1]])


def _quad(dim, nv, vmax):
    g = oracle.velocity_grid(dim, nv, vmax)
    return g, oracle.dv(nv, vmax) ** dim


@pytest.mark.parametrize("rho,U,T", [(1.0, (0.0, 0.0, 0.0), 1.0), (0.7, (0.3, -0.2, 0.1), 1.3), (1.9, (-0.5, 0.4, 0.0), 0.6)])
def test_maxwellian_3d_has_its_parameters_as_moments(rho, U, T):
    # Eq. (maxwellian) with the minus sign in the exponent: on a wide, fine grid the
    # rectangle rule is exact for Gaussians to rounding, so the discrete moments must
    # reproduce (rho, U, T) of Eqs. (moments), (internal_energy).
    p = _p(3, 36, 10.0)
    g, w = _quad(3, 36, 10.0)
    M = oracle.maxwellian(p, rho, U, T)[0]
    r = (M * w).sum()
    u = (g * M[:, None] * w).sum(0) / r
    e = ((((g - u) ** 2).sum(1)) * M * w).sum()
    assert abs(r - rho) < 1e-12 * rho
    assert np.allclose(u, U[:3], atol=1e-12)
    assert abs(e / (3 * r) - T) < 1e-12
    rr, uu, TT = oracle.moments_point(p, M[None, :])
    assert abs(rr - rho) < 1e-12 and np.allclose(uu, U[:3], atol=1e-12) and abs(TT - T) < 1e-12


@pytest.mark.parametrize("rho,U,T", [(1.0, (0.0, 0.0), 1.0), (0.5, (0.25, -0.4), 1.7), (1.4, (0.1, 0.1), 0.45)])
def test_chu_pair_has_its_parameters_as_moments(rho, U, T):
    # Eqs. (Maxw_G1), (Maxw_G2), (macroeq): rho = int G1, rho U = int v G1,
    # 3 rho T = int |v-U|^2 G1 + int G2.  Fails without the pi of G1's prefactor.
    p = _p(2, 60, 12.0)
    g, w = _quad(2, 60, 12.0)
    G = oracle.maxwellian(p, rho, U, T)
    r = (G[0] * w).sum()
    u = (g * G[0][:, None] * w).sum(0) / r
    e = ((((g - u) ** 2).sum(1)) * G[0] * w).sum() + (G[1] * w).sum()
    assert abs(r - rho) < 1e-12 * rho
    assert np.allclose(u, U, atol=1e-12)
    assert abs(e / (3 * r) - T) < 1e-12
    assert np.allclose(G[1], T * G[0], rtol=1e-15, atol=0)
    rr, uu, TT = oracle.moments_point(p, G)
    assert abs(rr - rho) < 1e-12 and np.allclose(uu, U, atol=1e-12) and abs(TT - T) < 1e-12


def test_chu_pair_is_the_v3_marginal_of_the_3d_maxwellian():
    # Sec. 2.1, Eqs. (reduced_g1), (reduced_g2): G1 = int M dv3, G2 = int v3^2 M dv3.
    nv, vmax = 28, 9.0
    rho, U, T = 1.2, (0.3, -0.15, 0.0), 0.9
    M3 = oracle.maxwellian(_p(3, nv, vmax), rho, U, T)[0].reshape(nv, nv, nv)  # [kz, ky, kx]
    v = oracle.velocity_nodes(nv, vmax)
    dv = oracle.dv(nv, vmax)
    G1 = (M3 * dv).sum(0).reshape(-1)
    G2 = (M3 * (v ** 2)[:, None, None] * dv).sum(0).reshape(-1)
    G = oracle.maxwellian(_p(2, nv, vmax), rho, U[:2], T)
    assert np.allclose(G[0], G1, rtol=0, atol=1e-13 * G1.max())
    assert np.allclose(G[1], G2, rtol=0, atol=1e-13 * G2.max())


def _golden_tau():
    vals, rows = {}, []
    with open(os.path.join(GOLDEN, "tau_argon.txt")) as fh:
        for line in fh:
            line = line.split("#")[0].split()
            if not line:
                continue
            if line[0] == "rho":
                rows.append((float(line[1]), float(line[3])))
            elif line[0] != "Kn":
                vals[line[0]] = float(line[1])
    return vals, rows


def test_tau_matches_printed_argon_values():
    # Sec. 5.1 prints tau = 3.7142e-10 s (rho0 = 1) and 3.7142e-9 s (rho0 = 0.1) for argon,
    # from Eqs. (tau), (lambda) with the printed constants.
    c, rows = _golden_tau()
    for rho, tau_printed in rows:
        t = oracle.tau_si(c["k_B"], c["R"], c["d"], rho, c["T0"])
        assert abs(t - tau_printed) < 5e-5 * tau_printed, (rho, t, tau_printed)


def test_nondimensional_tau_is_the_scaled_si_tau():
    # With L, sqrt(R T0), rho0 = 1, T0 as units, Eqs. (tau), (lambda) give
    # tau' = sqrt(2/pi) Kn / (rho sqrt(T)) with Kn = lambda(rho0) / L.
    c, _ = _golden_tau()
    for rho_si, T_si in [(1.0, 270.0), (0.37, 270.0), (1.0, 410.0), (2.5, 180.0)]:
        kn = oracle.lambda_si(c["k_B"], c["R"], c["d"], 1.0) / c["L"]
        t_si = oracle.tau_si(c["k_B"], c["R"], c["d"], rho_si, T_si)
        t_scaled = t_si * math.sqrt(c["R"] * c["T0"]) / c["L"]
        t_nd = oracle.tau(_p(2, 4, 1.0, kn=kn), rho_si / 1.0, T_si / c["T0"])
        assert abs(t_nd - t_scaled) < 1e-12 * t_scaled
    # the printed Kn 0.11 belongs to rho0 = 1 (the text swaps the pairing)
    kn1 = oracle.lambda_si(c["k_B"], c["R"], c["d"], 1.0) / c["L"]
    assert abs(kn1 - 0.11) < 0.005
    assert abs(oracle.tau(_p(2, 4, 1.0, kn=1.0, tau_mode=1), 3.0, 5.0) - math.sqrt(2 / math.pi)) < 1e-15


def _homogeneous_run(dim, nv, vmax, dt, nsteps, tau_mode=1):
    """A periodic box with a spatially uniform non-equilibrium f0 (two Maxwellians)."""
    p = bi.config("cavity2d_n41_v16_f64" if dim == 2 else "cavity3d_n41_v16_f32", nv=nv, vmax=vmax)
    p.update(periodic=1, n=4, h=0.3, dt=dt, tau_mode=tau_mode, kn=0.2, ale=0, max_nbrs=80)
    cloud = bi.periodic_box(dim, 4)
    U1, U2 = np.array([0.6, -0.3, 0.2])[:dim], np.array([-0.4, 0.5, -0.1])[:dim]
    r1, r2, T1, T2 = 0.7, 0.5, 0.8, 1.5
    f0 = oracle.maxwellian(p, r1, U1, T1) + oracle.maxwellian(p, r2, U2, T2)
    rho = r1 + r2
    U = (r1 * U1 + r2 * U2) / rho
    T = (r1 * (3 * T1 + ((U1 - U) ** 2).sum()) + r2 * (3 * T2 + ((U2 - U) ** 2).sum())) / (3 * rho)
    M = oracle.maxwellian(p, rho, U, T)
    sim = oracle.Simulation(p, cloud, f0=np.broadcast_to(f0, (cloud["x"].shape[0],) + f0.shape))
    sim.run(nsteps)
    return p, f0, M, sim, (rho, U, T)


@pytest.mark.parametrize("dim,nv,vmax", [(2, 60, 12.0), (3, 32, 10.0)])
def test_homogeneous_relaxation_closed_form(dim, nv, vmax):
    # Sec. 3.2: with transport inactive, f^{n+1} = (tau f^n + dt M)/(tau + dt) and M fixed,
    # so f^n = M + (f0 - M) (tau/(tau+dt))^n.  M is built from the closed-form moments of f0.
    nsteps, dt = 12, 0.05
    p, f0, M, sim, (rho, U, T) = _homogeneous_run(dim, nv, vmax, dt, nsteps)
    tau = math.sqrt(2 / math.pi) * p["kn"]
    expect = M + (f0 - M) * (tau / (tau + dt)) ** nsteps
    err = np.abs(sim.f - expect[None]).max() / np.abs(f0).max()
    assert err < 1e-13, err
    assert np.allclose(sim.rho, rho, rtol=1e-13) and np.allclose(sim.T, T, rtol=1e-13)
    assert np.allclose(sim.U, U[None], atol=1e-13)


def test_homogeneous_relaxation_converges_to_exponential_at_first_order():
    # The implicit step is first order: f(t) - f_exact(t) = O(dt), f_exact = M + (f0 - M) e^{-t/tau}.
    tfin, errs = 0.4, []
    for nsteps in (8, 16, 32):
        p, f0, M, sim, _ = _homogeneous_run(2, 60, 12.0, tfin / nsteps, nsteps)
        tau = math.sqrt(2 / math.pi) * p["kn"]
        exact = M + (f0 - M) * math.exp(-tfin / tau)
        errs.append(np.abs(sim.f[0] - exact).max())
    orders = [math.log2(errs[i] / errs[i + 1]) for i in range(2)]
    assert all(0.85 < o < 1.15 for o in orders), orders


def test_local_tau_uses_density_and_temperature():
    # tau = sqrt(2/pi) Kn / (rho sqrt T): doubling rho halves tau; T four times larger halves it too.
    p = _p(2, 4, 1.0, kn=0.3)
    t0 = oracle.tau(p, 1.0, 1.0)
    assert abs(t0 - math.sqrt(2 / math.pi) * 0.3) < 1e-15
    assert abs(oracle.tau(p, 2.0, 1.0) - t0 / 2) < 1e-15
    assert abs(oracle.tau(p, 1.0, 4.0) - t0 / 2) < 1e-15


def test_midpoint_velocity_grid():
    # vgrid 1: nv cells of width 2 vmax / nv over [-vmax, vmax], a node at each centre,
    # exactly symmetric; the midpoint rule integrates a Maxwellian to rounding on a wide grid
    for nv, vmax in [(16, 5.0), (17, 5.0), (2, 1.0)]:
        v = oracle.velocity_nodes(nv, vmax, 1)
        d = 2 * vmax / nv
        assert abs(oracle.dv(nv, vmax, 1) - d) < 1e-15
        assert abs(v[0] - (-vmax + d / 2)) < 1e-14 and abs(v[-1] - (vmax - d / 2)) < 1e-14
        assert np.allclose(np.diff(v), d, rtol=0, atol=1e-14)
        assert np.array_equal(v, -v[::-1])
    p = _p(2, 40, 10.0, vgrid=1)
    M = oracle.maxwellian(p, 0.8, (0.3, -0.2), 1.2)
    rho, U, T = oracle.moments_point(p, M)
    assert abs(rho - 0.8) < 1e-12 and np.abs(U - [0.3, -0.2]).max() < 1e-12 and abs(T - 1.2) < 1e-12
    # the same numbers as an explicit midpoint sum
    g = oracle.velocity_grid(2, 40, 10.0, 1)
    assert abs(M[0].sum() * oracle.dv(40, 10.0, 1) ** 2 - 0.8) < 1e-12
    assert np.abs(g[:40, 0] - oracle.velocity_nodes(40, 10.0, 1)).max() == 0.0


def test_global_maxwellian_stationary_on_the_midpoint_grid():
    # the midpoint grid (vgrid 1) through the whole step with walls at rest: a global
    # Maxwellian stays put to rounding on a grid wide and fine enough for its moments
    import bgk_inputs as bi
    p = bi.config("cavity2d_n41_v16_f64", n=9, nv=40, vmax=9.0, vgrid=1)
    p["lid_u"] = [0.0, 0.0, 0.0]
    sim = oracle.Simulation(p, bi.cavity(2, 9, 9))
    f0 = sim.f.copy()
    sim.run(50)
    assert np.abs(sim.f - f0).max() < 1e-12 * f0.max()
    assert np.abs(sim.rho - 1).max() < 1e-12 and np.abs(sim.T - 1).max() < 1e-12
