"""Pins of the oracle's discrete adjoint (fixed points).

The adjoint is not in the paper; it is the vector-Jacobian product of the
oracle's own step map.  It is pinned against that step map: the transpose
identity <L x, y> = <x, L^T y> for the (linear) collisionless transport, and
central finite differences of the full step and of the time-averaged lid-flux
objective in random directions and in the parameters (u_lid, Kn).
"""
import numpy as np
import pytest

import bgk_inputs as bi
import oracle


def _step(p, cl, f):
    sim = oracle.Simulation(p, cl, f0=f)
    sim.run(1)
    return sim.f


def _lists(p, cl):
    cnt, col = oracle.neighbours(cl["x"], p["h"], bool(p.get("periodic")), p["max_nbrs"])
    st = oracle.stencils(p, cl["x"], cl["kind"], cnt, col)
    return cnt, col, st


def _perturbed_maxwellian(p, n, seed):
    rng = np.random.default_rng(seed)
    M = oracle.maxwellian(p, 1.0, (0.05, -0.03, 0.02), 1.0)
    return M[None] * (1.0 + 0.2 * rng.uniform(-1, 1, size=(n,) + M.shape))


def test_transport_adjoint_is_the_transpose():
    # Collisionless periodic box: the step is the linear transport L, so <L x, y> = <x, L^T y>.
    cl = bi.periodic_box(2, 9, seed=3, jitter=0.1)
    p = {"dim": 2, "nv": 5, "vmax": 2.0, "kn": 1.0, "tau_mode": 2, "dt": 0.01, "h": 2.5 / 9, "alpha": 6.25,
         "max_nbrs": 48, "periodic": 1}
    cnt, col, st = _lists(p, cl)
    rng = np.random.default_rng(0)
    shape = (len(cl["kind"]), 2, 25)
    x, y = rng.normal(size=shape), rng.normal(size=shape)
    Lx = _step(p, cl, x)
    LTy, dth = oracle.adjoint_step(p, cl["kind"], cl["normal"], cnt, col, st, x, y)
    lhs, rhs = float((Lx * y).sum()), float((x * LTy).sum())
    assert abs(lhs - rhs) < 1e-12 * max(abs(lhs), 1.0)
    assert np.all(dth == 0.0)


@pytest.mark.parametrize("dim,tau_mode", [(2, 0), (2, 1), (3, 0)])
def test_step_vjp_matches_central_differences(dim, tau_mode):
    name = "cavity2d_n41_v16_f64" if dim == 2 else "cavity3d_n41_v16_f32"
    p = bi.config(name, n=7 if dim == 2 else 5, nv=6, vmax=4.0, tau_mode=tau_mode, kn=0.2)
    p["lid_u"] = [0.2, 0.0, 0.0]
    cl = bi.cloud_for(p)
    n = len(cl["kind"])
    cnt, col, st = _lists(p, cl)
    f = _perturbed_maxwellian(p, n, 1)
    rng = np.random.default_rng(2)
    lam, delta = rng.normal(size=f.shape), rng.normal(size=f.shape)
    lam0, dth = oracle.adjoint_step(p, cl["kind"], cl["normal"], cnt, col, st, f, lam)
    eps = 1e-5
    fd = ((_step(p, cl, f + eps * delta) - _step(p, cl, f - eps * delta)) * lam).sum() / (2 * eps)
    ad = (lam0 * delta).sum()
    assert abs(fd - ad) < 1e-6 * abs(ad), (fd, ad)
    # parameters: lid velocity (x component) and Kn
    for key, idx, h in (("lid", 0, 1e-5), ("kn", 3, 1e-6)):
        pp, pm = dict(p), dict(p)
        if key == "lid":
            pp["lid_u"] = [p["lid_u"][0] + h, 0.0, 0.0]
            pm["lid_u"] = [p["lid_u"][0] - h, 0.0, 0.0]
        else:
            pp["kn"], pm["kn"] = p["kn"] + h, p["kn"] - h
        fdp = ((_step(pp, cl, f) - _step(pm, cl, f)) * lam).sum() / (2 * h)
        assert abs(fdp - dth[idx]) < 1e-6 * max(abs(dth[idx]), 1e-8), (key, fdp, dth[idx])


def test_objective_gradient_matches_central_differences():
    # J = (1/N) sum_n lid x-momentum flux of f^n over N steps; central differences with eps = 1e-4
    p = bi.config("cavity2d_n41_v16_f64", n=9, nv=8, vmax=4.0, kn=0.1)
    p["lid_u"] = [0.1, 0.0, 0.0]
    cl = bi.cloud_for(p)
    N = 8

    def J_of(q, f0=None):
        sim = oracle.Simulation(q, cl, f0=f0)
        J = 0.0
        for _ in range(N):
            sim.run(1)
            J += oracle.objective(q, cl["kind"], sim.f) / N
        return J

    sim = oracle.Simulation(p, cl)
    f0 = sim.f.copy()
    J, dth, lam0 = sim.gradient(N)
    assert abs(J - J_of(p)) < 1e-14 * max(abs(J), 1e-30)
    eps = 1e-4
    for idx, key in ((0, "lid"), (3, "kn")):
        pp, pm = dict(p), dict(p)
        if key == "lid":
            pp["lid_u"], pm["lid_u"] = [p["lid_u"][0] + eps, 0, 0], [p["lid_u"][0] - eps, 0, 0]
        else:
            pp["kn"], pm["kn"] = p["kn"] + eps, p["kn"] - eps
        fd = (J_of(pp) - J_of(pm)) / (2 * eps)
        assert abs(fd - dth[idx]) < 1e-6 * abs(dth[idx]), (key, fd, dth[idx])
    delta = np.random.default_rng(4).normal(size=f0.shape) * f0
    fd = (J_of(p, f0 + eps * delta) - J_of(p, f0 - eps * delta)) / (2 * eps)
    ad = (lam0 * delta).sum()
    assert abs(fd - ad) < 1e-6 * abs(ad), (fd, ad)
