"""GPU discrete adjoint (bgk_adjoint_step, bgk_objective) against the FP64 oracle adjoint.

One adjoint step on random states and random adjoint vectors (FP64 to 1e-10,
FP32 to 1e-4 normwise); the checkpointed multi-step gradient of the lid-flux
objective against the oracle's gradient; and, on the 101^2 x 24^2 cavity over
1000 steps, the FP32 adjoint gradient against central finite differences of the
FP64 GPU path (eps = 1e-4, relative 1e-3) and against the FP64 adjoint.
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


def _pad(a, nvp):
    out = np.zeros(a.shape[:-1] + (nvp,))
    out[..., : a.shape[-1]] = a
    return out


@pytest.mark.parametrize("dim,storage,tau_mode,tol", [(2, "f64", 0, 1e-10), (2, "f64", 1, 1e-10), (3, "f64", 0, 1e-10),
                                                      (2, "f32", 0, 1e-4), (3, "f32", 0, 1e-4)])
def test_adjoint_step_matches_oracle(g, dim, storage, tau_mode, tol):
    import torch
    name = "cavity2d_n41_v16_f64" if dim == 2 else "cavity3d_n41_v16_f32"
    p = bi.config(name, n=11 if dim == 2 else 6, nv=6, vmax=4.0, kn=0.2, tau_mode=tau_mode, storage=storage)
    p["lid_u"] = [0.2, 0.0, 0.0]
    cl = bi.cloud_for(p)
    n = len(cl["kind"])
    rng = np.random.default_rng(11)
    M = oracle.maxwellian(p, 1.0, (0.05, -0.03, 0.02), 1.0)
    f = M[None] * (1.0 + 0.2 * rng.uniform(-1, 1, size=(n,) + M.shape))
    lam = rng.normal(size=f.shape)
    cnt, col = oracle.neighbours(cl["x"], p["h"], False, p["max_nbrs"])
    st = oracle.stencils(p, cl["x"], cl["kind"], cnt, col)
    lam0, dth = oracle.adjoint_step(p, cl["kind"], cl["normal"], cnt, col, st, f, lam)

    s = g.Solver([p], [cl])
    s.set_f(np.ascontiguousarray(f) if storage == "f64" else np.ascontiguousarray(f, dtype=np.float32))
    nvp = s.stats()["nv_pad"]
    cdt = torch.float64 if storage == "f64" else torch.float32
    lin = torch.tensor(_pad(lam, nvp), dtype=cdt, device="cuda")
    lout = torch.zeros_like(lin)
    dtg = torch.zeros(4, dtype=torch.float64, device="cuda")
    g.bgk_adjoint_step(s.ctx, 0, lin, lout, dtg)
    s.sync()
    lg = lout.double().cpu().numpy()[..., : M.shape[-1]]
    dg = dtg.cpu().numpy()
    assert np.abs(lg - lam0).max() <= tol * np.abs(lam0).max()
    assert np.abs(dg - dth).max() <= tol * np.abs(dth).max(), (dg, dth)


def test_objective_matches_oracle(g):
    import torch
    p = bi.config("cavity2d_n41_v16_f64", n=21, nv=8)
    cl = bi.cloud_for(p)
    sim = oracle.Simulation(p, cl)
    sim.run(3)
    s = g.Solver([p], [cl])
    s.set_maxwellian()
    s.step(3)
    J = torch.zeros(1, dtype=torch.float64, device="cuda")
    g.bgk_objective(s.ctx, 0, J)
    s.sync()
    Jo = oracle.objective(p, cl["kind"], sim.f)
    assert abs(J.item() - Jo) < 1e-10 * abs(Jo)


@pytest.mark.parametrize("storage,tol", [("f64", 1e-9), ("f32", 2e-4)])
def test_checkpointed_gradient_matches_oracle(g, storage, tol):
    from paper_2408_02350_gb300 import adjoint
    p = bi.config("cavity2d_n41_v16_f64", n=13, nv=8, vmax=4.0, kn=0.1, storage=storage)
    p["lid_u"] = [0.1, 0.0, 0.0]
    cl = bi.cloud_for(p)
    N = 8
    sim = oracle.Simulation(p, cl)
    Jo, dtho, lamo = sim.gradient(N)
    s = g.Solver([p], [cl])
    s.set_maxwellian()
    J, du, dkn, lam0 = adjoint.gradient(s, N, checkpoint_every=3)
    lam0 = lam0.double().cpu().numpy()
    assert abs(J - Jo) <= tol * abs(Jo)
    assert abs(du[0] - dtho[0]) <= tol * abs(dtho[0]), (du, dtho)
    assert abs(dkn - dtho[3]) <= tol * abs(dtho[3]), (dkn, dtho)
    assert np.abs(lam0 - lamo).max() <= tol * np.abs(lamo).max()


def test_adjoint_cavity_1000_steps_against_finite_differences(g):
    # 101^2 points, 24^2 velocities, Kn 0.1, 1000 steps, FP32 forward with checkpoints every 50
    import torch
    from paper_2408_02350_gb300 import adjoint
    p = bi.config("adjoint2d_n101_v24_f32")
    cl = bi.cloud_for(p)
    N = p["steps"]

    def J_of(q):
        s = g.Solver([q], [cl])
        s.set_maxwellian()
        Jd = torch.zeros(1, dtype=torch.float64, device="cuda")
        for _ in range(N):
            s.step(1)
            g.bgk_objective(s.ctx, 0, Jd)
        s.sync()
        s.close()
        return Jd.item() / N

    s32 = g.Solver([p], [cl])
    s32.set_maxwellian()
    J32, du32, dkn32, _ = adjoint.gradient(s32, N, checkpoint_every=50)
    p64 = dict(p, storage="f64")
    s64 = g.Solver([p64], [cl])
    s64.set_maxwellian()
    J64, du64, dkn64, _ = adjoint.gradient(s64, N, checkpoint_every=50)
    eps = 1e-4
    fd_u = (J_of(dict(p64, lid_u=[p["lid_u"][0] + eps, 0, 0])) - J_of(dict(p64, lid_u=[p["lid_u"][0] - eps, 0, 0]))) / (2 * eps)
    fd_k = (J_of(dict(p64, kn=p["kn"] + eps)) - J_of(dict(p64, kn=p["kn"] - eps))) / (2 * eps)
    assert abs(J32 - J64) <= 1e-3 * abs(J64)
    assert abs(du64[0] - fd_u) <= 1e-3 * abs(fd_u), (du64, fd_u)
    assert abs(dkn64 - fd_k) <= 1e-3 * abs(fd_k), (dkn64, fd_k)
    assert abs(du32[0] - fd_u) <= 1e-3 * abs(fd_u), (du32, fd_u)
    assert abs(dkn32 - fd_k) <= 1e-3 * abs(fd_k), (dkn32, fd_k)
    assert abs(du32[0] - du64[0]) <= 1e-3 * abs(du64[0])


@pytest.mark.parametrize("storage", ["f64", "f32"])
def test_autograd_function_gives_the_adjoint_gradient(g, storage):
    # torch.autograd through LidFluxObjective: the gradients equal adjoint.gradient's (the
    # same kernels in the same order: lam0 bit for bit; J and the parameter gradients are
    # sums of per-point terms added by FP64 atomics, whose order varies, so to 1e-12), and
    # (FP64) match central differences in u_lid and Kn and a directional difference in f0
    # to 1e-3
    import torch
    from paper_2408_02350_gb300 import adjoint
    p = bi.config("cavity2d_n41_v16_f64", n=21, nv=8, vmax=4.0, kn=0.1, storage=storage)
    p["lid_u"] = [0.1, 0.0, 0.0]
    cl = bi.cloud_for(p)
    N, K = 12, 5
    sdt = torch.float64 if storage == "f64" else torch.float32
    M = oracle.maxwellian(p, 1.0, (0.0, 0.0, 0.0), 1.0)
    n = len(cl["kind"])
    rng = np.random.default_rng(21)
    f0 = torch.tensor(M[None] * (1.0 + 0.05 * rng.uniform(-1, 1, size=(n,) + M.shape)), dtype=sdt, device="cuda")
    s = g.Solver([p], [cl])
    f0r = f0.clone().requires_grad_(True)
    lid = torch.tensor(0.1, dtype=torch.float64, requires_grad=True)
    kn = torch.tensor(0.1, dtype=torch.float64, requires_grad=True)
    J = adjoint.LidFluxObjective.apply(f0r, lid, kn, s, N, K)
    gf, gl, gk = torch.autograd.grad(J, (f0r, lid, kn))
    # the same gradient through adjoint.gradient on a fresh context
    s2 = g.Solver([p], [cl])
    J2, du, dkn, lam0 = adjoint.gradient(s2, N, checkpoint_every=K, f0=f0)
    assert abs(J.item() - J2) <= 1e-12 * abs(J2)
    assert abs(gl.item() - du[0]) <= 1e-12 * abs(du[0]) and abs(gk.item() - dkn) <= 1e-12 * abs(dkn)
    assert torch.equal(gf, lam0.to(gf.dtype))
    if storage == "f64":
        def J_of(lid_u, knv, f):
            with torch.no_grad():
                return adjoint.LidFluxObjective.apply(f, torch.tensor(lid_u, dtype=torch.float64),
                                                      torch.tensor(knv, dtype=torch.float64), s, N, K).item()
        eps = 1e-4
        fd_u = (J_of(0.1 + eps, 0.1, f0) - J_of(0.1 - eps, 0.1, f0)) / (2 * eps)
        fd_k = (J_of(0.1, 0.1 + eps, f0) - J_of(0.1, 0.1 - eps, f0)) / (2 * eps)
        d = torch.tensor(M[None] * rng.uniform(-1, 1, size=(n,) + M.shape), dtype=sdt, device="cuda")
        fd_f = (J_of(0.1, 0.1, f0 + eps * d) - J_of(0.1, 0.1, f0 - eps * d)) / (2 * eps)
        assert abs(gl.item() - fd_u) <= 1e-3 * abs(fd_u), (gl.item(), fd_u)
        assert abs(gk.item() - fd_k) <= 1e-3 * abs(fd_k), (gk.item(), fd_k)
        gd = float((gf * d).sum())
        assert abs(gd - fd_f) <= 1e-3 * abs(fd_f), (gd, fd_f)
    s.close()
    s2.close()
