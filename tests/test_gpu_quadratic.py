"""GPU parity of the second-order (quadratic) WLS stencils (Sec. 3.4.1, higher-order Taylor
expansion) against the oracle: the projected coefficients to rounding (FP64 solve on both
sides), the exact gradient of a quadratic from the GPU's own coefficients at a larger size,
and steps with the quadratic stencils (fixed points and ALE, FP64 and FP32) against the
oracle's.
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


def _name(dim):
    return "cavity2d_n41_v16_f64" if dim == 2 else "cavity3d_n41_v16_f32"


def _rel(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


@pytest.mark.parametrize("dim,n,storage,tol", [(2, 21, "f64", 1e-11), (3, 9, "f64", 1e-11), (2, 21, "f32", 1e-6)])
def test_quadratic_stencils_match(g, dim, n, storage, tol):
    p = bi.config(_name(dim), n=n, nv=4, storage=storage, wls_order=2)
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
            assert np.abs(P[k:k + m] - Po).max() <= tol * np.abs(Po).max(), i
        else:
            assert np.abs(R[k:k + m] - st["recon"][i, :m]).max() <= tol * max(1.0, np.abs(st["recon"][i]).max())
        k += m
    s.close()


def test_gpu_quadratic_gradient_is_exact(g):
    # sum_d P_d = coef_j; the gradient of q = a + b.x + x^T H x / 2 from the GPU's
    # coefficients equals b + H x_i at every interior point of a 61^2 jittered cavity
    p = bi.config("cavity2d_n41_v16_f64", n=61, nv=4, storage="f64", wls_order=2)
    cl = bi.cloud_for(p)
    s = g.Solver([p], [cl])
    s.neighbours()
    s.sync()
    rowptr, col = s.get_neighbours()
    P, _ = s.get_stencils()
    coef = P.sum(axis=1)
    rng = np.random.default_rng(5)
    b = rng.uniform(-1, 1, 2)
    H = rng.uniform(-2, 2, (2, 2))
    H = H + H.T
    x = cl["x"]
    q = 0.2 + x @ b + 0.5 * np.einsum("ni,ij,nj->n", x, H, x)
    worst = 0.0
    for i in np.where(cl["kind"] == 0)[0]:
        sl = slice(rowptr[i], rowptr[i + 1])
        grad = (coef[sl] * (q[col[sl]] - q[i])[:, None]).sum(0)
        worst = max(worst, np.abs(grad - (b + H @ x[i])).max())
    assert worst < 1e-9
    s.close()


@pytest.mark.parametrize("dim,n,nv,ale,storage,steps,tol", [
    (2, 21, 8, 0, "f64", 20, 1e-10), (2, 21, 8, 1, "f64", 10, 1e-10), (3, 7, 5, 0, "f64", 4, 1e-10),
    (2, 21, 8, 0, "f32", 20, 1e-4), (2, 21, 8, 1, "f32", 10, 1e-4)])
def test_quadratic_steps_match_oracle(g, dim, n, nv, ale, storage, steps, tol):
    p = bi.config(_name(dim), n=n, nv=nv, vmax=4.0, storage=storage, ale=ale, wls_order=2)
    cl = bi.cloud_for(p)
    sim = oracle.Simulation(p, cl)
    sim.run(steps)
    s = g.Solver([p], [cl])
    s.set_maxwellian()
    s.step(steps)
    s.sync()
    rho, u, T = s.moments()
    assert _rel(rho, sim.rho) < tol and _rel(T, sim.T) < tol and _rel(u, sim.U) < max(tol, 1e-12)
    if ale:
        assert np.abs(s.positions() - sim.x).max() < (1e-13 if storage == "f64" else 1e-7)
    s.close()


@pytest.mark.parametrize("dim,n,nv,ale,storage,steps,tol", [
    (2, 21, 8, 0, "f64", 10, 1e-10), (2, 21, 8, 1, "f64", 10, 1e-10), (3, 7, 6, 0, "f64", 10, 1e-10),
    (2, 21, 8, 0, "f32", 10, 1e-4), (2, 21, 8, 1, "f32", 10, 1e-4), (3, 7, 6, 0, "f32", 10, 1e-4)])
def test_negative_normal_coefficients_match_oracle(g, dim, n, nv, ale, storage, steps, tol):
    # Sec. 3.4.1 / 3.4.2 on a cloud jittered by 0.45 dx, where the second-order fit gives
    # negative projected normal coefficients abar_n (asserted on the oracle's stencils):
    # both sides use abar_d c_d - |abar_d||c_d| for every direction.
    p = bi.config(_name(dim), n=n, nv=nv, vmax=4.0, storage=storage, ale=ale, wls_order=2)
    cl = bi.cavity(dim, n, 2408011, 0.45)
    cnt, col = oracle.neighbours(cl["x"], p["h"], False, p["max_nbrs"])
    st = oracle.stencils(p, cl["x"], cl["kind"], cnt, col)
    interior = cl["kind"] == 0
    assert sum((st["abar"][i, :cnt[i], 0] < 0).sum() for i in np.where(interior)[0]) > 0
    sim = oracle.Simulation(p, cl)
    sim.run(steps)
    s = g.Solver([p], [cl])
    s.set_maxwellian()
    s.step(steps)
    s.sync()
    rho, u, T = s.moments()
    assert _rel(rho, sim.rho) < tol and _rel(T, sim.T) < tol and _rel(u, sim.U) < tol
    f = s.get_f()
    assert np.abs(f - sim.f).max() < tol * np.abs(sim.f).max()
    if ale:
        assert np.abs(s.positions() - sim.x).max() < (1e-13 if storage == "f64" else 1e-7)
    s.close()
