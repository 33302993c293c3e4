"""GPU point management (bgk_manage) against the oracle's or_manage.

A jittered cavity with a few close interior pairs and a hole: the GPU pass must
give the oracle's point count, kinds and positions bit for bit (FP64 without fused
multiply-add on both sides), f at the new points to rounding (FP64 storage 1e-12,
FP32 1e-5), and the moments recomputed from f.  Then steps from the managed state
(fixed points and ALE) against the oracle run from the oracle's managed state, the
capacity limit, and two passes in a row.
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


def _cloud(n=31, seed=3, ale=0):
    p = bi.config("cavity2d_n41_v16_f64", n=n, nv=8, vmax=4.0, ale=ale)
    cl = bi.cloud_for(p)
    x = cl["x"].copy()
    dx = 1.0 / (n - 1)
    inner = np.where(cl["kind"] == 0)[0]
    rng = np.random.default_rng(seed)
    for i in rng.choice(inner, size=8, replace=False):
        j = int(np.argmin(np.sum((x - (x[i] + [dx, 0.0])) ** 2, axis=1)))
        if cl["kind"][j] == 0:
            x[j] = x[i] + [0.1 * dx, 0.05 * dx]
    centre = np.array([0.62, 0.38])
    keep = ~((np.sum((x - centre) ** 2, axis=1) < 0.12 ** 2) & (cl["kind"] == 0))
    cl = {"x": x[keep], "kind": cl["kind"][keep], "normal": cl["normal"][keep]}
    return p, cl, 0.25 * dx, 14


def _f0(p, n, seed=4):
    M = oracle.maxwellian(p, 1.0, (0.0, 0.0, 0.0), 1.0)
    rng = np.random.default_rng(seed)
    return M[None] * (1.0 + 0.1 * rng.uniform(-1, 1, size=(n,) + M.shape))


def _oracle_manage(p, cl, f, rmin, mn, cap_out):
    cnt, col = oracle.neighbours(cl["x"], p["h"], False, p["max_nbrs"])
    return oracle.manage(p, cl["x"], cl["kind"], cl["normal"], f, cnt, col, rmin, mn, cap_out)


@pytest.mark.parametrize("storage,tol", [("f64", 1e-12), ("f32", 1e-5)])
def test_manage_matches_oracle(g, storage, tol):
    p, cl, rmin, mn = _cloud()
    p = dict(p, storage=storage, spare_points=64)
    n = len(cl["kind"])
    f = _f0(p, n)
    ref = _oracle_manage(p, cl, f, rmin, mn, n + 64)
    assert ref["merges"] >= 3 and ref["adds"] >= 1
    s = g.Solver([p], [cl])
    s.set_f(np.ascontiguousarray(f) if storage == "f64" else np.ascontiguousarray(f, dtype=np.float32))
    nn, removed, added = s.manage(rmin, mn)
    assert (nn, removed, added) == (len(ref["x"]), ref["merges"] + ref["wall_removals"], ref["adds"])
    assert np.array_equal(s.positions(), ref["x"])
    fg = s.get_f(0, np.float64)
    fo = ref["f"].reshape(fg.shape)
    assert np.abs(fg - fo).max() <= tol * np.abs(fo).max()
    rho, u, T = s.moments()
    ro, uo, To = oracle.moments(p, fo)
    assert np.abs(rho - ro).max() <= 10 * tol * np.abs(ro).max()
    assert np.abs(T - To).max() <= 10 * tol * np.abs(To).max()
    rowptr, col = s.get_neighbours()
    assert len(rowptr) == nn + 1
    s.close()


@pytest.mark.parametrize("ale", [0, 1])
def test_steps_after_manage_match_oracle(g, ale):
    p, cl, rmin, mn = _cloud(ale=ale)
    p = dict(p, storage="f64", spare_points=64)
    n = len(cl["kind"])
    f = _f0(p, n)
    s = g.Solver([p], [cl])
    s.set_f(np.ascontiguousarray(f))
    s.step(5)
    s.sync()
    # the oracle's state after the same 5 steps, then the same management pass
    sim = oracle.Simulation(p, cl, f0=f)
    sim.run(5)
    cl5 = {"x": sim.x, "kind": sim.kind, "normal": sim.normal}
    ref = _oracle_manage(p, cl5, sim.f, rmin, mn, n + 64)
    nn, removed, added = s.manage(rmin, mn)
    assert (nn, removed, added) == (len(ref["x"]), ref["merges"] + ref["wall_removals"], ref["adds"])
    assert np.abs(s.positions() - ref["x"]).max() < 1e-14
    s.step(10)
    s.sync()
    sim2 = oracle.Simulation(p, {"x": ref["x"], "kind": ref["kind"], "normal": ref["normal"]}, f0=ref["f"])
    sim2.run(10)
    rho, u, T = s.moments()
    assert np.abs(rho - sim2.rho).max() < 1e-10 * np.abs(sim2.rho).max()
    assert np.abs(T - sim2.T).max() < 1e-10 * np.abs(sim2.T).max()
    assert np.abs(u - sim2.U).max() < 1e-10 * max(np.abs(sim2.U).max(), 1e-3)
    if ale:
        assert np.abs(s.positions() - sim2.x).max() < 1e-13
    s.close()


def test_capacity_bounds_additions(g):
    p, cl, rmin, mn = _cloud()
    n = len(cl["kind"])
    full = _oracle_manage(p, cl, _f0(p, n), rmin, mn, n + 64)
    assert full["adds"] > 2
    merges = full["merges"] + full["wall_removals"]
    spare = 2
    p = dict(p, storage="f64", spare_points=spare)
    f = _f0(p, n)
    ref = _oracle_manage(p, cl, f, rmin, mn, n + spare)
    s = g.Solver([p], [cl])
    s.set_f(np.ascontiguousarray(f))
    nn, removed, added = s.manage(rmin, mn)
    assert ref["adds"] < full["adds"] and ref["adds"] == min(full["adds"], merges + spare)
    assert (nn, removed, added) == (len(ref["x"]), ref["merges"] + ref["wall_removals"], ref["adds"]) and nn <= n + spare
    assert np.array_equal(s.positions(), ref["x"])
    s.close()


def test_second_pass_after_first(g):
    # the first pass fills part of the hole; the second pass works on the new cloud
    p, cl, rmin, mn = _cloud()
    p = dict(p, storage="f64", spare_points=200)
    n = len(cl["kind"])
    f = _f0(p, n)
    s = g.Solver([p], [cl])
    s.set_f(np.ascontiguousarray(f))
    r1 = _oracle_manage(p, cl, f, rmin, mn, n + 200)
    s.manage(rmin, mn)
    cl1 = {"x": r1["x"], "kind": r1["kind"], "normal": r1["normal"]}
    r2 = _oracle_manage(p, cl1, r1["f"], rmin, mn, n + 200)
    nn, removed, added = s.manage(rmin, mn)
    assert (nn, removed, added) == (len(r2["x"]), r2["merges"] + r2["wall_removals"], r2["adds"])
    assert np.array_equal(s.positions(), r2["x"])
    fg = s.get_f(0, np.float64)
    assert np.abs(fg - r2["f"].reshape(fg.shape)).max() <= 1e-12 * np.abs(r2["f"]).max()
    s.close()


def test_points_next_to_walls_are_removed_as_in_oracle(g):
    p, cl, rmin, mn = _cloud()
    x = cl["x"].copy()
    dx = 1.0 / (p["n"] - 1)
    moved = 0
    for wx in (0.3, 0.5, 0.7):
        w = int(np.argmin(np.sum((x - [wx, 0.0]) ** 2, axis=1)))
        i = int(np.argmin(np.sum((x - [wx, dx]) ** 2, axis=1)))
        if cl["kind"][w] != 0 and cl["kind"][i] == 0:
            x[i] = x[w] + [0.02 * dx, 0.1 * dx]
            moved += 1
    cl = dict(cl, x=x)
    p = dict(p, storage="f64", spare_points=64)
    n = len(cl["kind"])
    f = _f0(p, n)
    ref = _oracle_manage(p, cl, f, rmin, mn, n + 64)
    assert ref["wall_removals"] == moved == 3
    s = g.Solver([p], [cl])
    s.set_f(np.ascontiguousarray(f))
    nn, removed, added = s.manage(rmin, mn)
    assert (nn, removed, added) == (len(ref["x"]), ref["merges"] + ref["wall_removals"], ref["adds"])
    assert np.array_equal(s.positions(), ref["x"])
    fg = s.get_f(0, np.float64)
    assert np.abs(fg - ref["f"].reshape(fg.shape)).max() <= 1e-12 * np.abs(ref["f"]).max()
    s.close()
