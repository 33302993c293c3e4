"""GPU parity of the moving rigid body (Sec. 3.4.1) against the oracle.

A 31^2 cavity with a disc of radius 0.2 moving through the gas under ALE: the body's
points and centre bit for bit (both sides form x + dt u in FP64 without fused
multiply-add), interior positions and moments to rounding (FP64 storage) or to the
FP32 bar, zero mass flux through the moving wall, the guard on points placed inside
the guard sphere, skin lists bit-identical to a full search every step while the
body outruns the gas, point management next to the body, a change of the body
velocity between steps, and a checkpoint that carries the centre.
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


def _case(storage="f64", u=(0.3, 0.1), n=31, nv=8, skin=0.0, **kw):
    p = bi.config("body2d_ale_n201_v32_f32", n=n, nv=nv, vmax=4.0, storage=storage, skin=skin,
                  body_u=list(u) + [0.0], body_radius=0.2, body_centre=[0.45, 0.5, 0.0], **kw)
    return p, bi.cloud_for(p)


def _rel(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


@pytest.mark.parametrize("skin", [0.0, 0.3])
def test_moving_body_matches_oracle_fp64(g, skin):
    p, cl = _case(skin=skin)
    s = g.Solver([p], [cl])
    s.set_maxwellian()
    s.step(12)
    s.sync()
    sim = oracle.Simulation(p, cl)
    sim.run(12)
    x = s.positions()
    body = cl["kind"] == p["body_wall"]
    assert np.array_equal(x[body], sim.x[body])
    assert np.array_equal(s.body_centre(), sim.body_c)
    assert np.abs(x - sim.x).max() < 1e-13
    rho, u, T = s.moments()
    assert _rel(rho, sim.rho) < 1e-10 and _rel(T, sim.T) < 1e-10 and _rel(u, sim.U) < 1e-10
    assert s.stats()["clamps"] == sim.clamps
    s.close()


def test_moving_body_matches_oracle_fp32(g):
    p, cl = _case(storage="f32", skin=0.2)
    s = g.Solver([p], [cl])
    s.set_maxwellian()
    s.step(12)
    s.sync()
    sim = oracle.Simulation(p, cl)
    sim.run(12)
    body = cl["kind"] == p["body_wall"]
    assert np.array_equal(s.positions()[body], sim.x[body])
    rho, u, T = s.moments()
    assert _rel(rho, sim.rho) < 1e-4 and _rel(T, sim.T) < 1e-4 and _rel(u, sim.U) < 1e-4
    s.close()


def test_no_mass_crosses_the_moving_wall_on_the_gpu(g):
    p, cl = _case(u=(-0.5, 0.4))
    s = g.Solver([p], [cl])
    s.set_maxwellian()
    vel = oracle.velocity_grid(2, p["nv"], p["vmax"])
    V = np.array([-0.5, 0.4])
    for _ in range(3):
        s.step(2)
        gb = s.get_f(0, np.float64)[:, 0, :]
        for b in np.where(cl["kind"] == p["body_wall"])[0]:
            c = (vel - V) @ cl["normal"][b]
            assert abs(np.dot(c, gb[b])) <= 1e-13 * np.dot(np.abs(c), gb[b])
    _, u, _ = s.moments()
    body = cl["kind"] == p["body_wall"]
    un = np.sum(u[body] * cl["normal"][body], axis=1)
    assert np.abs(un - cl["normal"][body] @ V).max() < 1e-12
    s.close()


def test_guard_puts_points_back(g):
    # interior points placed inside the guard sphere are put back on it at the first
    # step, on both sides, and counted
    p, cl = _case()
    dx = p["dx"]
    c0 = np.array([0.45, 0.5])
    th = 2 * np.pi * (np.arange(12) + 0.5) / 12
    extra = c0 + (p["body_radius"] + 0.05 * dx) * np.stack([np.cos(th), np.sin(th)], axis=1)
    cl = {"x": np.concatenate([cl["x"], extra]), "kind": np.concatenate([cl["kind"], np.zeros(12, np.int32)]),
          "normal": np.concatenate([cl["normal"], np.zeros((12, 2))])}
    s = g.Solver([p], [cl])
    s.set_maxwellian()
    s.step(3)
    s.sync()
    sim = oracle.Simulation(p, cl)
    sim.run(3)
    assert sim.clamps >= 12 and s.stats()["clamps"] == sim.clamps
    x = s.positions()
    assert np.abs(x - sim.x).max() < 1e-13
    r = np.linalg.norm(x[cl["kind"] == 0] - s.body_centre(), axis=1)
    assert r.min() >= (p["body_radius"] + p["guard"]) * (1 - 1e-14)
    s.close()


def test_skin_lists_follow_a_fast_body(g):
    # at Kn 1 the body moves about 30 % farther than any interior point in 24 steps, so
    # its own displacement decides the rebuilds
    p, cl = _case(storage="f32", u=(0.6, 0.0), nv=6, kn=1.0)

    def run(skin):
        s = g.Solver([dict(p, skin=skin)], [cl])
        s.set_maxwellian()
        s.step(24)
        s.sync()
        out = (s.positions(), s.get_neighbours(), s.get_f(0, np.float32))
        s.close()
        return out

    ref = run(0.0)
    for skin in (0.05, 0.5):
        x, (rp, col), f = run(skin)
        assert np.array_equal(x, ref[0])
        assert np.array_equal(rp, ref[1][0]) and np.array_equal(col, ref[1][1])
        assert np.array_equal(f, ref[2])


def test_manage_next_to_the_body_matches_oracle(g):
    # a body without boundary points inside a hole of radius 0.1: the additions that
    # would land inside its guard sphere (radius 0.08 + guard) are rejected, the rest kept
    p = bi.config("cavity2d_n41_v16_f64", n=41, nv=4, storage="f64", spare_points=200)
    cl = bi.cloud_for(p)
    c = np.array([0.5, 0.5])
    keep = ~((np.linalg.norm(cl["x"] - c, axis=1) < 0.1 + 0.5 * p["dx"]) & (cl["kind"] == 0))
    cl = {"x": cl["x"][keep], "kind": cl["kind"][keep], "normal": cl["normal"][keep]}
    n = len(cl["kind"])
    rng = np.random.default_rng(3)
    M = oracle.maxwellian(p, 1.0, (0.0, 0.0, 0.0), 1.0)
    f = M[None] * (1.0 + 0.1 * rng.uniform(-1, 1, size=(n,) + M.shape))
    cnt, col = oracle.neighbours(cl["x"], p["h"], False, p["max_nbrs"])
    rmin = 0.25 * p["dx"]
    free = oracle.manage(p, cl["x"], cl["kind"], cl["normal"], f, cnt, col, rmin, 14, n + 200)
    p = dict(p, body_wall=6, body_radius=0.08, body_centre=[0.5, 0.5, 0.0], body_u=[0.0, 0.0, 0.0])
    ref = oracle.manage(p, cl["x"], cl["kind"], cl["normal"], f, cnt, col, rmin, 14, n + 200)
    assert 0 < ref["adds"] < free["adds"]
    s = g.Solver([p], [cl])
    s.set_f(np.ascontiguousarray(f))
    nn, removed, added = s.manage(rmin, 14)
    assert (nn, removed, added) == (len(ref["x"]), ref["merges"] + ref["wall_removals"], ref["adds"])
    assert np.array_equal(s.positions(), ref["x"])
    s.close()


def test_body_velocity_change_and_checkpoint(g):
    p, cl = _case(u=(0.3, 0.1))
    s = g.Solver([p], [cl])
    s.set_maxwellian()
    s.step(3)
    blob = g.bgk_get_state(s.ctx)
    q = dict(p, body_u=[-0.2, 0.25, 0.0])
    g.bgk_set_params(s.ctx, 0, q)
    s.step(4)
    s.sync()
    x1, c1 = s.positions(), s.body_centre()
    sim = oracle.Simulation(p, cl)
    sim.run(3)
    sim.q.body_u[0], sim.q.body_u[1] = -0.2, 0.25
    sim.run(4)
    body = cl["kind"] == p["body_wall"]
    assert np.array_equal(x1[body], sim.x[body]) and np.array_equal(c1, sim.body_c)
    assert np.abs(x1 - sim.x).max() < 1e-13
    rho, _, T = s.moments()
    assert _rel(rho, sim.rho) < 1e-10 and _rel(T, sim.T) < 1e-10
    # back to the checkpoint (centre included) and the same 4 steps again
    g.bgk_set_state(s.ctx, blob)
    s.step(4)
    s.sync()
    assert np.array_equal(s.positions(), x1) and np.array_equal(s.body_centre(), c1)
    s.close()


def test_managed_moving_body_run_matches_oracle(g):
    # without management the hole behind a fast body starves the rear wall points of
    # interior neighbours; a pass every 10 steps fills it (additions outside the guard
    # sphere) and the run follows the oracle's managed run
    p, cl = _case(u=(0.6, 0.0), nv=6, spare_points=100)
    rmin, mn = 0.3 * p["dx"], 14
    s = g.Solver([p], [cl])
    s.set_maxwellian()
    sim = oracle.Simulation(p, cl)
    adds = 0
    for _ in range(3):
        s.step(10)
        sim.run(10)
        cnt, col = oracle.neighbours(sim.x, p["h"], False, p["max_nbrs"])
        ref = oracle.manage(sim.p, sim.x, sim.kind, sim.normal, sim.f, cnt, col, rmin, mn)
        nn, removed, added = s.manage(rmin, mn)
        assert (nn, removed, added) == (len(ref["x"]), ref["merges"] + ref["wall_removals"], ref["adds"])
        adds += added
        q = dict(sim.p, body_centre=list(sim.body_c) + [0.0])
        clamps = sim.clamps
        sim = oracle.Simulation(q, {"x": ref["x"], "kind": ref["kind"], "normal": ref["normal"]}, f0=ref["f"])
        sim.clamps = clamps
    assert adds > 0
    s.step(5)
    sim.run(5)
    s.sync()
    assert np.abs(s.positions() - sim.x).max() < 1e-12
    rho, u, T = s.moments()
    assert _rel(rho, sim.rho) < 1e-9 and _rel(T, sim.T) < 1e-9 and _rel(u, sim.U) < 1e-9
    assert np.array_equal(s.body_centre(), sim.body_c)
    s.close()


def test_moving_ball_3d_matches_oracle(g):
    # a ball of boundary points on a Fibonacci sphere in a 3D cavity, FP64
    p = bi.config("cavity3d_n41_v16_f32", n=11, nv=6, vmax=4.0, storage="f64", ale=1, skin=0.3)
    p.update(body_wall=8, body_u=[0.3, -0.2, 0.1], body_radius=0.25, body_centre=[0.5, 0.48, 0.52])
    cl = bi.cloud_for(p)
    assert (cl["kind"] == 8).sum() > 20
    s = g.Solver([p], [cl])
    s.set_maxwellian()
    s.step(5)
    s.sync()
    sim = oracle.Simulation(p, cl)
    sim.run(5)
    body = cl["kind"] == 8
    x = s.positions()
    assert np.array_equal(x[body], sim.x[body]) and np.array_equal(s.body_centre(), sim.body_c)
    assert np.abs(x - sim.x).max() < 1e-13
    rho, u, T = s.moments()
    assert _rel(rho, sim.rho) < 1e-10 and _rel(T, sim.T) < 1e-10 and _rel(u, sim.U) < 1e-10
    assert s.stats()["clamps"] == sim.clamps
    s.close()
