"""Pins of the oracle's moving rigid body (Sec. 3.4.1: boundary points move with the
boundary; diffuse reflection at a moving wall, Sec. 5.1 and 5.2).

The paper states that boundary points move together with a moving boundary and that
walls reflect diffusely; it prints no moving-body result.  The pins check what the
physics fixes: no mass crosses the moving wall, so the gas at a wall point moves
with the wall's normal velocity; the emitted half is a Maxwellian centred on the wall
velocity; the arriving half (classified by the velocity relative to the wall) is the
linear WLS reconstruction, exact on linear fields; the body translates rigidly by
n dt u; interior points are kept outside its guard sphere and put back on it along
the ray from the centre; point management adds no point inside it; a body at rest is
an ordinary wall.
"""
import numpy as np
import pytest

import bgk_inputs as bi
import oracle


def _body_case(n=31, nv=8, u=(0.3, 0.1), ale=1, kn=0.1):
    p = bi.config("body2d_ale_n201_v32_f32", n=n, nv=nv, vmax=4.0, storage="f64", ale=ale, kn=kn,
                  body_u=list(u) + [0.0], body_radius=0.2, body_centre=[0.45, 0.5, 0.0])
    cl = bi.cloud_for(p)
    return p, cl


def _vel(p):
    return oracle.velocity_grid(p["dim"], p["nv"], p["vmax"])


def test_body_at_rest_is_an_ordinary_wall():
    # body velocity 0 and no guard radius: the body path equals plain walls of that kind
    p, cl = _body_case(u=(0.0, 0.0))
    p = dict(p, body_radius=0.0)
    a = oracle.Simulation(p, cl)
    a.run(4)
    q = dict(p, body_wall=0)
    b = oracle.Simulation(q, cl)
    b.run(4)
    assert np.array_equal(a.f, b.f) and np.array_equal(a.x, b.x)
    assert np.array_equal(a.rho, b.rho) and np.array_equal(a.T, b.T)


@pytest.mark.parametrize("u", [(0.3, 0.1), (-0.5, 0.4)])
def test_no_mass_crosses_the_moving_wall(u):
    p, cl = _body_case(u=u)
    sim = oracle.Simulation(p, cl)
    vel = _vel(p)
    V = np.array(u)
    body = np.where(cl["kind"] == p["body_wall"])[0]
    walls = np.where((cl["kind"] != 0) & (cl["kind"] != p["body_wall"]))[0]
    nb = cl["normal"]
    for _ in range(3):
        sim.run(1)
        g = sim.f[:, 0, :]
        # relative normal velocity (v - V).n: the net flux vanishes at every body point
        for b in body:
            c = (vel - V) @ nb[b]
            flux = np.dot(c, g[b])
            assert abs(flux) <= 1e-13 * np.dot(np.abs(c), g[b])
            # so the gas at the wall point moves with the wall's normal velocity
            assert abs(np.dot(sim.U[b], nb[b]) - np.dot(V, nb[b])) < 1e-13
        for b in walls:
            c = vel @ nb[b]
            assert abs(np.dot(c, g[b])) <= 1e-13 * np.dot(np.abs(c), g[b])


def test_moving_wall_halves():
    # interior f linear in x for every velocity: after the boundary step, the body
    # point's arriving half ((v - V).n <= 0) is that linear field at the wall point and
    # the emitted half is rho_w M(v; 1, V, T_w) (h = T_w g there)
    p, cl = _body_case(u=(0.6, -0.2), ale=0)
    x, kind, normal = cl["x"], cl["kind"], cl["normal"]
    cnt, col = oracle.neighbours(x, p["h"], False, p["max_nbrs"])
    st = oracle.stencils(p, x, kind, cnt, col)
    NV = p["nv"] ** 2
    rng = np.random.default_rng(7)
    a = rng.uniform(1.0, 2.0, size=(2, NV))
    bvec = rng.uniform(-0.5, 0.5, size=(2, NV, 2))
    f = a[None] + np.einsum("qkd,nd->nqk", bvec, x)
    n = len(x)
    rho, U, T = np.ones(n), np.zeros((n, 2)), np.ones(n)
    assert oracle.boundary(p, kind, normal, cnt, col, st, f, rho, U, T) == 0
    vel = _vel(p)
    V = np.array(p["body_u"][:2])
    Mw = oracle.maxwellian(p, 1.0, V, p["wall_T"])
    body = np.where(kind == p["body_wall"])[0]
    both = 0
    for b in body:
        c = (vel - V) @ normal[b]
        arr, emit = c <= 0.0, c > 0.0
        both += int(np.sum(arr & (vel @ normal[b] > 0.0)))
        lin = a[:, arr] + bvec[:, arr, :] @ x[b]
        assert np.abs(f[b][:, arr] - lin).max() < 1e-12 * np.abs(lin).max()
        ratio = f[b][0, emit] / Mw[0, emit]
        assert np.ptp(ratio) < 1e-12 * ratio.mean()
        assert np.allclose(f[b][1, emit], p["wall_T"] * f[b][0, emit], rtol=1e-15, atol=0)
    # velocities that leave the wall in the absolute frame but arrive in the wall's frame
    assert both > 0


def test_body_translates_rigidly():
    p, cl = _body_case(u=(0.3, 0.1))
    sim = oracle.Simulation(p, cl)
    nsteps = 6
    sim.run(nsteps)
    body = cl["kind"] == p["body_wall"]
    disp = nsteps * p["dt"] * np.array([0.3, 0.1])
    assert np.abs(sim.x[body] - cl["x"][body] - disp).max() < 1e-15
    assert np.abs(sim.body_c - (np.array([0.45, 0.5]) + disp)).max() < 1e-15
    d0 = np.linalg.norm(cl["x"][body][:, None] - cl["x"][body][None], axis=2)
    d1 = np.linalg.norm(sim.x[body][:, None] - sim.x[body][None], axis=2)
    assert np.abs(d1 - d0).max() < 1e-15
    # the cavity walls stay put
    wall = (cl["kind"] != 0) & ~body
    assert np.array_equal(sim.x[wall], cl["x"][wall])


def test_guard_puts_points_back_on_the_sphere():
    p, cl = _body_case(u=(0.3, 0.1))
    x = cl["x"].copy()
    kind = cl["kind"]
    inner = kind == 0
    c0 = np.array(p["body_centre"][:2])
    # every interior point drifts towards the body centre by 0.3 of its distance
    U = np.zeros_like(x)
    U[inner] = -0.3 * (x[inner] - c0) / p["dt"]
    y = x + p["dt"] * U  # unguarded targets (bitwise as the oracle forms them)
    q = dict(p)
    nclamp = oracle.move(q, kind, U, x)
    c1 = c0 + p["dt"] * np.array([0.3, 0.1])
    assert np.abs(np.array(q["body_centre"][:2]) - c1).max() < 1e-16
    rg = p["body_radius"] + p["guard"]
    r_y = np.linalg.norm(y - c1, axis=1)
    inside = inner & (r_y < rg)
    assert inside.sum() > 10 and nclamp == inside.sum()
    r_x = np.linalg.norm(x - c1, axis=1)
    assert np.all(r_x[inner] >= rg * (1 - 1e-15))
    assert np.abs(r_x[inside] - rg).max() < 1e-15
    # put back along the ray from the centre
    d0, d1 = y[inside] - c1, x[inside] - c1
    cross = d0[:, 0] * d1[:, 1] - d0[:, 1] * d1[:, 0]
    assert np.abs(cross).max() < 1e-15 and np.all(np.sum(d0 * d1, axis=1) > 0)
    assert np.array_equal(x[inner & ~inside], y[inner & ~inside])


def test_manage_adds_no_point_inside_the_body():
    # a body without boundary points over a hole in the lattice: the rim points' new
    # points would go into the hole, which the body's guard sphere covers
    p = bi.config("cavity2d_n41_v16_f64", n=41, nv=4)
    cl = bi.cloud_for(p)
    c = np.array([0.5, 0.5])
    R = 0.1
    keep = ~((np.linalg.norm(cl["x"] - c, axis=1) < R + 0.5 * p["dx"]) & (cl["kind"] == 0))
    x, kind, normal = cl["x"][keep], cl["kind"][keep], cl["normal"][keep]
    cnt, col = oracle.neighbours(x, p["h"], False, p["max_nbrs"])
    f = np.ones((len(x), 2, 16))
    rmin = 0.25 * p["dx"]
    free = oracle.manage(p, x, kind, normal, f, cnt, col, rmin, 14)
    new = free["x"][free["origin"] < 0]
    assert np.sum(np.linalg.norm(new - c, axis=1) < R + p["guard"]) > 0
    pb = dict(p, body_wall=6, body_radius=R, body_centre=[0.5, 0.5, 0.0], body_u=[0.0, 0.0, 0.0])
    out = oracle.manage(pb, x, kind, normal, f, cnt, col, rmin, 14)
    new_b = out["x"][out["origin"] < 0]
    assert np.all(np.linalg.norm(new_b - c, axis=1) >= R + p["guard"])
    # exactly the additions outside the guard sphere remain, in the same order
    outside = np.linalg.norm(new - c, axis=1) >= R + p["guard"]
    assert np.array_equal(new_b, new[outside])
