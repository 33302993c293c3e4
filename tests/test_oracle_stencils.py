"""Pins of the oracle's neighbour search and weighted-least-squares stencils.

Neighbours: the cell search equals the O(n^2) definition; the relation is
symmetric; lattice counts match the integer-point count of a disc or ball.
Stencils: the WLS gradient reproduces linear functions exactly (and its
coefficients satisfy sum_j coef_j dr_j^T = I); the wall reconstruction
reproduces linear functions; the local frames are orthonormal, follow dr and
the paper's angle conventions; the projected coefficient along n is positive.
"""
import numpy as np
import pytest

import bgk_inputs as bi
import oracle


def _cloud(dim, n, seed, jitter=0.1):
    return bi.cavity(dim, n, seed, jitter)


def _random_cloud(dim, n, seed):
    return bi.uniform01(seed, n * dim).reshape(n, dim)


@pytest.mark.parametrize("dim,n,periodic,h", [
    (2, 41, False, 2.5 / 40), (3, 9, False, 2.5 / 8), (2, 0, False, 0.05), (3, 0, False, 0.12),
    (2, 0, True, 0.05), (3, 0, True, 0.2), (2, 0, True, 0.45), (3, 0, True, 0.4)])
def test_cell_search_equals_brute_force(dim, n, periodic, h):
    if n:
        x = _cloud(dim, n, 77)["x"]
    else:
        x = _random_cloud(dim, 900 if dim == 2 else 700, 1234 + dim)
    cap = 1000
    c1, l1 = oracle.neighbours(x, h, periodic, cap, "cells")
    c2, l2 = oracle.neighbours(x, h, periodic, cap, "brute")
    assert np.array_equal(c1, c2) and np.array_equal(l1, l2)
    # ascending, no self
    for i in range(len(c1)):
        row = l1[i, : c1[i]]
        assert np.all(np.diff(row) > 0) and i not in row


def test_neighbour_relation_is_symmetric():
    x = _cloud(2, 30, 5)["x"]
    cnt, col = oracle.neighbours(x, 2.5 / 29, False, 48)
    pairs = {(i, int(j)) for i in range(len(cnt)) for j in col[i, : cnt[i]]}
    assert all((j, i) in pairs for (i, j) in pairs)


@pytest.mark.parametrize("dim,expect", [(2, 20), (3, 80)])
def test_lattice_counts_match_integer_points_in_ball(dim, expect):
    # |a|^2 <= 6.25 over integer vectors a != 0: 20 in 2D, 80 in 3D.
    r = np.arange(-3, 4)
    grid = np.stack(np.meshgrid(*([r] * dim)), -1).reshape(-1, dim)
    assert ((grid ** 2).sum(1) <= 6.25).sum() - 1 == expect
    n = 11 if dim == 2 else 9
    c = _cloud(dim, n, 1, jitter=0.0)
    cnt, _ = oracle.neighbours(c["x"], 2.5 * c["dx"], False, 200)
    idx = np.indices((n,) * dim).reshape(dim, -1)[::-1].T
    far = np.all((idx >= 3) & (idx <= n - 4), axis=1)
    assert far.any() and np.all(cnt[far] == expect)


def test_overflow_is_reported():
    x = _cloud(2, 21, 3)["x"]
    with pytest.raises(OverflowError):
        oracle.neighbours(x, 2.5 / 20, False, 8)


def _stencil_case(dim, n, seed=11, jitter=0.1):
    name = "cavity2d_n41_v16_f64" if dim == 2 else "cavity3d_n41_v16_f32"
    p = bi.config(name, n=n, nv=4)
    c = bi.cavity(dim, n, seed, jitter)
    cnt, col = oracle.neighbours(c["x"], p["h"], False, p["max_nbrs"])
    st = oracle.stencils(p, c["x"], c["kind"], cnt, col)
    return p, c, cnt, col, st


def _dr(c, i, col, cnt):
    return c["x"][col[i, : cnt[i]]] - c["x"][i]


@pytest.mark.parametrize("dim,n", [(2, 15), (3, 7)])
def test_gradient_reproduces_linear_functions(dim, n):
    # Eqs. (x_derivative)-(z_derivative): for f = a + b.x the WLS gradient is b exactly,
    # so sum_j coef_j dr_j^T = I.
    p, c, cnt, col, st = _stencil_case(dim, n)
    b = np.array([0.7, -1.3, 2.1])[:dim]
    fval = 0.4 + c["x"] @ b
    for i in np.where(c["kind"] == 0)[0]:
        k = cnt[i]
        coef = st["coef"][i, :k]
        dr = _dr(c, i, col, cnt)
        assert np.allclose(coef.T @ dr, np.eye(dim), atol=1e-11)
        grad = (coef * (fval[col[i, :k]] - fval[i])[:, None]).sum(0)
        assert np.allclose(grad, b, atol=1e-11)


@pytest.mark.parametrize("dim,n", [(2, 15), (3, 7)])
def test_wall_reconstruction_reproduces_linear_functions(dim, n):
    p, c, cnt, col, st = _stencil_case(dim, n)
    b = np.array([0.3, 0.9, -0.6])[:dim]
    fval = 1.1 + c["x"] @ b
    nconst = 0
    for i in np.where(c["kind"] != 0)[0]:
        k = cnt[i]
        nb = col[i, :k]
        r = st["recon"][i, :k]
        inner = c["kind"][nb] == 0
        assert np.all(r[~inner] == 0.0)
        assert abs(r.sum() - 1.0) < 1e-12
        if inner.sum() >= dim + 1:
            dr = _dr(c, i, col, cnt)
            assert np.allclose((r[:, None] * dr).sum(0), 0.0, atol=1e-13)
            assert abs((r * fval[nb]).sum() - fval[i]) < 1e-12
        else:
            nconst += 1
            assert np.all(r[inner] > 0)
    assert dim == 3 or nconst == 0


def test_frames_2d_follow_the_angle_convention():
    # Sec. 3.4.2: n = (cos phi, sin phi), t = (-sin phi, cos phi), phi = atan2(dy, dx).
    rng = np.random.default_rng(0)
    for dr in list(rng.normal(size=(50, 2))) + [np.array([1.0, 0.0]), np.array([0.0, -2.0]), np.array([-1.0, 1e-300])]:
        F = oracle.frame(2, dr)
        n = dr / np.linalg.norm(dr)
        assert np.allclose(F[0], n, atol=1e-15)
        assert np.allclose(F[1], [-n[1], n[0]], atol=1e-15)


def test_frames_3d_are_right_handed_and_follow_the_angles():
    # Sec. 3.4.2: rows n, t, b of A from phi = atan2(dy, dx), theta = arccos(dz / r).
    rng = np.random.default_rng(1)
    cases = list(rng.normal(size=(100, 3))) + [np.array([0.0, 0.0, 1.0]), np.array([0.0, 0.0, -3.0]),
                                              np.array([1.0, 0.0, 0.0]), np.array([0.0, 2.0, 0.0])]
    for dr in cases:
        F = oracle.frame(3, dr)
        assert np.allclose(F @ F.T, np.eye(3), atol=1e-14)
        assert np.allclose(F[0], dr / np.linalg.norm(dr), atol=1e-14)
        assert np.allclose(np.cross(F[0], F[1]), F[2], atol=1e-14)
        assert F[2, 2] == 0.0
        rxy = np.hypot(dr[0], dr[1])
        cphi, sphi = (dr[0] / rxy, dr[1] / rxy) if rxy > 0 else (1.0, 0.0)
        assert np.allclose(F[2], [-sphi, cphi, 0.0], atol=1e-14)
    F = oracle.frame(3, np.array([0.0, 0.0, 1.0]))
    assert np.allclose(F, [[0, 0, 1], [1, 0, 0], [0, 1, 0]], atol=1e-15)


@pytest.mark.parametrize("dim,n", [(2, 15), (3, 7)])
def test_projected_coefficients(dim, n):
    # abar = (frame rows) . coef: abar_n = w r n^T S n > 0 (the paper's first term needs no sign);
    # the frame is orthonormal, so sum_d abar_d e_d = coef.
    p, c, cnt, col, st = _stencil_case(dim, n)
    for i in np.where(c["kind"] == 0)[0]:
        k = cnt[i]
        ab, F, coef = st["abar"][i, :k], st["frame"][i, :k], st["coef"][i, :k]
        assert np.all(ab[:, 0] > 0)
        assert np.allclose(np.einsum("kd,kda->ka", ab, F), coef, atol=1e-12 * np.abs(coef).max())


def test_unjittered_lattice_has_no_tangential_coefficient():
    # On a centrally symmetric neighbourhood coef_j is parallel to dr_j, so abar_t = abar_b = 0.
    p, c, cnt, col, st = _stencil_case(3, 9, jitter=0.0)
    idx = np.indices((9,) * 3).reshape(3, -1)[::-1].T
    far = np.where(np.all((idx >= 3) & (idx <= 5), axis=1))[0]
    for i in far:
        assert np.abs(st["abar"][i, : cnt[i], 1:]).max() < 1e-10 * st["abar"][i, : cnt[i], 0].max()


def _quad_case(dim, n, order, seed=11):
    name = "cavity2d_n41_v16_f64" if dim == 2 else "cavity3d_n41_v16_f32"
    p = bi.config(name, n=n, nv=4, wls_order=order)
    c = bi.cavity(dim, n, seed, 0.1)
    cnt, col = oracle.neighbours(c["x"], p["h"], False, p["max_nbrs"])
    st = oracle.stencils(p, c["x"], c["kind"], cnt, col)
    return p, c, cnt, col, st


@pytest.mark.parametrize("dim,n", [(2, 15), (3, 7)])
def test_quadratic_fit_gradient_is_exact_on_quadratics(dim, n):
    # Sec. 3.4.1: the higher-order Taylor expansion.  For q = a + b.x + x^T H x / 2 the
    # second-order fit's gradient rows give grad q(x_i) = b + H x_i exactly; the linear
    # fit's carry an O(h) error, which the test must see.
    rng = np.random.default_rng(3)
    b = rng.uniform(-1, 1, dim)
    H = rng.uniform(-2, 2, (dim, dim))
    H = H + H.T
    _, c, cnt, col, st2 = _quad_case(dim, n, 2)
    _, _, _, _, st1 = _quad_case(dim, n, 1)
    q = 0.3 + c["x"] @ b + 0.5 * np.einsum("ni,ij,nj->n", c["x"], H, c["x"])
    err1 = 0.0
    for i in np.where(c["kind"] == 0)[0]:
        k = cnt[i]
        exact = b + H @ c["x"][i]
        dq = q[col[i, :k]] - q[i]
        g2 = (st2["coef"][i, :k] * dq[:, None]).sum(0)
        assert np.abs(g2 - exact).max() < 1e-10 * max(1.0, np.abs(exact).max())
        # linear functions stay exact too: sum_j coef_j dr_j^T = I
        assert np.allclose(st2["coef"][i, :k].T @ _dr(c, i, col, cnt), np.eye(dim), atol=1e-11)
        g1 = (st1["coef"][i, :k] * dq[:, None]).sum(0)
        err1 = max(err1, np.abs(g1 - exact).max())
    assert err1 > 1e-4


@pytest.mark.parametrize("dim,n", [(2, 15), (3, 7)])
def test_quadratic_fit_projected_coefficients(dim, n):
    # the same frame construction as the linear fit: abar_d = e_d . coef_j and
    # sum_d abar_d e_d = coef_j
    _, c, cnt, col, st = _quad_case(dim, n, 2)
    for i in np.where(c["kind"] == 0)[0][:40]:
        for s in range(cnt[i]):
            fr = st["frame"][i, s]
            assert np.allclose(fr @ st["coef"][i, s], st["abar"][i, s], atol=1e-12)
            assert np.allclose(fr.T @ st["abar"][i, s], st["coef"][i, s], atol=1e-12)
