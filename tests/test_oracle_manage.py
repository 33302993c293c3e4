"""Pins of the oracle's point management (Sec. 3.5.2: removing and adding points).

The paper names the two operations (two points that come too close are replaced
by one at their midpoint; points are added where holes open) and says f at new
points comes from least squares, without thresholds.  The pins check what those
statements fix: a regular lattice is left alone, a close pair becomes its
midpoint and nothing else changes, only mutually nearest points pair up, the
least-squares value reproduces any linear field exactly at every new position,
a hole receives points inside it and away from the existing ones, the output
capacity bounds the additions, and periodic pairs merge across the box edge.
"""
import numpy as np

import bgk_inputs as bi
import oracle


def _setup(n=21, nv=4, jitter=0.0, periodic=False, seed=5):
    if periodic:
        cl = bi.periodic_box(2, n, seed=seed, jitter=jitter)
        p = {"dim": 2, "nv": nv, "vmax": 3.0, "kn": 0.1, "tau_mode": 0, "h": 2.5 / n, "alpha": 6.25, "wall_T": 1.0,
             "max_nbrs": 48, "periodic": 1, "guard": 0.0, "dt": 0.01}
    else:
        p = bi.config("cavity2d_n41_v16_f64", n=n, nv=nv)
        cl = bi.cloud_for(p)
        if jitter == 0.0:
            # unjittered lattice of the same cavity
            dx = 1.0 / (n - 1)
            idx = np.rint(cl["x"] / dx)
            cl = dict(cl, x=idx * dx)
    return p, cl


def _lists(p, x):
    return oracle.neighbours(x, p["h"], bool(p.get("periodic")), p["max_nbrs"])


def _linear_f(x, nrow, seed=1):
    # f_q(x) = a_q + b_q . x, one random linear field per row entry q
    rng = np.random.default_rng(seed)
    a = rng.uniform(1.0, 2.0, size=nrow)
    b = rng.uniform(-1.0, 1.0, size=(nrow, x.shape[1]))
    return a[None, :] + x @ b.T, a, b


def _f_shape(p):
    return (2, p["nv"] ** 2) if p["dim"] == 2 else (1, p["nv"] ** 3)


def test_regular_lattice_is_left_alone():
    p, cl = _setup()
    x = cl["x"]
    cnt, col = _lists(p, x)
    rng = np.random.default_rng(0)
    f = rng.uniform(0.5, 1.5, size=(len(x),) + _f_shape(p))
    dx = 1.0 / (p["n"] - 1)
    out = oracle.manage(p, x, cl["kind"], cl["normal"], f, cnt, col, 0.25 * dx, 10)
    assert out["merges"] == 0 and out["adds"] == 0
    assert np.array_equal(out["x"], x) and np.array_equal(out["f"], f)
    assert np.array_equal(out["origin"], np.arange(len(x)))
    assert np.array_equal(out["kind"], cl["kind"])


def test_close_pair_becomes_its_midpoint():
    p, cl = _setup()
    x = cl["x"].copy()
    dx = 1.0 / (p["n"] - 1)
    inner = np.where(cl["kind"] == 0)[0]
    i = inner[len(inner) // 2]
    # the interior point to the right of i, moved to 0.1 dx from i
    j = int(np.argmin(np.sum((x - (x[i] + [dx, 0.0])) ** 2, axis=1)))
    assert cl["kind"][j] == 0
    x[j] = x[i] + [0.1 * dx, 0.0]
    cnt, col = _lists(p, x)
    rng = np.random.default_rng(1)
    f = rng.uniform(0.5, 1.5, size=(len(x),) + _f_shape(p))
    out = oracle.manage(p, x, cl["kind"], cl["normal"], f, cnt, col, 0.25 * dx, 0)
    assert out["merges"] == 1 and out["adds"] == 0 and len(out["x"]) == len(x) - 1
    keep = np.array([k for k in range(len(x)) if k != max(i, j)])
    assert np.array_equal(out["origin"], keep)
    s = min(i, j)
    assert np.allclose(out["x"][s], 0.5 * (x[i] + x[j]), rtol=0, atol=1e-16)
    others = keep != s
    assert np.array_equal(out["x"][others], x[keep[others]])
    assert np.array_equal(out["f"][others], f[keep[others]])


def test_only_mutually_nearest_points_pair():
    p, cl = _setup()
    x = cl["x"].copy()
    dx = 1.0 / (p["n"] - 1)
    inner = np.where(cl["kind"] == 0)[0]
    a = inner[len(inner) // 2]
    # b and c on the line through a: |ab| = 0.05 dx, |bc| = 0.08 dx
    right = [int(np.argmin(np.sum((x - (x[a] + [k * dx, 0.0])) ** 2, axis=1))) for k in (1, 2)]
    b, c = right
    x[b] = x[a] + [0.05 * dx, 0.0]
    x[c] = x[a] + [0.13 * dx, 0.0]
    cnt, col = _lists(p, x)
    f = np.ones((len(x),) + _f_shape(p))
    out = oracle.manage(p, x, cl["kind"], cl["normal"], f, cnt, col, 0.25 * dx, 0)
    assert out["merges"] == 1
    assert c in out["origin"] and min(a, b) in out["origin"] and max(a, b) not in out["origin"]
    assert np.array_equal(out["x"][list(out["origin"]).index(c)], x[c])


def test_new_points_reproduce_linear_fields():
    p, cl = _setup(n=31)
    x = cl["x"].copy()
    dx = 1.0 / (p["n"] - 1)
    inner = np.where(cl["kind"] == 0)[0]
    rng = np.random.default_rng(2)
    # a few close pairs and a hole
    for i in rng.choice(inner, size=6, replace=False):
        j = int(np.argmin(np.sum((x - (x[i] + [0.0, dx])) ** 2, axis=1)))
        if cl["kind"][j] == 0:
            x[j] = x[i] + [0.0, 0.12 * dx]
    centre = np.array([0.3, 0.6])
    hole = (np.sum((x - centre) ** 2, axis=1) < (0.12) ** 2) & (cl["kind"] == 0)
    keep = ~hole
    x, kind, normal = x[keep], cl["kind"][keep], cl["normal"][keep]
    cnt, col = _lists(p, x)
    nrow = int(np.prod(_f_shape(p)))
    flin, a, b = _linear_f(x, nrow)
    f = flin.reshape((len(x),) + _f_shape(p))
    out = oracle.manage(p, x, kind, normal, f, cnt, col, 0.25 * dx, 14)
    assert out["merges"] >= 3 and out["adds"] >= 1
    new = out["origin"] < 0
    moved = np.zeros(len(out["x"]), dtype=bool)
    for k, o in enumerate(out["origin"]):
        if o >= 0 and not np.array_equal(out["x"][k], x[o]):
            moved[k] = True
    assert moved.sum() == out["merges"]
    for sel in (new, moved):
        y = out["x"][sel]
        expect = a[None, :] + y @ b.T
        got = out["f"][sel].reshape(len(y), nrow)
        assert np.abs(got - expect).max() < 1e-12 * np.abs(expect).max()


def test_hole_receives_points_inside_it():
    p, cl = _setup(n=41)
    x = cl["x"]
    dx = 1.0 / (p["n"] - 1)
    centre, rad = np.array([0.5, 0.5]), 0.1
    keep = ~((np.sum((x - centre) ** 2, axis=1) < rad ** 2) & (cl["kind"] == 0))
    x, kind, normal = x[keep], cl["kind"][keep], cl["normal"][keep]
    cnt, col = _lists(p, x)
    f = np.ones((len(x),) + _f_shape(p))
    rmin = 0.25 * dx
    out = oracle.manage(p, x, kind, normal, f, cnt, col, rmin, 14)
    assert out["adds"] > 0
    y = out["x"][out["origin"] < 0]
    # every new point is inside the hole's rim (closer to the centre than the hole radius plus h)
    assert np.all(np.sqrt(np.sum((y - centre) ** 2, axis=1)) < rad)
    # and at least rmin away from every old point
    d2 = np.sum((y[:, None, :] - x[None, :, :]) ** 2, axis=2)
    assert d2.min() >= rmin ** 2
    # the largest empty circle in the hole shrinks: farthest hole sample from any point
    g = centre + rad * 0.9 * np.stack(np.meshgrid(np.linspace(-1, 1, 21), np.linspace(-1, 1, 21)), -1).reshape(-1, 2)
    g = g[np.sum((g - centre) ** 2, axis=1) < (0.9 * rad) ** 2]
    before = np.sqrt(np.min(np.sum((g[:, None] - x[None]) ** 2, axis=2), axis=1)).max()
    after = np.sqrt(np.min(np.sum((g[:, None] - out["x"][None]) ** 2, axis=2), axis=1)).max()
    assert after < before


def test_capacity_bounds_additions():
    p, cl = _setup(n=41)
    x = cl["x"]
    centre, rad = np.array([0.5, 0.5]), 0.1
    keep = ~((np.sum((x - centre) ** 2, axis=1) < rad ** 2) & (cl["kind"] == 0))
    x, kind, normal = x[keep], cl["kind"][keep], cl["normal"][keep]
    cnt, col = _lists(p, x)
    f = np.ones((len(x),) + _f_shape(p))
    dx = 1.0 / (p["n"] - 1)
    full = oracle.manage(p, x, kind, normal, f, cnt, col, 0.25 * dx, 14)
    lim = oracle.manage(p, x, kind, normal, f, cnt, col, 0.25 * dx, 14, cap_out=len(x) + 2)
    assert full["adds"] > 2 and lim["adds"] == 2 and len(lim["x"]) == len(x) + 2
    assert np.array_equal(lim["x"], full["x"][: len(x) + 2])


def test_periodic_pair_merges_across_the_edge():
    p, cl = _setup(n=15, periodic=True)
    x = cl["x"].copy()
    dx = 1.0 / 15
    # two points on the same row, one at x = 0.01 dx, one at x = 1 - 0.02 dx
    row = np.where(np.isclose(x[:, 1], 7 * dx))[0]
    i = row[np.argmin(x[row, 0])]
    j = row[np.argmax(x[row, 0])]
    x[i, 0] = 0.01 * dx
    x[j, 0] = 1.0 - 0.02 * dx
    cnt, col = _lists(p, x)
    f = np.ones((len(x),) + _f_shape(p))
    out = oracle.manage(p, x, cl["kind"], cl["normal"], f, cnt, col, 0.25 * dx, 0)
    assert out["merges"] == 1
    s = list(out["origin"]).index(min(i, j))
    xm = out["x"][s, 0]
    assert abs(xm - (1.0 - 0.005 * dx)) < 1e-15 and abs(out["x"][s, 1] - 7 * dx) < 1e-15


def test_point_next_to_a_wall_is_removed():
    p, cl = _setup()
    x = cl["x"].copy()
    dx = 1.0 / (p["n"] - 1)
    # the interior point next to the wall point at (0.5, 0), moved to 0.1 dx above it
    w = int(np.argmin(np.sum((x - [0.5, 0.0]) ** 2, axis=1)))
    i = int(np.argmin(np.sum((x - [0.5, dx]) ** 2, axis=1)))
    assert cl["kind"][w] != 0 and cl["kind"][i] == 0
    x[i] = x[w] + [0.0, 0.1 * dx]
    cnt, col = _lists(p, x)
    rng = np.random.default_rng(4)
    f = rng.uniform(0.5, 1.5, size=(len(x),) + _f_shape(p))
    out = oracle.manage(p, x, cl["kind"], cl["normal"], f, cnt, col, 0.25 * dx, 0)
    assert out["wall_removals"] == 1 and out["merges"] == 0 and out["adds"] == 0
    keep = np.array([k for k in range(len(x)) if k != i])
    assert np.array_equal(out["origin"], keep)
    assert np.array_equal(out["x"], x[keep]) and np.array_equal(out["f"], f[keep])


def test_point_removed_at_a_wall_takes_no_partner():
    # a is 0.1 dx above a wall point and b 0.2 dx above a (0.3 dx from the wall, so
    # closer to a than rmin but not to the wall): a goes, b stays where it is
    p, cl = _setup()
    x = cl["x"].copy()
    dx = 1.0 / (p["n"] - 1)
    w = int(np.argmin(np.sum((x - [0.5, 0.0]) ** 2, axis=1)))
    a = int(np.argmin(np.sum((x - [0.5, dx]) ** 2, axis=1)))
    b = int(np.argmin(np.sum((x - [0.5, 2 * dx]) ** 2, axis=1)))
    x[a] = x[w] + [0.0, 0.1 * dx]
    x[b] = x[a] + [0.0, 0.2 * dx]
    cnt, col = _lists(p, x)
    f = np.ones((len(x),) + _f_shape(p))
    out = oracle.manage(p, x, cl["kind"], cl["normal"], f, cnt, col, 0.25 * dx, 0)
    assert out["wall_removals"] == 1 and out["merges"] == 0
    assert a not in out["origin"] and b in out["origin"]
    assert np.array_equal(out["x"][list(out["origin"]).index(b)], x[b])
    # without the wall point's pull the two would merge
    far = x.copy()
    far[a] = x[a] + [0.0, 3 * dx]
    far[b] = far[a] + [0.0, 0.2 * dx]
    cnt2, col2 = _lists(p, far)
    out2 = oracle.manage(p, far, cl["kind"], cl["normal"], f, cnt2, col2, 0.25 * dx, 0)
    assert out2["wall_removals"] == 0 and out2["merges"] == 1
