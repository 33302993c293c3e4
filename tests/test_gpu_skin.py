"""ALE neighbour lists with a skin (candidate lists re-filtered every step).

The exact test is applied to candidates of radius h (1 + skin) that are rebuilt
only after a point has moved h skin / 2; the lists, and so every state, must be
bit-identical to a full cell search every step (skin 0).  Small skins force a
rebuild almost every step; a fast lid and a drifting periodic box make points
move far (the periodic wrap forces a rebuild).
"""
import numpy as np
import pytest

import bgk_inputs as bi

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


def _run(g, p, cl, nsteps, u0=(0.0, 0.0, 0.0)):
    s = g.Solver([p], [cl])
    s.set_maxwellian(u0=u0)
    s.step(nsteps)
    s.sync()
    out = (s.get_f(0, np.float32 if p["storage"] != "f64" else np.float64), s.positions(0), s.get_neighbours(0),
           s.stats()["nnz"])
    s.close()
    return out


def _same(a, b):
    fa, xa, (ra, ca), za = a
    fb, xb, (rb, cb), zb = b
    assert np.array_equal(xa, xb)
    assert np.array_equal(ra, rb) and np.array_equal(ca, cb)
    assert za == zb
    assert np.array_equal(fa, fb)


@pytest.mark.parametrize("storage", ["f32", "f64"])
def test_cavity_skin_lists_are_bit_identical(g, storage):
    p = bi.config("cavity2d_ale_n201_v32_f32", n=41, nv=8, vmax=4.0, storage=storage)
    p["lid_u"] = [0.3, 0.0, 0.0]
    cl = bi.cloud_for(p)
    ref = _run(g, dict(p, skin=0.0), cl, 100)
    for skin in (0.01, 0.2, 1.0):
        _same(_run(g, dict(p, skin=skin), cl, 100), ref)


def test_3d_cavity_skin_lists_are_bit_identical(g):
    p = bi.config("cavity3d_n41_v16_f32", n=9, nv=6, vmax=4.0, ale=1)
    p["lid_u"] = [0.3, 0.0, 0.0]
    cl = bi.cloud_for(p)
    ref = _run(g, dict(p, skin=0.0), cl, 30)
    for skin in (0.02, 0.3):
        _same(_run(g, dict(p, skin=skin), cl, 30), ref)


def test_periodic_drift_wraps_and_rebuilds(g):
    n = 15
    cl = bi.periodic_box(2, n, seed=5, jitter=0.1)
    p = {"dim": 2, "nv": 8, "vmax": 4.0, "kn": 0.5, "tau_mode": 0, "h": 2.5 / n, "alpha": 6.25, "wall_T": 1.0,
         "max_nbrs": 48, "periodic": 1, "ale": 1, "storage": "f32", "dt": bi.cfl_dt(1.0 / n, 4.0, 2)}
    u0 = (0.9, -0.4, 0.0)  # uniform drift: every point crosses the box edge within the run
    ref = _run(g, dict(p, skin=0.0), cl, 120, u0)
    x0 = np.asarray(cl["x"])
    assert np.any(ref[1][:, 0] < x0[:, 0] - 0.1)  # the drift is in +x, so these points wrapped
    for skin in (0.02, 0.4):
        _same(_run(g, dict(p, skin=skin), cl, 120, u0), ref)
