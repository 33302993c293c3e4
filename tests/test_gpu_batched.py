"""Batched stepping of many independent cavities (one launch per step over all cases).

The batched kernels run the same per-point and per-wall-point code as the
per-case kernels, so every mode must give bit-identical states; one case of a
batch is also checked against the FP64 oracle.
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


def _mixed_cases():
    specs = [(21, 8, 0.1, 0.10), (33, 9, 0.02, 0.15), (17, 12, 1.0, 0.05), (41, 7, 0.3, 0.2), (25, 16, 0.05, 0.1),
             (29, 11, 0.5, 0.12)]
    ps, cls = [], []
    for k, (n, nv, kn, lid) in enumerate(specs):
        p = bi.config("cavity2d_n41_v16_f64", n=n, nv=nv, kn=kn, storage="f32", seed=2408500 + k)
        p["lid_u"] = [lid, 0.0, 0.0]
        ps.append(p)
        cls.append(bi.cloud_for(p))
    return ps, cls


def _run(g, ps, cls, mode, nsteps, tune=False):
    s = g.Solver(ps, cls)
    g.bgk_set_batching(s.ctx, mode)
    s.set_maxwellian()
    if tune:
        g.bgk_autotune(s.ctx)
    s.step(nsteps)
    s.sync()
    out = [s.get_f(c, np.float32) for c in range(len(ps))]
    st = s.stats()
    s.close()
    return out, st


def test_batched_modes_are_bit_identical_to_per_case_stepping(g):
    ps, cls = _mixed_cases()
    ref, st0 = _run(g, ps, cls, 0, 10)
    assert st0["batch_mode"] == 0
    for mode in (1, 2):
        got, st = _run(g, ps, cls, mode, 10, tune=(mode == 2))
        assert st["batch_mode"] == mode
        for c in range(len(ps)):
            assert np.array_equal(got[c], ref[c]), (mode, c)


def test_autotune_leaves_the_state_unchanged(g):
    ps, cls = _mixed_cases()
    s = g.Solver(ps, cls)
    s.set_maxwellian()
    s.step(2)
    s.sync()
    before = [s.get_f(c, np.float32) for c in range(len(ps))]
    g.bgk_autotune(s.ctx)
    s.sync()
    after = [s.get_f(c, np.float32) for c in range(len(ps))]
    st = s.stats()
    assert st["batch_warps"] in (4, 8)
    for c in range(len(ps)):
        assert np.array_equal(before[c], after[c])


def test_batched_case_matches_oracle(g):
    ps, cls = _mixed_cases()
    s = g.Solver(ps, cls)
    s.set_maxwellian()
    s.step(20)
    s.sync()
    for c in (1, 3):
        sim = oracle.Simulation(ps[c], cls[c])
        sim.run(20)
        rho, u, T = s.moments(c)
        assert np.abs(rho - sim.rho).max() < 1e-4 * np.abs(sim.rho).max()
        assert np.abs(T - sim.T).max() < 1e-4 * np.abs(sim.T).max()
        assert np.abs(u - sim.U).max() < 1e-4 * np.abs(sim.U).max()


def test_sixty_four_cavity_sweep_matches_per_case_stepping(g):
    # 64 cavities: sides uniform in [41, 121], velocity nodes uniform in [16, 32], Kn log-uniform in [0.01, 1]
    ps = bi.batched_cases(64)
    cls = [bi.cloud_for(p) for p in ps]
    ref, _ = _run(g, ps, cls, 0, 3)
    got, st = _run(g, ps, cls, 2, 3, tune=True)
    assert st["batch_mode"] == 2
    for c in range(len(ps)):
        assert np.array_equal(got[c], ref[c]), c
