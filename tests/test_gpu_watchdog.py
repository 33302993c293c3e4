"""Failure detection of the bounded device waits (no GPU fault involved): with the
watchdog limit at one poll, the grid barriers of the fused ALE list-build kernel give up
at once, the step reports BGK_E_TIMEOUT at the next bgk_sync, and the context stays
usable: after a checkpoint restore and the default limit, the run continues bit for bit
as a run that never timed out.
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


def test_watchdog_timeout_is_reported_and_recoverable(g):
    p = bi.config("cavity2d_ale_n201_v32_f32", n=41, nv=8, vmax=4.0)  # FP32, skin lists: fused list build
    cl = bi.cloud_for(p)
    s = g.Solver([p], [cl])
    s.set_maxwellian()
    s.step(2)
    s.sync()
    blob = g.bgk_get_state(s.ctx)
    s.step(3)
    s.sync()
    ref = s.get_f(0, np.float32)
    # every grid barrier gives up after one poll
    g.bgk_set_state(s.ctx, blob)
    g.bgk_set_watchdog(s.ctx, 1)
    s.step(3)
    with pytest.raises(g.BGKError) as e:
        s.sync()
    assert e.value.code == g.BGK_E_TIMEOUT
    # back to the default limit and the checkpoint: the same steps as the clean run
    g.bgk_set_watchdog(s.ctx, 0)
    g.bgk_set_state(s.ctx, blob)
    s.step(3)
    s.sync()
    assert np.array_equal(s.get_f(0, np.float32), ref)
    with pytest.raises(g.BGKError):
        g.bgk_set_watchdog(s.ctx, -1)
    s.close()


@pytest.mark.parametrize("body", [False, True])
def test_run_continues_after_timeout_without_restore(g, body):
    # A timeout in the side chain of the last step before bgk_sync: bgk_sync reports it,
    # resets the barrier state and drops the partly built lists; the next steps rebuild
    # them from the moved positions and match a run that never timed out, bit for bit.
    name = "body2d_ale_n201_v32_f32" if body else "cavity2d_ale_n201_v32_f32"
    p = bi.config(name, n=41, nv=8, vmax=4.0)
    cl = bi.cloud_for(p)
    ref = g.Solver([p], [cl])
    ref.set_maxwellian()
    ref.step(6)
    ref.sync()
    s = g.Solver([p], [cl])
    s.set_maxwellian()
    s.step(2)
    s.sync()
    g.bgk_set_watchdog(s.ctx, 1)
    s.step(1)
    with pytest.raises(g.BGKError) as e:
        s.sync()
    assert e.value.code == g.BGK_E_TIMEOUT
    g.bgk_set_watchdog(s.ctx, 0)
    s.step(3)
    s.sync()
    assert np.array_equal(s.positions(), ref.positions())
    assert np.array_equal(s.get_f(0, np.float32), ref.get_f(0, np.float32))
    if body:
        assert np.array_equal(s.body_centre(), ref.body_centre())
    # and the barriers keep working: more steps, no error
    s.step(5)
    ref.step(5)
    s.sync()
    ref.sync()
    assert np.array_equal(s.get_f(0, np.float32), ref.get_f(0, np.float32))
    s.close()
    ref.close()
