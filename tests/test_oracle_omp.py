"""The OpenMP build of the oracle (used only to time it on all host cores) computes
every point exactly as the plain build: f, moments and positions agree bit for bit
after several steps of a fixed and an ALE 2D cavity, a 3D cavity, the second-order
(quadratic) stencils and a moving body."""
import numpy as np
import pytest

import bgk_inputs as bi
import oracle


def _cases():
    yield "ale2d", bi.config("cavity2d_ale_n201_v32_f32", n=31, nv=12, kn=0.1), None
    yield "fixed2d", bi.config("cavity2d_n41_v16_f64", n=25, nv=10), None
    yield "cavity3d", bi.config("cavity3d_n41_v16_f32", n=7, nv=6, vmax=4.0), None
    yield "quadratic", bi.config("cavity2d_ale_n201_v32_f32", n=21, nv=8, vmax=4.0, wls_order=2), None
    p = bi.config("body2d_ale_n201_v32_f32", n=41, nv=8, vmax=4.0)
    yield "body", p, bi.cloud_for(p)


@pytest.mark.parametrize("name,p,cl", list(_cases()), ids=[c[0] for c in _cases()])
def test_openmp_build_equals_plain_build(name, p, cl):
    if cl is None:
        cl = bi.cloud_for(p)
    a = oracle.Simulation(p, cl)
    b = oracle.Simulation(p, cl, omp=True)
    a.run(4)
    b.run(4)
    assert oracle.threads(True) >= 1
    for u, v in ((a.f, b.f), (a.rho, b.rho), (a.U, b.U), (a.T, b.T), (a.x, b.x)):
        assert np.array_equal(u, v), name
    assert a.clamps == b.clamps
