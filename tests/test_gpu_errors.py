"""Error paths of the C ABI that the method's checks produce, with no GPU fault involved.

A state with a negative density reaches the relaxation, which flags it: the next
bgk_sync returns BGK_E_NONFINITE and clears the flag, and the context keeps
working.  A context whose arrays cannot fit in device memory fails in bgk_init with
BGK_E_NOMEM (cudaMalloc reports the failure; bgk_init frees what it had
allocated), after which a normal context still runs.
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


@pytest.mark.parametrize("storage,dim", [("f64", 2), ("f32", 2), ("f32", 3)])
def test_negative_density_is_reported_and_cleared(g, storage, dim):
    name = "cavity2d_n41_v16_f64" if dim == 2 else "cavity3d_n41_v16_f32"
    p = bi.config(name, n=13 if dim == 2 else 7, nv=8, storage=storage)
    cl = bi.cloud_for(p)
    M = oracle.maxwellian(p, 1.0, (0.0, 0.0, 0.0), 1.0)
    n = len(cl["kind"])
    f = np.broadcast_to(M, (n,) + M.shape).copy()
    i = int(np.where(cl["kind"] == 0)[0][len(np.where(cl["kind"] == 0)[0]) // 2])
    f[i] = -M  # negative density at one interior point
    s = g.Solver([p], [cl])
    s.set_f(f if storage == "f64" else f.astype(np.float32))
    s.step(1)
    with pytest.raises(g.BGKError) as e:
        s.sync()
    assert e.value.code == g.BGK_E_NONFINITE
    s.sync()  # the flag is cleared
    s.set_maxwellian()
    s.step(2)
    s.sync()
    rho, _, T = s.moments()
    assert np.all(rho > 0) and np.all(T > 0)
    s.close()


def test_arrays_beyond_device_memory_return_nomem(g):
    import torch
    p = bi.config("cavity2d_n41_v16_f64", n=11, nv=8, storage="f32", max_nbrs=512)
    cl = bi.cloud_for(p)
    n = len(cl["kind"])
    # 2^30 points of room: the neighbour lists alone would need 2 TB
    q = dict(p, spare_points=(1 << 30) - n)
    free0, _ = torch.cuda.mem_get_info()
    with pytest.raises(g.BGKError) as e:
        g.Solver([q], [cl])
    assert e.value.code == g.BGK_E_NOMEM
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 >= free0 - (64 << 20)  # what bgk_init had allocated is released
    s = g.Solver([p], [cl])
    s.set_maxwellian()
    s.step(2)
    s.sync()
    s.close()
