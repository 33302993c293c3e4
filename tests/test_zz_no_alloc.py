"""The allocation-free neighbour build against the context's neighbour build.

bgk_neighbours_noalloc serves callers that cannot allocate device memory: it
writes into buffers the caller owns and keeps its scratch in a fixed array in
device global memory.  Its lists must equal those of bgk_neighbours bit for bit,
also when consecutive calls reuse the shared scratch with different clouds, on a
periodic cloud (minimum image), and after a call that overflowed; with check = 1
an overflow is reported and the truncated rows hold true neighbours.  This file is
collected last on purpose.
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


def _context_lists(g, p, cl):
    s = g.Solver([p], [cl])
    s.neighbours()
    s.sync()
    rowptr, col = s.get_neighbours()
    s.close()
    return rowptr, col


def _noalloc_lists(g, p, cl):
    import torch
    n, dim = cl["x"].shape
    cap = p["max_nbrs"]
    x = torch.from_numpy(np.ascontiguousarray(cl["x"])).cuda()
    cnt = torch.full((n,), -1, dtype=torch.int32, device="cuda")
    ell = torch.full((n, cap), -7, dtype=torch.int32, device="cuda")
    g.bgk_neighbours_noalloc(dim, n, x, p["h"], int(p.get("periodic", 0)), cap, cnt, ell, 1)
    torch.cuda.synchronize()
    cnt, ell = cnt.cpu().numpy(), ell.cpu().numpy()
    rowptr = np.zeros(n + 1, dtype=np.int64)
    rowptr[1:] = np.cumsum(cnt)
    col = np.concatenate([ell[i, : cnt[i]] for i in range(n)])
    return rowptr, col


def test_noalloc_lists_equal_context_lists_on_consecutive_calls(g):
    cases = [bi.config("cavity2d_n41_v16_f64", n=101, nv=4),
             bi.config("cavity3d_n41_v16_f32", n=21, nv=4),
             bi.config("cavity2d_n41_v16_f64", n=61, nv=4, seed=77)]
    for p in cases:
        cl = bi.cloud_for(p)
        r0, c0 = _context_lists(g, p, cl)
        r1, c1 = _noalloc_lists(g, p, cl)
        assert np.array_equal(r0, r1) and np.array_equal(c0, c1), p["n"]


def test_noalloc_rejects_sizes_beyond_its_scratch(g):
    import torch
    n = 131073
    x = torch.zeros((n, 2), dtype=torch.float64, device="cuda")
    cnt = torch.zeros(n, dtype=torch.int32, device="cuda")
    col = torch.zeros((n, 8), dtype=torch.int32, device="cuda")
    with pytest.raises(g.BGKError) as e:
        g.bgk_neighbours_noalloc(2, n, x, 0.01, 0, 8, cnt, col, 1)
    assert e.value.code == g.BGK_E_INVAL


def test_noalloc_periodic_cloud_matches_context_and_oracle(g):
    import oracle
    x = bi.uniform01(99, 3000 * 2).reshape(-1, 2)
    cl = {"x": x, "kind": np.zeros(len(x), np.int32), "normal": np.zeros_like(x)}
    p = {"dim": 2, "nv": 4, "vmax": 1.0, "kn": 1.0, "tau_mode": 2, "dt": 1e-3, "h": 0.04, "alpha": 6.25,
         "max_nbrs": 64, "periodic": 1, "storage": "f64"}
    r0, c0 = _context_lists(g, p, cl)
    r1, c1 = _noalloc_lists(g, p, cl)
    assert np.array_equal(r0, r1) and np.array_equal(c0, c1)
    cnt, ocol = oracle.neighbours(x, p["h"], True, 64)
    orp, oc = oracle.to_csr(cnt, ocol)
    assert np.array_equal(r1, orp) and np.array_equal(c1, oc)


def test_noalloc_overflow_is_reported_with_check(g):
    import torch
    p = bi.config("cavity2d_n41_v16_f64", n=41, nv=4)
    cl = bi.cloud_for(p)
    r0, c0 = _context_lists(g, p, cl)
    n, dim = cl["x"].shape
    cap = 6
    x = torch.from_numpy(np.ascontiguousarray(cl["x"])).cuda()
    cnt = torch.full((n,), -1, dtype=torch.int32, device="cuda")
    ell = torch.full((n, cap), -7, dtype=torch.int32, device="cuda")
    with pytest.raises(g.BGKError) as e:
        g.bgk_neighbours_noalloc(dim, n, x, p["h"], 0, cap, cnt, ell, 1)
    assert e.value.code == g.BGK_E_NBR_OVERFLOW
    cnt, ell = cnt.cpu().numpy(), ell.cpu().numpy()
    full = np.diff(r0)
    assert np.array_equal(cnt, np.minimum(full, cap))
    for i in range(n):
        row = ell[i, :cnt[i]]
        true = set(c0[r0[i]:r0[i + 1]].tolist())
        assert set(row.tolist()) <= true and np.all(np.diff(row) > 0), i
    # the next call starts from a cleared status and gives the full lists again
    r1, c1 = _noalloc_lists(g, p, cl)
    assert np.array_equal(r0, r1) and np.array_equal(c0, c1)
