"""Caller-owned distribution storage (bgk_bind_f): a torch tensor bound as a case's f
holds the state after every call, bit-identical to the context's own storage, for odd
and even step counts, the ALE side chain, the second-order step, point management and
unbinding; writing into the tensor and calling bgk_set_f on it recomputes the moments.
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


def _tensor(p, n, spare=0):
    import torch
    dt = {"f64": torch.float64, "f32": torch.float32, "bf16": torch.bfloat16}[p["storage"]]
    nc = 2 if p["dim"] == 2 else 1
    return torch.full((n + spare, nc, p["nv"] ** p["dim"]), float("nan"), dtype=dt, device="cuda")


@pytest.mark.parametrize("storage,ale,order", [("f64", 0, 1), ("f32", 1, 1), ("bf16", 1, 1), ("f32", 0, 2)])
def test_bound_tensor_holds_the_state(g, storage, ale, order):
    import torch
    p = bi.config("cavity2d_n41_v16_f64", n=15, nv=8, vmax=3.0, storage=storage, ale=ale, time_order=order)
    cl = bi.cloud_for(p)
    n = len(cl["kind"])
    ref = g.Solver([p], [cl])
    ref.set_maxwellian()
    s = g.Solver([p], [cl])
    f = _tensor(p, n)
    s.bind_f(f)
    s.set_maxwellian()
    for k in (3, 2, 1):  # odd, even, odd step counts
        ref.step(k)
        s.step(k)
        torch.cuda.synchronize()
        want = ref.get_f(0, np.float64)
        got = f.double().cpu().numpy()
        assert np.array_equal(got, want), k
        assert np.array_equal(s.get_f(0, np.float64), want)
        assert np.array_equal(np.concatenate(s.moments()[:1]), np.concatenate(ref.moments()[:1]))
    # unbind: the state goes back into the context's buffer, stepping continues the same
    s.bind_f(None)
    f.fill_(float("nan"))
    ref.step(3)
    s.step(3)
    assert np.array_equal(s.get_f(0, np.float64), ref.get_f(0, np.float64))
    s.close()
    ref.close()


def test_writes_into_the_bound_tensor_and_set_f(g):
    import torch
    p = bi.config("cavity2d_n41_v16_f64", n=15, nv=8, vmax=3.0, storage="f32")
    cl = bi.cloud_for(p)
    n = len(cl["kind"])
    s = g.Solver([p], [cl])
    s.set_maxwellian()
    rho0, _, _ = s.moments()
    f = _tensor(p, n)
    s.bind_f(f)
    f.mul_(1.5)  # the caller changes the state in place
    g.bgk_set_f(s.ctx, 0, f, g.BGK_F32)  # the bound buffer itself: moments only
    rho, _, _ = s.moments()
    assert np.allclose(rho, 1.5 * rho0, rtol=1e-6)
    ref = g.Solver([p], [cl])
    ref.set_f(f.cpu())
    s.step(5)
    ref.step(5)
    torch.cuda.synchronize()
    assert np.array_equal(f.double().cpu().numpy(), ref.get_f(0, np.float64))
    s.close()
    ref.close()


def test_bound_tensor_through_point_management(g):
    import torch
    p = bi.config("cavity2d_ale_n201_v32_f32", n=21, nv=4, vmax=3.0, storage="f64", spare_points=200)
    cl = bi.cloud_for(p)
    n = len(cl["kind"])
    ref = g.Solver([p], [cl])
    s = g.Solver([p], [cl])
    f = _tensor(p, n, 200)
    s.bind_f(f)
    for x in (ref, s):
        x.set_maxwellian()
        x.step(7)
    r1 = ref.manage(0.35 * p["dx"], 14)
    r2 = s.manage(0.35 * p["dx"], 14)
    assert r1 == r2
    ref.step(3)
    s.step(3)
    torch.cuda.synchronize()
    m = r1[0]
    assert np.array_equal(f[:m].double().cpu().numpy(), ref.get_f(0, np.float64))
    s.close()
    ref.close()


def test_bind_rejects_bad_buffers(g):
    import torch
    p = bi.config("cavity2d_n41_v16_f64", n=9, nv=6, vmax=3.0, storage="f64")  # NV = 36
    cl = bi.cloud_for(p)
    n = len(cl["kind"])
    s = g.Solver([p], [cl])
    with pytest.raises(g.BGKError):
        s.bind_f(torch.zeros(n * 2 * 36 - 1, dtype=torch.float64, device="cuda"))  # too small
    with pytest.raises(g.BGKError):
        g.bgk_bind_f(s.ctx, 0, torch.zeros(n * 2 * 36, dtype=torch.float64))  # host memory
    s.close()
    p = bi.config("cavity2d_n41_v16_f64", n=9, nv=5, vmax=3.0, storage="f64")  # NV = 25: padded
    cl = bi.cloud_for(p)
    s = g.Solver([p], [cl])
    with pytest.raises(g.BGKError):
        s.bind_f(torch.zeros((len(cl["kind"]), 2, 28), dtype=torch.float64, device="cuda"))
    s.close()


@pytest.mark.parametrize("ale", [0, 1])
def test_staged_inputs_equal_set_f(g, ale):
    # bgk_stage_f uploads on another stream and the next step takes the input: the same
    # bits as bgk_set_f followed by the step, for a new input every step
    import torch
    p = bi.config("cavity2d_n41_v16_f64", n=15, nv=8, vmax=3.0, storage="f32", ale=ale)
    cl = bi.cloud_for(p)
    n = len(cl["kind"])
    gen = g.Solver([p], [cl])
    gen.set_maxwellian()
    a, b = g.Solver([p], [cl]), g.Solver([p], [cl])
    for k in range(4):
        gen.step(2)
        f_in = torch.from_numpy(gen.get_f(0, np.float32)).pin_memory()
        a.set_f(f_in)
        a.step(1)
        g.bgk_stage_f(b.ctx, 0, f_in, g.BGK_F32)
        b.step(1)
        b.sync()
        assert np.array_equal(b.get_f(0, np.float64), a.get_f(0, np.float64)), k
        for x, y in zip(b.moments(), a.moments()):
            assert np.array_equal(x, y)
    with pytest.raises(g.BGKError):  # pageable host memory
        g.bgk_stage_f(b.ctx, 0, np.zeros((n, 2, 64), np.float32), g.BGK_F32)
    g.bgk_stage_f(b.ctx, 0, f_in, g.BGK_F32)
    with pytest.raises(g.BGKError):  # binding while an input is pending
        b.bind_f(torch.zeros((n, 2, 64), dtype=torch.float32, device="cuda"))
    b.step(1)
    b.sync()
    for x in (gen, a, b):
        x.close()
