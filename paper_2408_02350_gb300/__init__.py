"""Python binding of libbgk, the GB300 library for the per-time-step hot path of the
meshfree ALE / weighted-least-squares scheme for the BGK equation (arXiv 2408.02350).

The functions below carry the names of the C ABI in ``include/bgk.h`` and only
marshal arguments (numpy host arrays, torch device tensors, CUDA streams) to
it; every step of the method runs in the library's CUDA kernels.  There is no
CPU fallback: importing this package without the built library raises.

``Solver`` is a convenience wrapper around one context.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
# BGK_LIBRARY selects a build variant (_build.build(variant=...)): "debug", the bounds-
# checked build (libbgk_debug.so: every neighbour and point index a kernel loads is
# checked against the point range, a bad one is recorded, BGK_E_BOUNDS at the next
# bgk_sync, and its access skipped), or "staged" (libbgk_staged.so: the 2D FP32 transport
# stages its neighbour rows in shared memory by bulk copies; same results, slower).
_VARIANT = os.environ.get("BGK_LIBRARY")
LIB_PATH = os.path.join(_HERE, "libbgk_%s.so" % _VARIANT if _VARIANT in ("debug", "staged") else "libbgk.so")

BGK_OK, BGK_E_INVAL, BGK_E_NOMEM, BGK_E_CUDA, BGK_E_SINGULAR = 0, 1, 2, 3, 4
BGK_E_NBR_OVERFLOW, BGK_E_NONFINITE, BGK_E_TIMEOUT, BGK_E_STATE, BGK_E_BOUNDS = 5, 6, 7, 8, 9
BGK_F64, BGK_F32, BGK_BF16 = 0, 1, 2
STORAGE = {"f64": BGK_F64, "f32": BGK_F32, "bf16": BGK_BF16}
K_TRANSPORT, K_WALLS, K_NBR, K_STENCIL, K_MOVE, K_ADJOINT, K_BATCH = 0, 1, 2, 3, 4, 5, 6

_STATUS_NAMES = {1: "BGK_E_INVAL", 2: "BGK_E_NOMEM", 3: "BGK_E_CUDA", 4: "BGK_E_SINGULAR",
                 5: "BGK_E_NBR_OVERFLOW", 6: "BGK_E_NONFINITE", 7: "BGK_E_TIMEOUT", 8: "BGK_E_STATE",
                 9: "BGK_E_BOUNDS"}


class BGKError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__("%s (%d): %s" % (_STATUS_NAMES.get(code, "?"), code, msg))
        self.code = code


class bgk_params(C.Structure):
    _fields_ = [
        ("dim", C.c_int32), ("nv", C.c_int32), ("vmax", C.c_double), ("kn", C.c_double),
        ("tau_mode", C.c_int32), ("ale", C.c_int32), ("periodic", C.c_int32), ("lid_wall", C.c_int32),
        ("max_nbrs", C.c_int32), ("storage", C.c_int32),
        ("dt", C.c_double), ("h", C.c_double), ("alpha", C.c_double), ("wall_T", C.c_double),
        ("guard", C.c_double), ("lid_u", C.c_double * 3), ("skin", C.c_double),
        ("spare_points", C.c_int32), ("pad2_", C.c_int32),
        ("body_wall", C.c_int32), ("wls_order", C.c_int32), ("body_u", C.c_double * 3),
        ("body_centre", C.c_double * 3), ("body_radius", C.c_double),
        ("vk_lo", C.c_int32), ("vk_hi", C.c_int32), ("time_order", C.c_int32), ("vgrid", C.c_int32),
    ]


class bgk_stats(C.Structure):
    _fields_ = [("steps", C.c_int64), ("launches", C.c_int64), ("clamps", C.c_int64), ("nnz", C.c_int64),
                ("nv_pad", C.c_int32), ("n_cases", C.c_int32), ("batch_mode", C.c_int32), ("batch_warps", C.c_int32),
                ("batch_grid", C.c_int32), ("pad_", C.c_int32)]


_P = C.c_void_p
_PD = C.POINTER(C.c_double)
_PI = C.POINTER(C.c_int32)
_PL = C.POINTER(C.c_int64)

_SIGS = {
    "bgk_version": (C.c_int, []),
    "bgk_peak_fp32": (C.c_int, [_PD, _PD, _PI, _P]),
    "bgk_peak_fp64": (C.c_int, [_PD, _P]),
    "bgk_init": (C.c_int, [C.POINTER(bgk_params), C.c_int32, _PL, _PD, _PI, _PD, C.POINTER(_P)]),
    "bgk_set_maxwellian": (C.c_int, [_P, C.c_double, _PD, C.c_double, _P]),
    "bgk_set_f": (C.c_int, [_P, C.c_int32, _P, C.c_int32, C.c_int32, _P]),
    "bgk_get_f": (C.c_int, [_P, C.c_int32, _P, C.c_int32, C.c_int32, _P]),
    "bgk_bind_f": (C.c_int, [_P, C.c_int32, _P, C.c_size_t, _P]),
    "bgk_stage_f": (C.c_int, [_P, C.c_int32, _P, C.c_int32]),
    "bgk_neighbours": (C.c_int, [_P, _P]),
    "bgk_get_neighbours": (C.c_int, [_P, C.c_int32, _PL, _PI, C.c_int64, _PL]),
    "bgk_get_stencils": (C.c_int, [_P, C.c_int32, _PD, _PD, C.c_int64]),
    "bgk_step": (C.c_int, [_P, C.c_int32, _P]),
    "bgk_moments": (C.c_int, [_P, C.c_int32, _P, _P, _P, C.c_int32, _P]),
    "bgk_get_positions": (C.c_int, [_P, C.c_int32, _P, C.c_int32, _P]),
    "bgk_get_body": (C.c_int, [_P, C.c_int32, _PD]),
    "bgk_sync": (C.c_int, [_P, _P]),
    "bgk_get_state": (C.c_int, [_P, _P, C.c_size_t, C.POINTER(C.c_size_t)]),
    "bgk_set_state": (C.c_int, [_P, _P, C.c_size_t]),
    "bgk_set_timing": (C.c_int, [_P, C.c_int32]),
    "bgk_set_watchdog": (C.c_int, [_P, C.c_int64]),
    "bgk_get_timing": (C.c_int, [_P, C.c_int32, _PD, _PL]),
    "bgk_get_stats": (C.c_int, [_P, C.POINTER(bgk_stats)]),
    "bgk_last_error": (C.c_char_p, [_P]),
    "bgk_free": (None, [_P]),
    "bgk_set_params": (C.c_int, [_P, C.c_int32, C.POINTER(bgk_params)]),
    "bgk_manage": (C.c_int, [_P, C.c_int32, C.c_double, C.c_int32, _PL, _P]),
    "bgk_set_batching": (C.c_int, [_P, C.c_int32]),
    "bgk_autotune": (C.c_int, [_P, _P]),
    "bgk_objective": (C.c_int, [_P, C.c_int32, _P, _P, C.c_double, _P]),
    "bgk_adjoint_step": (C.c_int, [_P, C.c_int32, _P, _P, _P, _P]),
    "bgk_neighbours_noalloc": (C.c_int, [C.c_int32, C.c_int64, _P, C.c_double, C.c_int32, C.c_int32, _P, _P,
                                         C.c_int32, _P]),
    "bgk_shard_sizes": (C.c_int, [_P, C.c_int32, _PL, _PL]),
    "bgk_shard_transport": (C.c_int, [_P, C.c_int32, _P, _P]),
    "bgk_shard_relax": (C.c_int, [_P, C.c_int32, _P, _P, _P]),
    "bgk_shard_walls": (C.c_int, [_P, C.c_int32, _P, _P]),
    "bgk_shard_partial": (C.c_int, [_P, C.c_int32, _P, _P]),
    "bgk_shard_set_moments": (C.c_int, [_P, C.c_int32, _P, _P]),
    "bgk_shard_allreduce": (C.c_int, [C.POINTER(_P), C.c_int32, C.c_int64, _P]),
}

_lib = None


def lib():
    """The loaded libbgk.so; raises if it has not been built."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError("libbgk.so is not built (%s); run `python -c \"import __graft_entry__ as g; g.build()\"`"
                              % LIB_PATH)
        h = C.CDLL(LIB_PATH)
        for name, (res, args) in _SIGS.items():
            fn = getattr(h, name)
            fn.restype = res
            fn.argtypes = args
        _lib = h
    return _lib


def exported_symbols() -> list:
    return list(_SIGS)


def _check(code: int, ctx=None) -> None:
    if code != BGK_OK:
        msg = lib().bgk_last_error(ctx)
        raise BGKError(code, msg.decode() if msg else "")


def _stream_ptr(stream) -> int | None:
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def _ptr(a) -> int:
    """Address of a numpy array or a torch tensor (contiguous)."""
    if isinstance(a, np.ndarray):
        assert a.flags.c_contiguous
        return a.ctypes.data
    assert a.is_contiguous()
    return a.data_ptr()


def _on_device(a) -> int:
    return 0 if isinstance(a, np.ndarray) else int(a.is_cuda)


# ---- the C ABI, one Python function per entry point ----

def bgk_version() -> int:
    return lib().bgk_version()


def bgk_peak_fp32(stream=None) -> dict:
    """Measured FP32 FMA rates of the device: scalar and packed FMAs per second, SM count."""
    a, b, n = C.c_double(0.0), C.c_double(0.0), C.c_int32(0)
    _check(lib().bgk_peak_fp32(C.byref(a), C.byref(b), C.byref(n), _stream_ptr(stream)))
    return {"fma_per_s": a.value, "fma2_per_s": b.value, "n_sm": n.value}


def bgk_peak_fp64(stream=None) -> float:
    """Measured FP64 FMAs per second of the device."""
    a = C.c_double(0.0)
    _check(lib().bgk_peak_fp64(C.byref(a), _stream_ptr(stream)))
    return a.value


def bgk_init(params: list, n_points, x, kind, normal) -> int:
    arr = (bgk_params * len(params))(*params)
    npts = np.ascontiguousarray(n_points, dtype=np.int64)
    x = np.ascontiguousarray(x, dtype=np.float64)
    kind = np.ascontiguousarray(kind, dtype=np.int32)
    normal = np.ascontiguousarray(normal, dtype=np.float64)
    ctx = _P()
    code = lib().bgk_init(arr, len(params), npts.ctypes.data_as(_PL), x.ctypes.data_as(_PD),
                          kind.ctypes.data_as(_PI), normal.ctypes.data_as(_PD), C.byref(ctx))
    _check(code, None)
    return ctx.value


def bgk_set_maxwellian(ctx, rho0: float, u0, T0: float, stream=None) -> None:
    u = np.zeros(3)
    u[: len(u0)] = u0
    _check(lib().bgk_set_maxwellian(ctx, rho0, u.ctypes.data_as(_PD), T0, _stream_ptr(stream)), ctx)


def bgk_set_f(ctx, case: int, f, dtype: int, stream=None) -> None:
    _check(lib().bgk_set_f(ctx, case, _ptr(f), dtype, _on_device(f), _stream_ptr(stream)), ctx)


def bgk_get_f(ctx, case: int, f, dtype: int, stream=None) -> None:
    _check(lib().bgk_get_f(ctx, case, _ptr(f), dtype, _on_device(f), _stream_ptr(stream)), ctx)


def bgk_stage_f(ctx, case: int, f, dtype: int) -> None:
    """Asynchronous upload of case's next input from page-locked host memory (a pinned
    torch tensor); the next bgk_step takes it."""
    _check(lib().bgk_stage_f(ctx, case, _ptr(f), dtype), ctx)


def bgk_bind_f(ctx, case: int, f, stream=None) -> None:
    """Use the device tensor f (contiguous, the storage dtype) as case's distribution
    storage; None unbinds."""
    if f is None:
        _check(lib().bgk_bind_f(ctx, case, None, 0, _stream_ptr(stream)), ctx)
    else:
        _check(lib().bgk_bind_f(ctx, case, _ptr(f), f.numel() * f.element_size(), _stream_ptr(stream)), ctx)


def bgk_neighbours(ctx, stream=None) -> None:
    _check(lib().bgk_neighbours(ctx, _stream_ptr(stream)), ctx)


def bgk_get_neighbours(ctx, case: int, n: int):
    rowptr = np.zeros(n + 1, dtype=np.int64)
    nnz = C.c_int64(0)
    _check(lib().bgk_get_neighbours(ctx, case, rowptr.ctypes.data_as(_PL), None, 0, C.byref(nnz)), ctx)
    col = np.zeros(max(nnz.value, 1), dtype=np.int32)
    _check(lib().bgk_get_neighbours(ctx, case, rowptr.ctypes.data_as(_PL), col.ctypes.data_as(_PI), col.size,
                                    C.byref(nnz)), ctx)
    return rowptr, col[: nnz.value]


def bgk_get_stencils(ctx, case: int, nnz: int, dim: int):
    P = np.zeros((max(nnz, 1), dim, dim))
    R = np.zeros(max(nnz, 1))
    _check(lib().bgk_get_stencils(ctx, case, P.ctypes.data_as(_PD), R.ctypes.data_as(_PD), nnz), ctx)
    return P[:nnz], R[:nnz]


def bgk_step(ctx, nsteps: int, stream=None) -> None:
    _check(lib().bgk_step(ctx, nsteps, _stream_ptr(stream)), ctx)


def bgk_moments(ctx, case: int, rho, u, T, stream=None) -> None:
    _check(lib().bgk_moments(ctx, case, _ptr(rho), _ptr(u), _ptr(T), _on_device(rho), _stream_ptr(stream)), ctx)


def bgk_get_positions(ctx, case: int, x, stream=None) -> None:
    _check(lib().bgk_get_positions(ctx, case, _ptr(x), _on_device(x), _stream_ptr(stream)), ctx)


def bgk_get_body(ctx, case: int, dim: int) -> np.ndarray:
    c = np.zeros(dim)
    _check(lib().bgk_get_body(ctx, case, c.ctypes.data_as(_PD)), ctx)
    return c


def bgk_set_watchdog(ctx, max_polls: int) -> None:
    _check(lib().bgk_set_watchdog(ctx, int(max_polls)), ctx)


def bgk_sync(ctx, stream=None) -> None:
    _check(lib().bgk_sync(ctx, _stream_ptr(stream)), ctx)


def bgk_get_state(ctx) -> bytes:
    used = C.c_size_t(0)
    _check(lib().bgk_get_state(ctx, None, 0, C.byref(used)), ctx)
    buf = C.create_string_buffer(used.value)
    _check(lib().bgk_get_state(ctx, C.cast(buf, _P), used.value, C.byref(used)), ctx)
    return buf.raw


def bgk_set_state(ctx, blob: bytes) -> None:
    buf = C.create_string_buffer(blob, len(blob))
    _check(lib().bgk_set_state(ctx, C.cast(buf, _P), len(blob)), ctx)


def bgk_set_timing(ctx, enable) -> None:
    """enable: True times every kernel group, False none, an int is the bit mask of group ids."""
    mask = (0x7F if enable else 0) if isinstance(enable, bool) else int(enable)
    _check(lib().bgk_set_timing(ctx, mask), ctx)


def bgk_get_timing(ctx, which: int):
    ms, n = C.c_double(0), C.c_int64(0)
    _check(lib().bgk_get_timing(ctx, which, C.byref(ms), C.byref(n)), ctx)
    return ms.value, n.value


def bgk_get_stats(ctx) -> dict:
    s = bgk_stats()
    _check(lib().bgk_get_stats(ctx, C.byref(s)), ctx)
    return {k: getattr(s, k) for k, _ in bgk_stats._fields_}


def bgk_last_error(ctx) -> str:
    msg = lib().bgk_last_error(ctx)
    return msg.decode() if msg else ""


def bgk_free(ctx) -> None:
    lib().bgk_free(ctx)


def bgk_set_params(ctx, case: int, params) -> None:
    q = params if isinstance(params, bgk_params) else params_from(params)
    _check(lib().bgk_set_params(ctx, case, C.byref(q)), ctx)


def bgk_manage(ctx, case: int, rmin: float, min_nbrs: int, stream=None):
    """One point-management pass; returns (new point count, removed by merging, added)."""
    counts = (C.c_int64 * 3)()
    _check(lib().bgk_manage(ctx, case, float(rmin), int(min_nbrs), counts, _stream_ptr(stream)), ctx)
    return int(counts[0]), int(counts[1]), int(counts[2])


def bgk_set_batching(ctx, mode: int) -> None:
    _check(lib().bgk_set_batching(ctx, mode), ctx)


def bgk_autotune(ctx, stream=None) -> None:
    _check(lib().bgk_autotune(ctx, _stream_ptr(stream)), ctx)


def bgk_objective(ctx, case: int, J=None, lam=None, scale: float = 1.0, stream=None) -> None:
    """J (device float64 tensor of one element) += lid flux; lam (device, internal layout) += scale dJ/df."""
    _check(lib().bgk_objective(ctx, case, _ptr(J) if J is not None else None, _ptr(lam) if lam is not None else None,
                               scale, _stream_ptr(stream)), ctx)


def bgk_adjoint_step(ctx, case: int, lam_in, lam_out, dtheta, stream=None) -> None:
    _check(lib().bgk_adjoint_step(ctx, case, _ptr(lam_in), _ptr(lam_out), _ptr(dtheta), _stream_ptr(stream)), ctx)


def bgk_neighbours_noalloc(dim: int, n: int, x, h: float, periodic: int, cap: int, cnt, col, check: int = 1,
                           stream=None) -> None:
    """Neighbour lists into caller-owned device tensors, without any device allocation.

    For callers that cannot allocate device memory.  x: [n, dim] float64, cnt: [n]
    int32, col: [n, cap] int32, all on the current CUDA device."""
    code = lib().bgk_neighbours_noalloc(dim, n, _ptr(x), h, periodic, cap, _ptr(cnt), _ptr(col), check,
                                        _stream_ptr(stream))
    if code != BGK_OK:
        raise BGKError(code, "bgk_neighbours_noalloc")


def bgk_shard_sizes(ctx, case: int):
    """Lengths (doubles) of the two exchange buffers of the sharded step: (xm, xw)."""
    a, b = C.c_int64(0), C.c_int64(0)
    _check(lib().bgk_shard_sizes(ctx, case, C.byref(a), C.byref(b)), ctx)
    return a.value, b.value


def bgk_shard_transport(ctx, case: int, xm, stream=None) -> None:
    _check(lib().bgk_shard_transport(ctx, case, _ptr(xm), _stream_ptr(stream)), ctx)


def bgk_shard_relax(ctx, case: int, xm, xw, stream=None) -> None:
    _check(lib().bgk_shard_relax(ctx, case, _ptr(xm), _ptr(xw) if xw is not None else None, _stream_ptr(stream)), ctx)


def bgk_shard_walls(ctx, case: int, xw, stream=None) -> None:
    _check(lib().bgk_shard_walls(ctx, case, _ptr(xw) if xw is not None else None, _stream_ptr(stream)), ctx)


def bgk_shard_partial(ctx, case: int, xm, stream=None) -> None:
    _check(lib().bgk_shard_partial(ctx, case, _ptr(xm), _stream_ptr(stream)), ctx)


def bgk_shard_set_moments(ctx, case: int, xm, stream=None) -> None:
    _check(lib().bgk_shard_set_moments(ctx, case, _ptr(xm), _stream_ptr(stream)), ctx)


def bgk_shard_allreduce(bufs: list, count: int, stream=None) -> None:
    """Elementwise sum of device buffers (tensors of float64) into each of them."""
    arr = (_P * len(bufs))(*[_ptr(b) for b in bufs])
    code = lib().bgk_shard_allreduce(arr, len(bufs), int(count), _stream_ptr(stream))
    if code != BGK_OK:
        raise BGKError(code, "bgk_shard_allreduce")


# ---- convenience ----

def params_from(p: dict) -> bgk_params:
    """bgk_params from a workload dict (dim, nv, vmax, kn, dt, h, alpha, ...)."""
    q = bgk_params()
    q.dim, q.nv, q.vmax, q.kn = int(p["dim"]), int(p["nv"]), float(p["vmax"]), float(p["kn"])
    q.tau_mode, q.ale, q.periodic = int(p.get("tau_mode", 0)), int(p.get("ale", 0)), int(p.get("periodic", 0))
    q.lid_wall, q.max_nbrs = int(p.get("lid_wall", 0)), int(p.get("max_nbrs", 48))
    st = p.get("storage", "f32")
    q.storage = STORAGE[st] if isinstance(st, str) else int(st)
    q.dt, q.h, q.alpha = float(p["dt"]), float(p["h"]), float(p["alpha"])
    q.wall_T, q.guard = float(p.get("wall_T", 1.0)), float(p.get("guard", 0.0))
    lu = list(p.get("lid_u", [0.0, 0.0, 0.0])) + [0.0, 0.0, 0.0]
    for a in range(3):
        q.lid_u[a] = float(lu[a])
    q.skin = float(p.get("skin", 0.2 if q.ale else 0.0))
    q.spare_points = int(p.get("spare_points", 0))
    q.body_wall = int(p.get("body_wall", 0))
    bu = list(p.get("body_u", [0.0, 0.0, 0.0])) + [0.0, 0.0, 0.0]
    bc = list(p.get("body_centre", [0.0, 0.0, 0.0])) + [0.0, 0.0, 0.0]
    for a in range(3):
        q.body_u[a] = float(bu[a])
        q.body_centre[a] = float(bc[a])
    q.body_radius = float(p.get("body_radius", 0.0))
    q.wls_order = int(p.get("wls_order", 1))
    q.vk_lo, q.vk_hi = int(p.get("vk_lo", 0)), int(p.get("vk_hi", 0))
    q.time_order = int(p.get("time_order", 1))
    q.vgrid = int(p.get("vgrid", 0))
    return q


class Solver:
    """One context holding one or more independent point clouds."""

    def __init__(self, params: list, clouds: list):
        self.params = [dict(p) for p in params]
        self.clouds = clouds
        self.n = [int(c["x"].shape[0]) for c in clouds]
        x = np.concatenate([np.ascontiguousarray(c["x"], dtype=np.float64).reshape(-1) for c in clouds])
        kind = np.concatenate([np.ascontiguousarray(c["kind"], dtype=np.int32) for c in clouds])
        normal = np.concatenate([np.ascontiguousarray(c["normal"], dtype=np.float64).reshape(-1) for c in clouds])
        self.ctx = bgk_init([params_from(p) for p in params], self.n, x, kind, normal)

    def close(self):
        if self.ctx:
            bgk_free(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def dims(self, case: int = 0):
        """(dim, ncomp, NV): NV velocities per row of f (those of the slab [vk_lo, vk_hi) if set)."""
        p = self.params[case]
        d = int(p["dim"])
        hi = int(p.get("vk_hi", 0))
        return d, (2 if d == 2 else 1), (hi - int(p.get("vk_lo", 0)) if hi else int(p["nv"]) ** d)

    def set_maxwellian(self, rho0=1.0, u0=(0.0, 0.0, 0.0), T0=1.0, stream=None):
        bgk_set_maxwellian(self.ctx, rho0, u0, T0, stream)

    def set_f(self, f, case: int = 0, stream=None):
        if isinstance(f, np.ndarray):
            dt = {np.dtype(np.float64): BGK_F64, np.dtype(np.float32): BGK_F32}[f.dtype]
        else:
            import torch
            dt = {torch.float64: BGK_F64, torch.float32: BGK_F32, torch.bfloat16: BGK_BF16}[f.dtype]
        bgk_set_f(self.ctx, case, f, dt, stream)

    def bind_f(self, f, case: int = 0, stream=None):
        """Keep case's distribution in the device tensor f ([n + spare_points][ncomp][NV],
        the storage dtype) from now on; f[:n] holds the state after every call.  None
        unbinds.  The solver keeps a reference to f while it is bound."""
        if not hasattr(self, "_bound"):
            self._bound = {}
        bgk_bind_f(self.ctx, case, f, stream)
        if f is None:
            self._bound.pop(case, None)
        else:
            self._bound[case] = f

    def get_f(self, case: int = 0, dtype=np.float64):
        d, nc, NV = self.dims(case)
        out = np.zeros((self.n[case], nc, NV), dtype=dtype)
        bgk_get_f(self.ctx, case, out, BGK_F64 if out.dtype == np.float64 else BGK_F32)
        return out

    def neighbours(self, stream=None):
        bgk_neighbours(self.ctx, stream)

    def get_neighbours(self, case: int = 0):
        return bgk_get_neighbours(self.ctx, case, self.n[case])

    def get_stencils(self, case: int = 0):
        rowptr, _ = self.get_neighbours(case)
        return bgk_get_stencils(self.ctx, case, int(rowptr[-1]), int(self.params[case]["dim"]))

    def step(self, nsteps: int = 1, stream=None):
        bgk_step(self.ctx, nsteps, stream)

    def manage(self, rmin: float, min_nbrs: int, case: int = 0, stream=None):
        """Point management pass; updates the point count; returns (n, removed, added)."""
        n, removed, added = bgk_manage(self.ctx, case, rmin, min_nbrs, stream)
        self.n[case] = n
        return n, removed, added

    def sync(self, stream=None):
        bgk_sync(self.ctx, stream)

    def moments(self, case: int = 0):
        d = int(self.params[case]["dim"])
        n = self.n[case]
        rho, u, T = np.zeros(n), np.zeros((n, d)), np.zeros(n)
        bgk_moments(self.ctx, case, rho, u, T)
        return rho, u, T

    def positions(self, case: int = 0):
        d = int(self.params[case]["dim"])
        x = np.zeros((self.n[case], d))
        bgk_get_positions(self.ctx, case, x)
        return x

    def body_centre(self, case: int = 0):
        """Current centre of case's moving body."""
        return bgk_get_body(self.ctx, case, int(self.params[case]["dim"]))

    def stats(self):
        return bgk_get_stats(self.ctx)
