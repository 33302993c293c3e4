"""FP64 CPU oracle for the meshfree ALE / WLS scheme for the BGK equation.

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the CPU
baseline leg of ``bench.py`` may use it; the CUDA library never does.  The
arithmetic lives in ``bgk_oracle.c`` (plain C, IEEE double, no fused
multiply-add); this module builds it with gcc and wraps it with ctypes and
numpy.  Every function names the passage of arXiv 2408.02350 it follows.

Parity status: every function is pinned by a test of ``tests/test_oracle_*``
against closed forms, invariants, brute force or the paper's printed numbers.
The driven-cavity flow fields themselves have no printed values in the paper
(its figures carry no data), so they rest on those pins and on GPU parity.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "bgk_oracle.c")
_OUT = os.path.join(_HERE, "_build", "liboracle.so")
_OUT_OMP = os.path.join(_HERE, "_build", "liboracle_omp.so")
_lock = threading.Lock()
_handle = None
_handle_omp = None

OK, E_OVERFLOW, E_SINGULAR, E_INVAL, E_NOMEM = 0, 1, 2, 3, 4


def build(force: bool = False, omp: bool = False) -> str:
    """Compile bgk_oracle.c into oracle/_build/liboracle.so (gcc -O2, no FMA contraction);
    with omp=True into liboracle_omp.so with -fopenmp (the loops over points split among
    threads, every point computed as in the plain build; used to time the oracle on all
    host cores)."""
    out = _OUT_OMP if omp else _OUT
    os.makedirs(os.path.dirname(out), exist_ok=True)
    import hashlib
    import platform
    with open(_SRC, "rb") as fh:
        stamp = hashlib.sha256(fh.read() + platform.machine().encode()).hexdigest()
    stamp_path = out + ".stamp"
    old = ""
    if os.path.exists(stamp_path):
        with open(stamp_path) as fh:
            old = fh.read()
    if force or old != stamp or not os.path.exists(out):
        tmp = out + ".%d.tmp" % os.getpid()
        cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off",
               "-fno-fast-math"] + (["-fopenmp"] if omp else []) + ["-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, out)
        with open(stamp_path, "w") as fh:
            fh.write(stamp)
    return out


class Params(C.Structure):
    _fields_ = [
        ("dim", C.c_int32), ("nv", C.c_int32), ("vmax", C.c_double), ("kn", C.c_double),
        ("tau_mode", C.c_int32), ("ale", C.c_int32), ("periodic", C.c_int32),
        ("lid_wall", C.c_int32), ("max_nbrs", C.c_int32), ("pad_", C.c_int32),
        ("dt", C.c_double), ("h", C.c_double), ("alpha", C.c_double), ("wall_T", C.c_double),
        ("guard", C.c_double), ("lid_u", C.c_double * 3),
        ("body_wall", C.c_int32), ("wls_order", C.c_int32), ("body_u", C.c_double * 3),
        ("body_c", C.c_double * 3), ("body_r", C.c_double), ("time_order", C.c_int32), ("vgrid", C.c_int32),
    ]


def params(p: dict) -> Params:
    """Oracle parameter block from a workload dict (see bgk_inputs)."""
    q = Params()
    q.dim, q.nv, q.vmax, q.kn = int(p["dim"]), int(p["nv"]), float(p["vmax"]), float(p["kn"])
    q.tau_mode, q.ale, q.periodic = int(p.get("tau_mode", 0)), int(p.get("ale", 0)), int(p.get("periodic", 0))
    q.lid_wall, q.max_nbrs = int(p.get("lid_wall", 0)), int(p.get("max_nbrs", 48))
    q.dt, q.h, q.alpha = float(p["dt"]), float(p["h"]), float(p["alpha"])
    q.wall_T, q.guard = float(p.get("wall_T", 1.0)), float(p.get("guard", 0.0))
    lu = list(p.get("lid_u", [0.0, 0.0, 0.0])) + [0.0, 0.0, 0.0]
    for a in range(3):
        q.lid_u[a] = float(lu[a])
    q.body_wall = int(p.get("body_wall", 0))
    bu = list(p.get("body_u", [0.0, 0.0, 0.0])) + [0.0, 0.0, 0.0]
    bc = list(p.get("body_centre", [0.0, 0.0, 0.0])) + [0.0, 0.0, 0.0]
    for a in range(3):
        q.body_u[a] = float(bu[a])
        q.body_c[a] = float(bc[a])
    q.body_r = float(p.get("body_radius", 0.0))
    q.wls_order = int(p.get("wls_order", 1))
    q.time_order = int(p.get("time_order", 1))
    q.vgrid = int(p.get("vgrid", 0))
    return q


_PD = C.POINTER(C.c_double)
_PI = C.POINTER(C.c_int32)
_PL = C.POINTER(C.c_int64)
_PP = C.POINTER(Params)


def lib(omp: bool = False):
    """The plain oracle library, or with omp=True its OpenMP build."""
    global _handle, _handle_omp
    with _lock:
        if (_handle_omp if omp else _handle) is None:
            h = C.CDLL(build(omp=omp))
            sig = {
                "or_dv": (C.c_double, [C.c_int32, C.c_double]),
                "or_velocity_nodes": (None, [C.c_int32, C.c_double, _PD]),
                "or_velocity_grid": (None, [C.c_int32, C.c_int32, C.c_double, _PD]),
                "or_dv_g": (C.c_double, [C.c_int32, C.c_double, C.c_int32]),
                "or_velocity_nodes_g": (None, [C.c_int32, C.c_double, C.c_int32, _PD]),
                "or_velocity_grid_g": (None, [C.c_int32, C.c_int32, C.c_double, C.c_int32, _PD]),
                "or_tau_si": (C.c_double, [C.c_double] * 5),
                "or_lambda_si": (C.c_double, [C.c_double] * 4),
                "or_tau": (C.c_double, [_PP, C.c_double, C.c_double]),
                "or_maxwellian": (None, [_PP, C.c_double, _PD, C.c_double, _PD]),
                "or_moments_point": (None, [_PP, _PD, _PD, _PD, _PD]),
                "or_neighbours_brute": (C.c_int64, [C.c_int32, C.c_int64, _PD, C.c_double, C.c_int32, C.c_int32, _PI, _PI]),
                "or_neighbours_cells": (C.c_int64, [C.c_int32, C.c_int64, _PD, C.c_double, C.c_int32, C.c_int32, _PI, _PI]),
                "or_frame": (None, [C.c_int32, _PD, _PD]),
                "or_stencils": (C.c_int, [_PP, C.c_int64, _PD, _PI, _PI, _PI, _PD, _PD, _PD, _PD]),
                "or_transport": (None, [_PP, C.c_int64, _PI, _PI, _PI, _PD, _PD, _PD, _PD, _PD]),
                "or_moments": (None, [_PP, C.c_int64, _PD, _PD, _PD, _PD]),
                "or_relax": (None, [_PP, C.c_int64, _PI, _PD, _PD, _PD, _PD, _PD]),
                "or_relax_exact": (None, [_PP, C.c_int64, _PI, _PD, C.c_double]),
                "or_transport_relax_points": (None, [_PP, C.c_int64, _PL, _PI, _PI, _PD, _PD, _PD, _PD, _PD, _PD]),
                "or_boundary": (C.c_int, [_PP, C.c_int64, _PI, _PD, _PI, _PI, _PD, _PD, _PD, _PD, _PD]),
                "or_move": (C.c_int64, [_PP, C.c_int64, _PI, _PD, _PD]),
                "or_init_maxwellian": (None, [_PP, C.c_int64, C.c_double, _PD, C.c_double, _PD, _PD, _PD, _PD]),
                "or_run": (C.c_int, [_PP, C.c_int64, _PD, _PI, _PD, _PD, _PD, _PD, _PD, C.c_int32, _PL]),
                "or_adjoint_step": (C.c_int, [_PP, C.c_int64, _PI, _PD, _PI, _PI, _PD, _PD, _PD, _PD, _PD, _PD, _PD]),
                "or_objective": (C.c_double, [_PP, C.c_int64, _PI, _PD, _PD, C.c_double]),
                "or_manage": (C.c_int64, [_PP, C.c_int64, _PD, _PI, _PD, _PD, _PI, _PI, C.c_double, C.c_int32,
                                          C.c_int64, _PD, _PI, _PD, _PD, _PL, _PL]),
                "or_threads": (C.c_int, []),
            }
            for name, (res, args) in sig.items():
                fn = getattr(h, name)
                fn.restype = res
                fn.argtypes = args
            if omp:
                _handle_omp = h
            else:
                _handle = h
    return _handle_omp if omp else _handle


def threads(omp: bool = False) -> int:
    """Threads the oracle's loops over points use (1 for the plain build)."""
    return int(lib(omp).or_threads())


def _d(a):
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(_PD)


def _i(a):
    assert a.dtype == np.int32 and a.flags.c_contiguous
    return a.ctypes.data_as(_PI)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _i32(a):
    return np.ascontiguousarray(a, dtype=np.int32)


def ncomp(dim: int) -> int:
    return 2 if dim == 2 else 1


def nvel(dim: int, nv: int) -> int:
    return nv ** dim


# ---- velocity grid (Sec. 3.3) ----

def dv(nv: int, vmax: float, vgrid: int = 0) -> float:
    """Node spacing: 2 vmax / (nv - 1) on the paper's endpoint grid, 2 vmax / nv on the
    midpoint grid (vgrid 1)."""
    return lib().or_dv_g(nv, vmax, vgrid)


def velocity_nodes(nv: int, vmax: float, vgrid: int = 0) -> np.ndarray:
    out = np.empty(nv)
    lib().or_velocity_nodes_g(nv, vmax, vgrid, _d(out))
    return out


def velocity_grid(dim: int, nv: int, vmax: float, vgrid: int = 0) -> np.ndarray:
    out = np.empty((nv ** dim, dim))
    lib().or_velocity_grid_g(dim, nv, vmax, vgrid, _d(out))
    return out


# ---- kinetic model (Sec. 2) ----

def tau_si(kb, R, diam, rho, T) -> float:
    return lib().or_tau_si(kb, R, diam, rho, T)


def lambda_si(kb, R, diam, rho) -> float:
    return lib().or_lambda_si(kb, R, diam, rho)


def tau(p: dict, rho: float, T: float) -> float:
    q = params(p)
    return lib().or_tau(C.byref(q), rho, T)


def maxwellian(p: dict, rho: float, U, T: float) -> np.ndarray:
    """[ncomp, NV] Maxwellian (3D) or Chu pair (G1, G2) (2D)."""
    q = params(p)
    U = _f64(np.resize(np.asarray(U, dtype=np.float64), 3))
    out = np.empty((ncomp(p["dim"]), nvel(p["dim"], p["nv"])))
    lib().or_maxwellian(C.byref(q), rho, _d(U), T, _d(out))
    return out


def moments_point(p: dict, fi: np.ndarray):
    q = params(p)
    fi = _f64(fi)
    rho, T, U = np.empty(1), np.empty(1), np.empty(3)
    lib().or_moments_point(C.byref(q), _d(fi), _d(rho), _d(U), _d(T))
    return float(rho[0]), U[: p["dim"]].copy(), float(T[0])


def moments(p: dict, f: np.ndarray):
    q = params(p)
    f = _f64(f)
    n = f.shape[0]
    rho, T, U = np.empty(n), np.empty(n), np.empty((n, p["dim"]))
    lib().or_moments(C.byref(q), n, _d(f), _d(rho), _d(U), _d(T))
    return rho, U, T


# ---- neighbours (Sec. 3.5.1, Sec. 4.2) ----

def neighbours(x: np.ndarray, h: float, periodic: bool = False, cap: int = 48, method: str = "cells"):
    """(cnt [n], col [n, cap]) ELL lists, ascending per row; raises on overflow."""
    x = _f64(x)
    n, dim = x.shape
    cnt = np.zeros(n, dtype=np.int32)
    col = np.full((n, cap), -1, dtype=np.int32)
    fn = lib().or_neighbours_cells if method == "cells" else lib().or_neighbours_brute
    nnz = fn(dim, n, _d(x), h, int(periodic), cap, _i(cnt), _i(col))
    if nnz < 0:
        raise OverflowError("neighbour list overflow (max count %d > cap %d)" % (cnt.max(), cap))
    return cnt, col


def to_csr(cnt: np.ndarray, col: np.ndarray):
    rowptr = np.zeros(len(cnt) + 1, dtype=np.int64)
    rowptr[1:] = np.cumsum(cnt)
    cols = np.concatenate([col[i, : cnt[i]] for i in range(len(cnt))]) if len(cnt) else np.zeros(0, np.int32)
    return rowptr, cols.astype(np.int32)


# ---- stencils (Sec. 3.4) ----

def frame(dim: int, dr) -> np.ndarray:
    dr = _f64(dr)
    out = np.empty((dim, dim))
    lib().or_frame(dim, _d(dr), _d(out))
    return out


def stencils(p: dict, x, kind, cnt, col) -> dict:
    q = params(p)
    x, kind, cnt, col = _f64(x), _i32(kind), _i32(cnt), _i32(col)
    n, dim = x.shape
    cap = q.max_nbrs
    assert col.shape == (n, cap)
    coef = np.empty((n, cap, dim))
    abar = np.empty((n, cap, dim))
    frm = np.empty((n, cap, dim, dim))
    recon = np.empty((n, cap))
    st = lib().or_stencils(C.byref(q), n, _d(x), _i(kind), _i(cnt), _i(col), _d(coef), _d(abar), _d(frm), _d(recon))
    if st != OK:
        raise ArithmeticError("or_stencils: singular WLS system (status %d)" % st)
    return {"coef": coef, "abar": abar, "frame": frm, "recon": recon}


# ---- step pieces (Sec. 3.2, 3.4.2, 5) ----

def transport(p: dict, kind, cnt, col, st: dict, U, f) -> np.ndarray:
    q = params(p)
    kind, cnt, col, f = _i32(kind), _i32(cnt), _i32(col), _f64(f)
    U = _f64(U)
    ft = np.empty_like(f)
    lib().or_transport(C.byref(q), f.shape[0], _i(kind), _i(cnt), _i(col), _d(_f64(st["abar"])),
                       _d(_f64(st["frame"])), _d(U), _d(f), _d(ft))
    return ft


def relax(p: dict, kind, ft, f, rho, U, T):
    """In place on f, rho, U, T (interior points)."""
    q = params(p)
    lib().or_relax(C.byref(q), ft.shape[0], _i(_i32(kind)), _d(_f64(ft)), _d(f), _d(rho), _d(U), _d(T))


def transport_relax_points(p: dict, idx, cnt, col, st: dict, U, f):
    """f^{n+1} and (rho, U, T) of the listed interior points after one transport + relaxation."""
    q = params(p)
    idx = np.ascontiguousarray(idx, dtype=np.int64)
    f = _f64(f)
    dim = p["dim"]
    out = np.empty((len(idx),) + f.shape[1:])
    mom = np.empty((len(idx), dim + 2))
    lib().or_transport_relax_points(C.byref(q), len(idx), idx.ctypes.data_as(_PL), _i(_i32(cnt)), _i(_i32(col)),
                                    _d(_f64(st["abar"])), _d(_f64(st["frame"])), _d(_f64(U)), _d(f), _d(out), _d(mom))
    return out, mom[:, 0], mom[:, 1:1 + dim], mom[:, 1 + dim]


def relax_exact(p: dict, kind, f, h: float) -> None:
    """In place on f: the exact relaxation over a time h at every interior point,
    f = M + (f - M) exp(-h / tau) with M, tau from the moments of f."""
    q = params(p)
    assert f.dtype == np.float64 and f.flags.c_contiguous
    lib().or_relax_exact(C.byref(q), f.shape[0], _i(_i32(kind)), _d(f), float(h))


def boundary(p: dict, kind, normal, cnt, col, st: dict, f, rho, U, T) -> int:
    q = params(p)
    return lib().or_boundary(C.byref(q), f.shape[0], _i(_i32(kind)), _d(_f64(normal)), _i(_i32(cnt)),
                             _i(_i32(col)), _d(_f64(st["recon"])), _d(f), _d(rho), _d(U), _d(T))


def move(p: dict, kind, U, x) -> int:
    """x += dt U in place (Eqs. originalALE1, ALE1) with the wall and body guards; with a
    body, its points move with it and p['body_centre'] advances.  Returns the clamps."""
    q = params(p)
    c = lib().or_move(C.byref(q), x.shape[0], _i(_i32(kind)), _d(_f64(U)), _d(x))
    if q.body_wall > 0:
        p["body_centre"] = [float(q.body_c[a]) for a in range(3)]
    return c


def manage(p: dict, x, kind, normal, f, cnt, col, rmin: float, min_nbrs: int, cap_out: int | None = None):
    """One pass of point management (Sec. 3.5.2): remove interior points closer than rmin
    to a wall point, merge mutually nearest remaining interior pairs closer than rmin at
    their midpoint, add points into holes next to interior points with fewer than
    min_nbrs neighbours; f at new positions by linear WLS reconstruction.  Returns
    dict(x, kind, normal, f, origin, merges, adds, wall_removals)."""
    q = params(p)
    x, f = _f64(x), _f64(f)
    n, dim = x.shape
    cap_out = int(cap_out if cap_out is not None else 2 * n)
    xo = np.zeros((cap_out, dim))
    ko = np.zeros(cap_out, dtype=np.int32)
    no = np.zeros((cap_out, dim))
    fo = np.zeros((cap_out,) + f.shape[1:])
    org = np.zeros(cap_out, dtype=np.int64)
    counts = np.zeros(3, dtype=np.int64)
    m = lib().or_manage(C.byref(q), n, _d(x), _i(_i32(kind)), _d(_f64(normal)), _d(f), _i(_i32(cnt)), _i(_i32(col)),
                        float(rmin), int(min_nbrs), cap_out, _d(xo), _i(ko), _d(no), _d(fo),
                        org.ctypes.data_as(_PL), counts.ctypes.data_as(_PL))
    if m < 0:
        raise MemoryError("or_manage")
    return {"x": xo[:m].copy(), "kind": ko[:m].copy(), "normal": no[:m].copy(), "f": fo[:m].copy(),
            "origin": org[:m].copy(), "merges": int(counts[0]), "adds": int(counts[1]),
            "wall_removals": int(counts[2])}


def adjoint_step(p: dict, kind, normal, cnt, col, st: dict, f, lam1):
    """(lam0, dtheta): lam0 = (dPhi/df)^T lam1 at state f; dtheta = [dJ/du_lid (3), dJ/dKn]."""
    q = params(p)
    f, lam1 = _f64(f), _f64(lam1)
    lam0 = np.empty_like(f)
    dth = np.zeros(4)
    lib().or_adjoint_step(C.byref(q), f.shape[0], _i(_i32(kind)), _d(_f64(normal)), _i(_i32(cnt)), _i(_i32(col)),
                          _d(_f64(st["abar"])), _d(_f64(st["frame"])), _d(_f64(st["recon"])), _d(f), _d(lam1),
                          _d(lam0), _d(dth))
    return lam0, dth


def objective(p: dict, kind, f, lam=None, scale: float = 1.0) -> float:
    """Lid x-momentum flux of state f; adds scale * dJ/df to lam when given."""
    q = params(p)
    f = _f64(f)
    lp = _d(lam) if lam is not None else None
    return lib().or_objective(C.byref(q), f.shape[0], _i(_i32(kind)), _d(f), lp, scale)


class Simulation:
    """State (x, f, rho, U, T) of one point cloud advanced by ``or_run``."""

    def __init__(self, p: dict, cloud: dict, rho0: float = 1.0, U0=(0.0, 0.0, 0.0), T0: float = 1.0, f0=None,
                 omp: bool = False):
        self.omp = omp  # run() through the OpenMP build (timing on all host cores)
        self.p = dict(p)
        self.q = params(p)
        self.x = _f64(cloud["x"]).copy()
        self.kind = _i32(cloud["kind"])
        self.normal = _f64(cloud["normal"])
        n, dim = self.x.shape
        self.n, self.dim = n, dim
        row = ncomp(dim) * nvel(dim, p["nv"])
        self.f = np.empty((n, ncomp(dim), nvel(dim, p["nv"])))
        self.rho, self.U, self.T = np.empty(n), np.empty((n, dim)), np.empty(n)
        U0 = _f64(np.resize(np.asarray(U0, dtype=np.float64), 3))
        lib().or_init_maxwellian(C.byref(self.q), n, rho0, _d(U0), T0, _d(self.f), _d(self.rho), _d(self.U), _d(self.T))
        if f0 is not None:
            self.f[...] = np.asarray(f0, dtype=np.float64).reshape(self.f.shape)
            self.rho, self.U, self.T = moments(self.p, self.f)
        self.clamps = 0
        self.steps = 0
        assert self.f.size == n * row

    def gradient(self, nsteps: int):
        """J = (1/N) sum_{n=1..N} J(f^n) from the current state, and its gradient with respect to
        (u_lid, Kn) and to the current f, by storing every state and sweeping the adjoint backwards.
        Fixed points only.  The state is advanced by nsteps."""
        assert not self.p.get("ale"), "the adjoint is for fixed points"
        cnt, col = neighbours(self.x, self.p["h"], bool(self.p.get("periodic")), int(self.p.get("max_nbrs", 48)))
        st = stencils(self.p, self.x, self.kind, cnt, col)
        states = [self.f.copy()]
        J = 0.0
        for _ in range(nsteps):
            self.run(1)
            states.append(self.f.copy())
            J += objective(self.p, self.kind, self.f) / nsteps
        lam = np.zeros_like(self.f)
        objective(self.p, self.kind, states[nsteps], lam, 1.0 / nsteps)
        dth = np.zeros(4)
        for k in range(nsteps - 1, -1, -1):
            lam, d = adjoint_step(self.p, self.kind, self.normal, cnt, col, st, states[k], lam)
            dth += d
            if k >= 1:
                objective(self.p, self.kind, states[k], lam, 1.0 / nsteps)
        return J, dth, lam

    def run(self, nsteps: int) -> None:
        cl = np.zeros(1, dtype=np.int64)
        st = lib(self.omp).or_run(C.byref(self.q), self.n, _d(self.x), _i(self.kind), _d(self.normal), _d(self.f),
                          _d(self.rho), _d(self.U), _d(self.T), nsteps, cl.ctypes.data_as(_PL))
        if st != OK:
            raise RuntimeError("oracle or_run failed with status %d" % st)
        self.clamps += int(cl[0])
        self.steps += nsteps
        if self.q.body_wall > 0:
            self.p["body_centre"] = self.body_c.tolist() + [0.0] * (3 - self.dim)

    @property
    def body_c(self) -> np.ndarray:
        """Current centre of the moving body."""
        return np.array([self.q.body_c[a] for a in range(self.dim)])
