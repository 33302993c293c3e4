"""Seeded synthetic inputs for the meshfree BGK driven-cavity workloads.

This module is shared by the FP64 CPU oracle (``oracle/``) and the CUDA
library (``paper_2408_02350_gb300``).  It holds geometry and parameters only:
point clouds, wall kinds, inward normals, and the configuration of each
workload.  It contains none of the method's arithmetic (no velocity grid, no
Maxwellian, no stencils), so neither side can inherit a mistake from the
other through it.

Geometry (Sec. 3.4 and Sec. 5 of arXiv 2408.02350): a unit square or cube
with boundary points on the walls and interior points that start on a
regular lattice.  The lattice spacing is dx = 1/(n-1).  Interior points get
i.i.d. uniform jitter in [-0.1 dx, 0.1 dx] per coordinate.  The jitter comes
from a SplitMix64 stream (Steele, Lea and Flood, OOPSLA 2014), one draw per
(point, axis) in point-major order.  Boundary points are not jittered.

Point order is lattice order with x fastest: p = ix + n*(iy + n*iz).

Wall kinds (the cavity walls of Sec. 5.1 and 5.2):
  0          interior point
  1, 2       faces x = 0 and x = 1
  3, 4       faces y = 0 and y = 1
  5, 6       faces z = 0 and z = 1 (3D only)
  2*dim + 1  edge or corner point: a wall at rest whose inward normal is the
             normalised sum of the adjacent face normals
  2*dim + 2  boundary point of a rigid body (a disc in 2D, a ball in 3D) that
             moves through the gas with a constant velocity (Sec. 3.4.1)
The lid is face y = 1 in 2D (kind 4) and face z = 1 in 3D (kind 6).  Only
points strictly inside the lid face move with the lid velocity.
"""
from __future__ import annotations

import json
import math
import os

import numpy as np

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(seed: int, count: int, start: int = 0) -> np.ndarray:
    """Outputs start..start+count-1 of the SplitMix64 stream seeded with ``seed``.

    Output k is mix(seed + (k+1) * 0x9E3779B97F4A7C15) with the published
    finaliser (xor-shift 30, multiply, xor-shift 27, multiply, xor-shift 31).
    """
    k = np.arange(start + 1, start + count + 1, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + k * _GOLDEN
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


def uniform01(seed: int, count: int, start: int = 0) -> np.ndarray:
    """Doubles in [0, 1): the top 53 bits of each SplitMix64 output times 2^-53."""
    z = splitmix64(seed, count, start)
    return (z >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


def cavity(dim: int, n: int, seed: int, jitter: float = 0.1) -> dict:
    """Jittered lattice in the unit square (dim=2) or cube (dim=3).

    Returns x [N, dim] float64, kind [N] int32, normal [N, dim] float64
    (inward unit normal, zero for interior points), dx, lid_wall and n.
    """
    if dim not in (2, 3) or n < 3:
        raise ValueError("cavity: dim must be 2 or 3 and n >= 3")
    dx = 1.0 / (n - 1)
    idx = np.indices((n,) * dim).reshape(dim, -1)[::-1].T  # columns (ix, iy[, iz]), x fastest
    npts = idx.shape[0]
    x = idx.astype(np.float64) * dx
    x[idx == n - 1] = 1.0  # exact wall coordinate
    on_lo = idx == 0
    on_hi = idx == n - 1
    nwalls = (on_lo | on_hi).sum(axis=1)
    kind = np.zeros(npts, dtype=np.int32)
    normal = np.zeros((npts, dim), dtype=np.float64)
    for a in range(dim):
        normal[on_lo[:, a], a] += 1.0
        normal[on_hi[:, a], a] -= 1.0
        kind[(nwalls == 1) & on_lo[:, a]] = 2 * a + 1
        kind[(nwalls == 1) & on_hi[:, a]] = 2 * a + 2
    kind[nwalls >= 2] = 2 * dim + 1
    nrm = np.sqrt((normal * normal).sum(axis=1))
    wall = nrm > 0
    normal[wall] /= nrm[wall, None]
    interior = kind == 0
    u = uniform01(seed, npts * dim).reshape(npts, dim)
    jit = (2.0 * u - 1.0) * (jitter * dx)
    x[interior] += jit[interior]
    return {"x": x, "kind": kind, "normal": normal, "dx": dx, "n": n,
            "lid_wall": 2 * dim, "dim": dim}


def periodic_box(dim: int, n: int, seed: int | None = None, jitter: float = 0.0) -> dict:
    """n^dim points on the periodic unit box, spacing 1/n, all interior."""
    dx = 1.0 / n
    idx = np.indices((n,) * dim).reshape(dim, -1)[::-1].T
    x = idx.astype(np.float64) * dx
    if seed is not None and jitter > 0.0:
        u = uniform01(seed, x.size).reshape(x.shape)
        x = np.mod(x + (2.0 * u - 1.0) * (jitter * dx), 1.0)
    npts = x.shape[0]
    return {"x": x, "kind": np.zeros(npts, dtype=np.int32),
            "normal": np.zeros((npts, dim)), "dx": dx, "n": n, "lid_wall": 0, "dim": dim}


def with_body(cl: dict, centre, radius: float, wall: int) -> dict:
    """The cloud ``cl`` with a rigid body of the given centre and radius.

    Interior points closer than radius + dx/2 to the centre are removed.  The body's
    boundary points (kind ``wall``) follow the cloud's points, spaced about dx on the
    circle (2D: equal angles) or sphere (3D: a Fibonacci spiral, equal areas); their
    inward normal (into the gas) points away from the centre.
    """
    dim, dx = cl["dim"], cl["dx"]
    c = np.asarray(centre, dtype=np.float64)[:dim]
    x = cl["x"]
    r = np.sqrt(((x - c) ** 2).sum(axis=1))
    keep = ~((cl["kind"] == 0) & (r < radius + 0.5 * dx))
    if dim == 2:
        m = max(8, int(round(2.0 * math.pi * radius / dx)))
        th = 2.0 * math.pi * np.arange(m) / m
        nb = np.stack([np.cos(th), np.sin(th)], axis=1)
    else:
        m = max(12, int(round(4.0 * math.pi * radius * radius / (dx * dx))))
        k = np.arange(m, dtype=np.float64)
        z = 1.0 - (2.0 * k + 1.0) / m
        rho = np.sqrt(1.0 - z * z)
        phi = k * (math.pi * (3.0 - math.sqrt(5.0)))
        nb = np.stack([rho * np.cos(phi), rho * np.sin(phi), z], axis=1)
    xb = c[None, :] + radius * nb
    out = dict(cl)
    out["x"] = np.concatenate([x[keep], xb])
    out["kind"] = np.concatenate([cl["kind"][keep], np.full(m, wall, dtype=np.int32)])
    out["normal"] = np.concatenate([cl["normal"][keep], nb])
    out["body_wall"] = wall
    return out


def cfl_dt(dx: float, vmax: float, dim: int, cfl: float = 0.5) -> float:
    """Time step cfl * dx / max|v|, with max|v| = vmax*sqrt(dim) at the grid corner."""
    return cfl * dx / (vmax * math.sqrt(dim))


def _params(dim, n, nv, vmax, kn, lid, steps, storage, ale, seed, cfl=0.5):
    dx = 1.0 / (n - 1)
    lid_u = [0.0, 0.0, 0.0]
    lid_u[0] = lid
    return {
        "dim": dim, "n": n, "nv": nv, "vmax": vmax, "kn": kn,
        "tau_mode": 0, "dt": cfl_dt(dx, vmax, dim, cfl), "h": 2.5 * dx,
        "alpha": 6.25, "wall_T": 1.0, "lid_u": lid_u, "lid_wall": 2 * dim,
        "ale": int(ale), "periodic": 0, "guard": 0.1 * dx, "steps": steps,
        "storage": storage, "seed": seed, "dx": dx,
        "max_nbrs": 48 if dim == 2 else 160,
    }


# The five driven-cavity workloads.  Seeds: 2408000 + k for workload k.
CONFIGS = {
    # 2D lid-driven cavity, plain FP64 method: 41^2 points, 16^2 velocities in [-5,5]^2.
    "cavity2d_n41_v16_f64": _params(2, 41, 16, 5.0, 0.1, 0.1, 100, "f64", False, 2408001),
    # 2D cavity with ALE motion: 201^2 points, 32^2 velocities in [-6,6]^2, Kn 0.1 (sweep 0.01/0.1/1).
    "cavity2d_ale_n201_v32_f32": _params(2, 201, 32, 6.0, 0.1, 0.1, 2000, "f32", True, 2408002),
    # 3D lid-driven cavity: 41^3 points, 16^3 velocities in [-5,5]^3.
    "cavity3d_n41_v16_f32": _params(3, 41, 16, 5.0, 0.1, 0.1, 500, "f32", False, 2408003),
    # 2D cavity for the adjoint: 101^2 points, 24^2 velocities in [-5,5]^2.
    "adjoint2d_n101_v24_f32": _params(2, 101, 24, 5.0, 0.1, 0.1, 1000, "f32", False, 2408005),
}

def _body(p: dict, centre, radius: float, u) -> dict:
    q = dict(p)
    q["body_wall"] = 2 * p["dim"] + 2
    q["body_centre"] = list(centre) + [0.0] * (3 - len(centre))
    q["body_radius"] = radius
    q["body_u"] = list(u) + [0.0] * (3 - len(u))
    return q


# The ALE cavity with a disc of radius 0.1 starting at (0.4, 0.5) and moving with (0.1, 0).
CONFIGS["body2d_ale_n201_v32_f32"] = _body(
    _params(2, 201, 32, 6.0, 0.1, 0.1, 2000, "f32", True, 2408006), (0.4, 0.5), 0.1, (0.1, 0.0))
KN_SWEEP_ALE = (0.01, 0.1, 1.0)


def config(name: str, **overrides) -> dict:
    """A copy of workload ``name`` with keyword overrides applied."""
    p = dict(CONFIGS[name])
    p["lid_u"] = list(p["lid_u"])
    for k in ("body_u", "body_centre"):
        if k in p:
            p[k] = list(p[k])
    for k, v in overrides.items():
        p[k] = v
    if "n" in overrides and ("h" not in overrides):
        dx = 1.0 / (p["n"] - 1)
        p["dx"] = dx
        p["h"] = 2.5 * dx
        p["guard"] = 0.1 * dx
        if "dt" not in overrides:
            p["dt"] = cfl_dt(dx, p["vmax"], p["dim"])
    if "vmax" in overrides and "dt" not in overrides:
        p["dt"] = cfl_dt(p["dx"], p["vmax"], p["dim"])
    return p


# One JSON file per workload (the parameters of CONFIGS[name], written by
# write_workload_files); a copy with some parameters changed describes a variant.
WORKLOAD_DIR = os.path.join(os.path.dirname(os.path.abspath(__file__)), "workloads")


def write_workload_files(folder: str = WORKLOAD_DIR) -> list[str]:
    """Write folder/<name>.json = {"workload": name, "params": CONFIGS[name]} for every workload."""
    os.makedirs(folder, exist_ok=True)
    paths = []
    for name in sorted(CONFIGS):
        path = os.path.join(folder, name + ".json")
        with open(path, "w") as fh:
            json.dump({"workload": name, "params": CONFIGS[name]}, fh, indent=1, sort_keys=True)
            fh.write("\n")
        paths.append(path)
    return paths


def workload_from_file(path: str) -> tuple[str, dict]:
    """(name, overrides) of a workload file {"workload": a CONFIGS name, "params": {...}}:
    the overrides are the parameters that differ from the named workload, so that
    config(name, **overrides) gives the file's parameters back.  Unknown names and keys
    raise ValueError."""
    with open(path) as fh:
        d = json.load(fh)
    name = d.get("workload")
    if name not in CONFIGS:
        raise ValueError("%s: workload %r is not one of %s" % (path, name, sorted(CONFIGS)))
    base = CONFIGS[name]
    params = d.get("params", {})
    unknown = sorted(set(params) - set(base) - {"time_order", "wls_order", "vgrid", "spare_points", "skin"})
    if unknown:
        raise ValueError("%s: unknown parameters %s" % (path, unknown))
    return name, {k: v for k, v in params.items() if base.get(k) != v}


def batched_cases(count: int = 64, seed0: int = 2408400) -> list[dict]:
    """Independent 2D cavities for the batched sweep.

    Case b draws from SplitMix64 seed seed0 + b: side n uniform-integer in
    [41, 121], velocity nodes per axis uniform-integer in [16, 32],
    Kn = 10^U(-2, 0), lid speed U(0.05, 0.2); v_max = 5.  Its point cloud
    uses the same seed.
    """
    out = []
    for b in range(count):
        u = uniform01(seed0 + b, 4, start=1 << 20)
        n = 41 + int(u[0] * 81)
        nv = 16 + int(u[1] * 17)
        kn = 10.0 ** (-2.0 + 2.0 * u[2])
        lid = 0.05 + 0.15 * u[3]
        p = _params(2, n, nv, 5.0, kn, lid, 100, "f32", False, seed0 + b)
        out.append(p)
    return out


def cloud_for(p: dict) -> dict:
    """The point cloud of a workload dict (cavity, with a body when p['body_wall'], or
    periodic box when p['periodic'])."""
    if p.get("periodic"):
        return periodic_box(p["dim"], p["n"])
    cl = cavity(p["dim"], p["n"], p["seed"])
    if p.get("body_wall"):
        cl = with_body(cl, p["body_centre"], p["body_radius"], p["body_wall"])
    return cl
