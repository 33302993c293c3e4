"""Gradients of the time-averaged lid flux through the discrete adjoint of bgk_step.

J = (1/N) sum_{n=1..N} J(f^n), J(f) the x-momentum flux through the lid plane
averaged over the lid points (bgk_objective).  gradient() returns J and
dJ/du_lid, dJ/dKn, dJ/df^0 for a fixed-point case, using uniform checkpointing:
the forward pass keeps f every `checkpoint_every` steps; the reverse pass
recomputes one segment at a time (keeping its states) and sweeps
bgk_adjoint_step backwards through it.  Device memory: N/K + K copies of f.
All arithmetic runs in the library's kernels; torch provides buffers and the
stream.  LidFluxObjective wraps gradient() as a torch.autograd.Function.
"""
from __future__ import annotations

import math

import torch

from . import (BGK_BF16, BGK_F32, BGK_F64, bgk_adjoint_step, bgk_get_f, bgk_objective, bgk_set_f,
               bgk_set_params, bgk_step, bgk_sync, params_from)

_TORCH = {BGK_F64: torch.float64, BGK_F32: torch.float32, BGK_BF16: torch.bfloat16}


def _dims(solver, case):
    p = solver.params[case]
    d = int(p["dim"])
    nc = 2 if d == 2 else 1
    NV = int(p["nv"]) ** d
    nvp = solver.stats()["nv_pad"]
    return d, nc, NV, nvp


def _storage(solver, case):
    st = solver.params[case].get("storage", "f32")
    return {"f64": BGK_F64, "f32": BGK_F32, "bf16": BGK_BF16}[st] if isinstance(st, str) else int(st)


def gradient(solver, nsteps: int, checkpoint_every: int = 50, case: int = 0, f0: torch.Tensor | None = None,
             stream=None):
    """(J, dJ/du_lid [3], dJ/dKn, dJ/df0 [n, ncomp, NV]) from the case's current state (or f0)."""
    assert not solver.params[case].get("ale"), "the discrete adjoint is for fixed points"
    dev = torch.device("cuda", torch.cuda.current_device())
    st = _storage(solver, case)
    sdt = _TORCH[st]
    cdt = torch.float64 if st == BGK_F64 else torch.float32
    d, nc, NV, nvp = _dims(solver, case)
    n = solver.n[case]
    ctx = solver.ctx
    if f0 is not None:
        bgk_set_f(ctx, case, f0.contiguous(), st, stream)
    K = max(1, min(checkpoint_every, nsteps))
    nseg = int(math.ceil(nsteps / K))
    ckpt = []
    J = torch.zeros(1, dtype=torch.float64, device=dev)
    for s in range(nseg):
        buf = torch.empty((n, nc, NV), dtype=sdt, device=dev)
        bgk_get_f(ctx, case, buf, st, stream)
        ckpt.append(buf)
        for _ in range(min(K, nsteps - s * K)):
            bgk_step(ctx, 1, stream)
            bgk_objective(ctx, case, J, None, 1.0, stream)
    J = J / nsteps
    lam = torch.zeros((n, nc, nvp), dtype=cdt, device=dev)
    lam2 = torch.zeros_like(lam)
    dth = torch.zeros(4, dtype=torch.float64, device=dev)
    bgk_objective(ctx, case, None, lam, 1.0 / nsteps, stream)  # dJ/df^N (current state is f^N)
    for s in range(nseg - 1, -1, -1):
        steps = min(K, nsteps - s * K)
        bgk_set_f(ctx, case, ckpt[s], st, stream)
        states = [ckpt[s]]
        for _ in range(steps - 1):
            bgk_step(ctx, 1, stream)
            buf = torch.empty((n, nc, NV), dtype=sdt, device=dev)
            bgk_get_f(ctx, case, buf, st, stream)
            states.append(buf)
        for k in range(steps - 1, -1, -1):
            bgk_set_f(ctx, case, states[k], st, stream)
            bgk_adjoint_step(ctx, case, lam, lam2, dth, stream)
            lam, lam2 = lam2, lam
            if s * K + k >= 1:
                bgk_objective(ctx, case, None, lam, 1.0 / nsteps, stream)
    bgk_sync(ctx, stream)
    return float(J.item()), dth[:3].cpu().numpy(), float(dth[3].item()), lam[..., :NV].contiguous()


class LidFluxObjective(torch.autograd.Function):
    """J(f0, u_lid_x, Kn) = time-averaged lid flux over `nsteps` steps; backward by the discrete adjoint."""

    @staticmethod
    def forward(ctx, f0, lid_u, kn, solver, nsteps: int, checkpoint_every: int = 50, case: int = 0):
        p = dict(solver.params[case])
        p["lid_u"] = [float(lid_u), 0.0, 0.0]
        p["kn"] = float(kn)
        solver.params[case] = p
        bgk_set_params(solver.ctx, case, params_from(p))
        J, du, dkn, lam0 = gradient(solver, nsteps, checkpoint_every, case, f0=f0)
        ctx.save_for_backward(lam0)
        ctx.du, ctx.dkn = float(du[0]), dkn
        return torch.tensor(J, dtype=torch.float64)

    @staticmethod
    def backward(ctx, gJ):
        (lam0,) = ctx.saved_tensors
        g = float(gJ)
        return (lam0 * g, torch.tensor(ctx.du * g, dtype=torch.float64), torch.tensor(ctx.dkn * g, dtype=torch.float64),
                None, None, None, None)
