"""Velocity-sharded stepping of one case: the discrete velocity grid split into slabs.

Transport and relaxation act on every discrete velocity separately (Sec. 3.2); the
velocities meet only in sums over the grid -- the moments of f~ (Eqs. fullmoment1a,
moment1a, moment1b) and, at a diffuse wall, the mass fluxes that fix rho_w and the wall
moments.  So a case can be split into slabs of its flattened velocity index, each slab
holding f for those velocities at every point, with positions, lists, stencils and
moments replicated.  One step of every slab is the library's three sharded calls with a
sum of two small buffers over all slabs between them (``bgk_shard_*`` in bgk.h):

    transport -> sum(xm) -> relax -> sum(xw) -> walls

The paper parallelises over points on one GPU (Sec. 5); this split is the library's
decomposition for several GPUs, one slab per rank with an allreduce of (dim + 2) n +
(2 dim + 6) n_wall doubles per step, against n ncomp NV / R values of f on each of R
ranks.  Slabs may also share one GPU, where ``bgk_shard_allreduce`` sums their buffers.

Everything here marshals calls: the arithmetic runs in the library's kernels and, for
ranks, in the collective of torch.distributed (NCCL between GPUs).
"""
from __future__ import annotations

from . import (BGK_E_INVAL, BGKError, Solver, bgk_set_maxwellian, bgk_shard_allreduce, bgk_shard_partial,
               bgk_shard_relax, bgk_shard_set_moments, bgk_shard_sizes, bgk_shard_transport, bgk_shard_walls)


def velocity_slabs(NV: int, parts: int, align: int = 4) -> list:
    """Split the flattened velocity index range [0, NV) into `parts` contiguous slabs
    [lo, hi) whose starts are multiples of `align` and whose sizes differ by at most
    `align` (the last one may be shorter by the ragged end of the grid)."""
    units = -(-int(NV) // align)
    if parts < 1 or parts > units:
        raise ValueError("cannot split %d velocities into %d slabs of %d-aligned starts" % (NV, parts, align))
    bounds = [min(int(NV), align * ((units * r) // parts)) for r in range(parts + 1)]
    return [(bounds[r], bounds[r + 1]) for r in range(parts)]


class Slab:
    """One velocity slab [lo, hi) of one case, in a library context of its own on the
    current CUDA device, with its two exchange buffers (device float64 tensors)."""

    def __init__(self, p: dict, cloud: dict, lo: int, hi: int):
        import torch
        self.p = dict(p, vk_lo=int(lo), vk_hi=int(hi))
        self.lo, self.hi = int(lo), int(hi)
        self.solver = Solver([self.p], [cloud])
        n_xm, n_xw = bgk_shard_sizes(self.solver.ctx, 0)
        self.xm = torch.zeros(n_xm, dtype=torch.float64, device="cuda")
        self.xw = torch.zeros(n_xw, dtype=torch.float64, device="cuda")

    @property
    def ctx(self):
        return self.solver.ctx

    def _xw(self):
        return self.xw if self.xw.numel() else None

    def set_maxwellian(self, rho0, u0, T0, stream=None):
        bgk_set_maxwellian(self.ctx, rho0, u0, T0, stream)

    def set_f(self, f, stream=None):
        """f: this slab's rows [n][ncomp][hi - lo] (host or device)."""
        self.solver.set_f(f, 0, stream)

    def partial(self, stream=None):
        bgk_shard_partial(self.ctx, 0, self.xm, stream)

    def set_moments(self, stream=None):
        bgk_shard_set_moments(self.ctx, 0, self.xm, stream)

    def transport(self, stream=None):
        bgk_shard_transport(self.ctx, 0, self.xm, stream)

    def relax(self, stream=None):
        bgk_shard_relax(self.ctx, 0, self.xm, self._xw(), stream)

    def walls(self, stream=None):
        bgk_shard_walls(self.ctx, 0, self._xw(), stream)

    def close(self):
        self.solver.close()


def local_exchange(bufs: list, stream=None) -> None:
    """Sum for slabs that share this GPU: every buffer becomes the sum of all of them."""
    if len(bufs) > 1 and bufs[0].numel():
        bgk_shard_allreduce(bufs, bufs[0].numel(), stream)


class TorchExchange:
    """Sum across the ranks of a torch.distributed group (NCCL between GPUs, gloo between
    CPU processes), one buffer per rank."""

    def __init__(self, group=None):
        self.group = group

    def __call__(self, bufs: list, stream=None) -> None:
        import torch
        import torch.distributed as dist
        if len(bufs) != 1:
            raise BGKError(BGK_E_INVAL, "TorchExchange: one slab per rank")
        b = bufs[0]
        if b.is_cuda and stream is not None:
            st = torch.cuda.ExternalStream(stream) if isinstance(stream, int) else stream
            with torch.cuda.stream(st):
                dist.all_reduce(b, group=self.group)
        else:
            dist.all_reduce(b, group=self.group)


class ShardedSolver:
    """One case stepped as velocity slabs.  `slabs`: the slabs this process holds (one
    per rank across GPUs, or all of them on one GPU); `exchange(bufs, stream)`: replaces
    every buffer by the sum of the corresponding buffers of all slabs of all processes.
    A slab is any object with the methods of `Slab` and its buffers xm, xw."""

    def __init__(self, slabs: list, exchange):
        self.slabs = list(slabs)
        self.exchange = exchange
        self.steps = 0

    @classmethod
    def on_one_device(cls, p: dict, cloud: dict, parts: int) -> "ShardedSolver":
        """All `parts` slabs of the case on the current GPU."""
        NV = int(p["nv"]) ** int(p["dim"])
        return cls([Slab(p, cloud, lo, hi) for lo, hi in velocity_slabs(NV, parts)], local_exchange)

    @classmethod
    def distributed(cls, p: dict, cloud: dict, group=None) -> "ShardedSolver":
        """This rank's slab of the case: slab r of world-size slabs."""
        import torch.distributed as dist
        rank, world = dist.get_rank(group), dist.get_world_size(group)
        NV = int(p["nv"]) ** int(p["dim"])
        lo, hi = velocity_slabs(NV, world)[rank]
        return cls([Slab(p, cloud, lo, hi)], TorchExchange(group))

    def refresh_moments(self, stream=None) -> None:
        """Stored moments of every slab from the current f of all slabs."""
        for s in self.slabs:
            s.partial(stream)
        self.exchange([s.xm for s in self.slabs], stream)
        for s in self.slabs:
            s.set_moments(stream)

    def set_maxwellian(self, rho0=1.0, u0=(0.0, 0.0, 0.0), T0=1.0, stream=None) -> None:
        for s in self.slabs:
            s.set_maxwellian(rho0, u0, T0, stream)
        self.refresh_moments(stream)

    def step(self, nsteps: int = 1, stream=None) -> None:
        walls = self.slabs[0].xw.numel() > 0
        for _ in range(nsteps):
            for s in self.slabs:
                s.transport(stream)
            self.exchange([s.xm for s in self.slabs], stream)
            for s in self.slabs:
                s.relax(stream)
            if walls:
                self.exchange([s.xw for s in self.slabs], stream)
            for s in self.slabs:
                s.walls(stream)
            self.steps += 1

    # ---- state of the replicated quantities (read from the first slab) ----

    def sync(self, stream=None) -> None:
        for s in self.slabs:
            s.solver.sync(stream)

    def moments(self):
        return self.slabs[0].solver.moments()

    def positions(self):
        return self.slabs[0].solver.positions()

    def get_f(self, dtype=None):
        """f of this process's slabs side by side along the velocity axis (all of f when
        every slab is here)."""
        import numpy as np
        parts = [s.solver.get_f(0, dtype or np.float64) for s in self.slabs]
        return np.concatenate(parts, axis=2)

    def close(self) -> None:
        for s in self.slabs:
            s.close()
