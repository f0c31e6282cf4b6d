"""Point sharding of one bundle across ranks, one GPU each (orchestration
only: every step runs in the library's kernels).

The points are split into contiguous ranges of their Morton order (whole
tiles of 32 except the last range), so a rank's points are neighbours in the
reference image and see similar frames. Every rank holds all frames, images
and poses and its own points; a point's residuals, H_fd, H_dd, g_d and depth
update stay on its rank. What couples the points are sums over points
(Sec. 3.5: the H_ff blocks, S_off = H_pd H_dd^-1 H_dp and the Schur
right-hand side), so each step runs in two halves with one sum over the
ranks in between: the IC precompute sums F x 21 frame sums and S_off once;
an IC iteration sums the F x 6 right-hand side; an FC iteration sums F x 27
frame sums and S_off. The solves then run on every rank with identical
inputs, so all ranks apply the same frame updates.
"""
from __future__ import annotations

import ctypes

import numpy as np

from .pba import Bundle, PbaError, _p

SHARD_IC_FRAME_SUMS, SHARD_SOFF, SHARD_IC_RHS, SHARD_FC_FRAME_SUMS = 0, 1, 2, 3
TILE = 32


def _spread16(x):
    x = np.asarray(x, dtype=np.uint64) & np.uint64(0xFFFF)
    for s, m in ((8, 0x00FF00FF), (4, 0x0F0F0F0F), (2, 0x33333333), (1, 0x55555555)):
        x = (x | (x << np.uint64(s))) & np.uint64(m)
    return x


def morton_order(uv) -> np.ndarray:
    """Caller indices of the points in the Morton order of their reference
    pixels (ties in caller order)."""
    uv = np.asarray(uv)
    code = _spread16(uv[:, 0]) | (_spread16(uv[:, 1]) << np.uint64(1))
    return np.argsort(code, kind="stable")


def shard_points(uv, world: int) -> list:
    """Caller indices of each rank's points: `world` contiguous ranges of
    the Morton order, as equal as whole tiles allow."""
    if world < 1:
        raise ValueError("world must be >= 1")
    order = morton_order(uv)
    n = order.shape[0]
    tiles = (n + TILE - 1) // TILE
    cuts = [min(n, TILE * ((tiles * r) // world)) for r in range(world + 1)]
    return [np.sort(order[cuts[r]:cuts[r + 1]]) for r in range(world)]


def reduce_stats(raw_ranks) -> np.ndarray:
    """Per-slot statistics of the whole bundle from every rank's raw slots
    ([slots, 6]: energy, sum r^2, count, max displacement, |Dtheta|^2,
    sum Dd^2): rows (energy, RMS, count, max displacement, |Dtheta|, |Dd|)
    as Bundle.iterate returns them."""
    raw = np.asarray(raw_ranks, dtype=np.float64)
    tot = raw.sum(axis=0)
    out = np.zeros((raw.shape[1], 6))
    out[:, 0] = tot[:, 0]
    out[:, 1] = np.sqrt(np.where(tot[:, 2] > 0, tot[:, 1] / np.maximum(tot[:, 2], 1), 0.0))
    out[:, 2] = tot[:, 2]
    out[:, 3] = raw[:, :, 3].max(axis=0)
    out[:, 4] = np.sqrt(raw[0, :, 4])
    out[:, 5] = np.sqrt(tot[:, 5])
    out[-1, 3:] = 0.0  # the final evaluation slot carries no step
    return out


class LibraryShard:
    """One rank's share of a bundle in a library context (a Bundle over the
    rank's points) and its split-phase steps."""

    def __init__(self, bundle: Bundle, device="cuda"):
        import torch
        self.b = bundle
        self.torch = torch
        self.bufs = {}
        for which in (SHARD_IC_FRAME_SUMS, SHARD_SOFF, SHARD_IC_RHS, SHARD_FC_FRAME_SUMS):
            n = ctypes.c_int64()
            self._check(self.b.lib.pba_shard_count(self.b.h, which, ctypes.byref(n)))
            self.bufs[which] = torch.zeros(int(n.value), dtype=torch.float64, device=device)

    def _check(self, st):
        self.b._check(st)

    def ic_precompute(self, half):
        self._check(self.b.lib.pba_shard_ic_precompute(self.b.h, half))

    def ic_step(self, k, half):
        self._check(self.b.lib.pba_shard_ic_step(self.b.h, k, half))

    def fc_step(self, k, half):
        self._check(self.b.lib.pba_shard_fc_step(self.b.h, k, half))

    def eval(self, fc, k):
        self._check(self.b.lib.pba_shard_eval(self.b.h, int(bool(fc)), k))

    def export(self, which):
        """The rank's buffer as a torch tensor (ordered on the context's
        stream, which is the current stream of the caller)."""
        t = self.bufs[which]
        self._check(self.b.lib.pba_shard_export(self.b.h, which, ctypes.c_void_p(t.data_ptr())))
        return t

    def import_(self, which, t):
        self._check(self.b.lib.pba_shard_import(self.b.h, which, ctypes.c_void_p(t.data_ptr())))

    def raw_stats(self, n_slots):
        raw = np.zeros((n_slots, 6))
        self._check(self.b.lib.pba_shard_stats(self.b.h, n_slots, _p(raw)))
        return raw


class ShardedSolve:
    """Runs IC and FC on one rank's shard. `reduce(tensor, op)` sums ("sum")
    or takes the maximum ("max") of a tensor over the ranks in place (e.g.
    torch.distributed.all_reduce); `shard` provides the halves (LibraryShard
    for the GPU path)."""

    def __init__(self, shard, reduce):
        self.shard = shard
        self.reduce = reduce

    def _sum(self, which):
        t = self.shard.export(which)
        self.reduce(t, "sum")
        self.shard.import_(which, t)

    def _stats(self, n_slots):
        import torch
        raw = torch.from_numpy(self.shard.raw_stats(n_slots))
        sums = raw.clone()
        self.reduce(sums, "sum")
        mx = raw[:, 3].clone().contiguous()
        self.reduce(mx, "max")
        merged = sums.numpy().copy()
        merged[:, 3] = mx.numpy()
        merged[:, 4] = raw[:, 4].numpy()
        return reduce_stats(merged[None])

    def precompute_ic(self):
        self.shard.ic_precompute(0)
        self._sum(SHARD_IC_FRAME_SUMS)
        self._sum(SHARD_SOFF)
        self.shard.ic_precompute(1)

    def iterate(self, n_iters):
        for k in range(n_iters):
            self.shard.ic_step(k, 0)
            self._sum(SHARD_IC_RHS)
            self.shard.ic_step(k, 1)
        self.shard.eval(False, n_iters)
        return self._stats(n_iters + 1)

    def solve_fc(self, n_iters):
        for k in range(n_iters):
            self.shard.fc_step(k, 0)
            self._sum(SHARD_FC_FRAME_SUMS)
            self._sum(SHARD_SOFF)
            self.shard.fc_step(k, 1)
        self.shard.eval(True, n_iters)
        return self._stats(n_iters + 1)


def torch_reduce(group=None):
    """reduce() over a torch.distributed process group."""
    import torch.distributed as dist

    def reduce(t, op):
        dist.all_reduce(t, op=dist.ReduceOp.SUM if op == "sum" else dist.ReduceOp.MAX, group=group)
    return reduce


def sharded_bundle(images, poses0, intrinsics, uv, inv_depth, vis, *, rank, world, reduce, **kw):
    """This rank's ShardedSolve of a bundle (its points: shard_points(uv,
    world)[rank]) and the caller indices of those points."""
    idx = shard_points(uv, world)[rank]
    if idx.size == 0:
        raise PbaError(-1, f"rank {rank} has no points")
    vis_r = None if vis is None else np.asarray(vis)[idx]
    b = Bundle(images, poses0, intrinsics, np.asarray(uv)[idx], np.asarray(inv_depth)[idx], vis_r, **kw)
    return ShardedSolve(LibraryShard(b), reduce), idx
