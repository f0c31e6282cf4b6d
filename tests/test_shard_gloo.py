"""Point sharding of one bundle (paper_1704_06967_gb300/shard.py) on the CPU.

The orchestration runs as two gloo ranks over a backend that computes each
rank's share with the FP64 oracle: per rank the H_ff blocks, S_off and the
Schur right-hand side of its own points (Sec. 3.5 steps 2-3), summed over
the ranks by the orchestrator's all-reduces, then the reduced system solved
on every rank and each rank's depths back-substituted from its own blocks.
The sharded IC and FC iterations must reproduce the oracle's steps on the
whole bundle: the coupling terms are sums over points, so the split is exact
up to the order of the sums. The partition and the statistics reduction are
checked on their own."""
import dataclasses
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

from paper_1704_06967_gb300 import shard  # noqa: E402


def test_shard_points_split_the_morton_order_into_whole_tiles():
    rng = np.random.default_rng(3)
    uv = rng.integers(0, 200, (1000, 2))
    order = shard.morton_order(uv)
    for world in (1, 2, 3, 7):
        parts = shard.shard_points(uv, world)
        assert len(parts) == world
        allidx = np.concatenate(parts)
        assert np.array_equal(np.sort(allidx), np.arange(1000))  # every point exactly once
        pos = np.empty(1000, int)
        pos[order] = np.arange(1000)
        for r, p in enumerate(parts):
            q = np.sort(pos[p])
            assert np.array_equal(q, np.arange(q[0], q[0] + q.size))  # contiguous in Morton order
            if r < world - 1:
                assert q.size % shard.TILE == 0  # whole tiles but the last
        sizes = [p.size for p in parts]
        assert max(sizes) - min(sizes) <= shard.TILE + 1000 % shard.TILE


def test_reduce_stats_sums_counts_and_takes_the_largest_displacement():
    a = np.array([[2.0, 8.0, 4.0, 1.5, 9.0, 4.0], [1.0, 2.0, 2.0, 0.0, 0.0, 0.0]])
    b = np.array([[1.0, 4.0, 4.0, 2.5, 9.0, 5.0], [3.0, 6.0, 2.0, 0.0, 0.0, 0.0]])
    out = shard.reduce_stats([a, b])
    assert np.allclose(out[0], [3.0, np.sqrt(12.0 / 8.0), 8.0, 2.5, 3.0, 3.0])
    assert np.allclose(out[1], [4.0, np.sqrt(8.0 / 4.0), 4.0, 0.0, 0.0, 0.0])


# ----------------------------------------------------------------------------
# a rank's share computed by the oracle
# ----------------------------------------------------------------------------
def _solve(Hff, Soff, y, t_anchor):
    """Delta theta = -S^-1 y with the oracle's gauge handling: frames without
    residuals get identity blocks, the scale prior mu t^ t^T on the first
    active frame's translation."""
    F = Hff.shape[0]
    n6 = 6 * (F - 1)
    S = -Soff.copy()
    b = -y.copy()
    active = [float(np.trace(Hff[f])) > 0 for f in range(F)]
    for f in range(1, F):
        S[6 * (f - 1):6 * f, 6 * (f - 1):6 * f] += Hff[f]
    diag = [S[i, i] for f in range(1, F) if active[f] for i in range(6 * (f - 1), 6 * f)]
    mu = float(np.mean(diag)) if diag else 0.0
    for f in range(1, F):
        if not active[f]:
            sl = slice(6 * (f - 1), 6 * f)
            S[sl, :] = 0.0
            S[:, sl] = 0.0
            S[sl, sl] = np.eye(6)
            b[sl] = 0.0
    anchor = next((f for f in range(1, F) if active[f]), -1)
    if anchor > 0:
        t = t_anchor[anchor] / np.linalg.norm(t_anchor[anchor])
        S[6 * (anchor - 1):6 * (anchor - 1) + 3, 6 * (anchor - 1):6 * (anchor - 1) + 3] += mu * np.outer(t, t)
    dth = np.zeros((F, 6))
    dth[1:] = np.linalg.solve(S, b).reshape(F - 1, 6)
    assert n6 == S.shape[0]
    return dth


class OracleShard:
    """One rank's points of a bundle, each half of a step by the oracle."""

    def __init__(self, sc, idx):
        import oracle
        self.o = oracle
        sub = dataclasses.replace(sc, uv=sc.uv[idx], vis=sc.vis[idx], depths_gt=sc.depths_gt[idx],
                                  depths0=sc.depths0[idx])
        self.sc = sub
        self.pb = oracle.Problem.from_scene(sub)
        self.poses, self.depths = sub.poses0.copy(), sub.depths0.copy()
        self.bufs = {}
        self.raw = []

    def _blocks(self, Hfd, Hdd):
        F, N = self.pb.F, self.pb.N
        U = Hfd[:, 1:, :].reshape(N, 6 * (F - 1))
        w = np.where(Hdd > 0, 1.0 / np.where(Hdd > 0, Hdd, 1.0), 0.0)
        return U, w

    def ic_precompute(self, half):
        if half == 0:
            self.pre = self.o.ic_precompute(self.pb, self.sc.poses0, self.sc.depths0)
            U, w = self._blocks(self.pre.Hfd, self.pre.Hdd)
            self.bufs[shard.SHARD_IC_FRAME_SUMS] = torch.from_numpy(self.pre.Hff.ravel().copy())
            self.bufs[shard.SHARD_SOFF] = torch.from_numpy(((U * w[:, None]).T @ U).ravel())
        else:
            F = self.pb.F
            self.Hff = self.bufs[shard.SHARD_IC_FRAME_SUMS].numpy().reshape(F, 6, 6)
            self.Soff = self.bufs[shard.SHARD_SOFF].numpy().reshape(6 * (F - 1), 6 * (F - 1))

    def _record(self, st, k):
        while len(self.raw) <= k:
            self.raw.append(np.zeros(6))
        self.raw[k][:3] = [st[0], st[1] ** 2 * st[2], st[2]]

    def ic_step(self, k, half):
        U, w = self._blocks(self.pre.Hfd, self.pre.Hdd)
        if half == 0:
            g_theta, self.g_d, st = self.o.ic_gradient(self.pb, self.pre, self.poses, self.depths)
            self._record(st, k)
            y = g_theta[1:].ravel() - U.T @ (w * self.g_d)
            self.bufs[shard.SHARD_IC_RHS] = torch.from_numpy(y.copy())
        else:
            y = self.bufs[shard.SHARD_IC_RHS].numpy()
            dth = _solve(self.Hff, self.Soff, y, self.sc.poses0[:, 9:])
            dd = -w * (self.g_d + U @ dth[1:].ravel())
            self.dth, self.dd = dth, dd
            self.poses, self.depths = self.o.ic_update(self.sc.poses0, self.sc.depths0, self.poses, self.depths,
                                                       dth, dd)

    def fc_step(self, k, half):
        F = self.pb.F
        if half == 0:
            Hff, Hfd, Hdd, g_theta, self.g_d, st = self.o.fc_linearize(self.pb, self.poses, self.depths)
            self._record(st, k)
            U, w = self._blocks(Hfd, Hdd)
            self.U, self.w = U, w
            y = g_theta[1:].ravel() - U.T @ (w * self.g_d)
            self.bufs[shard.SHARD_FC_FRAME_SUMS] = torch.from_numpy(np.concatenate([Hff.ravel(), y]))
            self.bufs[shard.SHARD_SOFF] = torch.from_numpy(((U * w[:, None]).T @ U).ravel())
        else:
            v = self.bufs[shard.SHARD_FC_FRAME_SUMS].numpy()
            Hff, y = v[:36 * F].reshape(F, 6, 6), v[36 * F:]
            Soff = self.bufs[shard.SHARD_SOFF].numpy().reshape(6 * (F - 1), 6 * (F - 1))
            dth = _solve(Hff, Soff, y, self.poses[:, 9:])
            dd = -self.w * (self.g_d + self.U @ dth[1:].ravel())
            self.dth, self.dd = dth, dd
            self.poses, self.depths = self.o.fc_update(self.poses, self.depths, dth, dd)

    def eval(self, fc, k):
        st = self.o.evaluate(self.pb, self.poses, self.depths)
        self._record(st, k)

    def export(self, which):
        return self.bufs[which]

    def import_(self, which, t):
        self.bufs[which] = t

    def raw_stats(self, n_slots):
        return np.array(self.raw[:n_slots])


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, q):
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import synth
    from paper_1704_06967_gb300 import shard as sh
    sc = synth.make_scene("small")
    idx = sh.shard_points(sc.uv, world)[rank]
    out = {"idx": idx}
    for method in ("ic", "fc"):
        be = OracleShard(sc, idx)
        solve = sh.ShardedSolve(be, sh.torch_reduce())
        if method == "ic":
            solve.precompute_ic()
            st = solve.iterate(2)
        else:
            st = solve.solve_fc(2)
        out[method] = (be.poses, be.depths, be.dth, be.dd, st)
    dist.barrier()
    q.put((rank, out))
    dist.destroy_process_group()


def test_two_gloo_ranks_reproduce_the_whole_bundle_iterations():
    import oracle
    import synth
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = dict(q.get(timeout=300) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    sc = synth.make_scene("small")
    pb = oracle.Problem.from_scene(sc)
    pre = oracle.ic_precompute(pb, sc.poses0, sc.depths0)
    P, D = sc.poses0, sc.depths0
    hist_ic = []
    for _ in range(2):
        dth, dd, P, D, st = oracle.ic_step(pb, pre, sc.poses0, sc.depths0, P, D)
        hist_ic.append(st)
    whole = {"ic": (P, D, dth, dd, hist_ic)}
    Pf, Df = sc.poses0, sc.depths0
    hist_fc = []
    for _ in range(2):
        fdth, fdd, Pf, Df, st = oracle.fc_step(pb, Pf, Df)
        hist_fc.append(st)
    whole["fc"] = (Pf, Df, fdth, fdd, hist_fc)
    for method in ("ic", "fc"):
        P_w, D_w, dth_w, dd_w, hist = whole[method]
        for rank in range(world):
            idx = res[rank]["idx"]
            P_r, D_r, dth_r, dd_r, st_r = res[rank][method]
            # every rank applies the whole bundle's frame update ...
            assert np.abs(dth_r - dth_w).max() <= 1e-9 * np.abs(dth_w).max(), method
            assert np.abs(P_r - P_w).max() <= 1e-10, method
            # ... and its own points' depth updates
            assert np.abs(dd_r - dd_w[idx]).max() <= 1e-9 * np.abs(dd_w).max(), method
            assert np.abs(D_r - D_w[idx]).max() <= 1e-10, method
            # statistics of the whole bundle from the ranks' sums
            for k in range(2):
                assert st_r[k, 2] == hist[k][oracle.ST_COUNT]
                assert abs(st_r[k, 0] - hist[k][oracle.ST_ENERGY]) <= 1e-12 * hist[k][oracle.ST_ENERGY]
