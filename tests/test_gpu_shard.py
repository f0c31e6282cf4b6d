"""Point sharding of one bundle through the library's split-phase C ABI on
one GPU: two contexts, each with a Morton-contiguous half of the points,
stepped in lockstep; between the halves of every step their frame sums and
S_off are added (a device sum standing in for the all-reduce of a
multi-GPU run; no kernel waits on another context). The two shards must
reproduce the single-context IC and FC iterations (the coupling terms are
sums over points; only the order of the frame sums differs: poses within
1e-7, inverse depths within 1e-6 and frame updates within 1e-5 relative,
RMS within 1e-6 relative) and the FP64
oracle's first steps; a single shard with no partner is the single-context
path itself."""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1704_06967_gb300 import build
    build.build()
    return torch


def _shards(sc, world):
    from paper_1704_06967_gb300 import Bundle
    from paper_1704_06967_gb300 import shard as sh
    from paper_1704_06967_gb300.pba import _scene_images
    img = _scene_images(sc)
    parts = sh.shard_points(sc.uv, world)
    out = []
    for idx in parts:
        b = Bundle(img, sc.poses0, sc.intrinsics, sc.uv[idx], sc.depths0[idx], sc.vis[idx],
                   pattern=sc.pattern, huber_k=sc.huber_k)
        out.append(sh.LibraryShard(b))
    return out, parts


def _sum(shards, which):
    ts = [s.export(which) for s in shards]
    tot = ts[0].clone()
    for t in ts[1:]:
        tot += t
    for s in shards:
        s.import_(which, tot)


def _run(shards, method, n):
    from paper_1704_06967_gb300 import shard as sh
    if method == "ic":
        for s in shards:
            s.ic_precompute(0)
        _sum(shards, sh.SHARD_IC_FRAME_SUMS)
        _sum(shards, sh.SHARD_SOFF)
        for s in shards:
            s.ic_precompute(1)
    for k in range(n):
        for s in shards:
            (s.ic_step if method == "ic" else s.fc_step)(k, 0)
        if method == "ic":
            _sum(shards, sh.SHARD_IC_RHS)
        else:
            _sum(shards, sh.SHARD_FC_FRAME_SUMS)
            _sum(shards, sh.SHARD_SOFF)
        for s in shards:
            (s.ic_step if method == "ic" else s.fc_step)(k, 1)
    for s in shards:
        s.eval(method == "fc", n)
    return sh.reduce_stats([s.raw_stats(n + 1) for s in shards])


@pytest.mark.parametrize("name", ["small", "ring5", "helix30"])
@pytest.mark.parametrize("method", ["ic", "fc"])
def test_two_point_shards_reproduce_the_single_context(torch_cuda, name, method):
    from paper_1704_06967_gb300 import Bundle
    sc = synth.make_scene(name)
    n = 3
    whole = Bundle.from_scene(sc)
    if method == "ic":
        whole.precompute_ic()
        st_w = whole.iterate(n)
    else:
        st_w = whole.solve_fc(n)
    P_w, D_w = whole.params()
    dth_w, _ = whole.last_update()
    whole.close()
    shards, parts = _shards(sc, 2)
    st = _run(shards, method, n)
    # the shards' frame sums and S_off are added in FP64 after each shard's
    # own fixed-order sums (double-float pairs, ~2^-48 of each entry; the
    # tensor-core S_off is exact), so the systems differ from the single
    # context's by that rounding, amplified by cond(S) in the steps
    for s, idx in zip(shards, parts):
        P, D = s.b.params()
        dth, _ = s.b.last_update()
        assert np.abs(P - P_w).max() <= 1e-7, method
        assert np.abs(D / D_w[idx] - 1).max() <= 1e-6, method
        assert np.abs(dth - dth_w).max() <= 1e-5 * np.abs(dth_w).max(), method
        s.b.close()
    assert np.array_equal(st[:, 2], st_w[:, 2])  # valid residual counts
    # the RMS follows the parameters: after three steps it differs by the
    # parameters' own difference times the residuals' sensitivity to them
    assert np.abs(st[:, 1] / st_w[:, 1] - 1).max() <= 1e-6
    assert np.abs(st[:-1, 3] / st_w[:-1, 3] - 1).max() <= 1e-4


def test_sharded_first_steps_match_the_oracle(torch_cuda):
    sc = synth.make_scene("ring5")
    pb = oracle.Problem.from_scene(sc)
    pre = oracle.ic_precompute(pb, sc.poses0, sc.depths0)
    o_dth, o_dd, _, _, _ = oracle.ic_step(pb, pre, sc.poses0, sc.depths0, sc.poses0, sc.depths0)
    f_dth, f_dd, _, _, _ = oracle.fc_step(pb, sc.poses0, sc.depths0)
    for method, (r_dth, r_dd) in (("ic", (o_dth, o_dd)), ("fc", (f_dth, f_dd))):
        shards, parts = _shards(sc, 2)
        _run(shards, method, 1)
        got_dd = np.zeros(sc.N)
        for s, idx in zip(shards, parts):
            dth, dd = s.b.last_update()
            got_dd[idx] = dd
            s.b.close()
        got = np.concatenate([dth[1:].ravel(), got_dd])
        ref = np.concatenate([r_dth[1:].ravel(), r_dd])
        err = np.linalg.norm(got - ref) / np.linalg.norm(ref)
        assert err <= 1e-4, (method, err)


def test_one_shard_is_the_single_context_path(torch_cuda):
    from paper_1704_06967_gb300 import Bundle
    from paper_1704_06967_gb300 import shard as sh
    sc = synth.make_scene("small")
    whole = Bundle.from_scene(sc)
    whole.precompute_ic()
    st_w = whole.iterate(4)
    P_w, D_w = whole.params()
    whole.close()
    shards, _ = _shards(sc, 1)
    solve = sh.ShardedSolve(shards[0], lambda t, op: None)
    solve.precompute_ic()
    st = solve.iterate(4)
    P, D = shards[0].b.params()
    assert np.array_equal(P, P_w) and np.array_equal(D, D_w)
    assert np.allclose(st, st_w, rtol=1e-12, atol=0)
    shards[0].b.close()
