"""Batched bundles: several independent bundles of uneven size in one context.

The batch concatenates the bundles' frames, tiles and entries, so each kernel
of an iteration covers all of them in one launch, while each bundle keeps its
own reference frame, gauge and reduced camera system. Every sum of the
method stays inside a bundle and keeps its order, so a bundle solved in a
batch must come out bit-identical to the same bundle solved alone; the
statistics are sums over the bundles. The first IC and FC steps of one
bundle of the batch are also checked against the FP64 oracle directly.
"""
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


def _scenes():
    """Three small bundles of different frame and point counts; the second
    has a target frame that sees none of its points."""
    base = synth.CONFIGS["small"]
    out = []
    for i, (F, N, az) in enumerate([(4, 120, (-12.0, 8.0, 16.0)), (6, 300, (-15.0, -7.5, 7.5, 15.0, 22.5)),
                                   (3, 64, (-10.0, 12.0))]):
        sc = synth.make_scene(base, seed_offset=100 + i, n_points=N, n_frames=F, azimuths_deg=az)
        out.append(sc)
    out[1].vis[:, 3] = 0
    return out


def _run(torch_cuda, scenes, method, iters, batched, **kw):
    from paper_1704_06967_gb300 import Batch, Bundle
    if batched:
        ctx = Batch.from_scenes(scenes, **kw)
        if method == "ic":
            ctx.precompute_ic()
            st = ctx.iterate(iters)
        else:
            st = ctx.solve_fc(iters)
        res = [ctx.params(b) for b in range(len(scenes))]
        ctx.close()
        return res, st
    res, sts = [], []
    for sc in scenes:
        b = Bundle.from_scene(sc, **kw)
        if method == "ic":
            b.precompute_ic()
            sts.append(b.iterate(iters))
        else:
            sts.append(b.solve_fc(iters))
        res.append(b.params())
        b.close()
    return res, sts


@pytest.mark.parametrize("method", ["ic", "fc"])
@pytest.mark.parametrize("graphs", [False, True])
def test_batch_equals_bundles_solved_alone(torch_cuda, method, graphs):
    scenes = _scenes()
    kw = dict(use_graphs=graphs, stream=torch_cuda.cuda.Stream()) if graphs else {}
    got, st = _run(torch_cuda, scenes, method, 6, True, **kw)
    ref, sts = _run(torch_cuda, scenes, method, 6, False)
    for b, ((P, D), (Pr, Dr)) in enumerate(zip(got, ref)):
        assert np.array_equal(P, Pr), (method, b, np.abs(P - Pr).max())
        assert np.array_equal(D, Dr), (method, b, np.abs(D - Dr).max())
    # statistics: sums over the bundles (counts exact, FP64 sums of FP32 tile
    # sums in another order otherwise)
    tot = sum(s for s in sts)
    assert np.array_equal(st[:, 2], tot[:, 2])
    assert np.allclose(st[:, 0], tot[:, 0], rtol=1e-6, atol=0.0)


def test_batch_reference_frames_stay_fixed(torch_cuda):
    from paper_1704_06967_gb300 import Batch
    scenes = _scenes()
    ctx = Batch.from_scenes(scenes)
    ctx.precompute_ic()
    ctx.iterate(4)
    for b in range(len(scenes)):
        P, _ = ctx.params(b)
        assert np.array_equal(P[0], np.array([1, 0, 0, 0, 1, 0, 0, 0, 1, 0, 0, 0], float))
        dth, _ = ctx.last_update(b)
        assert not dth[0].any()
    # the frame without observations keeps its pose and gets no update
    P, _ = ctx.params(1)
    assert np.array_equal(P[3], scenes[1].poses0[3])
    ctx.close()


@pytest.mark.parametrize("method", ["ic", "fc"])
def test_batch_step_matches_oracle(torch_cuda, method):
    from paper_1704_06967_gb300 import Batch
    scenes = _scenes()
    ctx = Batch.from_scenes(scenes)
    b = 1
    sc = scenes[b]
    pb = oracle.Problem.from_scene(sc)
    if method == "ic":
        ctx.precompute_ic()
        ctx.iterate(1)
        pre = oracle.ic_precompute(pb, sc.poses0, sc.depths0)
        o_dth, o_dd, _, _, _ = oracle.ic_step(pb, pre, sc.poses0, sc.depths0, sc.poses0, sc.depths0)
    else:
        ctx.solve_fc(1)
        o_dth, o_dd, _, _, _ = oracle.fc_step(pb, sc.poses0, sc.depths0)
    dth, dd = ctx.last_update(b)
    got = np.concatenate([dth[1:].ravel(), dd])
    ref = np.concatenate([o_dth[1:].ravel(), o_dd])
    assert np.linalg.norm(got - ref) <= 1e-4 * np.linalg.norm(ref)
    ctx.close()


def test_batch_system_slices_match_alone(torch_cuda):
    from paper_1704_06967_gb300 import Batch, Bundle
    scenes = _scenes()
    ctx = Batch.from_scenes(scenes)
    ctx.precompute_ic()
    for b, sc in enumerate(scenes):
        one = Bundle.from_scene(sc)
        one.precompute_ic()
        s1, s2 = ctx.system(bundle=b), one.system()
        for key in ("Hff", "Hfd", "Hdd", "S"):
            assert np.array_equal(s1[key], s2[key]), (b, key)
        assert ctx.n_residuals(b) == one.n_residuals() == sc.n_residuals()
        one.close()
    ctx.close()


def test_autotuned_shapes_leave_results_unchanged(torch_cuda):
    from paper_1704_06967_gb300 import Batch
    scenes = _scenes()
    res = []
    for tune in (False, True):
        ctx = Batch.from_scenes(scenes, autotune=tune)
        ctx.precompute_ic()
        ctx.iterate(4)
        w, c = ctx.tuning()
        assert w in (4, 8, 16) and c in (1, 2, 4, 8, 16)
        res.append([ctx.params(b) for b in range(len(scenes))])
        ctx.close()
    for (P1, D1), (P2, D2) in zip(*res):
        assert np.array_equal(P1, P2) and np.array_equal(D1, D2)


def test_set_launch_shapes_leave_results_unchanged(torch_cuda):
    """Shapes set by hand (as one context's autotuning would hand them to
    another) change no result; values outside the candidates are refused."""
    from paper_1704_06967_gb300 import Batch, PbaError
    scenes = _scenes()
    res = []
    for shape in (None, (4, 1), (16, 2)):
        ctx = Batch.from_scenes(scenes)
        if shape is not None:
            ctx.set_tuning(*shape)
            assert ctx.tuning() == shape
        ctx.precompute_ic()
        ctx.iterate(3)
        res.append([ctx.params(b) for b in range(len(scenes))])
        for bad in ((5, 1), (8, 3), (8, 0), (8, 64)):
            with pytest.raises(PbaError):
                ctx.set_tuning(*bad)
        ctx.close()
    for other in res[1:]:
        for (P1, D1), (P2, D2) in zip(res[0], other):
            assert np.array_equal(P1, P2) and np.array_equal(D1, D2)

