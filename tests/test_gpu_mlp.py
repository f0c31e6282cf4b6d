"""Learned inverse-depth proposal on the GPU against the FP64 oracle
(oracle/mlp.py): features, gradients, the Adam step, tensor-core inference,
the proposal written into a bundle, and what a trained network gains over
the constant-depth initialisation.

Tolerances. Features: FP32 projection and interpolation against FP64, the
values scaled by 1 / (sigma + 1/255) (<= 255): 2e-3 absolute, except that a
matching cost whose footprint sits on the image border may be valid on one
side only (at most 0.5 % of the costs). Gradients and the Adam step: FP32 sums
of <= 256 products against FP64: 1e-4 of each tensor's largest entry.
Inference: BF16 weights, BF16 inputs and BF16 hidden activations with FP32
accumulation; against the oracle run with the same roundings 3e-3 (1 + |y|)
(a hidden activation can round the other way, ~2^-8 of one of 128 terms),
against the unrounded oracle 6e-2 (1 + |y|) (2^-8 relative per layer).
"""
import numpy as np
import pytest

import synth
from oracle import mlp as omlp

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1704_06967_gb300 import build
    build.build()
    return torch


def _bf16(x):
    return synth.bf16_to_f32(synth.bf16_round(np.asarray(x, np.float32))).astype(np.float64)


def _oracle_bf16_forward(p, X):
    """The oracle forward with the GPU's roundings: BF16 weights, inputs and
    hidden activations h1, h2 (h3 and the output layer stay unrounded)."""
    q = {k: (_bf16(v) if k in ("W1", "W2", "W3") else v) for k, v in p.items()}
    h = _bf16(X)
    for layer in (1, 2, 3):
        z = h @ q[f"W{layer}"].T + q[f"b{layer}"]
        h = omlp.gelu(z)
        if layer < 3:
            h = _bf16(h)
    return h @ q["w4"] + q["b4"][0]


def test_features_match_oracle(torch_cuda):
    from paper_1704_06967_gb300 import Bundle
    sc = synth.make_scene("small")
    b = Bundle.from_scene(sc)
    got = b.depth_features().cpu().numpy().astype(np.float64)
    ref = omlp.features(sc.images_f32, sc.intrinsics, sc.poses0, sc.uv, sc.vis, sc.pattern)
    assert got.shape == ref.shape == (sc.N, 96)
    assert np.abs(got[:, :64] - ref[:, :64]).max() < 2e-3
    d = np.abs(got[:, 64:] - ref[:, 64:])
    # a bin's least cost can sit on the image border, where FP32 and FP64
    # disagree on whether the footprint is inside (a NO_DATA flip)
    assert np.mean(d > 2e-3) <= 5e-3, np.sort(d.ravel())[-10:]
    assert np.median(d) < 1e-4
    b.close()


def test_gradient_matches_oracle(torch_cuda):
    torch = torch_cuda
    from paper_1704_06967_gb300.learned import DepthMLP
    rng = np.random.default_rng(5)
    p = omlp.init_params(11)
    for k in p:
        p[k] = p[k] + 0.05 * rng.normal(size=p[k].shape)
    X = rng.normal(size=(200, 96))
    T = rng.normal(1.0, 0.3, size=200)
    net = DepthMLP(params=omlp.pack(p))
    loss, g = net.grad(torch.tensor(X, dtype=torch.float32, device="cuda"),
                       torch.tensor(T, dtype=torch.float32, device="cuda"))
    # the kernel takes FP32 parameters and inputs: give the oracle the same
    p32 = {k: v.astype(np.float32).astype(np.float64) for k, v in p.items()}
    lref, gref = omlp.loss_and_grad(p32, X.astype(np.float32).astype(np.float64), T.astype(np.float32))
    assert abs(float(loss) / 200 - lref) <= 1e-5 * lref
    gg = omlp.unpack(g.cpu().numpy().astype(np.float64))
    for k, _ in omlp.SHAPES:
        assert np.abs(gg[k] - gref[k]).max() <= 1e-4 * np.abs(gref[k]).max(), k


def test_adam_step_matches_oracle(torch_cuda):
    torch = torch_cuda
    from paper_1704_06967_gb300.learned import DepthMLP
    rng = np.random.default_rng(6)
    theta = omlp.pack(omlp.init_params(3)).astype(np.float32).astype(np.float64)
    X = rng.normal(size=(128, 96)).astype(np.float32)
    T = rng.normal(1.0, 0.3, size=128).astype(np.float32)
    net = DepthMLP(params=theta)
    Xt, Tt = torch.tensor(X, device="cuda"), torch.tensor(T, device="cuda")
    _, g = net.grad(Xt, Tt)
    gnp = g.cpu().numpy().astype(np.float64)
    # one step over the same samples in the same order: the step's gradient
    # is the one just read back
    import ctypes
    scratch = torch.empty(int(net.lib.pba_mlp_scratch_floats(128)), dtype=torch.float32, device="cuda")
    vp = lambda t: ctypes.c_void_p(t.data_ptr())
    st = net.lib.pba_mlp_train_step(vp(net.params), vp(net.m), vp(net.v), 1, ctypes.c_float(1e-3), 128, vp(Xt),
                                    vp(Tt), vp(scratch), None, ctypes.c_void_p(net.stream.cuda_stream))
    assert st == 0
    ref, mref, vref = omlp.adam_step(theta, gnp, np.zeros_like(theta), np.zeros_like(theta), 1, 1e-3)
    got = net.params.cpu().numpy().astype(np.float64)
    assert np.abs(got - ref).max() <= 1e-7
    assert np.allclose(net.m.cpu().numpy(), mref, rtol=1e-6, atol=0)
    assert np.allclose(net.v.cpu().numpy(), vref, rtol=1e-6, atol=0)


@pytest.mark.parametrize("n", [1, 127, 300, 4099])
def test_tensor_core_inference_matches_oracle(torch_cuda, n):
    torch = torch_cuda
    from paper_1704_06967_gb300.learned import DepthMLP
    rng = np.random.default_rng(n)
    p = omlp.init_params(21)
    X = rng.normal(size=(n, 96)) * 0.8
    net = DepthMLP(params=omlp.pack(p))
    y = net.infer(torch.tensor(X, dtype=torch.float32, device="cuda")).cpu().numpy().astype(np.float64)
    yb = _oracle_bf16_forward(p, X.astype(np.float32))
    y64, _ = omlp.forward(p, X)
    assert np.all(np.abs(y - yb) <= 3e-3 * (1 + np.abs(yb))), np.abs(y - yb).max()
    assert np.all(np.abs(y - y64) <= 6e-2 * (1 + np.abs(y64)))


def test_proposal_replaces_the_bundle_depths(torch_cuda):
    from paper_1704_06967_gb300 import Batch
    from paper_1704_06967_gb300.learned import DepthMLP
    sc = synth.make_scene("small")
    sc.vis[::7, :] = 0  # every seventh point observed by no target frame
    scenes = [sc]
    ctx = Batch.from_scenes([scenes[0]])
    net = DepthMLP(seed=4)
    X = ctx.depth_features(0)
    y = np.clip(net.infer(X).cpu().numpy(), 0.05, 20.0)
    _, before = ctx.params(0)
    net.propose(ctx, 0)
    _, d = ctx.params(0)
    seen = scenes[0].vis[:, 1:].any(1)
    assert seen.any() and (~seen).any()
    assert np.array_equal(d[seen], y.astype(np.float64)[seen])
    assert np.array_equal(d[~seen], before[~seen])  # the fallback
    # and the bundle still solves from there
    ctx.precompute_ic()
    st = ctx.iterate(3)
    assert np.isfinite(st[:, 0]).all()
    ctx.close()


def _learned_scene(i):
    # sphere and ground plane (depths vary across the image), poses known to
    # 0.1 deg / 0.001: the proposal's setting (new points of a tracked frame)
    r = float(np.random.default_rng(i).uniform(0.7, 1.5))
    return synth.make_scene("ring5", seed_offset=i, sphere_r=r, plane=True, n_points=1500, rot_deg=0.1,
                            trans=0.001, allow_fewer_points=True)


def test_trained_proposal_beats_constant_depth(torch_cuda):
    """Train on bundles the method solved, then initialise held-out bundles
    from the proposal and from the constant inverse depth 1: the proposal
    starts closer to the true depths, and the solve from it ends at a lower
    photometric cost (RMS). The depths after the solve are not compared with
    the truth: a monocular bundle's scale is a gauge freedom the solve may
    drift along (a uniform inverse-depth offset at an unchanged cost)."""
    torch = torch_cuda
    from paper_1704_06967_gb300 import Bundle
    from paper_1704_06967_gb300.learned import DepthMLP, training_pairs
    train = [_learned_scene(300 + i) for i in range(16)]
    held = [_learned_scene(900 + i) for i in range(2)]
    Xs, Ts = [], []
    for sc in train:
        tp = training_pairs(sc)
        if tp is None:
            continue
        X, d, use = tp
        Xs.append(X[torch.tensor(use, device="cuda")])
        Ts.append(torch.tensor(d[use], dtype=torch.float32, device="cuda"))
    X, T = torch.cat(Xs), torch.cat(Ts)
    net = DepthMLP(seed=0)
    hist = net.train(X, T, epochs=40, batch=512, lr=2e-3)
    assert hist[-1] < 0.5 * hist[0]
    for sc in held:
        res = {}
        for mode in ("constant", "proposal"):
            b = Bundle(synth_images(sc), sc.poses0, sc.intrinsics, sc.uv, np.ones(sc.N), sc.vis,
                       pattern=sc.pattern, huber_k=sc.huber_k, damping=0.01)
            if mode == "proposal":
                net.propose(b)
            _, d0 = b.params()
            st = b.solve_ic(20, reanchor_every=3)
            seen = sc.vis[:, 1:].any(1)  # the points the bundle adjustment estimates
            res[mode] = (np.median(np.abs(d0[seen] / sc.depths_gt[seen] - 1)), float(st[-1, 1]))
            b.close()
        assert res["proposal"][0] < 0.7 * res["constant"][0], res
        assert res["proposal"][1] < res["constant"][1], res


def synth_images(sc):
    from paper_1704_06967_gb300.pba import _scene_images
    return _scene_images(sc)


def test_bounded_wait_gives_up_and_reports_a_timeout(torch_cuda):
    """The bounded waits' give-up path, run on purpose: a wait on a barrier
    phase that nothing completes ends after its bound, the kernel exits
    normally, the host gets PBA_ERR_TIMEOUT, and the context keeps working."""
    import ctypes
    torch = torch_cuda
    from paper_1704_06967_gb300 import load
    lib = load()
    flag = torch.zeros(1, dtype=torch.int32, device="cuda")
    st = torch.cuda.current_stream().cuda_stream
    rc = lib.pba_wait_selftest(ctypes.c_void_p(flag.data_ptr()), ctypes.c_void_p(st))
    assert rc == 7  # PBA_ERR_TIMEOUT
    assert int(flag.item()) != 0
    x = torch.arange(1024, dtype=torch.float32, device="cuda")
    assert float((x * 2).sum().item()) == 2 * 1023 * 1024 / 2  # the context still runs kernels

