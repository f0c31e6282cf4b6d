"""Coarse-to-fine solving over an image pyramid (pba_downsample and
paper_1704_06967_gb300.pyramid): the level images against their definition
(2 x 2 means, FP64), and the wider basin: from a pose error beyond the fine
texture's reach, the coarse-to-fine solve ends near the true poses where the
same number of full-resolution iterations stops in a local minimum."""
import math

import numpy as np
import pytest

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


@pytest.mark.parametrize("dtype", ["f32", "f16"])
def test_downsample_is_the_mean_of_each_2x2_block(torch_cuda, dtype):
    torch = torch_cuda
    from paper_1704_06967_gb300.pyramid import downsample
    rng = np.random.default_rng(4)
    img = rng.uniform(0, 1, size=(2, 37, 50)).astype(np.float32)
    t = torch.tensor(img, device="cuda")
    if dtype == "f16":
        t = t.half()
        img = t.float().cpu().numpy()
    got = downsample(t).cpu().numpy().astype(np.float64)
    x = img.astype(np.float64)[:, :36, :50]
    ref = 0.25 * (x[:, 0::2, 0::2] + x[:, 0::2, 1::2] + x[:, 1::2, 0::2] + x[:, 1::2, 1::2])
    assert got.shape == (2, 18, 25)
    assert np.abs(got - ref).max() <= 2e-7


def _median_rot_err(Pa, Pb, active):
    out = []
    for f in range(1, Pa.shape[0]):
        if active[f]:
            Ra, Rb = Pa[f, :9].reshape(3, 3), Pb[f, :9].reshape(3, 3)
            out.append(math.degrees(math.acos(np.clip((np.trace(Ra @ Rb.T) - 1) / 2, -1, 1))))
    return float(np.median(out))


def test_coarse_to_fine_widens_the_basin(torch_cuda):
    """5-frame ring, poses perturbed by 3 deg / 0.03 (the texture's finest
    cells are 8 px; 3 degrees move the image ~15 px): at full resolution FC
    settles in a local minimum; coarse-to-fine over three levels ends near
    the true poses, at a lower photometric RMS."""
    from paper_1704_06967_gb300 import Bundle
    from paper_1704_06967_gb300.pba import _scene_images
    from paper_1704_06967_gb300.pyramid import solve_coarse_to_fine
    sc = synth.make_scene("ring5", rot_deg=3.0, trans=0.03)
    img = _scene_images(sc)
    act = sc.vis.sum(0) > 0
    b = Bundle(img, sc.poses0, sc.intrinsics, sc.uv, sc.depths0, sc.vis, pattern=sc.pattern,
               huber_k=sc.huber_k, damping=0.01)
    st_full = b.solve_fc(40)
    P_full, _ = b.params()
    b.close()
    P_ctf, _, stats = solve_coarse_to_fine(img, sc.poses0, sc.intrinsics, sc.uv, sc.depths0, sc.vis,
                                           pattern=sc.pattern, huber_k=sc.huber_k, levels=3, iters=(10, 10, 20),
                                           method="fc", damping=0.01)
    e_full = _median_rot_err(P_full, sc.poses_gt, act)
    e_ctf = _median_rot_err(P_ctf, sc.poses_gt, act)
    assert e_ctf < 0.5 * e_full, (e_full, e_ctf)
    assert stats[-1][-1, 1] < 0.7 * st_full[-1, 1], (stats[-1][-1, 1], st_full[-1, 1])
    assert len(stats) == 3 and all(np.isfinite(s).all() for s in stats)


def _python_levels(img, sc, levels, iters, method, damping):
    """The coarse-to-fine orchestration restated with one Bundle per level
    (the level geometry written out here): what pba_solve_pyramid must
    reproduce exactly, since it makes the same library calls."""
    from paper_1704_06967_gb300 import Bundle
    from paper_1704_06967_gb300.pyramid import downsample
    pyr = [img]
    for _ in range(levels - 1):
        pyr.append(downsample(pyr[-1]))
    poses, depth = sc.poses0.copy(), sc.depths0.copy()
    K = np.asarray(sc.intrinsics, np.float64)
    rad = int(np.abs(sc.pattern).max()) + 1
    stats = []
    for lvl in range(levels - 1, -1, -1):
        F, H, W = pyr[lvl].shape
        s = 2.0 ** lvl
        Kl = np.array([K[0] / s, K[1] / s, (K[2] + 0.5) / s - 0.5, (K[3] + 0.5) / s - 0.5])
        uvl = np.rint((sc.uv.astype(np.float64) + 0.5) / s - 0.5).astype(np.int32)
        keep = (uvl[:, 0] >= rad) & (uvl[:, 0] <= W - 1 - rad) & (uvl[:, 1] >= rad) & (uvl[:, 1] <= H - 1 - rad)
        b = Bundle(pyr[lvl].contiguous(), poses, Kl, uvl[keep], depth[keep], sc.vis[keep], pattern=sc.pattern,
                   huber_k=sc.huber_k, damping=damping)
        n = iters[levels - 1 - lvl]
        st = b.solve_ic(n, reanchor_every=3) if method == "ic" else b.solve_fc(n)
        poses, d = b.params()
        b.close()
        sub = depth[keep]
        good = np.isfinite(d) & (d > 0)
        sub[good] = d[good]
        depth[keep] = sub
        stats.append(st)
    return poses, depth, stats


@pytest.mark.parametrize("method", ["ic", "fc"])
def test_native_pyramid_makes_the_level_calls_in_order(torch_cuda, method):
    """pba_solve_pyramid against the same levels solved through the public
    API one context at a time: identical poses, inverse depths and
    statistics (bit for bit), and one device time per level."""
    from paper_1704_06967_gb300.pba import _scene_images
    from paper_1704_06967_gb300.pyramid import solve_coarse_to_fine
    sc = synth.make_scene("ring5", rot_deg=3.0, trans=0.03)
    img = _scene_images(sc)
    iters = (4, 3, 5)
    P_ref, D_ref, st_ref = _python_levels(img, sc, 3, iters, method, 0.01)
    ms = []
    P, D, st = solve_coarse_to_fine(img, sc.poses0, sc.intrinsics, sc.uv, sc.depths0, sc.vis, pattern=sc.pattern,
                                    huber_k=sc.huber_k, levels=3, iters=iters, method=method, damping=0.01,
                                    level_ms=ms)
    assert np.array_equal(P, P_ref) and np.array_equal(D, D_ref)
    assert len(st) == 3 and all(np.array_equal(a, b) for a, b in zip(st, st_ref))
    assert len(ms) == 3 and all(m > 0 for m in ms)


def test_native_pyramid_refuses_bad_arguments(torch_cuda):
    """Too many levels for the image size, several bundles, and a workspace
    smaller than the size query are refused; nothing is solved."""
    import ctypes
    torch = torch_cuda
    from paper_1704_06967_gb300.pba import Config, PBA_F32, _p, load
    lib = load()
    sc = synth.make_scene("tiny")
    pat = np.ascontiguousarray(sc.pattern, np.int32)
    cfg = Config(float(sc.huber_k), pat.shape[0], pat.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), 1.0, 0.0, 1,
                 None, 0, 256, 0, 0.0, 0)
    F, H, W = sc.F, sc.H, sc.W
    poses = np.ascontiguousarray(sc.poses0, np.float64)
    K = np.ascontiguousarray(sc.intrinsics, np.float64)
    uv = np.ascontiguousarray(sc.uv, np.int32)
    d = np.ascontiguousarray(sc.depths0, np.float64)
    nb = ctypes.c_size_t()
    assert lib.pba_pyramid_workspace_size(ctypes.byref(cfg), 8, F, W, H, _p(poses), _p(K), uv.shape[0], _p(uv),
                                          _p(d), None, ctypes.byref(nb)) == 1
    cfg.n_bundles = 2
    assert lib.pba_pyramid_workspace_size(ctypes.byref(cfg), 2, F, W, H, _p(poses), _p(K), uv.shape[0], _p(uv),
                                          _p(d), None, ctypes.byref(nb)) == 1
    cfg.n_bundles = 1
    assert lib.pba_pyramid_workspace_size(ctypes.byref(cfg), 2, F, W, H, _p(poses), _p(K), uv.shape[0], _p(uv),
                                          _p(d), None, ctypes.byref(nb)) == 0
    img = torch.tensor(sc.images_f32, device="cuda").contiguous()
    ws = torch.empty(int(nb.value) // 2 + 256, dtype=torch.uint8, device="cuda")
    base = (ws.data_ptr() + 255) // 256 * 256
    its = np.array([2, 2], np.int32)
    P0 = poses.copy()
    rc = lib.pba_solve_pyramid(ctypes.byref(cfg), 2, _p(its), 0, 0, ctypes.c_void_p(img.data_ptr()), PBA_F32, F, W, H,
                               W, _p(poses), _p(K), uv.shape[0], _p(uv), _p(d), None, ctypes.c_void_p(base),
                               int(nb.value) // 2, None, None)
    assert rc == 4  # PBA_ERR_NOMEM
    assert np.array_equal(poses, P0)
