"""Host-side checks of the C ABI: the library builds and loads, exports every
function include/pba.h declares, and rejects bad arguments and out-of-order
calls before touching the GPU."""
import ctypes

import numpy as np
import pytest

from paper_1704_06967_gb300 import build as pkg_build
from paper_1704_06967_gb300 import pba


@pytest.fixture(scope="module")
def lib():
    pkg_build.build()
    return pba.load()


def test_library_exports_every_declared_symbol(lib):
    names = pba.declared_symbols()
    assert len(names) >= 17
    for n in names:
        assert hasattr(lib, n), n


def _cfg(P=8, huber=9 / 255):
    pat = np.ascontiguousarray(np.zeros((P, 2)), dtype=np.int32)
    cfg = pba.Config(huber, P, pat.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), 0.0, 0.0, 1,
                     None, 0, 0)
    return cfg, pat


def test_create_rejects_bad_configs(lib):
    h = ctypes.c_void_p()
    cfg, pat = _cfg(huber=0.0)
    assert lib.pba_create(ctypes.byref(cfg), ctypes.byref(h)) == 1
    cfg, pat = _cfg(P=0)
    assert lib.pba_create(ctypes.byref(cfg), ctypes.byref(h)) == 1
    cfg, pat = _cfg(P=17)
    assert lib.pba_create(ctypes.byref(cfg), ctypes.byref(h)) == 1
    for nb in (-1, 65536):
        cfg, pat = _cfg()
        cfg.n_bundles = nb
        assert lib.pba_create(ctypes.byref(cfg), ctypes.byref(h)) == 1
    assert lib.pba_create(None, ctypes.byref(h)) == 1


def test_create_checks_the_brightness_options(lib):
    """photometric in {0, 1, 2}; the pairs as unknowns take one bundle per
    context; the prior weight is finite and >= 0."""
    h = ctypes.c_void_p()
    for mode, nb, prior, want in ((3, 1, 0.0, 1), (-1, 1, 0.0, 1), (2, 2, 0.0, 1), (2, 1, -0.5, 1),
                                  (2, 1, float("nan"), 1), (2, 1, float("inf"), 1), (1, 2, 0.0, 0),
                                  (2, 1, 0.01, 0), (2, 1, 0.0, 0), (0, 1, 0.0, 0)):
        cfg, pat = _cfg()
        cfg.n_bundles = nb
        cfg.photometric = mode
        cfg.photo_prior = prior
        st = lib.pba_create(ctypes.byref(cfg), ctypes.byref(h))
        assert st == want, (mode, nb, prior, st)
        if st == 0:
            lib.pba_destroy(h)


def test_call_order_and_argument_checks(lib):
    cfg, pat = _cfg()
    h = ctypes.c_void_p()
    assert lib.pba_create(ctypes.byref(cfg), ctypes.byref(h)) == 0
    try:
        # nothing set yet
        assert lib.pba_precompute_ic(h) == 2
        assert lib.pba_iterate(h, 1, None) == 2
        assert lib.pba_solve_fc(h, 1, None) == 2
        nb = ctypes.c_size_t()
        assert lib.pba_workspace_size(h, ctypes.byref(nb)) == 2
        uv = np.zeros((4, 2), np.int32) + 20
        d = np.ones(4)
        assert lib.pba_set_points(h, 0, 4, uv.ctypes.data, d.ctypes.data, None) == 2
        assert b"frames" in lib.pba_last_error(h)
        # frames: frame 0 must be the identity, F >= 2, bundle 0
        F, H, W = 3, 48, 64
        img = np.zeros((F, H, W), np.float32)
        poses = np.zeros((F, 12))
        poses[:, [0, 4, 8]] = 1.0
        K = np.array([50.0, 50.0, 31.5, 23.5])
        args = (F, W, H, W, 0, 1, img.ctypes.data, poses.ctypes.data, K.ctypes.data)
        assert lib.pba_set_frames(h, 1, *args) == 1
        bad = poses.copy()
        bad[0, 9] = 0.1
        assert lib.pba_set_frames(h, 0, F, W, H, W, 0, 1, img.ctypes.data, bad.ctypes.data,
                                  K.ctypes.data) == 1
        assert lib.pba_set_frames(h, 0, 1, W, H, W, 0, 1, img.ctypes.data, poses.ctypes.data,
                                  K.ctypes.data) == 1
        # a device image pointer off the element size (checked without touching it)
        assert lib.pba_set_frames(h, 0, F, W, H, W, 0, 0, 0x10002, poses.ctypes.data, K.ctypes.data) == 1
        assert b"misaligned" in lib.pba_last_error(h)
        assert lib.pba_set_frames(h, 0, *args) == 0
        # points: pattern footprint inside the reference, positive depths
        uv_bad = uv.copy()
        uv_bad[0] = (0, 0)
        assert lib.pba_set_points(h, 0, 4, uv_bad.ctypes.data, d.ctypes.data, None) == 1
        d_bad = d.copy()
        d_bad[1] = -1.0
        assert lib.pba_set_points(h, 0, 4, uv.ctypes.data, d_bad.ctypes.data, None) == 1
        assert lib.pba_set_points(h, 0, 4, uv.ctypes.data, d.ctypes.data, None) == 0
        assert lib.pba_workspace_size(h, ctypes.byref(nb)) == 0
        assert nb.value > 0
        n = ctypes.c_int64()
        assert lib.pba_num_residuals(h, 0, ctypes.byref(n)) == 0
        assert n.value == 4 * (F - 1) * 8
        # workspace: too small, misaligned, and calls that need it
        assert lib.pba_set_workspace(h, ctypes.c_void_p(256), 16) == 4
        assert lib.pba_set_workspace(h, ctypes.c_void_p(257), nb.value) == 1
        assert lib.pba_precompute_ic(h) == 2
        assert lib.pba_iterate(h, 1, None) == 2
    finally:
        lib.pba_destroy(h)


def test_workspace_grows_with_the_problem(lib):
    sizes = []
    for N in (10, 100, 1000):
        cfg, pat = _cfg()
        h = ctypes.c_void_p()
        assert lib.pba_create(ctypes.byref(cfg), ctypes.byref(h)) == 0
        F, H, W = 4, 120, 160
        img = np.zeros((F, H, W), np.float32)
        poses = np.zeros((F, 12))
        poses[:, [0, 4, 8]] = 1.0
        K = np.array([100.0, 100.0, 79.5, 59.5])
        assert lib.pba_set_frames(h, 0, F, W, H, W, 0, 0, img.ctypes.data, poses.ctypes.data,
                                  K.ctypes.data) == 0
        rng = np.random.default_rng(0)
        uv = np.stack([rng.integers(5, W - 5, N), rng.integers(5, H - 5, N)], 1).astype(np.int32)
        d = np.ones(N)
        assert lib.pba_set_points(h, 0, N, uv.ctypes.data, d.ctypes.data, None) == 0
        nb = ctypes.c_size_t()
        assert lib.pba_workspace_size(h, ctypes.byref(nb)) == 0
        sizes.append(nb.value)
        lib.pba_destroy(h)
    assert sizes[0] < sizes[1] < sizes[2]


def _frames(F, W=64, H=48, K=(50.0, 50.0, 31.5, 23.5)):
    img = np.zeros((F, H, W), np.float32)
    poses = np.zeros((F, 12))
    poses[:, [0, 4, 8]] = 1.0
    return img, poses, np.array(K)


def test_batched_bundles_share_the_camera_and_count_separately(lib):
    cfg, pat = _cfg()
    cfg.n_bundles = 3
    h = ctypes.c_void_p()
    assert lib.pba_create(ctypes.byref(cfg), ctypes.byref(h)) == 0
    try:
        W, H = 64, 48
        keep = []
        for b, F in enumerate((3, 5, 2)):
            img, poses, K = _frames(F)
            keep.append((img, poses, K))
            assert lib.pba_set_frames(h, b, F, W, H, W, 0, 1, img.ctypes.data, poses.ctypes.data,
                                      K.ctypes.data) == 0
        assert lib.pba_set_frames(h, 3, *((2, W, H, W, 0, 1) + tuple(
            a.ctypes.data for a in keep[2]))) == 1
        # another camera for bundle 1 while the others are set: refused
        img, poses, K = _frames(5, K=(60.0, 50.0, 31.5, 23.5))
        assert lib.pba_set_frames(h, 1, 5, W, H, W, 0, 1, img.ctypes.data, poses.ctypes.data,
                                  K.ctypes.data) == 1
        assert b"share" in lib.pba_last_error(h)
        img2, poses2, K2 = _frames(5, W=80)
        assert lib.pba_set_frames(h, 1, 5, 80, H, 80, 0, 1, img2.ctypes.data, poses2.ctypes.data,
                                  K2.ctypes.data) == 1
        nb = ctypes.c_size_t()
        rng = np.random.default_rng(1)
        counts = (7, 40, 33)
        for b, N in enumerate(counts):
            # the workspace needs every bundle's points
            assert lib.pba_workspace_size(h, ctypes.byref(nb)) == 2
            uv = np.stack([rng.integers(5, W - 5, N), rng.integers(5, H - 5, N)], 1).astype(np.int32)
            d = np.ones(N)
            assert lib.pba_set_points(h, b, N, uv.ctypes.data, d.ctypes.data, None) == 0
        assert lib.pba_workspace_size(h, ctypes.byref(nb)) == 0
        for b, (N, F) in enumerate(zip(counts, (3, 5, 2))):
            n = ctypes.c_int64()
            assert lib.pba_num_residuals(h, b, ctypes.byref(n)) == 0
            assert n.value == N * (F - 1) * 8
        # the batch holds every bundle's data: more than any one bundle needs
        # alone, and close to their sum (per-context pieces such as the
        # statistics slots are held once)
        total, largest = 0, 0
        for b, (N, F) in enumerate(zip(counts, (3, 5, 2))):
            cfg1, pat1 = _cfg()
            h1 = ctypes.c_void_p()
            assert lib.pba_create(ctypes.byref(cfg1), ctypes.byref(h1)) == 0
            img, poses, K = keep[b]
            assert lib.pba_set_frames(h1, 0, F, W, H, W, 0, 1, img.ctypes.data, poses.ctypes.data,
                                      K.ctypes.data) == 0
            rng1 = np.random.default_rng(b)
            uv = np.stack([rng1.integers(5, W - 5, N), rng1.integers(5, H - 5, N)], 1).astype(np.int32)
            d = np.ones(N)
            assert lib.pba_set_points(h1, 0, N, uv.ctypes.data, d.ctypes.data, None) == 0
            nb1 = ctypes.c_size_t()
            assert lib.pba_workspace_size(h1, ctypes.byref(nb1)) == 0
            total += nb1.value
            largest = max(largest, nb1.value)
            lib.pba_destroy(h1)
        assert largest < nb.value <= total
    finally:
        lib.pba_destroy(h)
