"""The no-allocation entry point (pba_reduced_system_noalloc) against the
context path.

It serves callers that cannot allocate device memory: it builds the anchored
reduced camera system from dense Hessian blocks with its scratch in a static
device array. Called twice in a row, through the C ABI, it must reproduce the
system the context built in its workspace (pba_get_system), for the IC
precompute and for an FC linearisation, within the tolerance the parity
tests use for S (1e-4 of its largest entry). This file is collected last so
that a failure here leaves every other test already run.
"""
import ctypes

import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu

PBA_OK, PBA_ERR_ARG, PBA_ERR_TOO_LARGE = 0, 1, 8


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1704_06967_gb300 import build, pba
    build.build()
    lib = pba.load()
    fn = lib.pba_reduced_system_noalloc
    vp = ctypes.c_void_p
    fn.argtypes = [ctypes.c_int, ctypes.c_int, vp, vp, vp, vp, ctypes.c_double, vp, vp]
    fn.restype = ctypes.c_int
    return torch, fn


def _dev(torch, a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()


def _call(torch, fn, F, N, Hff, Hfd, Hdd, poses, S, gauge_w=1.0):
    stream = torch.cuda.current_stream().cuda_stream
    return fn(F, N, Hff.data_ptr(), Hfd.data_ptr(), Hdd.data_ptr(), poses.data_ptr(), gauge_w,
              S.data_ptr(), ctypes.c_void_p(stream))


@pytest.mark.parametrize("fc", [False, True])
def test_noalloc_reduced_system_matches_context(env, fc):
    torch, fn = env
    from paper_1704_06967_gb300 import Bundle
    sc = synth.make_scene("small")
    b = Bundle.from_scene(sc)
    if fc:
        b.solve_fc(1)          # linearised at p_0; the gauge uses p_0's translations
    else:
        b.precompute_ic()
    ref = b.system(fc=fc)
    F, N = sc.F, sc.N
    n6 = 6 * (F - 1)
    Hff, Hfd, Hdd = _dev(torch, ref["Hff"]), _dev(torch, ref["Hfd"]), _dev(torch, ref["Hdd"])
    poses = _dev(torch, sc.poses0)
    S = torch.empty((n6, n6), dtype=torch.float64, device="cuda")
    tol = 1e-4 * np.abs(ref["S"]).max()
    for _ in range(2):
        S.fill_(float("nan"))
        assert _call(torch, fn, F, N, Hff, Hfd, Hdd, poses, S) == PBA_OK
        torch.cuda.synchronize()
        got = S.cpu().numpy()
        assert np.isfinite(got).all()
        assert np.abs(got - ref["S"]).max() <= tol
    b.close()


def test_noalloc_rejects_oversized_and_invalid_problems(env):
    torch, fn = env
    x = torch.zeros(8, dtype=torch.float64, device="cuda")
    assert _call(torch, fn, 66, 10, x, x, x, x, x) == PBA_ERR_TOO_LARGE
    assert _call(torch, fn, 1, 10, x, x, x, x, x) == PBA_ERR_ARG
    stream = torch.cuda.current_stream().cuda_stream
    assert fn(4, 10, None, x.data_ptr(), x.data_ptr(), x.data_ptr(), 1.0, x.data_ptr(),
              ctypes.c_void_p(stream)) == PBA_ERR_ARG


def _numpy_system(Hff, Hfd, Hdd, poses, gauge_w):
    """The system the header defines, written out in FP64 with numpy."""
    F = Hff.shape[0]
    n6 = 6 * (F - 1)
    U = Hfd[:, 1:, :].reshape(Hfd.shape[0], n6)
    w = np.where(Hdd > 0, 1.0 / np.where(Hdd > 0, Hdd, 1.0), 0.0)
    S = -(U * w[:, None]).T @ U
    active = [np.trace(Hff[f]) > 0 for f in range(F)]
    for f in range(1, F):
        S[6 * (f - 1):6 * f, 6 * (f - 1):6 * f] += Hff[f]
    mu = np.mean([S[i, i] for f in range(1, F) if active[f] for i in range(6 * (f - 1), 6 * f)])
    for f in range(1, F):
        if not active[f]:
            sl = slice(6 * (f - 1), 6 * f)
            S[sl, :] = 0.0
            S[:, sl] = 0.0
            S[sl, sl] = np.eye(6)
    fa = next(f for f in range(1, F) if active[f])
    t = poses[fa, 9:] / np.linalg.norm(poses[fa, 9:])
    S[6 * (fa - 1):6 * (fa - 1) + 3, 6 * (fa - 1):6 * (fa - 1) + 3] += (gauge_w or 1.0) * mu * np.outer(t, t)
    return S


def _random_blocks(F, N, seed):
    """Dense blocks of a random bundle: sparse visibility, H_ff the sum of
    the points' blocks plus a positive part, one frame without residuals."""
    rng = np.random.default_rng(seed)
    vis = rng.random((N, F)) < 0.3
    vis[:, 0] = False
    vis[:, F // 2] = False  # a frame nobody sees
    Hfd = rng.standard_normal((N, F, 6)) * vis[:, :, None]
    Hdd = rng.uniform(0.5, 4.0, N)
    Hdd[::17] = 0.0         # points without a depth block are skipped
    Hff = np.zeros((F, 6, 6))
    for f in range(F):
        if f == 0 or f == F // 2:
            continue
        G = rng.standard_normal((6, 6))
        Hff[f] = np.einsum("na,nb->ab", Hfd[:, f], Hfd[:, f]) / 0.5 + G @ G.T + 6 * np.eye(6)
    poses = np.tile(np.r_[np.eye(3).ravel(), 0.0, 0.0, 0.0], (F, 1))
    poses[:, 9:] = rng.standard_normal((F, 3))
    return Hff, Hfd, Hdd, poses


@pytest.mark.parametrize("F,gauge_w", [(65, 1.0), (12, 2.5)])
def test_noalloc_matches_the_schur_complement_written_out(env, F, gauge_w):
    """At the capacity (65 frames: the scratch array's last offsets) and
    with a gauge prior weight other than 1, against the definition in FP64
    numpy, on two calls in a row."""
    torch, fn = env
    N = 700
    Hff, Hfd, Hdd, poses = _random_blocks(F, N, seed=F)
    ref = _numpy_system(Hff, Hfd, Hdd, poses, gauge_w)
    n6 = 6 * (F - 1)
    dHff, dHfd, dHdd, dposes = (_dev(torch, a) for a in (Hff, Hfd, Hdd, poses))
    S = torch.empty((n6, n6), dtype=torch.float64, device="cuda")
    for _ in range(2):
        S.fill_(float("nan"))
        assert _call(torch, fn, F, N, dHff, dHfd, dHdd, dposes, S, gauge_w) == PBA_OK
        torch.cuda.synchronize()
        got = S.cpu().numpy()
        assert np.abs(got - ref).max() <= 1e-12 * np.abs(ref).max()
        assert np.array_equal(got, got.T)
