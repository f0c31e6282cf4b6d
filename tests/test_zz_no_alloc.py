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
