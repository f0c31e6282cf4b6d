"""Full-size precision workload (orbit101: reference + 100 frames, 1280x720
BF16 images, 200,000 points x 8-pixel pattern, 33.6 M residuals, a 600 x 600
reduced camera system): one teacher-forced IC step and one FC step against
the FP64 oracle at the step tolerance (relative error 1e-4).

The oracle needs ~2.5 minutes for this (its precompute, and the dense
600 x 600 Schur complements of its IC and FC steps, formed over every frame
pair of every point).
"""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

STEP_TOL = 1e-4


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1704_06967_gb300 import build
    build.build()
    return torch


def _step_err(dth, dd, o_dth, o_dd, ref0):
    got = np.concatenate([dth[1:].ravel(), dd])
    ref = np.concatenate([o_dth[1:].ravel(), o_dd])
    return np.linalg.norm(got - ref) / max(np.linalg.norm(ref), 1e-3 * ref0)


def test_orbit101_full_size_steps(torch_cuda):
    from paper_1704_06967_gb300 import Bundle
    sc = synth.make_scene("orbit101")
    assert sc.dtype == "bf16" and 6 * (sc.F - 1) == 600
    pb = oracle.Problem.from_scene(sc)
    b = Bundle.from_scene(sc)
    assert b.n_residuals() == sc.n_residuals()
    b.precompute_ic()
    st = b.iterate(1)
    dth, dd = b.last_update()
    pre = oracle.ic_precompute(pb, sc.poses0, sc.depths0)
    o_dth, o_dd, _, _, o_st = oracle.ic_step(pb, pre, sc.poses0, sc.depths0, sc.poses0, sc.depths0)
    ref0 = np.linalg.norm(np.concatenate([o_dth[1:].ravel(), o_dd]))
    err_ic = _step_err(dth, dd, o_dth, o_dd, ref0)
    print(f"orbit101 IC step error {err_ic:.3e}")
    assert err_ic <= STEP_TOL
    assert st[0, 2] == o_st[oracle.ST_COUNT]
    assert abs(st[0, 1] - o_st[oracle.ST_RMS]) <= 1e-5 * o_st[oracle.ST_RMS]
    assert abs(st[0, 3] - o_st[oracle.ST_MAXDISP]) <= 1e-4 * o_st[oracle.ST_MAXDISP] + 2e-3
    b.set_params(sc.poses0, sc.depths0)
    b.solve_fc(1)
    dth, dd = b.last_update()
    o_dth, o_dd, _, _, _ = oracle.fc_step(pb, sc.poses0, sc.depths0)
    ref0 = np.linalg.norm(np.concatenate([o_dth[1:].ravel(), o_dd]))
    err_fc = _step_err(dth, dd, o_dth, o_dd, ref0)
    print(f"orbit101 FC step error {err_fc:.3e}")
    assert err_fc <= STEP_TOL
    # 20 IC iterations run without device errors, counts stay sane
    b.set_params(sc.poses0, sc.depths0)
    st = b.iterate(20)
    assert np.isfinite(st).all() and (st[:, 2] > 0).all()
    b.close()
