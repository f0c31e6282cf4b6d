"""Coarse-to-fine solving over an image pyramid (pba_downsample and
paper_1704_06967_gb300.pyramid): the level images against their definition
(2 x 2 means, FP64), and the wider basin: from a pose error three times the
usual one, the coarse-to-fine IC solve ends closer to the true poses than
the same number of full-resolution iterations."""
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


def _pose_err(Pa, Pb):
    rot, tr = 0.0, 0.0
    for f in range(1, Pa.shape[0]):
        Ra, Rb = Pa[f, :9].reshape(3, 3), Pb[f, :9].reshape(3, 3)
        c = np.clip((np.trace(Ra @ Rb.T) - 1) / 2, -1, 1)
        rot = max(rot, math.degrees(math.acos(c)))
        tr = max(tr, np.abs(Pa[f, 9:] - Pb[f, 9:]).max())
    return rot, tr


def test_coarse_to_fine_widens_the_basin(torch_cuda):
    from paper_1704_06967_gb300 import Bundle
    from paper_1704_06967_gb300.pba import _scene_images
    from paper_1704_06967_gb300.pyramid import solve_coarse_to_fine
    sc = synth.make_scene("ring5", rot_deg=6.0, trans=0.06)
    img = _scene_images(sc)
    b = Bundle(img, sc.poses0, sc.intrinsics, sc.uv, sc.depths0, sc.vis, pattern=sc.pattern,
               huber_k=sc.huber_k)
    b.solve_ic(40, reanchor_every=3)
    P_full, _ = b.params()
    b.close()
    P_ctf, _, stats = solve_coarse_to_fine(img, sc.poses0, sc.intrinsics, sc.uv, sc.depths0, sc.vis,
                                           pattern=sc.pattern, huber_k=sc.huber_k, levels=3, iters=(10, 10, 20))
    r_full, t_full = _pose_err(P_full, sc.poses_gt)
    r_ctf, t_ctf = _pose_err(P_ctf, sc.poses_gt)
    r0, t0 = _pose_err(sc.poses0, sc.poses_gt)
    assert r_ctf < 0.5 * r0 and r_ctf < r_full, (r0, r_full, r_ctf)
    assert len(stats) == 3 and all(np.isfinite(s).all() for s in stats)
