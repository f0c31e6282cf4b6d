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
