"""The CUDA ray caster (synth/render_gpu.cu) against the host renderer
(synth/render.c): the same noise-free images bit for bit, the same object
ids, and so the same points, visibility and perturbation; the device noise
has the configured spread. Input generation only (no bundle adjustment
arithmetic on either side)."""
import dataclasses

import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    synth.build_renderer_gpu()
    return torch


def _cases():
    # sphere only, cards (rectangles), sphere on a ground plane (FP16 and
    # BF16 storage), at sizes the host renderer finishes in seconds
    return [
        ("tiny", {}),
        ("cards", {}),
        ("helix30", {"W": 160, "H": 120, "f": 131.25, "n_points": 400, "n_frames": 6, "plane": True,
                     "dtype": "f16"}),
        ("orbit101", {"W": 192, "H": 108, "f": 135.0, "n_points": 500, "n_frames": 5}),
    ]


@pytest.mark.parametrize("name,over", _cases())
def test_gpu_renderer_matches_host_renderer(torch_cuda, name, over):
    host = synth.make_scene(name, noise_free=True, **over)
    dev = synth.make_scene(name, noise_free=True, device="cuda", **over)
    got = dev.images_f32.cpu().numpy()
    assert got.shape == host.images_f32.shape
    assert np.array_equal(got, host.images_f32), np.abs(got - host.images_f32).max()
    assert np.array_equal(dev.uv, host.uv) and np.array_equal(dev.vis, host.vis)
    assert np.array_equal(dev.poses0, host.poses0) and np.array_equal(dev.depths0, host.depths0)


def test_gpu_renderer_noise_and_storage(torch_cuda):
    torch = torch_cuda
    cfg = dataclasses.replace(synth.CONFIGS["helix30"], W=160, H=120, f=131.25, n_points=400, n_frames=4,
                              dtype="bf16")
    clean = synth.make_scene(cfg, noise_free=True, device="cuda")
    noisy = synth.make_scene(cfg, device="cuda")
    assert noisy.images_store.dtype == torch.bfloat16 and noisy.images_store.is_cuda
    d = (noisy.images_f32 - clean.images_f32).double()
    # BF16 storage adds its rounding (relative 2^-9) to the N(0, sigma^2) noise
    assert abs(float(d.std()) - cfg.noise) < 0.25 * cfg.noise, float(d.std())
    assert abs(float(d.mean())) < 0.05 * cfg.noise
    again = synth.make_scene(cfg, device="cuda")  # seeded: the same bundle
    assert torch.equal(again.images_store, noisy.images_store)
