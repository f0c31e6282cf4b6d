"""Pins of the oracle's affine brightness option (or_photo_update, the
residual alpha_f I_f + beta_f): a closed-form fit that recovers known
brightness changes at the true parameters, the identity pair reproducing the
plain model, and a lower cost under lighting changes."""
import numpy as np
import pytest

import oracle
import synth


def _relit(sc, alphas, betas):
    """Target frames relit so that the template sees alpha_f I'_f + beta_f."""
    imgs = sc.images_f32.astype(np.float64).copy()
    for f in range(1, sc.F):
        imgs[f] = (imgs[f] - betas[f]) / alphas[f]
    return imgs


@pytest.fixture(scope="module")
def cards():
    return synth.make_scene("cards", noise_free=True)


def test_fit_recovers_known_brightness_at_the_true_parameters(cards):
    sc = cards
    rng = np.random.default_rng(12)
    alphas = np.r_[1.0, rng.uniform(0.7, 1.3, sc.F - 1)]
    betas = np.r_[0.0, rng.uniform(-0.1, 0.1, sc.F - 1)]
    pb = oracle.Problem(_relit(sc, alphas, betas), sc.uv, sc.pattern, sc.vis, sc.intrinsics, sc.huber_k,
                        photometric=True)
    oracle.photo_update(pb, sc.poses_gt, sc.depths_gt)
    got = pb.photo.reshape(sc.F, 2)
    assert np.abs(got[1:, 0] - alphas[1:]).max() < 5e-3, (got, alphas)
    assert np.abs(got[1:, 1] - betas[1:]).max() < 5e-3, (got, betas)
    assert np.array_equal(got[0], [1.0, 0.0])  # the reference frame has no pair to fit


def test_identity_pair_reproduces_the_plain_model():
    sc = synth.make_scene("tiny")
    plain = oracle.Problem.from_scene(sc)
    photo = oracle.Problem.from_scene(sc, photometric=True)
    pre_a = oracle.ic_precompute(plain, sc.poses0, sc.depths0)
    pre_b = oracle.ic_precompute(photo, sc.poses0, sc.depths0)
    a = oracle.ic_step(plain, pre_a, sc.poses0, sc.depths0, sc.poses0, sc.depths0)
    b = oracle.ic_step(photo, pre_b, sc.poses0, sc.depths0, sc.poses0, sc.depths0)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])
    fa = oracle.fc_step(plain, sc.poses0, sc.depths0)
    photo2 = oracle.Problem.from_scene(sc, photometric=True)
    fb = oracle.fc_step(photo2, sc.poses0, sc.depths0)
    assert np.array_equal(fa[0], fb[0]) and np.array_equal(fa[1], fb[1])
    # the step then fitted the pairs to its residuals (positive gains)
    assert np.all(photo2.photo[2::2] > 0) and np.isfinite(photo2.photo).all()


def test_brightness_model_lowers_the_cost_under_lighting_changes():
    sc = synth.make_scene("small")
    alphas = np.r_[1.0, 0.75, 1.25, 0.8, 1.2, 0.9]
    betas = np.r_[0.0, 0.06, -0.05, 0.04, -0.06, 0.03]
    imgs = _relit(sc, alphas, betas)
    rms = {}
    for on in (False, True):
        pb = oracle.Problem(imgs, sc.uv, sc.pattern, sc.vis, sc.intrinsics, sc.huber_k, photometric=on)
        _, _, h = oracle.fc_run(pb, sc.poses0, sc.depths0, 10)
        rms[on] = h[-1, oracle.ST_RMS]
        if on:
            got = pb.photo.reshape(sc.F, 2)
            assert np.abs(got[1:, 0] - alphas[1:]).max() < 0.05
    assert rms[True] < 0.5 * rms[False], rms
