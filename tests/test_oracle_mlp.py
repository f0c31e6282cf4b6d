"""Pins of the learned-proposal oracle (oracle/mlp.py) to facts outside it:
the normal distribution function at known points, central finite
differences of the loss, a one-path network evaluated by hand, Adam's first
step in closed form, and features of linear-ramp images whose patch
statistics and epipolar projections have closed forms."""
import math

import numpy as np
import pytest

from oracle import mlp

pytestmark = pytest.mark.filterwarnings("ignore::RuntimeWarning")


def test_gelu_at_known_points():
    # Phi(1) = 0.841344746068543, Phi(-1) = 0.158655253931457, Phi(2) = 0.977249868051821
    assert mlp.gelu(np.array([0.0]))[0] == 0.0
    assert abs(mlp.gelu(np.array([1.0]))[0] - 0.841344746068543) < 1e-15
    assert abs(mlp.gelu(np.array([-1.0]))[0] + 0.158655253931457) < 1e-15
    assert abs(mlp.gelu(np.array([2.0]))[0] - 2 * 0.977249868051821) < 1e-14
    assert abs(mlp.gelu(np.array([-30.0]))[0]) < 1e-100
    x = np.linspace(-4, 4, 41)
    h = 1e-6
    fd = (mlp.gelu(x + h) - mlp.gelu(x - h)) / (2 * h)
    assert np.abs(fd - mlp.gelu_grad(x)).max() < 1e-9


def test_one_path_network_by_hand():
    # only W1[5, 2], W2[7, 5], W3[3, 7] and w4[3] are non-zero: y is a chain
    # of scalar GELUs; a transposed weight would route through zeros
    p = {k: np.zeros(s) for k, s in mlp.SHAPES}
    p["W1"][5, 2] = 1.5
    p["b1"][5] = -0.25
    p["W2"][7, 5] = -0.75
    p["b2"][7] = 0.5
    p["W3"][3, 7] = 2.0
    p["b3"][3] = 0.125
    p["w4"][3] = 0.6
    p["b4"][0] = 0.9
    X = np.zeros((2, mlp.N_IN))
    X[0, 2] = 0.8
    X[1, 2] = -1.3

    def g(x):
        return 0.5 * x * (1.0 + math.erf(x / math.sqrt(2.0)))

    y, _ = mlp.forward(p, X)
    for b in range(2):
        h1 = g(1.5 * X[b, 2] - 0.25)
        h2 = g(-0.75 * h1 + 0.5)
        h3 = g(2.0 * h2 + 0.125)
        assert abs(y[b] - (0.6 * h3 + 0.9)) < 1e-15


def test_gradient_matches_central_differences():
    rng = np.random.default_rng(3)
    p = mlp.init_params(7)
    # shrink to keep the FD well conditioned, perturb biases off zero
    for k in p:
        p[k] = p[k] * 0.7 + 0.05 * rng.normal(size=p[k].shape)
    X = rng.normal(size=(5, mlp.N_IN))
    T = rng.normal(1.0, 0.3, size=5)
    _, g = mlp.loss_and_grad(p, X, T)
    h = 1e-6
    for k, s in mlp.SHAPES:
        flat = p[k].ravel()
        idx = rng.choice(flat.size, size=min(6, flat.size), replace=False)
        for i in idx:
            old = flat[i]
            flat[i] = old + h
            lp, _ = mlp.loss_and_grad(p, X, T)
            flat[i] = old - h
            lm, _ = mlp.loss_and_grad(p, X, T)
            flat[i] = old
            fd = (lp - lm) / (2 * h)
            an = g[k].ravel()[i]
            assert abs(fd - an) <= 1e-7 * max(1.0, abs(fd)), (k, i, fd, an)


def test_adam_first_step_closed_form():
    # step 1 with zero moments: m = (1 - b1) g, v = (1 - b2) g^2, the bias
    # corrections cancel, so the move is lr * g / (|g| + eps)
    th = np.array([1.0, -2.0, 0.5])
    gr = np.array([0.3, -4.0, 0.0])
    t, m, v = mlp.adam_step(th, gr, np.zeros(3), np.zeros(3), 1, lr=0.01)
    assert np.allclose(t, th - 0.01 * gr / (np.abs(gr) + 1e-8), rtol=0, atol=1e-15)
    assert np.allclose(m, 0.1 * gr) and np.allclose(v, 0.001 * gr * gr)


def test_pack_roundtrip_and_size():
    p = mlp.init_params(1)
    v = mlp.pack(p)
    assert v.size == mlp.N_PARAMS == 96 * 128 + 128 + 2 * (128 * 128 + 128) + 128 + 1
    q = mlp.unpack(v)
    for k, _ in mlp.SHAPES:
        assert np.array_equal(p[k], q[k])


def _ramp(F, H, W, a, b, c):
    y, x = np.mgrid[0:H, 0:W]
    return np.stack([a[f] * x + b[f] * y + c[f] for f in range(F)]).astype(np.float64)


def test_features_of_linear_ramps():
    # bilinear interpolation is exact on I = a x + b y + c_f; the patch
    # statistics have closed forms (offsets -3..4: mean 0.5, variance 5.25);
    # with R = I and t = (tx, 0, 0) every pattern pixel moves by fx d tx
    # along its row, so with a common slope the matching cost of inverse
    # depth d is ((a fx tx d + c_g - c_0) / (sigma + eps))^2 for every pixel
    F, H, W = 4, 60, 160
    a, b, c = 0.002, 0.001, [0.1, 0.2, 0.3, 0.4]
    imgs = _ramp(F, H, W, [a] * F, [b] * F, c)
    K = (100.0, 100.0, 79.5, 29.5)
    poses = np.zeros((F, 12))
    poses[:, [0, 4, 8]] = 1.0
    poses[1, 9], poses[2, 9], poses[3, 9] = 0.05, 0.1, -0.08
    uv = np.array([[60, 30], [70, 25]], dtype=np.int32)
    vis = np.ones((2, F), np.uint8)
    vis[:, 0] = 0
    vis[0, 1] = 0  # point 0: frames 2 and 3; point 1: frames 1 and 2
    pat = np.array([(-1, -1), (1, -1), (-1, 1), (1, 1), (-2, 0), (2, 0), (0, -2), (0, 2)], np.int32)
    X = mlp.features(imgs, K, poses, uv, vis, pat)
    sig = math.sqrt(5.25 * (a ** 2 + b ** 2))
    s = 1.0 / (sig + mlp.EPS)
    dm = 0.5 + (np.arange(256) + 0.5) * 1.5 / 256
    for n, frames in ((0, (2, 3)), (1, (1, 2))):
        u, v = uv[n]
        mu = a * (u + 0.5) + b * (v + 0.5) + c[0]
        for i in range(8):
            for j in range(8):
                ref = (a * (u - 3 + j) + b * (v - 3 + i) + c[0] - mu) * s
                assert abs(X[n, 8 * i + j] - ref) < 1e-12
        for fi, g in enumerate(frames):
            cost = ((a * K[0] * poses[g, 9] * dm + c[g] - c[0]) * s) ** 2
            ref = cost.reshape(16, 16).min(1)
            assert np.abs(X[n, 64 + 16 * fi:64 + 16 * (fi + 1)] - ref).max() < 1e-9 * max(1.0, ref.max()), (n, g)


def test_matching_cost_is_zero_at_the_true_depth():
    # a textured reference warped exactly by the pose and a constant inverse
    # depth d*: the bin holding d* has (near) zero cost and is the least
    rng = np.random.default_rng(8)
    H, W = 80, 200
    base = rng.uniform(0, 1, size=(H, W))
    K = (100.0, 100.0, 99.5, 39.5)
    dstar = 1.2
    tx = 0.1
    shift = K[0] * dstar * tx  # pixels; a pure x translation keeps rows
    # frame 1 shows frame 0 moved by `shift` pixels: I_1(x + shift, y) = I_0(x, y)
    x = np.arange(W)
    img1 = np.stack([np.interp(x - shift, x, base[y]) for y in range(H)])
    imgs = np.stack([base, img1, img1])
    poses = np.zeros((3, 12))
    poses[:, [0, 4, 8]] = 1.0
    poses[1, 9] = poses[2, 9] = tx
    pat = np.array([(-1, -1), (1, -1), (-1, 1), (1, 1), (-2, 0), (2, 0), (0, -2), (0, 2)], np.int32)
    uv = np.array([[60, 40]], np.int32)
    vis = np.array([[0, 1, 1]], np.uint8)
    X = mlp.features(imgs, K, poses, uv, vis, pat)
    k = int((dstar - 0.5) / (1.5 / 16))
    bins = X[0, 64:80]
    assert bins.argmin() == k and bins[k] < 1e-3


def test_features_without_observations_have_no_matching_data():
    F, H, W = 3, 40, 40
    imgs = _ramp(F, H, W, [0.01] * F, [0.0] * F, [0.0] * F)
    poses = np.zeros((F, 12))
    poses[:, [0, 4, 8]] = 1.0
    X = mlp.features(imgs, (50.0, 50.0, 19.5, 19.5), poses, np.array([[20, 20]], np.int32),
                     np.zeros((1, F), np.uint8), np.array([(-1, 0), (1, 0)], np.int32))
    assert np.all(X[0, 64:] == mlp.NO_DATA) and X[0, :64].any()
