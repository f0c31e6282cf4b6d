"""Pins of the FP64 CPU oracle to things other than itself.

Each test checks the oracle against what the paper or the mathematics fixes:
library routines for textbook pieces (SO(3)/SE(3) exponentials), exactness
properties (bilinear on affine images, central differences on quadratics),
the paper's stated identities (Eq. warp at the identity, phi(x;0) = x, the
closed form of dphi/dDelta d), a hand-derived golden value, finite
differences of the definitions, dense linear algebra on the assembled
normal equations, the gauge null vector, and recovery of known parameters on
noise-free scenes where the one-depth-per-point model is exact.
"""
import json
import math
import os

import numpy as np
import pytest

import oracle
import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _rand_rot(rng, scale=0.5):
    from scipy.spatial.transform import Rotation
    return Rotation.from_rotvec(rng.normal(size=3) * scale).as_matrix()


# ----------------------------------------------------------------------------
# Lie groups (Sec. 1, Sec. 3 Notation)
# ----------------------------------------------------------------------------
@pytest.mark.parametrize("scale", [0.0, 1e-9, 1e-5, 4e-4, 2e-3, 0.3, 2.5])
def test_so3_exp_matches_library(scale):
    from scipy.spatial.transform import Rotation
    rng = np.random.default_rng(11)
    for _ in range(5):
        w = rng.normal(size=3)
        w = w / np.linalg.norm(w) * scale
        R = oracle.so3_exp(w)
        assert np.allclose(R, Rotation.from_rotvec(w).as_matrix(), atol=1e-14, rtol=0)
        assert np.allclose(R @ R.T, np.eye(3), atol=1e-14)
        assert np.allclose(oracle.so3_exp(-w), R.T, atol=1e-15)


@pytest.mark.parametrize("scale", [0.0, 1e-7, 5e-4, 0.2, 1.7])
def test_se3_exp_matches_matrix_exponential(scale):
    from scipy.linalg import expm
    rng = np.random.default_rng(12)
    for _ in range(5):
        v = rng.normal(size=3)
        w = rng.normal(size=3)
        w = w / np.linalg.norm(w) * scale
        X = np.zeros((4, 4))
        X[:3, :3] = [[0, -w[2], w[1]], [w[2], 0, -w[0]], [-w[1], w[0], 0]]
        X[:3, 3] = v
        T = expm(X)
        R, t = oracle.se3_exp(np.concatenate([v, w]))
        assert np.allclose(R, T[:3, :3], atol=1e-13)
        assert np.allclose(t, T[:3, 3], atol=1e-13)


# ----------------------------------------------------------------------------
# images (Sec. 3 Notation: bilinear)
# ----------------------------------------------------------------------------
def test_bilinear_exact_on_affine_images_and_pixels():
    H, W = 20, 30
    vv, uu = np.mgrid[0:H, 0:W].astype(float)
    img = 0.3 + 0.01 * uu - 0.02 * vv
    rng = np.random.default_rng(3)
    for _ in range(200):
        u = rng.uniform(1.0, W - 2.0 - 1e-9)
        v = rng.uniform(1.0, H - 2.0 - 1e-9)
        assert oracle.bilinear(img, u, v) == pytest.approx(0.3 + 0.01 * u - 0.02 * v, abs=1e-14)
    rnd = rng.random((H, W))
    assert oracle.bilinear(rnd, 7.0, 5.0) == rnd[5, 7]
    # validity: the 2x2 footprint must lie in [1, W-2] x [1, H-2]
    assert oracle.bilinear(rnd, 0.999, 5.0) is None
    assert oracle.bilinear(rnd, 1.0, 5.0) is not None
    assert oracle.bilinear(rnd, W - 3.0 + 0.5, 5.0) is not None
    assert oracle.bilinear(rnd, W - 2.0, 5.0) is None
    assert oracle.bilinear(rnd, 5.0, H - 2.0) is None


def test_central_gradient_exact_on_quadratics():
    H, W = 12, 14
    vv, uu = np.mgrid[0:H, 0:W].astype(float)
    img = 0.5 + 0.1 * uu - 0.03 * vv + 0.002 * uu * uu + 0.004 * uu * vv - 0.001 * vv * vv
    for (x, y) in [(1, 1), (5, 7), (12, 10)]:
        gu, gv = oracle.grad_central(img, x, y)
        assert gu == pytest.approx(0.1 + 0.004 * x + 0.004 * y, abs=1e-14)
        assert gv == pytest.approx(-0.03 + 0.004 * x - 0.002 * y, abs=1e-14)


def test_huber_norm_and_weight():
    k = 9.0 / 255.0
    # continuous at |r| = k, IRLS weight = rho'(r) / r
    assert oracle.huber_rho(k, k) == pytest.approx(0.5 * k * k)
    assert oracle.huber_rho(k * (1 + 1e-12), k) == pytest.approx(0.5 * k * k, rel=1e-9)
    for r in [-0.3, -k, -1e-3, 0.0, 1e-3, k, 0.05, 2.0]:
        h = 1e-7
        if abs(r) > 2 * h:
            drho = (oracle.huber_rho(r + h, k) - oracle.huber_rho(r - h, k)) / (2 * h)
            assert oracle.huber_weight(r, k) == pytest.approx(drho / r, rel=1e-6)
        assert 0.0 < oracle.huber_weight(r, k) <= 1.0


# ----------------------------------------------------------------------------
# warps (Sec. 3.1, Eq. warp)
# ----------------------------------------------------------------------------
def test_ordinary_warp_identity_has_zero_depth_derivative():
    """Sec. 3.1: at R = I, t = 0 the warp is the identity for any inverse
    depth and dW/dd = 0, the degeneracy that rules out ordinary IC."""
    rng = np.random.default_rng(5)
    for _ in range(20):
        x, y = rng.normal(size=2) * 0.4
        d = rng.uniform(0.2, 3.0)
        w, _, front = oracle.warp(np.eye(3), np.zeros(3), d, x, y)
        assert front and np.allclose(w, [x, y], atol=1e-15)
        h = 1e-3
        wp, _, _ = oracle.warp(np.eye(3), np.zeros(3), d + h, x, y)
        wm, _, _ = oracle.warp(np.eye(3), np.zeros(3), d - h, x, y)
        assert np.array_equal(wp, wm)
        # with a translation the depth derivative is non-zero
        t = rng.normal(size=3) * 0.3
        wp, _, _ = oracle.warp(np.eye(3), t, d + h, x, y)
        wm, _, _ = oracle.warp(np.eye(3), t, d - h, x, y)
        assert np.linalg.norm(wp - wm) > 1e-6


def test_ground_truth_is_consistent_with_the_renderer():
    """The warp at the true parameters lands every template pixel on the same
    albedo in the target image (the renderer ray-casts independently); noise-
    free residuals at the truth are tiny against those at p0."""
    sc = synth.make_scene("cards", noise_free=True)
    pb = oracle.Problem.from_scene(sc)
    st_gt = oracle.evaluate(pb, sc.poses_gt, sc.depths_gt)
    st_0 = oracle.evaluate(pb, sc.poses0, sc.depths0)
    assert st_gt[oracle.ST_COUNT] == sc.n_residuals()
    assert st_gt[oracle.ST_RMS] < 0.1 / 255.0
    assert st_0[oracle.ST_RMS] > 20 * st_gt[oracle.ST_RMS]


# ----------------------------------------------------------------------------
# proxy warp (Sec. 3.2 - 3.4)
# ----------------------------------------------------------------------------
def _rand_p0(rng):
    return _rand_rot(rng, 0.3), rng.normal(size=3) * 0.4, rng.uniform(0.6, 1.5)


def test_proxy_warp_identity_at_zero_update():
    """Eq. phi: phi(x; 0) = x (the identity moved to p0)."""
    rng = np.random.default_rng(21)
    for _ in range(50):
        R0, t0, d0 = _rand_p0(rng)
        x, y = rng.normal(size=2) * 0.3
        assert np.allclose(oracle.phi(R0, t0, d0, x, y, np.zeros(7)), [x, y], atol=1e-13)


def test_proxy_warp_jacobian_matches_finite_differences():
    """Closed form of Sec. 3.4 against central differences of Eq. phi0."""
    rng = np.random.default_rng(22)
    for _ in range(25):
        R0, t0, d0 = _rand_p0(rng)
        x, y = rng.normal(size=2) * 0.3
        J = oracle.phi_jacobian(R0, t0, d0, x, y)
        h = 1e-6
        Jfd = np.zeros((2, 7))
        for k in range(7):
            e = np.zeros(7)
            e[k] = h
            Jfd[:, k] = (oracle.phi(R0, t0, d0, x, y, e) - oracle.phi(R0, t0, d0, x, y, -e)) / (2 * h)
        assert np.abs(J - Jfd).max() <= 1e-7 * np.abs(Jfd).max()


def test_proxy_warp_depth_derivative_closed_form():
    """Sec. 3.4: dphi*/dDelta d = M t0 and dphi/dDelta d is non-zero for a
    non-zero t0; with M t0 = (zbar0 - t0_z) R0^T t0 and phi*(x;0) = zbar0 x~,
    dphi/dDelta d = ((zbar0 - t0_z)/zbar0) [[1,0,-x],[0,1,-y]] R0^T t0."""
    rng = np.random.default_rng(23)
    for _ in range(25):
        R0, t0, d0 = _rand_p0(rng)
        x, y = rng.normal(size=2) * 0.3
        zbar0 = (R0 @ [x, y, 1.0] + d0 * t0)[2] / d0
        expect = (zbar0 - t0[2]) / zbar0 * np.array([[1, 0, -x], [0, 1, -y]]) @ (R0.T @ t0)
        J = oracle.phi_jacobian(R0, t0, d0, x, y)
        assert np.allclose(J[:, 6], expect, atol=1e-13)
        assert np.linalg.norm(J[:, 6]) > 1e-4
    # t0 = 0: the proxy warp degenerates to the ordinary warp, dphi/dd = 0
    J = oracle.phi_jacobian(np.eye(3), np.zeros(3), 1.3, 0.1, 0.2)
    assert np.array_equal(J[:, 6], np.zeros(2))


def test_proxy_warp_jacobian_golden_hand_value():
    g = json.load(open(os.path.join(GOLDEN, "proxy_warp_hand.json")))
    inp = g["inputs"]
    J = oracle.phi_jacobian(np.array(inp["R0"], float), np.array(inp["t0"]), inp["d0"],
                            *inp["x"])
    assert np.allclose(J, np.array(g["dphi_dp"]), atol=1e-14)


def test_update_form_of_proxy_warp():
    """Eq. phi_update keeps the identity; for Delta t = 0, omega = 0 it is
    blind to Delta d (only the scale of the projected vector changes)."""
    rng = np.random.default_rng(24)
    for _ in range(10):
        R0, t0, d0 = _rand_p0(rng)
        x, y = rng.normal(size=2) * 0.3
        assert np.allclose(oracle.phi_update(R0, t0, d0, x, y, np.zeros(7)), [x, y], atol=1e-13)
        dp = np.zeros(7)
        dp[6] = 0.1
        assert np.allclose(oracle.phi_update(R0, t0, d0, x, y, dp), [x, y], atol=1e-13)


# ----------------------------------------------------------------------------
# Jacobian rows (Sec. 3.5) on images where bilinear sampling is exact
# ----------------------------------------------------------------------------
def _ramp_problem(F=3, N=6, a=0.4, b=0.0021, c=-0.0013, seed=31):
    rng = np.random.default_rng(seed)
    W, H, f = 120, 90, 100.0
    vv, uu = np.mgrid[0:H, 0:W].astype(float)
    imgs = np.stack([a + b * uu + c * vv + 0.0005 * i * uu for i in range(F)])
    uv = np.stack([rng.integers(40, 80, N), rng.integers(30, 60, N)], axis=1)
    vis = np.ones((N, F), np.uint8)
    vis[:, 0] = 0
    pb = oracle.Problem(imgs, uv, synth.PATTERN8, vis, [f, f, (W - 1) / 2, (H - 1) / 2], 9 / 255)
    poses = np.zeros((F, 12))
    poses[:, :9] = np.eye(3).ravel()
    for i in range(1, F):
        poses[i, :9] = _rand_rot(rng, 0.02).ravel()
        poses[i, 9:] = rng.normal(size=3) * 0.05
    depths = rng.uniform(0.8, 1.2, N)
    return pb, poses, depths


def test_ic_jacobian_row_matches_finite_difference_of_template_composition():
    """J = grad I_0 dphi/dDelta p (Sec. 3.5) equals d/dDelta p I_0(phi(x; Delta p))
    on a linear template image, where the central differences are exact."""
    pb, poses, depths = _ramp_problem()
    b, c = 0.0021, -0.0013
    for n in range(pb.N):
        for f in (1, 2):
            for j in (0, 5):
                J, r0, ok = oracle.ic_residual(pb, poses, depths, n, f, j)
                assert ok
                px, py = pb.uv[n] + pb.pat[j]
                x, y = (px - pb.cx) / pb.fx, (py - pb.cy) / pb.fy
                R0, t0 = poses[f, :9].reshape(3, 3), poses[f, 9:]

                def I0(dp):
                    ph = oracle.phi(R0, t0, depths[n], x, y, dp)
                    return 0.4 + b * (pb.fx * ph[0] + pb.cx) + c * (pb.fy * ph[1] + pb.cy)

                h = 1e-6
                fd = np.array([(I0(h * e) - I0(-h * e)) / (2 * h) for e in np.eye(7)])
                assert np.allclose(J, fd, atol=1e-9 * np.abs(fd).max())


def test_fc_jacobian_row_matches_finite_difference_of_residual():
    """FC row J = dr/dDelta p for the boxplus update (Sec. 3 Notation) against
    central differences of the residual on a linear target image."""
    pb, poses, depths = _ramp_problem()
    for n in range(pb.N):
        for f in (1, 2):
            for j in (1, 6):
                J, r, ok = oracle.fc_residual(pb, poses, depths, n, f, j)
                assert ok
                h = 1e-6
                fd = np.zeros(7)
                for k in range(7):
                    rr = []
                    for s in (1.0, -1.0):
                        dth = np.zeros((pb.F, 6))
                        dd = np.zeros(pb.N)
                        if k < 6:
                            dth[f, k] = s * h
                        else:
                            dd[n] = s * h
                        P2, D2 = oracle.fc_update(poses, depths, dth, dd)
                        rr.append(oracle.fc_residual(pb, P2, D2, n, f, j)[1])
                    fd[k] = (rr[0] - rr[1]) / (2 * h)
                assert np.allclose(J, fd, atol=1e-8 * np.abs(fd).max())


def test_fc_depth_column_vanishes_at_identity_pose():
    pb, poses, depths = _ramp_problem()
    poses[1, :9] = np.eye(3).ravel()
    poses[1, 9:] = 0.0
    J, _, ok = oracle.fc_residual(pb, poses, depths, 0, 1, 0)
    assert ok and J[6] == 0.0


# ----------------------------------------------------------------------------
# normal equations, Schur complement and the gauge (Sec. 3.5)
# ----------------------------------------------------------------------------
def _dense_ic(pb, pre):
    F, N = pb.F, pb.N
    rows, w = [], []
    for n in range(N):
        for f in range(1, F):
            for j in range(pb.P):
                rid = pre.rid(pb, n, f, j)
                if not pre.valid0[rid]:
                    continue
                row = np.zeros(6 * (F - 1) + N)
                row[6 * (f - 1):6 * f] = pre.J[rid, :6]
                row[6 * (F - 1) + n] = pre.J[rid, 6]
                rows.append(row)
                w.append(pre.w0[rid])
    return np.array(rows), np.array(w)


@pytest.fixture(scope="module")
def tiny():
    sc = synth.make_scene("tiny")
    pb = oracle.Problem.from_scene(sc)
    pre = oracle.ic_precompute(pb, sc.poses0, sc.depths0)
    return sc, pb, pre


def test_hessian_blocks_equal_JtW0J_symmetric_psd_with_one_gauge(tiny):
    sc, pb, pre = tiny
    F, N = pb.F, pb.N
    J, w = _dense_ic(pb, pre)
    H = J.T @ (w[:, None] * J)
    for f in range(1, F):
        assert np.allclose(pre.Hff[f], H[6 * (f - 1):6 * f, 6 * (f - 1):6 * f], rtol=1e-12,
                           atol=1e-12 * np.abs(H).max())
    for n in range(N):
        assert pre.Hdd[n] == pytest.approx(H[6 * (F - 1) + n, 6 * (F - 1) + n], rel=1e-12, abs=1e-300)
        for f in range(1, F):
            assert np.allclose(pre.Hfd[n, f], H[6 * (f - 1):6 * f, 6 * (F - 1) + n],
                               atol=1e-12 * np.abs(H).max())
    assert np.array_equal(pre.Hff[1], pre.Hff[1].T)
    # keep only the points that have residuals (others are excluded by design)
    keep = np.concatenate([np.arange(6 * (F - 1)), 6 * (F - 1) + np.flatnonzero(pre.Hdd > 0)])
    ev = np.linalg.eigvalsh(H[np.ix_(keep, keep)])
    assert ev[0] >= -1e-12 * ev[-1]
    assert ev[0] < 1e-9 * ev[-1]          # the scale gauge
    assert ev[1] > 1e-7 * ev[-1]          # and nothing else


def test_gauge_null_vector_ic_and_fc(tiny):
    sc, pb, pre = tiny
    F, N = pb.F, pb.N
    J, _ = _dense_ic(pb, pre)
    v = np.zeros(6 * (F - 1) + N)
    for f in range(1, F):
        v[6 * (f - 1):6 * (f - 1) + 3] = -sc.poses0[f, 9:]
    v[6 * (F - 1):] = sc.depths0
    assert np.abs(J @ v).max() < 1e-12 * np.abs(J).max() * np.abs(v).max()
    # FC at p0: upsilon_f = -t_f, dd = d
    for n in range(N):
        for f in range(1, F):
            if not sc.vis[n, f]:
                continue
            for j in range(pb.P):
                Jr, _, ok = oracle.fc_residual(pb, sc.poses0, sc.depths0, n, f, j)
                if ok:
                    val = Jr[:3] @ (-sc.poses0[f, 9:]) + Jr[6] * sc.depths0[n]
                    assert abs(val) < 1e-12 * max(1.0, np.abs(Jr).max())


def test_schur_solution_solves_the_full_normal_equations(tiny):
    sc, pb, pre = tiny
    F, N = pb.F, pb.N
    g_theta, g_d, _ = oracle.ic_gradient(pb, pre, sc.poses0, sc.depths0)
    dtheta, dd, _ = oracle.schur_solve(F, N, pre.Hff, pre.Hfd, pre.Hdd, g_theta, g_d,
                                       sc.poses0[:, 9:])
    J, w = _dense_ic(pb, pre)
    H = J.T @ (w[:, None] * J)
    g = np.concatenate([g_theta[1:].ravel(), g_d])
    dp = np.concatenate([dtheta[1:].ravel(), dd])
    assert np.abs(H @ dp + g).max() < 1e-9 * np.abs(g).max()
    # a dense least-squares solve differs only along the gauge direction
    keep = np.concatenate([np.arange(6 * (F - 1)), 6 * (F - 1) + np.flatnonzero(pre.Hdd > 0)])
    dp_ls = np.zeros_like(dp)
    dp_ls[keep] = np.linalg.lstsq(H[np.ix_(keep, keep)], -g[keep], rcond=1e-12)[0]
    v = np.zeros_like(dp)
    for f in range(1, F):
        v[6 * (f - 1):6 * (f - 1) + 3] = -sc.poses0[f, 9:]
    v[6 * (F - 1):] = np.where(pre.Hdd > 0, sc.depths0, 0.0)
    diff = dp - dp_ls
    resid = diff - v * (diff @ v) / (v @ v)
    assert np.abs(resid).max() < 1e-8 * np.abs(dp).max()
    # the chosen gauge: no translation increment of the anchor frame along t0
    t1 = sc.poses0[1, 9:] / np.linalg.norm(sc.poses0[1, 9:])
    assert abs(dtheta[1, :3] @ t1) < 1e-10 * np.abs(dtheta).max()


@pytest.mark.parametrize("lam", [0.05, 0.7])
def test_damped_schur_solution_matches_the_dense_damped_solve(tiny, lam):
    """Levenberg-Marquardt (beyond the paper's Gauss-Newton): the Schur path
    with every diagonal entry of H scaled by 1 + lambda gives the frame update
    of the dense damped solve up to the scale null vector (Delta t_f ~ t_f),
    fixes the gauge (t_a . Delta t_a = 0) and back-substitutes the depths from
    the damped point equations."""
    sc, pb, pre = tiny
    F, N = pb.F, pb.N
    g_theta, g_d, _ = oracle.ic_gradient(pb, pre, sc.poses0, sc.depths0)
    dth, dd, _ = oracle.schur_solve(F, N, pre.Hff, pre.Hfd, pre.Hdd, g_theta, g_d, sc.poses0[:, 9:],
                                    damping=lam)
    J, w = _dense_ic(pb, pre)
    H = J.T @ (w[:, None] * J)
    H = H + lam * np.diag(np.diag(H))
    g = np.concatenate([g_theta[1:].ravel(), g_d])
    keep = np.concatenate([np.arange(6 * (F - 1)), 6 * (F - 1) + np.flatnonzero(pre.Hdd > 0)])
    dp = np.zeros(6 * (F - 1) + N)
    dp[keep] = np.linalg.solve(H[np.ix_(keep, keep)], -g[keep])
    diff = (dth[1:] - dp[:6 * (F - 1)].reshape(F - 1, 6))
    assert np.abs(diff[:, 3:]).max() < 1e-9 * np.abs(dth).max()
    t = sc.poses0[1:, 9:]
    alpha = -(diff[:, :3] * t).sum() / (t * t).sum()
    assert np.abs(diff[:, :3] + alpha * t).max() < 1e-9 * np.abs(dth).max()
    assert abs(alpha) > 1e-6 * np.abs(dth).max()  # the damped step does move along the gauge
    t1 = sc.poses0[1, 9:]
    assert abs(dth[1, :3] @ t1) < 1e-12 * np.abs(dth).max()
    Hdp = np.array([pre.Hfd[n, 1:].ravel() for n in range(N)])
    r = pre.Hdd * (1 + lam) * dd + Hdp @ dth[1:].ravel() + g_d
    assert np.abs(r[pre.Hdd > 0]).max() < 1e-9 * np.abs(g_d).max()


# ----------------------------------------------------------------------------
# updates (Sec. 3.6)
# ----------------------------------------------------------------------------
def test_ic_update_round_trip_is_second_order():
    """phi^-1 ~ phi(-Delta p) (Sec. 3.6): applying the update with Delta p and
    then -Delta p returns R exactly and t, d to O(|Delta p|^2)."""
    rng = np.random.default_rng(41)
    F, N = 4, 5
    poses0 = np.zeros((F, 12))
    poses0[:, :9] = np.eye(3).ravel()
    for f in range(1, F):
        poses0[f, :9] = _rand_rot(rng, 0.3).ravel()
        poses0[f, 9:] = rng.normal(size=3)
    depths0 = rng.uniform(0.5, 1.5, N)
    poses = poses0.copy()
    for f in range(1, F):
        poses[f, :9] = (_rand_rot(rng, 0.05) @ poses0[f, :9].reshape(3, 3)).ravel()
        poses[f, 9:] += rng.normal(size=3) * 0.05
    depths = depths0 * (1 + 0.05 * rng.normal(size=N))
    gaps = []
    for eps in (1e-2, 5e-3):
        dth = rng.normal(size=(F, 6)) * eps
        dth[0] = 0
        dd = rng.normal(size=N) * eps
        P1, D1 = oracle.ic_update(poses0, depths0, poses, depths, dth, dd)
        P2, D2 = oracle.ic_update(poses0, depths0, P1, D1, -dth, -dd)
        assert np.allclose(P2[:, :9], poses[:, :9], atol=1e-14)
        gaps.append(max(np.abs(P2 - poses).max(), np.abs(D2 - depths).max()) / eps ** 2)
        assert gaps[-1] < 10.0
    rng2 = np.random.default_rng(41)
    assert gaps[0] > 0


def test_ic_update_at_p0_is_boxplus_of_minus_dp():
    """At p = p0 the Sec. 3.6 rules give R = exp(-omega) R0, t = t0 - Dt,
    d = d0 - Dd, i.e. p0 (+) (-Delta p) with the proxy parameterisation."""
    rng = np.random.default_rng(42)
    F, N = 3, 4
    poses0 = np.zeros((F, 12))
    poses0[:, :9] = np.eye(3).ravel()
    for f in range(1, F):
        poses0[f, :9] = _rand_rot(rng).ravel()
        poses0[f, 9:] = rng.normal(size=3)
    depths0 = rng.uniform(0.5, 1.5, N)
    dth = rng.normal(size=(F, 6)) * 0.1
    dth[0] = 0
    dd = rng.normal(size=N) * 0.1
    P1, D1 = oracle.ic_update(poses0, depths0, poses0, depths0, dth, dd)
    from scipy.spatial.transform import Rotation
    for f in range(1, F):
        Rexp = Rotation.from_rotvec(-dth[f, 3:]).as_matrix() @ poses0[f, :9].reshape(3, 3)
        assert np.allclose(P1[f, :9].reshape(3, 3), Rexp, atol=1e-14)
        assert np.allclose(P1[f, 9:], poses0[f, 9:] - dth[f, :3], atol=1e-14)
    assert np.allclose(D1, depths0 - dd, atol=1e-15)


def _first_step_gap(eps):
    """Relative gaps between the parameters one IC step and one FC step reach
    from the same p_0 (rotation, translation, inverse depth blocks), on
    noise-free cards perturbed by eps times (0.5 deg, 0.005, 1 %)."""
    from scipy.spatial.transform import Rotation
    sc = synth.make_scene("cards", noise_free=True, rot_deg=0.5 * eps, trans=0.005 * eps, sigma_d=0.01 * eps)
    pb = oracle.Problem.from_scene(sc)
    pre = oracle.ic_precompute(pb, sc.poses0, sc.depths0)
    _, _, Pi, Di, _ = oracle.ic_step(pb, pre, sc.poses0, sc.depths0, sc.poses0, sc.depths0)
    _, _, Pf, Df, _ = oracle.fc_step(pb, sc.poses0, sc.depths0)
    P0 = sc.poses0
    blocks = {"rot": ([], []), "trans": ([], [])}
    for f in range(1, sc.F):
        R0t = P0[f, :9].reshape(3, 3).T
        for P, k in ((Pi, 0), (Pf, 1)):
            blocks["rot"][k].append(Rotation.from_matrix(P[f, :9].reshape(3, 3) @ R0t).as_rotvec())
            blocks["trans"][k].append(P[f, 9:] - P0[f, 9:])
    blocks["depth"] = ([Di - sc.depths0], [Df - sc.depths0])
    return {k: np.linalg.norm(np.concatenate(a) - np.concatenate(b)) / np.linalg.norm(np.concatenate(b))
            for k, (a, b) in blocks.items()}


def test_ic_and_fc_first_steps_agree_to_first_order():
    """Baker and Matthews' equivalence of the inverse and forwards
    compositional updates (cited in Sec. 2): from the same p_0 on exact data
    the two first steps differ by a term of second order in the
    perturbation, so their relative gap shrinks in proportion to it. A wrong
    sign or a swapped column in either Jacobian, or in either update rule,
    leaves a gap of order one."""
    g1, g2 = _first_step_gap(0.25), _first_step_gap(0.0625)
    for k in ("rot", "trans", "depth"):
        assert g2[k] < 0.15, (k, g1, g2)
        assert g1[k] / g2[k] > 2.5, (k, g1, g2)  # 4x smaller perturbation


# ----------------------------------------------------------------------------
# whole solves on noise-free data where the model is exact
# ----------------------------------------------------------------------------
def _errors(sc, poses, depths):
    s = (sc.depths_gt * depths).sum() / (depths * depths).sum()
    rot, tr = [], []
    for f in range(1, sc.F):
        if not sc.vis[:, f].any():
            continue
        R = poses[f, :9].reshape(3, 3)
        Rg = sc.poses_gt[f, :9].reshape(3, 3)
        rot.append(math.degrees(math.acos(np.clip((np.trace(R @ Rg.T) - 1) / 2, -1, 1))))
        tr.append(np.linalg.norm(poses[f, 9:] / s - sc.poses_gt[f, 9:]))
    return max(rot), max(tr), np.median(np.abs(s * depths / sc.depths_gt - 1))


def test_fc_recovers_known_parameters_on_noise_free_cards():
    sc = synth.make_scene("cards", noise_free=True)       # 2 deg / 0.02 / 5 %
    pb = oracle.Problem.from_scene(sc)
    P, D, hist = oracle.fc_run(pb, sc.poses0, sc.depths0, 20)
    rot, tr, dep = _errors(sc, P, D)
    assert rot < 0.05 and tr < 1e-3 and dep < 5e-3
    assert hist[-2, oracle.ST_MAXDISP] < 5e-3              # converged (Sec. 4.1 rule)
    gt = oracle.evaluate(pb, sc.poses_gt, sc.depths_gt)
    assert hist[-1, oracle.ST_RMS] <= 1.05 * gt[oracle.ST_RMS]


def test_ic_recovers_known_parameters_on_noise_free_cards():
    sc = synth.make_scene("cards", noise_free=True, rot_deg=0.5, trans=0.005, sigma_d=0.01)
    pb = oracle.Problem.from_scene(sc)
    P, D, hist = oracle.ic_run(pb, sc.poses0, sc.depths0, 25)
    rot, tr, dep = _errors(sc, P, D)
    assert rot < 0.05 and tr < 1e-3 and dep < 5e-3
    assert hist[-2, oracle.ST_MAXDISP] < 5e-3
    # IC's fixed point: J_0^T W r = 0 (its own stationarity condition)
    pre = oracle.ic_precompute(pb, sc.poses0, sc.depths0)
    g0 = oracle.ic_gradient(pb, pre, sc.poses0, sc.depths0)
    g1 = oracle.ic_gradient(pb, pre, P, D)
    assert np.abs(g1[0]).max() < 1e-3 * np.abs(g0[0]).max()
    # and it lands near FC's solution: the two fixed points differ (J_0 vs J(p)
    # in the stationarity condition) by the interpolation-limited bias only
    Pf, Df, _ = oracle.fc_run(pb, sc.poses0, sc.depths0, 20)
    assert oracle.max_reproj_disp(pb, P, D, Pf, Df) < 0.25


def test_ic_contracts_linearly_from_a_modest_perturbation():
    """The Sec. 3.6 update is p0 (+) (-Delta p) at p0 while the Jacobian holds
    the full first-order proxy warp, so IC contracts linearly; the step sizes
    of consecutive iterations shrink by a steady ratio below one."""
    sc = synth.make_scene("cards", noise_free=True, rot_deg=0.5, trans=0.005, sigma_d=0.01)
    pb = oracle.Problem.from_scene(sc)
    _, _, hist = oracle.ic_run(pb, sc.poses0, sc.depths0, 16)
    d = hist[:-1, oracle.ST_MAXDISP]
    ratios = d[9:15] / d[8:14]
    assert (ratios < 0.9).all() and (ratios > 0.05).all()


# ----------------------------------------------------------------------------
# the convergence measure of Sec. 4.1: the largest pattern-centre
# reprojection displacement between two parameter sets
# ----------------------------------------------------------------------------
def _disp_problem(F=4, N=7, seed=5):
    rng = np.random.default_rng(seed)
    W, H = 64, 48
    fx, fy, cx, cy = 300.0, 200.0, 31.5, 23.5
    uv = np.stack([rng.integers(4, W - 4, N), rng.integers(4, H - 4, N)], 1).astype(np.int32)
    vis = np.ones((N, F), np.uint8)
    pb = oracle.Problem(np.zeros((F, H, W)), uv, np.zeros((1, 2), np.int32), vis, (fx, fy, cx, cy), 0.1)
    depths = rng.uniform(0.5, 2.0, N)
    poses = np.tile(np.r_[np.eye(3).ravel(), 0.0, 0.0, 0.0], (F, 1))
    return pb, poses, depths


def test_max_reprojection_displacement_of_a_translation_is_f_d_delta():
    """With R = I and t_z = 0 the warp is x + d t, so shifting one frame's
    translation by (dx, dy, 0) moves every point it sees by
    d (f_x dx, f_y dy) pixels; the measure is that length at the largest
    inverse depth. Shifts along each axis separate f_x from f_y."""
    pb, poses, depths = _disp_problem()
    for delta, f_axis in (((1e-3, 0.0), pb.fx), ((0.0, 1e-3), pb.fy)):
        shifted = poses.copy()
        shifted[2, 9:11] += delta
        got = oracle.max_reproj_disp(pb, poses, depths, shifted, depths)
        assert got == pytest.approx(f_axis * depths.max() * 1e-3, rel=1e-12)
    # both axes at once: the Euclidean length of the pixel displacement
    shifted = poses.copy()
    shifted[1, 9:11] += (3e-4, 4e-4)
    got = oracle.max_reproj_disp(pb, poses, depths, shifted, depths)
    assert got == pytest.approx(depths.max() * math.hypot(pb.fx * 3e-4, pb.fy * 4e-4), rel=1e-12)


def test_max_reprojection_displacement_skips_unseen_pairs_and_the_reference():
    pb, poses, depths = _disp_problem()
    n_far = int(np.argmax(depths))
    shifted = poses.copy()
    shifted[0, 9] += 1.0      # the reference frame has no residuals
    shifted[3, 9] += 1e-3
    vis = pb.vis.copy()
    vis[n_far, 3] = 0         # the largest inverse depth is not seen in frame 3
    pb2 = oracle.Problem(pb.img, pb.uv, pb.pat, vis, (pb.fx, pb.fy, pb.cx, pb.cy), 0.1)
    got = oracle.max_reproj_disp(pb2, poses, depths, shifted, depths)
    second = np.sort(depths)[-2]
    assert got == pytest.approx(pb.fx * second * 1e-3, rel=1e-12)


def test_max_reprojection_displacement_of_a_depth_change_and_a_roll():
    pb, poses, depths = _disp_problem()
    # a depth change with t = (t_x, 0, 0): the point moves f_x t_x |Dd| pixels
    poses_t = poses.copy()
    poses_t[1:, 9] = 0.1
    dd = np.linspace(-2e-3, 3e-3, pb.N)
    got = oracle.max_reproj_disp(pb, poses_t, depths, poses_t, depths + dd)
    assert got == pytest.approx(pb.fx * 0.1 * np.abs(dd).max(), rel=1e-9)
    # a roll by theta about the optical axis at t = 0: the normalised centre
    # (x, y) turns in its plane, the pixel displacement scales by (f_x, f_y)
    th = 0.01
    rolled = poses.copy()
    c, s = math.cos(th), math.sin(th)
    rolled[2, :9] = [c, -s, 0, s, c, 0, 0, 0, 1]
    x = (pb.uv[:, 0] - pb.cx) / pb.fx
    y = (pb.uv[:, 1] - pb.cy) / pb.fy
    du = pb.fx * ((c - 1) * x - s * y)
    dv = pb.fy * (s * x + (c - 1) * y)
    got = oracle.max_reproj_disp(pb, poses, depths, rolled, depths)
    assert got == pytest.approx(np.hypot(du, dv).max(), rel=1e-9)
