"""Pins of the oracle's joint brightness step (or_ic_step_joint: the pairs
(alpha_f, beta_f) as Gauss-Newton unknowns of the IC system, an option
beyond the paper, whose Sec. 2 notes that direct methods must model
lighting), each against something other than the oracle's own formulas:

- exact recovery: with the identity warp and targets that are affine images
  of the template, the residual lies in the span of the two brightness
  columns, so one step must land on the true pairs and leave the geometry;
- dense least squares: the first step equals the minimiser of the weighted
  linearised cost over all unknowns (poses, pairs and depths in one dense
  system, solved by numpy) in every component the scale gauge leaves fixed;
- the composed update: the residual after or_photo_compose moves, to first
  order, by I_0 da + db (the template-side increment the columns model).
"""
import numpy as np
import pytest

import oracle
import synth


def _identity_warp_problem(alphas, betas, huber_k=None, photo_prior=0.0):
    """Every frame sees the template through the identity pose; frame f is
    the template mapped so that alpha_f I_f + beta_f = I_0."""
    sc = synth.make_scene("small", noise_free=True)
    I0 = sc.images_f32[0].astype(np.float64)
    imgs = np.stack([I0] + [(I0 - betas[f]) / alphas[f] for f in range(1, sc.F)])
    poses = np.zeros((sc.F, 12))
    poses[:, [0, 4, 8]] = 1.0
    vis = np.ones((sc.N, sc.F), np.uint8)
    k = sc.huber_k if huber_k is None else huber_k
    pb = oracle.Problem(imgs, sc.uv, sc.pattern, vis, sc.intrinsics, k, photometric=True,
                        photo_prior=photo_prior)
    return sc, pb, poses


def test_joint_step_recovers_affine_brightness_exactly():
    rng = np.random.default_rng(3)
    F = synth.make_scene("small", noise_free=True).F
    alphas = np.r_[1.0, rng.uniform(0.7, 1.3, F - 1)]
    betas = np.r_[0.0, rng.uniform(-0.1, 0.1, F - 1)]
    sc, pb, poses = _identity_warp_problem(alphas, betas)
    d = sc.depths_gt
    pre = oracle.ic_precompute(pb, poses, d)
    dth, dab, dd, P1, D1, _ = oracle.ic_step_joint(pb, pre, poses, d, poses, d)
    got = pb.photo.reshape(F, 2)
    assert np.abs(got[1:, 0] - alphas[1:]).max() < 1e-9, (got, alphas)
    assert np.abs(got[1:, 1] - betas[1:]).max() < 1e-9, (got, betas)
    assert np.array_equal(got[0], [1.0, 0.0])
    assert np.abs(dth).max() < 1e-9 and np.abs(dd).max() == 0.0
    # the increments themselves: (1 + da) I_0 + db = I_0 / alpha - beta / alpha
    assert np.allclose(dab[1:, 0], 1.0 / alphas[1:] - 1.0, atol=1e-9)
    assert np.allclose(dab[1:, 1], -betas[1:] / alphas[1:], atol=1e-9)
    # at the solution the next step is zero
    dth2, dab2, _, _, _, st = oracle.ic_step_joint(pb, pre, poses, d, P1, D1)
    assert np.abs(dab2).max() < 1e-9 and np.abs(dth2).max() < 1e-9
    assert st[oracle.ST_RMS] < 1e-9


def _dense_first_step(sc, pb, pre, prior=0.0):
    """Minimiser of sum w0 (r0 + J Delta)^2 over [per frame: Delta t, omega,
    da, db | per point: Delta d] from the precompute's rows (the step at p_0,
    where the current weights are W_0), by numpy least squares; with prior,
    also the rows sqrt(W_f) (ln alpha_f - da_f), sqrt(W_f) (beta_f - db_f),
    W_f = prior * sum of the frame's w0."""
    F, N, P = pb.F, pb.N, pb.P
    I0 = pb.img[0]
    rows, rhs = [], []
    nf = 8 * (F - 1)
    if prior > 0.0:
        for f in range(1, F):
            W = prior * sum(pre.w0[pre.rid(pb, n, f, j)] for n in range(N) for j in range(P)
                            if pre.valid0[pre.rid(pb, n, f, j)])
            for b, target in ((0, np.log(pb.photo[2 * f])), (1, pb.photo[2 * f + 1])):
                row = np.zeros(nf + N)
                row[8 * (f - 1) + 6 + b] = -np.sqrt(W)
                rows.append(row)
                rhs.append(-np.sqrt(W) * target)
    for n in range(N):
        for f in range(1, F):
            if not pb.vis[n, f]:
                continue
            for j in range(P):
                i = pre.rid(pb, n, f, j)
                if not pre.valid0[i]:
                    continue
                row = np.zeros(nf + N)
                px, py = pb.uv[n] + pb.pat[j]
                row[8 * (f - 1):8 * (f - 1) + 6] = pre.J[i, :6]
                row[8 * (f - 1) + 6] = I0[py, px]
                row[8 * (f - 1) + 7] = 1.0
                row[nf + n] = pre.J[i, 6]
                s = np.sqrt(pre.w0[i])
                rows.append(s * row)
                rhs.append(-s * pre.r0[i])
    x = np.linalg.lstsq(np.array(rows), np.array(rhs), rcond=None)[0]
    return x[:nf].reshape(F - 1, 8), x[nf:]


def test_joint_first_step_is_the_dense_least_squares_minimiser():
    """Components the scale gauge leaves fixed (rotations, brightness
    increments) match the dense minimiser; the gauge direction (translations
    and depths scaled together) is where the two may differ."""
    sc = synth.make_scene("tiny")
    rng = np.random.default_rng(5)
    alphas = np.r_[1.0, rng.uniform(0.8, 1.2, sc.F - 1)]
    betas = np.r_[0.0, rng.uniform(-0.05, 0.05, sc.F - 1)]
    imgs = sc.images_f32.astype(np.float64).copy()
    for f in range(1, sc.F):
        imgs[f] = (imgs[f] - betas[f]) / alphas[f]
    pb = oracle.Problem(imgs, sc.uv, sc.pattern, sc.vis, sc.intrinsics, sc.huber_k, photometric=True)
    pre = oracle.ic_precompute(pb, sc.poses0, sc.depths0)
    dense, _ = _dense_first_step(sc, pb, pre)
    dth, dab, _, _, _, _ = oracle.ic_step_joint(pb, pre, sc.poses0, sc.depths0, sc.poses0, sc.depths0)
    rot = dense[:, 3:6]
    assert np.abs(dth[1:, 3:] - rot).max() <= 1e-6 * np.abs(rot).max(), (dth[1:, 3:], rot)
    ph = dense[:, 6:]
    assert np.abs(dab[1:] - ph).max() <= 1e-6 * np.abs(ph).max(), (dab[1:], ph)
    # the translations differ from the dense minimiser by the scale gauge
    # only: t_f -> t_f + c Delta t_f with the same c for every frame
    t0 = sc.poses0[1:, 9:]
    diff = dth[1:, :3] - dense[:, :3]
    c = np.sum(diff * t0) / np.sum(t0 * t0)
    assert np.abs(diff - c * t0).max() <= 1e-5 * np.abs(dense[:, :3]).max()


@pytest.mark.parametrize("da,db", [(1e-6, 0.0), (0.0, 1e-6), (-7e-7, 4e-7)])
def test_composed_update_moves_the_residual_by_the_template_increment(da, db):
    rng = np.random.default_rng(9)
    F = synth.make_scene("small", noise_free=True).F
    alphas = np.r_[1.0, rng.uniform(0.7, 1.3, F - 1)]
    betas = np.r_[0.0, rng.uniform(-0.1, 0.1, F - 1)]
    sc, pb, poses = _identity_warp_problem(alphas, betas)
    pb.photo[:] = np.c_[alphas, betas].ravel()  # the true pairs: every residual is zero
    I0 = pb.img[0]
    for (n, f, j) in [(0, 1, 0), (17, 2, 5), (123, F - 1, 7)]:
        ab = pb.photo[2 * f:2 * f + 2].copy()
        _, r, ok = oracle.ic_residual(pb, poses, sc.depths_gt, n, f, j)
        assert ok and abs(r) < 1e-12
        pb.photo[2 * f:2 * f + 2] = oracle.photo_compose(ab, [da, db])
        _, r1, _ = oracle.ic_residual(pb, poses, sc.depths_gt, n, f, j)
        pb.photo[2 * f:2 * f + 2] = ab
        px, py = pb.uv[n] + pb.pat[j]
        model = I0[py, px] * da + db
        # exactly r1 = (I_0 da + db) / (1 + da): the model up to O(da (|da| + |db|))
        assert abs(r1 - model) <= 2.0 * abs(da) * (abs(da) + abs(db)) + 1e-14, (r1, model)
        assert abs(r1 - model) <= 1e-5 * abs(model)


def test_prior_step_is_the_dense_minimiser_with_the_prior_rows():
    """At pairs off the truth (identity warp, zero depth coupling), the step
    with the prior is the dense minimiser of the linearised data cost plus
    the prior rows; without the prior it is the exact recovery."""
    rng = np.random.default_rng(4)
    F = synth.make_scene("small", noise_free=True).F
    alphas = np.r_[1.0, rng.uniform(0.7, 1.3, F - 1)]
    betas = np.r_[0.0, rng.uniform(-0.1, 0.1, F - 1)]
    sc, pb, poses = _identity_warp_problem(alphas, betas, photo_prior=0.3)
    start = np.r_[1.0, 0.0, np.c_[rng.uniform(0.8, 1.2, F - 1), rng.uniform(-0.05, 0.05, F - 1)].ravel()]
    pb.photo[:] = start
    d = sc.depths_gt
    pre = oracle.ic_precompute(pb, poses, d)
    dense, _ = _dense_first_step(sc, pb, pre, prior=0.3)
    dth, dab, _, _, _, _ = oracle.ic_step_joint(pb, pre, poses, d, poses, d)
    assert np.abs(dab[1:] - dense[:, 6:]).max() <= 1e-8 * np.abs(dense[:, 6:]).max()
    assert np.abs(dth[1:] - dense[:, :6]).max() <= 1e-8 * max(np.abs(dense[:, :6]).max(), 1e-12)
    # the prior changes the step (without it the step lands on the truth)
    pb0 = _identity_warp_problem(alphas, betas)[1]
    pb0.photo[:] = start
    pre0 = oracle.ic_precompute(pb0, poses, d)
    _, dab0, _, _, _, _ = oracle.ic_step_joint(pb0, pre0, poses, d, poses, d)
    assert np.abs(dab0 - dab).max() > 1e-2
    assert np.abs(pb0.photo.reshape(F, 2)[1:] - np.c_[alphas, betas][1:]).max() < 1e-9


# ----------------------------------------------------------------------------
# FC with the pairs as unknowns (or_fc_step_joint): target-side columns
# -I_f and -1 at the current parameters, additive pair update
# ----------------------------------------------------------------------------
def _relit_tiny(seed=5):
    sc = synth.make_scene("tiny")
    rng = np.random.default_rng(seed)
    alphas = np.r_[1.0, rng.uniform(0.8, 1.2, sc.F - 1)]
    betas = np.r_[0.0, rng.uniform(-0.05, 0.05, sc.F - 1)]
    imgs = sc.images_f32.astype(np.float64).copy()
    for f in range(1, sc.F):
        imgs[f] = (imgs[f] - betas[f]) / alphas[f]
    return sc, imgs


def test_fc_joint_columns_are_finite_differences_of_the_residual():
    sc, imgs = _relit_tiny()
    pb = oracle.Problem(imgs, sc.uv, sc.pattern, sc.vis, sc.intrinsics, sc.huber_k, photometric=True)
    pb.photo[2:] = np.c_[np.linspace(0.9, 1.1, sc.F - 1), np.linspace(-0.02, 0.03, sc.F - 1)].ravel()
    P, D = sc.poses0, sc.depths0
    checked = 0
    for n in range(0, sc.N, 7):
        for f in range(1, sc.F):
            if not sc.vis[n, f]:
                continue
            J, r, ok = oracle.fc_residual_joint(pb, P, D, n, f, 3)
            if not ok:
                continue
            for k, idx in ((6, 2 * f), (7, 2 * f + 1)):
                h = 1e-6
                keep = pb.photo[idx]
                pb.photo[idx] = keep + h
                rp = oracle.fc_residual_joint(pb, P, D, n, f, 3)[1]
                pb.photo[idx] = keep - h
                rm = oracle.fc_residual_joint(pb, P, D, n, f, 3)[1]
                pb.photo[idx] = keep
                assert abs((rp - rm) / (2 * h) - J[k]) <= 1e-7, (n, f, k)
            # (the pose and depth columns use the central-difference image
            # gradient, pinned with or_fc_residual; they are not the
            # derivative of the bilinear sample)
            assert np.array_equal(J[[0, 1, 2, 3, 4, 5, 8]], oracle.fc_residual(pb, P, D, n, f, 3)[0])
            checked += 1
    assert checked > 20


def test_fc_joint_step_recovers_affine_brightness_exactly():
    rng = np.random.default_rng(7)
    F = synth.make_scene("small", noise_free=True).F
    alphas = np.r_[1.0, rng.uniform(0.7, 1.3, F - 1)]
    betas = np.r_[0.0, rng.uniform(-0.1, 0.1, F - 1)]
    sc, pb, poses = _identity_warp_problem(alphas, betas)
    d = sc.depths_gt
    dth, dab, dd, _, _, _ = oracle.fc_step_joint(pb, poses, d)
    got = pb.photo.reshape(F, 2)
    assert np.abs(got[1:, 0] - alphas[1:]).max() < 1e-9, (got, alphas)
    assert np.abs(got[1:, 1] - betas[1:]).max() < 1e-9, (got, betas)
    assert np.abs(dth).max() < 1e-9 and np.abs(dd).max() == 0.0


def test_fc_joint_step_is_the_dense_least_squares_minimiser():
    sc, imgs = _relit_tiny()
    pb = oracle.Problem(imgs, sc.uv, sc.pattern, sc.vis, sc.intrinsics, sc.huber_k, photometric=True)
    P, D = sc.poses0, sc.depths0
    F, N = pb.F, pb.N
    nf = 8 * (F - 1)
    rows, rhs = [], []
    for n in range(N):
        for f in range(1, F):
            if not pb.vis[n, f]:
                continue
            for j in range(pb.P):
                J, r, ok = oracle.fc_residual_joint(pb, P, D, n, f, j)
                if not ok:
                    continue
                w = oracle.huber_weight(r, pb.huber_k)
                row = np.zeros(nf + N)
                row[8 * (f - 1):8 * f] = J[:8]
                row[nf + n] = J[8]
                rows.append(np.sqrt(w) * row)
                rhs.append(-np.sqrt(w) * r)
    x = np.linalg.lstsq(np.array(rows), np.array(rhs), rcond=None)[0]
    dense = x[:nf].reshape(F - 1, 8)
    dth, dab, _, _, _, _ = oracle.fc_step_joint(pb, P, D)
    assert np.abs(dth[1:, 3:] - dense[:, 3:6]).max() <= 1e-6 * np.abs(dense[:, 3:6]).max()
    assert np.abs(dab[1:] - dense[:, 6:]).max() <= 1e-6 * np.abs(dense[:, 6:]).max()


@pytest.mark.parametrize("lam", [0.1, 1.0])
def test_damped_joint_step_is_the_damped_dense_solution(lam):
    """Levenberg-Marquardt damping of the 8-block system (every diagonal
    entry of H_pp and H_dd times 1 + lambda): the rotations and the pair
    increments equal those of the damped dense normal equations over all
    unknowns (numpy solve); the translations then take the scale-gauge
    projection, which leaves those components alone."""
    sc, imgs = _relit_tiny()
    pb = oracle.Problem(imgs, sc.uv, sc.pattern, sc.vis, sc.intrinsics, sc.huber_k, damping=lam,
                        photometric=True)
    P, D = sc.poses0, sc.depths0
    F, N = pb.F, pb.N
    nf = 8 * (F - 1)
    H = np.zeros((nf + N, nf + N))
    g = np.zeros(nf + N)
    for n in range(N):
        for f in range(1, F):
            if not pb.vis[n, f]:
                continue
            for j in range(pb.P):
                J, r, ok = oracle.fc_residual_joint(pb, P, D, n, f, j)
                if not ok:
                    continue
                w = oracle.huber_weight(r, pb.huber_k)
                row = np.zeros(nf + N)
                row[8 * (f - 1):8 * f] = J[:8]
                row[nf + n] = J[8]
                H += w * np.outer(row, row)
                g += w * r * row
    live = np.diag(H) > 0
    Hd = H + lam * np.diag(np.diag(H))
    x = np.zeros(nf + N)
    x[live] = np.linalg.solve(Hd[np.ix_(live, live)], -g[live])
    dense = x[:nf].reshape(F - 1, 8)
    dth, dab, _, _, _, _ = oracle.fc_step_joint(pb, P, D)
    assert np.abs(dth[1:, 3:] - dense[:, 3:6]).max() <= 1e-8 * np.abs(dense[:, 3:6]).max()
    assert np.abs(dab[1:] - dense[:, 6:]).max() <= 1e-8 * np.abs(dense[:, 6:]).max()
