"""FP64 CPU oracle for IC-PBA with proxy templates and FC-PBA.

TEST INFRASTRUCTURE ONLY: the plain, slow, obviously-correct reference of
Ham, Lucey and Singh (ICCV 2017, arXiv 1704.06967) that the GPU library is
checked against. Only the tests, the smoke check and the benchmark's
CPU-baseline leg may import this package; the library never does, and the two
share no code.

The arithmetic lives in pba_oracle.c (plain C, double precision, single
thread); this module compiles it with gcc on first use and marshals numpy
arrays. Every function cites the passage of the paper it follows in the C
source.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "pba_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

ST_ENERGY, ST_RMS, ST_COUNT, ST_MAXDISP, ST_DTHETA, ST_DD = range(6)
N_STATS = 8


def build(force: bool = False) -> str:
    """Compile the oracle (gcc -O2, no fast-math) if missing or stale."""
    with _lock:
        stale = (not os.path.exists(_LIB)) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC)
        if force or stale:
            tmp = _LIB + f".tmp{os.getpid()}"
            subprocess.check_call(["gcc", "-O2", "-fPIC", "-shared", "-std=c99",
                                   "-ffp-contract=off", _SRC, "-o", tmp, "-lm"])
            os.replace(tmp, _LIB)
    return _LIB


class _Problem(ctypes.Structure):
    _fields_ = [("W", ctypes.c_int), ("H", ctypes.c_int), ("F", ctypes.c_int),
                ("N", ctypes.c_int), ("P", ctypes.c_int),
                ("fx", ctypes.c_double), ("fy", ctypes.c_double), ("cx", ctypes.c_double),
                ("cy", ctypes.c_double), ("huber_k", ctypes.c_double),
                ("img", ctypes.c_void_p), ("uv", ctypes.c_void_p), ("pat", ctypes.c_void_p),
                ("vis", ctypes.c_void_p), ("damping", ctypes.c_double), ("photo", ctypes.c_void_p),
                ("photo_prior", ctypes.c_double)]


class _IcPre(ctypes.Structure):
    _fields_ = [("J", ctypes.c_void_p), ("r0", ctypes.c_void_p), ("w0", ctypes.c_void_p),
                ("valid0", ctypes.c_void_p), ("Hff", ctypes.c_void_p), ("Hfd", ctypes.c_void_p),
                ("Hdd", ctypes.c_void_p)]


def _L():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB)
        vp, d, i = ctypes.c_void_p, ctypes.c_double, ctypes.c_int
        pp = ctypes.POINTER(_Problem)
        sig = {
            "or_so3_exp": ([vp, vp], None),
            "or_se3_exp": ([vp, vp, vp], None),
            "or_bilinear": ([vp, i, i, d, d, vp], i),
            "or_grad_central": ([vp, i, i, i, i, vp, vp], None),
            "or_warp": ([vp, vp, d, d, d, vp, vp], i),
            "or_phi": ([vp, vp, d, d, d, vp, vp], None),
            "or_phi_update": ([vp, vp, d, d, d, vp, vp], None),
            "or_phi_jacobian": ([vp, vp, d, d, d, vp], None),
            "or_huber_rho": ([d, d], d),
            "or_huber_weight": ([d, d], d),
            "or_ic_residual": ([pp, vp, vp, i, i, i, vp, vp], i),
            "or_fc_residual": ([pp, vp, vp, i, i, i, vp, vp], i),
            "or_ic_precompute": ([pp, vp, vp, ctypes.POINTER(_IcPre)], None),
            "or_schur_solve": ([i, i, vp, vp, vp, vp, vp, vp, d, vp, vp, vp], i),
            "or_max_reproj_disp": ([pp, vp, vp, vp, vp], d),
            "or_ic_gradient": ([pp, ctypes.POINTER(_IcPre), vp, vp, vp, vp, vp], None),
            "or_ic_update": ([i, i, vp, vp, vp, vp, vp, vp, vp, vp], None),
            "or_ic_step": ([pp, ctypes.POINTER(_IcPre), vp, vp, vp, vp, vp, vp, vp, vp, vp], i),
            "or_fc_linearize": ([pp, vp, vp, vp, vp, vp, vp, vp, vp], None),
            "or_fc_update": ([i, i, vp, vp, vp, vp, vp, vp], None),
            "or_fc_step": ([pp, vp, vp, vp, vp, vp, vp, vp], i),
            "or_eval": ([pp, vp, vp, vp], None),
            "or_photo_update": ([pp, vp, vp], None),
            "or_photo_compose": ([vp, vp, vp], None),
            "or_ic_step_joint": ([pp, ctypes.POINTER(_IcPre), vp, vp, vp, vp, vp, vp, vp, vp, vp, vp], i),
            "or_fc_residual_joint": ([pp, vp, vp, i, i, i, vp, vp], i),
            "or_fc_step_joint": ([pp, vp, vp, vp, vp, vp, vp, vp, vp], i),
        }
        for name, (args, res) in sig.items():
            fn = getattr(lib, name)
            fn.argtypes = args
            fn.restype = res
        _lib = lib
    return _lib


def _p(a: np.ndarray):
    return a.ctypes.data


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


# ----------------------------------------------------------------------------
# elementary functions
# ----------------------------------------------------------------------------
def so3_exp(w) -> np.ndarray:
    w = _f64(w)
    R = np.empty(9)
    _L().or_so3_exp(_p(w), _p(R))
    return R.reshape(3, 3)


def se3_exp(xi):
    xi = _f64(xi)
    R, t = np.empty(9), np.empty(3)
    _L().or_se3_exp(_p(xi), _p(R), _p(t))
    return R.reshape(3, 3), t


def bilinear(img, u, v):
    img = _f64(img)
    out = np.empty(1)
    ok = _L().or_bilinear(_p(img), img.shape[1], img.shape[0], float(u), float(v), _p(out))
    return (float(out[0]) if ok else None)


def grad_central(img, x, y):
    img = _f64(img)
    gu, gv = np.empty(1), np.empty(1)
    _L().or_grad_central(_p(img), img.shape[1], img.shape[0], int(x), int(y), _p(gu), _p(gv))
    return float(gu[0]), float(gv[0])


def warp(R, t, d, x, y):
    R, t = _f64(R), _f64(t)
    out, q = np.empty(2), np.empty(3)
    front = _L().or_warp(_p(R), _p(t), float(d), float(x), float(y), _p(out), _p(q))
    return out, q, bool(front)


def phi(R0, t0, d0, x, y, dp):
    R0, t0, dp = _f64(R0), _f64(t0), _f64(dp)
    out = np.empty(2)
    _L().or_phi(_p(R0), _p(t0), float(d0), float(x), float(y), _p(dp), _p(out))
    return out


def phi_update(R0, t0, d0, x, y, dp):
    R0, t0, dp = _f64(R0), _f64(t0), _f64(dp)
    out = np.empty(2)
    _L().or_phi_update(_p(R0), _p(t0), float(d0), float(x), float(y), _p(dp), _p(out))
    return out


def phi_jacobian(R0, t0, d0, x, y) -> np.ndarray:
    R0, t0 = _f64(R0), _f64(t0)
    J = np.empty(14)
    _L().or_phi_jacobian(_p(R0), _p(t0), float(d0), float(x), float(y), _p(J))
    return J.reshape(2, 7)


def huber_rho(r, k):
    return _L().or_huber_rho(float(r), float(k))


def huber_weight(r, k):
    return _L().or_huber_weight(float(r), float(k))


# ----------------------------------------------------------------------------
# problems
# ----------------------------------------------------------------------------
class Problem:
    """A bundle as the oracle sees it: FP64 copies of the (dequantised) images,
    integer point pixels, pattern, visibility, intrinsics and Huber k."""

    def __init__(self, images, uv, pattern, vis, intrinsics, huber_k, damping=0.0, photometric=False,
                 photo_prior=0.0):
        self.img = _f64(images)
        self.F, self.H, self.W = self.img.shape
        self.uv = np.ascontiguousarray(uv, dtype=np.int32)
        self.pat = np.ascontiguousarray(pattern, dtype=np.int32)
        self.vis = np.ascontiguousarray(vis, dtype=np.uint8)
        self.N, self.P = self.uv.shape[0], self.pat.shape[0]
        fx, fy, cx, cy = [float(v) for v in intrinsics]
        self.fx, self.fy, self.cx, self.cy = fx, fy, cx, cy
        self.huber_k = float(huber_k)
        self.damping = float(damping)
        # affine brightness pairs (alpha_f, beta_f): the model's state, updated
        # in place by every step (None: model off)
        self.photo = np.tile([1.0, 0.0], self.F) if photometric else None
        self.c = _Problem(self.W, self.H, self.F, self.N, self.P, fx, fy, cx, cy,
                          self.huber_k, _p(self.img), _p(self.uv), _p(self.pat), _p(self.vis),
                          self.damping, _p(self.photo) if photometric else None, float(photo_prior))

    @classmethod
    def from_scene(cls, scene, damping=0.0, photometric=False, photo_prior=0.0):
        return cls(scene.images_f32, scene.uv, scene.pattern, scene.vis, scene.intrinsics,
                   scene.huber_k, damping, photometric, photo_prior)

    def ref(self):
        return ctypes.byref(self.c)


class IcPre:
    """Output of the IC precompute (Sec. 3.5): J rows, r0, W_0, H blocks."""

    def __init__(self, pb: Problem):
        R = pb.N * pb.F * pb.P
        self.J = np.zeros((R, 7))
        self.r0 = np.zeros(R)
        self.w0 = np.zeros(R)
        self.valid0 = np.zeros(R, np.uint8)
        self.Hff = np.zeros((pb.F, 6, 6))
        self.Hfd = np.zeros((pb.N, pb.F, 6))
        self.Hdd = np.zeros(pb.N)
        self.c = _IcPre(_p(self.J), _p(self.r0), _p(self.w0), _p(self.valid0), _p(self.Hff),
                        _p(self.Hfd), _p(self.Hdd))

    def ref(self):
        return ctypes.byref(self.c)

    def rid(self, pb, n, f, j):
        return (n * pb.F + f) * pb.P + j


def ic_residual(pb: Problem, poses0, depths0, n, f, j):
    poses0, depths0 = _f64(poses0), _f64(depths0)
    J, r = np.empty(7), np.empty(1)
    ok = _L().or_ic_residual(pb.ref(), _p(poses0), _p(depths0), n, f, j, _p(J), _p(r))
    return J, float(r[0]), bool(ok)


def fc_residual(pb: Problem, poses, depths, n, f, j):
    poses, depths = _f64(poses), _f64(depths)
    J, r = np.empty(7), np.empty(1)
    ok = _L().or_fc_residual(pb.ref(), _p(poses), _p(depths), n, f, j, _p(J), _p(r))
    return J, float(r[0]), bool(ok)


def ic_precompute(pb: Problem, poses0, depths0) -> IcPre:
    poses0, depths0 = _f64(poses0), _f64(depths0)
    pre = IcPre(pb)
    _L().or_ic_precompute(pb.ref(), _p(poses0), _p(depths0), pre.ref())
    return pre


def schur_solve(F, N, Hff, Hfd, Hdd, g_theta, g_d, t_anchor, want_S=False, damping=0.0):
    Hff, Hfd, Hdd = _f64(Hff), _f64(Hfd), _f64(Hdd)
    g_theta, g_d, t_anchor = _f64(g_theta), _f64(g_d), _f64(t_anchor)
    dtheta, dd = np.zeros(6 * F), np.zeros(N)
    n6 = 6 * (F - 1)
    S = np.zeros((n6, n6)) if want_S else None
    st = _L().or_schur_solve(F, N, _p(Hff), _p(Hfd), _p(Hdd), _p(g_theta), _p(g_d),
                             _p(t_anchor), float(damping), _p(dtheta), _p(dd), _p(S) if want_S else None)
    if st != 0:
        raise np.linalg.LinAlgError(f"reduced camera system not positive definite ({st})")
    return dtheta.reshape(F, 6), dd, S


def ic_gradient(pb: Problem, pre: IcPre, poses, depths):
    poses, depths = _f64(poses), _f64(depths)
    g_theta, g_d, stats = np.zeros(6 * pb.F), np.zeros(pb.N), np.zeros(N_STATS)
    _L().or_ic_gradient(pb.ref(), pre.ref(), _p(poses), _p(depths), _p(g_theta), _p(g_d),
                        _p(stats))
    return g_theta.reshape(pb.F, 6), g_d, stats


def ic_update(poses0, depths0, poses, depths, dtheta, dd):
    poses0, depths0, poses, depths = _f64(poses0), _f64(depths0), _f64(poses), _f64(depths)
    dtheta, dd = _f64(dtheta), _f64(dd)
    F, N = poses.shape[0], depths.shape[0]
    po, do = np.empty_like(poses), np.empty_like(depths)
    _L().or_ic_update(F, N, _p(poses0), _p(depths0), _p(poses), _p(depths), _p(dtheta), _p(dd),
                      _p(po), _p(do))
    return po, do


def fc_update(poses, depths, dtheta, dd):
    poses, depths, dtheta, dd = _f64(poses), _f64(depths), _f64(dtheta), _f64(dd)
    F, N = poses.shape[0], depths.shape[0]
    po, do = np.empty_like(poses), np.empty_like(depths)
    _L().or_fc_update(F, N, _p(poses), _p(depths), _p(dtheta), _p(dd), _p(po), _p(do))
    return po, do


def ic_step(pb: Problem, pre: IcPre, poses0, depths0, poses, depths):
    """One IC iteration; returns (dtheta [F,6], dd [N], poses', depths', stats)."""
    poses0, depths0, poses, depths = _f64(poses0), _f64(depths0), _f64(poses), _f64(depths)
    dtheta, dd = np.zeros(6 * pb.F), np.zeros(pb.N)
    po, do, stats = np.empty_like(poses), np.empty_like(depths), np.zeros(N_STATS)
    st = _L().or_ic_step(pb.ref(), pre.ref(), _p(poses0), _p(depths0), _p(poses), _p(depths),
                         _p(dtheta), _p(dd), _p(po), _p(do), _p(stats))
    if st != 0:
        raise np.linalg.LinAlgError("reduced camera system not positive definite")
    return dtheta.reshape(pb.F, 6), dd, po, do, stats


def photo_compose(ab, dab):
    """The brightness pair after a template-side increment (da, db)."""
    ab, dab, out = _f64(ab), _f64(dab), np.zeros(2)
    _L().or_photo_compose(_p(ab), _p(dab), _p(out))
    return out


def ic_step_joint(pb: Problem, pre: IcPre, poses0, depths0, poses, depths):
    """One IC iteration with the brightness pairs (pb.photo, updated in
    place) as Gauss-Newton unknowns; returns (dtheta [F,6], dab [F,2], dd
    [N], poses', depths', stats)."""
    if pb.photo is None:
        raise ValueError("the joint brightness step needs a problem with photometric=True")
    poses0, depths0, poses, depths = _f64(poses0), _f64(depths0), _f64(poses), _f64(depths)
    dtheta, dab, dd = np.zeros(6 * pb.F), np.zeros(2 * pb.F), np.zeros(pb.N)
    po, do, stats = np.empty_like(poses), np.empty_like(depths), np.zeros(N_STATS)
    st = _L().or_ic_step_joint(pb.ref(), pre.ref(), _p(poses0), _p(depths0), _p(poses), _p(depths),
                               _p(dtheta), _p(dab), _p(dd), _p(po), _p(do), _p(stats))
    if st != 0:
        raise np.linalg.LinAlgError("reduced camera system not positive definite")
    return dtheta.reshape(pb.F, 6), dab.reshape(pb.F, 2), dd, po, do, stats


def ic_run_joint(pb: Problem, poses0, depths0, iters: int):
    """IC-PBA with the brightness pairs as unknowns (same return layout as
    ic_run; pb.photo holds the final pairs)."""
    pre = ic_precompute(pb, poses0, depths0)
    poses, depths = _f64(poses0).copy(), _f64(depths0).copy()
    hist = np.zeros((iters + 1, N_STATS))
    for k in range(iters):
        _, _, _, poses, depths, hist[k] = ic_step_joint(pb, pre, poses0, depths0, poses, depths)
    hist[iters] = evaluate(pb, poses, depths)
    return poses, depths, hist


def fc_residual_joint(pb: Problem, poses, depths, n, f, j):
    """FC residual with the brightness columns: (J [9]: pose 6, -v, -1,
    depth; r; valid)."""
    poses, depths = _f64(poses), _f64(depths)
    J, r = np.empty(9), np.empty(1)
    ok = _L().or_fc_residual_joint(pb.ref(), _p(poses), _p(depths), n, f, j, _p(J), _p(r))
    return J, float(r[0]), bool(ok)


def fc_step_joint(pb: Problem, poses, depths):
    """One FC iteration with the brightness pairs (pb.photo, updated in
    place) as unknowns; returns (dtheta [F,6], dab [F,2], dd [N], poses',
    depths', stats)."""
    if pb.photo is None:
        raise ValueError("the joint brightness step needs a problem with photometric=True")
    poses, depths = _f64(poses), _f64(depths)
    dtheta, dab, dd = np.zeros(6 * pb.F), np.zeros(2 * pb.F), np.zeros(pb.N)
    po, do, stats = np.empty_like(poses), np.empty_like(depths), np.zeros(N_STATS)
    st = _L().or_fc_step_joint(pb.ref(), _p(poses), _p(depths), _p(dtheta), _p(dab), _p(dd), _p(po), _p(do),
                               _p(stats))
    if st != 0:
        raise np.linalg.LinAlgError("reduced camera system not positive definite")
    return dtheta.reshape(pb.F, 6), dab.reshape(pb.F, 2), dd, po, do, stats


def fc_linearize(pb: Problem, poses, depths):
    poses, depths = _f64(poses), _f64(depths)
    Hff, Hfd, Hdd = np.zeros((pb.F, 6, 6)), np.zeros((pb.N, pb.F, 6)), np.zeros(pb.N)
    g_theta, g_d, stats = np.zeros(6 * pb.F), np.zeros(pb.N), np.zeros(N_STATS)
    _L().or_fc_linearize(pb.ref(), _p(poses), _p(depths), _p(Hff), _p(Hfd), _p(Hdd),
                         _p(g_theta), _p(g_d), _p(stats))
    return Hff, Hfd, Hdd, g_theta.reshape(pb.F, 6), g_d, stats


def fc_step(pb: Problem, poses, depths):
    """One FC iteration; returns (dtheta [F,6], dd [N], poses', depths', stats)."""
    poses, depths = _f64(poses), _f64(depths)
    dtheta, dd = np.zeros(6 * pb.F), np.zeros(pb.N)
    po, do, stats = np.empty_like(poses), np.empty_like(depths), np.zeros(N_STATS)
    st = _L().or_fc_step(pb.ref(), _p(poses), _p(depths), _p(dtheta), _p(dd), _p(po), _p(do),
                         _p(stats))
    if st != 0:
        raise np.linalg.LinAlgError("reduced camera system not positive definite")
    return dtheta.reshape(pb.F, 6), dd, po, do, stats


def photo_update(pb: Problem, poses, depths):
    """Fits every target frame's brightness pair to the residuals at
    (poses, depths) in place (pb.photo); no-op with the model off."""
    poses, depths = _f64(poses), _f64(depths)
    _L().or_photo_update(pb.ref(), _p(poses), _p(depths))
    return pb.photo


def evaluate(pb: Problem, poses, depths):
    poses, depths = _f64(poses), _f64(depths)
    stats = np.zeros(N_STATS)
    _L().or_eval(pb.ref(), _p(poses), _p(depths), _p(stats))
    return stats


def max_reproj_disp(pb: Problem, poses_a, depths_a, poses_b, depths_b):
    a, b, c, d = _f64(poses_a), _f64(depths_a), _f64(poses_b), _f64(depths_b)
    return _L().or_max_reproj_disp(pb.ref(), _p(a), _p(b), _p(c), _p(d))


def ic_run(pb: Problem, poses0, depths0, iters: int):
    """IC-PBA from p0 for `iters` iterations. Returns (poses, depths, stats
    [iters+1, N_STATS]); row k holds the statistics at p_k (the last row only
    energy/RMS/count)."""
    pre = ic_precompute(pb, poses0, depths0)
    poses, depths = _f64(poses0).copy(), _f64(depths0).copy()
    hist = np.zeros((iters + 1, N_STATS))
    for k in range(iters):
        _, _, poses, depths, hist[k] = ic_step(pb, pre, poses0, depths0, poses, depths)
    hist[iters] = evaluate(pb, poses, depths)
    return poses, depths, hist


def fc_run(pb: Problem, poses0, depths0, iters: int):
    """FC-PBA from p0 for `iters` iterations (same return layout as ic_run)."""
    poses, depths = _f64(poses0).copy(), _f64(depths0).copy()
    hist = np.zeros((iters + 1, N_STATS))
    for k in range(iters):
        _, _, poses, depths, hist[k] = fc_step(pb, poses, depths)
    hist[iters] = evaluate(pb, poses, depths)
    return poses, depths, hist
