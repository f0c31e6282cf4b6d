"""Seeded synthetic bundles for photometric bundle adjustment.

Input generation only: this module renders images, picks template points,
marks visibility and perturbs the ground truth. It holds none of the bundle
adjustment arithmetic (no proxy warp, Jacobian, Hessian or update), so the
CPU oracle and the GPU path can both read its output without sharing any of
the method's code.

The paper's sequences (Stanford Bunny, Toy Robot, the Blender-rendered
synthetic set and the DSO dinosaur, Sec. 4) are not available; these scenes
stand in for them. They follow the paper's conventions where it states one:
one reference frame holding every point's inverse depth (Sec. 3, Eq. warp),
the mean point depth normalised to one (Sec. 4.1, "Magnitude of Noise"), and
parameter perturbations applied to a known solution (Sec. 4.1).

Recipe (all seeded):
  * object: sphere of radius `sphere_r` at the world origin, optionally a
    square ground plane z = -1; albedo = 4-octave value noise (render.c);
    background 0.5; images supersampled `ss` x `ss`.
  * cameras look at the origin (x right, y down, z forward); frame 0 is the
    reference and becomes the identity pose.
  * points: top pattern-summed squared central-difference gradient in frame 0,
    on-object pattern footprint, greedy minimum spacing, ties by raster index.
  * visibility (n,f): in front, unoccluded, surface normal within `max_view_deg`
    of the view ray, and the projection inside the image with a margin at both
    the true and the perturbed parameters. Target frames that see fewer than
    `min_pts_per_frame` points are marked inactive (their column cleared).
  * perturbation: each target pose is left-multiplied by a rotation of exactly
    `rot_deg` about a random axis and shifted by exactly `trans` in a random
    direction; inverse depths are scaled by (1 + sigma_d * eps), eps ~ N(0,1)
    truncated at 3.
  * image noise: additive N(0, sigma^2), unclamped, then quantised to the
    storage dtype (f32, f16 or bf16 with round-to-nearest-even).
"""
from __future__ import annotations

import ctypes
import dataclasses
import math
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "render.c")
_LIB = os.path.join(_HERE, "librender.so")
_SRC_GPU = os.path.join(_HERE, "render_gpu.cu")
_LIB_GPU = os.path.join(_HERE, "librender_gpu.so")
_lock = threading.Lock()
_lib = None
_lib_gpu = None

# 8-pixel pattern around each point; the point's own pixel is not part of it.
PATTERN8 = np.array([(-1, -1), (1, -1), (-1, 1), (1, 1), (-2, 0), (2, 0), (0, -2), (0, 2)],
                    dtype=np.int32)

SCENE_SEED, NOISE_SEED, PERTURB_SEED = 17040, 17041, 17042


def build_renderer(force: bool = False) -> str:
    """Compile render.c into librender.so (gcc, OpenMP) if missing or stale."""
    with _lock:
        stale = (not os.path.exists(_LIB)) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC)
        if force or stale:
            tmp = _LIB + f".tmp{os.getpid()}"
            # no multiply-add contraction: the same images on x86 and Arm,
            # and bit for bit those of the CUDA renderer
            subprocess.check_call(["gcc", "-O2", "-fPIC", "-shared", "-fopenmp", "-std=c99",
                                   "-ffp-contract=off", _SRC, "-o", tmp, "-lm"])
            os.replace(tmp, _LIB)
    return _LIB


def build_renderer_gpu(force: bool = False) -> str:
    """Compile render_gpu.cu into librender_gpu.so (nvcc, sm_103a, no
    multiply-add contraction) if missing or stale."""
    import shutil
    with _lock:
        stale = (not os.path.exists(_LIB_GPU)) or os.path.getmtime(_LIB_GPU) < os.path.getmtime(_SRC_GPU)
        if force or stale:
            nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
            tmp = _LIB_GPU + f".tmp{os.getpid()}"
            subprocess.check_call([nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-fmad=false",
                                   "-lineinfo", "-shared", "-Xcompiler", "-fPIC", _SRC_GPU, "-o", tmp])
            os.replace(tmp, _LIB_GPU)
    return _LIB_GPU


def _renderer_gpu():
    global _lib_gpu
    if _lib_gpu is None:
        build_renderer_gpu()
        lib = ctypes.CDLL(_LIB_GPU)
        d, i, vp = ctypes.c_double, ctypes.c_int, ctypes.c_void_p
        lib.synth_render_gpu.argtypes = [i, i, i, i, d, d, d, d, vp, d, i, vp, d, i, ctypes.c_uint64, d, vp, vp,
                                         vp]
        lib.synth_render_gpu.restype = i
        _lib_gpu = lib
    return _lib_gpu


def _renderer():
    global _lib
    if _lib is None:
        build_renderer()
        lib = ctypes.CDLL(_LIB)
        dp = ctypes.POINTER(ctypes.c_double)
        lib.synth_render.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                     ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                     ctypes.c_double, dp, dp, ctypes.c_double, ctypes.c_int,
                                     dp, ctypes.c_double, ctypes.c_int, ctypes.c_uint64,
                                     ctypes.c_double, ctypes.c_void_p, ctypes.c_void_p]
        lib.synth_cast_pixels.argtypes = [ctypes.c_int, dp, ctypes.c_double, ctypes.c_double,
                                          ctypes.c_double, ctypes.c_double, dp, dp,
                                          ctypes.c_double, ctypes.c_int, dp,
                                          ctypes.c_void_p, ctypes.c_void_p]
        lib.synth_unoccluded.argtypes = [ctypes.c_int, dp, dp, ctypes.c_double, ctypes.c_int,
                                         dp, ctypes.c_void_p]
        _lib = lib
    return _lib


def _dp(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


# ----------------------------------------------------------------------------
# small rigid-body helpers (scene construction only)
# ----------------------------------------------------------------------------
def _look_at(C: np.ndarray, target=(0.0, 0.0, 0.0), up=(0.0, 0.0, 1.0)):
    """World->camera rotation for a camera at C looking at target (y down)."""
    fwd = np.asarray(target, float) - C
    fwd /= np.linalg.norm(fwd)
    right = np.cross(fwd, np.asarray(up, float))
    right /= np.linalg.norm(right)
    down = np.cross(fwd, right)
    return np.stack([right, down, fwd])


def _rotvec_to_matrix(v: np.ndarray) -> np.ndarray:
    from scipy.spatial.transform import Rotation
    return Rotation.from_rotvec(v).as_matrix()


def bf16_round(x: np.ndarray) -> np.ndarray:
    """float32 -> bf16 bit patterns (uint16), round to nearest even."""
    u = np.ascontiguousarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    rounding = ((u >> 16) & 1) + 0x7FFF
    return ((u + rounding) >> 16).astype(np.uint16)


def bf16_to_f32(b: np.ndarray) -> np.ndarray:
    return (b.astype(np.uint32) << 16).view(np.float32)


# ----------------------------------------------------------------------------
# configurations
# ----------------------------------------------------------------------------
@dataclasses.dataclass
class SceneConfig:
    name: str
    W: int
    H: int
    f: float
    n_points: int
    path: str                       # "ring" | "helix" | "orbit"
    azimuths_deg: tuple = ()        # ring: target azimuths (reference at 0)
    n_frames: int = 5               # including the reference frame
    turns: float = 2.0              # helix
    height: float = 0.5             # helix: z from -height to +height
    elevation_deg: float = 30.0     # orbit
    radius: float = 3.0             # camera distance from the axis
    sphere_r: float = 1.0           # <= 0: no sphere
    plane: bool = False             # square ground plane z = -1, half size 4
    cards: int = 0                  # fronto-parallel (to frame 0) textured cards
    dtype: str = "f32"              # image storage: f32 | f16 | bf16
    rot_deg: float = 2.0
    trans: float = 0.02
    sigma_d: float = 0.05
    noise: float = 2.0 / 255.0
    huber_k: float = 9.0 / 255.0
    ss: int = 2
    tex_min_px: float = 8.0         # finest-octave cell size (px) at the nearest depth
    octaves: int = 4
    spacing: int = 2                # minimum Chebyshev distance between points
    max_view_deg: float = 72.0
    margin_px: float = 6.0
    min_pts_per_frame: int = 16
    edge_px: int = 1                # candidate points keep this distance from object edges
    allow_fewer_points: bool = False  # take all candidates when fewer than n_points exist


CONFIGS = {
    # 5 frames on a ring of radius 3 (reference at azimuth 0), 320x240, f=300,
    # 2,000 points; 2 deg / 0.02 pose noise, 5 % inverse-depth noise.
    "ring5": SceneConfig("ring5", 320, 240, 300.0, 2000, "ring",
                         azimuths_deg=(-20.0, -10.0, 10.0, 20.0), n_frames=5),
    # 30 frames on a 2-turn helix (radius 3, height +-0.5), 640x480, f=525,
    # 20,000 points: reduced camera system of 6*29 = 174.
    "helix30": SceneConfig("helix30", 640, 480, 525.0, 20000, "helix", n_frames=30, spacing=1),
    # 1 reference + 100 targets on a 30 deg orbit, 1280x720 bf16, f=900,
    # sphere + ground plane, 200,000 points: reduced camera system of 600.
    "orbit101": SceneConfig("orbit101", 1280, 720, 900.0, 200000, "orbit", n_frames=101,
                            plane=True, dtype="bf16", spacing=1),
    # small cases that the CPU oracle finishes in well under a second
    "tiny": SceneConfig("tiny", 128, 96, 120.0, 64, "ring",
                        azimuths_deg=(-15.0, 10.0, 20.0), n_frames=4, ss=2, tex_min_px=8.0),
    "small": SceneConfig("small", 160, 120, 150.0, 300, "ring",
                         azimuths_deg=(-15.0, -7.5, 7.5, 15.0, 22.5), n_frames=6),
    # six textured cards facing the reference camera at depths 2.4..3.3: every
    # pattern lies on a surface of constant reference depth, so the one-depth-
    # per-point model of the paper holds exactly and noise-free data admits
    # the true parameters as a zero-residual solution (up to interpolation).
    "cards": SceneConfig("cards", 200, 150, 130.0, 400, "ring",
                         azimuths_deg=(-12.0, -6.0, 6.0, 12.0), n_frames=5, sphere_r=0.0,
                         cards=6, tex_min_px=12.0, ss=4, edge_px=6, max_view_deg=80.0),
}


@dataclasses.dataclass
class Scene:
    cfg: SceneConfig
    W: int
    H: int
    fx: float
    fy: float
    cx: float
    cy: float
    images_f32: np.ndarray        # [F,H,W] float32 values the solver reads (dequantised)
    images_store: np.ndarray      # [F,H,W] storage array (float32 / float16 / uint16 bf16)
    dtype: str
    pattern: np.ndarray           # [P,2] int32 pixel offsets
    uv: np.ndarray                # [N,2] int32 pixel centres in frame 0
    vis: np.ndarray               # [N,F] uint8 (column 0 is 0)
    poses_gt: np.ndarray          # [F,12] float64 (row-major R | t), frame 0 = identity
    depths_gt: np.ndarray         # [N] float64 inverse depths (mean depth 1)
    poses0: np.ndarray            # perturbed initial poses
    depths0: np.ndarray           # perturbed initial inverse depths
    huber_k: float

    @property
    def F(self):
        return self.images_store.shape[0]

    @property
    def N(self):
        return self.uv.shape[0]

    @property
    def P(self):
        return self.pattern.shape[0]

    @property
    def intrinsics(self):
        return np.array([self.fx, self.fy, self.cx, self.cy], dtype=np.float64)

    def n_residuals(self) -> int:
        return int(self.vis.sum()) * self.P


def _rects(cfg: SceneConfig, R0w: np.ndarray, C0: np.ndarray):
    """Rectangles of the scene (11 doubles each) and the nearest surface depth."""
    rows = []
    near = cfg.radius - cfg.sphere_r if cfg.sphere_r > 0 else np.inf
    if cfg.plane:
        rows.append([0, 0, -1.0, 1, 0, 0, 0, 1, 0, 4.0, 4.0])
    if cfg.cards:
        # a 3 x 2 grid in the reference view, each card facing the reference
        right, down, fwd = R0w[0], R0w[1], R0w[2]
        depths = [2.4, 3.0, 2.7, 3.3, 2.6, 3.1]
        cols, rws = [-0.36, 0.0, 0.36], [-0.21, 0.21]
        for i in range(cfg.cards):
            xn, yn, z = cols[i % 3], rws[(i // 3) % 2], depths[i % len(depths)]
            c = C0 + z * (fwd + xn * right + yn * down)
            rows.append(list(c) + list(right) + list(down) + [0.14 * z, 0.17 * z])
            near = min(near, z)
    return np.ascontiguousarray(np.array(rows, dtype=np.float64).reshape(-1, 11)), near


def _camera_centres(cfg: SceneConfig) -> np.ndarray:
    if cfg.path == "ring":
        az = [0.0] + list(cfg.azimuths_deg)
        return np.array([[cfg.radius * math.cos(math.radians(a)),
                          cfg.radius * math.sin(math.radians(a)), 0.0] for a in az])
    if cfg.path == "helix":
        n = cfg.n_frames
        out = []
        for i in range(n):
            a = 2.0 * math.pi * cfg.turns * i / n
            z = -cfg.height + 2.0 * cfg.height * i / (n - 1)
            out.append([cfg.radius * math.cos(a), cfg.radius * math.sin(a), z])
        return np.array(out)
    if cfg.path == "orbit":
        n = cfg.n_frames
        el = math.radians(cfg.elevation_deg)
        out = []
        for i in range(n):
            a = 2.0 * math.pi * i / n
            out.append([cfg.radius * math.cos(el) * math.cos(a),
                        cfg.radius * math.cos(el) * math.sin(a), cfg.radius * math.sin(el)])
        return np.array(out)
    raise ValueError(cfg.path)


def _select_points(I0: np.ndarray, hit: np.ndarray, pattern: np.ndarray, n: int,
                   spacing: int, border: int, edge_px: int, allow_fewer: bool = False) -> np.ndarray:
    from scipy.ndimage import maximum_filter, minimum_filter
    H, W = I0.shape
    gx = np.zeros_like(I0, dtype=np.float64)
    gy = np.zeros_like(I0, dtype=np.float64)
    gx[:, 1:-1] = 0.5 * (I0[:, 2:].astype(np.float64) - I0[:, :-2])
    gy[1:-1, :] = 0.5 * (I0[2:, :].astype(np.float64) - I0[:-2, :])
    g2 = gx * gx + gy * gy
    score = np.zeros((H, W))
    ok = np.zeros((H, W), bool)
    ok[border:H - border, border:W - border] = True
    # the pattern footprint (+1 for gradients, + edge_px) sees one object only
    rad = int(np.abs(pattern).max()) + 1 + edge_px
    h = hit.astype(np.int32)
    size = 2 * rad + 1
    ok &= (maximum_filter(h, size=size) == minimum_filter(h, size=size))
    ok &= (h != 0) & (h != 255)
    for (ox, oy) in pattern:
        score += np.roll(np.roll(g2, -oy, axis=0), -ox, axis=1)
    cand = np.flatnonzero(ok.ravel())
    order = cand[np.argsort(-score.ravel()[cand], kind="stable")]
    taken = np.zeros((H, W), bool)
    pts = []
    r = spacing - 1
    for idx in order:
        v, u = divmod(int(idx), W)
        if r > 0 and taken[max(0, v - r):v + r + 1, max(0, u - r):u + r + 1].any():
            continue
        taken[v, u] = True
        pts.append((u, v))
        if len(pts) == n:
            break
    if len(pts) < n and not allow_fewer:
        raise ValueError(f"only {len(pts)} candidate points for {n} requested")
    return np.array(pts, dtype=np.int32)


def _render_frames_gpu(cfg, W, H, fx, fy, cx, cy, Rw, centres, rects, sphere_r, base_freq, tex_seed):
    """Every frame by the CUDA renderer (the same images as synth_render):
    a float32 torch tensor [F, H, W] on the current CUDA device and frame
    0's object ids (host)."""
    import torch
    F = centres.shape[0]
    RC = torch.tensor(np.concatenate([Rw.reshape(F, 9), centres], axis=1), dtype=torch.float64, device="cuda")
    out = torch.empty((F, H, W), dtype=torch.float32, device="cuda")
    hit = torch.empty((H, W), dtype=torch.uint8, device="cuda")
    st = torch.cuda.current_stream()
    rc = _renderer_gpu().synth_render_gpu(F, W, H, cfg.ss, fx, fy, cx, cy, RC.data_ptr(), sphere_r,
                                          rects.shape[0], rects.ctypes.data, base_freq, cfg.octaves, tex_seed,
                                          0.5, out.data_ptr(), hit.data_ptr(), ctypes.c_void_p(st.cuda_stream))
    if rc != 0:
        raise RuntimeError(f"synth_render_gpu failed ({rc})")
    return out, hit.cpu().numpy()


def make_scene(name_or_cfg, seed_offset: int = 0, noise_free: bool = False, device: str | None = None,
               **overrides) -> Scene:
    """Generate a bundle. `overrides` replace SceneConfig fields.

    device="cuda": the frames are rendered by the CUDA ray caster (the same
    noise-free images as the host renderer, bit for bit), the image noise is
    drawn on the device (torch's Philox generator seeded like the host's
    NOISE_SEED + seed_offset: other values than the host path's) and the
    scene's images_f32 / images_store are torch tensors on the device."""
    cfg = CONFIGS[name_or_cfg] if isinstance(name_or_cfg, str) else name_or_cfg
    if overrides:
        cfg = dataclasses.replace(cfg, **overrides)
    lib = _renderer()
    W, H, fx = cfg.W, cfg.H, cfg.f
    fy = fx
    cx, cy = (W - 1) / 2.0, (H - 1) / 2.0
    centres = _camera_centres(cfg)
    F = centres.shape[0]
    Rw = np.stack([_look_at(C) for C in centres])          # world->camera rotations
    rects, near = _rects(cfg, Rw[0], centres[0])
    base_freq = 1.0 / (cfg.tex_min_px * near / fx) / (2 ** (cfg.octaves - 1))
    n_rects = rects.shape[0]
    rects_p = _dp(rects)
    sphere_r = cfg.sphere_r
    tex_seed = SCENE_SEED + seed_offset

    if device is not None:
        return _finish_scene_gpu(cfg, seed_offset, noise_free, W, H, fx, fy, cx, cy, centres, Rw, rects,
                                 near, base_freq, sphere_r, tex_seed, lib)
    images = np.empty((F, H, W), np.float32)
    hit0 = np.empty((H, W), np.uint8)
    for f in range(F):
        R = np.ascontiguousarray(Rw[f], dtype=np.float64)
        C = np.ascontiguousarray(centres[f], dtype=np.float64)
        out = np.empty((H, W), np.float32)
        lib.synth_render(W, H, cfg.ss, fx, fy, cx, cy, _dp(R), _dp(C), sphere_r, n_rects,
                         rects_p, base_freq, cfg.octaves, tex_seed, 0.5, out.ctypes.data,
                         hit0.ctypes.data if f == 0 else None)
        images[f] = out

    if not noise_free and cfg.noise > 0:
        rng = np.random.default_rng(NOISE_SEED + seed_offset)
        images = (images + rng.normal(0.0, cfg.noise, images.shape)).astype(np.float32)
    if cfg.dtype == "f32":
        store = images
        deq = images
    elif cfg.dtype == "f16":
        store = images.astype(np.float16)
        deq = store.astype(np.float32)
    elif cfg.dtype == "bf16":
        store = bf16_round(images).reshape(images.shape)
        deq = bf16_to_f32(store).reshape(images.shape)
    else:
        raise ValueError(cfg.dtype)

    return _geometry(cfg, seed_offset, W, H, fx, fy, cx, cy, centres, Rw, rects, sphere_r, lib,
                     deq[0], hit0, np.ascontiguousarray(deq, dtype=np.float32), np.ascontiguousarray(store))


def _finish_scene_gpu(cfg, seed_offset, noise_free, W, H, fx, fy, cx, cy, centres, Rw, rects, near, base_freq,
                      sphere_r, tex_seed, lib):
    import torch
    images, hit0 = _render_frames_gpu(cfg, W, H, fx, fy, cx, cy, Rw, centres, rects, sphere_r, base_freq,
                                      tex_seed)
    if not noise_free and cfg.noise > 0:
        g = torch.Generator(device=images.device)
        g.manual_seed(NOISE_SEED + seed_offset)
        images = images + cfg.noise * torch.randn(images.shape, generator=g, device=images.device,
                                                  dtype=torch.float32)
    if cfg.dtype == "f32":
        store = images
    elif cfg.dtype == "f16":
        store = images.half()
    elif cfg.dtype == "bf16":
        store = images.bfloat16()  # round to nearest even, as bf16_round
    else:
        raise ValueError(cfg.dtype)
    deq = store.float()
    return _geometry(cfg, seed_offset, W, H, fx, fy, cx, cy, centres, Rw, rects, sphere_r, lib,
                     deq[0].cpu().numpy(), hit0, deq.contiguous(), store.contiguous())


def _geometry(cfg, seed_offset, W, H, fx, fy, cx, cy, centres, Rw, rects, sphere_r, lib, deq0, hit0,
              images_f32, images_store) -> Scene:
    """Points, ground truth, perturbation and visibility of a rendered
    bundle (frame 0's dequantised image deq0 and object ids hit0)."""
    F = centres.shape[0]
    n_rects = rects.shape[0]
    rects_p = _dp(rects)
    pattern = PATTERN8.copy()
    prad = int(np.abs(pattern).max())
    border = prad + 2 + int(math.ceil(cfg.margin_px))
    uv = _select_points(deq0, hit0, pattern, cfg.n_points, cfg.spacing, border, cfg.edge_px,
                        cfg.allow_fewer_points)
    N = uv.shape[0]

    # ground-truth 3-D points (world) from the reference camera's rays
    obj = np.empty(N, np.int32)
    Xw = np.empty((N, 3), np.float64)
    uvd = np.ascontiguousarray(uv, dtype=np.float64)
    R0w = np.ascontiguousarray(Rw[0], dtype=np.float64)
    C0 = np.ascontiguousarray(centres[0], dtype=np.float64)
    lib.synth_cast_pixels(N, _dp(uvd), fx, fy, cx, cy, _dp(R0w), _dp(C0), sphere_r, n_rects,
                          rects_p, obj.ctypes.data, Xw.ctypes.data)
    assert (obj > 0).all()
    normals = np.empty((N, 3))
    for i in range(N):
        if obj[i] == 1:
            normals[i] = Xw[i] / np.linalg.norm(Xw[i])
        else:
            r = rects[obj[i] - 2]
            normals[i] = np.cross(r[3:6], r[6:9])

    # poses relative to the reference: X_f = R X_0 + t with X_0 = R0w X_w + t0w
    tw = -np.einsum("fij,fj->fi", Rw, centres)
    Rrel = np.einsum("fij,kj->fik", Rw, Rw[0])
    trel = tw - np.einsum("fij,j->fi", Rrel, tw[0])
    X0 = Xw @ Rw[0].T + tw[0]                              # points in reference coords
    z0 = X0[:, 2]
    scale = float(z0.mean())                               # mean depth -> 1
    trel = trel / scale
    d_gt = scale / z0

    # perturbation of the known solution (reference frame stays fixed)
    rng = np.random.default_rng(PERTURB_SEED + seed_offset)
    R0p = Rrel.copy()
    t0p = trel.copy()
    for f in range(1, F):
        axis = rng.normal(size=3)
        axis /= np.linalg.norm(axis)
        dR = _rotvec_to_matrix(axis * math.radians(cfg.rot_deg))
        dirn = rng.normal(size=3)
        dirn /= np.linalg.norm(dirn)
        R0p[f] = dR @ Rrel[f]
        t0p[f] = trel[f] + cfg.trans * dirn
    eps = np.clip(rng.normal(size=N), -3.0, 3.0)
    d0 = d_gt * (1.0 + cfg.sigma_d * eps)

    # visibility per (point, frame)
    vis = np.zeros((N, F), np.uint8)
    cos_min = math.cos(math.radians(cfg.max_view_deg))
    lo = prad + 2 + cfg.margin_px
    xn = np.stack([(uv[:, 0] - cx) / fx, (uv[:, 1] - cy) / fy, np.ones(N)], axis=1)
    for f in range(1, F):
        C = np.ascontiguousarray(centres[f], dtype=np.float64)
        occ = np.empty(N, np.uint8)
        lib.synth_unoccluded(N, _dp(np.ascontiguousarray(Xw)), _dp(C), sphere_r, n_rects,
                             rects_p, occ.ctypes.data)
        tocam = C - Xw
        dist = np.linalg.norm(tocam, axis=1)
        cosv = (normals * tocam).sum(1) / dist
        facing = np.where(obj == 1, cosv, np.abs(cosv)) >= cos_min
        ok = (occ > 0) & facing
        # projection of the true and the perturbed 3-D point into frame f
        for (R, t, d) in ((Rrel[f], trel[f], d_gt), (R0p[f], t0p[f], d0)):
            Pc = (xn / d[:, None]) @ R.T + t
            front = Pc[:, 2] > 1e-3
            u = fx * Pc[:, 0] / np.where(front, Pc[:, 2], 1.0) + cx
            v = fy * Pc[:, 1] / np.where(front, Pc[:, 2], 1.0) + cy
            ok &= front & (u >= lo) & (u <= W - 1 - lo) & (v >= lo) & (v <= H - 1 - lo)
        vis[:, f] = ok
        if vis[:, f].sum() < cfg.min_pts_per_frame:
            vis[:, f] = 0

    def pack(R, t):
        out = np.zeros((F, 12))
        out[:, :9] = R.reshape(F, 9)
        out[:, 9:] = t
        return out

    return Scene(cfg=cfg, W=W, H=H, fx=fx, fy=fy, cx=cx, cy=cy,
                 images_f32=images_f32,
                 images_store=images_store, dtype=cfg.dtype,
                 pattern=pattern, uv=uv, vis=vis,
                 poses_gt=pack(Rrel, trel), depths_gt=d_gt,
                 poses0=pack(R0p, t0p), depths0=d0, huber_k=cfg.huber_k)


def point_subset(scene: Scene, stride: int, offset: int = 0) -> Scene:
    """The same bundle (frames, images, poses) with every `stride`-th point
    only, starting at `offset`: a bounded sample of a large workload."""
    idx = np.arange(offset, scene.N, stride)
    return dataclasses.replace(scene, uv=np.ascontiguousarray(scene.uv[idx]),
                               vis=np.ascontiguousarray(scene.vis[idx]),
                               depths_gt=scene.depths_gt[idx].copy(), depths0=scene.depths0[idx].copy())
