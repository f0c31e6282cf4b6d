"""Thin Python binding of libpba.so (the C ABI in include/pba.h).

Argument marshalling only: every step of the method runs in the library's
CUDA kernels. PyTorch supplies device memory (the workspace and, optionally,
the images) and the CUDA stream. There is no CPU fallback: if the library is
missing, loading raises.
"""
from __future__ import annotations

import ctypes
import os
import re

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libpba.so")
HEADERS = [os.path.join(os.path.dirname(HERE), "include", h) for h in ("pba.h", "pba_mlp.h")]

PBA_F32, PBA_F16, PBA_BF16 = 0, 1, 2
PBA_MEM_DEVICE, PBA_MEM_HOST = 0, 1
PBA_SCHUR_TENSOR, PBA_SCHUR_SIMT, PBA_SCHUR_AUTO = 0, 1, 2
TIMING_SLOTS = 7
TIMING_NAMES = ["precompute", "pass", "reduce", "schur", "solve", "eval", "point"]
STATUS = {0: "PBA_OK", 1: "PBA_ERR_ARG", 2: "PBA_ERR_STATE", 3: "PBA_ERR_CUDA",
          4: "PBA_ERR_NOMEM", 5: "PBA_ERR_NOT_PD", 6: "PBA_ERR_NONFINITE",
          7: "PBA_ERR_TIMEOUT"}

_lib = None


class PbaError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


class Config(ctypes.Structure):
    _fields_ = [("huber_k", ctypes.c_double), ("pattern_size", ctypes.c_int),
                ("pattern", ctypes.POINTER(ctypes.c_int32)), ("gauge_anchor_w", ctypes.c_double),
                ("conv_px", ctypes.c_double), ("n_bundles", ctypes.c_int),
                ("cuda_stream", ctypes.c_void_p), ("use_graphs", ctypes.c_int),
                ("max_stats_iters", ctypes.c_int), ("autotune", ctypes.c_int), ("damping", ctypes.c_double),
                ("photometric", ctypes.c_int), ("photo_prior", ctypes.c_double)]


class IterStats(ctypes.Structure):
    _fields_ = [(n, ctypes.c_double) for n in
                ("energy", "rms", "n_valid", "max_disp_px", "dtheta_norm", "dd_norm")]


def declared_symbols():
    """Function names declared in include/pba.h and include/pba_mlp.h."""
    text = "".join(open(h).read() for h in HEADERS)
    return sorted(set(re.findall(r"\b(pba_[a-z_0-9]+)\s*\(", text)))


def load(path: str = LIB_PATH) -> ctypes.CDLL:
    """Loads libpba.so and declares its signatures (raises when missing)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise PbaError(-1, f"{path} is missing: build it first (paper_1704_06967_gb300.build)")
    lib = ctypes.CDLL(path)
    vp, i, d, i64 = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_int64
    sigs = {
        "pba_create": ([ctypes.POINTER(Config), ctypes.POINTER(vp)], i),
        "pba_destroy": ([vp], None),
        "pba_last_error": ([vp], ctypes.c_char_p),
        "pba_set_frames": ([vp, i, i, i, i, i, i, i, vp, vp, vp], i),
        "pba_set_points": ([vp, i, i, vp, vp, vp], i),
        "pba_workspace_size": ([vp, ctypes.POINTER(ctypes.c_size_t)], i),
        "pba_set_workspace": ([vp, vp, ctypes.c_size_t], i),
        "pba_precompute_ic": ([vp], i),
        "pba_iterate": ([vp, i, vp], i),
        "pba_solve_fc": ([vp, i, vp], i),
        "pba_solve_ic": ([vp, i, i, vp], i),
        "pba_set_window": ([vp, i, vp], i),
        "pba_downsample": ([vp, i, i, i, i, i, vp, vp], i),
        "pba_pyramid_workspace_size": ([ctypes.POINTER(Config), i, i, i, i, vp, vp, i, vp, vp, vp,
                                        ctypes.POINTER(ctypes.c_size_t)], i),
        "pba_solve_pyramid": ([ctypes.POINTER(Config), i, vp, i, i, vp, i, i, i, i, i, vp, vp, i, vp, vp, vp, vp,
                               ctypes.c_size_t, vp, vp], i),
        "pba_get_brightness": ([vp, i, vp], i),
        "pba_set_brightness": ([vp, i, vp], i),
        "pba_update_ic": ([vp], i),
        "pba_get_params": ([vp, i, vp, vp], i),
        "pba_set_params": ([vp, i, vp, vp], i),
        "pba_get_last_update": ([vp, i, vp, vp], i),
        "pba_get_system": ([vp, i, i, vp, vp, vp, vp], i),
        "pba_num_residuals": ([vp, i, ctypes.POINTER(i64)], i),
        "pba_enable_timing": ([vp, i], i),
        "pba_last_timing": ([vp, vp], i),
        "pba_transfer_bytes": ([vp, ctypes.POINTER(i64), ctypes.POINTER(i64)], i),
        "pba_get_tuning": ([vp, ctypes.POINTER(i), ctypes.POINTER(i)], i),
        "pba_set_tuning": ([vp, i, i], i),
        "pba_set_schur_path": ([vp, i], i),
        "pba_shard_ic_precompute": ([vp, i], i),
        "pba_shard_ic_step": ([vp, i, i], i),
        "pba_shard_fc_step": ([vp, i, i], i),
        "pba_shard_eval": ([vp, i, i], i),
        "pba_shard_count": ([vp, i, ctypes.POINTER(i64)], i),
        "pba_shard_export": ([vp, i, vp], i),
        "pba_shard_import": ([vp, i, vp], i),
        "pba_shard_stats": ([vp, i, vp], i),
        "pba_bundle_errors": ([vp, vp], i),
        "pba_depth_features": ([vp, i, vp], i),
        "pba_mlp_pack": ([vp, vp, vp], i),
        "pba_mlp_infer": ([vp, i, vp, vp, vp, vp], i),
        "pba_mlp_scratch_floats": ([i], ctypes.c_size_t),
        "pba_wait_selftest": ([vp, vp], i),
        "pba_mlp_grad": ([vp, i, vp, vp, vp, vp, vp, vp], i),
        "pba_mlp_train_step": ([vp, vp, vp, i, ctypes.c_float, i, vp, vp, vp, vp, vp], i),
        "pba_propose_depths": ([vp, i, vp, vp], i),
    }
    for name, (args, res) in sigs.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = res
    _lib = lib
    return lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _photo_mode(photometric) -> int:
    """cfg.photometric from the binding's argument: False/0 off, True/1 or
    "fit" the per-step moment fit, 2 or "joint" the pairs as unknowns of the
    IC system."""
    if isinstance(photometric, str):
        modes = {"off": 0, "fit": 1, "joint": 2}
        if photometric not in modes:
            raise ValueError(f"photometric must be one of {sorted(modes)}")
        return modes[photometric]
    v = int(photometric)
    if v not in (0, 1, 2):
        raise ValueError("photometric must be 0, 1 or 2")
    return v


def _scene_images(scene, device_images=True):
    """A synth.Scene's image stack as a CUDA tensor (or the host array)."""
    import torch
    store = scene.images_store
    if isinstance(store, torch.Tensor):  # rendered on the device (synth.make_scene(device="cuda"))
        if device_images:
            return store.contiguous()
        return store.view(torch.int16).cpu().numpy().view(np.uint16) if store.dtype == torch.bfloat16 \
            else store.cpu().numpy()
    if not device_images:
        return store
    if scene.dtype == "bf16":
        t = torch.from_numpy(store.view(np.int16)).cuda().view(torch.bfloat16)
    else:
        t = torch.from_numpy(store).cuda()
    return t.contiguous()


class Batch:
    """Independent bundles solved together in one context: every kernel of
    an iteration runs over all of them in one launch, each bundle keeping its
    own reference frame, gauge and reduced camera system.

    items: sequence of (images, poses0, intrinsics, uv, inv_depth, vis) per
    bundle. images: torch tensor [F, H, W] on the GPU (float32, float16 or
    bfloat16; borrowed) or a host numpy array of the same layout (copied into
    the workspace by the library). The bundles share the camera (image size,
    type, intrinsics). The workspace is one torch uint8 tensor on the current
    CUDA device.
    """

    def __init__(self, items, *, pattern, huber_k, stream=None, gauge_anchor_w=1.0, max_stats_iters=256,
                 use_graphs=False, autotune=False, damping=0.0, photometric=False, photo_prior=0.0):
        import torch
        self.torch = torch
        lib = load()
        self.lib = lib
        if stream is None:
            stream = torch.cuda.current_stream()
        self.stream = stream
        pat = np.ascontiguousarray(pattern, dtype=np.int32)
        self._pat = pat
        items = list(items)
        self.B = len(items)
        cfg = Config(float(huber_k), pat.shape[0],
                     pat.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), float(gauge_anchor_w),
                     0.0, self.B, ctypes.c_void_p(stream.cuda_stream), int(bool(use_graphs)),
                     int(max_stats_iters), int(bool(autotune)), float(damping), _photo_mode(photometric),
                     float(photo_prior))
        h = ctypes.c_void_p()
        self.h = None
        self._check(lib.pba_create(ctypes.byref(cfg), ctypes.byref(h)), None)
        self.h = h
        self.P = pat.shape[0]
        self._keep = []
        self.Fs, self.Ns = [], []
        for b, (images, poses0, intrinsics, uv, inv_depth, vis) in enumerate(items):
            if isinstance(images, torch.Tensor):
                assert images.is_cuda and images.dim() == 3 and images.is_contiguous()
                dt = {torch.float32: PBA_F32, torch.float16: PBA_F16,
                      torch.bfloat16: PBA_BF16}[images.dtype]
                mem, ptr = PBA_MEM_DEVICE, ctypes.c_void_p(images.data_ptr())
                self._keep.append(images)
            else:
                arr = np.ascontiguousarray(images)
                dt = {np.dtype(np.float32): PBA_F32, np.dtype(np.float16): PBA_F16,
                      np.dtype(np.uint16): PBA_BF16}[arr.dtype]
                mem, ptr = PBA_MEM_HOST, _p(arr)
                self._keep.append(arr)
            F, H, W = images.shape
            self.H, self.W = int(H), int(W)
            self.Fs.append(int(F))
            poses0 = np.ascontiguousarray(poses0, dtype=np.float64)
            K = np.ascontiguousarray(intrinsics, dtype=np.float64)
            self._check(lib.pba_set_frames(h, b, int(F), self.W, self.H, self.W, dt, mem, ptr,
                                           _p(poses0), _p(K)))
            uv = np.ascontiguousarray(uv, dtype=np.int32)
            d0 = np.ascontiguousarray(inv_depth, dtype=np.float64)
            self.Ns.append(uv.shape[0])
            visp = None
            if vis is not None:
                vis = np.ascontiguousarray(vis, dtype=np.uint8)
                assert vis.shape == (uv.shape[0], int(F))
                visp = _p(vis)
                self._keep.append(vis)
            self._check(lib.pba_set_points(h, b, uv.shape[0], _p(uv), _p(d0), visp))
        nb = ctypes.c_size_t()
        self._check(lib.pba_workspace_size(h, ctypes.byref(nb)))
        self.workspace = torch.empty(int(nb.value) + 256, dtype=torch.uint8, device="cuda")
        base = self.workspace.data_ptr()
        aligned = (base + 255) // 256 * 256
        self._check(lib.pba_set_workspace(h, ctypes.c_void_p(aligned), int(nb.value)))
        self.workspace_bytes = int(nb.value)

    @classmethod
    def from_scenes(cls, scenes, device_images=True, **kw):
        """Batch from synth.Scene objects that share the camera and pattern."""
        s0 = scenes[0]
        items = [(_scene_images(sc, device_images), sc.poses0, sc.intrinsics, sc.uv, sc.depths0, sc.vis)
                 for sc in scenes]
        return cls(items, pattern=s0.pattern, huber_k=s0.huber_k, **kw)

    # ------------------------------------------------------------------
    def _check(self, st, h=True):
        if st != 0:
            msg = self.lib.pba_last_error(self.h if h else None)
            raise PbaError(st, msg.decode() if msg else "")

    def close(self):
        if getattr(self, "h", None):
            self.lib.pba_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def precompute_ic(self):
        self._check(self.lib.pba_precompute_ic(self.h))

    def _stats(self, fn, n_iters, stats):
        if stats:
            arr = (IterStats * (n_iters + 1))()
            self._check(fn(self.h, int(n_iters), ctypes.cast(arr, ctypes.c_void_p)))
            return np.array([[getattr(s, f) for f, _ in IterStats._fields_] for s in arr])
        self._check(fn(self.h, int(n_iters), None))
        return None

    def iterate(self, n_iters, stats=True):
        """IC iterations; returns stats [n+1, 6] (energy, rms, n_valid,
        max_disp_px, dtheta_norm, dd_norm) or None."""
        return self._stats(self.lib.pba_iterate, n_iters, stats)

    def brightness(self, bundle=0):
        """Affine brightness pairs [F_b, 2] (alpha_f, beta_f)."""
        ab = np.zeros((self.Fs[bundle], 2))
        self._check(self.lib.pba_get_brightness(self.h, bundle, _p(ab)))
        return ab

    def set_brightness(self, ab, bundle=0):
        ab = np.ascontiguousarray(ab, dtype=np.float64)
        assert ab.shape == (self.Fs[bundle], 2)
        self._check(self.lib.pba_set_brightness(self.h, bundle, _p(ab)))

    def set_window(self, in_window, bundle=0):
        """Frames of the bundle in the sliding window (F_b flags)."""
        flags = np.ascontiguousarray(np.asarray(in_window, dtype=bool).astype(np.uint8))
        assert flags.shape == (self.Fs[bundle],)
        self._check(self.lib.pba_set_window(self.h, bundle, _p(flags)))

    def update_ic(self):
        """Incremental IC system update after a window change."""
        self._check(self.lib.pba_update_ic(self.h))

    def solve_ic(self, n_iters, reanchor_every=0, stats=True):
        """Precompute + n_iters IC iterations, re-anchoring p_0 every
        reanchor_every iterations (0: never), in one library call."""
        fn = lambda h, n, p: self.lib.pba_solve_ic(h, n, int(reanchor_every), p)
        return self._stats(fn, n_iters, stats)

    def solve_fc(self, n_iters, stats=True):
        return self._stats(self.lib.pba_solve_fc, n_iters, stats)

    def params(self, bundle=0):
        poses = np.zeros((self.Fs[bundle], 12))
        d = np.zeros(self.Ns[bundle])
        self._check(self.lib.pba_get_params(self.h, bundle, _p(poses), _p(d)))
        return poses, d

    def set_params(self, poses, depths, bundle=0):
        poses = np.ascontiguousarray(poses, dtype=np.float64)
        depths = np.ascontiguousarray(depths, dtype=np.float64)
        self._check(self.lib.pba_set_params(self.h, bundle, _p(poses), _p(depths)))

    def last_update(self, bundle=0):
        dth = np.zeros((self.Fs[bundle], 6))
        dd = np.zeros(self.Ns[bundle])
        self._check(self.lib.pba_get_last_update(self.h, bundle, _p(dth), _p(dd)))
        return dth, dd

    def system(self, fc=False, bundle=0):
        F, N = self.Fs[bundle], self.Ns[bundle]
        n6 = 6 * (F - 1)
        Hff = np.zeros((F, 6, 6))
        Hfd = np.zeros((N, F, 6))
        Hdd = np.zeros(N)
        S = np.zeros((n6, n6))
        self._check(self.lib.pba_get_system(self.h, bundle, int(bool(fc)), _p(Hff), _p(Hfd), _p(Hdd), _p(S)))
        return dict(Hff=Hff, Hfd=Hfd, Hdd=Hdd, S=S)

    def n_residuals(self, bundle=None):
        """Residual count of one bundle, or of all (bundle=None)."""
        total = 0
        for b in (range(self.B) if bundle is None else [bundle]):
            n = ctypes.c_int64()
            self._check(self.lib.pba_num_residuals(self.h, b, ctypes.byref(n)))
            total += int(n.value)
        return total

    def enable_timing(self, mask=-1):
        """mask: bit s times slot s (TIMING_NAMES order); -1 all, 0 none."""
        self._check(self.lib.pba_enable_timing(self.h, int(mask)))

    def bundle_errors(self):
        """Per-bundle error bits of the last synchronising call (1: system
        not positive definite, 2: non-finite update)."""
        out = np.zeros(self.B, dtype=np.int32)
        self._check(self.lib.pba_bundle_errors(self.h, _p(out)))
        return out

    def depth_features(self, bundle=0):
        """Learned-proposal features of the bundle's points at the current
        poses: torch float32 [N, 96] on the GPU (caller's point order)."""
        t = self.torch.empty((self.Ns[bundle], 96), dtype=self.torch.float32, device="cuda")
        self._check(self.lib.pba_depth_features(self.h, bundle, ctypes.c_void_p(t.data_ptr())))
        return t

    def propose_depths(self, packed, bundle=0):
        """Replaces the bundle's inverse depths by the network's proposals
        (packed: the inference layout, a torch uint8 CUDA tensor)."""
        scratch = self.torch.empty(self.Ns[bundle] * 97 + 4, dtype=self.torch.float32, device="cuda")
        self._check(self.lib.pba_propose_depths(self.h, bundle, ctypes.c_void_p(packed.data_ptr()),
                                                ctypes.c_void_p(scratch.data_ptr())))

    def tuning(self):
        """(warps per CTA of the IC residual pass, CTAs per bundle of the factorisation)."""
        w, c = ctypes.c_int(), ctypes.c_int()
        self._check(self.lib.pba_get_tuning(self.h, ctypes.byref(w), ctypes.byref(c)))
        return int(w.value), int(c.value)

    def set_tuning(self, res_warps, ldl_cluster):
        """Sets the launch shapes (as tuning() returns them); results do not
        depend on them."""
        self._check(self.lib.pba_set_tuning(self.h, int(res_warps), int(ldl_cluster)))

    def set_schur_path(self, path):
        """How the Schur complement is formed: PBA_SCHUR_AUTO (the default: by
        the problem's size), PBA_SCHUR_TENSOR (tensor cores) or PBA_SCHUR_SIMT
        (exact products on the SIMT pipes)."""
        self._check(self.lib.pba_set_schur_path(self.h, int(path)))

    def transfer_bytes(self):
        a, b = ctypes.c_int64(), ctypes.c_int64()
        self._check(self.lib.pba_transfer_bytes(self.h, ctypes.byref(a), ctypes.byref(b)))
        return int(a.value), int(b.value)

    def timing(self):
        out = np.zeros(2 * TIMING_SLOTS + 1)
        self._check(self.lib.pba_last_timing(self.h, _p(out)))
        ms = dict(zip(TIMING_NAMES, out[:TIMING_SLOTS]))
        counts = dict(zip(TIMING_NAMES, out[TIMING_SLOTS + 1:].astype(int)))
        return ms, int(out[TIMING_SLOTS]), counts


class Bundle(Batch):
    """One bundle: reference + target images, p_0, points, visibility (a
    context of one bundle; see Batch for the arguments)."""

    def __init__(self, images, poses0, intrinsics, uv, inv_depth, vis=None, **kw):
        super().__init__([(images, poses0, intrinsics, uv, inv_depth, vis)], **kw)
        self.F, self.N = self.Fs[0], self.Ns[0]

    @classmethod
    def from_scene(cls, scene, device_images=True, **kw):
        """Bundle from a synth.Scene (images uploaded with torch, or host)."""
        return cls(_scene_images(scene, device_images), scene.poses0, scene.intrinsics, scene.uv,
                   scene.depths0, scene.vis, pattern=scene.pattern, huber_k=scene.huber_k, **kw)
