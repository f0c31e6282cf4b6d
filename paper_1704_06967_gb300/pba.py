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
HEADER = os.path.join(os.path.dirname(HERE), "include", "pba.h")

PBA_F32, PBA_F16, PBA_BF16 = 0, 1, 2
PBA_MEM_DEVICE, PBA_MEM_HOST = 0, 1
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
                ("max_stats_iters", ctypes.c_int)]


class IterStats(ctypes.Structure):
    _fields_ = [(n, ctypes.c_double) for n in
                ("energy", "rms", "n_valid", "max_disp_px", "dtheta_norm", "dd_norm")]


def declared_symbols():
    """Function names declared in include/pba.h."""
    text = open(HEADER).read()
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
        "pba_get_params": ([vp, i, vp, vp], i),
        "pba_set_params": ([vp, i, vp, vp], i),
        "pba_get_last_update": ([vp, i, vp, vp], i),
        "pba_get_system": ([vp, i, i, vp, vp, vp, vp], i),
        "pba_num_residuals": ([vp, i, ctypes.POINTER(i64)], i),
        "pba_enable_timing": ([vp, i], i),
        "pba_last_timing": ([vp, vp], i),
        "pba_transfer_bytes": ([vp, ctypes.POINTER(i64), ctypes.POINTER(i64)], i),
    }
    for name, (args, res) in sigs.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = res
    _lib = lib
    return lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


class Bundle:
    """One bundle: reference + target images, p_0, points, visibility.

    images: torch tensor [F, H, W] on the GPU (float32, float16 or bfloat16;
    borrowed) or a host numpy array of the same layout (copied into the
    workspace by the library: mem="host"). The workspace is one torch uint8
    tensor on the current CUDA device.
    """

    def __init__(self, images, poses0, intrinsics, uv, inv_depth, vis=None, *, pattern,
                 huber_k, stream=None, gauge_anchor_w=1.0, max_stats_iters=256, use_graphs=False):
        import torch
        self.torch = torch
        lib = load()
        self.lib = lib
        if stream is None:
            stream = torch.cuda.current_stream()
        self.stream = stream
        pat = np.ascontiguousarray(pattern, dtype=np.int32)
        self._pat = pat
        cfg = Config(float(huber_k), pat.shape[0],
                     pat.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), float(gauge_anchor_w),
                     0.0, 1, ctypes.c_void_p(stream.cuda_stream), int(bool(use_graphs)),
                     int(max_stats_iters))
        h = ctypes.c_void_p()
        self._check(lib.pba_create(ctypes.byref(cfg), ctypes.byref(h)), None)
        self.h = h
        self.P = pat.shape[0]
        self._keep = []
        if isinstance(images, torch.Tensor):
            assert images.is_cuda and images.dim() == 3 and images.is_contiguous()
            dt = {torch.float32: PBA_F32, torch.float16: PBA_F16, torch.bfloat16: PBA_BF16}[images.dtype]
            mem, ptr = PBA_MEM_DEVICE, ctypes.c_void_p(images.data_ptr())
            self._keep.append(images)
        else:
            arr = np.ascontiguousarray(images)
            dt = {np.dtype(np.float32): PBA_F32, np.dtype(np.float16): PBA_F16,
                  np.dtype(np.uint16): PBA_BF16}[arr.dtype]
            mem, ptr = PBA_MEM_HOST, _p(arr)
            self._keep.append(arr)
        F, H, W = images.shape
        self.F, self.H, self.W = int(F), int(H), int(W)
        poses0 = np.ascontiguousarray(poses0, dtype=np.float64)
        K = np.ascontiguousarray(intrinsics, dtype=np.float64)
        self._check(lib.pba_set_frames(h, 0, self.F, self.W, self.H, self.W, dt, mem, ptr,
                                       _p(poses0), _p(K)))
        uv = np.ascontiguousarray(uv, dtype=np.int32)
        d0 = np.ascontiguousarray(inv_depth, dtype=np.float64)
        self.N = uv.shape[0]
        visp = None
        if vis is not None:
            vis = np.ascontiguousarray(vis, dtype=np.uint8)
            assert vis.shape == (self.N, self.F)
            visp = _p(vis)
        self._check(lib.pba_set_points(h, 0, self.N, _p(uv), _p(d0), visp))
        nb = ctypes.c_size_t()
        self._check(lib.pba_workspace_size(h, ctypes.byref(nb)))
        self.workspace = torch.empty(int(nb.value) + 256, dtype=torch.uint8, device="cuda")
        base = self.workspace.data_ptr()
        aligned = (base + 255) // 256 * 256
        self._check(lib.pba_set_workspace(h, ctypes.c_void_p(aligned), int(nb.value)))
        self.workspace_bytes = int(nb.value)

    @classmethod
    def from_scene(cls, scene, device_images=True, **kw):
        """Bundle from a synth.Scene (images uploaded with torch, or host)."""
        import torch
        if device_images:
            store = scene.images_store
            if scene.dtype == "bf16":
                t = torch.from_numpy(store.view(np.int16)).cuda().view(torch.bfloat16)
            else:
                t = torch.from_numpy(store).cuda()
            images = t.contiguous()
        else:
            images = scene.images_store
        return cls(images, scene.poses0, scene.intrinsics, scene.uv, scene.depths0, scene.vis,
                   pattern=scene.pattern, huber_k=scene.huber_k, **kw)

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

    def solve_fc(self, n_iters, stats=True):
        return self._stats(self.lib.pba_solve_fc, n_iters, stats)

    def params(self):
        poses = np.zeros((self.F, 12))
        d = np.zeros(self.N)
        self._check(self.lib.pba_get_params(self.h, 0, _p(poses), _p(d)))
        return poses, d

    def set_params(self, poses, depths):
        poses = np.ascontiguousarray(poses, dtype=np.float64)
        depths = np.ascontiguousarray(depths, dtype=np.float64)
        self._check(self.lib.pba_set_params(self.h, 0, _p(poses), _p(depths)))

    def last_update(self):
        dth = np.zeros((self.F, 6))
        dd = np.zeros(self.N)
        self._check(self.lib.pba_get_last_update(self.h, 0, _p(dth), _p(dd)))
        return dth, dd

    def system(self, fc=False):
        n6 = 6 * (self.F - 1)
        Hff = np.zeros((self.F, 6, 6))
        Hfd = np.zeros((self.N, self.F, 6))
        Hdd = np.zeros(self.N)
        S = np.zeros((n6, n6))
        self._check(self.lib.pba_get_system(self.h, 0, int(bool(fc)), _p(Hff), _p(Hfd), _p(Hdd), _p(S)))
        return dict(Hff=Hff, Hfd=Hfd, Hdd=Hdd, S=S)

    def n_residuals(self):
        n = ctypes.c_int64()
        self._check(self.lib.pba_num_residuals(self.h, 0, ctypes.byref(n)))
        return int(n.value)

    def enable_timing(self, mask=-1):
        """mask: bit s times slot s (TIMING_NAMES order); -1 all, 0 none."""
        self._check(self.lib.pba_enable_timing(self.h, int(mask)))

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
