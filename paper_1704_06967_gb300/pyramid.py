"""Coarse-to-fine solving over an image pyramid (an addition beyond the
paper: a direct method's basin widens at coarse levels). Marshalling only:
pba_solve_pyramid (include/pba.h) forms the levels with pba_downsample and
solves them one context per level, coarsest first.

Level L halves the images L times (2 x 2 means), with intrinsics f / 2^L and
(c + 0.5) / 2^L - 0.5. A point keeps its parameter (one inverse depth along
its reference ray) at every level; its level-L pixel is the nearest pixel
centre, (u + 0.5) / 2^L - 0.5 rounded, and points whose pattern (and its
gradient neighbours) would leave a level's reference image sit that level
out. The poses and the inverse depths a level reaches start the next finer
level.
"""
from __future__ import annotations

import ctypes

import numpy as np

from .pba import PBA_BF16, PBA_F16, PBA_F32, Config, IterStats, PbaError, _p, load


def downsample(images):
    """One pyramid level of a [F, H, W] CUDA tensor (float32/float16/bfloat16)
    -> float32 [F, H // 2, W // 2]."""
    import torch
    lib = load()
    F, H, W = images.shape
    dt = {torch.float32: PBA_F32, torch.float16: PBA_F16, torch.bfloat16: PBA_BF16}[images.dtype]
    out = torch.empty((F, H // 2, W // 2), dtype=torch.float32, device=images.device)
    st = torch.cuda.current_stream().cuda_stream
    rc = lib.pba_downsample(ctypes.c_void_p(images.data_ptr()), dt, F, W, H, W, ctypes.c_void_p(out.data_ptr()),
                            ctypes.c_void_p(st))
    if rc != 0:
        raise PbaError(rc, "pba_downsample failed")
    return out


def solve_coarse_to_fine(images, poses0, intrinsics, uv, inv_depth, vis, *, pattern, huber_k, levels=3,
                         iters=(10, 10, 20), method="ic", reanchor_every=3, damping=0.0, stream=None,
                         gauge_anchor_w=1.0, level_ms=None):
    """Solves from the coarsest level (levels - 1) to the full resolution
    (pba_solve_pyramid). images: [F, H, W] CUDA tensor (float32, float16 or
    bfloat16); the rest as for Bundle. iters: iterations per level, coarsest
    first. Returns (poses, inv_depth, [statistics per level]). level_ms: a
    list that receives, per level, the device time (ms) of the level's solve
    call (the image reduction and the context set-up excluded)."""
    import torch
    lib = load()
    if stream is None:
        stream = torch.cuda.current_stream()
    assert images.is_cuda and images.dim() == 3 and images.is_contiguous()
    F, H, W = images.shape
    dt = {torch.float32: PBA_F32, torch.float16: PBA_F16, torch.bfloat16: PBA_BF16}[images.dtype]
    pat = np.ascontiguousarray(pattern, dtype=np.int32)
    cfg = Config(float(huber_k), pat.shape[0], pat.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                 float(gauge_anchor_w), 0.0, 1, ctypes.c_void_p(stream.cuda_stream), 0, 256, 0, float(damping), 0)
    poses = np.array(poses0, dtype=np.float64, order="C")
    depth = np.array(inv_depth, dtype=np.float64, order="C")
    K = np.ascontiguousarray(intrinsics, dtype=np.float64)
    uv = np.ascontiguousarray(uv, dtype=np.int32)
    visp = None
    if vis is not None:
        vis = np.ascontiguousarray(vis, dtype=np.uint8)
        visp = _p(vis)
    its = np.ascontiguousarray(iters[:levels], dtype=np.int32)
    assert its.shape[0] == levels
    nb = ctypes.c_size_t()
    rc = lib.pba_pyramid_workspace_size(ctypes.byref(cfg), levels, F, W, H, _p(poses), _p(K), uv.shape[0], _p(uv),
                                        _p(depth), visp, ctypes.byref(nb))
    if rc != 0:
        raise PbaError(rc, "pba_pyramid_workspace_size failed")
    ws = torch.empty(int(nb.value) + 256, dtype=torch.uint8, device=images.device)
    base = (ws.data_ptr() + 255) // 256 * 256
    arr = (IterStats * int(its.sum() + levels))()
    ms = np.zeros(levels)
    rc = lib.pba_solve_pyramid(ctypes.byref(cfg), levels, _p(its), 0 if method == "ic" else 1, int(reanchor_every),
                               ctypes.c_void_p(images.data_ptr()), dt, F, W, H, W, _p(poses), _p(K), uv.shape[0],
                               _p(uv), _p(depth), visp, ctypes.c_void_p(base), int(nb.value),
                               ctypes.cast(arr, ctypes.c_void_p), _p(ms))
    if rc != 0:
        raise PbaError(rc, "pba_solve_pyramid failed")
    if level_ms is not None:
        level_ms.extend(float(x) for x in ms)
    st = np.array([[getattr(s, f) for f, _ in IterStats._fields_] for s in arr])
    stats, k = [], 0
    for n in its:
        stats.append(st[k:k + n + 1])
        k += n + 1
    return poses, depth, stats
