"""Coarse-to-fine solving over an image pyramid (an addition beyond the
paper: a direct method's basin widens at coarse levels). Orchestration only:
the levels are formed by pba_downsample and every solve runs in the
library's kernels.

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

from .pba import PBA_BF16, PBA_F16, PBA_F32, Bundle, PbaError, load


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


def level_points(uv, level, W, H, pattern):
    """Pixels of the points at a level and which points take part there."""
    s = 2.0 ** level
    uvl = np.rint((np.asarray(uv, np.float64) + 0.5) / s - 0.5).astype(np.int32)
    rad = int(np.abs(pattern).max()) + 1
    keep = (uvl[:, 0] >= rad) & (uvl[:, 0] <= W - 1 - rad) & (uvl[:, 1] >= rad) & (uvl[:, 1] <= H - 1 - rad)
    return uvl, keep


def solve_coarse_to_fine(images, poses0, intrinsics, uv, inv_depth, vis, *, pattern, huber_k, levels=3,
                         iters=(10, 10, 20), method="ic", reanchor_every=3, damping=0.0, stream=None,
                         level_ms=None):
    """Solves from the coarsest level (levels - 1) to the full resolution.
    images: [F, H, W] CUDA tensor; the rest as for Bundle. iters: iterations
    per level, coarsest first. Returns (poses, inv_depth, [stats per level]).
    level_ms: a list that receives, per level, the device time (ms, CUDA
    events on the stream) of the level's solve call (the image reduction and
    the context set-up excluded)."""
    poses = np.array(poses0, dtype=np.float64)
    depth = np.array(inv_depth, dtype=np.float64)
    K = np.asarray(intrinsics, dtype=np.float64)
    pyr = [images]
    for _ in range(levels - 1):
        pyr.append(downsample(pyr[-1]))
    stats = []
    for lvl in range(levels - 1, -1, -1):
        img = pyr[lvl].contiguous()
        F, H, W = img.shape
        s = 2.0 ** lvl
        Kl = np.array([K[0] / s, K[1] / s, (K[2] + 0.5) / s - 0.5, (K[3] + 0.5) / s - 0.5])
        uvl, keep = level_points(uv, lvl, W, H, pattern)
        b = Bundle(img, poses, Kl, uvl[keep], depth[keep], None if vis is None else vis[keep], pattern=pattern,
                   huber_k=huber_k, stream=stream, damping=damping)
        n = iters[levels - 1 - lvl]
        if level_ms is not None:
            import torch
            s_ = b.stream
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(s_)
        if method == "ic":
            st = b.solve_ic(n, reanchor_every=reanchor_every)
        else:
            st = b.solve_fc(n)
        if level_ms is not None:
            e1.record(s_)
            e1.synchronize()
            level_ms.append(e0.elapsed_time(e1))
        p, d = b.params()
        b.close()
        poses = p
        # a point the level drove to a non-positive inverse depth keeps the
        # one it entered the level with
        sub = depth[keep]
        good = np.isfinite(d) & (d > 0)
        sub[good] = d[good]
        depth[keep] = sub
        stats.append(st)
    return poses, depth, stats
