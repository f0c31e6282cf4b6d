"""Seeded batches of independent bundles of uneven size.

Input generation only (no bundle-adjustment arithmetic). Recipe of a batch of
B bundles, all drawn from one generator seeded with BATCH_SEED:
  * frames F_b uniform in {4, ..., 64} (reference included), on a helix
    around the object with the per-frame step of the 30-frame helix (24 deg
    of azimuth per frame: F_b / 15 turns, height +-0.5, radius 3);
  * points N_b log-uniform in [500, 50,000]; a small sphere offers fewer
    candidate pixels than that, and then all of them are taken;
  * sphere radius uniform in [0.5, 2], texture seed = bundle index;
  * 640 x 480 FP16 images, f = 525, the 8-pixel pattern, and the
    perturbation and noise of the single-bundle scenes (2 deg / 0.02 pose
    error, 5 % inverse-depth error, noise 2/255, Huber k = 9/255).
Every bundle shares the camera (image size, type, intrinsics), as one
context of the library requires.
"""
from __future__ import annotations

import concurrent.futures as cf
import dataclasses
import math
import multiprocessing as mp
import os

import numpy as np

from .scene import SceneConfig, build_renderer, make_scene

BATCH_SEED = 17043


@dataclasses.dataclass(frozen=True)
class BundleDraw:
    index: int
    n_frames: int
    n_points: int
    sphere_r: float


def draw_batch(n_bundles: int, seed: int = BATCH_SEED, frames=(4, 64), points=(500, 50000),
               radii=(0.5, 2.0)) -> list[BundleDraw]:
    """The sizes of a batch (frames, requested points, sphere radius)."""
    rng = np.random.default_rng(seed)
    out = []
    lo, hi = math.log(points[0]), math.log(points[1])
    for b in range(n_bundles):
        F = int(rng.integers(frames[0], frames[1] + 1))
        N = int(round(math.exp(rng.uniform(lo, hi))))
        r = float(rng.uniform(radii[0], radii[1]))
        out.append(BundleDraw(b, F, N, r))
    return out


def bundle_config(d: BundleDraw, W: int = 640, H: int = 480, f: float = 525.0,
                  dtype: str = "f16") -> SceneConfig:
    return SceneConfig(f"batch{d.index}", W, H, f, d.n_points, "helix", n_frames=d.n_frames,
                       turns=d.n_frames / 15.0, sphere_r=d.sphere_r, dtype=dtype, spacing=1,
                       allow_fewer_points=True)


def _make_one(args):
    d, W, H, f, dtype, keep_f32 = args
    sc = make_scene(bundle_config(d, W, H, f, dtype), seed_offset=d.index)
    if not keep_f32:
        sc.images_f32 = None  # the storage array is what the solver reads
    return sc


def make_batch(n_bundles: int, seed: int = BATCH_SEED, W: int = 640, H: int = 480, f: float = 525.0,
               dtype: str = "f16", workers: int | None = None, keep_f32: bool = False, **draw_kw):
    """Generates the batch's scenes (in `workers` spawned processes; the
    renderer parallelises each image itself). Unless keep_f32, images_f32 is
    dropped from the returned scenes to save host memory (images_store holds
    the data the solver reads)."""
    draws = draw_batch(n_bundles, seed, **draw_kw)
    build_renderer()
    args = [(d, W, H, f, dtype, keep_f32) for d in draws]
    if workers is None:
        workers = max(1, min(8, (os.cpu_count() or 2) // 2))
    if workers <= 1 or n_bundles <= 1:
        return [_make_one(a) for a in args]
    with cf.ProcessPoolExecutor(max_workers=workers, mp_context=mp.get_context("spawn")) as ex:
        return list(ex.map(_make_one, args))
