"""Seeded synthetic inputs shared by the CPU oracle and the GPU path.

Holds no bundle-adjustment arithmetic; see scene.py for the recipe.
"""
from .batch import BATCH_SEED, BundleDraw, bundle_config, draw_batch, make_batch
from .scene import (CONFIGS, PATTERN8, Scene, SceneConfig, bf16_round, bf16_to_f32,
                    build_renderer, build_renderer_gpu, make_scene, point_subset)

__all__ = ["BATCH_SEED", "BundleDraw", "bundle_config", "draw_batch", "make_batch", "CONFIGS", "PATTERN8", "Scene", "SceneConfig", "bf16_round", "bf16_to_f32",
           "build_renderer", "build_renderer_gpu", "make_scene", "point_subset"]
