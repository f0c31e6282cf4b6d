"""Seeded synthetic inputs shared by the CPU oracle and the GPU path.

Holds no bundle-adjustment arithmetic; see scene.py for the recipe.
"""
from .scene import (CONFIGS, PATTERN8, Scene, SceneConfig, bf16_round, bf16_to_f32,
                    build_renderer, make_scene)

__all__ = ["CONFIGS", "PATTERN8", "Scene", "SceneConfig", "bf16_round", "bf16_to_f32",
           "build_renderer", "make_scene"]
