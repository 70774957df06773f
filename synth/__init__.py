"""Seeded synthetic inputs shared by the oracle tests and the CUDA path.

This package holds input generation only: scene descriptions (solids,
placements, materials with toy attenuation tables) and source descriptions.
It contains none of the navigation or transport arithmetic; both the oracle
(``oracle/``) and the CUDA library (``paper_1209_5235_gb300``) consume the
plain numbers it produces.
"""
from .materials import Material, make_material, toy_materials, E_GRID_MEV
from .scenes import (Scene, Source, Solid, Placement, VoxelSpec, tiny_scene, calorimeter_scene,
                     batched_scenes, barrel_scene, slab_scene, layered_scene, spheres_scene,
                     CONFIG_SEEDS)

__all__ = ["Material", "make_material", "toy_materials", "E_GRID_MEV", "Scene", "Source", "Solid",
           "Placement", "VoxelSpec", "tiny_scene", "calorimeter_scene", "batched_scenes", "barrel_scene",
           "slab_scene", "layered_scene", "spheres_scene", "CONFIG_SEEDS"]
