"""Seeded synthetic scenes and γ sources for the navigation/transport workloads.

A ``Scene`` is plain data: a list of solids, a list of placements (each
placement is a distinct volume; placement 0 is the world), the materials with
their attenuation tables and the voxelisation request for the accelerated
navigator.  A ``Source`` describes how track ``i`` draws its initial
position, direction and energy; the draws themselves are made by each
implementation from its own counter-based generator keyed by the track id.

Workloads (lengths in mm, energies in MeV):

* ``tiny_scene``: 1 m water-like cube holding 10 axis-aligned boxes with full
  edges uniform in [20, 100] mm at seeded non-overlapping positions; one
  8x8x8 voxel level; 1 MeV γ isotropic from the origin.
* ``calorimeter_scene``: 2 m vacuum world holding a 1000x1000x375 mm envelope
  tiled by 50 alternating lead-like (5 mm) / scintillator-like (10 mm) layers
  of 10x10 cells of 100x100 mm (5000 cells); two voxel levels (z: 50, x: 10);
  γ along +z with energy uniform in [0.1, 10] MeV and a Gaussian spot of
  sigma 10 mm starting at z = -10 mm.
* ``batched_scenes``: 256 water-like 1 m worlds with log-uniform daughter
  counts in [10, 5000] of mixed boxes/tubes/orbs rotated about z; 10^3..10^5
  γ each, log-uniform energy in [0.05, 5] MeV, isotropic from the centre.
* ``barrel_scene``: 30 concentric tube shells (r in [50, 1500] mm, half
  length 1500 mm), each tiled by 64 φ segments, with 2000 lead-like orbs of
  radius [5, 20] mm embedded in segments; γ log-uniform in [0.02, 20] MeV,
  isotropic from points on the axis with z uniform in [-1500, 1500] mm.
* ``spheres_scene``: the Spheres geometry of the paper's benchmark: 8000
  aluminium balls on a regular 20x20x20 grid in a 5 m vacuum cube.
* ``slab_scene`` / ``layered_scene``: one slab / a stack of slabs used by the
  attenuation tests.
"""
from __future__ import annotations

import dataclasses
import math
from typing import Optional

import numpy as np

from .materials import Material, toy_materials, constant_material, vacuum, E_GRID_MEV

BOX, TUBE, ORB, CONE = 0, 1, 2, 3
TWO_PI = 2.0 * math.pi
CONFIG_SEEDS = {i: (0x6E4A0000 + i, 0x7A0C0000 + i) for i in range(5)}   # (geometry seed, track seed)


@dataclasses.dataclass
class Solid:
    kind: int                 # BOX, TUBE, ORB or CONE (rmin1, rmax1, rmin2, rmax2, hz; full in phi)
    params: tuple             # box: (hx, hy, hz); tube: (rmin, rmax, hz, sphi, dphi); orb: (r,)


@dataclasses.dataclass
class Placement:
    mother: int               # -1 for the world
    solid: int
    material: int
    t: tuple                  # translation of the local origin in the mother frame
    rot: tuple = (1.0, 0.0)   # (cos θ, sin θ) of the rotation about z (local -> mother)


@dataclasses.dataclass
class VoxelSpec:
    """Voxelisation request: fixed levels (axes + slice counts) or the smart heuristic."""
    mode: str = "smart"                   # "smart" | "fixed" | "none"
    axes: tuple = ()                      # fixed: axis per level (0=x, 1=y, 2=z)
    slices: tuple = ()                    # fixed: slices per level
    smartless: float = 2.0                # smart: slices per daughter
    max_slices: int = 1000
    max_levels: int = 3
    refine_above: int = 4                 # smart: refine nodes with more candidates than this


@dataclasses.dataclass
class Source:
    """Per-track source recipe; every random quantity is drawn by the consumer."""
    pos: tuple = (0.0, 0.0, 0.0)
    spot_sigma: float = 0.0               # Gaussian spot in x, y (Marsaglia polar method)
    z_range: Optional[tuple] = None       # uniform z on a line parallel to the axis
    isotropic: bool = True
    direction: tuple = (0.0, 0.0, 1.0)
    e_kind: str = "mono"                  # "mono" | "uniform" | "loguniform"
    e0: float = 1.0
    e1: float = 1.0

    E_KINDS = {"mono": 0, "uniform": 1, "loguniform": 2}

    def as_array(self) -> np.ndarray:
        """Flat float64 record: pos[3], sigma, has_z, z0, z1, iso, dir[3], e_kind, e0, e1 (16 values)."""
        z = self.z_range if self.z_range is not None else (0.0, 0.0)
        return np.array([*self.pos, self.spot_sigma, 1.0 if self.z_range is not None else 0.0, z[0], z[1],
                         1.0 if self.isotropic else 0.0, *self.direction, float(self.E_KINDS[self.e_kind]),
                         self.e0, self.e1, 0.0], dtype=np.float64)


@dataclasses.dataclass
class Scene:
    name: str
    materials: list
    solids: list
    placements: list
    voxel: VoxelSpec = dataclasses.field(default_factory=VoxelSpec)

    @property
    def n_volumes(self) -> int:
        return len(self.placements)


def _mat_index(mats: list, m: Material) -> int:
    mats.append(m)
    return len(mats) - 1


def _std_materials():
    tm = toy_materials()
    mats = [tm["water"], tm["lead"], tm["scint"], tm["al"], tm["vacuum"]]
    return mats, {"water": 0, "lead": 1, "scint": 2, "al": 3, "vacuum": 4}


def tiny_scene(seed: int = CONFIG_SEEDS[0][0], n_boxes: int = 10, voxel: Optional[VoxelSpec] = None) -> Scene:
    """1 m water-like cube with ``n_boxes`` seeded, non-overlapping, axis-aligned boxes."""
    rng = np.random.default_rng(seed)
    mats, mi = _std_materials()
    solids = [Solid(BOX, (500.0, 500.0, 500.0))]
    places = [Placement(-1, 0, mi["water"], (0.0, 0.0, 0.0))]
    boxes = []
    while len(boxes) < n_boxes:
        h = rng.uniform(20.0, 100.0, 3) / 2.0
        c = rng.uniform(-500.0 + h, 500.0 - h)
        if any(np.all(np.abs(c - c2) < h + h2) for c2, h2 in boxes):
            continue
        boxes.append((c, h))
    for i, (c, h) in enumerate(boxes):
        solids.append(Solid(BOX, tuple(float(x) for x in h)))
        places.append(Placement(0, len(solids) - 1, mi["lead"] if i % 2 == 0 else mi["scint"],
                                tuple(float(x) for x in c)))
    vox = voxel or VoxelSpec(mode="fixed", axes=(0, 1, 2), slices=(8, 8, 8))
    return Scene("tiny", mats, solids, places, vox)


def tiny_source() -> Source:
    return Source(pos=(0.0, 0.0, 0.0), isotropic=True, e_kind="mono", e0=1.0, e1=1.0)


def calorimeter_scene(nx: int = 10, ny: int = 10, n_layers: int = 50, voxel: Optional[VoxelSpec] = None) -> Scene:
    """Sampling calorimeter: alternating 5 mm lead-like and 10 mm scintillator-like layers of 100 mm cells."""
    mats, mi = _std_materials()
    thick = [5.0 if k % 2 == 0 else 10.0 for k in range(n_layers)]
    depth = float(sum(thick))
    hx, hy = 50.0 * nx, 50.0 * ny
    solids = [Solid(BOX, (1000.0, 1000.0, 1000.0)), Solid(BOX, (hx, hy, depth / 2.0)),
              Solid(BOX, (50.0, 50.0, 2.5)), Solid(BOX, (50.0, 50.0, 5.0))]
    places = [Placement(-1, 0, mi["vacuum"], (0.0, 0.0, 0.0)),
              Placement(0, 1, mi["vacuum"], (0.0, 0.0, depth / 2.0))]
    z = 0.0
    for k in range(n_layers):
        zc = z + thick[k] / 2.0 - depth / 2.0
        for i in range(nx):
            for j in range(ny):
                places.append(Placement(1, 2 if k % 2 == 0 else 3, mi["lead"] if k % 2 == 0 else mi["scint"],
                                        (-hx + 50.0 + 100.0 * i, -hy + 50.0 + 100.0 * j, zc)))
        z += thick[k]
    vox = voxel or VoxelSpec(mode="fixed", axes=(2, 0), slices=(n_layers, nx))
    return Scene("calorimeter", mats, solids, places, vox)


def calorimeter_source() -> Source:
    return Source(pos=(0.0, 0.0, -10.0), spot_sigma=10.0, isotropic=False, direction=(0.0, 0.0, 1.0),
                  e_kind="uniform", e0=0.1, e1=10.0)


def _bounding_radius(s: Solid) -> float:
    if s.kind == BOX:
        return float(math.sqrt(sum(h * h for h in s.params)))
    if s.kind == TUBE:
        return float(math.hypot(s.params[1], s.params[2]))
    return float(s.params[0])


def _random_daughter(rng, kind: int, scale: float) -> Solid:
    if kind == BOX:
        return Solid(BOX, tuple(float(x) for x in rng.uniform(10.0, 50.0, 3) * scale / 2.0))
    if kind == TUBE:
        rmax = rng.uniform(5.0, 25.0) * scale
        rmin = 0.0 if rng.uniform() < 0.5 else rng.uniform(0.2, 0.7) * rmax
        hz = rng.uniform(5.0, 25.0) * scale
        if rng.uniform() < 0.5:
            return Solid(TUBE, (float(rmin), float(rmax), float(hz), 0.0, TWO_PI))
        sphi = rng.uniform(0.0, TWO_PI)
        dphi = rng.uniform(0.25 * math.pi, 1.75 * math.pi)
        return Solid(TUBE, (float(rmin), float(rmax), float(hz), float(sphi), float(dphi)))
    return Solid(ORB, (float(rng.uniform(5.0, 25.0) * scale),))


def random_world(rng, n_d: int, world_half: float = 500.0, fill: float = 0.12) -> tuple[list, list]:
    """Mixed boxes/tubes/orbs, rotated about z, kept apart by their bounding spheres (seeded)."""
    mean_r = 30.0  # rough mean bounding radius at scale 1
    scale = min(1.0, (fill * (2 * world_half) ** 3 / (n_d * 4.0 / 3.0 * math.pi * mean_r ** 3)) ** (1.0 / 3.0))
    solids, places = [], []
    cell = 2.0 * 45.0 * scale + 1e-6
    grid: dict = {}
    centres = []
    radii = []
    kinds = (BOX, TUBE, ORB)
    tries = 0
    while len(places) < n_d:
        tries += 1
        if tries > 200 * n_d:
            raise RuntimeError("could not place daughters")
        s = _random_daughter(rng, kinds[len(places) % 3], scale)
        r = _bounding_radius(s)
        c = rng.uniform(-world_half + r + 1e-3, world_half - r - 1e-3, 3)
        key = tuple(int(math.floor(x / cell)) for x in c)
        ok = True
        for dx in (-1, 0, 1):
            for dy in (-1, 0, 1):
                for dz in (-1, 0, 1):
                    for j in grid.get((key[0] + dx, key[1] + dy, key[2] + dz), ()):
                        if np.sum((centres[j] - c) ** 2) < (radii[j] + r + 1e-3) ** 2:
                            ok = False
                            break
                    if not ok:
                        break
                if not ok:
                    break
            if not ok:
                break
        if not ok:
            continue
        grid.setdefault(key, []).append(len(centres))
        centres.append(c)
        radii.append(r)
        th = rng.uniform(0.0, TWO_PI)
        solids.append(s)
        places.append((tuple(float(x) for x in c), (float(math.cos(th)), float(math.sin(th)))))
    return solids, places


def batched_scenes(n_geoms: int = 256, seed: int = CONFIG_SEEDS[2][0], d_range=(10, 5000),
                   tracks_range=(1000, 100000)) -> list[tuple[Scene, int]]:
    """Independent water-like worlds with log-uniform daughter counts; returns (scene, n_tracks) pairs."""
    rng = np.random.default_rng(seed)
    out = []
    for g in range(n_geoms):
        mats, mi = _std_materials()
        n_d = int(round(math.exp(rng.uniform(math.log(d_range[0]), math.log(d_range[1])))))
        n_t = int(round(math.exp(rng.uniform(math.log(tracks_range[0]), math.log(tracks_range[1])))))
        dsol, dpl = random_world(rng, n_d)
        solids = [Solid(BOX, (500.0, 500.0, 500.0))] + dsol
        places = [Placement(-1, 0, mi["water"], (0.0, 0.0, 0.0))]
        for i, (t, rot) in enumerate(dpl):
            places.append(Placement(0, i + 1, (mi["lead"], mi["scint"], mi["al"])[i % 3], t, rot))
        out.append((Scene(f"batched{g}", mats, solids, places, VoxelSpec(mode="smart")), n_t))
    return out


def batched_source() -> Source:
    return Source(pos=(0.0, 0.0, 0.0), isotropic=True, e_kind="loguniform", e0=0.05, e1=5.0)


def barrel_scene(seed: int = CONFIG_SEEDS[3][0], n_shells: int = 30, n_phi: int = 64, n_orbs: int = 2000,
                 r_in: float = 50.0, r_out: float = 1500.0, half_len: float = 1500.0) -> Scene:
    """Concentric shells tiled by φ segments with embedded orbs (depth 4: world/shell/segment/orb)."""
    rng = np.random.default_rng(seed)
    mats, mi = _std_materials()
    solids = [Solid(BOX, (2000.0, 2000.0, 2000.0))]
    places = [Placement(-1, 0, mi["vacuum"], (0.0, 0.0, 0.0))]
    dr = (r_out - r_in) / n_shells
    dphi = TWO_PI / n_phi
    seg_index = []   # (volume id, shell) per segment
    for i in range(n_shells):
        rmin, rmax = r_in + i * dr, r_in + (i + 1) * dr
        mat = mi["scint"] if i % 2 == 0 else mi["al"]
        solids.append(Solid(TUBE, (rmin, rmax, half_len, 0.0, TWO_PI)))
        places.append(Placement(0, len(solids) - 1, mat, (0.0, 0.0, 0.0)))
        shell_vol = len(places) - 1
        solids.append(Solid(TUBE, (rmin, rmax, half_len, 0.0, dphi)))
        seg_solid = len(solids) - 1
        for k in range(n_phi):
            th = k * dphi
            places.append(Placement(shell_vol, seg_solid, mat, (0.0, 0.0, 0.0), (math.cos(th), math.sin(th))))
            seg_index.append((len(places) - 1, i))
    orbs_in = {}
    margin = 0.5
    placed = 0
    tries = 0
    while placed < n_orbs:
        tries += 1
        if tries > 100 * n_orbs:
            raise RuntimeError("could not place orbs")
        vol, i = seg_index[int(rng.integers(len(seg_index)))]
        r = float(rng.uniform(5.0, 20.0))
        rmin, rmax = r_in + i * dr, r_in + (i + 1) * dr
        lo, hi = rmin + r + margin, rmax - r - margin
        if lo >= hi:
            continue
        rc = float(rng.uniform(lo, hi))
        half_ang = math.asin(min(1.0, (r + margin) / rc))
        if 2.0 * half_ang >= dphi:
            continue
        ph = float(rng.uniform(half_ang, dphi - half_ang))
        zc = float(rng.uniform(-half_len + r + margin, half_len - r - margin))
        c = np.array([rc * math.cos(ph), rc * math.sin(ph), zc])
        if any(np.sum((c - c2) ** 2) < (r + r2 + margin) ** 2 for c2, r2 in orbs_in.get(vol, [])):
            continue
        orbs_in.setdefault(vol, []).append((c, r))
        solids.append(Solid(ORB, (r,)))
        places.append(Placement(vol, len(solids) - 1, mi["lead"], tuple(float(x) for x in c)))
        placed += 1
    return Scene("barrel", mats, solids, places, VoxelSpec(mode="smart"))


def nested_barrel_scene(seed: int = CONFIG_SEEDS[3][0], n_shells: int = 30, n_phi: int = 64, n_orbs: int = 2000,
                        r_in: float = 50.0, r_out: float = 1500.0, half_len: float = 1500.0) -> Scene:
    """The barrel with deep nesting: full tube k (radius R_k = r_out - k dr, half-length half_len - k mm) is placed
    inside full tube k - 1; inside tube k the annulus [R_{k+1}, R_k] is tiled by n_phi φ segments (the innermost
    annulus down to r_in), and orbs sit in the segments of all but the innermost shell.  Depth: world, 30 tubes,
    a segment, an orb = 33 levels at most, 32 used (no orbs in the innermost shell)."""
    rng = np.random.default_rng(seed)
    mats, mi = _std_materials()
    solids = [Solid(BOX, (2000.0, 2000.0, 2000.0))]
    places = [Placement(-1, 0, mi["vacuum"], (0.0, 0.0, 0.0))]
    dr = (r_out - r_in) / n_shells
    dphi = TWO_PI / n_phi
    seg_index = []   # (segment volume, rmin, rmax, hz, shell)
    mother = 0
    for k in range(n_shells):
        R, Rin, hz = r_out - k * dr, r_out - (k + 1) * dr, half_len - k
        solids.append(Solid(TUBE, (0.0, R, hz, 0.0, TWO_PI)))
        places.append(Placement(mother, len(solids) - 1, mi["vacuum"], (0.0, 0.0, 0.0)))
        tube = len(places) - 1
        mat = mi["scint"] if k % 2 == 0 else mi["al"]
        solids.append(Solid(TUBE, (Rin, R, hz, 0.0, dphi)))
        seg_solid = len(solids) - 1
        for j in range(n_phi):
            th = j * dphi
            places.append(Placement(tube, seg_solid, mat, (0.0, 0.0, 0.0), (math.cos(th), math.sin(th))))
            if k < n_shells - 1:
                seg_index.append((len(places) - 1, Rin, R, hz))
        mother = tube
    orbs_in = {}
    margin = 0.5
    placed, tries = 0, 0
    while placed < n_orbs:
        tries += 1
        if tries > 100 * n_orbs:
            raise RuntimeError("could not place orbs")
        vol, rmin, rmax, hz = seg_index[int(rng.integers(len(seg_index)))]
        r = float(rng.uniform(5.0, 20.0))
        lo, hi = rmin + r + margin, rmax - r - margin
        if lo >= hi:
            continue
        rc = float(rng.uniform(lo, hi))
        half_ang = math.asin(min(1.0, (r + margin) / rc))
        if 2.0 * half_ang >= dphi:
            continue
        ph = float(rng.uniform(half_ang, dphi - half_ang))
        zc = float(rng.uniform(-hz + r + margin, hz - r - margin))
        c = np.array([rc * math.cos(ph), rc * math.sin(ph), zc])
        if any(np.sum((c - c2) ** 2) < (r + r2 + margin) ** 2 for c2, r2 in orbs_in.get(vol, [])):
            continue
        orbs_in.setdefault(vol, []).append((c, r))
        solids.append(Solid(ORB, (r,)))
        places.append(Placement(vol, len(solids) - 1, mi["lead"], tuple(float(x) for x in c)))
        placed += 1
    return Scene("nested_barrel", mats, solids, places, VoxelSpec(mode="smart"))


def barrel_source() -> Source:
    return Source(pos=(0.0, 0.0, 0.0), z_range=(-1500.0, 1500.0), isotropic=True, e_kind="loguniform",
                  e0=0.02, e1=20.0)


def spheres_scene(n_side: int = 20, radius: float = 100.0, pitch: float = 250.0, mu_al_mass: float = 0.06146) -> Scene:
    """Spheres benchmark geometry: aluminium balls on a regular grid in a 5 m vacuum cube.

    mu = rho * mu_Al(1 MeV) with mu_Al = 0.06146 cm^2/g (Sec. 3.4, Eq. 9); energy-independent table.
    """
    rho = 2.699
    mats = [vacuum(), constant_material("al_1MeV", rho, rho * mu_al_mass * 0.1)]
    solids = [Solid(BOX, (2500.0, 2500.0, 2500.0)), Solid(ORB, (radius,))]
    places = [Placement(-1, 0, 0, (0.0, 0.0, 0.0))]
    c0 = -pitch * (n_side - 1) / 2.0
    for i in range(n_side):
        for j in range(n_side):
            for k in range(n_side):
                places.append(Placement(0, 1, 1, (c0 + pitch * i, c0 + pitch * j, c0 + pitch * k)))
    return Scene("spheres", mats, solids, places, VoxelSpec(mode="smart"))


SPHERES_GRID = (400, 250)      # Regular target grid on the +z face (pixels along x, along y)
SPHERES_ENERGY = 1.0           # MeV: every particle of the Spheres benchmark has this energy


def spheres_rays(kind: str, n: int = 100_000, seed: int = 0x7A0C0005, half: float = 2500.0):
    """Inputs (x0, omega, Y) of the Spheres benchmark (Sec. 3.4, Algorithm 2 phases 2-3), all rays from the
    centre of the geometry.  'regular': towards the centres of a 400 x 250 pixel grid on the +z face,
    ray i*250 + j aims at x = -half + (i + 1/2) 2 half / 400, y = -half + (j + 1/2) 2 half / 250 (column-major
    pixel order), Y = 1 for every ray.  'random': directions uniform on the unit sphere, Y ~ Exp(1).
    Returns pos (n, 3), dir (n, 3), Y (n,) as float64 arrays."""
    if kind == "regular":
        nx, ny = SPHERES_GRID
        if n != nx * ny:
            raise ValueError("the regular grid has 400 x 250 rays")
        i, j = np.meshgrid(np.arange(nx), np.arange(ny), indexing="ij")
        tgt = np.stack([-half + (i.ravel() + 0.5) * (2 * half / nx), -half + (j.ravel() + 0.5) * (2 * half / ny),
                        np.full(n, half)], axis=1)
        d = tgt / np.linalg.norm(tgt, axis=1)[:, None]
        Y = np.ones(n)
    elif kind == "random":
        rng = np.random.default_rng(seed)
        d = rng.normal(size=(n, 3))
        d /= np.linalg.norm(d, axis=1)[:, None]
        Y = rng.exponential(1.0, size=n)
    else:
        raise ValueError(kind)
    return np.zeros((n, 3)), np.ascontiguousarray(d), Y


def slab_scene(thickness: float, material: Material, half_xy: float = 1.0e5) -> Scene:
    """One slab (z in [0, thickness]) of ``material`` inside a vacuum world: the Eq. 2-3 attenuation setup."""
    mats = [vacuum(material.energies), material]
    solids = [Solid(BOX, (half_xy * 2, half_xy * 2, 10.0 * thickness + 100.0)),
              Solid(BOX, (half_xy, half_xy, thickness / 2.0))]
    places = [Placement(-1, 0, 0, (0.0, 0.0, 0.0)), Placement(0, 1, 1, (0.0, 0.0, thickness / 2.0))]
    return Scene("slab", mats, solids, places, VoxelSpec(mode="none"))


def layered_scene(thicknesses: list, materials: list, half_xy: float = 1.0e5) -> Scene:
    """Touching slabs stacked along +z from z = 0: a piecewise-constant μ along the axis (Eq. 8)."""
    e = materials[0].energies
    mats = [vacuum(e)] + list(materials)
    total = float(sum(thicknesses))
    solids = [Solid(BOX, (half_xy * 2, half_xy * 2, 2.0 * total + 100.0))]
    places = [Placement(-1, 0, 0, (0.0, 0.0, 0.0))]
    z = 0.0
    for k, th in enumerate(thicknesses):
        solids.append(Solid(BOX, (half_xy, half_xy, th / 2.0)))
        places.append(Placement(0, len(solids) - 1, 1 + k, (0.0, 0.0, z + th / 2.0)))
        z += th
    return Scene("layered", mats, solids, places, VoxelSpec(mode="none"))


# ---------------------------------------------------------------- logical volumes (reuse)

@dataclasses.dataclass
class LogicalDaughter:
    lv: int                   # index of the daughter logical volume
    t: tuple                  # translation in the logical mother's frame
    rot: tuple = (1.0, 0.0)


@dataclasses.dataclass
class LogicalVolume:
    solid: int
    material: int
    daughters: list


@dataclasses.dataclass
class LogicalPlacement:
    mother: int               # physical volume of the base scene (or an earlier expansion)
    lv: int
    t: tuple
    rot: tuple = (1.0, 0.0)


def expand_logical(base: Scene, logicals: list, placements: list):
    """The flat scene of a base scene plus placed logical volumes: each placement expands its
    logical volume's subtree depth first (the volume, then its daughters' subtrees in order).
    Returns (scene, touchable) where touchable[v] = (logical volume, copy number) of volume v
    ((-1, -1) for the base placements)."""
    places = list(base.placements)
    touch = [(-1, -1)] * len(places)

    def expand(mother, lv, copy, t, rot):
        L = logicals[lv]
        places.append(Placement(mother, L.solid, L.material, tuple(t), tuple(rot)))
        touch.append((lv, copy))
        me = len(places) - 1
        for k, d in enumerate(L.daughters):
            expand(me, d.lv, k, d.t, d.rot)

    for p in placements:
        expand(p.mother, p.lv, 0, p.t, p.rot)
    return Scene(base.name + "_expanded", base.materials, base.solids, places, base.voxel), touch


def modular_calorimeter(n_mod: int = 2, n_tower: int = 4, n_pairs: int = 10):
    """A sampling calorimeter built from reused logical volumes: modules of n_tower x n_tower towers, each
    tower a stack of n_pairs (lead 5 mm + scintillator 10 mm) cells, n_mod x n_mod modules in a vacuum
    world.  Depth: world, module, tower, pair, cell.  Returns (base scene, logical volumes, placements)."""
    mats, mi = _std_materials()
    cell_xy, pb, sc = 20.0, 2.5, 5.0
    pair_hz = pb + sc
    tower_hz = n_pairs * pair_hz
    mod_half = n_tower * cell_xy
    solids = [Solid(BOX, (1000.0, 1000.0, 1000.0)),
              Solid(BOX, (cell_xy, cell_xy, pb)), Solid(BOX, (cell_xy, cell_xy, sc)),
              Solid(BOX, (cell_xy, cell_xy, pair_hz)), Solid(BOX, (cell_xy, cell_xy, tower_hz)),
              Solid(BOX, (mod_half, mod_half, tower_hz))]
    base = Scene("modular_calorimeter", mats, solids, [Placement(-1, 0, mi["vacuum"], (0.0, 0.0, 0.0))],
                 VoxelSpec(mode="smart"))
    lv_pb = LogicalVolume(1, mi["lead"], [])
    lv_sc = LogicalVolume(2, mi["scint"], [])
    lv_pair = LogicalVolume(3, mi["vacuum"], [LogicalDaughter(0, (0.0, 0.0, -sc)), LogicalDaughter(1, (0.0, 0.0, pb))])
    lv_tower = LogicalVolume(4, mi["vacuum"], [LogicalDaughter(2, (0.0, 0.0, -tower_hz + pair_hz * (2 * k + 1)))
                                               for k in range(n_pairs)])
    lv_mod = LogicalVolume(5, mi["vacuum"], [LogicalDaughter(3, (-mod_half + cell_xy * (2 * i + 1),
                                                                 -mod_half + cell_xy * (2 * j + 1), 0.0))
                                             for i in range(n_tower) for j in range(n_tower)])
    logicals = [lv_pb, lv_sc, lv_pair, lv_tower, lv_mod]
    placements = [LogicalPlacement(0, 4, (-n_mod * mod_half + mod_half * (2 * i + 1),
                                         -n_mod * mod_half + mod_half * (2 * j + 1), tower_hz))
                  for i in range(n_mod) for j in range(n_mod)]
    return base, logicals, placements


# Query workloads (locate / compute_step benchmarks): points uniform in a box that holds the detector
# and some of the world around it, directions isotropic.
QUERY_BOXES = {"calorimeter": ((-600.0, -600.0, -50.0), (600.0, 600.0, 425.0)),
               "barrel": ((-1600.0, -1600.0, -1600.0), (1600.0, 1600.0, 1600.0))}


def query_points(scene: str, n: int, seed: int):
    """(pos, dir) as (3, n) float64 arrays (structure of arrays): pos uniform in QUERY_BOXES[scene], dir
    isotropic (normalised Gaussian triples)."""
    lo, hi = (np.asarray(b) for b in QUERY_BOXES[scene])
    rng = np.random.default_rng(seed)
    p = lo[:, None] + (hi - lo)[:, None] * rng.random((3, n))
    v = rng.standard_normal((3, n))
    v /= np.sqrt((v * v).sum(axis=0))[None, :]
    return np.ascontiguousarray(p), np.ascontiguousarray(v)


def reversed_stack_scene(n_plates: int = 24, pitch: float = 40.0) -> Scene:
    """A 200 x 200 x 1000 mm vacuum box holding n_plates aluminium-like plates (80 x 80 x 5 mm) stacked along z,
    placed (hence numbered) from the top down, without voxels: one candidate list in id order, which puts the
    plates farthest along an upward ray first -- the order a learned proposal can improve on."""
    mats, mi = _std_materials()
    solids = [Solid(BOX, (100.0, 100.0, 500.0)), Solid(BOX, (40.0, 40.0, 2.5))]
    places = [Placement(-1, 0, mi["vacuum"], (0.0, 0.0, 0.0))]
    for k in range(n_plates):
        places.append(Placement(0, 1, mi["al"], (0.0, 0.0, 450.0 - pitch * k)))
    return Scene("reversed_stack", mats, solids, places, VoxelSpec(mode="none"))


def reversed_stack_source() -> Source:
    return Source(pos=(0.0, 0.0, -495.0), spot_sigma=15.0, isotropic=False, direction=(0.0, 0.0, 1.0),
                  e_kind="loguniform", e0=0.1, e1=3.0)
