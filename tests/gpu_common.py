"""Shared helpers of the GPU parity tests: one library context per session,
seeded query generation, and the scene workloads used in the parity cases."""
import math

import numpy as np

import oracle
import synth
from synth.scenes import Scene, Solid, Placement, VoxelSpec, BOX, TUBE, ORB, CONE
from synth.materials import toy_materials


def world_half(scene):
    return np.array(scene.solids[scene.placements[0].solid].params[:3]) if scene.solids[0].kind == BOX else None


def mixed_scene(seed=5, n=120, half=300.0, voxel=None):
    rng = np.random.default_rng(seed)
    m = toy_materials()
    dsol, dpl = synth.scenes.random_world(rng, n, world_half=half, fill=0.15)
    solids = [Solid(BOX, (half, half, half))] + dsol
    places = [Placement(-1, 0, 0, (0, 0, 0))] + [Placement(0, i + 1, 1 + i % 3, t, rot) for i, (t, rot) in enumerate(dpl)]
    return Scene("mixed", [m["water"], m["lead"], m["scint"], m["al"]], solids, places, voxel or VoxelSpec(mode="smart"))


def nested_scene():
    """World + 7 nested levels (box > tube > orb > box > ...), each holder rotated about z, with a small
    sibling beside every holder and a wide tube segment beside the tube holders: the maximum depth."""
    m = toy_materials()
    mats = [m["water"], m["lead"], m["scint"], m["al"]]
    S = 400.0
    solids = [Solid(BOX, (S, S, S))]
    places = [Placement(-1, 0, 0, (0, 0, 0))]
    mother, mkind, size = 0, BOX, S
    for lev in range(7):
        th = 0.3 * (lev + 1)
        rot = (math.cos(th), math.sin(th))
        if mkind == BOX:        # tube holder in a box mother, sibling boxes in the corners
            hold = Solid(TUBE, (0.0, 0.6 * size, 0.6 * size, 0.0, 2 * math.pi))
            sib = [(Solid(BOX, (0.05 * size,) * 3), (0.85 * size, 0.85 * size, 0.0)),
                   (Solid(TUBE, (0.02 * size, 0.1 * size, 0.1 * size, 0.3, 4.5)), (-0.8 * size, -0.8 * size, 0.0))]
            nkind, nsize = TUBE, 0.6 * size
        elif mkind == TUBE:     # orb holder in a tube mother, sibling on the axis
            hold = Solid(ORB, (0.55 * size,))
            sib = [(Solid(BOX, (0.05 * size,) * 3), (0.0, 0.0, 0.8 * size))]
            nkind, nsize = ORB, 0.55 * size
        else:                   # box holder in an orb mother
            hold = Solid(BOX, (0.5 * size,) * 3)
            sib = [(Solid(BOX, (0.05 * size,) * 3), (0.0, 0.0, 0.75 * size))]
            nkind, nsize = BOX, 0.5 * size
        solids.append(hold)
        places.append(Placement(mother, len(solids) - 1, (lev + 1) % 4, (0.0, 0.0, 0.0), rot))
        holder = len(places) - 1
        for k, (so, t) in enumerate(sib):
            solids.append(so)
            places.append(Placement(mother, len(solids) - 1, (lev + 2 + k) % 4, t, (math.cos(0.7 * k), math.sin(0.7 * k))))
        mother, mkind, size = holder, nkind, nsize
    return Scene("nested", mats, solids, places, VoxelSpec(mode="smart"))


def segments_scene():
    """Tube segments (narrow, wide, exactly pi; with and without bore) at a systematic grid of start
    angles and rotations, including combinations whose rotated phi range runs past 4 pi."""
    m = toy_materials()
    solids = [Solid(BOX, (400.0, 400.0, 400.0))]
    places = [Placement(-1, 0, 0, (0, 0, 0))]
    k = 0
    for i, sphi in enumerate(np.linspace(0.0, 2 * math.pi, 6, endpoint=False) + 0.1):
        for j, dphi in enumerate((0.4, 2.0, math.pi, 4.0, 5.36, 6.0)):
            th = (k * 0.7361) % (2 * math.pi) - math.pi
            rmin = 0.0 if (i + j) % 2 else 8.0
            solids.append(Solid(TUBE, (rmin, 17.0, 12.0, float(sphi), float(dphi))))
            cx, cy, cz = -330.0 + 60.0 * i, -330.0 + 60.0 * j, 30.0 * ((k % 5) - 2)
            places.append(Placement(0, len(solids) - 1, 1 + k % 3, (cx, cy, cz), (math.cos(th), math.sin(th))))
            k += 1
    return Scene("segments", [m["water"], m["lead"], m["scint"], m["al"]], solids, places, VoxelSpec(mode="smart"))


def random_queries(og, scene, n, seed, box_half=None, surface_frac=0.5, aim_frac=0.0):
    """Points inside the world (half of them moved onto a boundary along a random ray) with
    random unit directions, a fraction `aim_frac` of them aimed near a random daughter.
    Surface points are produced by the oracle's own compute_step."""
    rng = np.random.default_rng(seed)
    h = np.asarray(box_half if box_half is not None else world_half(scene) * 0.98)
    p = rng.uniform(-h, h, size=(n, 3))
    v = rng.normal(size=(n, 3))
    if aim_frac > 0 and scene.n_volumes > 1:
        k = rng.uniform(size=n) < aim_frac
        tgt = np.array([scene.placements[int(i)].t for i in rng.integers(1, scene.n_volumes, n)])
        tgt += rng.uniform(-10.0, 10.0, size=(n, 3))
        v[k] = tgt[k] - p[k]
    v /= np.linalg.norm(v, axis=1)[:, None]
    k = int(n * surface_frac)
    if k:
        d, pa = og.locate_many(p[:k], v[:k])
        ok = d > 0
        s, lim, _ = og.compute_step_many(p[:k][ok], v[:k][ok], d[ok], pa[ok])
        idx = np.nonzero(ok)[0]
        p[idx] = p[idx] + s[:, None] * v[idx]
        # half of the surface points get a fresh random direction
        w = rng.normal(size=(idx.size, 3))
        w /= np.linalg.norm(w, axis=1)[:, None]
        flip = rng.uniform(size=idx.size) < 0.5
        v[idx[flip]] = w[flip]
    return p, v


def to_soa(a, torch, device="cuda"):
    return torch.tensor(np.ascontiguousarray(a.T), dtype=torch.float64, device=device)


def cones_scene(seed=21, n_random=40, half=500.0):
    """Cones as leaves and as mothers: a solid cone holding a box, an orb and a small hollow cone; a hollow
    cone with orbs in its wall; and seeded random cones (solid and hollow, widening and narrowing, rotated
    about z) kept apart by their bounding spheres, among a few boxes."""
    rng = np.random.default_rng(seed)
    m = toy_materials()
    mats = [m["water"], m["lead"], m["scint"], m["al"]]
    solids = [Solid(BOX, (half, half, half)),
              Solid(CONE, (0.0, 200.0, 0.0, 120.0, 150.0)),      # 1 solid cone mother
              Solid(BOX, (20.0, 20.0, 20.0)),                    # 2
              Solid(ORB, (30.0,)),                               # 3
              Solid(CONE, (10.0, 40.0, 15.0, 30.0, 40.0)),       # 4 small hollow cone
              Solid(CONE, (30.0, 80.0, 50.0, 120.0, 100.0)),     # 5 hollow cone mother
              Solid(ORB, (15.0,))]                               # 6
    places = [Placement(-1, 0, 0, (0.0, 0.0, 0.0)),
              Placement(0, 1, 1, (200.0, 200.0, 0.0)),
              Placement(1, 2, 2, (0.0, 0.0, -50.0)),
              Placement(1, 3, 3, (0.0, 0.0, 60.0)),
              Placement(1, 4, 2, (60.0, 0.0, -40.0), (math.cos(0.4), math.sin(0.4))),
              Placement(0, 5, 3, (-250.0, -100.0, 100.0), (math.cos(1.1), math.sin(1.1)))]
    for k in range(6):
        a = k * math.pi / 3
        places.append(Placement(5, 6, 1, (70.0 * math.cos(a), 70.0 * math.sin(a), 0.0)))
    centres = [np.array([200.0, 200.0, 0.0]), np.array([-250.0, -100.0, 100.0])]
    radii = [math.hypot(200.0, 150.0), math.hypot(120.0, 100.0)]
    placed = tries = 0
    while placed < n_random and tries < 100000:
        tries += 1
        if placed % 4 == 3:
            so = Solid(BOX, tuple(float(x) for x in rng.uniform(10.0, 40.0, 3)))
            r = float(np.linalg.norm(so.params))
        else:
            hz = float(rng.uniform(10.0, 40.0))
            rmax1, rmax2 = (float(x) for x in rng.uniform(8.0, 45.0, 2))
            if rng.uniform() < 0.5:
                rmin1, rmin2 = 0.0, 0.0
            else:
                rmin1, rmin2 = float(rng.uniform(0.2, 0.7) * rmax1), float(rng.uniform(0.2, 0.7) * rmax2)
            so = Solid(CONE, (rmin1, rmax1, rmin2, rmax2, hz))
            r = math.hypot(max(rmax1, rmax2), hz)
        c = rng.uniform(-half + r + 1.0, half - r - 1.0, 3)
        if any(np.linalg.norm(c - c2) < r + r2 + 1.0 for c2, r2 in zip(centres, radii)):
            continue
        centres.append(c)
        radii.append(r)
        solids.append(so)
        th = float(rng.uniform(0.0, 2 * math.pi))
        places.append(Placement(0, len(solids) - 1, 1 + placed % 3, tuple(float(x) for x in c), (math.cos(th), math.sin(th))))
        placed += 1
    return Scene("cones", mats, solids, places, VoxelSpec(mode="smart"))
