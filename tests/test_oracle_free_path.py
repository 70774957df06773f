"""The oracle's Algorithm 1 free path on the Spheres benchmark geometry (Sec. 3.4), pinned by the
closed-form chord of a ray through a ball centre, and its batch form against the per-ray form."""
import math

import numpy as np

import oracle
import synth

MU_AL = 2.699 * 0.06146 * 0.1   # 1/mm: rho x mass attenuation coefficient of Al at 1 MeV (Eq. 9)


def test_ray_through_ball_centre_closed_form():
    sc = synth.scenes.spheres_scene()
    og = oracle.Geometry(sc)
    c = np.array([125.0, 125.0, 125.0])       # nearest ball centre to the origin
    d = c / np.linalg.norm(c)
    entry = np.linalg.norm(c) - 100.0
    for Y in (0.25, 1.0, 3.0):
        T, steps = og.free_path(np.zeros(3), d, 1.0, Y)
        assert math.isclose(T, entry + Y / MU_AL, rel_tol=0, abs_tol=1e-9)
        assert steps == 2                    # vacuum to the ball, then inside it
    # Y beyond the chord's optical depth: the ray leaves the ball and goes on to the next ball on the diagonal
    Ychord = 200.0 * MU_AL
    T, steps = og.free_path(np.zeros(3), d, 1.0, Ychord + 0.5)
    c2 = c + 250.0
    entry2 = np.linalg.norm(c2) - 100.0
    assert math.isclose(T, entry2 + 0.5 / MU_AL, rel_tol=0, abs_tol=1e-9)
    # a ray between the balls along an axis through no ball escapes
    T, _ = og.free_path(np.zeros(3), np.array([1.0, 0.0, 0.0]), 1.0, 1.0)
    assert math.isinf(T)


def test_batch_equals_single():
    sc = synth.scenes.spheres_scene()
    og = oracle.Geometry(sc)
    p, v, Y = synth.scenes.spheres_rays("random", n=300, seed=9)
    T, ns, used = og.free_path_many(p, v, 1.0, Y)
    for i in range(300):
        t1, s1 = og.free_path(p[i], v[i], 1.0, Y[i])
        assert (t1 == T[i]) or (math.isinf(t1) and math.isinf(T[i]))
        assert s1 == ns[i]
    assert used >= 1


def test_regular_rays_aim_at_pixel_centres():
    p, v, Y = synth.scenes.spheres_rays("regular")
    assert p.shape == (100_000, 3) and np.all(Y == 1.0) and np.all(p == 0.0)
    # ray i*250 + j hits the +z face at the centre of pixel (i, j)
    for i, j in ((0, 0), (399, 249), (123, 45)):
        r = i * 250 + j
        hit = v[r] * (2500.0 / v[r, 2])
        assert np.allclose(hit[:2], [-2500 + (i + 0.5) * 12.5, -2500 + (j + 0.5) * 20.0], atol=1e-9)
