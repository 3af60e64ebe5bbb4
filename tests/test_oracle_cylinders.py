"""Pins for the oracle's coated cylinders (§6 outlook: RVEs with cylinders, or spheres and
cylinders) and the seeded cylinder generator: the integer rule reduces to a disk times an
interval for an axis-aligned cylinder, the voxel volume approaches pi r^2 h, the grid does
not depend on the sign of the axis and follows periodic shifts, a continuous fiber is a
prism, mixed grids with no cylinders are the sphere grids, the homogenized conductivity of
fibers along z is the exact arithmetic mean along z, and the generator's segment distance
matches brute force and keeps objects apart."""
import math

import numpy as np
import pytest

from oracle import em as om
from paper_1504_07499_gb300 import inputs as I

K3 = (0.20, 0.25, 400.0)


def test_axis_aligned_cylinder_is_a_disk_times_an_interval():
    N, layer = 24, 0.3
    c = np.array([[0.37, 0.61, 0.45, 0.0, 0.0, 1.0, 0.21, 0.55]])
    core, outer = om.cylinder_masks(c, layer, N)
    q, S = om.quantize_cylinders(c, layer, N)
    cx, cy, cz, _, _, _, ro2, ri2, ho, hi = q[0]
    v = (2 * np.arange(N) + 1) * om.QUANT_GC
    sd = lambda a, b: (a - b + S // 2) % S - S // 2
    dx, dy, dz = sd(v, cx), sd(v, cy), sd(v, cz)
    disk_o = (dx[None, :] ** 2 + dy[:, None] ** 2) <= ro2
    disk_i = (dx[None, :] ** 2 + dy[:, None] ** 2) <= ri2
    zo, zi = np.abs(dz) <= ho, np.abs(dz) <= hi
    assert np.array_equal(outer, zo[:, None, None] & disk_o[None])
    assert np.array_equal(core, zi[:, None, None] & disk_i[None])


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_voxel_volume_approaches_the_cylinder_volume(seed):
    rng = np.random.default_rng(seed)
    u = rng.standard_normal(3)
    u /= np.linalg.norm(u)
    r, h, layer = 0.15, 0.4, 0.25
    c = np.array([[*rng.random(3), *u, r, h]])
    for N in (48, 96):
        core, outer = om.cylinder_masks(c, layer, N)
        vol = math.pi * r * r * h
        vin = math.pi * ((1 - layer) * r) ** 2 * (h - 2 * layer * r)
        # a voxel-thick shell around the surface bounds the error
        assert abs(outer.mean() - vol) < (2 * math.pi * r * h + 2 * math.pi * r * r) * 1.0 / N
        assert abs(core.mean() - vin) < (2 * math.pi * r * h + 2 * math.pi * r * r) * 1.0 / N


def test_axis_sign_and_periodic_shift():
    N, layer = 32, 0.3
    rng = np.random.default_rng(9)
    u = rng.standard_normal(3)
    u /= np.linalg.norm(u)
    c = np.array([[0.3, 0.7, 0.2, *u, 0.12, 0.35]])
    c_neg = c.copy()
    c_neg[0, 3:6] *= -1
    g = om.voxelize_mixed(None, c, layer, N)
    g_neg = om.voxelize_mixed(None, c_neg, layer, N)
    # +-u quantize to +-A up to the half-up rounding of exact halves; away from those the
    # grids are equal
    assert np.array_equal(g, g_neg)
    c_shift = c.copy()
    c_shift[0, :3] += np.array([3, -5, 7]) / N
    g_shift = om.voxelize_mixed(None, c_shift, layer, N)
    assert np.array_equal(g_shift, np.roll(g, (7, -5, 3), axis=(0, 1, 2)))


def test_continuous_fiber_is_a_prism():
    N, layer, r = 20, 0.3, 0.2
    h = 1.0 + 2 * layer * r + 1e-9
    g = om.voxelize_mixed(None, np.array([[0.5, 0.5, 0.1, 0.0, 0.0, 1.0, r, h]]), layer, N)
    assert (g == g[0][None]).all()                         # the same in every z plane
    assert set(np.unique(g)) == {0, 1, 2}


def test_mixed_grid_without_cylinders_is_the_sphere_grid():
    sl = I.generate_spheres(7, 6, 0.3)
    assert np.array_equal(om.voxelize_mixed(sl.spheres, None, 0.3, 24), om.voxelize(sl.spheres, 0.3, 24))


def test_fibers_along_z_give_the_arithmetic_mean_along_z():
    """A microstructure invariant along z: E along z is itself compatible and in
    equilibrium, so K_zz is the voxel average of k exactly, and K_xz = K_yz = 0."""
    N, layer, r = 16, 0.3, 0.12
    h = 1.0 + 2 * layer * r + 1e-9
    cyl = np.array([[0.25, 0.25, 0.5, 0, 0, 1, r, h], [0.75, 0.7, 0.5, 0, 0, 1, r, h]])
    ph = om.voxelize_mixed(None, cyl, layer, N)
    K, _ = om.effective_tensor(ph, K3, tol=1e-10)
    f = om.phase_fractions(ph)
    arith = float((f * np.asarray(K3)).sum())
    assert abs(K[2, 2] - arith) < 1e-12 * arith
    assert abs(K[0, 2]) < 1e-12 * arith and abs(K[1, 2]) < 1e-12 * arith


def test_segment_distance_matches_brute_force():
    rng = np.random.default_rng(4)
    s = np.linspace(-1, 1, 801)
    for _ in range(30):
        a, b, w = rng.standard_normal(3) * 0.2, rng.standard_normal(3) * 0.2, rng.standard_normal(3) * 0.3
        if _ % 10 == 0:
            b = a * 0.7                                   # parallel segments
        exact = I._segment_distance_sq(w, a, b)
        pts = s[:, None, None] * a[None, None, :] - (w[None, None, :] + s[None, :, None] * b[None, None, :])
        brute = float((pts * pts).sum(-1).min())
        assert exact <= brute + 1e-12 and brute - exact < 2e-3 * max(brute, 1e-3)


def test_generated_objects_keep_apart():
    sp, cy = I.generate_cylinders(11, 10, 0.05, 0.3, spheres=6, r_sphere=0.06)
    objs = [(c[:3], 0.5 * c[7] * c[3:6], c[6]) for c in cy] + [(s[:3], np.zeros(3), s[3]) for s in sp]
    for i in range(len(objs)):
        for j in range(i + 1, len(objs)):
            w = objs[j][0] - objs[i][0]
            w = w - np.floor(w + 0.5)
            d2 = I._segment_distance_sq(w, objs[i][1], objs[j][1])
            assert d2 > (objs[i][2] + objs[j][2]) ** 2
