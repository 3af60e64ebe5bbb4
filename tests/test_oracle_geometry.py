"""Pins for the geometry side: the paper's Tables 0-3 (§5), the reference medium (§5),
the sphere-radius reading, and the integer voxelization rule of coated spheres (§2)."""
import math

import numpy as np
import pytest

from conftest import read_golden
from oracle import em as om
from paper_1504_07499_gb300 import inputs as I


def test_table0_coating_fraction():
    for layer, f in read_golden("table0_coating_fraction.txt"):
        assert abs(om.coating_fraction(layer, 0.3) - f) <= 0.00051


def test_tables1_3_coating_voxels_pin_radius_reading():
    rows = read_golden("tables1_3_coating_voxels.txt")
    assert len(rows) == 20
    for row in rows:
        res, layer, vals = int(row[0]), row[1], row[2:]
        for n, printed in zip(range(30, 101, 10), vals):
            got = om.coating_voxels(layer, res, n)
            assert abs(got - printed) <= 0.0051, (res, layer, n, got, printed)
            # the input generator's radius is the same reading (n in the denominator)
            assert abs(layer * res * I.sphere_radius(n, 0.3) - got) < 1e-12
            # n_sp in the numerator, as printed under the tables, misses them by far
            wrong = layer * res * (3 * 0.3 * n / (4 * math.pi)) ** (1 / 3)
            assert abs(wrong - printed) > 0.05


def test_reference_medium_value():
    (km, ki, kc, L0abs, cmin, cmax), = read_golden("reference_medium.txt")
    assert abs(om.reference_k0((km, ki, kc)) - L0abs) < 1e-12
    assert abs(4 * math.sqrt(5) - L0abs) < 1e-12
    ks = sorted((km, ki, kc))
    assert abs(ks[1] / ks[0] - cmin) < 1e-12 and abs(ks[2] / ks[0] - cmax) < 1e-9


def _float_phase(spheres, layer, N):
    """Floating-point evaluation of the same rule, for voxels away from the boundary."""
    v = (np.arange(N) + 0.5) / N
    incl = np.zeros((N, N, N), bool)
    coat = np.zeros((N, N, N), bool)
    near = np.zeros((N, N, N), bool)
    for cx, cy, cz, r in spheres:
        d = []
        for c in (cx, cy, cz):
            dd = np.abs(v - c)
            dd = np.minimum(dd, 1 - dd)
            d.append(dd * dd)
        d2 = d[2][:, None, None] + d[1][None, :, None] + d[0][None, None, :]
        dist = np.sqrt(d2)
        ri = (1 - layer) * r
        incl |= dist < ri
        coat |= dist < r
        near |= (np.abs(dist - ri) < 1e-6) | (np.abs(dist - r) < 1e-6)
    ph = np.zeros((N, N, N), np.uint8)
    ph[coat] = 2
    ph[incl] = 1
    return ph, near


@pytest.mark.parametrize("seed,N,n,f,layer", [(1, 24, 10, 0.3, 0.3), (2, 32, 30, 0.2, 0.1), (3, 20, 5, 0.35, 0.6)])
def test_voxelize_matches_float_rule_off_boundary(seed, N, n, f, layer):
    sl = I.generate_spheres(seed, n, f)
    ph = om.voxelize(sl.spheres, layer, N)
    ref, near = _float_phase(sl.spheres, layer, N)
    assert (ph[~near] == ref[~near]).all()


def test_centred_sphere_has_cubic_symmetry_and_counts():
    N = 32
    ph = om.voxelize(I.centred_sphere(0.25), 0.25, N)
    for axes in [(0, 1, 2), (1, 0, 2), (2, 1, 0), (0, 2, 1)]:
        assert (np.transpose(ph, axes) == ph).all()
    assert (np.flip(ph, 0) == ph).all() and (np.flip(ph, 2) == ph).all()
    counts = np.bincount(ph.reshape(-1), minlength=3)
    # continuum volumes of core (r = 6 voxels) and shell (6..8 voxels)
    v_core = 4 / 3 * math.pi * 6 ** 3
    v_shell = 4 / 3 * math.pi * (8 ** 3 - 6 ** 3)
    assert abs(counts[1] - v_core) / v_core < 0.06
    assert abs(counts[2] - v_shell) / v_shell < 0.06


def test_voxel_counts_converge_to_sphere_volume():
    sph = np.array([[0.31, 0.47, 0.62, 0.2]])
    errs = []
    for N in (16, 32, 64):
        ph = om.voxelize(sph, 0.4, N)
        frac_core = (ph == 1).mean()
        errs.append(abs(frac_core - 4 / 3 * math.pi * (0.6 * 0.2) ** 3))
    assert errs[2] < errs[0] and errs[2] < 2e-4


def test_periodic_wrap_equals_roll():
    N = 16
    a = om.voxelize(np.array([[0.5, 0.5, 0.5, 0.3]]), 0.3, N)
    b = om.voxelize(np.array([[0.0, 0.0, 1.0, 0.3]]), 0.3, N)   # same sphere shifted by N/2
    assert (np.roll(a, (N // 2, N // 2, N // 2), axis=(0, 1, 2)) == b).all()


def test_quantization_rule_values():
    q, S = om.quantize_spheres(np.array([[0.5, 0.25, 1.0 - 2 ** -30, 0.125]]), 0.5, 8)
    assert S == 2 * 8 * 4096
    cx, cy, cz, ro2, ri2 = q[0]
    assert cx == S // 2 and cy == S // 4 and cz == 0      # wraps to 0
    assert ro2 == (S // 8) ** 2 and ri2 == (S // 16) ** 2


def test_thin_coating_is_lost_when_below_a_voxel():
    # §5: coatings thinner than a voxel can be missed by the voxelization
    N = 32
    thin = om.voxelize(I.centred_sphere(0.25), 0.01, N)   # 0.08 voxel thick
    assert (thin == 2).sum() < 0.2 * (om.voxelize(I.centred_sphere(0.25), 0.25, N) == 2).sum()
