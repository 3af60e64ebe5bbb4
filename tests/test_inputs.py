"""Checks of the seeded input generators (§2: up to 100 identical non-overlapping
spheres at up to 40 % volume fraction)."""
import math

import numpy as np
import pytest

from paper_1504_07499_gb300 import inputs as I


def test_splitmix64_published_vector():
    # first outputs of SplitMix64 seeded with 0 (reference implementation by S. Vigna)
    got = [int(v) for v in I.SplitMix64(0).take(3)]
    assert got == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]


def test_uniform_range_and_determinism():
    a = I.SplitMix64(5).uniform(10000)
    b = I.SplitMix64(5).uniform(10000)
    assert (a == b).all() and a.min() >= 0 and a.max() < 1
    assert abs(a.mean() - 0.5) < 0.01


def _check_spheres(sl, n, f):
    c = sl.spheres[:, :3]
    r = sl.spheres[:, 3]
    assert len(c) == n and np.all(r == r[0])
    assert abs(n * 4 / 3 * math.pi * r[0] ** 3 - f) < 1e-12
    d = np.abs(c[:, None] - c[None])
    d = np.minimum(d, 1 - d)
    d2 = (d * d).sum(-1)
    np.fill_diagonal(d2, np.inf)
    assert d2.min() > (2 * r[0]) ** 2
    assert (c >= 0).all() and (c < 1).all()


@pytest.mark.parametrize("seed,n,f", [(1000, 30, 0.20), (4001, 10, 0.35), (7, 100, 0.30)])
def test_rsa_non_overlapping(seed, n, f):
    sl = I.generate_spheres(seed, n, f)
    _check_spheres(sl, n, f)
    again = I.generate_spheres(seed, n, f)
    assert (again.spheres == sl.spheres).all()


@pytest.mark.slow
def test_forty_percent_uses_fallback():
    sl = I.generate_spheres(3000, 100, 0.40)
    _check_spheres(sl, 100, 0.40)
    assert sl.generator == "rsa+grow"


def test_batch_recipe_ranges():
    rec = I.batch_recipe()
    assert len(rec) == 64
    assert sorted({r["N"] for r in rec}) == [64, 96, 128]
    assert sum(r["N"] == 128 for r in rec) == 16
    for r in rec:
        assert 10 <= r["n"] <= 100 and 0.10 <= r["f"] <= 0.40 and 0.1 <= r["layer"] <= 0.5


def test_laminate_and_random_grids():
    g = I.laminate_grid(8, 3, axis=0)
    assert (g[:, :, :3] == 2).all() and (g[:, :, 3:] == 0).all()
    r = I.random_phase_grid(1, 16, probs=(0.5, 0.25, 0.25))
    frac = np.bincount(r.reshape(-1), minlength=3) / r.size
    assert np.abs(frac - [0.5, 0.25, 0.25]).max() < 0.03
