"""Seeded synthetic inputs: sphere lists (RSA placement, §2) and phase grids for tests.

This module only *generates inputs*.  It holds none of the homogenization
arithmetic (no voxelization rule, no conductivity map, no Fourier step), so both
the CUDA path and the CPU oracle may draw their inputs from it.

Random numbers come from SplitMix64, a counter-based generator: output ``i`` of
stream ``seed`` is ``mix(seed + (i + 1) * 0x9E3779B97F4A7C15 mod 2**64)`` with the
published finalizer (Steele, Lea & Flood, "Fast splittable pseudorandom number
generators", OOPSLA 2014).  Uniform doubles take the top 53 bits.  Being
counter-based, a block of outputs is computed vectorized and the sequence does not
depend on the platform or on numpy's own generators.

Sphere placement follows §2: up to 100 identical, non-overlapping spheres in the
periodic unit cube, at most 40 % volume fraction, each sphere given by its centre
and its outer radius ``r_s`` (inclusion plus coating).  The radius follows from
the sphere volume fraction ``f`` (coating included, §2) and the count ``n``:
``r_s = (3 f / (4 pi n))**(1/3)`` -- the reading of the voxel-thickness formula
under Tables 1-3 with ``n_sp`` in the denominator, which reproduces the tables.

Plain random sequential adsorption jams near 38 % for hard spheres, so above it
(and whenever the candidate cap runs out) a seeded fallback is used: RSA at a
reduced radius followed by Monte-Carlo displacement sweeps that grow the radius to
its target.  ``generate_spheres`` reports which generator produced the list.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)
_MASK64 = (1 << 64) - 1


class SplitMix64:
    """Counter-based SplitMix64 stream; ``take(k)`` returns the next ``k`` outputs."""

    def __init__(self, seed: int, stream: int = 0):
        # Distinct streams of one seed are separated by a large odd offset.
        self.base = (int(seed) + int(stream) * 0xD1B54A32D192ED03) & _MASK64
        self.counter = 0

    def take(self, k: int) -> np.ndarray:
        idx = np.arange(self.counter + 1, self.counter + 1 + k, dtype=np.uint64)
        self.counter += k
        with np.errstate(over="ignore"):
            z = np.uint64(self.base) + idx * _GAMMA
            z = (z ^ (z >> np.uint64(30))) * _M1
            z = (z ^ (z >> np.uint64(27))) * _M2
            z = z ^ (z >> np.uint64(31))
        return z

    def uniform(self, k: int) -> np.ndarray:
        """``k`` doubles uniform in [0, 1) from the top 53 bits."""
        return (self.take(k) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


def sphere_radius(n: int, f: float) -> float:
    """Outer radius of ``n`` identical spheres filling volume fraction ``f`` of the unit cube."""
    return (3.0 * f / (4.0 * math.pi * n)) ** (1.0 / 3.0)


def _min_image_sq(a: np.ndarray, b: np.ndarray) -> np.ndarray:
    """Squared periodic minimum-image distances between rows of ``a`` (k,3) and ``b`` (m,3).
    Every operation rounds on its own in a fixed order, (dx^2 + dy^2) + dz^2 with
    d = min(|a - b|, 1 - |a - b|), so the value is the same on every platform (and on
    the GPU generator, which follows the same steps)."""
    d = np.abs(a[:, None, :] - b[None, :, :])
    d = np.minimum(d, 1.0 - d)
    return (d[..., 0] * d[..., 0] + d[..., 1] * d[..., 1]) + d[..., 2] * d[..., 2]


def _wrap1(x: np.ndarray) -> np.ndarray:
    """x wrapped into [0, 1): the exact remainder fmod(x, 1), plus 1 (one rounding) where
    it is negative; a zero remainder is +0."""
    m = np.fmod(x, 1.0)
    return np.where(m < 0.0, m + 1.0, m) + 0.0


def _sq(x: float) -> float:
    """x * x (a single rounded product, unlike pow)."""
    return x * x


def rsa(seed: int, n: int, r: float, max_candidates: int = 2_000_000,
        batch: int = 8192, stream: int = 0) -> np.ndarray | None:
    """Sequential RSA: candidates uniform in [0,1)^3 are accepted, in draw order, when
    their periodic distance to every accepted centre exceeds ``2 r``.  Returns the
    (n, 3) centres, or None when ``max_candidates`` draws do not place ``n`` spheres."""
    rng = SplitMix64(seed, stream)
    acc = np.empty((0, 3))
    lim = _sq(2.0 * r)
    used = 0
    while used < max_candidates:
        cand = rng.uniform(3 * batch).reshape(batch, 3)
        used += batch
        ok = np.ones(batch, dtype=bool)
        if len(acc):
            ok &= (_min_image_sq(cand, acc) > lim).all(axis=1)
        start = 0
        while True:
            nz = np.flatnonzero(ok[start:])
            if nz.size == 0:
                break
            i = start + int(nz[0])
            acc = np.vstack([acc, cand[i]])
            if len(acc) == n:
                return acc
            rest = cand[i + 1:]
            ok[i + 1:] &= _min_image_sq(rest, cand[i:i + 1])[:, 0] > lim
            start = i + 1
    return None


def grow_mc(seed: int, centres: np.ndarray, r_target: float, max_sweeps: int = 20000,
            stream: int = 1) -> np.ndarray | None:
    """Monte-Carlo displacement sweeps that let the common radius grow to ``r_target``.

    After every sweep the working radius becomes ``min(r_target, 0.5 * min pair
    distance)``; a move is accepted when the moved centre keeps distance
    ``> 2 r_work`` to all others.  Returns the centres or None if the cap is hit."""
    rng = SplitMix64(seed, stream)
    c = centres.copy()
    n = len(c)
    if n == 1:
        return c
    for _ in range(max_sweeps):
        d2 = _min_image_sq(c, c)
        np.fill_diagonal(d2, np.inf)
        r_work = min(r_target, 0.5 * math.sqrt(d2.min()))
        if r_work >= r_target and d2.min() > _sq(2.0 * r_target):
            return c
        step = max(0.25 * r_target, 1e-3)
        u = rng.uniform(4 * n).reshape(n, 4)
        lim = _sq(2.0 * r_work)
        for i in range(n):
            trial = _wrap1(c[i] + step * (2.0 * u[i, :3] - 1.0))
            others = np.delete(c, i, axis=0)
            if (_min_image_sq(trial[None, :], others)[0] > lim).all():
                c[i] = trial
        # Radius growth happens through r_work on the next sweep.
    return None


@dataclass
class SphereList:
    """Sphere list in unit-cube coordinates: columns cx, cy, cz, r (outer radius)."""
    spheres: np.ndarray
    generator: str
    seed: int
    n: int
    f: float
    extra: dict = field(default_factory=dict)

    @property
    def radius(self) -> float:
        return float(self.spheres[0, 3])


def generate_spheres(seed: int, n: int, f: float, max_candidates: int = 400_000) -> SphereList:
    """Seeded sphere list for ``n`` spheres at volume fraction ``f`` (coating included).

    Plain RSA first; if it cannot place ``n`` spheres within ``max_candidates`` draws
    (RSA jams near 38 %), RSA at 85 % of the radius followed by growth sweeps."""
    if not (1 <= n <= 100) or not (0.0 < f <= 0.4):
        raise ValueError("need 1 <= n <= 100 and 0 < f <= 0.4")
    r = sphere_radius(n, f)
    if r >= 0.5:
        raise ValueError("radius must stay below half the cell")
    gen = "rsa"
    cen = rsa(seed, n, r, max_candidates=max_candidates)
    if cen is None:
        gen = "rsa+grow"
        seed_c = rsa(seed, n, 0.85 * r, max_candidates=max_candidates, stream=2)
        if seed_c is None:
            raise RuntimeError("RSA at reduced radius failed")
        cen = grow_mc(seed, seed_c, r)
        if cen is None:
            raise RuntimeError("growth sweeps did not reach the target radius")
    sph = np.column_stack([cen, np.full(n, r)])
    return SphereList(sph, gen, seed, n, f)


def random_axis(u1: float, u2: float) -> np.ndarray:
    """Unit vector uniform on the sphere from two uniforms (z = 2 u1 - 1, azimuth 2 pi u2)."""
    z = 2.0 * u1 - 1.0
    s = math.sqrt(max(0.0, 1.0 - z * z))
    phi = 2.0 * math.pi * u2
    return np.array([s * math.cos(phi), s * math.sin(phi), z])


def _segment_distance_sq(w: np.ndarray, a: np.ndarray, b: np.ndarray) -> float:
    """Smallest squared distance between the segments s a (s in [-1, 1]) and w + t b
    (t in [-1, 1]): the minimum of the convex quadratic |s a - t b - w|^2 over the square,
    inside it or on one of its four edges."""
    aa, bb, ab = float(a @ a), float(b @ b), float(a @ b)
    aw, bw = float(a @ w), float(b @ w)

    def f(s, t):
        d = s * a - t * b - w
        return float(d @ d)

    def clamp(x):
        return min(1.0, max(-1.0, x))

    best = math.inf
    det = aa * bb - ab * ab
    if det > 1e-14 * max(aa * bb, 1e-300):
        s = (aw * bb - ab * bw) / det
        t = (ab * aw - aa * bw) / det
        if -1.0 <= s <= 1.0 and -1.0 <= t <= 1.0:
            return f(s, t)
    for s in (-1.0, 1.0):   # edges s = +-1: t minimizes |s a - w - t b|^2
        t = clamp((s * ab - bw) / bb) if bb > 0 else 0.0
        best = min(best, f(s, t))
    for t in (-1.0, 1.0):
        s = clamp((t * ab + aw) / aa) if aa > 0 else 0.0
        best = min(best, f(s, t))
    return best


def generate_cylinders(seed: int, n: int, r: float, h: float, axis=None, spheres: int = 0, r_sphere: float = 0.0,
                       max_candidates: int = 400_000):
    """Seeded RSA of ``n`` coated cylinders (outer radius r, outer length h) and
    ``spheres`` spheres of radius r_sphere in the periodic unit cube (§6: RVEs with
    cylinders, or spheres and cylinders).  Cylinders come first, then spheres; a
    candidate is accepted when its capsule (its axis segment of half-length h/2 inflated
    by its radius; a sphere is a point inflated by its radius) keeps clear of every
    accepted object's capsule; a flat-ended cylinder lies inside its capsule, so the
    objects never overlap.
    Each cylinder candidate draws 5 uniforms (centre, then the axis unless ``axis`` fixes
    it), each sphere candidate 3.  Needs h/2 + r <= 1/4 (one periodic image per pair).
    Returns (spheres (k, 4), cylinders (n, 8): cx, cy, cz, ux, uy, uz, r, h)."""
    if not (0.5 * h + max(r, r_sphere) <= 0.25 + 1e-12):
        raise ValueError("objects must fit a quarter of the cell (h/2 + r <= 1/4)")
    rng = SplitMix64(seed, 5)
    objs = []   # (centre, half-axis vector, radius)
    cyl, sph = [], []
    used = 0
    fixed = None if axis is None else np.asarray(axis, dtype=np.float64) / np.linalg.norm(axis)
    while (len(cyl) < n or len(sph) < spheres) and used < max_candidates:
        is_cyl = len(cyl) < n
        u = rng.uniform(5 if is_cyl else 3)
        used += 1
        c = u[:3]
        if is_cyl:
            ax = fixed if fixed is not None else random_axis(u[3], u[4])
            half, rad = 0.5 * h * ax, r
        else:
            ax = np.zeros(3)
            half, rad = np.zeros(3), r_sphere
        ok = True
        for c2, h2, r2 in objs:
            w = c2 - c
            w = w - np.floor(w + 0.5)                      # minimum image of the centre offset
            if _segment_distance_sq(w, half, h2) <= (rad + r2) * (rad + r2):
                ok = False
                break
        if not ok:
            continue
        objs.append((c, half, rad))
        if is_cyl:
            cyl.append([c[0], c[1], c[2], ax[0], ax[1], ax[2], r, h])
        else:
            sph.append([c[0], c[1], c[2], r_sphere])
    if len(cyl) < n or len(sph) < spheres:
        raise RuntimeError("RSA of cylinders and spheres did not place every object")
    return np.array(sph).reshape(-1, 4), np.array(cyl).reshape(-1, 8)


def centred_sphere(r: float = 0.25) -> np.ndarray:
    """One sphere centred at (0.5, 0.5, 0.5): a voxel corner for every even N."""
    return np.array([[0.5, 0.5, 0.5, r]])


def laminate_grid(N: int, thickness: int, axis: int = 0, phase_a: int = 2,
                  phase_b: int = 0) -> np.ndarray:
    """Phase grid (z, y, x order) of slabs normal to ``axis`` (0 = x): the first
    ``thickness`` planes hold ``phase_a``, the rest ``phase_b``."""
    g = np.full((N, N, N), phase_b, dtype=np.uint8)
    sl = [slice(None)] * 3
    sl[2 - axis] = slice(0, thickness)
    g[tuple(sl)] = phase_a
    return g


def random_phase_grid(seed: int, N: int, probs=(0.5, 0.25, 0.25)) -> np.ndarray:
    """Voxel-wise i.i.d. phases 0/1/2 with the given probabilities (z, y, x order)."""
    u = SplitMix64(seed, 7).uniform(N ** 3).reshape(N, N, N)
    c = np.cumsum(probs)
    return (u >= c[0]).astype(np.uint8) + (u >= c[1]).astype(np.uint8)


# ---------------------------------------------------------------------------
# Workload recipes (the paper's RVE shapes, §2 and §5): sizes and parameters only.
# ---------------------------------------------------------------------------
K_PHASES = (0.20, 0.25, 400.0)   # matrix, inclusion, coating conductivities

WORKLOADS = {
    # 32^3, one centred coated sphere, r_s = 8 voxels, l = 0.25, FP64 plain method
    "sphere32": dict(N=32, spheres="centred", r=0.25, layer=0.25, k=K_PHASES, tol=1e-8),
    # 128^3, 30 RSA spheres at 20 %, l = 0.3 (seeds 1000..1004)
    "rsa128": dict(N=128, n=30, f=0.20, layer=0.3, k=K_PHASES, tol=1e-8, seeds=list(range(1000, 1005))),
    # 256^3, 100 spheres at 40 %, l in {0.1,0.3,0.5}, k_coat in {2,40,400,4000} (seed 3000)
    "rsa256": dict(N=256, n=100, f=0.40, layers=(0.1, 0.3, 0.5), k_coats=(2.0, 40.0, 400.0, 4000.0),
                   k=K_PHASES, tol=1e-8, seed=3000),
}


def batch_recipe(seed0: int = 4000, count: int = 64):
    """Mixed-size stochastic-averaging batch: 24 x 64^3, 24 x 96^3, 16 x 128^3 RVEs with
    n ~ U{10..100}, f ~ U[0.10, 0.40], l ~ U[0.1, 0.5] (one SplitMix64 stream per RVE)."""
    sizes = [64] * 24 + [96] * 24 + [128] * 16
    out = []
    for i in range(count):
        s = seed0 + i
        u = SplitMix64(s, 11).uniform(3)
        n = 10 + int(u[0] * 91)
        f = 0.10 + 0.30 * float(u[1])
        layer = 0.1 + 0.4 * float(u[2])
        out.append(dict(seed=s, N=sizes[i % len(sizes)], n=n, f=f, layer=layer))
    return out


def poisson_arrivals(seed: int, rate_hz: float, count: int):
    """Arrival times (s) of a Poisson stream: exponential gaps from SplitMix64 uniforms."""
    u = SplitMix64(seed, 13).uniform(count)
    gaps = -np.log1p(-u) / rate_hz
    return np.cumsum(gaps)
