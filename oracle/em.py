"""CPU oracle for the Eyre-Milton FFT homogenization scheme (and the basic scheme it is
compared with) -- TEST INFRASTRUCTURE ONLY.

Only the test suite, the smoke check and the CPU-baseline leg of the benchmark may
import this module.  The product path (the CUDA library and its Python binding)
never calls it and shares no code with it.

Everything here is plain FP64 numpy written from the paper:

* §2 / Fig. 1: coated spheres -- outer radius r_s, layer l = coating width / r_s,
  core radius (1 - l) r_s -- voxelized into three phases (matrix 0, inclusion 1,
  coating 2).  Voxelization is integer arithmetic on quantized coordinates so the
  phase grid is defined bit for bit (rule below).
* §3, eq. 1: polarization form with a constant reference medium L0 = -k0 I,
  k0 = sqrt(min k * max k) (§5).
* §3, Green operator under eq. 3: Gamma0_ij(xi) = xi_i xi_j / (xi . L0 xi).
* §3, Algorithm, steps 1-7, in the paper's order and notation (gradient form e = grad theta).
* §3 last paragraph: <phi> = -L_hom grad Theta gives the effective tensor.
* §3 (the list of FFT-based schemes) and eqs. 1-3: the basic scheme, the plain
  fixed-point iteration of the Lippmann-Schwinger equation (``basic_solve``), the
  augmented Lagrangian scheme from its Lagrangian (``al_solve``), and the polarization
  scheme read as step 7 with a relaxation beta in place of 2 (``em_solve(beta=...)``).

The 3D DFT is the direct sum (``dft3_direct``, taken axis by axis) on grids up to
16^3, and the library FFT (scipy.fft) above that, which the tests pin against the
direct sum.

Readings where the paper is silent or garbled (each is also listed in the design
notes):

* Sign of L0: taken as -k0 I with k0 > 0 in every formula, which is the only
  reading under which the printed steps converge.  The basic scheme takes the
  positive reference +k0 I, k0 = (min k + max k) / 2, the only sign under which
  the plain iteration converges.
* DC of step 4 with an unnormalized DFT: the mean gradient times N^3.
* Wavevector and Nyquist rule: m_j in (-N/2, N/2], xi_j = 2 pi m_j / N (voxel
  units).  Nyquist components (m_j = N/2, N even) are dropped from xi, except in a
  mode whose only nonzero component is a Nyquist one, which keeps it.  The
  projector P = xi xi^T / |xi|^2 (zero where xi = 0) is then real, even in m,
  an orthogonal projector at every mode, and invariant under the reflections and
  axis permutations of the grid: at the modes with two or three Nyquist components
  and nothing else, where +pi and -pi are the same frequency, any rank-one choice
  would break the reflection symmetry, so P = 0 there.  Single-axis Nyquist modes
  keep P = e_j e_j^T, which makes laminates exact.
* Equilibrium residual of step 1: the divergence xi . phi_hat with
  phi_hat = DFT(phi) / N^3, summed over nonzero modes, over |phi_hat(0)|.
* Step 1 uses the eps_comp of the previous sweep (infinite before the first) and
  tests the current iterate; the same tolerance serves both tests.
* Voxelization: voxel (i, j, k) has centre ((i+1/2)/N, ...); coordinates are
  quantized to S = 2 N G units with G = 4096 (voxel centres at odd multiples of
  G); centre C = floor(c S + 1/2) mod S after wrapping c into [0, 1);
  R_out^2 = floor((r S)^2 + 1/2), R_in^2 = floor(((1 - l) r S)^2 + 1/2);
  periodic minimum-image squared distance d^2 in int64; phase 1 if any sphere has
  d^2 <= R_in^2, else 2 if any has d^2 <= R_out^2, else 0.

Parity pins: every function here is checked in ``tests/test_oracle_*.py`` against
closed forms (homogeneous medium, laminates), a dense direct solve of the discrete
equations on tiny grids, the Wiener and Hashin-Shtrikman bounds, the contraction
rate of the iteration, symmetry and metamorphic relations, and the paper's
Tables 0-3.
"""
from __future__ import annotations

import math
import os
from dataclasses import dataclass, field

import numpy as np

try:  # library FFT; pinned against the direct sum in the tests
    import scipy.fft as _sfft
except ImportError:  # pragma: no cover
    _sfft = None

MATRIX, INCLUSION, COATING = 0, 1, 2
QUANT_G = 4096

# ---------------------------------------------------------------------------
# §2 geometry: coated spheres -> three-phase voxel grid
# ---------------------------------------------------------------------------


def quantize_spheres(spheres, layer: float, N: int):
    """Integer sphere data for the voxelization rule: centres (n, 3) in units of
    1 / (2 N G), and squared outer / core radii in the same units."""
    S = 2 * N * QUANT_G
    out = []
    for cx, cy, cz, r in np.asarray(spheres, dtype=np.float64):
        cen = []
        for c in (cx, cy, cz):
            cw = c - math.floor(c)
            q = math.floor(cw * S + 0.5)
            cen.append(q % S)
        t_out = r * S
        t_in = (1.0 - layer) * r * S
        out.append((cen[0], cen[1], cen[2],
                    math.floor(t_out * t_out + 0.5), math.floor(t_in * t_in + 0.5)))
    return np.array(out, dtype=np.int64).reshape(-1, 5), S


def voxelize(spheres, layer: float, N: int) -> np.ndarray:
    """Three-phase grid (z, y, x order, uint8) of coated spheres (§2, Fig. 1)."""
    q, S = quantize_spheres(spheres, layer, N)
    v = (2 * np.arange(N, dtype=np.int64) + 1) * QUANT_G  # voxel-centre coordinates
    incl = np.zeros((N, N, N), dtype=bool)
    coat = np.zeros((N, N, N), dtype=bool)
    for cx, cy, cz, ro2, ri2 in q:
        d = []
        for c in (cx, cy, cz):
            delta = (v - c) % S
            dd = np.minimum(delta, S - delta)
            d.append(dd * dd)
        d2 = d[2][:, None, None] + d[1][None, :, None] + d[0][None, None, :]
        incl |= d2 <= ri2
        coat |= d2 <= ro2
    phase = np.zeros((N, N, N), dtype=np.uint8)
    phase[coat] = COATING
    phase[incl] = INCLUSION
    return phase


# Coated cylinders (§6: RVEs "with cylinders or both spheres and cylinders").  A cylinder
# has a centre, a unit axis u, an outer radius r and an outer length h; the coating has the
# same thickness l r on the lateral surface and on the flat ends, so the core has radius
# (1 - l) r and length h - 2 l r.  Integer rule (coordinates in units of 1 / (2 N GC),
# voxel centres at odd multiples of GC): the centre maps like a sphere's; the axis to
# A = floor(u 1024 + 1/2) per component; squared radii to floor((r S)^2 + 1/2) and
# floor(((1 - l) r S)^2 + 1/2); half-lengths to floor((h/2) S + 1/2) and
# floor((h/2 - l r) S + 1/2).  With d the signed minimum-image offset of a voxel centre
# from the cylinder centre (each component in [-S/2, S/2)) and t = d . A, the voxel lies in
# the cylinder when |d|^2 |A|^2 - t^2 <= R^2 |A|^2 (radial) and t^2 <= H^2 |A|^2 (axial),
# in int64 (the quantization keeps every product below 2^63 up to N = 512).

QUANT_GC = 256
AXIS_Q = 1024


def quantize_cylinders(cylinders, layer: float, N: int):
    """Integer cylinder data: (n, 10) rows (Cx, Cy, Cz, Ax, Ay, Az, R_out^2, R_in^2, H_out,
    H_in), and S."""
    S = 2 * N * QUANT_GC
    out = []
    for cx, cy, cz, ux, uy, uz, r, h in np.asarray(cylinders, dtype=np.float64).reshape(-1, 8):
        cen = []
        for c in (cx, cy, cz):
            cw = c - math.floor(c)
            cen.append(math.floor(cw * S + 0.5) % S)
        ax = [math.floor(u * AXIS_Q + 0.5) for u in (ux, uy, uz)]
        t_out = r * S
        t_in = (1.0 - layer) * r * S
        out.append((*cen, *ax, math.floor(t_out * t_out + 0.5), math.floor(t_in * t_in + 0.5),
                    math.floor(0.5 * h * S + 0.5), math.floor((0.5 * h - layer * r) * S + 0.5)))
    return np.array(out, dtype=np.int64).reshape(-1, 10), S


def cylinder_masks(cylinders, layer: float, N: int):
    """(core, outer) boolean grids (z, y, x) of the coated cylinders."""
    q, S = quantize_cylinders(cylinders, layer, N)
    v = (2 * np.arange(N, dtype=np.int64) + 1) * QUANT_GC
    core = np.zeros((N, N, N), dtype=bool)
    outer = np.zeros((N, N, N), dtype=bool)
    for cx, cy, cz, ax, ay, az, ro2, ri2, ho, hi in q:
        d = []
        for c in (cx, cy, cz):
            d.append((v - c + S // 2) % S - S // 2)          # signed minimum image
        dx, dy, dz = d[0][None, None, :], d[1][None, :, None], d[2][:, None, None]
        a2 = ax * ax + ay * ay + az * az
        t = dx * ax + dy * ay + dz * az
        rad = (dx * dx + dy * dy + dz * dz) * a2 - t * t
        t2 = t * t
        outer |= (rad <= ro2 * a2) & (t2 <= ho * ho * a2)
        if hi > 0:
            core |= (rad <= ri2 * a2) & (t2 <= hi * hi * a2)
    return core, outer


def voxelize_mixed(spheres, cylinders, layer: float, N: int) -> np.ndarray:
    """Three-phase grid of coated spheres and coated cylinders (same layer l): inclusion
    inside any core, else coating inside any outer shape, else matrix."""
    phase = np.zeros((N, N, N), dtype=np.uint8)
    incl = np.zeros((N, N, N), dtype=bool)
    coat = np.zeros((N, N, N), dtype=bool)
    if spheres is not None and len(spheres):
        ph_s = voxelize(spheres, layer, N)
        incl |= ph_s == INCLUSION
        coat |= ph_s != MATRIX
    if cylinders is not None and len(cylinders):
        core, outer = cylinder_masks(cylinders, layer, N)
        incl |= core
        coat |= outer
    phase[coat] = COATING
    phase[incl] = INCLUSION
    return phase


def coating_fraction(layer: float, f_sp: float) -> float:
    """Coating volume fraction of spheres of total fraction f_sp (§5, Table 0)."""
    return (1.0 - (1.0 - layer) ** 3) * f_sp


def coating_voxels(layer: float, res: int, n_sp: int, f_sp: float = 0.3) -> float:
    """Coating thickness in voxels, l * Res * r_s with r_s = (3 f / (4 pi n))^(1/3)
    (§5, Tables 1-3; n_sp read in the denominator)."""
    return layer * res * (3.0 * f_sp / (4.0 * math.pi * n_sp)) ** (1.0 / 3.0)


# ---------------------------------------------------------------------------
# §5 reference medium
# ---------------------------------------------------------------------------


def reference_k0(k_phases) -> float:
    """k0 = sqrt(min k * max k) over the phase conductivities (§5); L0 = -k0 I."""
    return math.sqrt(min(k_phases) * max(k_phases))


# ---------------------------------------------------------------------------
# 3D DFT: direct sum and library
# ---------------------------------------------------------------------------

_DFT_CACHE: dict = {}


def _dft_matrix(N: int) -> np.ndarray:
    """Matrix of the 3D DFT on N^3 points (z, y, x flattening), by the definition
    X[k] = sum_n x[n] exp(-2 pi i (k . n) / N).  Built row-block by row-block."""
    if N not in _DFT_CACHE:
        idx = np.indices((N, N, N)).reshape(3, -1).T  # (N^3, 3) = (z, y, x)
        M = np.empty((N ** 3, N ** 3), dtype=np.complex128)
        for a in range(0, N ** 3, 256):
            kn = (idx[a:a + 256, None, :] * idx[None, :, :]).sum(-1) % N
            M[a:a + 256] = np.exp(-2j * np.pi * kn / N)
        _DFT_CACHE[N] = M
    return _DFT_CACHE[N]


def dft3_dense(x: np.ndarray, inverse: bool = False) -> np.ndarray:
    """Unnormalized 3D DFT as one dense N^3 x N^3 matrix product (the definition
    written out; meant for N <= 8, where it pins ``dft3_direct``)."""
    N = x.shape[-1]
    M = _dft_matrix(N)
    flat = x.reshape(x.shape[:-3] + (N ** 3,)).astype(np.complex128)
    y = flat @ (M.conj().T if inverse else M.T)
    return y.reshape(x.shape)


def dft3_direct(x: np.ndarray, inverse: bool = False) -> np.ndarray:
    """Unnormalized 3D DFT by the direct sum (inverse: conjugate kernel, no 1/N^3).
    exp(-2 pi i k.n/N) factors into one exponential per axis, so the triple sum is
    taken one axis at a time with the N x N matrix W[k, n] = exp(-+2 pi i (k n mod N)/N):
    O(N^4) work, no fast algorithm."""
    N = x.shape[-1]
    kn = np.outer(np.arange(N), np.arange(N)) % N
    W = np.exp((2j if inverse else -2j) * np.pi * kn / N)
    y = x.astype(np.complex128)
    for axis in (-1, -2, -3):
        y = np.moveaxis(np.tensordot(y, W, axes=([axis], [1])), -1, axis)
    return y


def _workers() -> int:
    return int(os.environ.get("HMG_ORACLE_THREADS", os.cpu_count() or 1))


def fft3(x: np.ndarray) -> np.ndarray:
    """Unnormalized forward 3D DFT over the last three axes: the direct sum on grids up
    to 16^3, the library FFT above (pinned against the direct sum in the tests)."""
    N = x.shape[-1]
    if N <= 16:
        return dft3_direct(x)
    if _sfft is None:
        return np.fft.fftn(x, axes=(-3, -2, -1))
    return _sfft.fftn(x, axes=(-3, -2, -1), workers=_workers())


def ifft3_unnorm(X: np.ndarray) -> np.ndarray:
    """Unnormalized inverse 3D DFT (kernel exp(+2 pi i k.n/N), no 1/N^3)."""
    N = X.shape[-1]
    if N <= 16:
        return dft3_direct(X, inverse=True)
    if _sfft is None:
        return np.fft.ifftn(X, axes=(-3, -2, -1)) * N ** 3
    return _sfft.ifftn(X, axes=(-3, -2, -1), workers=_workers(), norm="forward")


# ---------------------------------------------------------------------------
# §3 wavevectors and the Green operator
# ---------------------------------------------------------------------------


def mode_indices(N: int) -> np.ndarray:
    """Signed mode numbers m in (-N/2, N/2] for DFT indices 0..N-1."""
    k = np.arange(N)
    return np.where(k <= N // 2, k, k - N)


def wavevectors(N: int) -> np.ndarray:
    """Wavevector field xi' (3, N, N, N) in (z, y, x) grid order, components (x, y, z),
    with the Nyquist rule stated in the module docstring (zero at DC and at the modes
    made only of two or three Nyquist components)."""
    m = mode_indices(N)
    mz, my, mx = np.meshgrid(m, m, m, indexing="ij")
    comps = [mx, my, mz]
    nyq = [(N % 2 == 0) & (c == N // 2) for c in comps]
    nonzero = (mx != 0).astype(int) + (my != 0) + (mz != 0)
    xi = np.empty((3, N, N, N))
    for j in range(3):
        keep = ~nyq[j] | (nonzero == 1)
        xi[j] = np.where(keep, 2.0 * np.pi * comps[j] / N, 0.0)
    return xi


def gamma0_apply(xi: np.ndarray, L0: float, tau_hat: np.ndarray) -> np.ndarray:
    """Gamma0(xi) tau_hat with Gamma0_ij = xi_i xi_j / (xi . L0 xi) for an isotropic
    L0 = L0 * I (§3); zero at xi = 0."""
    xi2 = (xi * xi).sum(0)
    dot = (xi * tau_hat).sum(0)
    with np.errstate(invalid="ignore", divide="ignore"):
        coef = np.where(xi2 > 0, dot / (L0 * np.where(xi2 > 0, xi2, 1.0)), 0.0)
    return xi * coef


# ---------------------------------------------------------------------------
# §3 Algorithm
# ---------------------------------------------------------------------------


@dataclass
class EMResult:
    e: np.ndarray                 # final gradient field (3, N, N, N), components (x, y, z)
    flux_mean: np.ndarray         # <phi> of the final field (paper's sign: phi = -k e)
    iters: int                    # number of sweeps through steps 2-7
    converged: bool
    eps_eq: float
    eps_comp_hist: list = field(default_factory=list)
    eps_eq_hist: list = field(default_factory=list)


def equilibrium_residual(k_field: np.ndarray, e: np.ndarray, xi: np.ndarray):
    """Step 1: phi = -L grad theta, phi_hat = DFT(phi)/N^3,
    eps_eq = sqrt(sum_{xi != 0} |xi . phi_hat|^2) / |phi_hat(0)|.  Returns (eps_eq, <phi>)."""
    N = e.shape[-1]
    phi = -k_field[None] * e
    phi_hat = fft3(phi) / N ** 3
    div = (xi * phi_hat).sum(0)
    div[0, 0, 0] = 0.0
    mean = phi_hat[:, 0, 0, 0].real
    return math.sqrt(float((np.abs(div) ** 2).sum())) / float(np.linalg.norm(mean)), mean


def compatibility_residual(e: np.ndarray, ec: np.ndarray, normE: float) -> float:
    """Step 6: eps_comp = sqrt(<|e - e_comp|^2>) / |grad Theta|, the volume average
    <.> being the mean over the N^3 voxels."""
    return math.sqrt(float(((e - ec) ** 2).sum(0).mean())) / normE


def em_solve(phase: np.ndarray, k_phases, grad_Theta, tol: float = 1e-8,
             max_iter: int = 20000, record: bool = False, e0: np.ndarray | None = None,
             beta: float = 2.0) -> EMResult:
    """Eyre-Milton accelerated scheme of §3 (Algorithm, steps 1-7) for one macroscopic
    gradient grad_Theta, in the gradient form and the paper's notation.

    ``beta`` replaces the factor 2 of step 7 (the polarization family read for the
    polarization scheme §3 names: 2 is the accelerated scheme itself)."""
    N = phase.shape[0]
    k_field = np.asarray(k_phases, dtype=np.float64)[phase]
    L0 = -reference_k0(k_phases)                 # L0 = -sqrt(min * max) I   (§5)
    xi = wavevectors(N)
    E = np.asarray(grad_Theta, dtype=np.float64)
    normE = float(np.linalg.norm(E))
    # Initialization: grad theta^0 = grad Theta everywhere.
    e = np.broadcast_to(E[:, None, None, None], (3, N, N, N)).copy() if e0 is None else e0.copy()
    eps_comp = math.inf
    hist_c, hist_q = [], []
    eps_eq = math.inf
    for n in range(max_iter):
        # Step 1: convergence test on the current iterate.
        if eps_comp < tol:
            eps_eq, mean_phi = equilibrium_residual(k_field, e, xi)
            hist_q.append(eps_eq)
            if eps_eq < tol:
                return EMResult(e, mean_phi, n, True, eps_eq, hist_c, hist_q)
        # Step 2: tau = -(L + L0) grad theta.
        tau = -(k_field + L0)[None] * e
        # Step 3: tau_hat = FFT(tau).
        tau_hat = fft3(tau)
        # Step 4: e_comp_hat = -Gamma0 tau_hat for xi != 0, = grad Theta at xi = 0.
        ec_hat = -gamma0_apply(xi, L0, tau_hat)
        ec_hat[:, 0, 0, 0] = E * N ** 3
        # Step 5: inverse FFT.
        ec_c = ifft3_unnorm(ec_hat) / N ** 3
        ec = ec_c.real
        # Step 6: eps_comp = sqrt(<|e - e_comp|^2>) / |grad Theta|.
        eps_comp = compatibility_residual(e, ec, normE)
        if record:
            hist_c.append(eps_comp)
        if not math.isfinite(eps_comp):
            break
        # Step 7: e^{n+1} = e^n - 2 (L - L0)^{-1} L0 (e_comp - e^n)  (beta in place of 2).
        e = e - beta * (L0 / (k_field - L0))[None] * (ec - e)
    eps_eq, mean_phi = equilibrium_residual(k_field, e, xi)
    return EMResult(e, mean_phi, max_iter, False, eps_eq, hist_c, hist_q)


def effective_tensor(phase: np.ndarray, k_phases, tol: float = 1e-8, max_iter: int = 20000,
                     beta: float = 2.0):
    """L_hom from <phi> = -L_hom grad Theta for the three unit gradients (§3).
    Returns (K (3x3, column j answers gradient e_j), [EMResult] * 3)."""
    K = np.zeros((3, 3))
    res = []
    for j in range(3):
        E = np.zeros(3)
        E[j] = 1.0
        r = em_solve(phase, k_phases, E, tol, max_iter, beta=beta)
        K[:, j] = -r.flux_mean
        res.append(r)
    return K, res


# ---------------------------------------------------------------------------
# §3 augmented Lagrangian scheme (named in §3's list of FFT-based schemes; the
# paper prints no formula).  Written from its definition in Michel, Moulinec &
# Suquet (2001), cited in §5: the cell problem is the minimization of <e.k e>/2
# over compatible fields e with mean grad Theta; a free field d with the constraint
# d = e and a multiplier lambda give the augmented Lagrangian
#     <d.k d>/2 + <lambda.(e - d)> + k0 <|e - d|^2>/2,
# minimized alternately over e (compatible: a Fourier projection) and d (pointwise),
# followed by the multiplier step.  Reading: penalty k0 = sqrt(min k * max k) as for
# the accelerated scheme (§5); the two tests of the §3 Algorithm are applied to the
# iterate d (step 6: |d - e| of the compatible field e it gives; step 1: equilibrium
# of the flux lambda).
# ---------------------------------------------------------------------------


def al_solve(phase: np.ndarray, k_phases, grad_Theta, tol: float = 1e-8,
             max_iter: int = 40000, record: bool = False) -> EMResult:
    """Augmented Lagrangian scheme for one macroscopic gradient.  EMResult.e is the
    final iterate d; its flux is lambda."""
    N = phase.shape[0]
    k_field = np.asarray(k_phases, dtype=np.float64)[phase]
    k0 = reference_k0(k_phases)
    xi = wavevectors(N)
    E = np.asarray(grad_Theta, dtype=np.float64)
    normE = float(np.linalg.norm(E))
    d = np.broadcast_to(E[:, None, None, None], (3, N, N, N)).copy()
    lam = k_field[None] * d                        # multiplier: the flux of d
    eps_comp = math.inf
    hist_c, hist_q = [], []
    eps_eq = math.inf
    for n in range(max_iter):
        # Step 1 on the current iterate: equilibrium of its flux
        if eps_comp < tol:
            eps_eq, mean_phi = equilibrium_residual(k_field, d, xi)
            hist_q.append(eps_eq)
            if eps_eq < tol:
                return EMResult(d, mean_phi, n, True, eps_eq, hist_c, hist_q)
        # e: minimize <lambda.e> + k0 <|e - d|^2>/2 over e = grad Theta + compatible
        # fluctuation: e = grad Theta + P(d - lambda / k0), P = k0 Gamma0 for L0 = k0
        q_hat = fft3(d - lam / k0)
        e_hat = gamma0_apply(xi, k0, q_hat) * k0
        e_hat[:, 0, 0, 0] = E * N ** 3
        e = (ifft3_unnorm(e_hat) / N ** 3).real
        # step 6 on the iterate d
        eps_comp = compatibility_residual(d, e, normE)
        if record:
            hist_c.append(eps_comp)
        if not math.isfinite(eps_comp):
            break
        # d: minimize <d.k d>/2 - <lambda.d> + k0 <|e - d|^2>/2 pointwise
        d = (lam + k0 * e) / (k_field + k0)[None]
        # multiplier step
        lam = lam + k0 * (e - d)
    eps_eq, mean_phi = equilibrium_residual(k_field, d, xi)
    return EMResult(d, mean_phi, max_iter, False, eps_eq, hist_c, hist_q)


def al_effective_tensor(phase: np.ndarray, k_phases, tol: float = 1e-8, max_iter: int = 40000):
    """L_hom of the augmented Lagrangian scheme for the three unit gradients."""
    K = np.zeros((3, 3))
    res = []
    for j in range(3):
        E = np.zeros(3)
        E[j] = 1.0
        r = al_solve(phase, k_phases, E, tol, max_iter)
        K[:, j] = -r.flux_mean
        res.append(r)
    return K, res


# ---------------------------------------------------------------------------
# §3 basic scheme (named in §3 among the FFT-based schemes; the paper prints only
# the accelerated one).  It iterates the Lippmann-Schwinger equation of eqs. 1-3
# directly: grad theta = grad Theta - Gamma0 * tau, tau = (L - L0) grad theta.
# Reading: the reference medium is positive, L0 = k0 I with k0 = (min k + max k) / 2
# (with the negative L0 of the accelerated scheme the plain iteration diverges);
# the two convergence tests are steps 1 and 6 of the §3 Algorithm, and the new
# iterate is the compatible field of step 5.
# ---------------------------------------------------------------------------


def basic_reference_k0(k_phases) -> float:
    """k0 of the basic scheme: the centre of the conductivity range (L0 = +k0 I)."""
    k = np.asarray(k_phases, dtype=np.float64)
    return 0.5 * (float(k.min()) + float(k.max()))


def basic_solve(phase: np.ndarray, k_phases, grad_Theta, tol: float = 1e-8,
                max_iter: int = 200000, record: bool = False) -> EMResult:
    """Basic scheme for one macroscopic gradient, in the steps of the §3 Algorithm
    without its acceleration (step 7 keeps the compatible field)."""
    N = phase.shape[0]
    k_field = np.asarray(k_phases, dtype=np.float64)[phase]
    L0 = basic_reference_k0(k_phases)             # L0 = +k0 I
    xi = wavevectors(N)
    E = np.asarray(grad_Theta, dtype=np.float64)
    normE = float(np.linalg.norm(E))
    e = np.broadcast_to(E[:, None, None, None], (3, N, N, N)).copy()
    eps_comp = math.inf
    hist_c, hist_q = [], []
    eps_eq = math.inf
    for n in range(max_iter):
        # Step 1: convergence test on the current iterate.
        if eps_comp < tol:
            eps_eq, mean_phi = equilibrium_residual(k_field, e, xi)
            hist_q.append(eps_eq)
            if eps_eq < tol:
                return EMResult(e, mean_phi, n, True, eps_eq, hist_c, hist_q)
        # Polarization tau = (L - L0) grad theta (eq. 1).
        tau = (k_field - L0)[None] * e
        tau_hat = fft3(tau)
        # grad theta_hat = -Gamma0 tau_hat for xi != 0, grad Theta at xi = 0 (eqs. 2-3).
        ec_hat = -gamma0_apply(xi, L0, tau_hat)
        ec_hat[:, 0, 0, 0] = E * N ** 3
        ec = (ifft3_unnorm(ec_hat) / N ** 3).real
        # Step 6: eps_comp = sqrt(<|e - e_comp|^2>) / |grad Theta|.
        eps_comp = compatibility_residual(e, ec, normE)
        if record:
            hist_c.append(eps_comp)
        if not math.isfinite(eps_comp):
            break
        e = ec
    eps_eq, mean_phi = equilibrium_residual(k_field, e, xi)
    return EMResult(e, mean_phi, max_iter, False, eps_eq, hist_c, hist_q)


def basic_effective_tensor(phase: np.ndarray, k_phases, tol: float = 1e-8, max_iter: int = 200000):
    """L_hom of the basic scheme for the three unit gradients (same reading of K as
    ``effective_tensor``).  Returns (K, [EMResult] * 3)."""
    K = np.zeros((3, 3))
    res = []
    for j in range(3):
        E = np.zeros(3)
        E[j] = 1.0
        r = basic_solve(phase, k_phases, E, tol, max_iter)
        K[:, j] = -r.flux_mean
        res.append(r)
    return K, res


# ---------------------------------------------------------------------------
# Independent checks used to pin the iteration
# ---------------------------------------------------------------------------


def projector_matrix(N: int) -> np.ndarray:
    """Dense real matrix of the compatible-field projector P (3N^3 x 3N^3) acting on
    stacked components (x, y, z), assembled column by column from the DFT."""
    xi = wavevectors(N)
    n = N ** 3
    P = np.zeros((3 * n, 3 * n))
    xi2 = (xi * xi).sum(0)
    for col in range(3 * n):
        v = np.zeros(3 * n)
        v[col] = 1.0
        vh = fft3(v.reshape(3, N, N, N))
        dot = (xi * vh).sum(0)
        ph = xi * np.where(xi2 > 0, dot / np.where(xi2 > 0, xi2, 1.0), 0.0)
        P[:, col] = (ifft3_unnorm(ph) / n).real.reshape(-1)
    return P


def direct_solve(phase: np.ndarray, k_phases) -> np.ndarray:
    """Effective tensor from a dense solve of the discrete cell problem
    (I - P + P diag(k)) e = E: compatibility (I - P) e = E and equilibrium
    P (k e) = 0.  Independent of the iteration; meant for N <= 6."""
    N = phase.shape[0]
    n = N ** 3
    k = np.asarray(k_phases, dtype=np.float64)[phase].reshape(-1)
    kk = np.concatenate([k, k, k])
    P = projector_matrix(N)
    A = np.eye(3 * n) - P + P * kk[None, :]
    K = np.zeros((3, 3))
    for j in range(3):
        rhs = np.zeros(3 * n)
        rhs[j * n:(j + 1) * n] = 1.0
        e = np.linalg.solve(A, rhs)
        K[:, j] = (kk * e).reshape(3, n).mean(1)
    return K


def phase_fractions(phase: np.ndarray) -> np.ndarray:
    return np.bincount(phase.reshape(-1), minlength=3)[:3] / phase.size


def wiener_bounds(phase: np.ndarray, k_phases):
    """Harmonic and arithmetic means of k over the voxel phase fractions."""
    f = phase_fractions(phase)
    k = np.asarray(k_phases, dtype=np.float64)
    return 1.0 / float((f / k).sum()), float((f * k).sum())


def hashin_shtrikman_bounds(phase: np.ndarray, k_phases):
    """Isotropic Hashin-Shtrikman bounds for the voxel phase fractions:
    k_HS(k*) = [sum_i f_i / (k_i + 2 k*)]^-1 - 2 k*, with k* = min k (lower) and max k (upper)."""
    f = phase_fractions(phase)
    k = np.asarray(k_phases, dtype=np.float64)
    present = f > 0
    f, k = f[present], k[present]

    def hs(ks):
        return 1.0 / float((f / (k + 2.0 * ks)).sum()) - 2.0 * ks

    return hs(k.min()), hs(k.max())


def contraction_rate(k_phases) -> float:
    """Bound rho = max |(k - k0)/(k + k0)| = (sqrt(c) - 1)/(sqrt(c) + 1) on the rate at
    which successive eps_comp decrease, c = max k / min k."""
    c = max(k_phases) / min(k_phases)
    return (math.sqrt(c) - 1.0) / (math.sqrt(c) + 1.0)
