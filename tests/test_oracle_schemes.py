"""Pins for the oracle's augmented Lagrangian scheme (``al_solve``, written from its
Lagrangian) and the relaxed polarization iteration (``em_solve`` with beta in place of
the factor 2 of step 7), two of the FFT-based schemes §3 lists beside the accelerated
one: closed forms (homogeneous medium, laminates), the dense direct solve of the
discrete cell problem, agreement with the accelerated scheme, the contraction rate
1 - beta (1 - rho) / 2, the first compatibility residual of a laminate, and the
identity of the augmented Lagrangian iterates with the beta = 1 iterates (derived by
eliminating e and lambda: lambda = k d after every step, so d^{n+1} is
d^n + k0 / (k + k0) (e_comp(d^n) - d^n)).  Planted mistakes must fail."""
import math

import numpy as np
import pytest

from oracle import em as om
from paper_1504_07499_gb300 import inputs as I

K3 = (0.20, 0.25, 400.0)


def test_homogeneous_medium_is_exact():
    ph = I.random_phase_grid(3, 8)
    for K, res in (om.al_effective_tensor(ph, (1.5, 1.5, 1.5)), om.effective_tensor(ph, (1.5, 1.5, 1.5), beta=1.3)):
        assert np.abs(K - 1.5 * np.eye(3)).max() < 1e-13
        assert all(r.converged for r in res)


@pytest.mark.parametrize("N,thick,axis", [(6, 2, 0), (9, 4, 2), (12, 5, 1)])
def test_laminate_means(N, thick, axis):
    ph = I.laminate_grid(N, thick, axis=axis, phase_a=2, phase_b=0)
    f = thick / N
    harm = 1.0 / (f / K3[2] + (1 - f) / K3[0])
    arith = f * K3[2] + (1 - f) * K3[0]
    expect = np.full(3, arith)
    expect[axis] = harm
    for K, _ in (om.al_effective_tensor(ph, K3, tol=1e-10), om.effective_tensor(ph, K3, tol=1e-10, beta=1.5)):
        assert (np.abs(np.diag(K) - expect) <= 1e-8 * expect).all()
        assert np.abs(K - np.diag(np.diag(K))).max() < 1e-9


@pytest.mark.parametrize("N,seed", [(3, 1), (4, 2), (5, 3), (6, 4)])
def test_matches_dense_direct_solve(N, seed):
    ph = I.random_phase_grid(seed, N, probs=(0.4, 0.3, 0.3))
    Kd = om.direct_solve(ph, K3)
    Ka, _ = om.al_effective_tensor(ph, K3, tol=1e-11)
    Kp, _ = om.effective_tensor(ph, K3, tol=1e-11, beta=0.8)
    assert np.abs(Ka - Kd).max() < 1e-9 * np.abs(Kd).max()
    assert np.abs(Kp - Kd).max() < 1e-9 * np.abs(Kd).max()


def test_agrees_with_the_accelerated_scheme():
    N = 16
    sl = I.generate_spheres(5, 6, 0.3)
    ph = om.voxelize(sl.spheres, 0.3, N)
    Ke, re = om.effective_tensor(ph, K3, tol=1e-10)
    Ka, ra = om.al_effective_tensor(ph, K3, tol=1e-10)
    assert np.abs(Ka - Ke).max() < 1e-8 * np.abs(Ke).max()
    # the accelerated scheme needs fewer sweeps than the augmented Lagrangian one
    assert all(a.iters > e.iters for a, e in zip(ra, re))


def test_al_iterates_equal_relaxation_one():
    N = 8
    ph = I.random_phase_grid(21, N)
    E = np.array([0.2, 1.0, -0.4])
    for n in (1, 2, 7):
        ra = om.al_solve(ph, K3, E, tol=0.0, max_iter=n, record=True)
        rp = om.em_solve(ph, K3, E, tol=0.0, max_iter=n, record=True, beta=1.0)
        assert np.abs(ra.e - rp.e).max() < 1e-12 * np.abs(rp.e).max()
        assert np.allclose(ra.eps_comp_hist, rp.eps_comp_hist, rtol=1e-10)


@pytest.mark.parametrize("beta", [1.0, 1.5])
def test_contraction_rate(beta):
    ph = I.random_phase_grid(11, 8)
    rho = om.contraction_rate(K3)
    bound = 1.0 - 0.5 * beta * (1.0 - rho)
    r = om.em_solve(ph, K3, (1.0, 0.0, 0.0), tol=1e-12, max_iter=4000, record=True, beta=beta)
    h = np.array(r.eps_comp_hist)
    ok = h[:-1] > 1e-11
    assert (h[1:][ok] <= bound * h[:-1][ok] * (1 + 1e-9)).all()
    ra = om.al_solve(ph, K3, (1.0, 0.0, 0.0), tol=1e-12, record=True)
    ha = np.array(ra.eps_comp_hist)
    oka = ha[:-1] > 1e-11
    rho_al = 0.5 * (1.0 + rho)
    assert (ha[1:][oka] <= rho_al * ha[:-1][oka] * (1 + 1e-9)).all()


def test_first_compatibility_residual_of_a_laminate():
    # the first compatible field of d^0 = E is the accelerated scheme's: eps = std(k) / k0
    N, thick = 10, 4
    ph = I.laminate_grid(N, thick, axis=1, phase_a=2, phase_b=0)
    r = om.al_solve(ph, K3, (0.0, 2.0, 0.0), tol=1e-30, max_iter=1, record=True)
    f = thick / N
    expect = abs(K3[2] - K3[0]) * math.sqrt(f * (1 - f)) / om.reference_k0(K3)
    assert abs(r.eps_comp_hist[0] - expect) <= 1e-12 * expect


# --- planted mistakes -----------------------------------------------------------


def _al_variant(ph, E, n, multiplier_sign=1.0, penalty_d=1.0):
    """al_solve's steps with one planted change (for the tests below only)."""
    N = ph.shape[0]
    k = np.asarray(K3)[ph]
    k0 = om.reference_k0(K3)
    xi = om.wavevectors(N)
    d = np.broadcast_to(E[:, None, None, None], (3, N, N, N)).copy()
    lam = k[None] * d
    for _ in range(n):
        e_hat = om.gamma0_apply(xi, k0, om.fft3(d - lam / k0)) * k0
        e_hat[:, 0, 0, 0] = E * N ** 3
        e = (om.ifft3_unnorm(e_hat) / N ** 3).real
        d = (lam + penalty_d * k0 * e) / (k + penalty_d * k0)[None]
        lam = lam + multiplier_sign * k0 * (e - d)
    return d


@pytest.mark.parametrize("change", [dict(multiplier_sign=-1.0), dict(penalty_d=2.0)])
def test_planted_mistakes_break_the_iterate_identity(change):
    N = 8
    ph = I.random_phase_grid(21, N)
    E = np.array([0.2, 1.0, -0.4])
    good = _al_variant(ph, E, 5)
    ref = om.em_solve(ph, K3, E, tol=0.0, max_iter=5, beta=1.0).e
    assert np.abs(good - ref).max() < 1e-12 * np.abs(ref).max()
    bad = _al_variant(ph, E, 5, **change)
    assert np.abs(bad - ref).max() > 1e-6 * np.abs(ref).max()
