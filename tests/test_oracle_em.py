"""Pins for the oracle's Eyre-Milton iteration (§3, Algorithm) and effective tensor:
closed forms (homogeneous medium, laminates), a dense direct solve of the discrete
cell problem, the contraction rate, the Wiener and Hashin-Shtrikman bounds,
symmetry, metamorphic relations, and planted mistakes that these pins must catch."""
import math

import numpy as np
import pytest

from oracle import em as om
from paper_1504_07499_gb300 import inputs as I

K3 = (0.20, 0.25, 400.0)


def test_homogeneous_medium_is_exact():
    ph = I.random_phase_grid(3, 8)
    K, res = om.effective_tensor(ph, (2.5, 2.5, 2.5))
    assert np.abs(K - 2.5 * np.eye(3)).max() < 1e-13
    for r in res:
        assert r.iters == 1 and r.converged
    r = om.em_solve(ph, (2.5, 2.5, 2.5), (0.0, 1.0, 0.0), record=True)
    assert r.eps_comp_hist[0] < 1e-14


@pytest.mark.parametrize("N,thick,axis", [(6, 2, 0), (8, 3, 1), (9, 4, 2), (10, 5, 0), (12, 1, 2)])
def test_laminate_means(N, thick, axis):
    ph = I.laminate_grid(N, thick, axis=axis, phase_a=2, phase_b=0)
    K, res = om.effective_tensor(ph, K3, tol=1e-10)
    f = thick / N
    harm = 1.0 / (f / K3[2] + (1 - f) / K3[0])
    arith = f * K3[2] + (1 - f) * K3[0]
    expect = np.full(3, arith)
    expect[axis] = harm
    assert (np.abs(np.diag(K) - expect) <= 1e-8 * expect).all()
    assert np.abs(K - np.diag(np.diag(K))).max() < 1e-9


@pytest.mark.parametrize("N,seed", [(3, 1), (4, 2), (5, 3), (6, 4)])
def test_matches_dense_direct_solve(N, seed):
    ph = I.random_phase_grid(seed, N, probs=(0.4, 0.3, 0.3))
    Kd = om.direct_solve(ph, K3)
    K, _ = om.effective_tensor(ph, K3, tol=1e-11)
    assert np.abs(K - Kd).max() < 1e-9 * np.abs(Kd).max()


def test_dense_solve_of_centred_sphere_is_isotropic():
    # reflection and permutation symmetry of the grid -> K = kappa I for the exact
    # discrete solution (this pins the Nyquist rule at multi-Nyquist modes)
    ph = om.voxelize(I.centred_sphere(0.3), 0.3, 6)
    Kd = om.direct_solve(ph, K3)
    assert np.abs(Kd - Kd[0, 0] * np.eye(3)).max() < 1e-12


def test_matches_dense_direct_solve_coated_sphere():
    ph = om.voxelize(np.array([[0.41, 0.55, 0.48, 0.33]]), 0.3, 6)
    assert set(np.unique(ph)) == {0, 1, 2}
    Kd = om.direct_solve(ph, K3)
    K, _ = om.effective_tensor(ph, K3, tol=1e-11)
    assert np.abs(K - Kd).max() < 1e-9 * np.abs(Kd).max()


def test_contraction_rate_of_eps_comp():
    ph = I.random_phase_grid(11, 8)
    rho = om.contraction_rate(K3)
    r = om.em_solve(ph, K3, (1.0, 0.0, 0.0), tol=1e-12, record=True)
    h = np.array(r.eps_comp_hist)
    ok = h[:-1] > 1e-11
    assert (h[1:][ok] <= rho * h[:-1][ok] * (1 + 1e-9)).all()
    # the bound is nearly attained for a high-contrast grid
    assert (h[1:][ok] / h[:-1][ok]).max() > 0.5 * rho


def test_wiener_bounds_and_spd():
    for seed, N in [(21, 8), (22, 12)]:
        ph = I.random_phase_grid(seed, N, probs=(0.5, 0.2, 0.3))
        K, _ = om.effective_tensor(ph, K3)
        assert np.abs(K - K.T).max() < 1e-6 * np.abs(K).max()
        ev = np.linalg.eigvalsh(0.5 * (K + K.T))
        lo, hi = om.wiener_bounds(ph, K3)
        assert ev.min() > lo * (1 - 1e-9) and ev.max() < hi * (1 + 1e-9)


def test_centred_coated_sphere_isotropic_within_hs_bounds():
    N = 16
    ph = om.voxelize(I.centred_sphere(0.25), 0.25, N)
    K, res = om.effective_tensor(ph, K3)
    d = np.diag(K)
    # cubic symmetry of the grid makes K isotropic (up to the stopping tolerance)
    assert np.abs(d - d.mean()).max() < 1e-9 * d.mean()
    assert np.abs(K - np.diag(d)).max() < 1e-12 * d.mean()
    lo, hi = om.hashin_shtrikman_bounds(ph, K3)
    assert lo < d.mean() < hi
    assert all(r.converged and r.eps_eq < 1e-8 for r in res)


def test_metamorphic_shift_permute_scale():
    N = 10
    sl = I.generate_spheres(31, 4, 0.3)
    ph = om.voxelize(sl.spheres, 0.3, N)
    K, _ = om.effective_tensor(ph, K3)
    Ks, _ = om.effective_tensor(np.roll(ph, (3, -2, 5), axis=(0, 1, 2)), K3)
    assert np.abs(Ks - K).max() < 1e-7 * np.abs(K).max()
    # swapping grid axes x <-> z swaps tensor indices 0 <-> 2
    Kp, _ = om.effective_tensor(np.ascontiguousarray(np.transpose(ph, (2, 1, 0))), K3)
    perm = [2, 1, 0]
    assert np.abs(Kp - K[np.ix_(perm, perm)]).max() < 1e-7 * np.abs(K).max()
    Kx, _ = om.effective_tensor(ph, tuple(3.0 * k for k in K3))
    assert np.abs(Kx - 3.0 * K).max() < 1e-7 * np.abs(K).max()


def test_residuals_vanish_at_convergence():
    ph = I.random_phase_grid(41, 8)
    r = om.em_solve(ph, K3, (0.0, 0.0, 1.0), tol=1e-10, record=True)
    assert r.converged and r.eps_eq < 1e-10 and r.eps_comp_hist[-1] < 1e-10
    k = np.asarray(K3)[ph]
    eps, _ = om.equilibrium_residual(k, r.e, om.wavevectors(8))
    assert eps < 1e-10
    # compatibility: the mean gradient is the imposed one
    assert np.abs(r.e.mean(axis=(1, 2, 3)) - np.array([0, 0, 1.0])).max() < 1e-12


@pytest.mark.parametrize("N", [4, 6, 8])
def test_nyquist_rule_gives_real_trace_one_projectors(N):
    xi = om.wavevectors(N)
    xi2 = (xi * xi).sum(0)
    nz = xi2 > 0
    # xi' = 0 only at DC and at the 4 modes built from two or three Nyquist components
    assert nz.sum() == N ** 3 - 5
    h = N // 2
    for m in [(h, h, 0), (h, 0, h), (0, h, h), (h, h, h), (0, 0, 0)]:
        assert xi2[m] == 0
    for m in [(h, 0, 0), (0, h, 0), (0, 0, h)]:
        assert xi2[m] > 0
    # even in m: P(-m) = P(m)  <=> xi'(-m) = +-xi'(m)
    neg = np.roll(np.flip(xi, axis=(1, 2, 3)), 1, axis=(1, 2, 3))
    cross = np.cross(xi, neg, axis=0)
    assert np.abs(cross).max() < 1e-12
    # a real field stays real through the Green operator
    rng = np.random.default_rng(N)
    tau = rng.standard_normal((3, N, N, N))
    out = om.ifft3_unnorm(om.gamma0_apply(xi, -1.0, om.fft3(tau))) / N ** 3
    assert np.abs(out.imag).max() < 1e-12


def test_tau_form_identity():
    """(k + k0) e^{n+1} = (I - 2P)((k - k0) e^n) + 2 k0 E, the form used on the GPU."""
    N = 8
    ph = I.random_phase_grid(51, N)
    k = np.asarray(K3)[ph]
    k0 = om.reference_k0(K3)
    E = np.array([0.3, -0.5, 0.8])
    rng = np.random.default_rng(5)
    e = E[:, None, None, None] + 0.1 * rng.standard_normal((3, N, N, N))
    e1 = om.em_solve(ph, K3, E, max_iter=1, e0=e).e
    xi = om.wavevectors(N)
    s_hat = om.fft3((k - k0)[None] * e)
    refl = s_hat + 2.0 * k0 * om.gamma0_apply(xi, k0, s_hat) * (-1.0)
    refl[:, 0, 0, 0] += 2 * k0 * E * N ** 3
    tau1 = (om.ifft3_unnorm(refl) / N ** 3).real
    assert np.abs(tau1 - (k + k0)[None] * e1).max() < 1e-11 * np.abs(tau1).max()


# --- planted mistakes: each must be caught by one of the pins above -------------


def test_planted_sign_error_in_gamma_is_caught(monkeypatch):
    real = om.gamma0_apply
    monkeypatch.setattr(om, "gamma0_apply", lambda xi, L0, t: real(xi, -L0, t))
    ph = I.laminate_grid(6, 2)
    K, res = om.effective_tensor(ph, K3, max_iter=300)
    f = 2 / 6
    harm = 1.0 / (f / K3[2] + (1 - f) / K3[0])
    assert not (res[0].converged and abs(K[0, 0] - harm) < 1e-6 * harm)


def test_planted_dropped_nyquist_rule_is_caught(monkeypatch):
    real = om.wavevectors

    def naive(N):
        m = om.mode_indices(N)
        mz, my, mx = np.meshgrid(m, m, m, indexing="ij")
        return np.stack([2 * np.pi * mx / N, 2 * np.pi * my / N, 2 * np.pi * mz / N])

    monkeypatch.setattr(om, "wavevectors", naive)
    rng = np.random.default_rng(3)
    tau = rng.standard_normal((3, 6, 6, 6))
    out = om.ifft3_unnorm(om.gamma0_apply(om.wavevectors(6), -1.0, om.fft3(tau))) / 6 ** 3
    assert np.abs(out.imag).max() > 1e-6
    monkeypatch.setattr(om, "wavevectors", real)


def _tau_form_step(ph, e, E):
    N = ph.shape[0]
    k = np.asarray(K3)[ph]
    k0 = om.reference_k0(K3)
    xi = om.wavevectors(N)
    s_hat = om.fft3((k - k0)[None] * e)
    refl = s_hat - 2.0 * k0 * om.gamma0_apply(xi, k0, s_hat)
    refl[:, 0, 0, 0] += 2 * k0 * E * N ** 3
    return (om.ifft3_unnorm(refl) / N ** 3).real, k + k0


def test_planted_wrong_update_factor_is_caught():
    # step 7 with the factor 2 replaced by 1 keeps the fixed point (so K alone cannot
    # see it) but breaks the one-step identity pinned in test_tau_form_identity
    N = 8
    ph = I.random_phase_grid(51, N)
    E = np.array([0.3, -0.5, 0.8])
    e = E[:, None, None, None] + 0.1 * np.random.default_rng(5).standard_normal((3, N, N, N))
    e1 = om.em_solve(ph, K3, E, max_iter=1, e0=e).e
    e1_bad = e + 0.5 * (e1 - e)            # what factor 1 would have produced
    tau1, kk = _tau_form_step(ph, e, E)
    good = np.abs(tau1 - kk[None] * e1).max() / np.abs(tau1).max()
    bad = np.abs(tau1 - kk[None] * e1_bad).max() / np.abs(tau1).max()
    assert good < 1e-11 and bad > 1e-3
