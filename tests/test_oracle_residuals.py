"""Pins for the scales of the two residuals of the §3 Algorithm, which decide when
every solve stops: the equilibrium residual of step 1 (its wavevector scale
xi = 2 pi m / N and the normalization phi_hat = DFT(phi) / N^3) and the compatibility
residual of step 6 (a mean over voxels, divided by |grad Theta|).

The projector P = xi xi^T / |xi|^2 is blind to the scale of xi, and a contraction
ratio is blind to a constant factor in eps_comp, so the other oracle pins cannot see
these scales.  Here each residual is compared with a value worked out by hand for a
field whose spectrum has only a few modes, and planted mistakes (xi = m without
2 pi / N, |xi| in place of the divergence, a sum in place of the mean) must fail.
"""
import math

import numpy as np
import pytest

from oracle import em as om
from paper_1504_07499_gb300 import inputs as I


def _cos_field(N, m, comp, a, b):
    """k = 1 and e chosen so that phi = -k e has phi_comp = a + b cos(2 pi (m . x) / N)
    varying along the grid axes listed in `m` (x, y, z), other components 0."""
    z, y, x = np.indices((N, N, N))
    arg = 2 * np.pi * (m[0] * x + m[1] * y + m[2] * z) / N
    phi = np.zeros((3, N, N, N))
    phi[comp] = a + b * np.cos(arg)
    return np.ones((N, N, N)), -phi


@pytest.mark.parametrize("N,m,comp,a,b", [
    (8, (1, 0, 0), 0, 2.0, 0.5),      # phi_x varies along x: full divergence
    (12, (3, 0, 0), 0, -1.5, 0.25),
    (10, (0, 2, 0), 1, 0.7, -0.3),    # phi_y along y
    (9, (0, 0, 4), 2, 1.0, 0.125),    # odd N, phi_z along z
    (12, (2, 5, 0), 0, 1.25, 0.4),    # oblique mode: only xi_x enters the divergence
])
def test_equilibrium_residual_of_one_cosine_mode(N, m, comp, a, b):
    # phi_hat(0) = a e_comp and phi_hat(+-m) = b/2 e_comp, so
    # xi . phi_hat(+-m) = +-(2 pi m_comp / N) b / 2 and
    # eps_eq = sqrt(2 (2 pi m_comp / N)^2 b^2 / 4) / |a| = (2 pi m_comp / N) |b| / (sqrt 2 |a|)
    k, e = _cos_field(N, m, comp, a, b)
    eps, mean = om.equilibrium_residual(k, e, om.wavevectors(N))
    expect = (2 * np.pi * m[comp] / N) * abs(b) / (math.sqrt(2.0) * abs(a))
    assert abs(eps - expect) <= 1e-12 * expect
    ref_mean = np.zeros(3)
    ref_mean[comp] = a
    assert np.abs(mean - ref_mean).max() < 1e-13


def test_equilibrium_residual_of_divergence_free_flux_is_zero():
    # phi_x varies along y only: xi . phi_hat = xi_x phi_hat_x = 0 at modes (0, m, 0),
    # although |xi| |phi_hat| is not zero there (the divergence, not a norm, reading)
    k, e = _cos_field(12, (0, 3, 0), 0, 1.0, 0.5)
    eps, _ = om.equilibrium_residual(k, e, om.wavevectors(12))
    assert eps < 1e-14


def test_equilibrium_residual_with_two_components():
    # phi = (a + b cos(2 pi m x / N), c, c' cos(2 pi m' z / N)):
    # eps_eq^2 = [(2 pi m/N)^2 b^2 + (2 pi m'/N)^2 c'^2] / 2 / (a^2 + c^2)
    N, m, mp, a, b, c, cp = 16, 3, 5, 1.1, 0.3, -0.8, 0.2
    z, y, x = np.indices((N, N, N))
    phi = np.zeros((3, N, N, N))
    phi[0] = a + b * np.cos(2 * np.pi * m * x / N)
    phi[1] = c
    phi[2] = cp * np.cos(2 * np.pi * mp * z / N)
    kk = np.full((N, N, N), 2.0)  # e = -phi / k
    eps, _ = om.equilibrium_residual(kk, -phi / 2.0, om.wavevectors(N))
    xm, xmp = 2 * np.pi * m / N, 2 * np.pi * mp / N
    expect = math.sqrt((xm ** 2 * b ** 2 + xmp ** 2 * cp ** 2) / 2.0 / (a * a + c * c))
    assert abs(eps - expect) <= 1e-12 * expect


@pytest.mark.parametrize("N,thick,axis,Emag", [(8, 3, 0, 1.0), (12, 5, 2, 2.0), (9, 4, 1, 0.5)])
def test_first_compatibility_residual_of_a_laminate(N, thick, axis, Emag):
    # e^0 = E across the layers: tau = (k - k0) E is a function of the layer
    # coordinate only, its modes lie on that axis where P = e_axis e_axis^T, so
    # e_comp = E - (tau - <tau>) / k0 and e^0 - e_comp = (k - <k>) E / k0:
    # eps_comp^1 = std(k) |E| / (k0 |E|) = |k_a - k_b| sqrt(f (1 - f)) / k0.
    K3 = (0.20, 0.25, 400.0)
    ph = I.laminate_grid(N, thick, axis=axis, phase_a=2, phase_b=0)
    E = np.zeros(3)
    E[axis] = Emag
    r = om.em_solve(ph, K3, E, tol=1e-30, max_iter=1, record=True)
    f = thick / N
    expect = abs(K3[2] - K3[0]) * math.sqrt(f * (1 - f)) / om.reference_k0(K3)
    assert abs(r.eps_comp_hist[0] - expect) <= 1e-12 * expect
    # along the layers the first compatible field is E itself
    E2 = np.zeros(3)
    E2[(axis + 1) % 3] = Emag
    r2 = om.em_solve(ph, K3, E2, tol=1e-30, max_iter=1, record=True)
    assert r2.eps_comp_hist[0] < 1e-14


def test_first_compatibility_residual_of_the_basic_scheme():
    # the basic scheme's first sweep gives the same compatible field formula with its
    # own reference k0 = (min k + max k) / 2
    K3 = (0.20, 0.25, 400.0)
    N, thick = 10, 3
    ph = I.laminate_grid(N, thick, axis=0, phase_a=2, phase_b=0)
    r = om.basic_solve(ph, K3, (1.0, 0.0, 0.0), tol=1e-30, max_iter=1, record=True)
    f = thick / N
    expect = abs(K3[2] - K3[0]) * math.sqrt(f * (1 - f)) / om.basic_reference_k0(K3)
    assert abs(r.eps_comp_hist[0] - expect) <= 1e-12 * expect


# --- planted mistakes: each must fail one of the pins above --------------------


def test_planted_wavevector_without_two_pi_over_N_is_caught(monkeypatch):
    real = om.wavevectors
    monkeypatch.setattr(om, "wavevectors", lambda N: real(N) * N / (2 * np.pi))
    N, m, a, b = 12, (3, 0, 0), -1.5, 0.25
    k, e = _cos_field(N, m, 0, a, b)
    eps, _ = om.equilibrium_residual(k, e, om.wavevectors(N))
    expect = (2 * np.pi * m[0] / N) * abs(b) / (math.sqrt(2.0) * abs(a))
    assert abs(eps - expect) > 0.1 * expect


def test_planted_norm_in_place_of_divergence_is_caught(monkeypatch):
    # |xi| |phi_hat| instead of xi . phi_hat: the divergence-free flux is no longer 0
    def norm_form(k_field, e, xi):
        N = e.shape[-1]
        phi_hat = om.fft3(-k_field[None] * e) / N ** 3
        nrm = np.sqrt((xi * xi).sum(0)) * np.sqrt((np.abs(phi_hat) ** 2).sum(0))
        nrm[0, 0, 0] = 0.0
        mean = phi_hat[:, 0, 0, 0].real
        return math.sqrt(float((nrm ** 2).sum())) / float(np.linalg.norm(mean)), mean

    monkeypatch.setattr(om, "equilibrium_residual", norm_form)
    k, e = _cos_field(12, (0, 3, 0), 0, 1.0, 0.5)
    eps, _ = om.equilibrium_residual(k, e, om.wavevectors(12))
    assert eps > 1e-3


def test_planted_sum_in_place_of_mean_is_caught(monkeypatch):
    monkeypatch.setattr(om, "compatibility_residual",
                        lambda e, ec, normE: math.sqrt(float(((e - ec) ** 2).sum())) / normE)
    K3 = (0.20, 0.25, 400.0)
    N, thick = 8, 3
    ph = I.laminate_grid(N, thick, axis=0, phase_a=2, phase_b=0)
    r = om.em_solve(ph, K3, (1.0, 0.0, 0.0), tol=1e-30, max_iter=1, record=True)
    f = thick / N
    expect = abs(K3[2] - K3[0]) * math.sqrt(f * (1 - f)) / om.reference_k0(K3)
    assert abs(r.eps_comp_hist[0] - expect) > 0.1 * expect


def test_planted_missing_gradient_normalization_is_caught(monkeypatch):
    monkeypatch.setattr(om, "compatibility_residual",
                        lambda e, ec, normE: math.sqrt(float(((e - ec) ** 2).sum(0).mean())))
    K3 = (0.20, 0.25, 400.0)
    ph = I.laminate_grid(12, 5, axis=2, phase_a=2, phase_b=0)
    r = om.em_solve(ph, K3, (0.0, 0.0, 2.0), tol=1e-30, max_iter=1, record=True)
    f = 5 / 12
    expect = abs(K3[2] - K3[0]) * math.sqrt(f * (1 - f)) / om.reference_k0(K3)
    assert abs(r.eps_comp_hist[0] - expect) > 0.1 * expect
