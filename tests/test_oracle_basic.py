"""Pins for the oracle's basic scheme (§3 names it among the FFT-based schemes; it
iterates the Lippmann-Schwinger equation of eqs. 1-3 with a positive reference medium):
the homogeneous medium, laminate closed forms, a dense direct solve of the discrete cell
problem (the same discrete solution as the accelerated scheme), the contraction rate
(c - 1)/(c + 1), and planted mistakes that these pins must catch."""
import math

import numpy as np
import pytest

from oracle import em as om
from paper_1504_07499_gb300 import inputs as I

K3 = (0.20, 0.25, 4.0)        # contrast 20: a few hundred basic sweeps


def test_reference_is_the_centre_of_the_range():
    assert om.basic_reference_k0((0.2, 0.25, 4.0)) == pytest.approx(2.1, abs=1e-15)
    assert om.basic_reference_k0((3.0, 1.0, 2.0)) == 2.0


def test_homogeneous_medium_is_exact():
    ph = I.random_phase_grid(5, 8)
    K, res = om.basic_effective_tensor(ph, (1.7, 1.7, 1.7))
    assert np.abs(K - 1.7 * np.eye(3)).max() < 1e-13
    for r in res:
        assert r.iters == 1 and r.converged


@pytest.mark.parametrize("N,thick,axis", [(6, 2, 0), (9, 4, 2), (10, 3, 1)])
def test_laminate_means(N, thick, axis):
    ph = I.laminate_grid(N, thick, axis=axis, phase_a=2, phase_b=0)
    K, _ = om.basic_effective_tensor(ph, K3, tol=1e-11)
    f = thick / N
    ka, kb = K3[2], K3[0]
    harm = 1.0 / (f / ka + (1 - f) / kb)
    arith = f * ka + (1 - f) * kb
    for i in range(3):
        assert K[i, i] == pytest.approx(harm if i == axis else arith, rel=1e-9)
    assert np.abs(K - np.diag(np.diag(K))).max() < 1e-9 * arith


@pytest.mark.parametrize("N,seed", [(3, 1), (4, 2), (5, 3), (6, 4)])
def test_matches_dense_direct_solve(N, seed):
    ph = I.random_phase_grid(seed, N)
    K, _ = om.basic_effective_tensor(ph, K3, tol=1e-12)
    assert np.abs(K - om.direct_solve(ph, K3)).max() < 1e-9 * np.abs(K).max()


def test_same_solution_as_the_accelerated_scheme():
    ph = om.voxelize(I.centred_sphere(0.25), 0.25, 8)
    Kb, rb = om.basic_effective_tensor(ph, K3, tol=1e-10)
    Ke, re = om.effective_tensor(ph, K3, tol=1e-10)
    assert np.abs(Kb - Ke).max() < 1e-8 * np.abs(Ke).max()
    # and the basic scheme needs more sweeps at this contrast
    assert min(r.iters for r in rb) > max(r.iters for r in re)


def test_contraction_rate_of_eps_comp():
    """|e^{n+1} - e^{n+2}| <= rho |e^n - e^{n+1}| with rho = (c - 1)/(c + 1): the step
    error map is -P Y with |Y| = |k - k0| / k0 <= rho and P an orthogonal projector."""
    ph = I.random_phase_grid(7, 8)
    c = max(K3) / min(K3)
    rho = (c - 1) / (c + 1)
    r = om.basic_solve(ph, K3, (1.0, 0.0, 0.0), tol=0.0, max_iter=60, record=True)
    h = r.eps_comp_hist
    assert all(h[n + 1] <= rho * h[n] * (1 + 1e-10) for n in range(len(h) - 1))
    # and the bound is nearly attained: the rate is close to rho, far above the
    # accelerated scheme's (sqrt c - 1)/(sqrt c + 1)
    assert h[-1] / h[-2] > (math.sqrt(c) - 1) / (math.sqrt(c) + 1)


# --- planted mistakes: each must be caught by one of the pins above -------------


def test_planted_negative_reference_is_caught(monkeypatch):
    """The accelerated scheme's sign of L0 makes the plain iteration diverge."""
    monkeypatch.setattr(om, "basic_reference_k0", lambda k: -0.5 * (min(k) + max(k)))
    ph = I.random_phase_grid(2, 4)
    r = om.basic_solve(ph, K3, (1.0, 0.0, 0.0), tol=1e-10, max_iter=300, record=True)
    assert not r.converged or np.abs(-r.flux_mean - om.direct_solve(ph, K3)[:, 0]).max() > 1e-6


def test_planted_wrong_reference_value_changes_only_the_rate(monkeypatch):
    """A different positive k0 converges to the same K (the fixed point does not depend
    on k0) -- the dense-solve pin stays green -- but the contraction pin catches a k0
    below the centre of the range (rate above rho)."""
    ph = I.random_phase_grid(7, 8)
    monkeypatch.setattr(om, "basic_reference_k0", lambda k: 0.75 * (min(k) + max(k)))
    K, _ = om.basic_effective_tensor(I.random_phase_grid(2, 4), K3, tol=1e-12)
    assert np.abs(K - om.direct_solve(I.random_phase_grid(2, 4), K3)).max() < 1e-8
    monkeypatch.setattr(om, "basic_reference_k0", lambda k: 0.3 * (min(k) + max(k)))
    c = max(K3) / min(K3)
    rho = (c - 1) / (c + 1)
    r = om.basic_solve(ph, K3, (1.0, 0.0, 0.0), tol=0.0, max_iter=40, record=True)
    h = r.eps_comp_hist
    assert any(h[n + 1] > rho * h[n] * (1 + 1e-10) for n in range(len(h) - 1))
