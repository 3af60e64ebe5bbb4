"""The augmented Lagrangian scheme (hmg_solve_scheme with HMG_SCHEME_AUGMENTED_LAGRANGIAN)
and the relaxed polarization iteration (hmg_solve_polarization) on the GPU against the
oracle's al_solve and em_solve(beta): plain FP64 (K to 1e-9, the oracle's sweep counts
+-1) on the generic kernels, FP32 bulk (K to 1e-5, fields to 1e-4 relative L2) on the
generic and the register-resident kernels; beta = 2 is exactly the accelerated scheme;
bad relaxations are rejected."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import em as om
from paper_1504_07499_gb300 import hmg, inputs as I

from test_gpu_parity import kerr

K3 = (0.20, 0.25, 40.0)    # contrast 200


@pytest.fixture(scope="module")
def ctx():
    from paper_1504_07499_gb300 import build
    build.build()
    c = hmg.Context(0)
    yield c
    c.close()


def _grid(N, seed=1000):
    sl = I.generate_spheres(seed, 20, 0.3)
    return om.voxelize(sl.spheres, 0.3, N)


@pytest.mark.parametrize("N", [16, 24])
def test_al_fp64_matches_oracle(ctx, N):
    ph = _grid(N)
    Kref, res = om.al_effective_tensor(ph, K3, tol=1e-8)
    e = np.empty((3, 3, N, N, N))
    K, info, st = hmg.hmg_solve_scheme(ctx.handle, ph, N, K3, 1e-8, hmg.HMG_FP64, hmg.HMG_SCHEME_AUGMENTED_LAGRANGIAN, e)
    assert st == hmg.HMG_OK
    assert kerr(K, Kref) < 1e-9
    for j in range(3):
        assert abs(info["iters"][j] - res[j].iters) <= 1
        assert np.abs(e[j] - res[j].e).max() < 1e-9 * np.abs(res[j].e).max()


@pytest.mark.parametrize("N,beta", [(16, 1.5), (24, 0.7)])
def test_polarization_fp64_matches_oracle(ctx, N, beta):
    ph = _grid(N, 1001)
    Kref, res = om.effective_tensor(ph, K3, tol=1e-8, beta=beta)
    K, info, st = hmg.hmg_solve_polarization(ctx.handle, ph, N, K3, 1e-8, hmg.HMG_FP64, beta)
    assert st == hmg.HMG_OK
    assert kerr(K, Kref) < 1e-9
    for j in range(3):
        assert abs(info["iters"][j] - res[j].iters) <= 1


@pytest.mark.parametrize("N", [48, 64])
def test_al_fp32bulk_matches_oracle(ctx, N):
    ph = _grid(N)
    Kref, res = om.al_effective_tensor(ph, K3, tol=1e-8)
    e = np.empty((3, 3, N, N, N))
    K, info, st = hmg.hmg_solve_scheme(ctx.handle, ph, N, K3, 1e-8, hmg.HMG_FP32_BULK,
                                       hmg.HMG_SCHEME_AUGMENTED_LAGRANGIAN, e)
    assert st == hmg.HMG_OK
    assert kerr(K, Kref) < 1e-5
    for j in range(3):
        assert np.linalg.norm(e[j] - res[j].e) < 1e-4 * np.linalg.norm(res[j].e)
        assert info["eps_eq"][j] < 1e-8


def test_polarization_fp32bulk_matches_oracle(ctx):
    N, beta = 64, 1.5
    ph = _grid(N, 1002)
    Kref, res = om.effective_tensor(ph, K3, tol=1e-8, beta=beta)
    e = np.empty((3, 3, N, N, N))
    K, info, st = hmg.hmg_solve_polarization(ctx.handle, ph, N, K3, 1e-8, hmg.HMG_FP32_BULK, beta, e)
    assert st == hmg.HMG_OK
    assert kerr(K, Kref) < 1e-5
    for j in range(3):
        assert np.linalg.norm(e[j] - res[j].e) < 1e-4 * np.linalg.norm(res[j].e)


def test_beta_two_is_the_accelerated_scheme(ctx):
    N = 64
    ph = _grid(N, 1003)
    Kp, ip, _ = hmg.hmg_solve_polarization(ctx.handle, ph, N, K3, 1e-8, hmg.HMG_FP32_BULK, 2.0)
    Ke, ie, _ = hmg.hmg_solve(ctx.handle, ph, N, K3, 1e-8, hmg.HMG_FP32_BULK)
    assert np.array_equal(Kp, Ke) and list(ip["iters"]) == list(ie["iters"])
    Ka, ia, _ = hmg.hmg_solve_scheme(ctx.handle, ph, N, K3, 1e-8, hmg.HMG_FP32_BULK,
                                     hmg.HMG_SCHEME_AUGMENTED_LAGRANGIAN)
    assert kerr(Ka, Ke) < 1e-5
    assert min(ia["iters"]) > max(ie["iters"])   # half steps: more sweeps


@pytest.mark.parametrize("beta", [0.0, -1.0, 2.5, float("nan")])
def test_bad_relaxation_is_rejected(ctx, beta):
    ph = _grid(16)
    with pytest.raises(hmg.HmgError) as ex:
        hmg.hmg_solve_polarization(ctx.handle, ph, 16, K3, 1e-8, hmg.HMG_FP64, beta)
    assert ex.value.status == hmg.HMG_INVALID_ARG
