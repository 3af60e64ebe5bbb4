"""The basic scheme on the GPU (hmg_solve_scheme with HMG_SCHEME_BASIC) against the
oracle's basic scheme: plain FP64 (K to 1e-9, the same sweep counts +-1) on the
generic kernels, FP32 bulk (K to 1e-5, fields to 1e-4 relative L2) on the generic and
the register-resident kernels, agreement with the accelerated scheme, bad arguments."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import em as om
from paper_1504_07499_gb300 import hmg, inputs as I

from test_gpu_parity import kerr

K3 = (0.20, 0.25, 4.0)    # contrast 20


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
def test_basic_fp64_matches_oracle(ctx, N):
    ph = _grid(N)
    Kref, res = om.basic_effective_tensor(ph, K3, tol=1e-8)
    K, info, st = hmg.hmg_solve_scheme(ctx.handle, ph, N, K3, 1e-8, hmg.HMG_FP64, hmg.HMG_SCHEME_BASIC)
    assert st == hmg.HMG_OK
    assert kerr(K, Kref) < 1e-9
    for j in range(3):
        assert abs(info["iters"][j] - res[j].iters) <= 1
        assert info["eps_eq"][j] < 1e-8


@pytest.mark.parametrize("N", [48, 64, 96])
def test_basic_fp32bulk_matches_oracle(ctx, N):
    ph = _grid(N)
    Kref, res = om.basic_effective_tensor(ph, K3, tol=1e-8)
    e = np.empty((3, 3, N, N, N))
    K, info, st = hmg.hmg_solve_scheme(ctx.handle, ph, N, K3, 1e-8, hmg.HMG_FP32_BULK, hmg.HMG_SCHEME_BASIC, e)
    assert st == hmg.HMG_OK
    assert kerr(K, Kref) < 1e-5
    for j in range(3):
        assert np.linalg.norm(e[j] - res[j].e) < 1e-4 * np.linalg.norm(res[j].e)
        assert info["eps_eq"][j] < 1e-8


def test_basic_and_accelerated_agree(ctx):
    N = 64
    ph = _grid(N, 1001)
    Kb, ib, _ = hmg.hmg_solve_scheme(ctx.handle, ph, N, K3, 1e-8, hmg.HMG_FP32_BULK, hmg.HMG_SCHEME_BASIC)
    Ke, ie, _ = hmg.hmg_solve_scheme(ctx.handle, ph, N, K3, 1e-8, hmg.HMG_FP32_BULK, hmg.HMG_SCHEME_EYRE_MILTON)
    assert kerr(Kb, Ke) < 1e-5
    assert min(ib["iters"]) > max(ie["iters"])   # the basic scheme needs more sweeps
    Kp, _, _ = hmg.hmg_solve(ctx.handle, ph, N, K3, 1e-8, hmg.HMG_FP32_BULK)
    assert np.array_equal(Kp, Ke)                  # Eyre-Milton is exactly hmg_solve


def test_unknown_scheme_is_rejected(ctx):
    ph = _grid(16)
    with pytest.raises(hmg.HmgError) as ex:
        hmg.hmg_solve_scheme(ctx.handle, ph, 16, K3, 1e-8, hmg.HMG_FP64, 7)
    assert ex.value.status == hmg.HMG_INVALID_ARG
