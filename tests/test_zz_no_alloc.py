"""hmg_equilibrium_noalloc: the equilibrium residual for callers that cannot allocate
device memory (hosts whose own pool owns the device memory, or that must not risk an
allocation failure or cudaMalloc's implicit synchronization mid-run).  Its scratch is
static device memory, so it is checked here against hmg_equilibrium, which allocates,
on two calls in a row.  This file is collected last on purpose."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1504_07499_gb300 import hmg, inputs as I

K3 = I.K_PHASES
TOL = 1e-10          # FP64 equilibrium tolerance used by the parity tests


@pytest.fixture(scope="module")
def ctx():
    from paper_1504_07499_gb300 import build
    build.build()
    c = hmg.Context(0)
    yield c
    c.close()


def _field(N, seed):
    rng = np.random.default_rng(seed)
    E = np.array([1.0, 0.0, 0.0])
    return np.ascontiguousarray(E[:, None, None, None] + 0.2 * rng.standard_normal((3, N, N, N)))


@pytest.mark.parametrize("N", [16, 64])
def test_noalloc_matches_allocating_entry_point_twice(ctx, N):
    torch.cuda.set_device(0)
    ph = I.random_phase_grid(N, N, probs=(0.5, 0.2, 0.3))
    e = _field(N, N)
    ref_eps, ref_flux = hmg.hmg_equilibrium(ctx.handle, ph, N, K3, hmg.HMG_FP64, e)
    ph_d = torch.from_numpy(ph.reshape(-1)).cuda()
    e_d = torch.from_numpy(e.reshape(-1)).cuda()
    torch.cuda.synchronize()
    results = []
    free = []
    for call in range(2):
        eps, flux = hmg.hmg_equilibrium_noalloc(ph_d, N, K3, e_d)
        results.append((eps, flux))
        free.append(torch.cuda.mem_get_info()[0])
    for eps, flux in results:
        assert abs(eps - ref_eps) <= TOL * ref_eps
        assert np.abs(flux - ref_flux).max() <= TOL * np.abs(ref_flux).max()
    assert free[0] == free[1]           # the second call took no device memory
    # host inputs work too
    eps_h, flux_h = hmg.hmg_equilibrium_noalloc(ph, N, K3, e)
    assert abs(eps_h - ref_eps) <= TOL * ref_eps


def test_noalloc_rejects_sizes_beyond_its_static_scratch():
    N = 2 * hmg.HMG_NOALLOC_MAX_N
    ph = np.zeros((N, N, N), np.uint8)
    e = np.zeros((3, N, N, N))
    with pytest.raises(hmg.HmgError) as err:
        hmg.hmg_equilibrium_noalloc(ph, N, K3, e)
    assert err.value.status == hmg.HMG_INVALID_ARG
    assert "static scratch" in str(err.value)
