"""Sphere placement on the GPU (hmg_rsa, hmg_rve) against the library's seeded host
generator (paper_1504_07499_gb300/inputs.py, the reference for the placement rule):
the same sphere lists bit for bit -- plain RSA and, above the jamming limit, the
reduced-radius RSA with growth sweeps -- and the same phase grids as the oracle's
voxelization of the host list; bounded failure; bad arguments."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import em as om
from paper_1504_07499_gb300 import hmg, inputs as I


@pytest.fixture(scope="module")
def ctx():
    from paper_1504_07499_gb300 import build
    build.build()
    c = hmg.Context(0)
    yield c
    c.close()


CASES = [(3000, 100, 0.40), (1000, 30, 0.20), (1, 3, 0.3), (7, 50, 0.35), (11, 100, 0.3), (12, 10, 0.4),
         (4005, 64, 0.31), (6001, 70, 0.3), (5, 1, 0.2)]


@pytest.mark.parametrize("seed,n,f", CASES)
def test_device_placement_equals_host_generator(ctx, seed, n, f):
    ref = I.generate_spheres(seed, n, f)
    got, gen = hmg.hmg_rsa(ctx.handle, seed, n, I.sphere_radius(n, f))
    assert np.array_equal(got, ref.spheres)
    assert gen == (0 if ref.generator == "rsa" else 1)


def test_device_placement_into_device_memory(ctx):
    seed, n, f = 3000, 100, 0.40
    out = torch.empty((n, 4), dtype=torch.float64, device="cuda")
    hmg.hmg_rsa(ctx.handle, seed, n, I.sphere_radius(n, f), spheres_out=out)
    assert np.array_equal(out.cpu().numpy(), I.generate_spheres(seed, n, f).spheres)


@pytest.mark.parametrize("seed,n,f,layer,N", [(3000, 100, 0.40, 0.3, 256), (1000, 30, 0.20, 0.3, 128),
                                             (12, 10, 0.4, 0.9, 24)])
def test_device_rve_equals_oracle_voxelization(ctx, seed, n, f, layer, N):
    ref = I.generate_spheres(seed, n, f)
    ph = torch.empty(N ** 3, dtype=torch.uint8, device="cuda")
    sph = np.empty((n, 4))
    gen = hmg.hmg_rve(ctx.handle, seed, n, I.sphere_radius(n, f), layer, N, ph, spheres_out=sph)
    assert np.array_equal(sph, ref.spheres)
    assert (ph.cpu().numpy().reshape(N, N, N) == om.voxelize(ref.spheres, layer, N)).all()
    assert gen == (0 if ref.generator == "rsa" else 1)


def test_impossible_packing_fails_with_a_status(ctx):
    # 100 spheres of radius 0.2 cannot fit the unit cell: both placement steps give up
    with pytest.raises(hmg.HmgError) as ex:
        hmg.hmg_rsa(ctx.handle, 9, 100, 0.2, max_candidates=20000)
    assert ex.value.status == hmg.HMG_NOT_CONVERGED
    # the context stays usable
    got, _ = hmg.hmg_rsa(ctx.handle, 1, 3, I.sphere_radius(3, 0.3))
    assert np.array_equal(got, I.generate_spheres(1, 3, 0.3).spheres)


@pytest.mark.parametrize("n,r,cap", [(0, 0.1, 1000), (2000, 0.01, 1000), (5, 0.0, 1000), (5, 0.5, 1000),
                                     (5, 0.1, 0), (5, float("nan"), 1000)])
def test_bad_arguments_are_rejected(ctx, n, r, cap):
    with pytest.raises(hmg.HmgError) as ex:
        hmg.hmg_rsa(ctx.handle, 1, n, r, max_candidates=cap, spheres_out=np.empty((max(n, 1), 4)))
    assert ex.value.status == hmg.HMG_INVALID_ARG


def test_served_rve_requests_match_solves_of_the_host_generated_grids(ctx):
    """hmg_submit_rve: the request loop places, voxelizes and solves on the device; each
    K equals (within the FP32-bulk tolerance) the solve of the host generator's grid."""
    from test_gpu_parity import kerr
    k = (0.20, 0.25, 40.0)
    reqs = [(4001, 40, 0.3, 0.3, 64), (4002, 60, 0.35, 0.2, 96), (3000, 100, 0.40, 0.3, 64)]
    with hmg.Context(0) as srv:
        tickets = [hmg.hmg_submit_rve(srv.handle, s, n, I.sphere_radius(n, f), l, N, k, 1e-8, hmg.HMG_FP32_BULK)
                   for s, n, f, l, N in reqs]
        out = {}
        import time
        t0 = time.time()
        while len(out) < len(tickets) and time.time() - t0 < 300:
            for t in tickets:
                if t not in out:
                    st, K, info = hmg.hmg_poll(srv.handle, t)
                    if st != hmg.HMG_PENDING:
                        out[t] = (st, K)
            time.sleep(0.01)
    assert len(out) == len(tickets)
    for (s, n, f, l, N), t in zip(reqs, tickets):
        st, K = out[t]
        assert st == hmg.HMG_OK
        ph = om.voxelize(I.generate_spheres(s, n, f).spheres, l, N)
        Kref, _, _ = hmg.hmg_solve(ctx.handle, ph, N, k, 1e-8, hmg.HMG_FP32_BULK)
        assert kerr(K, Kref) < 1e-5
