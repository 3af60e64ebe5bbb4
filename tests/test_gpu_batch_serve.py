"""Many RVEs at once: hmg_solve_batch (one CUDA-graph launch advances every RVE) and the
continuous-batching request loop behind hmg_submit / hmg_poll.

The engine runs each gradient through the same sequence of sweeps as a single solve
(per-gradient arithmetic never mixes RVEs), so results are compared with single solves
at the FP32-bulk tolerance (1e-5 per K entry) and with the oracle for one entry.
"""
import time

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import em as om
from paper_1504_07499_gb300 import hmg, inputs as I

from test_gpu_parity import kerr


@pytest.fixture(scope="module")
def ctx():
    from paper_1504_07499_gb300 import build
    build.build()
    c = hmg.Context(0)
    yield c
    c.close()


def _rves():
    """Mixed sizes: a generic-kernel size (32), register-path sizes (64, 96) and a size
    with the fused cluster kernels (128)."""
    out = []
    for i, (N, n, f, layer, kc) in enumerate([(32, 8, 0.25, 0.3, 400.0), (64, 20, 0.3, 0.2, 40.0),
                                              (32, 5, 0.2, 0.5, 4000.0), (96, 30, 0.25, 0.3, 400.0),
                                              (64, 12, 0.35, 0.4, 400.0), (128, 30, 0.2, 0.3, 400.0)]):
        sl = I.generate_spheres(100 + i, n, f)
        out.append((om.voxelize(sl.spheres, layer, N), N, (0.20, 0.25, kc)))
    return out


def test_batch_matches_single_solves_and_oracle(ctx):
    rves = _rves()
    phases = [r[0] for r in rves]
    Ns = [r[1] for r in rves]
    k3 = np.array([r[2] for r in rves])
    K, infos, st = hmg.hmg_solve_batch(ctx.handle, phases, Ns, k3, 1e-8, hmg.HMG_FP32_BULK)
    assert st == hmg.HMG_OK
    for i, (ph, N, k) in enumerate(rves):
        Ks, _, _ = ctx.solve(ph, k, 1e-8, hmg.HMG_FP32_BULK)
        assert kerr(K[i], Ks) < 1e-5, i
        assert all(e < 1e-8 for e in infos[i]["eps_eq"])
    Kref, _ = om.effective_tensor(rves[0][0], rves[0][2], tol=1e-8)
    assert kerr(K[0], Kref) < 1e-5


def test_batch_fp64_is_the_plain_method(ctx):
    rves = _rves()[:2]
    K, infos, st = hmg.hmg_solve_batch(ctx.handle, [r[0] for r in rves], [r[1] for r in rves],
                                       np.array([r[2] for r in rves]), 1e-8, hmg.HMG_FP64)
    for i, (ph, N, k) in enumerate(rves):
        Ks, _, _ = ctx.solve(ph, k, 1e-8, hmg.HMG_FP64)
        assert np.array_equal(K[i], Ks)


def _wait(handle, tickets, timeout=300):
    res = {}
    t0 = time.time()
    while len(res) < len(tickets):
        for t in tickets:
            if t in res:
                continue
            st, K, info = hmg.hmg_poll(handle, t)
            if st != hmg.HMG_PENDING:
                res[t] = (st, K, info)
        assert time.time() - t0 < timeout
        time.sleep(0.005)
    return res


def test_serving_same_alone_and_in_the_mix():
    rves = _rves()
    with hmg.Context(0) as alone_ctx:
        alone = {}
        for i, (ph, N, k) in enumerate(rves):
            t = hmg.hmg_submit(alone_ctx.handle, ph, N, k, 1e-8, hmg.HMG_FP32_BULK)
            alone[i] = _wait(alone_ctx.handle, [t])[t]
        assert hmg.hmg_server_stats(alone_ctx.handle)["max_resident"] == 1
    with hmg.Context(0) as mix_ctx:
        tickets = [hmg.hmg_submit(mix_ctx.handle, ph, N, k, 1e-8, hmg.HMG_FP32_BULK) for ph, N, k in rves]
        res = _wait(mix_ctx.handle, tickets)
        stats = hmg.hmg_server_stats(mix_ctx.handle)
    assert stats["completed"] == len(rves) and stats["max_resident"] > 1
    assert stats["graph_launches"] > 0
    for i, t in enumerate(tickets):
        st, K, info = res[t]
        assert st == hmg.HMG_OK
        assert kerr(K, alone[i][1]) < 1e-5
        assert info["eps_eq"][0] < 1e-8


def test_serving_admits_as_memory_frees_up():
    N = 64
    budget = int(2.5 * hmg.hmg_footprint(N, hmg.HMG_FP32_BULK))   # two requests at a time
    rves = [r for r in _rves() if r[1] == N]
    reqs = rves * 2
    with hmg.Context(0, budget) as c:
        tickets = [hmg.hmg_submit(c.handle, ph, N, k, 1e-8, hmg.HMG_FP32_BULK) for ph, _, k in reqs]
        res = _wait(c.handle, tickets)
        stats = hmg.hmg_server_stats(c.handle)
        assert all(res[t][0] == hmg.HMG_OK for t in tickets)
        assert stats["max_resident"] == 2
        assert kerr(res[tickets[0]][1], res[tickets[2]][1]) < 1e-12   # same input, same result
        # a request that cannot fit the budget at all is refused at submit time
        with pytest.raises(hmg.HmgError) as e:
            ph = np.zeros((256, 256, 256), np.uint8)
            hmg.hmg_submit(c.handle, ph, 256, (0.2, 0.25, 400.0), 1e-8, hmg.HMG_FP32_BULK)
        assert e.value.status == hmg.HMG_OUT_OF_MEMORY


def test_poll_unknown_ticket(ctx):
    with pytest.raises(hmg.HmgError) as e:
        hmg.hmg_poll(ctx.handle, 987654321)
    assert e.value.status == hmg.HMG_UNKNOWN_TICKET


def test_small_requests_do_not_wait_for_a_large_one(ctx):
    """Large (192^3 and up) and small grids run in separate lanes of the request loop:
    small requests submitted after a large one finish first, and every result equals the
    single solve of its grid."""
    big_ph = om.voxelize(I.generate_spheres(3000, 100, 0.40).spheres, 0.3, 192)
    small = [(ph, N, k) for ph, N, k in _rves() if N == 64]
    with hmg.Context(0) as c:
        tb = hmg.hmg_submit(c.handle, big_ph, 192, I.K_PHASES, 1e-8, hmg.HMG_FP32_BULK)
        ts = [hmg.hmg_submit(c.handle, ph, N, k, 1e-8, hmg.HMG_FP32_BULK) for ph, N, k in small]
        res = _wait(c.handle, [tb] + ts)
    assert all(res[t][0] == hmg.HMG_OK for t in [tb] + ts)
    assert max(res[t][2]["seconds"] for t in ts) < res[tb][2]["seconds"]
    Kb, _, _ = ctx.solve(big_ph, I.K_PHASES, 1e-8, hmg.HMG_FP32_BULK)
    assert kerr(res[tb][1], Kb) < 1e-5
    for (ph, N, k), t in zip(small, ts):
        Ks, _, _ = ctx.solve(ph, k, 1e-8, hmg.HMG_FP32_BULK)
        assert kerr(res[t][1], Ks) < 1e-5
