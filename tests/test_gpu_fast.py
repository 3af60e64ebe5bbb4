"""The register-resident FP32 kernels (grid sizes 64, 96, 128, 192, 256) against the
oracle, including the benchmark's full 256^3 size (one sweep, all voxels compared).

Tolerances as in test_gpu_parity: FP32 transforms 2e-6 of the largest coefficient,
FP32 sweeps 1e-5 relative, FP32-bulk solves 1e-5 on K and 1e-4 relative L2 on the field.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import em as om
from paper_1504_07499_gb300 import hmg, inputs as I

from test_gpu_parity import kerr, unpack_spectrum

K3 = I.K_PHASES


@pytest.fixture(scope="module")
def ctx():
    from paper_1504_07499_gb300 import build
    build.build()
    c = hmg.Context(0)
    yield c
    c.close()


@pytest.fixture(params=[0, 1, 2, 3], ids=["z0", "z1", "z0-fusedxy", "z1-fusedxy"])
def zvar(request, ctx):
    """Runs a test once per kernel variant (z pass, fused x + y), pinned for every fast size."""
    for n in (64, 96, 128, 192, 256):
        hmg.hmg_set_variant(ctx.handle, n, request.param)
    yield request.param
    for n in (64, 96, 128, 192, 256):
        hmg.hmg_set_variant(ctx.handle, n, -1)


@pytest.mark.parametrize("N,count", [(64, 4), (128, 3), (192, 1), (256, 1)])
def test_fast_fft_forward_inverse(ctx, zvar, N, count):
    rng = np.random.default_rng(N)
    x = rng.standard_normal((count, N, N, N))
    ref = np.fft.fftn(x, axes=(1, 2, 3))
    Z = np.empty((count, N * N * N // 2, 2))
    hmg.hmg_fft_forward(ctx.handle, N, count, hmg.HMG_FP32_BULK, x, Z)
    Zc = Z[..., 0] + 1j * Z[..., 1]
    for i in range(count):
        full = unpack_spectrum(Zc[i], N)
        assert np.abs(full - ref[i]).max() < 2e-6 * np.abs(ref[i]).max(), (N, i)
    back = np.empty_like(x)
    hmg.hmg_fft_inverse(ctx.handle, N, count, hmg.HMG_FP32_BULK, Z, back)
    assert np.abs(back / N ** 3 - x).max() < 2e-5 * np.abs(x).max()


@pytest.mark.parametrize("N", [64, 96, 128])
def test_fast_sweeps_match_oracle(ctx, zvar, N):
    sl = I.generate_spheres(N, 20, 0.3)
    ph = om.voxelize(sl.spheres, 0.3, N)
    E = np.array([0.3, -1.0, 0.5])
    rng = np.random.default_rng(N)
    e0 = E[:, None, None, None] + 0.3 * rng.standard_normal((3, N, N, N))
    ref = om.em_solve(ph, K3, E, tol=0.0, max_iter=2, record=True, e0=e0)
    e = e0.copy()
    eps = hmg.hmg_em_iterate(ctx.handle, ph, N, K3, E, hmg.HMG_FP32_BULK, 2, e)
    assert np.abs(e - ref.e).max() < 1e-5 * np.abs(ref.e).max()
    assert np.allclose(eps, ref.eps_comp_hist, rtol=1e-4)


def test_fast_equilibrium_fp32(ctx, zvar):
    N = 64
    ph = I.random_phase_grid(8, N)
    r = om.em_solve(ph, K3, (0.0, 1.0, 0.0), tol=0.0, max_iter=20)
    ref_eps, ref_mean = om.equilibrium_residual(np.asarray(K3)[ph], r.e, om.wavevectors(N))
    eps, flux = hmg.hmg_equilibrium(ctx.handle, ph, N, K3, hmg.HMG_FP32_BULK, np.ascontiguousarray(r.e))
    assert abs(eps - ref_eps) < 1e-4 * ref_eps
    assert np.abs(flux + ref_mean).max() < 1e-5 * np.abs(ref_mean).max()


@pytest.mark.parametrize("N", [64, 128])
def test_fast_bulk_solve_matches_oracle(ctx, zvar, N):
    sl = I.generate_spheres(1000, 30, 0.2)
    ph = om.voxelize(sl.spheres, 0.3, N)
    k = (0.20, 0.25, 40.0)          # contrast 200 keeps the oracle solve short
    Kref, res = om.effective_tensor(ph, k, tol=1e-8)
    e = np.empty((3, 3, N, N, N))
    K, info, _ = hmg.hmg_solve_fields(ctx.handle, ph, N, k, 1e-8, hmg.HMG_FP32_BULK, e)
    assert kerr(K, Kref) < 1e-5
    for j in range(3):
        assert np.linalg.norm(e[j] - res[j].e) < 1e-4 * np.linalg.norm(res[j].e)
        assert info["eps_eq"][j] < 1e-8


def test_full_size_256_one_sweep_matches_oracle(ctx, zvar):
    """The benchmark's grid (256^3, 100 spheres at 40 %, l = 0.3): one sweep from the
    initial field, every voxel of all three components against the oracle."""
    N = 256
    sl = I.generate_spheres(3000, 100, 0.40)
    ph_d = torch.empty(N ** 3, dtype=torch.uint8, device="cuda")
    hmg.hmg_voxelize(ctx.handle, torch.from_numpy(np.ascontiguousarray(sl.spheres)).cuda(), 0.3, N, ph_d)
    ph = ph_d.cpu().numpy().reshape(N, N, N)
    assert (ph == om.voxelize(sl.spheres, 0.3, N)).all()          # bit-exact at full size
    E = np.array([1.0, 0.0, 0.0])
    ref = om.em_solve(ph, K3, E, tol=0.0, max_iter=1, record=True)
    e = torch.zeros((3, N ** 3), dtype=torch.float64, device="cuda")
    e[0] = 1.0
    eps = hmg.hmg_em_iterate(ctx.handle, ph_d, N, K3, E, hmg.HMG_FP32_BULK, 1, e)
    got = e.cpu().numpy().reshape(3, N, N, N)
    assert np.abs(got - ref.e).max() < 1e-5 * np.abs(ref.e).max()
    assert abs(eps[0] - ref.eps_comp_hist[0]) < 1e-5 * ref.eps_comp_hist[0]


def test_autotuner_records_a_variant(ctx):
    N = 128
    hmg.hmg_set_variant(ctx.handle, N, -1)
    assert hmg.hmg_get_variant(ctx.handle, N) == -1
    ph = I.random_phase_grid(3, N)
    e = np.zeros((3, N, N, N))
    e[0] = 1.0
    hmg.hmg_em_iterate(ctx.handle, ph, N, K3, (1.0, 0.0, 0.0), hmg.HMG_FP32_BULK, 1, e)
    v = hmg.hmg_get_variant(ctx.handle, N)
    assert 0 <= v < 32 and not (v & 4)            # bits 0, 1, 3, 4 chosen; chaining kept on


@pytest.mark.parametrize("N", [64, 96, 128])
def test_chained_sweeps_are_bit_identical(ctx, N):
    """Chained FP32 sweeps (variant bit 2 clear: x inverse + next x forward in one kernel)
    against unchained ones (bit 2 set): the same K, sweep counts and fields, bit for bit."""
    sl = I.generate_spheres(1000, 30, 0.2)
    ph = om.voxelize(sl.spheres, 0.3, N)
    k = (0.20, 0.25, 40.0)
    out = []
    for v in (0, 4):
        hmg.hmg_set_variant(ctx.handle, N, v)
        e = np.empty((3, 3, N, N, N))
        K, info, st = hmg.hmg_solve_fields(ctx.handle, ph, N, k, 1e-8, hmg.HMG_FP32_BULK, e)
        assert st == hmg.HMG_OK
        out.append((K, info, e))
    hmg.hmg_set_variant(ctx.handle, N, -1)
    assert np.array_equal(out[0][0], out[1][0])
    assert list(out[0][1]["iters"]) == list(out[1][1]["iters"])
    assert np.array_equal(out[0][2], out[1][2])


def test_chained_engine_batch_is_bit_identical(ctx):
    """The engine's graph of chained blocks against unchained blocks (hmg_solve_batch)."""
    N = 64
    phs = [om.voxelize(I.generate_spheres(s, 20, 0.3).spheres, 0.3, N) for s in (11, 12)]
    res = []
    for v in (0, 4):
        hmg.hmg_set_variant(ctx.handle, N, v)
        K, infos, st = hmg.hmg_solve_batch(ctx.handle, phs, [N, N], np.array([I.K_PHASES, (0.2, 0.25, 40.0)]),
                                           1e-8, hmg.HMG_FP32_BULK)
        assert st == hmg.HMG_OK
        res.append((K, infos))
    hmg.hmg_set_variant(ctx.handle, N, -1)
    assert np.array_equal(res[0][0], res[1][0])
    for a, b in zip(res[0][1], res[1][1]):
        assert list(a["iters"]) == list(b["iters"])


@pytest.mark.parametrize("N,pers", [(64, 8), (96, 8), (128, 8), (64, 16), (96, 16), (128, 16), (128, 24)])
def test_persistent_kernels_are_bit_identical(ctx, N, pers):
    """Chained sweeps with the persistent x round trip (variant bit 3: bulk copies stage
    the next row block) and/or the persistent z pass (bit 4: tensor copies stage the next
    column block) against the plain kernels: the same K, sweep counts and fields, bit for
    bit, correction sweeps (r added) included."""
    sl = I.generate_spheres(1000, 30, 0.2)
    ph = om.voxelize(sl.spheres, 0.3, N)
    k = (0.20, 0.25, 40.0)
    out = []
    for v in (0, pers):
        hmg.hmg_set_variant(ctx.handle, N, v)
        e = np.empty((3, 3, N, N, N))
        K, info, st = hmg.hmg_solve_fields(ctx.handle, ph, N, k, 1e-8, hmg.HMG_FP32_BULK, e)
        assert st == hmg.HMG_OK
        assert info["fp64_rounds"] > 0          # correction sweeps ran
        out.append((K, info, e))
    hmg.hmg_set_variant(ctx.handle, N, -1)
    assert np.array_equal(out[0][0], out[1][0])
    assert list(out[0][1]["iters"]) == list(out[1][1]["iters"])
    assert np.array_equal(out[0][2], out[1][2])


@pytest.mark.parametrize("N,base", [(64, 0), (128, 0), (128, 16), (192, 0), (192, 16)])
def test_plane_kernel_is_bit_identical(ctx, N, base):
    """Chained sweeps with the plane kernel (variant bit 5: the y inverse, the x round trip
    and the next sweep's y forward of each (component, z) plane in one persistent launch)
    against the separate passes: the same K, sweep counts and fields, bit for bit,
    correction sweeps (r added) and the stored field of the residual sweep included."""
    sl = I.generate_spheres(1000, 30, 0.2)
    ph = om.voxelize(sl.spheres, 0.3, N)
    k = (0.20, 0.25, 40.0)
    out = []
    for v in (base, base | 32):
        hmg.hmg_set_variant(ctx.handle, N, v)
        e = np.empty((3, 3, N, N, N))
        K, info, st = hmg.hmg_solve_fields(ctx.handle, ph, N, k, 1e-8, hmg.HMG_FP32_BULK, e)
        assert st == hmg.HMG_OK
        assert info["fp64_rounds"] > 0          # correction sweeps ran
        out.append((K, info, e))
    hmg.hmg_set_variant(ctx.handle, N, -1)
    assert np.array_equal(out[0][0], out[1][0])
    assert list(out[0][1]["iters"]) == list(out[1][1]["iters"])
    assert np.array_equal(out[0][2], out[1][2])


def test_plane_kernel_in_the_batch_engine_is_bit_identical(ctx):
    """The many-RVE engine's chained blocks (per-slot flags, correction sweeps, one graph
    per round) with and without the plane kernel: the same K and sweep counts."""
    Ns = [64, 128, 64, 128, 64]
    phases = [om.voxelize(I.generate_spheres(40 + i, 25, 0.2).spheres, 0.3, N) for i, N in enumerate(Ns)]
    res = []
    for v in (0, 32):
        for N in (64, 128):
            hmg.hmg_set_variant(ctx.handle, N, v)
        K, infos, st = hmg.hmg_solve_batch(ctx.handle, phases, Ns, np.tile((0.20, 0.25, 40.0), (len(Ns), 1)),
                                           1e-8, hmg.HMG_FP32_BULK)
        assert st == hmg.HMG_OK
        res.append((K, infos))
    for N in (64, 128):
        hmg.hmg_set_variant(ctx.handle, N, -1)
    assert np.array_equal(res[0][0], res[1][0])
    for a, b in zip(res[0][1], res[1][1]):
        assert list(a["iters"]) == list(b["iters"])


def test_autotuner_choices_persist_on_disk(tmp_path):
    """With HMG_TUNE_CACHE set, a fresh process records the variant it times, and a later
    process takes the recorded choice (here overwritten with another valid one) instead of
    timing."""
    import os
    import subprocess
    import sys
    from conftest import ROOT
    cache = tmp_path / "variants"
    prog = (
        "import sys, numpy as np; sys.path.insert(0, sys.argv[1])\n"
        "from paper_1504_07499_gb300 import hmg, inputs as I\n"
        "c = hmg.Context(0)\n"
        "ph = I.random_phase_grid(3, 64)\n"
        "e = np.zeros((3, 64, 64, 64)); e[0] = 1.0\n"
        "hmg.hmg_solve(c.handle, ph, 64, I.K_PHASES, 1e-8, hmg.HMG_FP32_BULK, max_iter=8,"
        " allow=(hmg.HMG_NOT_CONVERGED,))\n"
        "print(hmg.hmg_get_variant(c.handle, 64))\n")
    env = dict(os.environ, HMG_TUNE_CACHE=str(cache))
    r = subprocess.run([sys.executable, "-c", prog, ROOT], env=env, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr[-2000:]
    first = int(r.stdout.split()[-1])
    lines = cache.read_text().splitlines()
    assert len(lines) == 1 and lines[0].endswith(f"|64|{first}")
    other = 17 if first != 17 else 1
    cache.write_text(lines[0].rsplit("|", 1)[0] + f"|{other}\n")
    r = subprocess.run([sys.executable, "-c", prog, ROOT], env=env, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr[-2000:]
    assert int(r.stdout.split()[-1]) == other
    assert len(cache.read_text().splitlines()) == 1          # nothing timed, nothing appended
