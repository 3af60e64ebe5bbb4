"""512^3, the largest grid of the library (a single RVE of 134 M voxels; the FP32-bulk state
is 11 GB): the register-resident kernels of length 512 (y and z passes) and 256 (x passes)
against numpy's FFT and the oracle, and a full solve against a closed form.  Tolerances as
in test_gpu_parity: FP32 transforms 2e-6 of the largest coefficient, one FP32 sweep 1e-5
relative, FP32-bulk K 1e-5."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import em as om
from paper_1504_07499_gb300 import hmg, inputs as I

from test_gpu_parity import unpack_spectrum

N = 512
K3 = I.K_PHASES


@pytest.fixture(scope="module")
def ctx():
    from paper_1504_07499_gb300 import build
    build.build()
    c = hmg.Context(0)
    yield c
    c.close()


def test_fft_512_forward_inverse(ctx):
    x = np.random.default_rng(512).standard_normal((1, N, N, N))
    Z = np.empty((1, N * N * N // 2, 2))
    hmg.hmg_fft_forward(ctx.handle, N, 1, hmg.HMG_FP32_BULK, x, Z)
    ref = np.fft.fftn(x[0])
    full = unpack_spectrum(Z[0, :, 0] + 1j * Z[0, :, 1], N)
    assert np.abs(full - ref).max() < 2e-6 * np.abs(ref).max()
    del full, ref
    back = np.empty_like(x)
    hmg.hmg_fft_inverse(ctx.handle, N, 1, hmg.HMG_FP32_BULK, Z, back)
    assert np.abs(back / N ** 3 - x).max() < 2e-5 * np.abs(x).max()


def test_one_sweep_512_matches_oracle(ctx):
    """100 spheres at 40 % on 512^3 (the benchmark's RVE at twice the resolution): the
    voxelization bit for bit, then one FP32 sweep from the initial field on every voxel."""
    sl = I.generate_spheres(3000, 100, 0.40)
    ph_d = torch.empty(N ** 3, dtype=torch.uint8, device="cuda")
    hmg.hmg_voxelize(ctx.handle, torch.from_numpy(np.ascontiguousarray(sl.spheres)).cuda(), 0.3, N, ph_d)
    ph = ph_d.cpu().numpy().reshape(N, N, N)
    assert (ph == om.voxelize(sl.spheres, 0.3, N)).all()
    E = np.array([0.0, 0.0, 1.0])
    ref = om.em_solve(ph, K3, E, tol=0.0, max_iter=1, record=True)
    e = torch.zeros((3, N ** 3), dtype=torch.float64, device="cuda")
    e[2] = 1.0
    eps = hmg.hmg_em_iterate(ctx.handle, ph_d, N, K3, E, hmg.HMG_FP32_BULK, 1, e)
    got = e.cpu().numpy().reshape(3, N, N, N)
    assert np.abs(got - ref.e).max() < 1e-5 * np.abs(ref.e).max()
    assert abs(eps[0] - ref.eps_comp_hist[0]) < 1e-5 * ref.eps_comp_hist[0]


def test_laminate_512_fp32bulk_closed_form(ctx):
    """Slabs of coating and matrix normal to y: K_yy is the harmonic mean, K_xx = K_zz the
    arithmetic mean of the voxel fractions, off-diagonals zero (exact for the discrete
    scheme under the Nyquist rule)."""
    thick = 197
    ph = I.laminate_grid(N, thick, axis=1, phase_a=2, phase_b=0)
    K, info, st = hmg.hmg_solve(ctx.handle, torch.from_numpy(ph.reshape(-1)).cuda(), N, K3, 1e-8,
                                hmg.HMG_FP32_BULK)
    assert st == hmg.HMG_OK
    f = thick / N
    ka, kb = K3[2], K3[0]
    harm, arith = 1.0 / (f / ka + (1 - f) / kb), f * ka + (1 - f) * kb
    assert abs(K[1, 1] - harm) < 1e-5 * harm
    assert abs(K[0, 0] - arith) < 1e-5 * arith and abs(K[2, 2] - arith) < 1e-5 * arith
    assert np.abs(K - np.diag(np.diag(K))).max() < 1e-5 * harm
