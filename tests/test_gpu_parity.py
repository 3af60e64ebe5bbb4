"""CUDA path against the CPU oracle, element by element, through the C ABI.

Tolerances:
* voxelization: bit-exact (integer rule).
* FP64 transforms and sweeps: 1e-11 relative (rounding-order differences only).
* FP32 transforms: 2e-6 relative to the largest coefficient (FP32 FFT error
  ~ eps32 * log2(N^3)); FP32 sweeps: 1e-5 relative.
* Full solves: FP64 K within 1e-9 relative and the same sweep counts (+-1);
  FP32-bulk K within 1e-5 relative on each entry (entries below 1 % of the largest
  diagonal entry relative to that 1 %, see ``kerr``) and the gradient field within
  1e-4 relative L2.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import em as om
from paper_1504_07499_gb300 import hmg, inputs as I

K3 = I.K_PHASES


@pytest.fixture(scope="module")
def ctx():
    from paper_1504_07499_gb300 import build
    build.build()
    c = hmg.Context(0)
    yield c
    c.close()


def unpack_spectrum(Z, N):
    """Full N^3 spectrum (z, y, x order) from the packed layout of hmg_fft_forward."""
    M = N // 2
    Z = Z.reshape(N, N, M)
    full = np.zeros((N, N, N), complex)
    full[:, :, 1:M] = Z[:, :, 1:]
    col = Z[:, :, 0]
    neg = np.roll(np.flip(col, axis=(0, 1)), 1, axis=(0, 1))
    A = 0.5 * (col + neg.conj())
    B = (col - neg.conj()) / 2j
    full[:, :, 0] = A
    full[:, :, M] = B
    # Hermitian completion for kx > N/2
    for kx in range(M + 1, N):
        src = full[:, :, N - kx]
        full[:, :, kx] = np.roll(np.flip(src, axis=(0, 1)), 1, axis=(0, 1)).conj()
    return full


KERR_FLOOR = 1e-2


def kerr(K, Kref):
    """Largest relative error over the entries of K.  Each entry is compared with
    itself (|K_ij - Kref_ij| / |Kref_ij|) when it is at least KERR_FLOOR times the
    largest diagonal entry; smaller entries (off-diagonals that vanish by symmetry or
    nearly so) are compared with that floor instead."""
    floor = KERR_FLOOR * np.abs(np.diag(Kref)).max()
    return (np.abs(K - Kref) / np.maximum(np.abs(Kref), floor)).max()


# --- voxelization (§2) -------------------------------------------------------------

@pytest.mark.parametrize("seed,N,n,f,layer", [(1, 16, 3, 0.3, 0.3), (1000, 64, 30, 0.2, 0.3),
                                              (7, 96, 50, 0.35, 0.1), (11, 128, 100, 0.3, 0.5),
                                              (12, 24, 10, 0.4, 0.9)])
def test_voxelize_bit_exact(ctx, seed, N, n, f, layer):
    sl = I.generate_spheres(seed, n, f)
    got = ctx.voxelize(sl.spheres, layer, N)
    ref = om.voxelize(sl.spheres, layer, N)
    assert (got == ref).all()
    # device output buffer too
    out = torch.empty(N ** 3, dtype=torch.uint8, device="cuda")
    ctx.voxelize(sl.spheres, layer, N, out=out)
    assert (out.cpu().numpy().reshape(N, N, N) == ref).all()


def test_voxelize_centred_sphere_and_wrap(ctx):
    for sph in (I.centred_sphere(0.25), np.array([[0.999999, 0.0, 0.5, 0.3]]), np.array([[-0.25, 1.75, 0.1, 0.2]])):
        assert (ctx.voxelize(sph, 0.25, 32) == om.voxelize(sph, 0.25, 32)).all()


def test_voxelize_rejects_bad_input(ctx):
    with pytest.raises(hmg.HmgError) as e:
        ctx.voxelize(np.array([[0.1, 0.1, 0.1, 0.2], [0.2, 0.1, 0.1, 0.2]]), 0.3, 16)
    assert e.value.status == hmg.HMG_INVALID_ARG
    for bad in ([[0.5, 0.5, 0.5, 0.6]], [[np.nan, 0.5, 0.5, 0.1]]):
        with pytest.raises(hmg.HmgError):
            ctx.voxelize(np.array(bad), 0.3, 16)
    with pytest.raises(hmg.HmgError):
        ctx.voxelize(I.centred_sphere(), 0.3, 10)     # N = 10 is not 2^a 3^b
    with pytest.raises(hmg.HmgError):
        ctx.voxelize(I.centred_sphere(), 1.0, 16)     # layer outside (0, 1)


# --- transforms (§3 steps 3 and 5) ---------------------------------------------------

@pytest.mark.parametrize("N", [8, 12, 16, 24, 32, 48, 64, 96])
def test_fft_forward_inverse(ctx, N):
    rng = np.random.default_rng(N)
    x = rng.standard_normal((4, N, N, N))
    ref = np.fft.fftn(x, axes=(1, 2, 3))
    for prec, tol in ((hmg.HMG_FP64, 1e-12), (hmg.HMG_FP32_BULK, 2e-6)):
        Z = np.empty((4, N * N * N // 2, 2))
        hmg.hmg_fft_forward(ctx.handle, N, 4, prec, x, Z)
        Zc = Z[..., 0] + 1j * Z[..., 1]
        for i in range(4):
            full = unpack_spectrum(Zc[i], N)
            assert np.abs(full - ref[i]).max() < tol * np.abs(ref[i]).max(), (N, prec, i)
        back = np.empty_like(x)
        hmg.hmg_fft_inverse(ctx.handle, N, 4, prec, Z, back)
        assert np.abs(back / N ** 3 - x).max() < 10 * tol * np.abs(x).max()


# --- one sweep of steps 2-7 ----------------------------------------------------------

@pytest.mark.parametrize("N,seed", [(16, 1), (24, 2), (32, 3)])
def test_em_sweeps_match_oracle(ctx, N, seed):
    ph = I.random_phase_grid(seed, N, probs=(0.5, 0.2, 0.3))
    E = np.array([0.2, 1.0, -0.4])
    rng = np.random.default_rng(seed)
    e0 = E[:, None, None, None] + 0.3 * rng.standard_normal((3, N, N, N))
    n = 3
    ref = om.em_solve(ph, K3, E, tol=0.0, max_iter=n, record=True, e0=e0)
    for prec, tol in ((hmg.HMG_FP64, 1e-11), (hmg.HMG_FP32_BULK, 1e-5)):
        e = e0.copy()
        eps = hmg.hmg_em_iterate(ctx.handle, ph, N, K3, E, prec, n, e)
        assert np.abs(e - ref.e).max() < tol * np.abs(ref.e).max(), prec
        assert np.allclose(eps, ref.eps_comp_hist, rtol=max(tol, 1e-10) * 100), (eps, ref.eps_comp_hist)


def test_equilibrium_residual_matches_oracle(ctx):
    N = 24
    ph = I.random_phase_grid(5, N)
    r = om.em_solve(ph, K3, (1.0, 0.0, 0.0), tol=0.0, max_iter=40)
    ref_eps, ref_mean = om.equilibrium_residual(np.asarray(K3)[ph], r.e, om.wavevectors(N))
    for prec, tol in ((hmg.HMG_FP64, 1e-10), (hmg.HMG_FP32_BULK, 1e-4)):
        eps, flux = hmg.hmg_equilibrium(ctx.handle, ph, N, K3, prec, np.ascontiguousarray(r.e))
        assert abs(eps - ref_eps) < tol * ref_eps, (prec, eps, ref_eps)
        assert np.abs(flux + ref_mean).max() < tol * np.abs(ref_mean).max()


# --- full solves (§3 Algorithm + effective tensor) -----------------------------------

def test_homogeneous_and_laminate_closed_forms(ctx):
    N = 16
    ph = I.random_phase_grid(9, N)
    for prec in (hmg.HMG_FP64, hmg.HMG_FP32_BULK):
        K, info, _ = ctx.solve(ph, (1.7, 1.7, 1.7), 1e-8, prec)
        assert np.abs(K - 1.7 * np.eye(3)).max() < 1e-12
    lam = I.laminate_grid(N, 5, axis=1)
    f = 5 / N
    harm = 1 / (f / K3[2] + (1 - f) / K3[0])
    arith = f * K3[2] + (1 - f) * K3[0]
    for prec in (hmg.HMG_FP64, hmg.HMG_FP32_BULK):
        K, info, _ = ctx.solve(lam, K3, 1e-9, prec)
        assert abs(K[1, 1] - harm) < 1e-7 * harm and abs(K[0, 0] - arith) < 1e-7 * arith
        assert abs(K[2, 2] - arith) < 1e-7 * arith


@pytest.mark.parametrize("N,kind", [(16, "sphere"), (24, "random"), (32, "rsa")])
def test_solve_fp64_matches_oracle(ctx, N, kind):
    if kind == "sphere":
        ph = om.voxelize(I.centred_sphere(0.25), 0.25, N)
    elif kind == "random":
        ph = I.random_phase_grid(77, N, probs=(0.6, 0.2, 0.2))
    else:
        ph = om.voxelize(I.generate_spheres(5, 8, 0.25).spheres, 0.3, N)
    Kref, res = om.effective_tensor(ph, K3, tol=1e-8)
    e = np.empty((3, 3, N, N, N))
    K, info, _ = hmg.hmg_solve_fields(ctx.handle, ph, N, K3, 1e-8, hmg.HMG_FP64, e)
    assert kerr(K, Kref) < 1e-9
    for j in range(3):
        assert abs(info["iters"][j] - res[j].iters) <= 1
        assert np.linalg.norm(e[j] - res[j].e) < 1e-7 * np.linalg.norm(res[j].e)
        assert info["eps_eq"][j] < 1e-8


@pytest.mark.parametrize("N,kind", [(16, "sphere"), (24, "random"), (32, "rsa")])
def test_solve_fp32_bulk_matches_oracle(ctx, N, kind):
    if kind == "sphere":
        ph = om.voxelize(I.centred_sphere(0.25), 0.25, N)
    elif kind == "random":
        ph = I.random_phase_grid(77, N, probs=(0.6, 0.2, 0.2))
    else:
        ph = om.voxelize(I.generate_spheres(5, 8, 0.25).spheres, 0.3, N)
    Kref, res = om.effective_tensor(ph, K3, tol=1e-8)
    e = np.empty((3, 3, N, N, N))
    K, info, _ = hmg.hmg_solve_fields(ctx.handle, ph, N, K3, 1e-8, hmg.HMG_FP32_BULK, e)
    assert kerr(K, Kref) < 1e-5
    for j in range(3):
        assert np.linalg.norm(e[j] - res[j].e) < 1e-4 * np.linalg.norm(res[j].e)
        assert info["eps_eq"][j] < 1e-8
    assert info["fp64_rounds"] >= 1


def test_not_converged_and_invalid_arguments(ctx):
    N = 16
    ph = om.voxelize(I.centred_sphere(0.25), 0.25, N)
    K, info, st = ctx.solve(ph, K3, 1e-8, hmg.HMG_FP64, max_iter=5, allow=(hmg.HMG_NOT_CONVERGED,))
    assert st == hmg.HMG_NOT_CONVERGED and info["iters"] == [5, 5, 5]
    assert np.isfinite(K).all()
    with pytest.raises(hmg.HmgError):
        ctx.solve(ph, (0.2, -1.0, 400.0))
    with pytest.raises(hmg.HmgError):
        hmg.hmg_solve(ctx.handle, ph, 14, K3, 1e-8, hmg.HMG_FP64)


def test_device_resident_phase(ctx):
    N = 16
    ph = om.voxelize(I.centred_sphere(0.25), 0.25, N)
    d = torch.from_numpy(ph.reshape(-1)).cuda()
    K1, _, _ = ctx.solve(ph, K3, 1e-8, hmg.HMG_FP64)
    K2, _, _ = hmg.hmg_solve(ctx.handle, d, N, K3, 1e-8, hmg.HMG_FP64)
    assert np.array_equal(K1, K2)   # same inputs, same launch order: bitwise identical


def test_fp64_rate_is_measured(ctx):
    """The FP64 FMA-rate probe behind the FP64 form's roofline returns a finite rate in
    the range of any current GPU (0.1 to 100 TFLOP/s)."""
    r = hmg.hmg_fp64_rate(ctx.handle)
    assert 1e11 < r < 1e14
