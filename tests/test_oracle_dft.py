"""Pins for the oracle's 3D DFT: the direct sum against closed forms, and the library
FFT against the direct sum (§3, steps 3 and 5 rely on an unnormalized DFT pair)."""
import numpy as np
import pytest

from oracle import em as om


@pytest.mark.parametrize("N", [2, 3, 4, 5, 6, 12, 16])
def test_plane_wave_maps_to_delta(N):
    # x[n] = exp(+2 pi i k0.n / N)  ->  X[k] = N^3 delta(k - k0)
    k0 = np.array([1, N - 1, 2 % N])  # (z, y, x)
    z, y, x = np.indices((N, N, N))
    sig = np.exp(2j * np.pi * (k0[0] * z + k0[1] * y + k0[2] * x) / N)
    expect = np.zeros((N, N, N), complex)
    expect[tuple(k0)] = N ** 3
    assert np.abs(om.dft3_direct(sig) - expect).max() < 1e-9 * N ** 3
    if N <= 6:
        assert np.abs(om.dft3_dense(sig) - expect).max() < 1e-9 * N ** 3


@pytest.mark.parametrize("N", [3, 4, 6, 8])
def test_axis_by_axis_sum_matches_dense_definition(N):
    # the direct sum taken one axis at a time against the whole N^3 x N^3 DFT matrix
    rng = np.random.default_rng(N)
    x = rng.standard_normal((2, N, N, N)) + 1j * rng.standard_normal((2, N, N, N))
    for inv in (False, True):
        d = om.dft3_direct(x, inverse=inv)
        assert np.abs(d - om.dft3_dense(x, inverse=inv)).max() < 1e-10 * N ** 3


def test_direct_sum_of_a_single_voxel():
    # x = delta at n0  ->  X[k] = exp(-2 pi i k . n0 / N), on a grid the dense matrix
    # would not fit (16^3 -> 4096^2 complex entries)
    N = 16
    n0 = (3, 11, 7)  # (z, y, x)
    x = np.zeros((N, N, N))
    x[n0] = 1.0
    kz, ky, kx = np.indices((N, N, N))
    expect = np.exp(-2j * np.pi * (kz * n0[0] + ky * n0[1] + kx * n0[2]) / N)
    assert np.abs(om.dft3_direct(x) - expect).max() < 1e-12
    assert np.abs(om.fft3(x) - expect).max() < 1e-12


@pytest.mark.parametrize("N", [4, 6, 8, 9, 12, 16, 24])
def test_library_fft_matches_direct_sum(N):
    rng = np.random.default_rng(100 + N)
    x = rng.standard_normal((3, N, N, N))
    d = om.dft3_direct(x)
    if om._sfft is not None:
        lib = om._sfft.fftn(x, axes=(-3, -2, -1))
        assert np.abs(lib - d).max() < 1e-10 * N ** 3
    assert np.abs(om.fft3(x) - d).max() < 1e-10 * N ** 3
    if N <= 16:  # the oracle's own transform up to 16^3 is the direct sum
        assert np.array_equal(om.fft3(x), d)
    back = om.ifft3_unnorm(om.fft3(x)) / N ** 3
    assert np.abs(back - x).max() < 1e-12


@pytest.mark.parametrize("N", [5, 8, 16, 24])
def test_parseval_and_real_symmetry(N):
    rng = np.random.default_rng(7 * N)
    x = rng.standard_normal((N, N, N))
    X = om.fft3(x)
    assert abs((np.abs(X) ** 2).sum() / N ** 3 - (x ** 2).sum()) < 1e-9 * (x ** 2).sum()
    # Hermitian symmetry of a real signal: X[-k] = conj X[k]
    Xm = np.roll(np.flip(X, axis=(0, 1, 2)), 1, axis=(0, 1, 2))
    assert np.abs(Xm - X.conj()).max() < 1e-9 * N ** 3
