"""Coated cylinders and mixed sphere/cylinder RVEs on the GPU (hmg_voxelize_mixed, §6
outlook) against the oracle: bit-exact phase grids from host or device object lists,
solves of mixed grids against the oracle's K, the exact arithmetic mean along continuous
fibers, and rejected bad cylinders."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import em as om
from paper_1504_07499_gb300 import hmg, inputs as I

from test_gpu_parity import kerr

K3 = (0.20, 0.25, 400.0)


@pytest.fixture(scope="module")
def ctx():
    from paper_1504_07499_gb300 import build
    build.build()
    c = hmg.Context(0)
    yield c
    c.close()


@pytest.mark.parametrize("seed,nc,ns,N,layer,axis", [(1, 8, 0, 24, 0.3, None), (2, 6, 6, 64, 0.2, None),
                                                    (3, 12, 4, 128, 0.4, (0, 0, 1)), (4, 10, 10, 96, 0.5, None),
                                                    (5, 4, 8, 256, 0.3, None)])
def test_mixed_voxelization_bit_exact(ctx, seed, nc, ns, N, layer, axis):
    sp, cy = I.generate_cylinders(seed, nc, 0.05, 0.3, axis=axis, spheres=ns, r_sphere=0.06)
    ref = om.voxelize_mixed(sp if ns else None, cy, layer, N)
    got = np.empty((N, N, N), np.uint8)
    hmg.hmg_voxelize_mixed(ctx.handle, sp if ns else None, cy, layer, N, got)
    assert (got == ref).all()
    # device object lists and a device output grid
    out = torch.empty(N ** 3, dtype=torch.uint8, device="cuda")
    hmg.hmg_voxelize_mixed(ctx.handle, torch.from_numpy(sp).cuda() if ns else None, torch.from_numpy(cy).cuda(),
                           layer, N, out)
    assert (out.cpu().numpy().reshape(N, N, N) == ref).all()


def test_mixed_grid_without_cylinders_equals_hmg_voxelize(ctx):
    sl = I.generate_spheres(3000, 100, 0.40)
    a = np.empty((64, 64, 64), np.uint8)
    b = np.empty((64, 64, 64), np.uint8)
    hmg.hmg_voxelize(ctx.handle, sl.spheres, 0.3, 64, a)
    hmg.hmg_voxelize_mixed(ctx.handle, sl.spheres, None, 0.3, 64, b)
    assert np.array_equal(a, b)


@pytest.mark.parametrize("prec,tol", [(hmg.HMG_FP64, 1e-9), (hmg.HMG_FP32_BULK, 1e-5)])
def test_mixed_rve_solve_matches_oracle(ctx, prec, tol):
    N = 24
    sp, cy = I.generate_cylinders(21, 6, 0.06, 0.3, spheres=4, r_sphere=0.07)
    ph = om.voxelize_mixed(sp, cy, 0.3, N)
    Kref, _ = om.effective_tensor(ph, K3, tol=1e-8)
    K, info, st = hmg.hmg_solve(ctx.handle, ph, N, K3, 1e-8, prec)
    assert st == hmg.HMG_OK
    assert kerr(K, Kref) < tol


@pytest.mark.parametrize("prec,tol", [(hmg.HMG_FP64, 1e-12), (hmg.HMG_FP32_BULK, 1e-9)])
def test_continuous_fibers_give_the_arithmetic_mean_along_them(ctx, prec, tol):
    N, layer, r = 64, 0.3, 0.1
    h = 1.0 + 2 * layer * r + 1e-9
    cyl = np.array([[0.25, 0.25, 0.5, 0, 0, 1, r, h], [0.75, 0.7, 0.3, 0, 0, 1, r, h],
                    [0.3, 0.72, 0.9, 0, 0, 1, r, h]])
    ph = np.empty((N, N, N), np.uint8)
    hmg.hmg_voxelize_mixed(ctx.handle, None, cyl, layer, N, ph)
    K, info, st = hmg.hmg_solve(ctx.handle, ph, N, K3, 1e-8, prec)
    assert st == hmg.HMG_OK
    f = om.phase_fractions(ph)
    arith = float((f * np.asarray(K3)).sum())
    assert abs(K[2, 2] - arith) < tol * arith
    assert max(abs(K[0, 2]), abs(K[1, 2])) < tol * arith


@pytest.mark.parametrize("bad", [dict(r=0.0), dict(r=0.6), dict(h=0.0), dict(h=2.5), dict(ux=0.5),
                                 dict(cx=float("nan"))])
def test_bad_cylinders_are_rejected(ctx, bad):
    c = dict(cx=0.5, cy=0.5, cz=0.5, ux=0.0, uy=0.0, uz=1.0, r=0.1, h=0.3)
    c.update(bad)
    cyl = np.array([[c[k] for k in ("cx", "cy", "cz", "ux", "uy", "uz", "r", "h")]])
    with pytest.raises(hmg.HmgError) as ex:
        hmg.hmg_voxelize_mixed(ctx.handle, None, cyl, 0.3, 16, np.empty((16, 16, 16), np.uint8))
    assert ex.value.status == hmg.HMG_INVALID_ARG
