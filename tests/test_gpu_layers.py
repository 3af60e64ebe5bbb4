"""A thicker coating (larger l, same sphere centres and outer radius) only turns inclusion
voxels (k = 0.2) into coating voxels (k = 400).  The effective tensor of the discrete
problem is monotone in every voxel's conductivity (it minimizes <e . k e> over the
compatible fields), so K(l2) - K(l1) must be positive semidefinite for l2 > l1: a property
of the exact solution that the GPU solve has to reproduce (the paper observes the rise of
the homogenized conductivity with the layer thickness in §5)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1504_07499_gb300 import hmg, inputs as I

K_PAPER = (1.0, 0.2, 400.0)     # matrix, inclusion, coating (§5)


@pytest.fixture(scope="module")
def ctx():
    from paper_1504_07499_gb300 import build
    build.build()
    c = hmg.Context(0)
    yield c
    c.close()


@pytest.mark.parametrize("N", [64, 128])
def test_k_is_monotone_in_the_layer(ctx, N):
    sl = I.generate_spheres(6000, 30, 0.3)
    Ks = []
    for layer in (0.1, 0.3, 0.6):
        ph = ctx.voxelize(sl.spheres, layer, N)
        K, _, st = ctx.solve(ph, K_PAPER, 1e-8, hmg.HMG_FP32_BULK)
        assert st == hmg.HMG_OK
        Ks.append(0.5 * (K + K.T))
    for a, b in zip(Ks, Ks[1:]):
        ev = np.linalg.eigvalsh(b - a)
        assert ev.min() > -1e-6 * np.trace(a)          # K(l2) >= K(l1) in the Loewner order
        assert np.trace(b) > np.trace(a)                # and the layer does change the grid
