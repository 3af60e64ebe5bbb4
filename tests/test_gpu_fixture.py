"""Full-size parity for the 128^3 workload (30 RSA spheres at 20 %, layer 0.3, contrast
2000, tol 1e-8): the GPU solves against the oracle's stored result
(tests/golden/oracle_rsa128_s1000.json, written by tests/golden/make_oracle_fixtures.py
from oracle/ only).  FP32 bulk: K within 1e-5 per entry; FP64: 1e-9 and the same sweep
counts (+-1)."""
import hashlib
import json
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from conftest import GOLDEN
from paper_1504_07499_gb300 import hmg, inputs as I

from test_gpu_parity import kerr


@pytest.fixture(scope="module")
def case():
    with open(os.path.join(GOLDEN, "oracle_rsa128_s1000.json")) as fh:
        return json.load(fh)


@pytest.fixture(scope="module")
def ctx():
    from paper_1504_07499_gb300 import build
    build.build()
    c = hmg.Context(0)
    yield c
    c.close()


@pytest.fixture(scope="module")
def phase(case, ctx):
    p = case["params"]
    sl = I.generate_spheres(p["seed"], p["n"], p["f"])
    N = p["N"]
    ph = ctx.voxelize(sl.spheres, p["layer"], N)
    assert hashlib.sha256(ph.tobytes()).hexdigest() == case["phase_sha256"]   # the same grid
    return ph


@pytest.mark.parametrize("prec,tol,iters_exact", [(hmg.HMG_FP32_BULK, 1e-5, False), (hmg.HMG_FP64, 1e-9, True)])
def test_rsa128_against_stored_oracle(case, ctx, phase, prec, tol, iters_exact):
    p = case["params"]
    Kref = np.array(case["K"])
    K, info, st = ctx.solve(phase, tuple(p["k"]), p["tol"], prec)
    assert st == hmg.HMG_OK
    assert kerr(K, Kref) < tol
    assert all(e < p["tol"] for e in info["eps_eq"])
    if iters_exact:
        assert all(abs(a - b) <= 1 for a, b in zip(info["iters"], case["iters"]))
