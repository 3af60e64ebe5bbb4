"""hmg_equilibrium_noalloc: the equilibrium residual for callers that cannot allocate
device memory (hosts whose own pool owns the device memory, or that must not risk an
allocation failure or cudaMalloc's implicit synchronization mid-run).  Its scratch is
static device memory.  It is checked here against hmg_equilibrium, which allocates,
and against the oracle's equilibrium residual, on two calls in a row; a fresh process
checks that not even the first call changes the device's free memory.  This file is
collected last on purpose."""
import json
import os
import subprocess
import sys

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from conftest import ROOT
from oracle import em as om
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
def test_noalloc_matches_allocating_entry_point_and_oracle_twice(ctx, N):
    torch.cuda.set_device(0)
    ph = I.random_phase_grid(N, N, probs=(0.5, 0.2, 0.3))
    e = _field(N, N)
    ref_eps, ref_flux = hmg.hmg_equilibrium(ctx.handle, ph, N, K3, hmg.HMG_FP64, e)
    ora_eps, ora_mean = om.equilibrium_residual(np.asarray(K3)[ph], e, om.wavevectors(N))
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
        # the oracle's phi = -k e: its mean flux is minus <k e>
        assert abs(eps - ora_eps) <= TOL * ora_eps
        assert np.abs(flux + ora_mean).max() <= TOL * np.abs(ora_mean).max()
    assert free[0] == free[1]           # the second call took no device memory
    # host inputs work too
    eps_h, flux_h = hmg.hmg_equilibrium_noalloc(ph, N, K3, e)
    assert abs(eps_h - ref_eps) <= TOL * ref_eps


# Run in a fresh process with every module loaded when the CUDA context is created
# (CUDA_MODULE_LOADING=EAGER), so that the static arrays are already mapped in; the
# process makes no allocation of its own and reads the device's free memory around
# each call through the CUDA runtime libhmg is linked against.
_FIRST_CALL = r"""
import ctypes, json, sys
import numpy as np
sys.path.insert(0, sys.argv[1])
from paper_1504_07499_gb300 import hmg, inputs as I
L = hmg.lib()
rt_path = [ln.split()[-1] for ln in open("/proc/self/maps") if "libcudart" in ln][0]
rt = ctypes.CDLL(rt_path)
assert rt.cudaSetDevice(0) == 0 and rt.cudaDeviceSynchronize() == 0
def free():
    f, t = ctypes.c_size_t(), ctypes.c_size_t()
    assert rt.cudaMemGetInfo(ctypes.byref(f), ctypes.byref(t)) == 0
    return f.value
N = int(sys.argv[2])
ph = I.random_phase_grid(N, N, probs=(0.5, 0.2, 0.3))
rng = np.random.default_rng(N)
e = np.ascontiguousarray(np.array([1.0, 0.0, 0.0])[:, None, None, None] + 0.2 * rng.standard_normal((3, N, N, N)))
out = {"free": [free()], "eps": [], "flux": []}
for call in range(2):
    eps, flux = hmg.hmg_equilibrium_noalloc(ph, N, I.K_PHASES, e)
    out["free"].append(free())
    out["eps"].append(eps)
    out["flux"].append(list(flux))
print(json.dumps(out))
"""


def test_noalloc_first_call_in_a_fresh_process_takes_no_device_memory(ctx):
    N = 32
    env = dict(os.environ, CUDA_MODULE_LOADING="EAGER")
    r = subprocess.run([sys.executable, "-c", _FIRST_CALL, ROOT, str(N)], env=env, capture_output=True,
                       text=True, timeout=300)
    assert r.returncode == 0, r.stderr[-2000:]
    out = json.loads(r.stdout.strip().splitlines()[-1])
    assert out["free"][0] == out["free"][1] == out["free"][2], out["free"]
    ph = I.random_phase_grid(N, N, probs=(0.5, 0.2, 0.3))
    rng = np.random.default_rng(N)
    e = np.array([1.0, 0.0, 0.0])[:, None, None, None] + 0.2 * rng.standard_normal((3, N, N, N))
    ora_eps, ora_mean = om.equilibrium_residual(np.asarray(K3)[ph], e, om.wavevectors(N))
    for eps, flux in zip(out["eps"], out["flux"]):
        assert abs(eps - ora_eps) <= TOL * ora_eps
        assert np.abs(np.array(flux) + ora_mean).max() <= TOL * np.abs(ora_mean).max()


def test_noalloc_rejects_sizes_beyond_its_static_scratch():
    N = 2 * hmg.HMG_NOALLOC_MAX_N
    ph = np.zeros((N, N, N), np.uint8)
    e = np.zeros((3, N, N, N))
    with pytest.raises(hmg.HmgError) as err:
        hmg.hmg_equilibrium_noalloc(ph, N, K3, e)
    assert err.value.status == hmg.HMG_INVALID_ARG
    assert "static scratch" in str(err.value)
