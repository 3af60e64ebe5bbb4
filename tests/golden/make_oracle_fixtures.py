"""Writes the stored oracle results used by the GPU parity tests at full workload size.

Every value comes from the CPU oracle (oracle/em.py) on seeded inputs from
paper_1504_07499_gb300/inputs.py; nothing here touches the CUDA path.

    python tests/golden/make_oracle_fixtures.py rsa128_s1000

Each case stores K, the sweep counts, eps_eq, and a checksum of the voxelized phase
grid (so a test can confirm it solves the same grid):

rsa128_s1000: the 128^3 RVE of 30 RSA spheres at 20 % volume fraction (seed 1000),
  layer 0.3, conductivities 0.20 / 0.25 / 400, tol 1e-8.
rsa256_s3000: the 256^3 RVE of 100 spheres at 40 % (seed 3000, growth-sweep fallback),
  layer 0.3, conductivities 0.20 / 0.25 / 400 (contrast 2000), tol 1e-8 -- the
  benchmark's own workload (hours of CPU time).
rsa64_s3000_c2e4: the same 100 spheres at 40 % on a 64^3 grid with coating
  conductivity 4000 (contrast 2e4, the highest of the contrast sweep), tol 1e-8.
sphere32: one coated sphere centred in the cell (r_s = 0.25, l = 0.25) on 32^3,
  conductivities 0.20 / 0.25 / 400, tol 1e-8 (its K is isotropic).
"""
import concurrent.futures as cf
import hashlib
import json
import multiprocessing as mp
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

from oracle import em as om  # noqa: E402
from paper_1504_07499_gb300 import inputs as I  # noqa: E402

CASES = {
    "rsa128_s1000": dict(N=128, n=30, f=0.20, layer=0.3, seed=1000, k=(0.20, 0.25, 400.0), tol=1e-8),
    "rsa256_s3000": dict(N=256, n=100, f=0.40, layer=0.3, seed=3000, k=(0.20, 0.25, 400.0), tol=1e-8),
    "rsa64_s3000_c2e4": dict(N=64, n=100, f=0.40, layer=0.3, seed=3000, k=(0.20, 0.25, 4000.0), tol=1e-8),
    "sphere32": dict(N=32, centred=0.25, layer=0.25, k=(0.20, 0.25, 400.0), tol=1e-8),
}


def _solve_one(args):
    ph, k, tol, j = args
    E = np.zeros(3)
    E[j] = 1.0
    r = om.em_solve(ph, k, E, tol)
    r.e = None  # the field is not stored
    return r


def make(name: str) -> dict:
    c = CASES[name]
    if "centred" in c:
        spheres, generator = I.centred_sphere(c["centred"]), "centred"
    else:
        sl = I.generate_spheres(c["seed"], c["n"], c["f"])
        spheres, generator = sl.spheres, sl.generator
    ph = om.voxelize(spheres, c["layer"], c["N"])
    t0 = time.time()
    if c["N"] >= 128:
        # the three gradients are independent solves: one process each
        with cf.ProcessPoolExecutor(3, mp_context=mp.get_context("spawn")) as ex:
            res = list(ex.map(_solve_one, [(ph, c["k"], c["tol"], j) for j in range(3)]))
        K = np.stack([-r.flux_mean for r in res], axis=1)
    else:
        K, res = om.effective_tensor(ph, c["k"], tol=c["tol"])
    return {"case": name, "params": {k: (list(v) if isinstance(v, tuple) else v) for k, v in c.items()},
            "phase_sha256": hashlib.sha256(ph.tobytes()).hexdigest(),
            "phase_counts": [int((ph == p).sum()) for p in range(3)],
            "K": K.tolist(), "iters": [r.iters for r in res], "eps_eq": [r.eps_eq for r in res],
            "converged": [bool(r.converged) for r in res], "generator": generator,
            "oracle_seconds": time.time() - t0}


if __name__ == "__main__":
    for name in sys.argv[1:] or list(CASES):
        out = make(name)
        with open(os.path.join(HERE, f"oracle_{name}.json"), "w") as fh:
            json.dump(out, fh, indent=1)
        print(name, out["iters"], out["oracle_seconds"])
