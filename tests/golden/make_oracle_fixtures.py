"""Writes the stored oracle results used by the GPU parity tests at full workload size.

Every value comes from the CPU oracle (oracle/em.py) on seeded inputs from
paper_1504_07499_gb300/inputs.py; nothing here touches the CUDA path.

    python tests/golden/make_oracle_fixtures.py rsa128_s1000

rsa128_s1000: the 128^3 RVE of 30 RSA spheres at 20 % volume fraction (seed 1000),
layer 0.3, conductivities 0.20 / 0.25 / 400, tol 1e-8: K, sweep counts, eps_eq, and a
checksum of the voxelized phase grid (so a test can confirm it solves the same grid).
"""
import hashlib
import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

from oracle import em as om  # noqa: E402
from paper_1504_07499_gb300 import inputs as I  # noqa: E402

CASES = {
    "rsa128_s1000": dict(N=128, n=30, f=0.20, layer=0.3, seed=1000, k=(0.20, 0.25, 400.0), tol=1e-8),
}


def make(name: str) -> dict:
    c = CASES[name]
    sl = I.generate_spheres(c["seed"], c["n"], c["f"])
    ph = om.voxelize(sl.spheres, c["layer"], c["N"])
    t0 = time.time()
    K, res = om.effective_tensor(ph, c["k"], tol=c["tol"])
    return {"case": name, "params": {k: (list(v) if isinstance(v, tuple) else v) for k, v in c.items()},
            "phase_sha256": hashlib.sha256(ph.tobytes()).hexdigest(),
            "phase_counts": [int((ph == p).sum()) for p in range(3)],
            "K": K.tolist(), "iters": [r.iters for r in res], "eps_eq": [r.eps_eq for r in res],
            "converged": [bool(r.converged) for r in res], "generator": sl.generator,
            "oracle_seconds": time.time() - t0}


if __name__ == "__main__":
    for name in sys.argv[1:] or list(CASES):
        out = make(name)
        with open(os.path.join(HERE, f"oracle_{name}.json"), "w") as fh:
            json.dump(out, fh, indent=1)
        print(name, out["iters"], out["oracle_seconds"])
