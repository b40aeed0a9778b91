"""Write the stored expected values of the GPU tests.  Calls only the oracle (and the
input generators); nothing here touches the CUDA library.

    python tests/golden/make_golden.py

bar1d_2000_solve.json: the oracle's enhanced ParaSLRF (Alg. 2) on the 1D linear-FEM bar
n = 2000, gamma = 4150.528, block 32, m = 8, It_max = 200, start block Gaussian(seed 1):
eigenvalues, residuals, outer iterations and the number of pairs locked per iteration.
"""
import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import slrf_inputs as si  # noqa: E402
from oracle import slrf_oracle as orc  # noqa: E402


def bar1d_2000():
    wl = si.bar1d(2000)
    V1 = si.start_block(wl.n, wl.block, wl.seed)
    t = time.time()
    r = orc.enhanced_slrf(wl.pencil.A(), wl.pencil.B(), wl.gamma, V1, m=wl.m, it_max=200, tol_in=1e-10,
                          tol_eig=1e-8, outer_max=60, keep_trace=True)
    return {
        "workload": "bar1d_2000", "gamma": wl.gamma, "block": wl.block, "m": wl.m, "it_max": 200, "seed": wl.seed,
        "status": int(r.status), "evals": r.evals.tolist(), "resid": r.resid.tolist(),
        "outer_iters": int(r.outer_iters), "locks": [int(d["n_lock"]) for d in r.trace],
        "oracle_seconds": time.time() - t,
    }


if __name__ == "__main__":
    out = bar1d_2000()
    with open(os.path.join(HERE, "bar1d_2000_solve.json"), "w") as fh:
        json.dump(out, fh, indent=1)
    print(out["status"], len(out["evals"]), out["outer_iters"], out["locks"])
