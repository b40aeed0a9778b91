"""Writes the reference values of the 64 x 64 x 32 Q1 elasticity box (z = 0 clamped, E
lognormal(0, 0.5) seed 3) from oracle/ only:
  spectrum -> tests/golden/elast_64_spectrum.json: the 330 lowest eigenvalues by
              shift-invert Lanczos;
  inertia  -> tests/golden/elast_64_count.json: the number of eigenvalues below gamma by
              Sylvester's law of inertia (a symmetric sparse LU of A - gamma B).
Each takes up to about an hour and ~25 GB of host memory.

    python tests/golden/make_elast64.py [spectrum|inertia]
"""
import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import slrf_oracle as orc  # noqa: E402
from slrf_inputs import elastic as se  # noqa: E402

def main(what):
    out = os.path.join(HERE, "elast_64_spectrum.json" if what == "spectrum" else "elast_64_count.json")
    tab = {}
    p = se.pencil("elast_64")
    A, B = p.A(), p.B()
    if what == "spectrum":
        lam = orc.shift_invert_spectrum(A, B, 330)
        tab["lambdas"] = [float(v) for v in lam]
        tab["source_lambdas"] = "oracle.shift_invert_spectrum (scipy eigsh, shift-invert at 0, tol 1e-12), k = 330"
    else:
        gamma, _ = se.gamma("elast_64")
        cnt, ok = orc.inertia_count(A, B, gamma)
        tab["gamma"] = gamma
        tab["inertia_count"] = cnt
        tab["inertia_symmetric_ordering"] = ok
        tab["source_inertia"] = "oracle.inertia_count (SuperLU, symmetric mode, diagonal pivots) of A - gamma B"
    tab["n"] = p.n
    tab["nnz"] = p.nnz
    with open(out, "w") as fh:
        json.dump(tab, fh, indent=1)
    print({k: (v if not isinstance(v, list) else len(v)) for k, v in tab.items()})


if __name__ == "__main__":
    main(sys.argv[1] if len(sys.argv) > 1 else "spectrum")
