"""Writes tests/golden/elast_64_spectrum.json: the reference spectrum of the 64 x 64 x 32 Q1
elasticity box (z = 0 clamped, E lognormal(0, 0.5) seed 3) and the count of eigenvalues in
(0, gamma] -- from oracle/ only (shift-invert Lanczos and a Sylvester-inertia count).  Takes
about an hour and ~25 GB of host memory.

    python tests/golden/make_elast64.py [spectrum|inertia]
"""
import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import slrf_oracle as orc  # noqa: E402
from slrf_inputs import elastic as se  # noqa: E402

OUT = os.path.join(HERE, "elast_64_spectrum.json")


def main(what):
    tab = {}
    if os.path.exists(OUT):
        with open(OUT) as fh:
            tab = json.load(fh)
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
    with open(OUT, "w") as fh:
        json.dump(tab, fh, indent=1)
    print({k: (v if not isinstance(v, list) else len(v)) for k, v in tab.items()})


if __name__ == "__main__":
    main(sys.argv[1] if len(sys.argv) > 1 else "spectrum")
