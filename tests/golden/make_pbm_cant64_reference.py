"""Writes tests/golden/pbm_cant64_oracle.json: the oracle's Algorithm 1 (oracle/pbm.py `pbm`) on the 64 x 32 x 32
cantilever (face x = 0 clamped, unit downward load split over the bottom edge at x = 64, volume fraction 0.3,
density bounds 1e-3 and 1, E = 1, nu = 0.3) from the paper's initial point, with the paper's parameters
(eps_PBM = 1e-5, beta = gamma = 0.3, p_min = 1e-8, eps_NWT from 1 down to 1e-3) and MG-MINRES inner solves
(5-level Galerkin V-cycle, initial eps_MR = 1e-4 sqrt(n) adapted as in Section 5.3).

Only oracle/ and synthetic/ are used: the stored values are the oracle's. Run from the repository root:
    python tests/golden/make_pbm_cant64_reference.py
"""
import json
import math
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import synthetic  # noqa: E402
from oracle import fem, pbm  # noqa: E402


def main():
    nx, ny, nz = 64, 32, 32
    g = fem.Grid(nx, ny, nz, "cantilever")
    f = synthetic.load_vector(nx, ny, nz, "end_edge")
    pb = pbm.Problem(g, f, 0.3 * g.m, 1e-3, 1.0)
    t0 = time.time()
    res = pbm.pbm(pb, eps_pbm=1e-5, eps_mr=1e-4 * math.sqrt(g.n), levels=5)
    st = res.state
    out = {
        "workload": "64x32x32 cantilever, end_edge load, volume fraction 0.3, rho in [1e-3, 1], E 1, nu 0.3",
        "algorithm": "oracle/pbm.py pbm(eps_pbm=1e-5, eps_mr=1e-4 sqrt(n), levels=5), paper's initial point",
        "compliance": float(0.5 * pb.f @ pbm.masked(pb, st.u)),
        "volume": float(st.rho.sum()),
        "gap_ratio": float(res.gap_ratio),
        "outer": int(res.outer),
        "newton": int(res.newton),
        "minres": int(res.minres),
        "rho_min": float(st.rho.min()),
        "rho_max": float(st.rho.max()),
        "seconds": time.time() - t0,
    }
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "pbm_cant64_oracle.json")
    with open(path, "w") as fh:
        json.dump(out, fh, indent=1)
        fh.write("\n")
    print(json.dumps(out))


if __name__ == "__main__":
    main()
