"""Writes the oracle's reference solution of the 128 x 64 x 64 bridge's reduced Newton system:
tests/golden/bridge128_dz_ref.npy (n + 1 float64 entries, alpha last) and tests/golden/bridge128_dz_ref.json.

The system is eq. (system) with S of eq. (S) at the synthetic Newton state of the bridge workload: the four bottom
corner nodes fixed, a uniform downward traction of total 1 on the top face, densities from 32 Gaussian bumps at
volume fraction 0.2 (seed 0), mu = nu = 1, alpha = 1, p = q = 1, and the displacement u the seeded smooth field
(seed 5, max |u| = 1, zero on the supported dofs). The oracle assembles S and the right-hand side in CSR and solves
with its own MG-MINRES (6-level Galerkin V-cycle, Chebyshev smoothing) driven toward a true relative residual of
1e-14 for at most 80 iterations (FP64 levels off near 2e-14 on this system); anything above 1e-13 is refused. Only oracle/ and synthetic/ are used. The JSON records the residual
reached, the iteration counts to 1e-8 and to the reference, and sums and norms of the inputs (rho, f, u) so that
readers can check they hold the same system. Run from the repository root (about three minutes):
    python tests/golden/make_bridge128_reference.py
"""
import json
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import synthetic  # noqa: E402
from oracle import fem, pbm, solvers  # noqa: E402

HERE = os.path.dirname(os.path.abspath(__file__))
U_SEED, U_AMPLITUDE = 5, 1.0


def inputs():
    """(grid, rho, f, u, state dict) of the bridge workload's reduced system."""
    w = synthetic.WORKLOADS["bridge128"]
    g = fem.Grid(w.nx, w.ny, w.nz, w.bc)
    rho = synthetic.density_for(w)
    f = synthetic.load_vector(w.nx, w.ny, w.nz, w.loads[0])
    u = synthetic.state_displacement(w)
    assert w.extra["u"] == ("smooth", U_SEED, U_AMPLITUDE)
    return w, g, rho, f, u, synthetic.synthetic_state(w, u)


def input_check(rho, f, u) -> dict:
    """Sums and norms of the inputs (float64): a reader regenerates the inputs from synthetic/ and compares these
    to 1e-12 relative (the platforms' exp and sin may differ in the last bit, so no bitwise digest)."""
    ramp = np.linspace(1.0, 2.0, u.size)
    return {"rho_sum": float(rho.sum()), "rho_norm": float(np.linalg.norm(rho)), "f_norm": float(np.linalg.norm(f)),
            "u_norm": float(np.linalg.norm(u)), "u_ramp": float(u @ ramp)}


def main():
    t0 = time.time()
    w, g, rho, f, u, d = inputs()
    pb = pbm.Problem(g, f, d["V"], d["rho_lo"], d["rho_up"])
    st = pbm.State.from_dict(d)
    cf = pbm.coeffs(pb, st)
    S = pbm.assemble_S(pb, st, cf)
    rhs = pbm.rhs_closed(pb, st, cf)
    h = solvers.Hierarchy(g, S, w.levels, has_alpha=True, smoother="chebyshev")
    r8 = solvers.minres(lambda v: S @ v, rhs, h.vcycle, rtol=1e-8, maxit=2000)
    ref = solvers.minres(lambda v: S @ v, rhs, h.vcycle, rtol=1e-14, maxit=80)   # FP64 levels off near 2e-14
    if not ref.relres < 1e-13:
        raise SystemExit(f"reference solve reached only {ref.relres:.3e}")
    np.save(os.path.join(HERE, "bridge128_dz_ref.npy"), ref.x)
    meta = {
        "system": "eq. (system) / eq. (S) of the 128x64x64 bridge workload at its synthetic Newton state",
        "state": {"u": f"synthetic.smooth_displacement(seed={U_SEED}, amplitude={U_AMPLITUDE}), supported dofs 0",
                  "rho": "synthetic.density_bumps(vf=0.2, seed=0)", "mu_lo": 1, "mu_up": 1, "nu_lo": 1, "nu_up": 1,
                  "alpha": 1, "p": 1, "q": 1, "V": w.V, "rho_lo": w.rho_lo, "rho_up": w.rho_up},
        "inputs_check": input_check(rho, f, u),
        "n_plus_1": int(ref.x.size),
        "solver": "oracle MINRES + 6-level Galerkin V-cycle, Chebyshev smoothing",
        "relres": ref.relres, "iterations": ref.iters,
        "iterations_to_1e-8": r8.iters, "relres_at_1e-8": r8.relres,
        "error_of_1e-8_solve": float(np.linalg.norm(r8.x - ref.x) / np.linalg.norm(ref.x)),
        "seconds": time.time() - t0,
    }
    with open(os.path.join(HERE, "bridge128_dz_ref.json"), "w") as fh:
        json.dump(meta, fh, indent=1)
        fh.write("\n")
    print(json.dumps(meta))


if __name__ == "__main__":
    main()
