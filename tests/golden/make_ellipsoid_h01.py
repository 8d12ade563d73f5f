"""Writes the oracle's FP64 solve of the ellipsoid at h = 0.1 (M = 44 597) for the GPU solve tests.

The convergence study of Sec. 3.3.2 on an ellipsoid (semi-axes 4, 3, 2; three seeded charges; eps_I = 1,
eps_E = 80, kappa = 0.1257; tube 2h): the system of Eq. (2.30) solved by the oracle's GMRES to 1e-12,
psi_rxn at the charges by Eq. (2.31) and G_pol by Eq. (3.3).  The file keeps G_pol, psi_rxn, the
largest |psi| and |dpsi_n| and both at 512 seeded sample nodes (by grid linear index).  Calls only
oracle/ and the seeded input generators; run from the repo root:
    python tests/golden/make_ellipsoid_h01.py
"""
import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import synthetic as syn  # noqa: E402
from oracle import energy, tables  # noqa: E402
from oracle.system import OracleSystem  # noqa: E402

H = 0.1
N_SAMPLES = 512


def main():
    t0 = time.time()
    prob = syn.ellipsoid_problem(h=H)
    S = OracleSystem.from_problem(prob, tables=tables.build_tables(os.path.join(ROOT, "oracle", "_build", "cache")))
    psi, dpsi, info = S.solve(tol=1e-12, max_iter=400)
    assert info["converged"], info
    G, prx = energy.polarization_energy(S, psi, dpsi)
    rng = np.random.Generator(np.random.PCG64(7))
    idx = np.sort(rng.choice(S.M, size=N_SAMPLES, replace=False))
    out = {
        "citation": "Sec. 3.3.2 convergence study (ellipsoid), system Eq. (2.30), psi_rxn Eq. (2.31), "
                    "G_pol Eq. (3.3); oracle FP64 GMRES to 1e-12",
        "workload": "synthetic.ellipsoid_problem(h=0.1): semi-axes 4, 3, 2, three seeded charges, "
                    "eps_in 1, eps_out 80, kappa 0.1257, tube 2h",
        "M": int(S.M), "iterations": int(info["iterations"]), "G_pol": G, "psi_rxn": [float(v) for v in prx],
        "psi_max": float(np.max(np.abs(psi))), "dpsi_max": float(np.max(np.abs(dpsi))),
        "grid_index": [int(v) for v in S.geo.lin[idx]],
        "psi": [float(v) for v in psi[idx]], "dpsi": [float(v) for v in dpsi[idx]],
        "oracle_seconds": time.time() - t0,
    }
    with open(os.path.join(HERE, "ellipsoid_h0.1_oracle_solve.json"), "w") as f:
        json.dump(out, f, indent=0)
    print(f"M={S.M} iterations={info['iterations']} G_pol={G:.12e} ({time.time() - t0:.0f} s)")


if __name__ == "__main__":
    main()
