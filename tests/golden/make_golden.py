"""Writes the closed-form golden values used by the oracle pin tests.

Calls only oracle/ (the closed forms of oracle.exact); run from the repo root:
    python tests/golden/make_golden.py
"""
import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import exact  # noqa: E402

q, R, eps_in, eps_out, kappa = 1.0, 2.0, 1.0, 80.0, 0.1257
out = {
    "citation": "Sec. 2.6, exact sphere solution and psi_rxn(0) (one power of q; "
                "Coulomb term with eps_I), G_pol by Eq. (3.3)",
    "q": q, "R": R, "eps_in": eps_in, "eps_out": eps_out, "kappa": kappa,
    "psi_rxn_0": exact.kirkwood_reaction_potential(q, R, eps_in, eps_out, kappa),
    "G_pol": exact.kirkwood_energy(q, R, eps_in, eps_out, kappa),
    "psi_boundary": exact.sphere_boundary_values(q, R, eps_in, eps_out, kappa)[0],
    "dpsi_boundary": exact.sphere_boundary_values(q, R, eps_in, eps_out, kappa)[1],
}
with open(os.path.join(HERE, "kirkwood_sphere_R2.json"), "w") as f:
    json.dump(out, f, indent=1)
print(json.dumps(out, indent=1))
