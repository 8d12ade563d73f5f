"""Reaction potential and polarization energy (Secs. 2.6 and 3.3).

psi_rxn(z) of Eq. (2.31) by the standard trapezoidal rule on the tube (the
evaluation point is away from the surface, so no correction applies):
    psi_rxn(z) = h^3 sum_j W_j [ ((eps_E/eps_I) dGk/dn_y - dG0/dn_y)(z, P_j) psi_j
                                 + (G0 - Gk)(z, P_j) dpsi_j ]
G_pol = 1/2 sum_k q_k psi_rxn(z_k), Eq. (3.3).

Parity status: pinned (Kirkwood closed form for the sphere).
"""
from __future__ import annotations

import numpy as np

from . import native


def reaction_potential(system, psi, dpsi, z) -> np.ndarray:
    z = np.ascontiguousarray(np.asarray(z, dtype=np.float64).reshape(-1, 3))
    out = np.zeros(z.shape[0])
    psi = np.ascontiguousarray(psi, dtype=np.float64)
    dpsi = np.ascontiguousarray(dpsi, dtype=np.float64)
    native.lib().oracle_reaction_potential(system.M, native.dptr(system._P), native.dptr(system._N),
                                           native.dptr(system._W), native.dptr(psi), native.dptr(dpsi),
                                           system.h, system.kappa, system.ratio, z.shape[0],
                                           native.dptr(z), native.dptr(out))
    return out


def polarization_energy(system, psi, dpsi):
    prx = reaction_potential(system, psi, dpsi, system.charge_xyz)
    return 0.5 * float(np.sum(system.charge_q * prx)), prx
