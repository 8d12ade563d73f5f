"""Closed forms used to pin the oracle (Sec. 2.6 sphere test; tube-rule identities).

Sphere of radius R, one charge q at its centre (Sec. 2.6), read with the two
printed typos fixed: inside, the Coulomb term is q/(4 pi eps_I |x|) (continuity
of psi and of eps psi_n across |x| = R require it), and psi_rxn(0) is
q/(4 pi R) (1/(eps_E (1 + kappa R)) - 1/eps_I) (one power of q; the paper
prints q^2, which is q times this value, i.e. 2 G_pol).

On a sphere every kernel of Eq. (1.4) between two surface points depends on
r = |x - y| only: (x - y).n_x = r^2/(2R), (x - y).n_y = -r^2/(2R),
n_x.n_y = 1 - r^2/(2 R^2), and dsigma = 2 pi r dr/... integrated on r in [0, 2R]
(dsigma = (R / R) 2 pi r dr for a sphere: r dr = R^2 sin(theta) dtheta).

Parity status: these closed forms are the pins; each is checked against an independent route in the
tests (the boundary integral equations on the sphere, the sphere kernel integrals, Kirkwood's energy).
"""
from __future__ import annotations

import math

import numpy as np


def sphere_boundary_values(q, R, eps_in, eps_out, kappa):
    """(psi, interior dpsi/dn) on |x| = R of the exact sphere solution (Sec. 2.6)."""
    psi = q / (4.0 * math.pi * eps_out * (1.0 + kappa * R) * R)
    dpsi = -q / (4.0 * math.pi * eps_in * R * R)
    return psi, dpsi


def kirkwood_reaction_potential(q, R, eps_in, eps_out, kappa):
    """psi_rxn at the centre: q/(4 pi R) (1/(eps_E (1 + kappa R)) - 1/eps_I)."""
    return q / (4.0 * math.pi * R) * (1.0 / (eps_out * (1.0 + kappa * R)) - 1.0 / eps_in)


def kirkwood_energy(q, R, eps_in, eps_out, kappa):
    """G_pol = 1/2 q psi_rxn(0) (Eq. (3.3) with one charge)."""
    return 0.5 * q * kirkwood_reaction_potential(q, R, eps_in, eps_out, kappa)


def sphere_kernel_integrals(R, eps_in, eps_out, kappa, n=4000):
    """int_Gamma K_ij(x, y) dsigma_y for x on the sphere, by Gauss-Legendre in r.

    Integrands written from the definitions of Eq. (1.4) with the sphere
    relations above; every K_ij is at most O(1/r) and r dr makes them smooth.
    """
    xg, wg = np.polynomial.legendre.leggauss(n)
    r = R * (xg + 1.0)             # [0, 2R]
    w = R * wg * 2.0 * math.pi * r  # dsigma = 2 pi r dr
    E = np.exp(-kappa * r)
    fp = 4.0 * math.pi
    dnx = r * r / (2.0 * R)        # (x - y).n_x
    dny = -r * r / (2.0 * R)       # (x - y).n_y
    nn = 1.0 - r * r / (2.0 * R * R)
    dG0_dny = dny / (fp * r ** 3)
    dGk_dny = E * (1 + kappa * r) * dny / (fp * r ** 3)
    dG0_dnx = -dnx / (fp * r ** 3)
    dGk_dnx = -E * (1 + kappa * r) * dnx / (fp * r ** 3)
    d2G0 = nn / (fp * r ** 3) - 3.0 * dnx * dny / (fp * r ** 5)
    d2Gk = E * ((1 + kappa * r) * nn / (fp * r ** 3) - (3 + 3 * kappa * r + (kappa * r) ** 2) * dnx * dny / (fp * r ** 5))
    ratio = eps_out / eps_in
    K11 = dG0_dny - ratio * dGk_dny
    K12 = (1.0 - E) / (fp * r)
    K21 = d2G0 - d2Gk
    K22 = dG0_dnx - (1.0 / ratio) * dGk_dnx
    return {k: float(np.sum(w * v)) for k, v in (("K11", K11), ("K12", K12), ("K21", K21), ("K22", K22))}


def sphere_double_layer_yukawa(R, kappa):
    """int_Gamma dGk/dn_y(x, y) dsigma_y for x on the sphere: -(1 - e^{-2 kappa R}(1 + kappa R))/(2 kappa R)."""
    if kappa == 0.0:
        return -0.5
    return -(1.0 - math.exp(-2.0 * kappa * R) * (1.0 + kappa * R)) / (2.0 * kappa * R)
