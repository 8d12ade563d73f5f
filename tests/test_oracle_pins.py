"""Pins of the CPU oracle against closed forms, identities and independent computations.

Each test fixes a quantity by something other than the oracle itself:
closed forms (lattice zeta constant, Kirkwood energy, sphere geometry),
an independent Ewald evaluation of the correction weights, integral
identities of the boundary operators on a sphere, and a dense direct solve.
Several tests plant a mistake in a copy of the oracle's data and check that
the pin catches it.
"""
import json
import math
import os

import numpy as np
import pytest
from scipy.special import gamma, gammainc, gammaincc

import synthetic as syn
from oracle import correction, energy, exact, geometry, gmres, tables
from oracle.system import OracleSystem

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ---------------------------------------------------------------- weights
def _ewald_weight(k, a):
    """omega[|y|^-1 e^{i k psi}; a] = -(regularised sum_{n != 0} f(n - a)) by Ewald splitting.

    Written independently of the oracle from the Mellin representation
    |x|^{-2s} = pi^s/Gamma(s) int t^{s-1} e^{-pi t |x|^2} dt, s = (k+1)/2,
    split at t = 1, the small-t part Poisson-summed with Hecke's identity.
    """
    s = (k + 1) / 2.0
    R = 8
    rng = np.arange(-R, R + 1)
    n1, n2 = [v.ravel().astype(float) for v in np.meshgrid(rng, rng, indexing="ij")]
    nz = ~((n1 == 0) & (n2 == 0))
    x1, x2 = n1 - a[0], n2 - a[1]
    r2 = x1 * x1 + x2 * x2
    real = np.sum(((x1 + 1j * x2) ** k * gammaincc(s, np.pi * r2) / r2 ** s)[nz])
    ra2 = a[0] ** 2 + a[1] ** 2
    if ra2 > 0:
        zero = -(-a[0] - 1j * a[1]) ** k * gammainc(s, np.pi * ra2) / ra2 ** s
    else:
        zero = -(np.pi ** s) / gamma(s + 1) if k == 0 else 0.0
    m1, m2 = n1[nz], n2[nz]
    mr2 = m1 * m1 + m2 * m2
    rec = (-1j) ** k * np.sum((m1 + 1j * m2) ** k * np.exp(-2j * np.pi * (m1 * a[0] + m2 * a[1]))
                              * gammaincc(s, np.pi * mr2) / mr2 ** s)
    m0 = -2.0 if k == 0 else 0.0
    return -(real + zero + rec + m0)


def test_weight_square_lattice_constant():
    g = json.load(open(os.path.join(GOLDEN, "square_lattice_zeta.json")))
    closed = -4.0 * g["zeta_half"] * g["dirichlet_beta_half"]
    om, n_used = tables.omega_limit([0.0], [0.0], kmax=0)
    assert abs(om[0, 0].real - closed) < 1e-11
    assert abs(om[0, 0].imag) < 1e-14


@pytest.mark.parametrize("k,a", [(0, (0.3, -0.2)), (2, (0.3, -0.2)), (4, (0.1, 0.45)), (6, (-0.49, 0.2)),
                                 (8, (0.5, -0.5)), (12, (-0.3, -0.37)), (16, (0.25, 0.33)), (2, (0.56, 0.0))])
def test_weight_limit_matches_ewald(k, a):
    om, _ = tables.omega_limit([a[0]], [a[1]], kmax=k, kstep=2)
    ref = _ewald_weight(k, a)
    assert abs(om[0, k // 2] - ref) < 2e-11 * max(1.0, abs(ref))


def test_weight_table_symmetries(oracle_tables):
    T = oracle_tables
    # even harmonics: omega(-alpha, -beta) = omega(alpha, beta)
    assert np.allclose(T, T[:, :, ::-1, ::-1], atol=1e-12, rtol=0)
    c = tables.HALF
    for mi, k in enumerate(tables.MODES):
        assert abs(T[1, mi, c, c]) < 1e-12              # sin terms vanish at (0, 0)
        if k % 4 == 2:
            assert abs(T[0, mi, c, c]) < 1e-12          # square-lattice symmetry
    # the table is smooth: interpolation reproduces off-grid limits (the high
    # harmonics oscillate faster in (alpha, beta), so their error is larger; they
    # enter the weights multiplied by geometrically small Fourier coefficients)
    for (a, b) in [(0.123, -0.377), (-0.49, 0.31), (0.07, 0.0)]:
        Ti = tables.interpolate(T, a, b)
        om, _ = tables.omega_limit([a], [b], kmax=tables.N_MODES, kstep=2)
        tol = 2e-7 * 4.0 ** (np.array(tables.MODES) / 2)
        assert np.all(np.abs(Ti[0] - om[0].real) < tol)
        assert np.all(np.abs(Ti[1] - om[0].imag) < tol)


def test_weight_of_constant_is_one():
    for (a, b) in [(0.0, 0.0), (0.3, -0.41), (-0.5, 0.5)]:
        assert abs(tables.omega_one(a, b, 2.0 ** -7) - 1.0) < 1e-8


def test_plane_rule_second_order(oracle_tables):
    """2-D corrected rule (Eq. (2.23)) on s(u - u0) v(u), s = |y|^-1 l(theta), l anisotropic.

    Uses the oracle's FFT + table interpolation path (correction.fourier_coefficients,
    tables.interpolate).  Exact value by polar quadrature about u0.
    """
    T = oracle_tables
    Amat = np.array([[1.0, 0.3], [-0.2, 0.7]])

    def ell(th):
        c, s = np.cos(th), np.sin(th)
        v1 = Amat[0, 0] * c + Amat[0, 1] * s
        v2 = Amat[1, 0] * c + Amat[1, 1] * s
        return 1.0 / np.sqrt(v1 * v1 + v2 * v2)

    v = lambda x, y: np.exp(-(x * x + 2 * y * y) / 4 + 0.3 * x)  # noqa: E731
    a_c, b_c = correction.fourier_coefficients(ell(2 * np.pi * np.arange(correction.N_SAMPLES)
                                                   / correction.N_SAMPLES)[None, :])
    shift = np.array([0.371, -0.217])        # fixed (alpha, beta): u0 = h (alpha, beta)
    th = 2 * np.pi * np.arange(512) / 512
    rr, wr = np.polynomial.legendre.leggauss(300)
    Rmax = 16.0
    r = 0.5 * Rmax * (rr + 1)
    wr = 0.5 * Rmax * wr
    Ti = tables.interpolate(T, shift[0], shift[1])[None]
    om = correction.weights_from_coefficients(a_c, b_c, Ti)[0]
    errs, errs_plain = [], []
    for h in (0.1, 0.05, 0.025):
        u0 = h * shift
        X = u0[0] + r[:, None] * np.cos(th)[None, :]
        Y = u0[1] + r[:, None] * np.sin(th)[None, :]
        exact_val = np.sum(wr[:, None] * v(X, Y) * ell(th)[None, :]) * (2 * np.pi / 512)
        n = np.arange(-int(14 / h), int(14 / h) + 1)
        XX, YY = np.meshgrid(h * n, h * n, indexing="ij")
        dx, dy = XX - u0[0], YY - u0[1]
        c = len(n) // 2
        dx[c, c] = 1.0                           # the node nearest to u0 is omitted below
        val = ell(np.arctan2(dy, dx)) / np.hypot(dx, dy) * v(XX, YY)
        mask = np.ones_like(val, bool)
        mask[c, c] = False
        plain = h * h * np.sum(val[mask])
        corrected = plain + h * om * v(0.0, 0.0)
        errs.append(abs(corrected - exact_val))
        errs_plain.append(abs(plain - exact_val))
    assert errs[1] < errs[0] / 3.0 and errs[2] < errs[1] / 3.0      # second order (4x per halving)
    assert errs[2] < 5e-4
    assert errs[2] < errs_plain[2] / 100.0          # the correction is what makes it accurate


# ---------------------------------------------------------------- geometry
def test_sphere_geometry_and_area(sphere_c1):
    prob, S = sphere_c1
    geo = S.geo
    R = 2.0
    r = np.linalg.norm(geo.y, axis=1)
    # normals and closest points (second-order FD on an exact distance)
    assert np.max(np.linalg.norm(geo.n - geo.y / r[:, None], axis=1)) < 5e-3
    assert np.max(np.abs(np.linalg.norm(geo.P, axis=1) - R)) < 5e-3
    # level-set curvatures 1/(R + d), Jacobian (R/(R + d))^2, surface curvature 1/R
    assert np.max(np.abs(geo.kprime - (1.0 / r)[:, None])) < 2e-2
    assert np.max(np.abs(geo.J - (R / r) ** 2)) < 2e-2
    assert np.max(np.abs(geo.kappa_s - 1.0 / R)) < 2e-2
    # tube rule of Eq. (2.6) with f = 1: area 4 pi R^2
    assert abs(S.area() / (4 * np.pi * R * R) - 1.0) < 1e-4


def test_ellipsoid_area(oracle_tables):
    prob = syn.ellipsoid_problem(h=0.2)
    geo = geometry.tube_geometry(prob.grid.n, prob.grid.origin, prob.grid.h, prob.sdist, prob.tube)
    A_ref = syn.ellipsoid_area((4.0, 3.0, 2.0))
    assert abs(geometry.tube_area(geo) / A_ref - 1.0) < 2e-3


def test_tube_and_stencil_checks():
    grid = syn.box_grid((-2.5,) * 3, (2.5,) * 3, 0.25)
    sd = syn.sphere_sdist(grid, 2.0)
    with pytest.raises(ValueError):
        geometry.tube_geometry(grid.n, grid.origin, grid.h, sd, 0.5)   # stencil leaves the grid


# ---------------------------------------------------------------- correction nodes
def test_correction_nodes_structure(sphere_c1):
    prob, S = sphere_c1
    c = S.corr
    counts = np.diff(c.ptr)
    # at most 2 eps/h + 1 = 5 corrected nodes per target at eps = 2h (Sec. 2.5, figure of Omega)
    assert counts.max() <= 5 and counts.min() >= 1
    assert 3.0 <= counts.mean() <= 5.0
    # the target itself is a correction node with (alpha, beta) = (0, 0) (it lies on its normal line)
    for i in range(S.M):
        s, e = c.ptr[i], c.ptr[i + 1]
        hit = np.nonzero(c.node[s:e] == i)[0]
        assert hit.size == 1
        assert abs(c.alpha[s + hit[0]]) < 1e-9 and abs(c.beta[s + hit[0]]) < 1e-9
    assert np.all((c.alpha >= -0.5) & (c.alpha < 0.5) & (c.beta >= -0.5) & (c.beta < 0.5))


# ---------------------------------------------------------------- operator identities
def _consistency(S, q=1.0, R=2.0):
    psiG, dpsiG = exact.sphere_boundary_values(q, R, S.eps_in, S.eps_out, S.kappa)
    M = S.M
    p = np.concatenate([np.full(M, psiG), np.full(M, dpsiG)])
    g = S.rhs()
    r = S.matvec(p) - g
    return (np.abs(r[:M]).mean() / np.abs(g[:M]).mean(), np.abs(r[M:]).mean() / np.abs(g[M:]).mean())


def test_rhs_on_sphere(sphere_c1):
    prob, S = sphere_c1
    g = S.rhs()
    M = S.M
    R = np.linalg.norm(S.geo.P, axis=1)
    assert np.allclose(g[:M], 1.0 / (4 * np.pi * R), rtol=1e-12)
    assert np.allclose(g[M:], -1.0 / (4 * np.pi * R * R), rtol=1e-2)


def test_sphere_kernel_integrals_closed_form():
    # the 1-D sphere integrals reproduce the Gauss identity and the Yukawa double layer
    R, kap = 2.0, 0.7
    I = exact.sphere_kernel_integrals(R, 1.0, 1.0, kap)
    dl = exact.sphere_double_layer_yukawa(R, kap)
    assert abs(I["K11"] - (-0.5 - dl)) < 1e-12
    assert abs(exact.sphere_kernel_integrals(R, 1.0, 1.0, 1e-9)["K11"]) < 1e-8


def test_exact_solution_satisfies_bie():
    # the exact boundary values satisfy the continuous BIE (1.2)-(1.3) on the sphere
    for (eo, kap) in [(80.0, 0.1257), (4.0, 3.0)]:
        R, q = 2.0, 1.0
        psi, dpsi = exact.sphere_boundary_values(q, R, 1.0, eo, kap)
        I = exact.sphere_kernel_integrals(R, 1.0, eo, kap)
        lam1, lam2 = 0.5 * (1 + eo), 0.5 * (1 + 1.0 / eo)
        g1, g2 = q / (4 * np.pi * R), -q / (4 * np.pi * R * R)
        assert abs(lam1 * psi + I["K11"] * psi - I["K12"] * dpsi - g1) < 1e-10 * abs(g1)
        assert abs(lam2 * dpsi + I["K21"] * psi - I["K22"] * dpsi - g2) < 1e-10 * abs(g2)


def test_double_layer_identity(sphere_c1):
    prob, S = sphere_c1
    M = S.M
    row1 = S.matvec(np.concatenate([np.ones(M), np.zeros(M)]))[:M]
    ex = S.lam1 - 0.5 - S.ratio * exact.sphere_double_layer_yukawa(2.0, S.kappa)
    assert np.abs(row1 - ex).mean() < 1e-3 * ex


def test_operator_consistency_and_planted_mistakes(oracle_tables):
    """A applied to the exact sphere solution returns g up to O(h); wrong corrections do not."""
    prob = syn.sphere_problem(h=0.25, kappa=3.0, eps_out=4.0)
    S = OracleSystem.from_problem(prob, tables=oracle_tables)
    r1, r2 = _consistency(S)
    assert r1 < 2e-3 and r2 < 5e-3
    base = (S.omega11.copy(), S.omega21.copy(), S.omega22.copy(), S.omega12)
    for which in range(4):
        vals = list(base)
        vals[which] = -vals[which]                   # planted sign error
        S.omega11, S.omega21, S.omega22, S.omega12 = vals
        b1, b2 = _consistency(S)
        assert max(b1 / r1, b2 / r2) > 3.0, which
    S.omega11, S.omega21, S.omega22, S.omega12 = base
    S.omega21 = base[1] / S.kappa ** 2               # planted: the printed s0^(21) without kappa^2
    b1, b2 = _consistency(S)
    assert b2 / r2 > 3.0


def test_consistency_converges(oracle_tables):
    errs = []
    for h in (0.25, 0.125):
        S = OracleSystem.from_problem(syn.sphere_problem(h=h), tables=oracle_tables)
        errs.append(max(_consistency(S)))
    assert errs[1] < 0.6 * errs[0]


# ---------------------------------------------------------------- solver and energy
def test_gmres_matches_dense_solve(oracle_tables):
    prob = syn.sphere_problem(h=0.25, R=1.0, half_box=1.75)
    S = OracleSystem.from_problem(prob, tables=oracle_tables)
    assert S.M < 1200
    A = S.dense()
    g = S.rhs()
    x_ref = np.linalg.solve(A, g)
    psi, dpsi, info = S.solve(tol=1e-14)
    x = np.concatenate([psi, dpsi])
    assert info["converged"]
    assert np.max(np.abs(x - x_ref)) < 1e-11 * np.max(np.abs(x_ref))
    # restarted GMRES reaches the same solution
    x2, _ = gmres.gmres(S.matvec, g, tol=1e-14, max_iter=400, restart=8)
    assert np.max(np.abs(x2 - x_ref)) < 1e-10 * np.max(np.abs(x_ref))


def test_reaction_potential_of_exact_solution(sphere_c1):
    prob, S = sphere_c1
    gold = json.load(open(os.path.join(GOLDEN, "kirkwood_sphere_R2.json")))
    M = S.M
    prx = energy.reaction_potential(S, np.full(M, gold["psi_boundary"]), np.full(M, gold["dpsi_boundary"]),
                                    np.zeros((1, 3)))
    assert abs(prx[0] / gold["psi_rxn_0"] - 1.0) < 1e-3


def test_kirkwood_energy(sphere_c1):
    prob, S = sphere_c1
    gold = json.load(open(os.path.join(GOLDEN, "kirkwood_sphere_R2.json")))
    psi, dpsi, info = S.solve(tol=1e-12)
    assert info["converged"] and 5 <= info["iterations"] <= 40
    G, prx = energy.polarization_energy(S, psi, dpsi)
    assert abs(G / gold["G_pol"] - 1.0) < 5e-4
    assert np.abs(psi / gold["psi_boundary"] - 1.0).max() < 2e-2
    assert np.abs(dpsi / gold["dpsi_boundary"] - 1.0).max() < 2e-2


# ---------------------------------------------------------------- K-reg / HYB (Secs. 2.3, 3.2)
def test_kreg_constant_is_disc_average():
    """C12 of Sec. 2.3 equals the tangent-disc average of (G0 - Gk) (independent quadrature)."""
    from oracle.correction import kreg_constant
    for kappa, tau in [(0.1257, 0.5), (1.0, 0.25), (3.0, 0.1)]:
        x, w = np.polynomial.legendre.leggauss(200)
        r = 0.5 * tau * (x + 1)
        wr = 0.5 * tau * w
        avg = np.sum(wr * 2 * np.pi * r * (1 - np.exp(-kappa * r)) / (4 * np.pi * r)) / (np.pi * tau * tau)
        assert abs(kreg_constant(kappa, tau) - avg) < 1e-13
    assert kreg_constant(0.0, 0.5) == 0.0


def test_kreg_is_first_order_and_worse_than_ctr2(oracle_tables):
    """Paper Sec. 2.6: K-reg has order 1 and an error constant far above CTR2's."""
    gold = json.load(open(os.path.join(GOLDEN, "kirkwood_sphere_R2.json")))
    prob = syn.sphere_problem(h=0.25)
    S = OracleSystem.from_problem(prob, tables=oracle_tables, method="kreg")
    assert S.geo.bad.all() and np.allclose(S.geo.J, 1.0)
    psi, dpsi, info = S.solve(tol=1e-11)
    G, _ = energy.polarization_energy(S, psi, dpsi)
    err_kreg = abs(G / gold["G_pol"] - 1)
    assert 1e-2 < err_kreg < 0.1
    # every K-reg row corrects the nodes of its tangent cylinder (tens of nodes at tau = 2h)
    assert 30 < np.diff(S.corr.ptr).mean() < 70 and np.all(S.corr.kreg)


def test_hybrid_classification_on_smooth_and_kinked_surfaces(oracle_tables):
    prob = syn.ellipsoid_problem(h=0.2)
    geo = geometry.tube_geometry(prob.grid.n, prob.grid.origin, prob.grid.h, prob.sdist, prob.tube)
    assert not geo.bad.any()                 # smooth, resolved: HYB is plain CTR2
    mol = syn.molecule_problem(n_atoms=30, seed=1, h=0.5)
    geo = geometry.tube_geometry(mol.grid.n, mol.grid.origin, mol.grid.h, mol.sdist, mol.tube)
    assert geo.bad.any() and not geo.bad.all()
    assert np.all(geo.J[geo.bad] == 1.0) and np.all(np.isfinite(geo.W)) and np.all(geo.W >= 0)


def test_hybrid_threshold_on_a_quadratic_level_set():
    """HYB classification (Sec. 3.2) against its closed form: with d = (|x|^2 - 1)/2 the finite differences
    are exact, the surface curvature at a node is 1/(r - d), r = |y|, and a node is bad iff
    (eps + h) / (r - d) >= 0.8.  eps + h = 0.75 puts the threshold inside the tube: nodes with
    r <= 1 - sqrt(1/8) or r >= 1 + sqrt(1/8) are bad, the band between is not."""
    prob = syn.quadratic_sphere_problem(h=0.1, tube=0.65)
    g = prob.grid
    geo = geometry.tube_geometry(g.n, g.origin, g.h, prob.sdist, prob.tube)
    r = np.linalg.norm(geo.y, axis=1)
    val = (prob.tube + g.h) / (r - geo.d)
    clear = np.abs(val - 0.8) > 1e-9
    assert clear.sum() > 0.99 * geo.M
    assert np.array_equal(geo.bad[clear], val[clear] >= 0.8)
    assert geo.bad.any() and not geo.bad.all()
    assert np.all(geo.bad[r < 0.6]) and not np.any(geo.bad[(r > 0.7) & (r < 1.3)]) and np.all(geo.bad[r > 1.4])
    # the closed form's other parts: level-set curvature 1/r (both principal values), W uses J = 1 at bad nodes
    kp = geo.kprime[~geo.bad]
    assert np.allclose(kp, 1.0 / r[~geo.bad, None], rtol=1e-12)
    assert np.all(geo.J[geo.bad] == 1.0)


def test_kreg_cylinder_on_a_flat_face():
    """K-reg correction sets (Sec. 2.3) where the surface is a plane (the centre of a flat face, z = c): the
    tube nodes whose tangent-plane distance to the target's P is below tau = 2h are the 9 lattice columns
    with a^2 + b^2 < 4 times the 3 tube layers |z - c| < 2h, 27 nodes for every such target; a brute force
    over every tube node on that face gives the same sets."""
    from oracle.correction import correction_nodes
    prob = syn.flat_cylinder_problem(h=0.25, R=1.5, c=1.0)
    g = prob.grid
    geo = geometry.tube_geometry(g.n, g.origin, g.h, prob.sdist, prob.tube, method="kreg")
    assert geo.bad.all()
    ent, _ = correction_nodes(geo)
    tgt = ent[:, 0].astype(int)
    node = ent[:, 1].astype(int)
    tau = 2.0 * g.h
    rho = np.linalg.norm(geo.y[:, :2], axis=1)
    face = (rho <= 0.4 + 1e-9) & (np.abs(np.abs(geo.y[:, 2]) - 1.0) < 0.3)
    assert np.allclose(np.abs(geo.n[face, 2]), 1.0, atol=1e-14)
    counts = np.bincount(tgt, minlength=geo.M)
    assert face.sum() >= 50 and np.all(counts[face] == 27)
    for i in np.nonzero(face)[0]:
        same_side = np.sign(geo.y[:, 2]) == np.sign(geo.y[i, 2])
        v = geo.y - geo.P[i]
        t = v - np.outer(v @ geo.n[i], geo.n[i])
        brute = np.nonzero(same_side & (np.sum(t * t, axis=1) < tau * tau))[0]
        assert np.array_equal(np.sort(node[tgt == i]), brute)


def test_oracle_torus_area_converges():
    """Rotated torus of Sec. 3.3.2 (R1 = 1, R2 = 1/2): the tube rule with J_h (Eq. 2.6, f = 1) against the
    closed form 4 pi^2 R1 R2 at eps = 2h; at least second order (the paper tabulates 1e-6..1e-5 errors)."""
    from oracle.geometry import tube_area, tube_geometry
    errs = []
    for h in (0.1, 0.05):
        p = syn.torus_problem(h)
        g = p.grid
        geo = tube_geometry(g.n, g.origin, g.h, p.sdist, p.tube)
        errs.append(abs(tube_area(geo) / syn.torus_area() - 1))
    assert errs[0] < 5e-4 and errs[1] < 1e-4
    assert errs[0] / errs[1] > 4.0
