"""Tube nodes and their geometry from a signed distance grid (Sec. 2.1).

Follows Sec. 2.1 and the finite-difference remark of Sec. 3.3.1:
  * tube nodes: T^h_eps = {grid nodes with |d| < eps}, Eq. (2.4) with the
    boundary excluded (phi(+-1) = 0 gives those nodes zero weight anyway);
  * gradient: second-order central differences; Hessian: central difference
    of the central-difference gradient (5 nodes per direction, Sec. 3.3.1);
  * unit normal n = grad d / |grad d| (outward, since d > 0 outside);
  * closest point P = y - d n  (Sec. 2.1, P(x) = x - d grad d);
  * level-set principal curvatures k'_1, k'_2 and directions tau_1, tau_2 from
    the Hessian restricted to the tangent plane (divided by |grad d|);
  * Jacobian J = (1 - d k'_1)(1 - d k'_2): Eq. (2.8) written with d > 0 outside
    and level-set curvatures (1 + 2 d H + d^2 G with the paper's sign of d);
  * surface principal curvatures k_i = k'_i / (1 - d k'_i), and the matrix of
    Theorem (Sec. 2.4.1) M = diag(-k_1, -k_2): the surface is locally
    P + w + (1/2) w^T M w n in principal coordinates w (a sphere: M = -I/R);
  * W = J * delta_eps(d), delta_eps(eta) = phi(eta/eps)/eps with
    phi(x) = (1 + cos(pi x))/2 on |x| <= 1 (Sec. 2.6).

Hybrid classification (Sec. 3.2, HYB-IBIM): a node is "bad" when its
finite-difference geometry cannot be trusted -- reading of the paper's "stencil
negatively impacted by the curvature discontinuity": a non-finite value, or a
surface principal curvature with |k_i| (eps + h) >= 0.8, i.e. the tube (and
every correction plane, |eta| <= eps + h) would reach within 20% of the focal
distance 1/|k_i|.  Bad nodes take J = 1 (Eq. (3.2)); their rows use K-reg
(module correction).  Method "kreg" marks every node bad (the K-reg method of
Sec. 2.3 with J = 1, as in the paper's comparison).

Arithmetic order matters where a floating-point value decides an integer
(tube membership, the correction planes and nodes): y = origin + h*i,
g_c = (d[+] - d[-]) / (2h), |g| = sqrt((g0*g0 + g1*g1) + g2*g2), n_c = g_c/|g|,
P_c = y_c - d*n_c, each a single IEEE FP64 operation without fusion.

Parity status: pinned (sphere: J, curvatures, area; ellipsoid area).
"""
from __future__ import annotations

import dataclasses

import numpy as np


@dataclasses.dataclass
class TubeGeometry:
    h: float
    eps: float
    grid_n: tuple
    origin: tuple
    lin: np.ndarray        # (M,) int64 grid linear index of each tube node
    ijk: np.ndarray        # (M, 3) int64 grid index (i, j, k)
    y: np.ndarray          # (M, 3) node coordinates
    d: np.ndarray          # (M,) signed distance
    grad_norm: np.ndarray  # (M,) |grad d|
    n: np.ndarray          # (M, 3) unit normal
    P: np.ndarray          # (M, 3) closest point
    kprime: np.ndarray     # (M, 2) level-set principal curvatures
    tau: np.ndarray        # (M, 2, 3) principal directions
    kappa_s: np.ndarray    # (M, 2) surface principal curvatures (convex > 0)
    bad: np.ndarray        # (M,) bool: hybrid classification (Sec. 3.2)
    J: np.ndarray          # (M,)
    W: np.ndarray          # (M,) J * delta_eps(d)
    node_of: np.ndarray    # grid-sized int64 map: linear index -> node id or -1

    @property
    def M(self) -> int:
        return int(self.lin.size)


def phi(x):
    """Averaging kernel of Sec. 2.6: (1 + cos(pi x))/2 on |x| <= 1, else 0."""
    x = np.asarray(x, dtype=np.float64)
    return np.where(np.abs(x) <= 1.0, 0.5 * (1.0 + np.cos(np.pi * x)), 0.0)


def delta_eps(eta, eps):
    """delta_eps(eta) = phi(eta/eps)/eps, Eq. (2.7)."""
    return phi(np.asarray(eta) / eps) / eps


BAD_CURVATURE = 0.8   # |k_i| (eps + h) at or above this marks a node bad


def tube_geometry(grid_n, origin, h, sdist, eps, method: str = "hyb") -> TubeGeometry:
    """method: "hyb" (CTR2 with the hybrid classification) or "kreg" (every node bad)."""
    nx, ny, nz = (int(v) for v in grid_n)
    D = np.asarray(sdist, dtype=np.float64).reshape(nz, ny, nx)
    flat = D.ravel()
    lin = np.nonzero(np.abs(flat) < eps)[0].astype(np.int64)
    if lin.size == 0:
        raise ValueError("empty tube")
    i = lin % nx
    j = (lin // nx) % ny
    k = lin // (nx * ny)
    ijk = np.stack([i, j, k], axis=1)
    for c, nc in enumerate((nx, ny, nz)):
        if ijk[:, c].min() < 2 or ijk[:, c].max() > nc - 3:
            raise ValueError("tube node within 2 nodes of the grid boundary")

    def at(di, dj, dk):
        return D[k + dk, j + dj, i + di]

    two_h = 2.0 * h
    g = np.stack([(at(1, 0, 0) - at(-1, 0, 0)) / two_h,
                  (at(0, 1, 0) - at(0, -1, 0)) / two_h,
                  (at(0, 0, 1) - at(0, 0, -1)) / two_h], axis=1)
    four_h2 = 4.0 * h * h
    unit = [(1, 0, 0), (0, 1, 0), (0, 0, 1)]
    H = np.zeros((lin.size, 3, 3))
    for a in range(3):
        ea = unit[a]
        H[:, a, a] = (at(*[2 * v for v in ea]) - 2.0 * at(0, 0, 0) + at(*[-2 * v for v in ea])) / four_h2
        for b in range(a + 1, 3):
            eb = unit[b]
            pp = at(ea[0] + eb[0], ea[1] + eb[1], ea[2] + eb[2])
            pm = at(ea[0] - eb[0], ea[1] - eb[1], ea[2] - eb[2])
            mp = at(-ea[0] + eb[0], -ea[1] + eb[1], -ea[2] + eb[2])
            mm = at(-ea[0] - eb[0], -ea[1] - eb[1], -ea[2] - eb[2])
            H[:, a, b] = H[:, b, a] = (pp - pm - mp + mm) / four_h2

    gn = np.sqrt(g[:, 0] * g[:, 0] + g[:, 1] * g[:, 1] + g[:, 2] * g[:, 2])
    n = g / gn[:, None]
    dd = flat[lin]
    y = np.stack([origin[0] + h * i.astype(np.float64),
                  origin[1] + h * j.astype(np.float64),
                  origin[2] + h * k.astype(np.float64)], axis=1)
    P = y - dd[:, None] * n

    # tangent basis: e1 = n x e_c (c = axis of smallest |n_c|), e2 = n x e1
    c_small = np.argmin(np.abs(n), axis=1)
    ec = np.eye(3)[c_small]
    e1 = np.cross(n, ec)
    e1 /= np.linalg.norm(e1, axis=1)[:, None]
    e2 = np.cross(n, e1)
    E = np.stack([e1, e2], axis=1)                               # (M, 2, 3)
    S = np.einsum("mai,mij,mbj->mab", E, H, E) / gn[:, None, None]
    S = 0.5 * (S + np.transpose(S, (0, 2, 1)))
    kp, V = np.linalg.eigh(S)                                    # ascending
    tau = np.einsum("mab,mai->mbi", V, E)                        # tau[:, b] = sum_a V[a, b] E[a]
    J = (1.0 - dd * kp[:, 0]) * (1.0 - dd * kp[:, 1])
    ks = kp / (1.0 - dd[:, None] * kp)
    finite = np.isfinite(J) & np.all(np.isfinite(ks), axis=1) & np.all(np.isfinite(tau.reshape(lin.size, -1)), axis=1)
    with np.errstate(invalid="ignore"):
        bad = (~finite) | (np.max(np.abs(ks), axis=1) * (eps + h) >= BAD_CURVATURE)
    if method == "kreg":
        bad[:] = True
    elif method != "hyb":
        raise ValueError("method must be 'hyb' or 'kreg'")
    J = np.where(bad, 1.0, J)                    # Eq. (3.2): J = 1 at bad nodes
    W = J * delta_eps(dd, eps)
    node_of = np.full(flat.size, -1, dtype=np.int64)
    node_of[lin] = np.arange(lin.size, dtype=np.int64)
    return TubeGeometry(h=float(h), eps=float(eps), grid_n=(nx, ny, nz), origin=tuple(float(v) for v in origin),
                        lin=lin, ijk=ijk, y=y, d=dd, grad_norm=gn, n=n, P=P, kprime=kp, tau=tau,
                        kappa_s=ks, bad=bad, J=J, W=W, node_of=node_of)


def tube_area(geo: TubeGeometry) -> float:
    """Surface area by the tube rule, Eq. (2.6) with f = 1: h^3 sum_j J_j delta_eps(d_j)."""
    return float(geo.h ** 3 * np.sum(geo.W))
