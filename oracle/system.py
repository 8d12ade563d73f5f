"""The discrete CTR-IBIM operator and right-hand side (Secs. 2.1, 2.2, 2.5).

Linear system Eq. (2.30), Lambda p + h^3 K W p + h^2 Omega W p = g, row by row
as Eqs. (2.14)-(2.15):

  (A p)_1,i = lambda_1 rho1_i + h^3 sum_{j not in N(i)} W_j (K11 rho1_j - K12 rho2_j)
              + sum_{m in N(i)} W_m (h^2 omega11 rho1_m - h^3 omega12 rho2_m)
  (A p)_2,i = lambda_2 rho2_i + h^3 sum_{j not in N(i)} W_j (K21 rho1_j - K22 rho2_j)
              + sum_{m in N(i)} W_m (h^2 omega21 rho1_m - h^2 omega22 rho2_m)

kernels at (P_i, n_i; P_j, n_j) (Eq. (2.11), K(x, P y)), lambda_1,2 and g_1,2
of Eq. (2.12) evaluated at P_i.  The unknowns are ordered p = [rho1; rho2].

Parity status: pinned (sphere operator identities, brute-force dense solve).
"""
from __future__ import annotations

import math

import numpy as np

from . import native
from . import tables as tb
from .correction import Correction, build_correction, kreg_constant
from .geometry import TubeGeometry, tube_area, tube_geometry
from .gmres import gmres


class OracleSystem:
    """Setup (tube, geometry, correction, rhs) and the operator of Eq. (2.30)."""

    def __init__(self, grid_n, origin, h, sdist, eps_in, eps_out, kappa, charge_xyz, charge_q, tube,
                 tables=None, table_cache=None, rows=None, method="hyb"):
        """rows: optional subset of target rows whose corrections are built (sampled checks);
        matvec is then valid for those rows only.  method: "hyb" (CTR2, K-reg at bad
        nodes, Sec. 3.2) or "kreg" (K-reg everywhere, Sec. 2.3)."""
        self.h = float(h)
        self.eps_in, self.eps_out, self.kappa = float(eps_in), float(eps_out), float(kappa)
        self.ratio = self.eps_out / self.eps_in                         # eps_E / eps_I
        self.lam1 = 0.5 * (1.0 + self.eps_out / self.eps_in)
        self.lam2 = 0.5 * (1.0 + self.eps_in / self.eps_out)
        self.charge_xyz = np.ascontiguousarray(charge_xyz, dtype=np.float64).reshape(-1, 3)
        self.charge_q = np.ascontiguousarray(charge_q, dtype=np.float64).ravel()
        self.geo: TubeGeometry = tube_geometry(grid_n, origin, h, sdist, tube, method=method)
        self.T = tables if tables is not None else tb.build_tables(table_cache)
        self.rows = None if rows is None else np.array(sorted(int(r) for r in rows), dtype=np.int64)
        self.corr: Correction = build_correction(self.geo, self.T, targets=self.rows)
        self.omega11 = (1.0 - self.eps_out / self.eps_in) * self.corr.omega_A
        self.omega22 = (1.0 - self.eps_in / self.eps_out) * self.corr.omega_A
        self.omega21 = self.kappa ** 2 * self.corr.omega_B
        self.omega12 = np.where(self.corr.kreg, kreg_constant(self.kappa, 2.0 * self.h),
                                self.kappa / (4.0 * math.pi))
        self.excl_ptr, self.excl_idx = self.corr.excl_csr()
        self._P = np.ascontiguousarray(self.geo.P)
        self._N = np.ascontiguousarray(self.geo.n)
        self._W = np.ascontiguousarray(self.geo.W)

    @classmethod
    def from_problem(cls, prob, **kw):
        """System for a synthetic.Problem; keyword arguments go to the constructor."""
        g = prob.grid
        return cls(g.n, g.origin, g.h, prob.sdist, prob.eps_in, prob.eps_out, prob.kappa,
                   prob.charge_xyz, prob.charge_q, prob.tube, **kw)

    @property
    def M(self) -> int:
        return self.geo.M

    # ------------------------------------------------------------ rhs
    def rhs(self) -> np.ndarray:
        """g_1 = sum_k q_k/eps_I G0(P_i, z_k), g_2 = sum_k q_k/eps_I dG0/dn_x(P_i, z_k) (Eq. (2.12))."""
        P, n = self.geo.P, self.geo.n
        g1 = np.zeros(self.M)
        g2 = np.zeros(self.M)
        for z, q in zip(self.charge_xyz, self.charge_q):
            d = P - z[None, :]
            r = np.sqrt(np.sum(d * d, axis=1))
            g1 += q / self.eps_in / (4.0 * math.pi * r)
            # dG0/dn_x(x, z) = -(x - z).n_x / (4 pi r^3)
            g2 += q / self.eps_in * (-np.sum(d * n, axis=1)) / (4.0 * math.pi * r ** 3)
        return np.concatenate([g1, g2])

    # ------------------------------------------------------------ operator pieces
    def punctured_sum(self, p: np.ndarray, rows=None):
        """h^3 sum_{j not in N(i)} W_j (K_i1 rho1_j - K_i2 rho2_j) for the requested rows."""
        M = self.M
        p = np.ascontiguousarray(p, dtype=np.float64)
        rho1 = np.ascontiguousarray(p[:M])
        rho2 = np.ascontiguousarray(p[M:])
        rows = np.arange(M, dtype=np.int64) if rows is None else np.ascontiguousarray(rows, dtype=np.int64)
        o1 = np.zeros(rows.size)
        o2 = np.zeros(rows.size)
        native.lib().oracle_punctured_sum(M, native.dptr(self._P), native.dptr(self._N), native.dptr(self._W),
                                          native.dptr(rho1), native.dptr(rho2), self.h, self.kappa, self.ratio,
                                          native.iptr(self.excl_ptr), native.iptr(self.excl_idx),
                                          native.iptr(rows), rows.size, native.dptr(o1), native.dptr(o2))
        return o1, o2

    def correction_apply(self, p: np.ndarray, rows=None):
        """sum_{m in N(i)} W_m (h^2 w11 rho1_m - h^3 w12 rho2_m), W_m (h^2 w21 rho1_m - h^2 w22 rho2_m)."""
        M = self.M
        rho1, rho2 = p[:M], p[M:]
        rows = np.arange(M) if rows is None else np.asarray(rows)
        h2, h3 = self.h ** 2, self.h ** 3
        c = self.corr
        o1 = np.zeros(rows.size)
        o2 = np.zeros(rows.size)
        for t, i in enumerate(rows):
            s, e = c.ptr[i], c.ptr[i + 1]
            m = c.node[s:e]
            Wm = self.geo.W[m]
            o1[t] = np.sum(Wm * (h2 * self.omega11[s:e] * rho1[m] - h3 * self.omega12[s:e] * rho2[m]))
            o2[t] = np.sum(Wm * (h2 * self.omega21[s:e] * rho1[m] - h2 * self.omega22[s:e] * rho2[m]))
        return o1, o2

    def matvec(self, p: np.ndarray, rows=None) -> np.ndarray:
        """(A p) of Eq. (2.30); with `rows`, only those target rows: [out1(rows); out2(rows)]."""
        M = self.M
        p = np.asarray(p, dtype=np.float64)
        r = np.arange(M) if rows is None else np.asarray(rows)
        if self.rows is not None and not np.all(np.isin(r, self.rows)):
            raise ValueError("corrections were built for a subset of rows only")
        s1, s2 = self.punctured_sum(p, r)
        c1, c2 = self.correction_apply(p, r)
        out1 = self.lam1 * p[:M][r] + s1 + c1
        out2 = self.lam2 * p[M:][r] + s2 + c2
        return np.concatenate([out1, out2])

    def dense(self) -> np.ndarray:
        """The 2M x 2M matrix of Eq. (2.30), column by column (tiny problems only)."""
        n = 2 * self.M
        A = np.zeros((n, n))
        e = np.zeros(n)
        for j in range(n):
            e[:] = 0.0
            e[j] = 1.0
            A[:, j] = self.matvec(e)
        return A

    def area(self) -> float:
        return tube_area(self.geo)

    # ------------------------------------------------------------ solve
    def solve(self, tol: float = 1e-13, max_iter: int = 300, restart: int | None = None):
        g = self.rhs()
        x, info = gmres(self.matvec, g, tol=tol, max_iter=max_iter, restart=restart)
        return x[:self.M], x[self.M:], info
