"""Far-field acceleration of the dense sum K v (Sec. 2.5) -- TEST INFRASTRUCTURE ONLY.

The paper solves Eq. (2.30) with GMRES and multiplies by the dense part K
through a black-box fast multipole method (Sec. 2.5): the kernel is
interpolated at Chebyshev points of well-separated clusters.  This module is
the plain definition of the approximation the CUDA path computes, a
particle-cluster treecode with the same interpolation:

1. Tree.  Octree over the tube nodes' integer grid indices (i, j, k): a cell
   is the tight integer box [lo, hi) of its nodes; a cell of more than `leaf`
   nodes is split at mid = lo + (hi - lo) // 2 in every axis with hi - lo >= 2
   into octants, visited in the order x-bit + 2 y-bit + 4 z-bit; empty octants
   are dropped.  The leaves in depth-first order give the tree positions
   p = 0..M-1 (perm[p] = node); a leaf lists its nodes by increasing index.
   Every cell is a cluster: the positions [begin, end).
2. Target blocks.  Positions [I BS, (I+1) BS); BS is the arithmetic's block.
3. Separation test (exact integer arithmetic).  A set of nodes with integer
   box [lo, hi) holds its closest points P inside the box widened by
   g = ceil(eps/h) grid units (|y - P| = |d| < eps).  In doubled grid units
   the widened box has centre c2 = lo + hi - 1 and half-extent e2 =
   hi - 1 - lo + 2 g; R2 = |e2|^2 and D2 = |c2_B - c2_C|^2.  With
   theta = tq / 1024, tq = floor(1024 theta + 1/2), the block B and cluster C
   are well separated when theta dist > r_B + r_C, i.e.
       A = tq^2 D2 - 2^20 (R2_B + R2_C) > 0  and  A^2 > 2^42 R2_B R2_C.
4. Lists.  From the root: a well-separated cluster that holds none of the
   block's correction nodes N(i) is approximated when it has more than
   (n+1)^3 nodes and summed directly otherwise; any other cluster is summed
   directly if it is a leaf and opened otherwise.  Direct ("near") position
   ranges are merged when adjacent.  The correction pairs therefore always lie
   in the near field, where they are skipped exactly as in Eqs. (2.14)-(2.15).
5. Interpolation.  A far cluster's proxy points are the tensor Chebyshev
   points of the second kind s_a[m] = c_a + w_a x_m, x_m = cos(m pi / n),
   m = 0..n, on the tight box of its points P (c = (lo+hi)/2,
   w = max((hi-lo)/2, h/1024)); barycentric weights (-1)^m, halved at m = 0, n.
   Lagrange basis l_m(u), u = (t - c)/w, by the barycentric formula (l = e_m
   when u hits x_m exactly), and its derivative l' = (l D)/w with the
   differentiation matrix D[m,q] = (w_q/w_m)/(x_m - x_q), D[m,m] = -sum_q D[m,q].
6. Modified charges (the kernel's source variable y is interpolated:
   G(x, y) ~ sum_k G(x, s_k) L_k(y), so d/dn_y falls on L_k):
       Dk = sum_j a_j n_j . grad L_k(P_j),  Sk = sum_j b_j L_k(P_j),
       a = h^3 W rho1, b = h^3 W rho2,
       Q0 = Dk - Sk,  Qk = -(eps_E/eps_I) Dk + Sk,  Qk' = -Dk + (eps_I/eps_E) Sk,
   so that, from K11..K22 of Eq. (1.4),
       out1 += sum_k G0(x, s_k) Q0 + Gk(x, s_k) Qk,
       out2 += sum_k dG0/dn_x(x, s_k) Q0 + dGk/dn_x(x, s_k) Qk'.

Parity status: pinned -- theta = 0 reduces to the direct punctured sum of
Eqs. (2.14)-(2.15); the modified charges reproduce every polynomial moment of
degree <= n per axis exactly; the error against the direct sum falls
geometrically with n; the integer separation test agrees with the real
inequality evaluated in 60-digit decimal arithmetic.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

from . import native


@dataclass
class Tree:
    perm: np.ndarray                     # (M,) node at each tree position
    begin: list = field(default_factory=list)
    end: list = field(default_factory=list)
    lo: list = field(default_factory=list)     # integer box [lo, hi) per cluster
    hi: list = field(default_factory=list)
    children: list = field(default_factory=list)

    @property
    def n_clusters(self) -> int:
        return len(self.begin)


def build_tree(ijk: np.ndarray, leaf: int) -> Tree:
    """Step 1: the octree over integer grid indices and the tree positions."""
    ijk = np.asarray(ijk, dtype=np.int64)
    order: list = []
    t = Tree(perm=np.zeros(0, dtype=np.int64))

    def split(idx: np.ndarray) -> int:
        cid = t.n_clusters
        lo = ijk[idx].min(axis=0)
        hi = ijk[idx].max(axis=0) + 1
        t.begin.append(len(order))
        t.end.append(-1)
        t.lo.append(lo)
        t.hi.append(hi)
        t.children.append([])
        if idx.size <= leaf:
            order.extend(np.sort(idx).tolist())
        else:
            mid = lo + (hi - lo) // 2
            code = np.zeros(idx.size, dtype=np.int64)
            for a in range(3):
                if hi[a] - lo[a] >= 2:
                    code += (ijk[idx, a] >= mid[a]).astype(np.int64) << a
            for c in range(8):
                sub = idx[code == c]
                if sub.size:
                    t.children[cid].append(split(sub))
        t.end[cid] = len(order)
        return cid

    split(np.arange(ijk.shape[0], dtype=np.int64))
    t.perm = np.array(order, dtype=np.int64)
    return t


def theta_q(theta: float) -> int:
    return int(math.floor(1024.0 * theta + 0.5))


def widened(lo, hi, g):
    """Doubled centre and half-extent of the box [lo, hi) widened by g (step 3), as Python ints."""
    c2 = [int(lo[a]) + int(hi[a]) - 1 for a in range(3)]
    e2 = [int(hi[a]) - 1 - int(lo[a]) + 2 * g for a in range(3)]
    return c2, sum(e * e for e in e2)


def separated(cB, R2B, cC, R2C, tq: int) -> bool:
    """Step 3: theta |c_B - c_C| > r_B + r_C in exact integer arithmetic."""
    D2 = sum((cB[a] - cC[a]) ** 2 for a in range(3))
    A = tq * tq * D2 - (1 << 20) * (R2B + R2C)
    return A > 0 and A * A > (1 << 42) * R2B * R2C


@dataclass
class Lists:
    BS: int
    near_ptr: np.ndarray
    near_rng: np.ndarray       # (n_near, 2) position ranges
    far_ptr: np.ndarray
    far_cl: np.ndarray         # cluster ids


def interaction_lists(tree: Tree, ijk, excl_ptr, excl_idx, BS: int, theta: float, degree: int,
                      g: int, min_far: int | None = None) -> Lists:
    """Steps 2-4: near ranges and far clusters of every target block.  A well-separated cluster is
    approximated when it has more than min_far nodes (default (n+1)^3, the proxy count)."""
    ijk = np.asarray(ijk, dtype=np.int64)
    M = tree.perm.size
    pos = np.empty(M, dtype=np.int64)
    pos[tree.perm] = np.arange(M)
    tq = theta_q(theta)
    n_proxy = (degree + 1) ** 3 if min_far is None else int(min_far)
    box = [widened(tree.lo[c], tree.hi[c], g) for c in range(tree.n_clusters)]
    nb = (M + BS - 1) // BS
    near_ptr, near_rng, far_ptr, far_cl = [0], [], [0], []
    for I in range(nb):
        p0, p1 = I * BS, min(M, (I + 1) * BS)
        nodes = tree.perm[p0:p1]
        cB, R2B = widened(ijk[nodes].min(axis=0), ijk[nodes].max(axis=0) + 1, g)
        ex = np.unique(pos[np.concatenate([excl_idx[excl_ptr[i]:excl_ptr[i + 1]] for i in nodes])])
        ranges = []

        def holds_excluded(c):
            k = np.searchsorted(ex, tree.begin[c])
            return k < ex.size and ex[k] < tree.end[c]

        def visit(c):
            if separated(cB, R2B, box[c][0], box[c][1], tq) and not holds_excluded(c):
                if tree.end[c] - tree.begin[c] > n_proxy:
                    far_cl.append(c)
                else:
                    ranges.append([tree.begin[c], tree.end[c]])
            elif not tree.children[c]:
                ranges.append([tree.begin[c], tree.end[c]])
            else:
                for ch in tree.children[c]:
                    visit(ch)

        visit(0)
        merged = []
        for b, e in ranges:
            if merged and merged[-1][1] == b:
                merged[-1][1] = e
            else:
                merged.append([b, e])
        near_rng.extend(merged)
        near_ptr.append(len(near_rng))
        far_ptr.append(len(far_cl))
    return Lists(BS, np.array(near_ptr, dtype=np.int64), np.array(near_rng, dtype=np.int64).reshape(-1, 2),
                 np.array(far_ptr, dtype=np.int64), np.array(far_cl, dtype=np.int64))


def chebyshev(degree: int):
    """Step 5: reference nodes x_m = cos(m pi/n), barycentric weights, differentiation matrix."""
    n = degree
    x = np.cos(np.pi * np.arange(n + 1) / n)
    w = (-1.0) ** np.arange(n + 1)
    w[0] *= 0.5
    w[n] *= 0.5
    D = np.zeros((n + 1, n + 1))
    for m in range(n + 1):
        for q in range(n + 1):
            if q != m:
                D[m, q] = (w[q] / w[m]) / (x[m] - x[q])
        D[m, m] = -np.sum(D[m, :])
    return x, w, D


def lagrange(u: np.ndarray, x: np.ndarray, w: np.ndarray) -> np.ndarray:
    """l_m(u) for every u (rows) by the barycentric formula; exact node hits give e_m."""
    u = np.asarray(u, dtype=np.float64)
    diff = u[:, None] - x[None, :]
    hit = diff == 0.0
    with np.errstate(divide="ignore", invalid="ignore"):
        t = w[None, :] / diff
        L = t / np.sum(t, axis=1, keepdims=True)
    rows = np.any(hit, axis=1)
    L[rows] = hit[rows].astype(np.float64)
    return L


def cluster_box(P: np.ndarray, h: float):
    lo = P.min(axis=0)
    hi = P.max(axis=0)
    c = 0.5 * (lo + hi)
    w = np.maximum(0.5 * (hi - lo), h / 1024.0)
    return c, w


def proxy_points(P: np.ndarray, h: float, degree: int) -> np.ndarray:
    """(3, n+1) proxy coordinates s_a[m] of a cluster whose points are P."""
    x, _, _ = chebyshev(degree)
    c, w = cluster_box(P, h)
    return c[:, None] + w[:, None] * x[None, :]


def moments(P, N, a, b, h: float, degree: int):
    """Step 6: Dk = sum_j a_j n_j . grad L_k(P_j) and Sk = sum_j b_j L_k(P_j) of one cluster,
    each (n+1)^3 in the order k = (k3 n1 + k2) n1 + k1."""
    x, w, Dm = chebyshev(degree)
    c, wd = cluster_box(P, h)
    l = [lagrange((P[:, ax] - c[ax]) / wd[ax], x, w) for ax in range(3)]
    dl = [(l[ax] @ Dm) / wd[ax] for ax in range(3)]
    # sum over sources j; array axes (k3, k2, k1)
    S = np.einsum("j,jc,jb,ja->cba", b, l[2], l[1], l[0])
    D = (np.einsum("j,jc,jb,ja->cba", a * N[:, 0], l[2], l[1], dl[0])
         + np.einsum("j,jc,jb,ja->cba", a * N[:, 1], l[2], dl[1], l[0])
         + np.einsum("j,jc,jb,ja->cba", a * N[:, 2], dl[2], l[1], l[0]))
    return D.ravel(), S.ravel()


def modified_charges(P, N, a, b, h: float, degree: int, ratio: float):
    """Step 6: (Q0, Qk, Qk') of one cluster; ratio = eps_E/eps_I."""
    D, S = moments(P, N, a, b, h, degree)
    return np.stack([D - S, -ratio * D + S, -D + S / ratio])


class TreeOperator:
    """The punctured sum of Eqs. (2.14)-(2.15) with the far field of steps 1-6 (one system)."""

    def __init__(self, system, BS: int, degree: int, theta: float, leaf: int, min_far: int | None = None):
        geo = system.geo
        self.sys = system
        self.degree, self.theta, self.leaf, self.BS = degree, theta, leaf, BS
        self.g = int(math.ceil(geo.eps / geo.h))
        self.tree = build_tree(geo.ijk, leaf)
        self.lists = interaction_lists(self.tree, geo.ijk, system.excl_ptr, system.excl_idx, BS, theta,
                                       degree, self.g, min_far)
        self.far_ids, self.far_index = np.unique(self.lists.far_cl, return_inverse=True)
        self.sx = np.zeros((self.far_ids.size, 3, degree + 1))
        for q, c in enumerate(self.far_ids):
            nodes = self.tree.perm[self.tree.begin[c]:self.tree.end[c]]
            self.sx[q] = proxy_points(geo.P[nodes], geo.h, degree)

    def counts(self):
        """(near pair evaluations, far proxy evaluations) of one application."""
        M = self.tree.perm.size
        L = self.lists
        near = far = 0
        for I in range(L.near_ptr.size - 1):
            nt = min(M, (I + 1) * self.BS) - I * self.BS
            r = L.near_rng[L.near_ptr[I]:L.near_ptr[I + 1]]
            near += nt * int(np.sum(r[:, 1] - r[:, 0]))
            far += nt * (L.far_ptr[I + 1] - L.far_ptr[I]) * (self.degree + 1) ** 3
        return near, far

    def charges(self, p: np.ndarray) -> np.ndarray:
        s = self.sys
        geo = s.geo
        M = geo.M
        h3 = geo.h ** 3
        a = h3 * geo.W * p[:M]
        b = h3 * geo.W * p[M:]
        Q = np.zeros((self.far_ids.size, 3, (self.degree + 1) ** 3))
        for q, c in enumerate(self.far_ids):
            nodes = self.tree.perm[self.tree.begin[c]:self.tree.end[c]]
            Q[q] = modified_charges(geo.P[nodes], geo.n[nodes], a[nodes], b[nodes], geo.h, self.degree, s.ratio)
        return Q

    def punctured_sum(self, p: np.ndarray):
        s = self.sys
        M = s.M
        p = np.ascontiguousarray(p, dtype=np.float64)
        rho1 = np.ascontiguousarray(p[:M])
        rho2 = np.ascontiguousarray(p[M:])
        L = self.lists
        o1 = np.zeros(M)
        o2 = np.zeros(M)
        perm = np.ascontiguousarray(self.tree.perm)
        rng = np.ascontiguousarray(L.near_rng.reshape(-1))
        lib = native.lib()
        lib.oracle_tree_near(M, native.dptr(s._P), native.dptr(s._N), native.dptr(s._W), native.dptr(rho1),
                             native.dptr(rho2), s.h, s.kappa, s.ratio, native.iptr(s.excl_ptr),
                             native.iptr(s.excl_idx), native.iptr(perm), self.BS, native.iptr(L.near_ptr),
                             native.iptr(rng), native.dptr(o1), native.dptr(o2))
        if self.far_ids.size:
            Q = np.ascontiguousarray(self.charges(p))
            sx = np.ascontiguousarray(self.sx)
            far_cl = np.ascontiguousarray(self.far_index.astype(np.int64))
            lib.oracle_tree_far(M, native.dptr(s._P), native.dptr(s._N), s.kappa, native.iptr(perm), self.BS,
                                native.iptr(L.far_ptr), native.iptr(far_cl), self.degree + 1, native.dptr(sx),
                                native.dptr(Q), native.dptr(o1), native.dptr(o2))
        return o1, o2

    def matvec(self, p: np.ndarray) -> np.ndarray:
        """(A p) of Eq. (2.30) with the accelerated dense sum."""
        s = self.sys
        M = s.M
        p = np.asarray(p, dtype=np.float64)
        s1, s2 = self.punctured_sum(p)
        c1, c2 = s.correction_apply(p)
        return np.concatenate([s.lam1 * p[:M] + s1 + c1, s.lam2 * p[M:] + s2 + c2])
