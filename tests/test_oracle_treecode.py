"""Pins of the oracle's far-field acceleration (oracle/treecode.py) -- CPU only.

The accelerated sum is fixed by what does not depend on it: with theta = 0 it
must be the direct punctured sum of Eqs. (2.14)-(2.15); its modified charges
must reproduce every polynomial moment up to the interpolation degree; its
error against the direct sum must fall geometrically with the degree; its
integer separation test must agree with the real inequality in high-precision
decimal arithmetic; its tree and lists must partition the nodes.
"""
import math
from decimal import Decimal, getcontext

import numpy as np
import pytest

import synthetic as syn
from oracle import treecode as tc
from oracle.system import OracleSystem


@pytest.fixture(scope="module")
def ellipsoid_02(oracle_tables):
    prob = syn.ellipsoid_problem(h=0.2)
    return OracleSystem.from_problem(prob, tables=oracle_tables)


@pytest.fixture(scope="module")
def direct_02(ellipsoid_02):
    rng = np.random.Generator(np.random.PCG64(5))
    p = rng.standard_normal(2 * ellipsoid_02.M)
    return p, ellipsoid_02.punctured_sum(p)


def _rel(a, b):
    return max(np.abs(a[0] - b[0]).max() / np.abs(b[0]).max(), np.abs(a[1] - b[1]).max() / np.abs(b[1]).max())


def test_theta_zero_is_the_direct_sum(ellipsoid_02, direct_02):
    p, ref = direct_02
    op = tc.TreeOperator(ellipsoid_02, BS=256, degree=4, theta=0.0, leaf=64)
    assert op.lists.far_cl.size == 0
    assert _rel(op.punctured_sum(p), ref) < 1e-14


def _far_pair_share(op, M):
    t, L = op.tree, op.lists
    fp = 0
    for I in range(L.far_ptr.size - 1):
        nt = min(M, (I + 1) * op.BS) - I * op.BS
        fp += nt * sum(t.end[c] - t.begin[c] for c in L.far_cl[L.far_ptr[I]:L.far_ptr[I + 1]])
    return fp / M ** 2


def test_error_falls_geometrically_with_degree(ellipsoid_02, direct_02):
    """Same tree and lists for every degree (small blocks, leaves and far-cluster threshold, so that
    a third of the pairs lie in the far field at this size); only the interpolation degree changes."""
    p, ref = direct_02
    errs = []
    for n in (2, 4, 6, 8, 10):
        op = tc.TreeOperator(ellipsoid_02, BS=32, degree=n, theta=0.7, leaf=16, min_far=48)
        assert _far_pair_share(op, ellipsoid_02.M) > 0.3
        errs.append(_rel(op.punctured_sum(p), ref))
    for a, b in zip(errs, errs[1:]):
        assert b < a / 4, errs
    assert errs[-1] < 1e-6, errs


def test_planted_sign_error_is_caught(ellipsoid_02, direct_02, monkeypatch):
    """A flipped sign in the dn_x charges (Qk') must break the convergence pin."""
    p, ref = direct_02
    good = tc.modified_charges

    def bad(*args):
        Q = good(*args)
        Q[2] = -Q[2]
        return Q

    monkeypatch.setattr(tc, "modified_charges", bad)
    op = tc.TreeOperator(ellipsoid_02, BS=32, degree=8, theta=0.7, leaf=16, min_far=48)
    assert _rel(op.punctured_sum(p), ref) > 1e-3


@pytest.mark.parametrize("degree", [3, 6, 10])
def test_moments_reproduce_polynomials(degree):
    """sum_k Sk p(s_k) = sum_j b_j p(P_j) and sum_k Dk p(s_k) = sum_j a_j n_j . grad p(P_j)
    for every monomial of degree <= n per axis (the interpolation is exact on them)."""
    rng = np.random.Generator(np.random.PCG64(degree))
    P = rng.uniform([-1.0, 0.5, 2.0], [0.2, 1.1, 2.3], size=(300, 3))
    P[:5] = P[5:10].min(axis=0)          # points on the box corners: exact proxy hits
    N = rng.standard_normal((300, 3))
    N /= np.linalg.norm(N, axis=1, keepdims=True)
    a = rng.standard_normal(300)
    b = rng.standard_normal(300)
    D, S = tc.moments(P, N, a, b, 0.05, degree)
    s = tc.proxy_points(P, 0.05, degree)
    n1 = degree + 1
    k1, k2, k3 = np.meshgrid(np.arange(n1), np.arange(n1), np.arange(n1), indexing="ij")
    order = (k3 * n1 + k2) * n1 + k1
    X, Y, Z = s[0][k1], s[1][k2], s[2][k3]
    c = P.mean(axis=0)
    for al, be, ga in [(0, 0, 0), (1, 0, 0), (0, 2, 1), (degree, degree, degree), (degree, 0, 3 % n1)]:
        def poly(x, y, z):
            return (x - c[0]) ** al * (y - c[1]) ** be * (z - c[2]) ** ga

        def grad(x, y, z):
            gx = al * (x - c[0]) ** max(al - 1, 0) * (y - c[1]) ** be * (z - c[2]) ** ga
            gy = be * (x - c[0]) ** al * (y - c[1]) ** max(be - 1, 0) * (z - c[2]) ** ga
            gz = ga * (x - c[0]) ** al * (y - c[1]) ** be * (z - c[2]) ** max(ga - 1, 0)
            return gx, gy, gz

        pk = np.zeros(n1 ** 3)
        pk[order.ravel()] = poly(X, Y, Z).ravel()
        exact_S = np.sum(b * poly(P[:, 0], P[:, 1], P[:, 2]))
        g = grad(P[:, 0], P[:, 1], P[:, 2])
        exact_D = np.sum(a * (N[:, 0] * g[0] + N[:, 1] * g[1] + N[:, 2] * g[2]))
        scale = np.sum(np.abs(b)) + np.sum(np.abs(a))
        assert abs(np.dot(S, pk) - exact_S) < 1e-11 * scale
        assert abs(np.dot(D, pk) - exact_D) < 1e-10 * scale * max(1, degree)


def test_separation_test_is_exact():
    getcontext().prec = 60
    rng = np.random.Generator(np.random.PCG64(11))
    agree = 0
    for _ in range(4000):
        lo = [rng.integers(0, 400, 3) for _ in range(2)]
        hi = [l + rng.integers(1, 60, 3) for l in lo]
        g = int(rng.integers(1, 4))
        theta = float(rng.choice([0.5, 0.7, 0.8, 0.61]))
        tq = tc.theta_q(theta)
        cB, R2B = tc.widened(lo[0], hi[0], g)
        cC, R2C = tc.widened(lo[1], hi[1], g)
        dist = Decimal(sum((cB[a] - cC[a]) ** 2 for a in range(3))).sqrt()
        lhs = Decimal(tq) / Decimal(1024) * dist - Decimal(R2B).sqrt() - Decimal(R2C).sqrt()
        if lhs == 0:
            continue
        assert tc.separated(cB, R2B, cC, R2C, tq) == (lhs > 0)
        agree += 1
    assert agree > 3900


def test_tree_and_lists_partition_the_nodes(ellipsoid_02):
    S = ellipsoid_02
    op = tc.TreeOperator(S, BS=256, degree=6, theta=0.8, leaf=64)
    t = op.tree
    M = S.M
    assert np.array_equal(np.sort(t.perm), np.arange(M))
    ijk = S.geo.ijk
    for c in range(t.n_clusters):
        nodes = t.perm[t.begin[c]:t.end[c]]
        assert np.array_equal(ijk[nodes].min(axis=0), t.lo[c])
        assert np.array_equal(ijk[nodes].max(axis=0) + 1, t.hi[c])
        if t.children[c]:
            spans = [(t.begin[k], t.end[k]) for k in t.children[c]]
            assert spans[0][0] == t.begin[c] and spans[-1][1] == t.end[c]
            assert all(spans[i][1] == spans[i + 1][0] for i in range(len(spans) - 1))
        else:
            assert nodes.size <= 64 and np.all(np.diff(nodes) > 0)
    pos = np.empty(M, dtype=np.int64)
    pos[t.perm] = np.arange(M)
    L = op.lists
    nfar = 0
    for I in range(L.near_ptr.size - 1):
        cover = np.zeros(M, dtype=np.int64)
        for b, e in L.near_rng[L.near_ptr[I]:L.near_ptr[I + 1]]:
            cover[b:e] += 1
        near_mask = cover.copy()
        for c in L.far_cl[L.far_ptr[I]:L.far_ptr[I + 1]]:
            cover[t.begin[c]:t.end[c]] += 1
            assert t.end[c] - t.begin[c] > 7 ** 3
            nfar += 1
        assert np.all(cover == 1)
        for i in t.perm[I * 256:(I + 1) * 256]:
            ex = pos[S.excl_idx[S.excl_ptr[i]:S.excl_ptr[i + 1]]]
            assert np.all(near_mask[ex] == 1)
    assert nfar > 0
