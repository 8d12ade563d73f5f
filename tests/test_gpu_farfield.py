"""The treecode (farfield = CTR_FARFIELD_TREECODE) through the C ABI against the oracle.

Tolerances:
  * tree order and work counts: exact (integer work, the oracle's own tree and lists);
  * FP64 operator against the oracle's accelerated operator (same tree, same interpolation):
    1e-12 relative (max norm);
  * float-float operator (near and far field float-float, FP64 moments and charges): 1e-11;
  * FP32 operator: 2e-5, as for the direct sum;
  * against the exact punctured sum (the approximation itself): 1e-6 at the default
    degree 10, theta 0.8 (the oracle measures ~6e-8); 4e-5 for the FP32 operator (its own
    degree 6, theta 0.9: ~7e-6, plus the FP32 rounding);
  * FP32-refined solves to 1e-10 on the treecode (float-float residual operator): converged; the
    polarization energy within 1e-10 of the direct solve at degree 10 and within 1e-11 at degree 12,
    theta 0.6 (measured 6.7e-12 and 1.2e-13: the interpolation error of the treecode's operator).
"""
import math

import numpy as np
import pytest

import synthetic as syn
from oracle import treecode as tc
from oracle.system import OracleSystem

pytestmark = pytest.mark.gpu

SMALL = dict(tree_degree=4, tree_theta=0.7, tree_leaf=32, tree_degree_fp32=4,
             tree_theta_fp32=0.7)   # a large far field at test sizes, the same degree in every arithmetic


def _rel(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


@pytest.fixture(scope="module")
def ctr():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2210_03699_gb300 as ctr
    return ctr


@pytest.fixture(scope="module")
def ellipsoid(ctr, oracle_tables):
    prob = syn.ellipsoid_problem(h=0.1)
    S = OracleSystem.from_problem(prob, tables=oracle_tables)
    G = ctr.CtrIbim.from_problem(prob, options=ctr.Options(tube_halfwidth=prob.tube,
                                                           farfield=ctr.FARFIELD_TREECODE, **SMALL))
    yield prob, S, G
    G.close()


BLOCK = {1: 1024, 2: 256, 0: 256}   # target block of each arithmetic: FP32_REFINE, DF64, FP64
MIN_FAR_DIV = {1: 1, 2: 2, 0: 1}    # approximated clusters exceed (degree+1)^3 / this many nodes


def _oracle_op(S, prec, degree=4, theta=0.7, leaf=32):
    return tc.TreeOperator(S, BS=BLOCK[prec], degree=degree, theta=theta, leaf=leaf,
                           min_far=(degree + 1) ** 3 // MIN_FAR_DIV[prec])


@pytest.mark.parametrize("prec", [0, 1, 2])
def test_tree_structure_matches_oracle(ctr, ellipsoid, prec):
    prob, S, G = ellipsoid
    info = G.farfield_info(prec)
    op = _oracle_op(S, prec)
    near, far = op.counts()
    assert np.array_equal(info["perm"], op.tree.perm)
    assert info["near_pairs"] == near
    assert info["far_evaluations"] == far
    assert info["far_interactions"] == op.lists.far_cl.size
    assert info["far_clusters"] == op.far_ids.size
    assert far > 0.05 * S.M ** 2


@pytest.mark.parametrize("prec,tol", [(0, 1e-12), (2, 1e-11), (1, 2e-5)])
def test_tree_operator_matches_oracle(ctr, ellipsoid, prec, tol):
    prob, S, G = ellipsoid
    p = syn.random_density(S.M, seed=23, smooth_points=S.geo.P)
    ref = _oracle_op(S, prec).matvec(p)
    y = G.matvec(p, prec)
    assert np.all(np.isfinite(y))
    assert _rel(y, ref) < tol


def test_tree_fp64_on_molecule_matches_oracle(ctr, oracle_tables):
    """SES molecule with K-reg rows (wide exclusion sets) at the bad nodes."""
    prob = syn.molecule_problem(n_atoms=60, seed=11, h=0.5)
    S = OracleSystem.from_problem(prob, tables=oracle_tables)
    G = ctr.CtrIbim.from_problem(prob, options=ctr.Options(tube_halfwidth=prob.tube,
                                                           farfield=ctr.FARFIELD_TREECODE, tree_degree=3,
                                                           tree_theta=0.61, tree_leaf=16))
    op = tc.TreeOperator(S, BS=256, degree=3, theta=0.61, leaf=16)
    assert op.lists.far_cl.size > 0
    p = syn.random_density(S.M, seed=29, smooth_points=S.geo.P)
    assert _rel(G.matvec(p, ctr.FP64), op.matvec(p)) < 1e-12
    G.close()


def test_time_operator_phases(ctr, ellipsoid):
    """ctr_ibim_time_operator: the far phase is timed for a treecode handle, zero without one."""
    prob, S, G = ellipsoid
    t = G.time_operator(ctr.FP32_REFINE, reps=2)
    assert t["far_ms"] > 0 and t["pairs_ms"] > 0 and t["pack_ms"] >= 0 and t["finish_ms"] > 0
    D = ctr.CtrIbim.from_problem(prob, options=ctr.Options(tube_halfwidth=prob.tube))
    d = D.time_operator(ctr.DF64, reps=1)
    assert d["far_ms"] < 0.05 and d["pairs_ms"] > 0
    D.close()


def test_tree_default_parameters_close_to_direct(ctr, ellipsoid):
    """Default degree 10, theta 0.8: the accelerated operator within 1e-6 of the direct one; the FP32 operator
    (degree 6, theta 0.9, ~7e-6, below its own rounding) within 4e-5."""
    prob, S, _ = ellipsoid
    G = ctr.CtrIbim.from_problem(prob, options=ctr.Options(tube_halfwidth=prob.tube,
                                                           farfield=ctr.FARFIELD_TREECODE))
    D = ctr.CtrIbim.from_problem(prob, options=ctr.Options(tube_halfwidth=prob.tube))
    p = syn.random_density(S.M, seed=31, smooth_points=S.geo.P)
    yd = D.matvec(p, ctr.FP64)
    assert _rel(G.matvec(p, ctr.FP64), yd) < 1e-6
    assert _rel(G.matvec(p, ctr.DF64), yd) < 1e-6
    assert _rel(G.matvec(p, ctr.FP32_REFINE), yd) < 4e-5
    G.close()
    D.close()


def test_tree_solve_energy_and_batching(ctr, ellipsoid):
    """FP32-refined solves on the treecode (the engine's treecode kernels) to 1e-10: the float-float residual
    operator is consistent to ~1e-13, so refinement reaches the tolerance; the energy differs from the direct
    solve's by the interpolation error only (degree 10: 1e-10; degree 12, theta 0.6: 1e-11); solving in one
    engine with a direct-sum system changes neither result."""
    prob, S, _ = ellipsoid
    opt = dict(tube_halfwidth=prob.tube, precision=ctr.FP32_REFINE, tol=1e-10)
    D = ctr.CtrIbim.from_problem(prob, options=ctr.Options(**opt))
    psi_d, dpsi_d, idd = D.solve()
    assert idd.converged
    Ed = D.energy(psi_d, dpsi_d)[0]
    for extra, tol in ((dict(), 1e-10), (dict(tree_degree=12, tree_theta=0.6), 1e-11)):
        T = ctr.CtrIbim.from_problem(prob, options=ctr.Options(farfield=ctr.FARFIELD_TREECODE, **opt, **extra))
        psi_t, dpsi_t, it = T.solve()
        assert it.converged and it.residual <= 1e-10, it
        # the residual of the treecode's own float-float operator, recomputed
        x = np.concatenate([psi_t, dpsi_t])
        g = T.rhs()
        assert np.linalg.norm(g - T.matvec(x, ctr.DF64)) / np.linalg.norm(g) < 2e-10
        Et = T.energy(psi_t, dpsi_t)[0]
        assert abs(Et / Ed - 1) < tol, (extra, Et, Ed)
        if not extra:
            out = ctr.batch_solve([T, D])
            assert np.array_equal(out[0][0], psi_t) and np.array_equal(out[0][1], dpsi_t)
            assert np.array_equal(out[1][0], psi_d) and np.array_equal(out[1][1], dpsi_d)
        T.close()
    D.close()


def test_tree_full_size_sampled_rows(ctr, oracle_tables):
    """Ellipsoid at h = 0.025 (~714k nodes), the far-field benchmark's workload, default parameters:
    sampled rows against the oracle's exact punctured sum."""
    prob = syn.ellipsoid_problem(h=0.025)
    G = ctr.CtrIbim.from_problem(prob, options=ctr.Options(tube_halfwidth=prob.tube, farfield=ctr.FARFIELD_TREECODE))
    rng = np.random.Generator(np.random.PCG64(37))
    rows = np.unique(np.concatenate([[0, G.M - 1], rng.integers(0, G.M, size=30)]))
    S = OracleSystem.from_problem(prob, tables=oracle_tables, rows=rows)
    assert G.M == S.M > 700_000
    p = syn.random_density(S.M, seed=41, smooth_points=S.geo.P)
    ref = S.matvec(p, rows=rows)
    sel = np.concatenate([rows, G.M + rows])
    ydf = G.matvec(p, ctr.DF64)
    y32 = G.matvec(p, ctr.FP32_REFINE)
    assert np.all(np.isfinite(ydf)) and np.all(np.isfinite(y32))
    assert _rel(ydf[sel], ref) < 1e-6
    assert _rel(y32[sel], ref) < 4e-5
    G.close()


def test_server_mixes_treecode_and_direct_requests(ctr):
    """The server admits treecode requests beside direct-sum ones (the engine runs both kinds of pair
    work and the far-field kernels in one step); each result equals the system solved alone, bitwise."""
    import time
    probs = [syn.ellipsoid_problem(h=0.1), syn.ellipsoid_problem(h=0.2, seed=1),
             syn.molecule_problem(n_atoms=40, seed=5, h=0.5), syn.ellipsoid_problem(h=0.1, seed=2)]
    tree = dict(farfield=ctr.FARFIELD_TREECODE, tol=1e-6, **SMALL)
    opts = [ctr.Options(tube_halfwidth=probs[0].tube, precision=ctr.FP32_REFINE, **tree),
            ctr.Options(tube_halfwidth=probs[1].tube, precision=ctr.FP32_REFINE),
            ctr.Options(tube_halfwidth=probs[2].tube, precision=ctr.FP32_REFINE, farfield=ctr.FARFIELD_TREECODE,
                        tol=1e-6),
            ctr.Options(tube_halfwidth=probs[3].tube, precision=ctr.FP64, **tree)]
    alone = []
    for p, o in zip(probs, opts):
        G = ctr.CtrIbim.from_problem(p, options=o)
        psi, dpsi, info = G.solve()
        alone.append((psi, dpsi, G.energy(psi, dpsi)[0], info))
        G.close()
    with ctr.Server(max_slots=3) as sv:
        tickets = []
        for k, (p, o) in enumerate(zip(probs, opts)):
            tickets.append(sv.submit_problem(p, o))
            time.sleep(0.01 * k)
        results = [sv.wait(t, timeout=600) for t in tickets]
        for t, r, (psi, dpsi, Gp, info) in zip(tickets, results, alone):
            assert r.status == 0 and r.info.converged, r
            bpsi, bdpsi = sv.fetch(t, r.M)
            assert np.array_equal(bpsi, psi) and np.array_equal(bdpsi, dpsi)
            assert r.G_pol == Gp
            sv.release(t)
