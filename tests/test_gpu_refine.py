"""FP32 + FP64-accurate refinement against the oracle at the convergence study's second spacing, the
residual-update refinement against full residuals, and a batched molecule against the oracle's rows.

Tolerances: the FP32+refinement solve 1e-6 relative in psi, dpsi_n and G_pol (max norm, against the
oracle's FP64 solve); the residual of a refined solution recomputed with the FP64 operator within
2x the solve tolerance; oracle rows of a batched solution 1e-8 of max|g| (the solve stops at 1e-10).
"""
import json
import os

import numpy as np
import pytest

import synthetic as syn
from oracle.system import OracleSystem

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "ellipsoid_h0.1_oracle_solve.json")


@pytest.fixture(scope="module")
def ctr():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2210_03699_gb300 as ctr
    return ctr


def _true_residual(G, ctr, psi, dpsi):
    x = np.concatenate([psi, dpsi])
    g = G.rhs()
    return float(np.linalg.norm(g - G.matvec(x, ctr.FP64)) / np.linalg.norm(g))


def test_residual_update_matches_full_residuals(ctr):
    prob = syn.ellipsoid_problem(h=0.2)
    out = {}
    for mode in (ctr.RESIDUAL_UPDATE, ctr.RESIDUAL_FULL):
        opts = ctr.Options(tube_halfwidth=prob.tube, precision=ctr.FP32_REFINE, tol=1e-10, residual_mode=mode)
        with ctr.CtrIbim.from_problem(prob, options=opts) as G:
            psi, dpsi, info = G.solve()
            assert info.converged and info.residual <= 1e-10
            # the FP64 operator's residual of the returned solution: the update's error is far below tol
            assert _true_residual(G, ctr, psi, dpsi) < 2e-10
            out[mode] = (psi, dpsi, info, G.energy(psi, dpsi)[0])
    _, _, iu, Gu = out[ctr.RESIDUAL_UPDATE]
    _, _, if_, Gf = out[ctr.RESIDUAL_FULL]
    assert iu.matvecs_fp64 == 1 and if_.matvecs_fp64 == if_.refinements >= 2
    assert iu.refinements == if_.refinements
    for a, b in zip(out[ctr.RESIDUAL_UPDATE][:2], out[ctr.RESIDUAL_FULL][:2]):
        assert np.max(np.abs(a - b)) / np.max(np.abs(b)) < 1e-8
    assert abs(Gu / Gf - 1) < 1e-9


def test_solve_fp32_refine_ellipsoid_h01_against_oracle(ctr):
    """The ellipsoid of the convergence study at h = 0.1 (M = 44 597): FP32 pairs with both residual
    modes and both residual arithmetics, against the oracle's FP64 solve (tests/golden, written by
    make_ellipsoid_h01.py from oracle/ only)."""
    ref = json.load(open(GOLDEN))
    prob = syn.ellipsoid_problem(h=0.1)
    for residual, mode in ((ctr.DF64, ctr.RESIDUAL_UPDATE), (ctr.DF64, ctr.RESIDUAL_FULL),
                           (ctr.FP64, ctr.RESIDUAL_UPDATE)):
        opts = ctr.Options(tube_halfwidth=prob.tube, precision=ctr.FP32_REFINE, tol=1e-10, residual=residual,
                           residual_mode=mode)
        with ctr.CtrIbim.from_problem(prob, options=opts) as G:
            assert G.M == ref["M"]
            psi, dpsi, info = G.solve()
            assert info.converged
            lin = G.nodes()
            pos = np.searchsorted(lin, np.asarray(ref["grid_index"], dtype=np.int64))
            assert np.array_equal(lin[pos], ref["grid_index"])
            assert np.max(np.abs(psi[pos] - ref["psi"])) / ref["psi_max"] < 1e-6
            assert np.max(np.abs(dpsi[pos] - ref["dpsi"])) / ref["dpsi_max"] < 1e-6
            assert abs(np.max(np.abs(psi)) / ref["psi_max"] - 1) < 1e-6
            Gp, prx = G.energy(psi, dpsi)
            assert abs(Gp / ref["G_pol"] - 1) < 1e-6
            assert np.max(np.abs(prx - ref["psi_rxn"])) / np.max(np.abs(ref["psi_rxn"])) < 1e-6


def test_batched_molecule_member_satisfies_oracle_rows(ctr, oracle_tables):
    """A molecule shaped like the batched workload's members (SES of a random-walk molecule, h = 0.35)
    solved inside a mixed batch: its solution, put into the oracle's rows of Eq. (2.30) on sampled
    targets, reproduces the right-hand side; the batch result equals the solve alone bit for bit."""
    mol = syn.molecule_problem(n_atoms=120, seed=11, h=0.35)
    others = [syn.sphere_problem(h=0.25), syn.ellipsoid_problem(h=0.2, seed=2)]
    opts = lambda p: ctr.Options(tube_halfwidth=p.tube, precision=ctr.FP32_REFINE, tol=1e-10)  # noqa: E731
    systems = [ctr.CtrIbim.from_problem(p, options=opts(p)) for p in [others[0], mol, others[1]]]
    out = ctr.batch_solve(systems)
    psi, dpsi, info = out[1]
    assert all(o[2].converged for o in out)
    with ctr.CtrIbim.from_problem(mol, options=opts(mol)) as G:
        psi_a, dpsi_a, _ = G.solve()
        assert np.array_equal(psi, psi_a) and np.array_equal(dpsi, dpsi_a)
        M = G.M
    rng = np.random.Generator(np.random.PCG64(3))
    rows = np.sort(rng.choice(M, size=96, replace=False))
    S = OracleSystem.from_problem(mol, tables=oracle_tables, rows=rows)
    assert S.M == M
    x = np.concatenate([psi, dpsi])
    g = S.rhs()
    Ax = S.matvec(x, rows)
    gr = np.concatenate([g[:M][rows], g[M:][rows]])
    assert np.max(np.abs(Ax - gr)) / np.max(np.abs(g)) < 1e-8
    for s in systems:
        s.close()
