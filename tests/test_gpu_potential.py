"""Potential maps: psi_rxn of Eq. (2.31) at many points (ctr_ibim_potential_map) against the oracle.

Tolerances (max norm, relative to the largest |psi_rxn| of the map): FP32 pairs 2e-6 (inputs rounded to
FP32, SFU rsqrt/ex2, FP64 tile sums); float-float and FP64 1e-12.
"""
import json
import os

import numpy as np
import pytest

import synthetic as syn
from oracle import energy as oenergy
from oracle.system import OracleSystem

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctr():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2210_03699_gb300 as ctr
    return ctr


def _points(prob, n, seed, margin):
    """n points of the grid's box whose signed distance (linear interpolation of the grid values is not
    needed: points are kept only where every surrounding grid value is beyond the margin) lies outside
    the band |d| <= margin, inside and outside the surface."""
    g = prob.grid
    rng = np.random.Generator(np.random.PCG64(seed))
    lo = np.asarray(g.origin)
    hi = lo + g.h * (np.asarray(g.n) - 1)
    sd = prob.sdist.reshape(g.n[2], g.n[1], g.n[0])
    out = []
    while sum(len(o) for o in out) < n:
        p = rng.uniform(lo, hi, size=(4 * n, 3))
        c = np.floor((p - lo) / g.h).astype(int)
        c = np.minimum(c, np.asarray(g.n) - 2)
        ok = np.ones(len(p), dtype=bool)
        for dz in (0, 1):
            for dy in (0, 1):
                for dx in (0, 1):
                    ok &= np.abs(sd[c[:, 2] + dz, c[:, 1] + dy, c[:, 0] + dx]) > margin
        out.append(p[ok])
    return np.concatenate(out)[:n]


@pytest.mark.parametrize("which", ["sphere", "ellipsoid"])
def test_potential_map_against_oracle(ctr, oracle_tables, which):
    prob = syn.sphere_problem(h=0.25) if which == "sphere" else syn.ellipsoid_problem(h=0.2)
    S = OracleSystem.from_problem(prob, tables=oracle_tables)
    with ctr.CtrIbim.from_problem(prob, options=ctr.Options(tube_halfwidth=prob.tube, tol=1e-12)) as G:
        psi, dpsi, info = G.solve()
        assert info.converged
        z = _points(prob, 12000, seed=5, margin=2 * prob.tube)
        ref = oenergy.reaction_potential(S, psi, dpsi, z)
        scale = np.max(np.abs(ref))
        tol = {ctr.FP32_REFINE: 2e-6, ctr.DF64: 1e-12, ctr.FP64: 1e-12}
        got = {}
        for prec, t in tol.items():
            got[prec] = G.potential_map(psi, dpsi, z, prec)
            err = np.max(np.abs(got[prec] - ref)) / scale
            assert err < t, (prec, err)
        # the FP64 map is the energy's kernel: ctr_ibim_reaction_potential gives the same numbers
        assert np.array_equal(G.reaction_potential(psi, dpsi, z[:100]), got[ctr.FP64][:100])
        # repeated calls reuse the handle's buffers and give the same bits; fewer points as well
        assert np.array_equal(G.potential_map(psi, dpsi, z, ctr.FP32_REFINE), got[ctr.FP32_REFINE])
        assert np.array_equal(G.potential_map(psi, dpsi, z[:7], ctr.DF64), got[ctr.DF64][:7])


def test_potential_map_device_arrays_and_edges(ctr):
    import torch
    prob = syn.sphere_problem(h=0.25)
    with ctr.CtrIbim.from_problem(prob) as G:
        psi, dpsi, _ = G.solve()
        z = np.array([[0.0, 0.0, 0.0], [0.4, -0.3, 0.2], [3.5, 0.0, 0.0]])
        host = G.potential_map(psi, dpsi, z, ctr.FP32_REFINE)
        dev = G.potential_map(torch.tensor(psi, device="cuda"), torch.tensor(dpsi, device="cuda"),
                              torch.tensor(z, device="cuda"), ctr.FP32_REFINE)
        assert np.array_equal(dev.cpu().numpy(), host)
        assert G.potential_map(psi, dpsi, np.zeros((0, 3)), ctr.FP64).size == 0
        with pytest.raises(ctr.CtrError):
            G.potential_map(psi, dpsi, z, 7)
        # the Kirkwood field inside the sphere: psi_rxn(0) of the closed form (discretization error)
        gold = json.load(open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden",
                                           "kirkwood_sphere_R2.json")))
        assert abs(host[0] / gold["psi_rxn_0"] - 1) < 5e-4
