"""The treecode's host logic in the library (ctr_farfield_plan) against the oracle's tree -- CPU only.

The tree, the separation test and the interaction lists are integer work: the library's
permutation, near ranges and far clusters must equal the oracle's exactly.
"""
import math

import numpy as np
import pytest

import synthetic as syn
from oracle import treecode as tc
from oracle.system import OracleSystem

ctr = pytest.importorskip("paper_2210_03699_gb300")


@pytest.fixture(scope="module")
def systems(oracle_tables):
    out = {}
    for name, prob in [("ellipsoid_0.2", syn.ellipsoid_problem(h=0.2)),
                       ("molecule_60", syn.molecule_problem(n_atoms=60, seed=11, h=0.5))]:
        out[name] = OracleSystem.from_problem(prob, tables=oracle_tables)
    return out


@pytest.mark.parametrize("name", ["ellipsoid_0.2", "molecule_60"])
@pytest.mark.parametrize("block,degree,theta,leaf,min_far", [(256, 10, 0.8, 128, 0), (1024, 10, 0.8, 128, 0),
                                                             (256, 10, 0.8, 128, 1331 // 16), (256, 4, 0.7, 32, 0),
                                                             (64, 3, 0.61, 16, 0), (256, 4, 0.7, 32, 7)])
def test_plan_matches_oracle(systems, name, block, degree, theta, leaf, min_far):
    S = systems[name]
    g = int(math.ceil(S.geo.eps / S.geo.h))
    plan = ctr.farfield_plan(S.geo.ijk, S.excl_ptr, S.excl_idx, g, degree, theta, leaf, block, min_far)
    tree = tc.build_tree(S.geo.ijk, leaf)
    L = tc.interaction_lists(tree, S.geo.ijk, S.excl_ptr, S.excl_idx, block, theta, degree, g,
                             min_far=min_far if min_far > 0 else None)
    assert np.array_equal(plan["perm"], tree.perm)
    assert np.array_equal(plan["near_ptr"], L.near_ptr)
    assert np.array_equal(plan["near_rng"], L.near_rng)
    assert np.array_equal(plan["far_ptr"], L.far_ptr)
    assert np.array_equal(plan["far_begin"], np.array([tree.begin[c] for c in L.far_cl], dtype=np.int64))
    assert np.array_equal(plan["far_end"], np.array([tree.end[c] for c in L.far_cl], dtype=np.int64))
    if degree <= 4:
        assert L.far_cl.size > 0


def test_plan_theta_zero_and_bad_arguments(systems):
    S = systems["ellipsoid_0.2"]
    plan = ctr.farfield_plan(S.geo.ijk, S.excl_ptr, S.excl_idx, 2, 6, 0.0, 64, 256)
    assert plan["far_begin"].size == 0
    r = plan["near_rng"]
    assert np.all(r[:, 1] > r[:, 0]) and int(np.sum(r[:, 1] - r[:, 0])) == S.M * (plan["near_ptr"].size - 1)
    with pytest.raises(ctr.CtrError):
        ctr.farfield_plan(S.geo.ijk, S.excl_ptr, S.excl_idx, 2, 13, 0.8, 64, 256)
    with pytest.raises(ctr.CtrError):
        ctr.farfield_plan(S.geo.ijk, S.excl_ptr, S.excl_idx, 2, 10, 1.0, 64, 256)
