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
    op_near = op_far = 0
    for I in range(L.near_ptr.size - 1):
        nt = min(S.M, (I + 1) * block) - I * block
        r = L.near_rng[L.near_ptr[I]:L.near_ptr[I + 1]]
        op_near += nt * int(np.sum(r[:, 1] - r[:, 0]))
        op_far += nt * int(L.far_ptr[I + 1] - L.far_ptr[I]) * (degree + 1) ** 3
    assert plan["near_pairs"] == op_near and plan["far_evaluations"] == op_far


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
    # a malformed exclusion CSR is rejected before it indexes anything
    ptr = np.asarray(S.excl_ptr, dtype=np.int64)
    idx = np.asarray(S.excl_idx, dtype=np.int64)
    bad_first = ptr.copy()
    bad_first[0] = 1
    bad_order = ptr.copy()
    bad_order[5] = bad_order[6] + 1
    bad_node = idx.copy()
    bad_node[3] = S.M
    neg_node = idx.copy()
    neg_node[0] = -1
    for p_, i_ in ((bad_first, idx), (bad_order, idx), (ptr, bad_node), (ptr, neg_node)):
        with pytest.raises(ctr.CtrError, match="farfield plan"):
            ctr.farfield_plan(S.geo.ijk, p_, i_, 2, 6, 0.8, 64, 256)
    huge = np.asarray(S.geo.ijk, dtype=np.int64).copy()
    huge[0, 0] = 1 << 30
    with pytest.raises(ctr.CtrError, match="grid indices"):
        ctr.farfield_plan(huge, ptr, idx, 2, 6, 0.8, 64, 256)


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_plan_matches_oracle_on_random_point_sets(seed):
    """Random integer point sets (a dense blob, a flat slab one cell thick, scattered points) with random
    exclusion sets: cells that cannot be split along every axis, uneven octants, empty ones."""
    rng = np.random.Generator(np.random.PCG64(100 + seed))
    blob = rng.integers(0, 24, size=(1500, 3))
    slab = np.column_stack([rng.integers(30, 90, 1200), rng.integers(0, 60, 1200), np.full(1200, 7)])
    far = rng.integers(-200, 200, size=(300, 3))
    pts = np.unique(np.concatenate([blob, slab, far]), axis=0)
    pts = pts[rng.permutation(pts.shape[0])]
    M = pts.shape[0]
    cnt = rng.integers(0, 6, size=M) * (rng.random(M) < 0.02)   # scattered exclusions: most clusters stay free
    ptr = np.concatenate([[0], np.cumsum(cnt)]).astype(np.int64)
    idx = np.concatenate([np.sort(rng.choice(M, size=c, replace=False)) for c in cnt]).astype(np.int64)
    n_far = 0
    for block, degree, theta, leaf, g in [(64, 2, 0.5, 8, 1), (256, 3, 0.8, 16, 2), (32, 2, 0.95, 4, 0)]:
        plan = ctr.farfield_plan(pts, ptr, idx, g, degree, theta, leaf, block, 20)
        tree = tc.build_tree(pts, leaf)
        L = tc.interaction_lists(tree, pts, ptr, idx, block, theta, degree, g, min_far=20)
        assert np.array_equal(plan["perm"], tree.perm)
        assert np.array_equal(plan["near_ptr"], L.near_ptr)
        assert np.array_equal(plan["near_rng"], L.near_rng)
        assert np.array_equal(plan["far_ptr"], L.far_ptr)
        assert np.array_equal(plan["far_begin"], np.array([tree.begin[c] for c in L.far_cl], dtype=np.int64))
        n_far += L.far_cl.size
    assert n_far > 0


def test_separation_ties_are_not_separated():
    """theta |c_B - c_C| = r_B + r_C exactly is not separated (strict inequality), on both sides of it."""
    # radii 3 and 3 in doubled units (R2 = 9), theta = 1/2: separated iff the doubled distance exceeds 12
    assert not tc.separated([0, 0, 0], 9, [12, 0, 0], 9, 512)
    assert tc.separated([0, 0, 0], 9, [13, 0, 0], 9, 512)
    assert not tc.separated([0, 0, 0], 9, [0, 0, 0], 9, 1023)
