"""Per-system FP32 pair-kernel variants (targets per block, source tile): each system's shape is fixed at
setup, so its results are the same alone and in a batch that mixes shapes; every shape matches the oracle
within the FP32 operator tolerance (2e-5, max norm)."""
import numpy as np
import pytest

import synthetic as syn
from oracle.system import OracleSystem

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctr():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2210_03699_gb300 as ctr
    return ctr


SHAPES = [(1024, 256), (512, 256), (1024, 128), (512, 128)]


def test_every_fp32_shape_matches_oracle(ctr, oracle_tables):
    prob = syn.ellipsoid_problem(h=0.2)
    S = OracleSystem.from_problem(prob, tables=oracle_tables)
    x = syn.random_density(S.M, seed=9)
    ref = S.matvec(x)
    for bs, tile in SHAPES:
        opts = ctr.Options(tube_halfwidth=prob.tube, fp32_block=bs, fp32_tile=tile)
        with ctr.CtrIbim.from_problem(prob, options=opts) as G:
            t = G.pair_tuning(ctr.FP32_REFINE)
            assert (t["block_targets"], t["tile"]) == (bs, tile)
            y = G.matvec(x, ctr.FP32_REFINE)
            assert np.max(np.abs(y - ref)) / np.max(np.abs(ref)) < 2e-5
    with pytest.raises(ctr.CtrError):
        ctr.CtrIbim.from_problem(prob, options=ctr.Options(tube_halfwidth=prob.tube, fp32_block=768))


def test_mixed_shapes_batch_bitwise(ctr):
    probs = [syn.sphere_problem(h=0.25), syn.ellipsoid_problem(h=0.2), syn.molecule_problem(n_atoms=40, seed=3, h=0.5),
             syn.ellipsoid_problem(h=0.2, seed=4)]
    opts = [ctr.Options(tube_halfwidth=p.tube, precision=ctr.FP32_REFINE, fp32_block=bs, fp32_tile=tile)
            for p, (bs, tile) in zip(probs, SHAPES)]
    alone = []
    for p, o in zip(probs, opts):
        with ctr.CtrIbim.from_problem(p, options=o) as G:
            alone.append(G.solve())
    systems = [ctr.CtrIbim.from_problem(p, options=o) for p, o in zip(probs, opts)]
    batch = ctr.batch_solve(systems)
    for (psi, dpsi, info), (bpsi, bdpsi, binfo) in zip(alone, batch):
        assert binfo.converged
        assert np.array_equal(psi, bpsi) and np.array_equal(dpsi, bdpsi)
        assert info.iterations == binfo.iterations
    for s in systems:
        s.close()


def test_tuned_variant_is_cached_per_size_bucket(ctr):
    """Without a requested shape the setup times the variants on the system and keeps the choice for
    its size bucket: a second system of the bucket gets the same shape; the choice is reported."""
    prob = syn.ellipsoid_problem(h=0.2)
    with ctr.CtrIbim.from_problem(prob) as A, ctr.CtrIbim.from_problem(syn.ellipsoid_problem(h=0.2, seed=5)) as B:
        ta, tb = A.pair_tuning(ctr.FP32_REFINE), B.pair_tuning(ctr.FP32_REFINE)
        assert ta == tb
        assert (ta["block_targets"], ta["tile"]) in SHAPES and ta["chunk"] in (4, 8) and ta["unroll"] in (1, 2)
        R, V, U = ctr.tuning_info()
        assert R * 256 == ta["block_targets"] and (V, U) == (ta["chunk"], ta["unroll"])
        assert A.pair_tuning(ctr.DF64) == {"block_targets": 256, "tile": 128, "chunk": 8, "unroll": 1}
