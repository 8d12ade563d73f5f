"""Split operator applications in the server (step_quantum_ms).

A system whose pair sum would take longer than the quantum runs each operator application in parts
(balanced sets of its schedule's items) over consecutive engine steps, while the other slots take
their whole iteration every step.  The node accumulators are exact (integer addition), so every
result equals the system's solve alone bit for bit, whatever the split and whatever else is resident.
"""
import time

import numpy as np
import pytest

import synthetic as syn

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctr():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2210_03699_gb300 as ctr
    return ctr


def _alone(ctr, prob, opt):
    with ctr.CtrIbim.from_problem(prob, options=opt) as G:
        psi, dpsi, info = G.solve()
        Gp, _ = G.energy(psi, dpsi)
    assert info.converged
    return psi, dpsi, Gp, info


def _check(sv, ticket, ref):
    psi, dpsi, Gp, info = ref
    r = sv.wait(ticket, 600)
    assert r.status == 0 and r.info.converged
    bpsi, bdpsi = sv.fetch(ticket, r.M)
    assert np.array_equal(bpsi, psi) and np.array_equal(bdpsi, dpsi)
    assert r.G_pol == Gp
    assert (r.info.iterations, r.info.refinements, r.info.matvecs_fp32, r.info.matvecs_fp64) == \
           (info.iterations, info.refinements, info.matvecs_fp32, info.matvecs_fp64)
    sv.release(ticket)


def test_split_application_equals_alone_and_takes_more_steps(ctr):
    """The ellipsoid at h = 0.1 (44,597 nodes, about 1,300 items per arithmetic) alone in a server:
    whole applications (quantum 0) and applications split into up to 20 parts give the same bits as
    the solve alone; the split run takes several engine steps per application."""
    big = syn.ellipsoid_problem(h=0.1)
    opt = ctr.Options(tube_halfwidth=big.tube, precision=ctr.FP32_REFINE)
    ref = _alone(ctr, big, opt)
    steps = {}
    for q in (0.0, 0.05):
        with ctr.Server(max_slots=2, step_quantum_ms=q) as sv:
            _check(sv, sv.submit_problem(big, opt), ref)
            steps[q] = sv.stats()["steps"]
    assert steps[0.05] > 5 * steps[0.0]


def test_mixed_split_and_whole_slots_equal_alone(ctr):
    """Staggered arrivals of a split FP32+refinement system, a split plain-FP64 system and small
    systems that run whole (FP32+refinement, float-float K-reg): every result equals its solve alone."""
    cases = [
        (syn.ellipsoid_problem(h=0.1), ctr.FP32_REFINE, ctr.METHOD_HYB),
        (syn.sphere_problem(h=0.25), ctr.FP32_REFINE, ctr.METHOD_HYB),
        (syn.ellipsoid_problem(h=0.2, seed=2), ctr.FP64, ctr.METHOD_HYB),
        (syn.sphere_problem(h=0.25, kappa=1.0), ctr.DF64, ctr.METHOD_KREG),
        (syn.molecule_problem(n_atoms=40, seed=5, h=0.5), ctr.FP32_REFINE, ctr.METHOD_HYB),
    ]
    opts = [ctr.Options(tube_halfwidth=p.tube, precision=pr, method=m) for p, pr, m in cases]
    refs = [_alone(ctr, p, o) for (p, _, _), o in zip(cases, opts)]
    with ctr.Server(max_slots=4, step_quantum_ms=0.05) as sv:
        tickets = []
        for k, ((p, _, _), o) in enumerate(zip(cases, opts)):
            tickets.append(sv.submit_problem(p, o))
            time.sleep(0.02 * k)
        for t, ref in zip(tickets, refs):
            _check(sv, t, ref)
        st = sv.stats()
        assert st["running"] == 0 and st["waiting"] == 0 and st["used_bytes"] == 0


def test_cancel_between_parts(ctr):
    """A split plain-FP64 system (44,597 nodes: about 130 ms per application, in up to 127 parts of
    1 ms) cancelled while it runs leaves its slot between two steps; the same problem submitted
    again, and a small one running beside it, still equal their solves alone."""
    big = syn.ellipsoid_problem(h=0.1)
    small = syn.sphere_problem(h=0.25)
    ob = ctr.Options(tube_halfwidth=big.tube, precision=ctr.FP64)
    os_ = ctr.Options(tube_halfwidth=small.tube, precision=ctr.FP32_REFINE)
    ref_big, ref_small = _alone(ctr, big, ob), _alone(ctr, small, os_)
    with ctr.Server(max_slots=2, step_quantum_ms=1.0) as sv:
        t1 = sv.submit_problem(big, ob)
        t0 = time.time()
        while sv.stats()["running"] == 0 and time.time() - t0 < 120:
            time.sleep(0.005)
        time.sleep(0.5)                 # a few of its 11 iterations (about 0.16 s each), not all
        sv.cancel(t1)
        r1 = sv.wait(t1, 120)
        assert r1.status == ctr.ERR_CANCELLED and r1.info.iterations > 0
        sv.release(t1)
        t2 = sv.submit_problem(big, ob)
        t3 = sv.submit_problem(small, os_)
        _check(sv, t2, ref_big)
        _check(sv, t3, ref_small)


def test_step_quantum_is_validated(ctr):
    for bad in (-1.0, float("nan"), float("inf")):
        with pytest.raises(ctr.CtrError):
            ctr.Server(max_slots=1, step_quantum_ms=bad)
