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
    """A sphere of about 250k nodes alone in a server (FP32 application about 50 ms, float-float about
    0.5 s): whole applications (quantum 0) and applications split into parts of about 10 ms (3 FP32
    parts, some 50 float-float ones) give the same bits as the solve alone; the split run takes
    several engine steps per application."""
    big = syn.sphere_with_nodes(250000)
    opt = ctr.Options(tube_halfwidth=big.tube, precision=ctr.FP32_REFINE)
    ref = _alone(ctr, big, opt)
    steps = {}
    for q in (0.0, 10.0):
        with ctr.Server(max_slots=2, step_quantum_ms=q) as sv:
            _check(sv, sv.submit_problem(big, opt), ref)
            steps[q] = sv.stats()["steps"]
    assert steps[10.0] > 3 * steps[0.0]


def test_mixed_split_and_whole_slots_equal_alone(ctr):
    """Staggered arrivals of split systems (FP32+refinement at 250k nodes, plain FP64 at 44,597 nodes)
    and small systems that run whole (FP32+refinement, float-float K-reg, a molecule): every result
    equals its solve alone."""
    cases = [
        (syn.sphere_with_nodes(250000, q=-1.0), ctr.FP32_REFINE, ctr.METHOD_HYB),
        (syn.sphere_problem(h=0.25), ctr.FP32_REFINE, ctr.METHOD_HYB),
        (syn.ellipsoid_problem(h=0.1, seed=2), ctr.FP64, ctr.METHOD_HYB),
        (syn.sphere_problem(h=0.25, kappa=1.0), ctr.DF64, ctr.METHOD_KREG),
        (syn.molecule_problem(n_atoms=40, seed=5, h=0.5), ctr.FP32_REFINE, ctr.METHOD_HYB),
    ]
    opts = [ctr.Options(tube_halfwidth=p.tube, precision=pr, method=m) for p, pr, m in cases]
    refs = [_alone(ctr, p, o) for (p, _, _), o in zip(cases, opts)]
    with ctr.Server(max_slots=4, step_quantum_ms=5.0) as sv:
        tickets = []
        for k, ((p, _, _), o) in enumerate(zip(cases, opts)):
            tickets.append(sv.submit_problem(p, o))
            time.sleep(0.02 * k)
        for t, ref in zip(tickets, refs):
            _check(sv, t, ref)
        st = sv.stats()
        assert st["running"] == 0 and st["waiting"] == 0 and st["used_bytes"] == 0


def test_cancel_between_parts(ctr):
    """A split plain-FP64 system (44,597 nodes: about 130 ms per application, in parts of about 10 ms)
    cancelled while it runs leaves its slot between two steps; the same problem submitted again, and a
    small one running beside it, still equal their solves alone."""
    big = syn.ellipsoid_problem(h=0.1)
    small = syn.sphere_problem(h=0.25)
    ob = ctr.Options(tube_halfwidth=big.tube, precision=ctr.FP64)
    os_ = ctr.Options(tube_halfwidth=small.tube, precision=ctr.FP32_REFINE)
    ref_big, ref_small = _alone(ctr, big, ob), _alone(ctr, small, os_)
    with ctr.Server(max_slots=2, step_quantum_ms=10.0) as sv:
        t1 = sv.submit_problem(big, ob)
        t0 = time.time()
        while sv.stats()["running"] == 0 and time.time() - t0 < 120:
            time.sleep(0.005)
        time.sleep(0.6)                 # a few of its 11 iterations (about 0.15 s each), not all
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


def test_many_requests_at_once_are_all_admitted(ctr):
    """Many small requests submitted at once to a server with few slots: the setup thread counts the
    systems the worker is admitting as holding slots, so no set-up system finds the engine full
    (before, such a system failed with CTR_ERR_CAPACITY)."""
    probs = [syn.sphere_problem(h=0.25, R=1.5, half_box=2.5), syn.sphere_problem(h=0.25),
             syn.sphere_problem(h=0.25, kappa=0.5)]
    refs = [_alone(ctr, p, ctr.Options(tube_halfwidth=p.tube)) for p in probs]
    with ctr.Server(max_slots=2) as sv:
        tickets = [(k % 3, sv.submit_problem(probs[k % 3])) for k in range(36)]
        for k, t in tickets:
            r = sv.wait(t, 300)
            assert r.status == 0 and r.G_pol == refs[k][2]
            sv.release(t)
        assert sv.stats()["peak_slots"] <= 2


def test_served_result_matches_oracle(ctr, sphere_c1):
    """A small request served beside a split 250k-node system, checked against the oracle's own solve
    (FP64, GMRES to 1e-13) of the same sphere: psi, dpsi_n and G_pol within 1e-6 (the FP32+refinement
    bar; observed about 1e-9)."""
    from oracle import energy as oenergy
    prob, S = sphere_c1
    psi_o, dpsi_o, _ = S.solve(tol=1e-13)
    Go, _ = oenergy.polarization_energy(S, psi_o, dpsi_o)
    big = syn.sphere_with_nodes(250000)
    with ctr.Server(max_slots=2, step_quantum_ms=10.0) as sv:
        tb = sv.submit_problem(big, ctr.Options(tube_halfwidth=big.tube, precision=ctr.FP32_REFINE))
        time.sleep(0.3)
        ts = sv.submit_problem(prob, ctr.Options(tube_halfwidth=prob.tube, precision=ctr.FP32_REFINE))
        r = sv.wait(ts, 300)
        assert r.status == 0
        psi, dpsi = sv.fetch(ts, r.M)
        assert np.max(np.abs(psi - psi_o)) / np.max(np.abs(psi_o)) < 1e-6
        assert np.max(np.abs(dpsi - dpsi_o)) / np.max(np.abs(dpsi_o)) < 1e-6
        assert abs(r.G_pol / Go - 1) < 1e-6
        assert sv.wait(tb, 300).status == 0
