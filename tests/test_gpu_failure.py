"""Failure paths of the GPU library, made on the host or by a bounded wait told to give up at once.

No test here faults, traps or hangs the GPU: bad inputs are rejected by the library's own checks, the
device-wait test sets the pair kernels' poll limit to 0 (every bounded wait returns "expired" without
polling; the blocks let their bulk copies land and return), and cancellation acts between engine steps.
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


def test_iteration_limit_reports_not_converged(ctr):
    prob = syn.sphere_problem(h=0.25)
    with ctr.CtrIbim.from_problem(prob, options=ctr.Options(tube_halfwidth=prob.tube, max_iter=3)) as G:
        psi, dpsi, info = G.solve()
        assert info.status == 1 and not info.converged          # CTR_NOT_CONVERGED, result still written
        assert info.iterations == 3 and 1e-10 < info.residual < 1.0
        assert np.all(np.isfinite(psi)) and np.max(np.abs(psi)) > 0
    opts = ctr.Options(tube_halfwidth=prob.tube, precision=ctr.FP32_REFINE, max_refine=1, tol=1e-12)
    with ctr.CtrIbim.from_problem(prob, options=opts) as G:
        _, _, info = G.solve()
        assert info.status == 1 and info.refinements == 1


def test_non_finite_inputs_are_rejected(ctr):
    prob = syn.sphere_problem(h=0.25)
    g = prob.grid
    for where in (0, int(np.argmin(np.abs(prob.sdist)))):    # a grid corner, and a node on the surface
        sd = prob.sdist.copy()
        sd[where] = np.nan
        with pytest.raises(ctr.CtrError) as e:
            ctr.CtrIbim(g.n, g.origin, g.h, sd, 1.0, 80.0, 0.1257, prob.charge_xyz, prob.charge_q)
        assert e.value.status == -6
    for xyz, q in (([[np.nan, 0.0, 0.0]], [1.0]), ([[0.0, 0.0, 0.0]], [np.inf])):
        with pytest.raises(ctr.CtrError) as e:
            ctr.CtrIbim(g.n, g.origin, g.h, prob.sdist, 1.0, 80.0, 0.1257, np.array(xyz), np.array(q))
        assert e.value.status == -6
    # served: the bad request fails alone, the others match their solve alone bit for bit
    with ctr.CtrIbim.from_problem(prob) as G:
        psi, dpsi, _ = G.solve()
        G_alone, _ = G.energy(psi, dpsi)
    bad = prob.sdist.copy()
    bad[int(np.argmin(np.abs(prob.sdist)))] = np.nan
    with ctr.Server(max_slots=2) as sv:
        t1 = sv.submit_problem(prob)
        tb = sv.submit(g.n, g.origin, g.h, bad, prob.eps_in, prob.eps_out, prob.kappa, prob.charge_xyz,
                       prob.charge_q, ctr.Options(tube_halfwidth=prob.tube))
        tq = sv.submit(g.n, g.origin, g.h, prob.sdist, prob.eps_in, prob.eps_out, prob.kappa, prob.charge_xyz,
                       np.array([np.nan]), ctr.Options(tube_halfwidth=prob.tube))
        t2 = sv.submit_problem(prob)
        r1, rb, rq, r2 = (sv.wait(t, 120) for t in (t1, tb, tq, t2))
        assert rb.status == -6 and rq.status == -6
        assert r1.status == 0 and r2.status == 0 and r1.G_pol == G_alone == r2.G_pol


def test_expired_device_wait_returns_status(ctr):
    """Poll limit 0: every pair block's first source-tile wait gives up; the call reports
    CTR_ERR_DEVICE_WAIT and the handle and the device stay usable."""
    prob = syn.sphere_problem(h=0.25)
    with ctr.CtrIbim.from_problem(prob) as G:
        x = syn.random_density(G.M, seed=4)
        ref = {p: G.matvec(x, p) for p in (ctr.FP32_REFINE, ctr.DF64, ctr.FP64)}
        try:
            ctr.set_wait_limit(0)
            for p in ref:
                with pytest.raises(ctr.CtrError) as e:
                    G.matvec(x, p)
                assert e.value.status == ctr.ERR_DEVICE_WAIT
            with pytest.raises(ctr.CtrError) as e:
                G.solve()
            assert e.value.status == ctr.ERR_DEVICE_WAIT
        finally:
            ctr.set_wait_limit(-1)
        for p, y in ref.items():
            assert np.array_equal(G.matvec(x, p), y)
        _, _, info = G.solve()
        assert info.converged


def test_server_cancel_waiting_and_running(ctr):
    """One slot: a long FP64 request runs, two wait.  Cancelling a waiting one and the running one
    frees the slot; the remaining requests match their solves alone bit for bit."""
    long_prob = syn.ellipsoid_problem(h=0.1)
    small = [syn.sphere_problem(h=0.25), syn.sphere_problem(h=0.25, R=1.5, half_box=2.5)]
    alone = []
    for p in small:
        with ctr.CtrIbim.from_problem(p, options=ctr.Options(tube_halfwidth=p.tube)) as G:
            psi, dpsi, _ = G.solve()
            alone.append(G.energy(psi, dpsi)[0])
    with ctr.Server(max_slots=1) as sv:
        t_long = sv.submit_problem(long_prob, ctr.Options(tube_halfwidth=long_prob.tube, precision=ctr.FP64))
        t_a = sv.submit_problem(small[0])
        t_b = sv.submit_problem(small[1])
        sv.cancel(t_b)                                  # still queued behind the slot
        rb = sv.wait(t_b, 60)
        assert rb.status == ctr.ERR_CANCELLED
        t0 = time.time()
        while sv.stats()["running"] == 0 and time.time() - t0 < 60:
            time.sleep(0.01)
        assert sv.stats()["running"] == 1
        time.sleep(0.2)                                 # a few engine steps of the long solve
        sv.cancel(t_long)
        rl = sv.wait(t_long, 120)
        assert rl.status == ctr.ERR_CANCELLED and rl.info.iterations > 0 and not rl.info.converged
        t_c = sv.submit_problem(small[1])               # arrives after the cancellations
        ra, rc = sv.wait(t_a, 120), sv.wait(t_c, 120)
        assert ra.status == 0 and rc.status == 0
        assert ra.G_pol == alone[0] and rc.G_pol == alone[1]
        with pytest.raises(ctr.CtrError):
            sv.cancel(t_a)                              # already finished
        st = sv.stats()
        assert st["running"] == 0 and st["waiting"] == 0 and st["used_bytes"] == 0
        for t in (t_long, t_a, t_b, t_c):
            sv.release(t)


def test_server_admits_over_budget_requests_alone(ctr):
    """A budget smaller than any request: each is admitted alone when nothing else is resident."""
    probs = [syn.sphere_problem(h=0.25), syn.ellipsoid_problem(h=0.2), syn.sphere_problem(h=0.25, kappa=0.5)]
    alone = []
    for p in probs:
        with ctr.CtrIbim.from_problem(p, options=ctr.Options(tube_halfwidth=p.tube)) as G:
            psi, dpsi, _ = G.solve()
            alone.append(G.energy(psi, dpsi)[0])
    with ctr.Server(max_slots=4, hbm_budget_bytes=1) as sv:
        ts = [sv.submit_problem(p) for p in probs]
        rs = [sv.wait(t, 120) for t in ts]
        assert all(r.status == 0 for r in rs)
        assert [r.G_pol for r in rs] == alone
        assert sv.stats()["peak_slots"] == 1


def test_server_submissions_to_an_idle_server(ctr):
    """Each request arrives when the previous one has finished and both server threads are idle: every
    submission must reach the setup thread (a wakeup taken by the idle worker would leave it queued)."""
    prob = syn.sphere_problem(h=0.25, R=1.5, half_box=2.5)
    with ctr.Server(max_slots=2) as sv:
        G = None
        for k in range(12):
            t = sv.submit_problem(prob)
            r = sv.wait(t, 60)
            assert r.status == 0
            G = r.G_pol if G is None else G
            assert r.G_pol == G
            sv.release(t)
            time.sleep(0.05)                            # let both threads go idle
