"""GPU path (through the C ABI) against the FP64 CPU oracle, element by element.

Tolerances (arithmetic behind them in the design notes):
  * integer / decision outputs (tube nodes, correction CSR, node ids): exact;
  * P and n: exact (both sides evaluate the same unfused IEEE sequence);
  * W, correction weights, rhs: 1e-12 relative to the largest magnitude;
  * FP64 and float-float (DF64) operators: 1e-12 relative (max norm);
  * FP64 solve: 1e-10 relative;
  * FP32-pair operator: 2e-5 relative (FP32 pair terms, FP64 accumulation per tile);
  * FP32 + FP64-refinement solve: 1e-6 relative in psi, dpsi and G_pol.
"""
import math

import numpy as np
import pytest

import synthetic as syn
from oracle import energy as oenergy
from oracle.system import OracleSystem

pytestmark = pytest.mark.gpu


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
def sphere(ctr, oracle_tables):
    prob = syn.sphere_problem(h=0.25)
    S = OracleSystem.from_problem(prob, tables=oracle_tables)
    G = ctr.CtrIbim.from_problem(prob)
    yield prob, S, G
    G.close()


@pytest.fixture(scope="module")
def ellipsoid(ctr, oracle_tables):
    prob = syn.ellipsoid_problem(h=0.2)
    S = OracleSystem.from_problem(prob, tables=oracle_tables)
    G = ctr.CtrIbim.from_problem(prob)
    yield prob, S, G
    G.close()


def test_weight_tables_match_oracle(ctr, oracle_tables):
    T = ctr.weight_tables()
    assert T.shape == oracle_tables.shape == (2, 9, 39, 39)
    assert np.max(np.abs(T - oracle_tables)) < 1e-11


@pytest.fixture(scope="module")
def molecule(ctr, oracle_tables):
    """60-atom synthetic molecule, SES at h = 0.5: HYB-IBIM with many bad nodes."""
    prob = syn.molecule_problem(n_atoms=60, seed=0, h=0.5)
    S = OracleSystem.from_problem(prob, tables=oracle_tables)
    G = ctr.CtrIbim.from_problem(prob)
    yield prob, S, G
    G.close()


@pytest.fixture(scope="module")
def quadsphere(ctr, oracle_tables):
    """Exact finite-difference geometry (quadratic level set): the HYB threshold cuts through the tube."""
    prob = syn.quadratic_sphere_problem(h=0.1, tube=0.65)
    S = OracleSystem.from_problem(prob, tables=oracle_tables)
    G = ctr.CtrIbim.from_problem(prob)
    yield prob, S, G
    G.close()


@pytest.fixture(scope="module")
def flatcyl_kreg(ctr, oracle_tables):
    """Flat faces (exact planes near their centres), K-reg rows everywhere."""
    prob = syn.flat_cylinder_problem(h=0.25)
    S = OracleSystem.from_problem(prob, tables=oracle_tables, method="kreg")
    G = ctr.CtrIbim.from_problem(prob, options=ctr.Options(tube_halfwidth=prob.tube, method=ctr.METHOD_KREG))
    yield prob, S, G
    G.close()


@pytest.fixture(scope="module")
def sphere_kreg(ctr, oracle_tables):
    """The K-reg method (Sec. 2.3) everywhere on the sphere."""
    prob = syn.sphere_problem(h=0.25)
    S = OracleSystem.from_problem(prob, tables=oracle_tables, method="kreg")
    G = ctr.CtrIbim.from_problem(prob, options=ctr.Options(tube_halfwidth=prob.tube, method=ctr.METHOD_KREG))
    yield prob, S, G
    G.close()


@pytest.mark.parametrize("which", ["sphere", "ellipsoid", "molecule", "sphere_kreg", "quadsphere", "flatcyl_kreg"])
def test_setup_parity(which, request):
    prob, S, G = request.getfixturevalue(which)
    assert G.M == S.M
    assert np.array_equal(G.nodes(), S.geo.lin)
    P, n, W = G.geometry()
    assert np.array_equal(P, S.geo.P)
    assert np.array_equal(n, S.geo.n)
    assert _rel(W, S.geo.W) < 1e-12
    assert np.array_equal(G.bad_nodes(), S.geo.bad)
    ptr, node, w = G.corrections()
    assert np.array_equal(ptr, S.corr.ptr)
    assert np.array_equal(node, S.corr.node)
    assert _rel(w[0], S.omega11) < 1e-10
    assert _rel(w[1], S.omega21) < 1e-10
    assert _rel(w[2], S.omega22) < 1e-10
    assert _rel(w[3], S.omega12) < 1e-14
    assert _rel(G.rhs(), S.rhs()) < 1e-12
    assert abs(G.area() / S.area() - 1) < 1e-12


@pytest.mark.parametrize("which", ["sphere", "ellipsoid", "molecule", "sphere_kreg", "quadsphere", "flatcyl_kreg"])
def test_operator_parity(which, request, ctr):
    prob, S, G = request.getfixturevalue(which)
    p = syn.random_density(S.M, seed=11, smooth_points=S.geo.P)
    ref = S.matvec(p)
    y64 = G.matvec(p, ctr.FP64)
    assert _rel(y64, ref) < 1e-12
    ydf = G.matvec(p, ctr.DF64)
    assert _rel(ydf, ref) < 1e-12
    y32 = G.matvec(p, ctr.FP32_REFINE)
    assert _rel(y32, ref) < 2e-5
    # deterministic: fixed-order reductions
    assert np.array_equal(G.matvec(p, ctr.FP64), y64)
    assert np.array_equal(G.matvec(p, ctr.FP32_REFINE), y32)


def test_operator_parity_all_rows_many_blocks(ctr, oracle_tables):
    """Ellipsoid at h = 0.1 (~45k nodes): ~44 FP32 and ~175 float-float target blocks, so the
    schedules hold near (one-sided, masked) items, split symmetric items and a ragged last block;
    every row against the oracle."""
    prob = syn.ellipsoid_problem(h=0.1)
    S = OracleSystem.from_problem(prob, tables=oracle_tables)
    G = ctr.CtrIbim.from_problem(prob)
    assert G.M == S.M > 40_000 and G.M % 1024 != 0
    for prec in (ctr.FP32_REFINE, ctr.DF64, ctr.FP64):   # every ordered pair covered exactly once
        sc = G.pair_schedule(prec)
        assert sc["one_sided_pairs"] + 2 * sc["symmetric_pairs"] == G.M * G.M
        assert sc["symmetric_pairs"] > 0.3 * G.M * G.M
    p = syn.random_density(S.M, seed=17, smooth_points=S.geo.P)
    ref = S.matvec(p)
    y64 = G.matvec(p, ctr.FP64)
    ydf = G.matvec(p, ctr.DF64)
    y32 = G.matvec(p, ctr.FP32_REFINE)
    assert _rel(y64, ref) < 1e-12
    assert _rel(ydf, ref) < 1e-12
    assert _rel(y32, ref) < 2e-5
    # row by row too (rows below 1e-3 of the largest are measured against that floor): FP64 and
    # float-float (about 2^-44 per operation) keep every row to the oracle's digits less the
    # cancellation of that row's terms; FP32 keeps about 4 digits
    for name, y, tol in (("fp64", y64, 1e-11), ("df64", ydf, 1e-10), ("fp32", y32, 1e-3)):
        err = np.abs(y - ref) / np.maximum(np.abs(ref), 1e-3 * np.max(np.abs(ref)))
        assert np.max(err) < tol, (name, float(np.max(err)))
    G.close()


def test_operator_device_buffers(sphere, ctr):
    import torch
    prob, S, G = sphere
    p = syn.random_density(S.M, seed=3)
    x = torch.tensor(p, dtype=torch.float64, device="cuda")
    y = G.matvec(x, ctr.FP64)
    assert isinstance(y, torch.Tensor) and y.is_cuda
    assert np.array_equal(y.cpu().numpy(), G.matvec(p, ctr.FP64))


def test_solve_fp64_parity(sphere, ctr):
    prob, S, G = sphere
    psi_o, dpsi_o, info_o = S.solve(tol=1e-13)
    G.options.tol = 1e-13
    G2 = ctr.CtrIbim.from_problem(prob, options=ctr.Options(tube_halfwidth=prob.tube, tol=1e-13))
    psi, dpsi, info = G2.solve()
    assert info.converged and info.residual <= 1e-13
    assert 5 <= info.iterations <= 60
    assert _rel(psi, psi_o) < 1e-10
    assert _rel(dpsi, dpsi_o) < 1e-10
    Gp, prx = G2.energy(psi, dpsi)
    Go, prx_o = oenergy.polarization_energy(S, psi_o, dpsi_o)
    assert abs(Gp / Go - 1) < 1e-10
    # Kirkwood closed form (discretization error at h = 0.25)
    assert abs(Gp / -0.019695646775266615 - 1) < 5e-4
    G2.close()


def test_solve_fp32_refine_parity(ellipsoid, ctr):
    prob, S, G = ellipsoid
    psi_o, dpsi_o, info_o = S.solve(tol=1e-13)
    Go, _ = oenergy.polarization_energy(S, psi_o, dpsi_o)
    for residual in (ctr.DF64, ctr.FP64):
        G32 = ctr.CtrIbim.from_problem(prob, options=ctr.Options(tube_halfwidth=prob.tube, residual=residual,
                                                                   precision=ctr.FP32_REFINE, tol=1e-11))
        psi, dpsi, info = G32.solve()
        assert info.converged and info.refinements >= 1 and info.matvecs_fp32 > info.matvecs_fp64
        assert _rel(psi, psi_o) < 1e-6
        assert _rel(dpsi, dpsi_o) < 1e-6
        Gp, _ = G32.energy(psi, dpsi)
        assert abs(Gp / Go - 1) < 1e-6
        G32.close()
    # FP64 GPU path on the same system
    G64 = ctr.CtrIbim.from_problem(prob, options=ctr.Options(tube_halfwidth=prob.tube, tol=1e-13))
    psi64, dpsi64, _ = G64.solve()
    assert _rel(psi64, psi_o) < 1e-10
    G64.close()
    # float-float operator as a plain solve mode
    Gdf = ctr.CtrIbim.from_problem(prob, options=ctr.Options(tube_halfwidth=prob.tube, tol=1e-13,
                                                               precision=ctr.DF64))
    psid, dpsid, info = Gdf.solve()
    assert info.converged
    assert _rel(psid, psi_o) < 1e-10 and _rel(dpsid, dpsi_o) < 1e-10
    Gdf.close()


def test_solve_molecule_hyb_parity(molecule, ctr):
    prob, S, G = molecule
    assert 0 < S.geo.bad.sum() < S.M
    psi_o, dpsi_o, info_o = S.solve(tol=1e-12, max_iter=400)
    assert info_o["converged"]
    Go, _ = oenergy.polarization_energy(S, psi_o, dpsi_o)
    G32 = ctr.CtrIbim.from_problem(prob, options=ctr.Options(tube_halfwidth=prob.tube, precision=ctr.FP32_REFINE,
                                                               tol=1e-11))
    psi, dpsi, info = G32.solve()
    assert info.converged
    assert _rel(psi, psi_o) < 1e-6 and _rel(dpsi, dpsi_o) < 1e-6
    Gp, _ = G32.energy(psi, dpsi)
    assert abs(Gp / Go - 1) < 1e-6
    G32.close()


def test_solve_kreg_parity(sphere_kreg, ctr):
    prob, S, G = sphere_kreg
    psi_o, dpsi_o, _ = S.solve(tol=1e-13)
    Gk = ctr.CtrIbim.from_problem(prob, options=ctr.Options(tube_halfwidth=prob.tube, method=ctr.METHOD_KREG,
                                                              tol=1e-13))
    psi, dpsi, info = Gk.solve()
    assert info.converged
    assert _rel(psi, psi_o) < 1e-10 and _rel(dpsi, dpsi_o) < 1e-10
    Gp, _ = Gk.energy(psi, dpsi)
    # K-reg is first order: a few percent from Kirkwood at h = 0.25 (CTR2: 1e-6)
    assert 1e-3 < abs(Gp / -0.019695646775266615 - 1) < 0.1
    Gk.close()


def test_solve_on_device_buffers(sphere, ctr):
    import torch
    prob, S, G = sphere
    psi_h, dpsi_h, _ = G.solve()
    psi_d, dpsi_d, info = G.solve(device=True)
    assert isinstance(psi_d, torch.Tensor)
    assert np.array_equal(psi_d.cpu().numpy(), psi_h)
    Gh, _ = G.energy(psi_h, dpsi_h)
    Gd, _ = G.energy(psi_d, dpsi_d)
    assert Gh == Gd


def test_reaction_potential_points(sphere):
    prob, S, G = sphere
    psi, dpsi, _ = G.solve()
    z = np.array([[0.0, 0.0, 0.0], [0.3, -0.2, 0.1], [0.0, 0.5, -0.4]])
    got = G.reaction_potential(psi, dpsi, z)
    ref = oenergy.reaction_potential(S, psi, dpsi, z)
    assert _rel(got, ref) < 1e-12


# ---------------------------------------------------------------- edge cases
def test_small_system_and_laplace(ctr, oracle_tables):
    # fewer nodes than one thread block; kappa = 0 (pure Laplace kernels)
    prob = syn.sphere_problem(h=0.25, R=0.75, half_box=1.5, kappa=0.0)
    S = OracleSystem.from_problem(prob, tables=oracle_tables)
    G = ctr.CtrIbim.from_problem(prob)
    assert G.M == S.M and G.M < 512
    p = syn.random_density(S.M, seed=5)
    assert _rel(G.matvec(p, ctr.FP64), S.matvec(p)) < 1e-12
    assert _rel(G.matvec(p, ctr.DF64), S.matvec(p)) < 1e-12
    assert _rel(G.matvec(p, ctr.FP32_REFINE), S.matvec(p)) < 2e-5
    G.close()


def test_no_charges_gives_zero_solution(ctr):
    prob = syn.sphere_problem(h=0.25)
    G = ctr.CtrIbim(prob.grid.n, prob.grid.origin, prob.grid.h, prob.sdist, 1.0, 80.0, 0.1257,
                    np.zeros((0, 3)), np.zeros(0))
    assert np.all(G.rhs() == 0)
    psi, dpsi, info = G.solve()
    assert info.converged and np.all(psi == 0) and np.all(dpsi == 0)
    Gp, prx = G.energy(psi, dpsi)
    assert Gp == 0.0 and prx.size == 0
    G.close()


def test_error_statuses(ctr):
    prob = syn.sphere_problem(h=0.25)
    with pytest.raises(ctr.CtrError) as e:       # empty tube
        ctr.CtrIbim(prob.grid.n, prob.grid.origin, prob.grid.h, np.full(prob.grid.size, 10.0), 1.0, 80.0, 0.1,
                    np.zeros((1, 3)), np.ones(1))
    assert e.value.status == -2
    g = syn.box_grid((-2.25,) * 3, (2.25,) * 3, 0.25)   # sphere reaches the grid margin
    with pytest.raises(ctr.CtrError) as e:
        ctr.CtrIbim(g.n, g.origin, g.h, syn.sphere_sdist(g, 2.0), 1.0, 80.0, 0.1, np.zeros((1, 3)), np.ones(1))
    assert e.value.status == -3


# ---------------------------------------------------------------- full size, sampled rows
def test_full_size_sampled_rows(ctr, oracle_tables):
    """Ellipsoid at h = 0.05 (~178k nodes), the benchmark's launch configuration; rows sampled."""
    prob = syn.ellipsoid_problem(h=0.05)
    G = ctr.CtrIbim.from_problem(prob, options=ctr.Options(tube_halfwidth=prob.tube))
    rng = np.random.Generator(np.random.PCG64(7))
    rows = np.unique(np.concatenate([[0, G.M - 1], rng.integers(0, G.M, size=46)]))
    S = OracleSystem.from_problem(prob, tables=oracle_tables, rows=rows)
    assert G.M == S.M > 150_000
    p = syn.random_density(S.M, seed=13, smooth_points=S.geo.P)
    ref = S.matvec(p, rows=rows)
    y64 = G.matvec(p, ctr.FP64)
    ydf = G.matvec(p, ctr.DF64)
    y32 = G.matvec(p, ctr.FP32_REFINE)
    sel = np.concatenate([rows, G.M + rows])
    assert _rel(y64[sel], ref) < 1e-12
    assert _rel(ydf[sel], ref) < 1e-12
    assert _rel(y32[sel], ref) < 2e-5
    assert np.all(np.isfinite(y32)) and np.all(np.isfinite(y64))
    G.close()


def test_full_size_molecule_sampled_rows_and_energy(ctr, oracle_tables):
    """The 500-atom SES molecule at h = 0.5 (the single-molecule workload, ~90k nodes; HYB with K-reg rows
    at the bad nodes): every ordered pair covered once by each schedule, sampled rows against the oracle
    in the three arithmetics, and the FP32-refined polarization energy within 1e-6 of the plain FP64
    solve on the GPU."""
    prob = syn.molecule_problem(n_atoms=500, seed=0, h=0.5)
    G = ctr.CtrIbim.from_problem(prob, options=ctr.Options(tube_halfwidth=prob.tube, precision=ctr.FP32_REFINE))
    assert G.M > 80_000 and G.bad_nodes().sum() > 0
    for prec in (ctr.FP32_REFINE, ctr.DF64, ctr.FP64):
        sc = G.pair_schedule(prec)
        assert sc["one_sided_pairs"] + 2 * sc["symmetric_pairs"] == G.M * G.M
    rng = np.random.Generator(np.random.PCG64(11))
    bad = np.nonzero(G.bad_nodes())[0]
    rows = np.unique(np.concatenate([[0, G.M - 1], rng.integers(0, G.M, size=38), rng.choice(bad, size=8)]))
    S = OracleSystem.from_problem(prob, tables=oracle_tables, rows=rows)
    assert S.M == G.M
    p = syn.random_density(S.M, seed=19, smooth_points=S.geo.P)
    ref = S.matvec(p, rows=rows)
    sel = np.concatenate([rows, G.M + rows])
    assert _rel(G.matvec(p, ctr.FP64)[sel], ref) < 1e-12
    assert _rel(G.matvec(p, ctr.DF64)[sel], ref) < 1e-12
    assert _rel(G.matvec(p, ctr.FP32_REFINE)[sel], ref) < 2e-5
    psi, dpsi, info = G.solve()
    assert info.converged and info.residual < 1e-10
    E32 = G.energy(psi, dpsi)[0]
    G.close()
    with ctr.CtrIbim.from_problem(prob, options=ctr.Options(tube_halfwidth=prob.tube, precision=ctr.FP64)) as G64:
        psi64, dpsi64, info64 = G64.solve()
        assert info64.converged
        E64 = G64.energy(psi64, dpsi64)[0]
    assert abs(E32 / E64 - 1) < 1e-6


# ---------------------------------------------------------------- batched engine (many systems, one engine)
def test_batch_matches_alone_bitwise(ctr, oracle_tables):
    """Each system's result is the same alone and in a mixed batch (sizes, methods, precisions)."""
    probs = [
        (syn.sphere_problem(h=0.25), ctr.Options(tube_halfwidth=0.5, precision=ctr.FP32_REFINE)),
        (syn.ellipsoid_problem(h=0.2), ctr.Options(tube_halfwidth=0.4, precision=ctr.FP32_REFINE)),
        (syn.molecule_problem(n_atoms=40, seed=3, h=0.5), ctr.Options(tube_halfwidth=1.0,
                                                                      precision=ctr.FP32_REFINE)),
        (syn.sphere_problem(h=0.25, R=1.5, half_box=2.5), ctr.Options(tube_halfwidth=0.5, precision=ctr.FP64)),
        (syn.sphere_problem(h=0.25, kappa=1.0), ctr.Options(tube_halfwidth=0.5, precision=ctr.DF64,
                                                            method=ctr.METHOD_KREG)),
    ]
    alone = []
    for prob, opt in probs:
        G = ctr.CtrIbim.from_problem(prob, options=opt)
        psi, dpsi, info = G.solve()
        assert info.converged
        alone.append((psi, dpsi, info))
        G.close()
    systems = [ctr.CtrIbim.from_problem(prob, options=opt) for prob, opt in probs]
    batch = ctr.batch_solve(systems)
    for (psi, dpsi, info), (bpsi, bdpsi, binfo) in zip(alone, batch):
        assert binfo.converged
        assert np.array_equal(psi, bpsi) and np.array_equal(dpsi, bdpsi)
        assert (info.iterations, info.refinements, info.matvecs_fp32, info.matvecs_fp64) == \
               (binfo.iterations, binfo.refinements, binfo.matvecs_fp32, binfo.matvecs_fp64)
    # a second batch in another order gives the same results again
    batch2 = ctr.batch_solve(list(reversed(systems)))
    for (psi, dpsi, _), (bpsi, bdpsi, _) in zip(alone, reversed(batch2)):
        assert np.array_equal(psi, bpsi) and np.array_equal(dpsi, bdpsi)
    for G in systems:
        G.close()


# ---------------------------------------------------------------- serving (continuous batching)
def test_server_results_equal_alone_under_staggered_arrivals(ctr):
    """Requests submitted while others run are admitted as slots free up; each result is the
    same as the system solved alone (bitwise), and the memory budget is respected."""
    import time
    probs = [syn.sphere_problem(h=0.25), syn.ellipsoid_problem(h=0.2),
             syn.molecule_problem(n_atoms=40, seed=5, h=0.5), syn.sphere_problem(h=0.25, R=1.5, half_box=2.5),
             syn.ellipsoid_problem(h=0.2, seed=1), syn.sphere_problem(h=0.25, kappa=0.5)]
    opts = [ctr.Options(tube_halfwidth=p.tube, precision=ctr.FP32_REFINE) for p in probs]
    alone = []
    for p, o in zip(probs, opts):
        G = ctr.CtrIbim.from_problem(p, options=o)
        psi, dpsi, info = G.solve()
        Gp, _ = G.energy(psi, dpsi)
        alone.append((psi, dpsi, Gp, info))
        G.close()
    with ctr.Server(max_slots=3, hbm_budget_bytes=int(1.5e9)) as sv:
        tickets = []
        for k, (p, o) in enumerate(zip(probs, opts)):
            tickets.append(sv.submit_problem(p, o))
            time.sleep(0.01 * k)                      # staggered arrivals
        results = [sv.wait(t, timeout=300) for t in tickets]
        st = sv.stats()
        assert st["peak_slots"] <= 3 and st["peak_used_bytes"] <= st["budget_bytes"]
        assert st["running"] == 0 and st["waiting"] == 0
        for t, r, (psi, dpsi, Gp, info) in zip(tickets, results, alone):
            assert r.status == 0 and r.info.converged
            assert r.t_submit <= r.t_admit <= r.t_done
            bpsi, bdpsi = sv.fetch(t, r.M)
            assert np.array_equal(bpsi, psi) and np.array_equal(bdpsi, dpsi)
            assert r.G_pol == Gp
            assert r.info.iterations == info.iterations
            sv.release(t)


def test_server_isolates_failed_requests(ctr):
    """A request whose setup fails (empty tube) reports its status; the others complete."""
    good = syn.sphere_problem(h=0.25)
    with ctr.Server(max_slots=2) as sv:
        t1 = sv.submit_problem(good)
        t_bad = sv.submit(good.grid.n, good.grid.origin, good.grid.h, np.full(good.grid.size, 9.0), 1.0, 80.0, 0.1,
                          np.zeros((1, 3)), np.ones(1))
        t2 = sv.submit_problem(good)
        r1, rb, r2 = sv.wait(t1, 120), sv.wait(t_bad, 120), sv.wait(t2, 120)
        assert r1.status == 0 and r2.status == 0 and rb.status == -2
        assert r1.G_pol == r2.G_pol


# ---------------------------------------------------------------- convergence studies (Sec. 3.3.2)
def test_torus_area_and_potential_convergence(ctr, oracle_tables):
    """Rotated torus (R1 = 1, R2 = 1/2, eps = 2h): the GPU area equals the oracle's, its error against
    4 pi^2 R1 R2 falls at least fourfold per halving of h, and psi_rxn(0) (Eq. 2.31) converges: the
    successive differences shrink (the paper's 'diff' column falls 3.8x and 5.2x)."""
    from oracle.geometry import tube_area, tube_geometry
    areas, rx = [], []
    for h in (0.1, 0.05, 0.025):
        p = syn.torus_problem(h)
        with ctr.CtrIbim.from_problem(p, options=ctr.Options(tube_halfwidth=p.tube, precision=ctr.FP32_REFINE)) as G:
            areas.append(G.area())
            psi, dpsi, info = G.solve()
            assert info.converged
            rx.append(G.reaction_potential(psi, dpsi, np.zeros((1, 3)))[0])
            if h == 0.1:
                g = p.grid
                geo = tube_geometry(g.n, g.origin, g.h, p.sdist, p.tube)
                assert abs(areas[0] / tube_area(geo) - 1) < 1e-12
    err = [abs(a / syn.torus_area() - 1) for a in areas]
    assert err[0] / err[1] > 4.0 and err[1] / err[2] > 4.0 and err[2] < 1e-5
    d1, d2 = abs(rx[1] - rx[0]), abs(rx[2] - rx[1])
    assert d1 / d2 > 2.5


def test_sphere_r10_ctr2_beats_kreg(ctr):
    """Sphere r = 10, one unit charge at the centre, eps = 2h (Sec. 3.3.2, Fig. 2): psi_rxn(0) against the
    closed form.  CTR2 converges (order about 1 at eps = 2h) and its error is at least ten times smaller
    than K-reg's at every h, as the paper reports; K-reg converges at first order."""
    R, q = 10.0, 1.0
    exact = q / (4 * math.pi * R) * (1 / (syn.EPS_OUT * (1 + syn.KAPPA * R)) - 1 / syn.EPS_IN)
    e_ctr, e_kreg = [], []
    for h in (1.0, 0.5, 0.25):
        p = syn.sphere_problem(h=h, R=R, half_box=R + 5 * h, q=q)
        for meth, errs in ((ctr.METHOD_HYB, e_ctr), (ctr.METHOD_KREG, e_kreg)):
            with ctr.CtrIbim.from_problem(p, options=ctr.Options(tube_halfwidth=p.tube, precision=ctr.FP32_REFINE,
                                                                 method=meth)) as G:
                psi, dpsi, info = G.solve()
                assert info.converged
                errs.append(abs(G.reaction_potential(psi, dpsi, np.zeros((1, 3)))[0] / exact - 1))
    assert all(a * 10 < b for a, b in zip(e_ctr, e_kreg))
    assert e_ctr[0] > e_ctr[1] > e_ctr[2] and e_ctr[2] < 2e-5
    assert all(1.6 < e_kreg[k] / e_kreg[k + 1] < 2.5 for k in range(2))
