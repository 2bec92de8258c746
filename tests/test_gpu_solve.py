"""Solve parity through the C ABI (mg_solve / mg_batch_solve / serving) against the
oracle's exact discrete solution phi* (oracle iterated to FP64 stagnation):
FP64 path <= 1e-10 relative L2 error over the unknowns, mixed path <= 1e-9."""
import numpy as np
import pytest

from paper_2602_01888_gb300 import inputs as I

pytestmark = pytest.mark.gpu

FP64_TOL = 1e-10
MIXED_TOL = 1e-9


def _ref(oracle, inst):
    P = oracle.prepare(inst)
    phi, it, hist = oracle.pcg_solve(P.A, P.b, P.phi0, rtol=0.0, max_iters=400, stagnate=10)
    return phi


def _err(oracle, inst, phi, ref):
    return oracle.rel_l2(phi, ref, inst.grid.interior_mask())


@pytest.fixture(scope="module")
def ctx(libmg, cuda):
    c = libmg.Context(0)
    yield c
    c.close()


CASES = {
    "config1_129": (lambda: I.config1(129), 1e-10),
    "inclusion_257": (lambda: I.inclusion_instance(257, 0.25, 10.0, 2), 1e-10),
    "annulus_129": (lambda: I.annulus_log(129), 1e-11),
    "circle_65": (lambda: I.circle_poisson(65), 1e-10),
    "affine_33": (lambda: I.affine_quadratic(33), 1e-11),
    "rect_65x33": (lambda: I.Instance("rect", I.Grid(65, 33, 0.0, 0.0, 1.0, 0.5),
                                      I.MapSpec("sine_warp", (0.05,)),
                                      I.random_field((33, 65), 1)), 1e-10),
}


@pytest.mark.parametrize("case", list(CASES))
@pytest.mark.parametrize("precision,outer", [("fp64", "fcg"), ("fp64", "vcycle"), ("mixed", "fcg"),
                                             ("mixed", "vcycle")])
def test_solve_matches_oracle(libmg, oracle, ctx, case, precision, outer):
    make, rtol = CASES[case]
    inst = make()
    ref = _ref(oracle, inst)
    opts = libmg.make_opts(precision, outer, rtol=rtol, max_iters=400)
    prob = libmg.Problem(ctx, inst, opts)
    phi, st = prob.solve()
    tol = FP64_TOL if precision == "fp64" else MIXED_TOL
    err = _err(oracle, inst, phi, ref)
    assert err <= tol, (case, precision, outer, err, st.iters)
    assert st.rel_residual <= rtol
    # boundary ring carries the Dirichlet data
    m = ~inst.grid.interior_mask()
    bc = np.zeros(inst.grid.shape) if inst.bc is None else inst.bc
    assert np.array_equal(phi[m], bc[m])
    prob.close()


def test_config1_accuracy_vs_manufactured_solution(libmg, oracle, ctx):
    """The GPU solution reproduces the oracle's discretization error (Eqs. 25-27)."""
    inst = I.config1(129)
    prob = libmg.Problem(ctx, inst, libmg.make_opts("fp64", "vcycle", rtol=1e-10))
    phi, st = prob.solve()
    ref = _ref(oracle, inst)
    g_norms = oracle.error_norms(inst.exact, phi)
    o_norms = oracle.error_norms(inst.exact, ref)
    assert np.allclose(g_norms, o_norms, rtol=1e-6)
    assert st.iters <= 15


def test_host_and_device_memory_give_identical_results(libmg, ctx, cuda):
    torch = cuda
    inst = I.inclusion_instance(129, 0.25, 10.0, 3)
    opts = libmg.make_opts("mixed", "fcg", rtol=1e-10)
    prob_h = libmg.Problem(ctx, inst, opts)
    prob_d = libmg.Problem(ctx, inst, opts, device_inputs=True)
    phi_h, _ = prob_h.solve()
    rho = torch.from_numpy(np.ascontiguousarray(inst.rho_phys)).cuda()
    phi_d = torch.zeros(inst.grid.shape, dtype=torch.float64, device="cuda")
    prob_d.solve(rho=rho, phi=phi_d)
    torch.cuda.synchronize()
    assert np.array_equal(phi_h, phi_d.cpu().numpy())
    # a second solve on the same problem is bitwise reproducible
    phi_h2, _ = prob_h.solve()
    assert np.array_equal(phi_h, phi_h2)


def test_page_locked_host_arrays_are_used_in_place(libmg, ctx, cuda):
    """Page-locked host arrays (read and written by the kernels over the host link), pageable
    ones (staged) and device arrays give the same solution, cold and warm started."""
    torch = cuda
    inst = I.annulus_log(129)
    opts = libmg.make_opts("mixed", "fcg", rtol=1e-10, smoother="xline", nu1=1, nu2=1)
    prob = libmg.Problem(ctx, inst, opts)
    rho, bc = np.ascontiguousarray(inst.rho_phys), np.ascontiguousarray(inst.bc)
    pin = lambda a: torch.from_numpy(np.array(a)).pin_memory()
    rho_p, bc_p = pin(rho), pin(bc)
    phi_p = torch.zeros(inst.grid.shape, dtype=torch.float64).pin_memory()
    phi_h = np.zeros(inst.grid.shape)
    prob.solve(rho=rho, bc=bc, phi=phi_h)
    libmg.mg_solve(prob.h, rho_p.numpy(), bc_p.numpy(), phi_p.numpy(), opts)
    phi_d = torch.zeros(inst.grid.shape, dtype=torch.float64, device="cuda")
    libmg.mg_solve(prob.h, torch.from_numpy(rho).cuda(), torch.from_numpy(bc).cuda(), phi_d, opts)
    torch.cuda.synchronize()
    assert np.array_equal(phi_p.numpy(), phi_h)
    assert np.array_equal(phi_d.cpu().numpy(), phi_h)
    warm = libmg.make_opts("mixed", "fcg", rtol=1e-10, smoother="xline", nu1=1, nu2=1, warm_start=True)
    st = libmg.mg_solve(prob.h, rho_p.numpy(), bc_p.numpy(), phi_p.numpy(), warm)
    assert st.iters <= 1  # started from the converged solution, read in place
    ring = ~inst.grid.interior_mask()
    assert np.array_equal(phi_p.numpy()[ring], bc[ring])
    prob.close()


def test_warm_start_from_solution(libmg, ctx):
    inst = I.config1(65)
    opts = libmg.make_opts("fp64", "fcg", rtol=1e-9)
    prob = libmg.Problem(ctx, inst, opts)
    phi, st = prob.solve()
    opts2 = libmg.make_opts("fp64", "fcg", rtol=1e-9, warm_start=True)
    phi2 = phi.copy()
    _, st2 = prob.solve(phi=phi2, opts=opts2)
    assert st2.iters <= 1


@pytest.mark.parametrize("shape", [(3, 3), (5, 5), (9, 9), (33, 17), (17, 65)])
def test_small_and_rectangular_grids(libmg, oracle, ctx, shape):
    nx, ny = shape
    inst = I.Instance("small", I.Grid(nx, ny, 0.0, 0.0, 1.0, (ny - 1) / (nx - 1)),
                      I.MapSpec("sine_warp", (0.05,)), I.random_field((ny, nx), nx * ny))
    ref = _ref(oracle, inst)
    prob = libmg.Problem(ctx, inst, libmg.make_opts("fp64", "fcg", rtol=1e-12))
    phi, st = prob.solve()
    assert _err(oracle, inst, phi, ref) <= FP64_TOL


def test_error_reporting(libmg, ctx):
    folded = I.affine_quadratic(9, (1.0, 0.0, 0.0, -1.0))
    with pytest.raises(libmg.MGError) as e:
        libmg.Problem(ctx, folded)
    assert e.value.status == libmg.MG_ERR_MAP_FOLDED
    bad = I.Instance("bad", I.Grid(1000, 1000), I.MapSpec("identity"), np.zeros((1000, 1000)))
    with pytest.raises(libmg.MGError) as e:
        libmg.Problem(ctx, bad)
    assert e.value.status == libmg.MG_ERR_SIZE
    inst = I.config1(65)
    prob = libmg.Problem(ctx, inst, libmg.make_opts("fp64", "vcycle", rtol=1e-14, max_iters=1))
    phi = np.zeros(inst.grid.shape)
    st = libmg.mg_solve(prob.h, np.ascontiguousarray(inst.rho_phys), None, phi, prob.opts,
                        allow_not_converged=True)
    assert st.iters == 1 and st.rel_residual > 1e-14
    with pytest.raises(libmg.MGError) as e:
        libmg.mg_solve(prob.h, np.ascontiguousarray(inst.rho_phys), None, phi, prob.opts)
    assert e.value.status == libmg.MG_ERR_NOT_CONVERGED


def test_batch_equals_individual_solves_bitwise(libmg, ctx):
    specs = [(65, 0.2, 5.0, 1), (129, 0.3, 20.0, 2), (257, 0.15, 40.0, 3), (65, 0.25, 1.0, 4),
             (129, 0.12, 2.0, 5)]
    insts = [I.inclusion_instance(*s) for s in specs]
    opts = libmg.make_opts("mixed", "fcg", rtol=1e-10)
    probs = [libmg.Problem(ctx, inst, opts) for inst in insts]
    alone = [p.solve()[0] for p in probs]
    rhos = [np.ascontiguousarray(i.rho_phys) for i in insts]
    phis = [np.zeros(i.grid.shape) for i in insts]
    libmg.mg_batch_solve(ctx.h, [p.h for p in probs], rhos, None, phis, opts)
    for a, b in zip(alone, phis):
        assert np.array_equal(a, b)


def test_server_results_equal_mg_solve_bitwise(libmg, ctx):
    specs = [(65, 0.2, 5.0, 11), (129, 0.3, 20.0, 12), (257, 0.15, 40.0, 13), (129, 0.25, 3.0, 14)]
    insts = [I.inclusion_instance(*s) for s in specs]
    opts = libmg.make_opts("mixed", "fcg", rtol=1e-10)
    alone = []
    for inst in insts:
        p = libmg.Problem(ctx, inst, opts)
        alone.append(p.solve()[0])
        p.close()
    srv = libmg.mg_server_start(ctx.h, max_inflight=3)
    tickets = []
    for inst in insts:
        st, t = libmg.mg_serve_submit(srv, inst.grid, inst.map, np.ascontiguousarray(inst.rho_phys),
                                      None, np.ascontiguousarray(inst.eps_phys), opts)
        assert st == 0
        tickets.append(t)
    for inst, t, a in zip(insts, tickets, alone):
        out = np.zeros(inst.grid.shape)
        st, stats = libmg.mg_serve_poll(srv, t, 60000, out)
        assert st == 0
        assert np.array_equal(out, a)
    rep = libmg.mg_server_stop(srv)
    assert rep.completed == len(insts) and rep.failed == 0
    assert rep.p99_ms >= rep.p50_ms > 0


def test_full_size_inclusion_1025(libmg, oracle, ctx):
    """The 1025^2 inclusion workload at the settings the benchmark uses (FP64 and mixed,
    flexible CG, residual tolerance 3e-8): error against the oracle's phi* within a tenth
    of the 1e-9 target."""
    inst = I.config2(1025)
    ref = _ref(oracle, inst)
    for prec, tol in (("fp64", 1e-10), ("mixed", 1e-10)):
        prob = libmg.Problem(ctx, inst, libmg.make_opts(prec, "fcg", rtol=3e-8))
        phi, st = prob.solve()
        err = _err(oracle, inst, phi, ref)
        assert err <= tol, (prec, err, st.iters)
        prob.close()


def test_server_reuses_resident_hierarchies_with_identical_results(libmg, ctx):
    """Twelve requests over three grid sides through two slots: later requests run on
    hierarchies left resident by earlier ones (coefficients rebuilt in place) and still
    return exactly what a fresh mg_setup_transform + mg_solve returns."""
    sides = [65, 129, 97, 65, 129, 97, 129, 65, 97, 65, 129, 97]
    specs = [(n, 0.12 + 0.02 * k, 2.0 + 3.0 * k, 100 + k) for k, n in enumerate(sides)]
    insts = [I.inclusion_instance(*s) for s in specs]
    opts = libmg.make_opts("mixed", "fcg", rtol=1e-10)
    alone = []
    for inst in insts:
        p = libmg.Problem(ctx, inst, opts)
        alone.append(p.solve()[0])
        p.close()
    srv = libmg.mg_server_start(ctx.h, max_inflight=2)
    tickets = []
    for inst in insts:
        st, t = libmg.mg_serve_submit(srv, inst.grid, inst.map, np.ascontiguousarray(inst.rho_phys),
                                      None, np.ascontiguousarray(inst.eps_phys), opts)
        assert st == 0
        tickets.append(t)
    for inst, t, a in zip(insts, tickets, alone):
        out = np.zeros(inst.grid.shape)
        st, _ = libmg.mg_serve_poll(srv, t, 60000, out)
        assert st == 0
        assert np.array_equal(out, a), inst.name
    rep = libmg.mg_server_stop(srv)
    assert rep.completed == len(insts) and rep.failed == 0
    assert rep.reused >= len(insts) - 2 * 3


def test_server_host_staging_budget_gives_busy_then_recovers(libmg, ctx):
    """Submitted arrays live in page-locked staging until their ticket is polled; a full
    staging budget makes mg_serve_submit return MG_ERR_BUSY, and polling frees room."""
    insts = [I.inclusion_instance(65, 0.2, 3.0 + k, 300 + k) for k in range(3)]
    one = 6 * 65 * 65 * 8  # rho, phi, eps, xp, yp and rounding slack
    opts = libmg.make_opts("mixed", "fcg", rtol=1e-10)
    srv = libmg.mg_server_start(ctx.h, max_inflight=2, host_budget=2 * one + 4096)
    sub = lambda x: libmg.mg_serve_submit(srv, x.grid, x.map, np.ascontiguousarray(x.rho_phys), None,
                                          np.ascontiguousarray(x.eps_phys), opts)
    st0, t0 = sub(insts[0])
    st1, t1 = sub(insts[1])
    st2, _ = sub(insts[2])
    assert (st0, st1, st2) == (0, 0, libmg.MG_ERR_BUSY)
    out = np.zeros(insts[0].grid.shape)
    assert libmg.mg_serve_poll(srv, t0, 60000, out)[0] == 0
    st2, t2 = sub(insts[2])
    assert st2 == 0
    for t in (t1, t2):
        assert libmg.mg_serve_poll(srv, t, 60000, None)[0] == 0
    rep = libmg.mg_server_stop(srv)
    assert rep.completed == 3 and rep.failed == 0


def test_cycle_time_of_a_resident_problem(libmg, cuda):
    """mg_cycle_time runs the problem's own cycle: positive, below the whole solve's time per
    iteration (which adds the outer FP64 vector work), refused for the SOR iteration, and it
    leaves the next solve's result unchanged (bitwise)."""
    ctx = libmg.Context(0)
    inst = I.config2(257)
    for prec in ("fp64", "mixed"):
        opts = libmg.make_opts(prec, "fcg", rtol=1e-10)
        pr = libmg.Problem(ctx, inst, opts)
        phi0, st = pr.solve()
        ms = libmg.mg_cycle_time(pr.h, opts, reps=10)
        assert 0.0 < ms < st.solve_ms / max(st.iters, 1) * 1.5, (prec, ms, st.solve_ms, st.iters)
        phi1, _ = pr.solve()
        assert np.array_equal(phi0, phi1)
        if prec == "fp64":
            with pytest.raises(libmg.MGError):
                libmg.mg_cycle_time(pr.h, libmg.make_opts("fp64", "sor", nu1=4, omega_j=1.5))
        pr.close()
    ctx.close()


@pytest.mark.parametrize("case", ["config1_129", "inclusion_257", "annulus_129"])
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_jacobi_smoothed_solve_matches_oracle(libmg, oracle, ctx, case, precision):
    """Weighted Jacobi (omega_J = 4/5, the smoother option of Sec. 3) inside flexible CG: the
    solution reaches the oracle's phi* like the Gauss-Seidel solves do."""
    make, rtol = CASES[case]
    inst = make()
    ref = _ref(oracle, inst)
    opts = libmg.make_opts(precision, "fcg", rtol=rtol, max_iters=400, smoother="jacobi", omega_j=0.8)
    prob = libmg.Problem(ctx, inst, opts)
    phi, st = prob.solve()
    err = _err(oracle, inst, phi, ref)
    assert err <= (FP64_TOL if precision == "fp64" else MIXED_TOL), (case, precision, err, st.iters)
    assert st.rel_residual <= rtol
    # the smoother is in use: the residual history differs from the Gauss-Seidel solve's
    gs = libmg.Problem(ctx, inst, libmg.make_opts(precision, "fcg", rtol=rtol, max_iters=400))
    _, st_gs = gs.solve()
    assert st.hist[1] != st_gs.hist[1], (st.hist[1], st_gs.hist[1])
    gs.close()
    prob.close()


def test_served_results_match_oracle(libmg, oracle, ctx):
    """Requests of three grid sides and different geometries submitted while earlier ones are
    still on the device (three slots, seven requests), polled in a different order than
    submitted: every served result is within the mixed path's 1e-9 of the oracle's phi*."""
    specs = [(257, 0.3, 40.0, 21), (65, 0.2, 5.0, 22), (129, 0.15, 12.0, 23), (257, 0.25, 2.0, 24),
             (129, 0.3, 49.0, 25), (65, 0.1, 30.0, 26), (129, 0.2, 1.0, 27)]
    insts = [I.inclusion_instance(*s) for s in specs]
    opts = libmg.make_opts("mixed", "fcg", rtol=1e-9, max_iters=400)
    srv = libmg.mg_server_start(ctx.h, max_inflight=3)
    tickets = []
    for inst in insts:
        st, t = libmg.mg_serve_submit(srv, inst.grid, inst.map, np.ascontiguousarray(inst.rho_phys),
                                      None, np.ascontiguousarray(inst.eps_phys), opts)
        assert st == 0
        tickets.append(t)
    order = [3, 0, 6, 1, 5, 2, 4]
    for k in order:
        inst = insts[k]
        out = np.zeros(inst.grid.shape)
        st, stats = libmg.mg_serve_poll(srv, tickets[k], 120000, out)
        assert st == 0, (k, st)
        err = _err(oracle, inst, out, _ref(oracle, inst))
        assert err <= MIXED_TOL, (inst.name, err, stats.iters)
    rep = libmg.mg_server_stop(srv)
    assert rep.completed == len(insts) and rep.failed == 0


def test_server_request_whose_completion_query_fails_is_reported_and_stop_returns(libmg, ctx):
    """A request whose completion query reports an error (made on the host by the server's
    test hook, nothing faults on the device) finishes with MG_ERR_CUDA instead of staying in
    flight; its slot is freed, later requests are served normally and mg_server_stop
    returns with the failure counted."""
    insts = [I.inclusion_instance(65, 0.2, 3.0 + k, 400 + k) for k in range(3)]
    opts = libmg.make_opts("mixed", "fcg", rtol=1e-10)
    srv = libmg.mg_server_start(ctx.h, max_inflight=1)
    sub = lambda x: libmg.mg_serve_submit(srv, x.grid, x.map, np.ascontiguousarray(x.rho_phys), None,
                                          np.ascontiguousarray(x.eps_phys), opts)
    try:
        libmg.lib().mgk_server_fail_event_queries(1)
        st0, t0 = sub(insts[0])
        assert st0 == 0
        st, _ = libmg.mg_serve_poll(srv, t0, 60000, np.zeros(insts[0].grid.shape))
        assert st == libmg.MG_ERR_CUDA, st
    finally:
        libmg.lib().mgk_server_fail_event_queries(0)
    outs = []
    for x in insts[1:]:
        st, t = sub(x)
        assert st == 0
        out = np.zeros(x.grid.shape)
        assert libmg.mg_serve_poll(srv, t, 60000, out)[0] == 0
        outs.append(out)
    rep = libmg.mg_server_stop(srv)
    assert rep.failed == 1 and rep.completed == 2
    for x, out in zip(insts[1:], outs):
        p = libmg.Problem(ctx, x, opts)
        want, _ = p.solve()
        p.close()
        assert np.array_equal(out, want)
