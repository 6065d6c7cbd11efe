"""GPU parity of the CUDA path (through the C ABI) against the oracle.

Criteria: primal solution within 1e-6 relative (max-norm, scaled by
max(1, |y|_inf)); the GPU's primal-dual point has scaled KKT error
E_0 <= 1e-8 when evaluated by the oracle's own evaluator; equal
interior-point iteration counts on the same seeds.

Iteration counts are compared with the GPU eliminating in the oracle's own
order (stage order; the oracle's banded Cholesky), so both sides see the
same pivot sequence up to rounding, and against the oracle's rounding spread:
the oracle is re-run with its inputs perturbed by 1e-15..1e-13 relative.
When that leaves its count unchanged the GPU count must be equal; when
rounding alone moves the oracle's count, the GPU count must lie within the
oracle's own range.  With nested dissection (the performance default) the
pivots differ, so the pivot test of the inertia correction can decide
differently; there the counts must be equal unless the first iteration at
which the traces differ is an inertia-correction decision.  The heated plate's
primal solution is only determined to ~1e-3 at tol 1e-8 (its reduced Hessian
is nearly flat), so its primal parity is checked at tol 1e-12.
"""
import numpy as np
import pytest

import paper_2606_04725_gb300.inputs as I

pytestmark = pytest.mark.gpu

TOL_Y = 1e-6
TOL_KKT = 1e-8


@pytest.fixture(scope="module")
def P():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2606_04725_gb300 as P
    P.build()
    return P


def _oracle_problem(O, kind, T, x0, sp, uprev=I.U_REF, **kw):
    if kind == "distill12":
        return O.distillation(12, 5, T, x0, np.full(T, sp) if np.isscalar(sp) else sp, uprev)
    if kind == "distill34":
        return O.distillation(34, 17, T, x0, np.full(T, sp) if np.isscalar(sp) else sp, uprev)
    if kind.startswith("plate"):
        g, S = kw["g"], kw["S"]
        return O.plate(g, S, T, x0, sp)
    if kind == "toy":
        return O.toy(T, x0, sp, dt=kw["dt"])
    raise ValueError(kind)


NATURAL = 1  # elimination in stage order, as the oracle's banded Cholesky


def _gpu_solver(P, kind, horizons, **kw):
    kw.setdefault("opts", P.options(ordering=NATURAL))
    if kind == "distill12":
        return P.Solver(P.MODEL_DISTILLATION, horizons, N=12, Nf=5, **kw)
    if kind == "distill34":
        return P.Solver(P.MODEL_DISTILLATION, horizons, N=34, Nf=17, **kw)
    if kind == "toy":
        dt = kw.pop("dt")
        return P.Solver(P.MODEL_TOY, horizons, dt=dt, **kw)
    raise ValueError(kind)


def _state_from_gpu(O, solver, inst, n, m):
    y, du = solver.get_solution(inst, duals=True)
    st = O.State(n, m)
    st.y[:] = y
    for k in ("zL", "zU", "s_p", "s_m", "w_p", "w_m", "b_p", "b_m"):
        getattr(st, k)[:] = du[k]
    return st


def _oracle_spread(O, prob, state=None, warm=False, **opts):
    """Iteration counts of the oracle under 1e-15..1e-13 relative input
    perturbations (same problem otherwise)."""
    counts = set()
    x0 = prob.x0.copy()
    for k, eps in enumerate((0.0, 1e-15, 1e-14, 1e-13)):
        rng = np.random.default_rng(77 + k)
        prob.set_params(x0=x0 * (1.0 + eps * rng.uniform(-1, 1, x0.size)))
        _, info, _ = O.solve(prob, state=None if state is None else state.copy(), warm=warm, **opts)
        counts.add(info["iters"])
    prob.set_params(x0=x0)
    return counts


def _first_divergence(tr_gpu, tr_or):
    for k in range(min(len(tr_gpu), len(tr_or))):
        if not np.allclose(tr_gpu[k], tr_or[k], rtol=1e-6, atol=1e-300):
            return k, tr_gpu[k], tr_or[k]
    return None


def _compare(O, prob, solver, inst, st_or, info_or, info_gpu, check_iters=True, tol_y=TOL_Y,
             tol_kkt=TOL_KKT, spread=None, tr_or=None, opts=None):
    assert info_or["status"] == 0, info_or
    assert info_gpu["status"] == 0, info_gpu
    st_gpu = _state_from_gpu(O, solver, inst, prob.n, prob.m)
    err = np.max(np.abs(st_gpu.y - st_or.y)) / max(1.0, np.max(np.abs(st_or.y)))
    es, _ = O.kkt_error(prob, st_gpu, **(opts or {}))
    msg = f"y err {err:.2e}, oracle-evaluated E0 {es:.2e}, iters gpu {info_gpu['iters']} oracle {info_or['iters']}"
    if tr_or is not None:
        msg += f", first trace divergence {_first_divergence(solver.trace(inst), tr_or)}"
    assert err <= tol_y, msg
    assert es <= tol_kkt, msg
    if check_iters:
        if spread is None or len(spread) == 1:
            assert info_gpu["iters"] == info_or["iters"], msg
        else:
            assert min(spread) <= info_gpu["iters"] <= max(spread), msg + f", oracle spread {sorted(spread)}"
    return err


def test_distillation_N12_cold_solve(P, oracle):
    T = 20
    x0 = I.distillation_x0(12, 5, seed=1)
    sp, _ = I.distillation_setpoints(12, seed=1)
    prob = _oracle_problem(oracle, "distill12", T, x0, sp)
    st_or, info_or, tr = oracle.solve(prob)
    s = _gpu_solver(P, "distill12", [T])
    s.set_params(x0=x0, setpoint=np.full(T, sp), u_prev=np.array([I.U_REF]))
    info = s.solve(warm=False)[0]
    _compare(oracle, prob, s, 0, st_or, info_or, info, spread=_oracle_spread(oracle, prob), tr_or=tr)


def test_distillation_N12_closed_loop(P, oracle):
    """Five re-solves (the first cold), both sides fed the oracle's parameters."""
    T = 20
    x0 = I.distillation_x0(12, 5, seed=1)
    sp, _ = I.distillation_setpoints(12, seed=1)
    prob = _oracle_problem(oracle, "distill12", T, x0, sp)
    s = _gpu_solver(P, "distill12", [T])
    st_or, uprev = None, I.U_REF
    for k in range(5):
        s.set_params(x0=prob.x0.copy(), setpoint=np.full(T, sp), u_prev=np.array([uprev]))
        spread = _oracle_spread(oracle, prob, state=st_or, warm=k > 0)
        st_or, info_or, tr = oracle.solve(prob, state=st_or, warm=k > 0)
        info = s.solve(warm=k > 0)[0]
        _compare(oracle, prob, s, 0, st_or, info_or, info, spread=spread, tr_or=tr)
        uprev = st_or.y[prob.off_u(1)]
        prob.set_params(x0=st_or.y[prob.off_x(1):prob.off_x(1) + 12].copy(), uprev=uprev)


def test_distillation_N34_T200_resolves(P, oracle):
    """Distillation N=34, T=200: cold solve plus warm re-solves across a setpoint switch."""
    T = 200
    x0 = I.distillation_x0(34, 17, seed=2)
    a, b = I.distillation_setpoints(34, seed=2)
    prob = _oracle_problem(oracle, "distill34", T, x0, a)
    s = _gpu_solver(P, "distill34", [T])
    st_or, uprev = None, I.U_REF
    for k, spk in enumerate([a, a, a, b, b]):
        prob.set_params(sp=np.full(T, spk))
        s.set_params(x0=prob.x0.copy(), setpoint=np.full(T, spk), u_prev=np.array([uprev]))
        spread = _oracle_spread(oracle, prob, state=st_or, warm=k > 0)
        st_or, info_or, tr = oracle.solve(prob, state=st_or, warm=k > 0)
        info = s.solve(warm=k > 0)[0]
        _compare(oracle, prob, s, 0, st_or, info_or, info, spread=spread, tr_or=tr)
        uprev = st_or.y[prob.off_u(1)]
        prob.set_params(x0=st_or.y[prob.off_x(1):prob.off_x(1) + 34].copy(), uprev=uprev)


def test_paper_distillation_closed_loop(P, oracle):
    """The paper's own column (Sec. 4.1: N = 32, feed tray 17, holdups
    0.5 / 0.25 / 1.0, dt = 2, 90 intervals, stage cost (x_1 - xbar)^2 +
    0.1 (u - ubar)^2): a cold solve and four warm re-solves of the closed loop."""
    N, Nf, T = 32, 17, 90
    x0 = I.distillation_x0(N, Nf, seed=6)
    sp = np.full(T, I.PAPER_XBAR)
    prob = oracle.distillation(N, Nf, T, x0, sp, I.U_REF, **I.PAPER_COLUMN)
    s = P.Solver(P.MODEL_DISTILLATION, [T], N=N, Nf=Nf, opts=P.options(ordering=NATURAL), **I.PAPER_COLUMN)
    st_or, uprev = None, I.U_REF
    for k in range(5):
        s.set_params(x0=prob.x0.copy(), setpoint=sp, u_prev=np.array([uprev]))
        spread = _oracle_spread(oracle, prob, state=st_or, warm=k > 0)
        st_or, info_or, tr = oracle.solve(prob, state=st_or, warm=k > 0)
        info = s.solve(warm=k > 0)[0]
        _compare(oracle, prob, s, 0, st_or, info_or, info, spread=spread, tr_or=tr)
        uprev = st_or.y[prob.off_u(1)]
        prob.set_params(x0=st_or.y[prob.off_x(1):prob.off_x(1) + N].copy(), uprev=uprev)


def test_toy_code_listing_problem(P, oracle):
    T = 14
    dt = 10.0 / T
    t = dt * np.arange(1, T + 1)
    prob = oracle.toy(T, 1.0, np.sin(t), dt=dt)
    st_or, info_or, tr = oracle.solve(prob)
    s = _gpu_solver(P, "toy", [T], dt=dt)
    s.set_params(x0=np.array([1.0]), setpoint=np.sin(t))
    info = s.solve()[0]
    _compare(oracle, prob, s, 0, st_or, info_or, info, spread=_oracle_spread(oracle, prob), tr_or=tr)


@pytest.mark.parametrize("g,S,T", [(8, 8, 5), (12, 12, 4)])
def test_plate_small(P, oracle, g, S, T):
    tgt = I.plate_target(g, seed=3)
    x0 = np.zeros(g * g)
    prob = oracle.plate(g, S, T, x0, tgt)
    # at the default tolerance: both converge, the GPU point is KKT-optimal by
    # the oracle's evaluator, and the iteration count is within the spread
    st_or, info_or, tr = oracle.solve(prob)
    s = P.Solver(P.MODEL_PLATE, [T], g=g, S=S, opts=P.options(ordering=NATURAL))
    s.set_params(x0=x0, setpoint=tgt)
    info = s.solve()[0]
    _compare(oracle, prob, s, 0, st_or, info_or, info, tol_y=1e-2, spread=_oracle_spread(oracle, prob), tr_or=tr)
    # primal parity where the tolerance ball is small enough to define it
    st_or, info_or, _ = oracle.solve(prob, tol=1e-12)
    s = P.Solver(P.MODEL_PLATE, [T], g=g, S=S, opts=P.options(tol=1e-12, ordering=NATURAL))
    s.set_params(x0=x0, setpoint=tgt)
    info = s.solve()[0]
    _compare(oracle, prob, s, 0, st_or, info_or, info, check_iters=False, tol_kkt=1e-12, opts=dict(tol=1e-12))


def test_batched_instances_match_individual_oracle_solves(P, oracle):
    """Block-diagonal batch with uneven horizons: each instance equals its own
    oracle solve (same iterations), in one batched GPU solve."""
    hz = [20, 7, 13, 20, 5]
    s = _gpu_solver(P, "distill12", hz)
    for i, T in enumerate(hz):
        x0 = I.distillation_x0(12, 5, seed=10 + i)
        sp = 0.76 + 0.02 * i
        s.set_params(instance=i, x0=x0, setpoint=np.full(T, sp), u_prev=np.array([I.U_REF]))
    infos = s.solve()
    for i, T in enumerate(hz):
        x0 = I.distillation_x0(12, 5, seed=10 + i)
        prob = _oracle_problem(oracle, "distill12", T, x0, 0.76 + 0.02 * i)
        st_or, info_or, tr = oracle.solve(prob)
        _compare(oracle, prob, s, i, st_or, info_or, infos[i], spread=_oracle_spread(oracle, prob), tr_or=tr)


def test_one_iteration_matches_oracle(P, oracle):
    """After exactly one interior-point iteration (max_iter = 1) the GPU
    iterate equals the oracle's: evaluation, assembly, factorization, solve,
    step recovery, line search and update of Algorithm 2 agree."""
    T = 20
    x0 = I.distillation_x0(12, 5, seed=1)
    prob = _oracle_problem(oracle, "distill12", T, x0, 0.8)
    for iters in (1, 2, 5):
        st_or, info_or, _ = oracle.solve(prob, max_iter=iters)
        s = _gpu_solver(P, "distill12", [T], opts=P.options(max_iter=iters, ordering=NATURAL))
        s.set_params(x0=x0, setpoint=np.full(T, 0.8), u_prev=np.array([I.U_REF]))
        info = s.solve()[0]
        assert info["iters"] == info_or["iters"]
        st_gpu = _state_from_gpu(oracle, s, 0, prob.n, prob.m)
        for k in ("y", "s_p", "s_m", "w_p", "w_m", "b_p", "b_m", "zL", "zU"):
            a, b = getattr(st_gpu, k), getattr(st_or, k)
            np.testing.assert_allclose(a, b, rtol=1e-7, atol=1e-9 * (1 + np.abs(b).max()), err_msg=f"{iters} {k}")


def test_nested_dissection_matches_oracle(P, oracle):
    """The performance configuration (nested dissection, cluster fronts) on the
    34-tray, 200-interval column: same solution and KKT error as the oracle;
    iteration counts equal unless the traces first part at an inertia
    decision (a different pivot sequence meets the pivot test differently)."""
    T = 200
    x0 = I.distillation_x0(34, 17, seed=2)
    a, b = I.distillation_setpoints(34, seed=2)
    prob = _oracle_problem(oracle, "distill34", T, x0, a)
    s = P.Solver(P.MODEL_DISTILLATION, [T], N=34, Nf=17, opts=P.options(ordering=2))
    st_or, uprev = None, I.U_REF
    for k, spk in enumerate([a, a, b]):
        prob.set_params(sp=np.full(T, spk))
        s.set_params(x0=prob.x0.copy(), setpoint=np.full(T, spk), u_prev=np.array([uprev]))
        st_or, info_or, tr = oracle.solve(prob, state=st_or, warm=k > 0)
        info = s.solve(warm=k > 0)[0]
        _compare(oracle, prob, s, 0, st_or, info_or, info, check_iters=False)
        if info["iters"] != info_or["iters"]:
            div = _first_divergence(s.trace(0), tr)
            assert div is not None and div[1][3] != div[2][3], ("iterations differ without an inertia decision", div)
        uprev = st_or.y[prob.off_u(1)]
        prob.set_params(x0=st_or.y[prob.off_x(1):prob.off_x(1) + 34].copy(), uprev=uprev)


def test_nested_dissection_default_options_exact_iteration_count(P, oracle):
    """The library's defaults (nested dissection for this horizon, cluster
    fronts, sibling-limited supernodes) on the 12-tray, 20-interval column of
    seed 1: the cold solve and four warm closed-loop re-solves take exactly
    the oracle's iteration counts (no rounding-spread allowance)."""
    T = 20
    x0 = I.distillation_x0(12, 5, seed=1)
    sp, _ = I.distillation_setpoints(12, seed=1)
    prob = _oracle_problem(oracle, "distill12", T, x0, sp)
    s = P.Solver(P.MODEL_DISTILLATION, [T], N=12, Nf=5)
    assert s.stats()["ordering_used"] == 2
    st_or, uprev = None, I.U_REF
    for k in range(5):
        s.set_params(x0=prob.x0.copy(), setpoint=np.full(T, sp), u_prev=np.array([uprev]))
        st_or, info_or, tr = oracle.solve(prob, state=st_or, warm=k > 0)
        info = s.solve(warm=k > 0)[0]
        _compare(oracle, prob, s, 0, st_or, info_or, info, check_iters=True, tr_or=tr)
        uprev = st_or.y[prob.off_u(1)]
        prob.set_params(x0=st_or.y[prob.off_x(1):prob.off_x(1) + 12].copy(), uprev=uprev)


def test_ordering_does_not_change_the_solution(P):
    T = 40
    x0 = I.distillation_x0(12, 5, seed=5)
    ys, its = [], []
    for ordering in (1, 2):
        s = P.Solver(P.MODEL_DISTILLATION, [T], N=12, Nf=5, opts=P.options(ordering=ordering))
        s.set_params(x0=x0, setpoint=np.full(T, 0.8), u_prev=np.array([I.U_REF]))
        info = s.solve()[0]
        assert info["status"] == 0
        ys.append(s.get_solution(0))
        its.append(info["iters"])
    assert abs(its[0] - its[1]) <= 3  # different pivot sequences meet the inertia test differently
    assert np.max(np.abs(ys[0] - ys[1])) < 1e-6


def test_cluster_and_single_cta_factorizations_agree(P):
    """The cluster-cooperative front kernel (several CTAs per front, panels
    shared through distributed shared memory) and the one-CTA kernel compute
    the same factor up to rounding: same solution, same iteration count."""
    T = 200
    x0 = I.distillation_x0(34, 17, seed=2)
    a, _ = I.distillation_setpoints(34, seed=2)
    ys, its = [], []
    for mode in (0, 1):
        s = _gpu_solver(P, "distill34", [T], opts=P.options(factor_mode=mode, ordering=2))
        s.set_params(x0=x0, setpoint=np.full(T, a), u_prev=np.array([I.U_REF]))
        info = s.solve()[0]
        assert info["status"] == 0
        ys.append(s.get_solution(0))
        its.append(info["iters"])
    assert abs(its[0] - its[1]) <= 1
    assert np.max(np.abs(ys[0] - ys[1])) < 1e-6


def test_amalgamation_modes_agree(P, oracle):
    """Relaxed and sibling-limited supernode partitions of the nested-
    dissection ordering factor the same matrix in other groupings: the same
    solution up to rounding (each within the parity bar of the converged
    point, so within twice it of each other), both KKT-optimal by the
    oracle's evaluator, iteration counts within one."""
    T = 200
    x0 = I.distillation_x0(34, 17, seed=2)
    a, _ = I.distillation_setpoints(34, seed=2)
    prob = _oracle_problem(oracle, "distill34", T, x0, a)
    ys, its = [], []
    for am in (1, 2):
        s = _gpu_solver(P, "distill34", [T], opts=P.options(amalgamation=am, ordering=2))
        s.set_params(x0=x0, setpoint=np.full(T, a), u_prev=np.array([I.U_REF]))
        info = s.solve()[0]
        assert info["status"] == 0
        es, _ = oracle.kkt_error(prob, _state_from_gpu(oracle, s, 0, prob.n, prob.m))
        assert es <= TOL_KKT, (am, es)
        ys.append(s.get_solution(0))
        its.append(info["iters"])
    assert abs(its[0] - its[1]) <= 1, its
    assert np.max(np.abs(ys[0] - ys[1])) / max(1.0, np.max(np.abs(ys[0]))) <= 2 * TOL_Y


@pytest.mark.parametrize("hz", [[200], [30, 45, 60, 20]])
def test_solve_forms_agree(P, oracle, hz):
    """The three forms of the small-front solves: the panel transformed with
    the rows below each 16-column block scaled by the block's inverse (one
    product per block), the diagonal blocks inverted only (two products per
    block), and plain column substitution.  Same iteration counts up to
    rounding, every point KKT-optimal by the oracle's evaluator, and primal
    points within 2 TOL_Y of each other (relative to max(1, |y|)): each is held
    to TOL_Y of the converged point by the parity bar, so two of them may
    differ by twice that."""
    x0s = [I.distillation_x0(34, 17, seed=40 + i) for i in range(len(hz))]
    sps = [0.78 + 0.02 * i for i in range(len(hz))]
    ys, its = [], []
    for mode in (1, 2, 3):
        s = _gpu_solver(P, "distill34", hz, opts=P.options(panel_scale=mode, ordering=2))
        for i, T in enumerate(hz):
            s.set_params(instance=i, x0=x0s[i], setpoint=np.full(T, sps[i]), u_prev=np.array([I.U_REF]))
        infos = s.solve()
        assert all(inf["status"] == 0 for inf in infos), infos
        ys.append([s.get_solution(i) for i in range(len(hz))])
        its.append([inf["iters"] for inf in infos])
        for i, T in enumerate(hz):
            prob = oracle.distillation(34, 17, T, x0s[i], np.full(T, sps[i]), I.U_REF)
            es, _ = oracle.kkt_error(prob, _state_from_gpu(oracle, s, i, prob.n, prob.m))
            assert es <= TOL_KKT, (mode, i, es)
    for k in (1, 2):
        for i in range(len(hz)):
            assert abs(its[0][i] - its[k][i]) <= 1, its
            assert np.max(np.abs(ys[0][i] - ys[k][i])) / max(1.0, np.max(np.abs(ys[0][i]))) <= 2 * TOL_Y


def test_device_parameters_equal_host_parameters_and_runs_are_deterministic(P):
    import torch
    T = 20
    x0 = I.distillation_x0(12, 5, seed=3)
    s = _gpu_solver(P, "distill12", [T])
    s.set_params(x0=x0, setpoint=np.full(T, 0.8), u_prev=np.array([I.U_REF]))
    s.solve()
    y_host = s.get_solution(0)
    dev = torch.device("cuda")
    s.set_params(x0=torch.tensor(x0, device=dev), setpoint=torch.full((T,), 0.8, dtype=torch.float64, device=dev),
                 u_prev=torch.tensor([I.U_REF], dtype=torch.float64, device=dev))
    s.solve()
    y_dev = s.get_solution(0)
    assert np.array_equal(y_host, y_dev)  # bitwise: fixed-order reductions, no atomics
    out = torch.empty(len(y_host), dtype=torch.float64, device=dev)
    s.get_solution(0, out=(out, None))
    assert np.array_equal(out.cpu().numpy(), y_host)


def test_warm_start_without_solution_falls_back_to_cold_and_errors_are_reported(P):
    T = 10
    s = _gpu_solver(P, "distill12", [T])
    with pytest.raises(P.NmpcError):
        s.set_params(instance=3, x0=np.zeros(12))
    s.set_params(x0=I.distillation_x0(12, 5, 1), setpoint=np.full(T, 0.8), u_prev=np.array([I.U_REF]))
    info = s.solve(warm=True)[0]
    assert info["status"] == 0
