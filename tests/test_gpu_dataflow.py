"""The dataflow factorization (factor_mode 3) and the two-sided stage order
(ordering 3) on the GPU.

Pins:
  * the dataflow launch computes each front with the same arithmetic, in the
    same order, as the per-level cluster kernel: the same iterations and the
    same solution to rounding level, under nested dissection and stage order;
  * the two-sided order eliminates the same matrix in another order: against
    the oracle, the solution within the parity bar and KKT-optimal by the
    oracle's own evaluator, iteration counts equal unless the traces first
    part at an inertia decision (as for nested dissection) or in the end game,
    where the constraint violation theta is at rounding level (below 1e-10)
    and the elimination order's rounding moves the last steps, and then
    within two;
  * a batch of uneven horizons in the two-sided order with the dataflow
    launch matches the oracle instance by instance, and the batch calls
    (all instances' parameters in one call, every solution in one read)
    agree with the per-instance calls.
"""
import numpy as np
import pytest

import paper_2606_04725_gb300.inputs as I
from test_gpu_parity import _compare, _first_divergence, _oracle_problem

pytestmark = pytest.mark.gpu

TWO_SIDED, ND, NATURAL = 3, 2, 1


def _check_counts(info, info_or, div):
    """Equal counts, or a first trace difference at an inertia decision
    (trace column 3, delta_w) or at rounding level in the end game (theta,
    column 4, below 1e-10 on both sides), with counts within two."""
    if info["iters"] == info_or["iters"]:
        return
    assert div is not None, "counts differ with identical traces"
    k, tg, to = div
    inertia = tg[3] != to[3]
    end_game = max(tg[4], to[4]) <= 1e-10
    assert (inertia or end_game) and abs(info["iters"] - info_or["iters"]) <= 2, (info["iters"], info_or["iters"], div)


@pytest.fixture(scope="module")
def P():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2606_04725_gb300 as P
    P.build()
    return P


@pytest.mark.parametrize("ordering", [ND, NATURAL])
def test_dataflow_launch_equals_level_launches(P, ordering):
    T = 200
    x0 = I.distillation_x0(34, 17, seed=2)
    a, _ = I.distillation_setpoints(34, seed=2)
    ys, its = [], []
    for mode in (0, 3):
        s = P.Solver(P.MODEL_DISTILLATION, [T], N=34, Nf=17,
                     opts=P.options(ordering=ordering, factor_mode=mode, amalgamation=2))
        s.set_params(x0=x0, setpoint=np.full(T, a), u_prev=np.array([I.U_REF]))
        info = s.solve()[0]
        assert info["status"] == 0, (mode, info)
        ys.append(s.get_solution(0))
        its.append(info["iters"])
    assert its[0] == its[1], its
    assert np.max(np.abs(ys[0] - ys[1])) <= 1e-12 * max(1.0, np.max(np.abs(ys[0])))


def test_two_sided_order_matches_oracle(P, oracle):
    T = 200
    x0 = I.distillation_x0(34, 17, seed=2)
    a, b = I.distillation_setpoints(34, seed=2)
    prob = _oracle_problem(oracle, "distill34", T, x0, a)
    s = P.Solver(P.MODEL_DISTILLATION, [T], N=34, Nf=17, opts=P.options(ordering=TWO_SIDED, factor_mode=3))
    st = s.stats()
    assert st["ordering_used"] == TWO_SIDED and st["n_levels"] < 100  # about half the chain of stage order
    st_or, uprev = None, I.U_REF
    for k, spk in enumerate([a, a, b]):
        prob.set_params(sp=np.full(T, spk))
        s.set_params(x0=prob.x0.copy(), setpoint=np.full(T, spk), u_prev=np.array([uprev]))
        st_or, info_or, tr = oracle.solve(prob, state=st_or, warm=k > 0)
        info = s.solve(warm=k > 0)[0]
        _compare(oracle, prob, s, 0, st_or, info_or, info, check_iters=False)
        _check_counts(info, info_or, _first_divergence(s.trace(0), tr))
        uprev = st_or.y[prob.off_u(1)]
        prob.set_params(x0=st_or.y[prob.off_x(1):prob.off_x(1) + 34].copy(), uprev=uprev)


def test_two_sided_dataflow_batch_matches_oracle_and_batch_calls(P, oracle):
    hz = np.array([20, 7, 13, 20, 5, 16], dtype=np.int32)
    x0s = np.stack([I.distillation_x0(12, 5, seed=40 + i) for i in range(hz.size)])
    sps = 0.76 + 0.015 * np.arange(hz.size)
    s = P.Solver(P.MODEL_DISTILLATION, hz, N=12, Nf=5, opts=P.options(ordering=TWO_SIDED, factor_mode=3))
    # all instances in one call: setpoints of unequal horizons packed one after another
    s.set_params(x0=x0s.ravel().copy(), setpoint=np.concatenate([np.full(T, v) for T, v in zip(hz, sps)]),
                 u_prev=np.full(hz.size, I.U_REF))
    infos = s.solve()
    y_all = s.get_solution(-1)
    off = 0
    for i, T in enumerate(hz):
        y = s.get_solution(i)
        assert np.array_equal(y_all[off:off + y.size], y)
        off += y.size
        prob = _oracle_problem(oracle, "distill12", int(T), x0s[i].copy(), float(sps[i]))
        st_or, info_or, tr = oracle.solve(prob)
        _compare(oracle, prob, s, i, st_or, info_or, infos[i], check_iters=False)
        _check_counts(infos[i], info_or, _first_divergence(s.trace(i), tr))
    assert off == y_all.size
    # a warm re-solve of every instance from its own x_1 and u_1, set in one call,
    # equals the same re-solve with the parameters set instance by instance
    x1 = np.concatenate([s.get_solution(i)[12:24] for i in range(hz.size)])
    u1 = np.array([s.get_solution(i)[24] for i in range(hz.size)])
    sp_packed = np.concatenate([np.full(T, v) for T, v in zip(hz, sps)])
    s2 = P.Solver(P.MODEL_DISTILLATION, hz, N=12, Nf=5, opts=P.options(ordering=TWO_SIDED, factor_mode=3))
    for i, T in enumerate(hz):
        s2.set_params(instance=i, x0=x0s[i], setpoint=np.full(T, sps[i]), u_prev=np.array([I.U_REF]))
    s2.solve()
    s.set_params(x0=x1, setpoint=sp_packed, u_prev=u1)
    a = s.solve(warm=True)
    for i, T in enumerate(hz):
        s2.set_params(instance=i, x0=x1[12 * i:12 * i + 12], setpoint=np.full(T, sps[i]), u_prev=u1[i:i + 1])
    b = s2.solve(warm=True)
    assert [f["iters"] for f in a] == [f["iters"] for f in b]
    assert np.array_equal(s.get_solution(-1), s2.get_solution(-1))


def test_two_sided_dataflow_batch_of_columns_matches_single_solves(P):
    n_inst = 12
    hz = I.batch_horizons(n_inst, 50, 200, seed=4)
    x0s, sps = I.batch_distillation(n_inst, 34, 17, seed=4)
    opts = dict(ordering=TWO_SIDED, factor_mode=3, panel_scale=3)
    s = P.Solver(P.MODEL_DISTILLATION, hz, N=34, Nf=17, opts=P.options(**opts))
    s.set_params(x0=x0s.ravel().copy(), setpoint=np.concatenate([np.full(T, v) for T, v in zip(hz, sps)]),
                 u_prev=np.full(n_inst, I.U_REF))
    infos = s.solve()
    assert all(f["status"] == 0 for f in infos), [f["status"] for f in infos]
    for i in (0, 5, 11):
        T = hz[i]
        s1 = P.Solver(P.MODEL_DISTILLATION, [T], N=34, Nf=17, opts=P.options(**opts))
        s1.set_params(x0=x0s[i], setpoint=np.full(T, sps[i]), u_prev=np.array([I.U_REF]))
        info1 = s1.solve()[0]
        assert info1["status"] == 0
        assert infos[i]["iters"] == info1["iters"], (i, infos[i]["iters"], info1["iters"])
        assert np.max(np.abs(s.get_solution(i) - s1.get_solution(0))) <= 1e-9
