"""GPU parity of the HyKKT form (NMPC_KKT_HYKKT) against the oracle's HyKKT
form: the equalities keep their multipliers, K_gamma = W + Sigma +
delta_w I + gamma H^T H goes through the same assembly, factorization and
solves, and conjugate gradients on H K_gamma^-1 H^T give the multipliers'
step (Sec. 3.2.2's alternative to Lifted-KKT).

Criteria as for the lifted form: primal within 1e-6 relative, E_0 <= 1e-8
by the oracle's HyKKT evaluator at the GPU's point, iteration counts in
stage order equal or inside the oracle's rounding spread; CG iteration
totals within one per Newton step of the oracle's.
"""
import numpy as np
import pytest

import paper_2606_04725_gb300.inputs as I
from test_gpu_parity import _compare, _oracle_spread, _state_from_gpu

pytestmark = pytest.mark.gpu

HY = dict(kkt=1)


@pytest.fixture(scope="module")
def P():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2606_04725_gb300 as P
    P.build()
    return P


def _cg_close(info, info_or):
    assert abs(info["cg_iters"] - info_or["cg_iters"]) <= max(1, info_or["iters"]), (info, info_or)


@pytest.mark.parametrize("use_graph", [1, 0])
def test_hykkt_N12_closed_loop_stage_order(P, oracle, use_graph):
    T = 20
    x0 = I.distillation_x0(12, 5, seed=1)
    sp, _ = I.distillation_setpoints(12, seed=1)
    prob = oracle.distillation(12, 5, T, x0.copy(), np.full(T, sp), I.U_REF)
    s = P.Solver(P.MODEL_DISTILLATION, [T], N=12, Nf=5,
                 opts=P.options(ordering=1, kkt=P.KKT_HYKKT, use_graph=use_graph))
    st_or, uprev = None, I.U_REF
    for k in range(5):
        s.set_params(x0=prob.x0.copy(), setpoint=np.full(T, sp), u_prev=np.array([uprev]))
        spread = _oracle_spread(oracle, prob, state=st_or, warm=k > 0, **HY)
        st_or, info_or, tr = oracle.solve(prob, state=st_or, warm=k > 0, **HY)
        info = s.solve(warm=k > 0)[0]
        _compare(oracle, prob, s, 0, st_or, info_or, info, spread=spread, tr_or=tr, opts=HY)
        _cg_close(info, info_or)
        assert info["cg_iters"] > 0
        uprev = st_or.y[prob.off_u(1)]
        prob.set_params(x0=st_or.y[prob.off_x(1):prob.off_x(1) + 12].copy(), uprev=uprev)


def test_hykkt_multipliers_match_the_oracle(P, oracle):
    """lambda itself (not only the primal point) agrees with the oracle's."""
    T = 20
    x0 = I.distillation_x0(12, 5, seed=3)
    sp, _ = I.distillation_setpoints(12, seed=3)
    prob = oracle.distillation(12, 5, T, x0.copy(), np.full(T, sp), I.U_REF)
    st_or, info_or, _ = oracle.solve(prob, tol=1e-11, **HY)
    s = P.Solver(P.MODEL_DISTILLATION, [T], N=12, Nf=5, opts=P.options(ordering=1, kkt=P.KKT_HYKKT, tol=1e-11))
    s.set_params(x0=x0, setpoint=np.full(T, sp), u_prev=np.array([I.U_REF]))
    assert s.solve()[0]["status"] == 0
    st = _state_from_gpu(oracle, s, 0, prob.n, prob.m)
    np.testing.assert_allclose(st.w_p, st_or.w_p, rtol=1e-6, atol=1e-8 * np.abs(st_or.w_p).max())
    assert np.all(st.w_m == 0.0)


def test_hykkt_truncated_cg_matches_the_oracle(P, oracle):
    """With at most 2 CG steps per Newton step both sides take the same
    inexact steps (stage order): the truncation is part of the method."""
    T = 20
    x0 = I.distillation_x0(12, 5, seed=1)
    sp, _ = I.distillation_setpoints(12, seed=1)
    prob = oracle.distillation(12, 5, T, x0.copy(), np.full(T, sp), I.U_REF)
    opts = dict(kkt=1, cg_max_iter=2)
    st_or, info_or, tr = oracle.solve(prob, **opts)
    s = P.Solver(P.MODEL_DISTILLATION, [T], N=12, Nf=5, opts=P.options(ordering=1, kkt=P.KKT_HYKKT, cg_max_iter=2))
    s.set_params(x0=x0, setpoint=np.full(T, sp), u_prev=np.array([I.U_REF]))
    info = s.solve()[0]
    _compare(oracle, prob, s, 0, st_or, info_or, info, spread=_oracle_spread(oracle, prob, **opts), tr_or=tr, opts=HY)
    assert info["cg_iters"] <= 2 * info["iters"]
    _cg_close(info, info_or)


def test_hykkt_N34_T200_defaults(P, oracle):
    """Nested dissection and the dataflow factorization (the library's
    defaults) on the N=34, T=200 column: cold plus three warm re-solves."""
    T = 200
    x0 = I.distillation_x0(34, 17, seed=2)
    a, _ = I.distillation_setpoints(34, seed=2)
    prob = oracle.distillation(34, 17, T, x0.copy(), np.full(T, a), I.U_REF)
    s = P.Solver(P.MODEL_DISTILLATION, [T], N=34, Nf=17, opts=P.options(kkt=P.KKT_HYKKT))
    st_or, uprev = None, I.U_REF
    for k in range(4):
        s.set_params(x0=prob.x0.copy(), setpoint=np.full(T, a), u_prev=np.array([uprev]))
        st_or, info_or, _ = oracle.solve(prob, state=st_or, warm=k > 0, **HY)
        info = s.solve(warm=k > 0)[0]
        _compare(oracle, prob, s, 0, st_or, info_or, info, check_iters=False, opts=HY)
        assert abs(info["iters"] - info_or["iters"]) <= 2
        uprev = st_or.y[prob.off_u(1)]
        prob.set_params(x0=st_or.y[prob.off_x(1):prob.off_x(1) + 34].copy(), uprev=uprev)


def test_hykkt_uneven_batch_matches_single_solves(P):
    """Each instance of a batch runs its own CG: a 3-instance batch gives each
    instance's single solve."""
    hz = [15, 20, 27]
    x0s = [I.distillation_x0(12, 5, seed=10 + i) for i in range(3)]
    sps = [I.distillation_setpoints(12, seed=10 + i)[0] for i in range(3)]
    o = P.options(ordering=1, kkt=P.KKT_HYKKT)
    b = P.Solver(P.MODEL_DISTILLATION, hz, N=12, Nf=5, opts=o)
    for i in range(3):
        b.set_params(instance=i, x0=x0s[i], setpoint=np.full(hz[i], sps[i]), u_prev=np.array([I.U_REF]))
    ib = b.solve()
    for i in range(3):
        s = P.Solver(P.MODEL_DISTILLATION, [hz[i]], N=12, Nf=5, opts=o)
        s.set_params(x0=x0s[i], setpoint=np.full(hz[i], sps[i]), u_prev=np.array([I.U_REF]))
        info = s.solve()[0]
        assert info["status"] == 0 and ib[i]["status"] == 0
        assert abs(info["iters"] - ib[i]["iters"]) <= 1
        assert np.max(np.abs(s.get_solution(0) - b.get_solution(i))) <= 1e-7


def test_hykkt_paper_plate_matches_oracle(P, oracle):
    """The paper's nonlinear plate (n = 7) in the HyKKT form, stage order:
    cold solve and two closed-loop re-solves."""
    n, T, dt = 7, 12, 0.08
    x0 = np.full((n - 2) ** 2, 50.0)
    prob = oracle.paper_plate(n, T, x0.copy(), I.paper_plate_setpoints(0.0, T, dt), 50.0)
    s = P.Solver(P.MODEL_PAPER_PLATE, [T], g=n, opts=P.options(ordering=1, kkt=P.KKT_HYKKT))
    st_or = None
    for r in range(3):
        sp = I.paper_plate_setpoints(r * dt, T, dt)
        prob.set_params(sp=sp)
        s.set_params(x0=prob.x0.copy(), setpoint=sp, u_prev=np.array([50.0]))
        spread = _oracle_spread(oracle, prob, state=st_or, warm=r > 0, **HY)
        st_or, info_or, tr = oracle.solve(prob, state=st_or, warm=r > 0, **HY)
        info = s.solve(warm=r > 0)[0]
        _compare(oracle, prob, s, 0, st_or, info_or, info, spread=spread, tr_or=tr, opts=HY)
        prob.set_params(x0=st_or.y[prob.off_x(1):prob.off_x(1) + (n - 2) ** 2].copy())


def test_hykkt_sensitivity_needs_the_lifted_form(P):
    s = P.Solver(P.MODEL_TOY, [6], dt=0.5, opts=P.options(kkt=P.KKT_HYKKT))
    s.set_params(x0=np.array([1.0]), setpoint=np.sin(np.arange(6)))
    assert s.solve()[0]["status"] == 0
    with pytest.raises(P.NmpcError):
        s.sensitivity(0, np.ones(s.dims[0][0]))
