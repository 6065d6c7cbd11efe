"""The paper's column with its algebraic variables (eq. distill-ocp as
printed: y, L, V and S as variables with their own rows) on the GPU.

Pins:
  * against the oracle's DAE column: the solution within 1e-6 relative and
    optimal by the oracle's evaluator, on the 12-tray column in stage order
    (iteration counts inside the oracle's rounding spread) and on the paper's
    own column (32 trays, 90 intervals, its holdups and cost) under the
    library's defaults, cold and over three warm closed-loop re-solves;
  * eliminating y, L, V and S gives the substituted model the other columns
    use: the GPU's x and u trajectories of both forms agree.
"""
import numpy as np
import pytest

import paper_2606_04725_gb300.inputs as I
from test_gpu_parity import _compare, _oracle_spread

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2606_04725_gb300 as P
    P.build()
    return P


def test_dae_column_N12_matches_oracle(P, oracle):
    T = 20
    x0 = I.distillation_x0(12, 5, seed=1)
    sp, _ = I.distillation_setpoints(12, seed=1)
    prob = oracle.distillation_dae(12, 5, T, x0.copy(), np.full(T, sp), I.U_REF)
    st_or, info_or, tr = oracle.solve(prob)
    s = P.Solver(P.MODEL_DISTILLATION_DAE, [T], N=12, Nf=5, opts=P.options(ordering=1))
    s.set_params(x0=x0, setpoint=np.full(T, sp), u_prev=np.array([I.U_REF]))
    info = s.solve()[0]
    _compare(oracle, prob, s, 0, st_or, info_or, info, spread=_oracle_spread(oracle, prob), tr_or=tr)


def test_paper_column_dae_closed_loop_matches_oracle(P, oracle):
    wl = I.WORKLOADS["paper_distillation_N32_T90"]
    N, Nf, T = wl["N"], wl["Nf"], wl["T"]
    x0 = I.distillation_x0(N, Nf, wl["seed"])
    sp = np.full(T, I.PAPER_XBAR)
    prob = oracle.distillation_dae(N, Nf, T, x0.copy(), sp, I.U_REF, **I.PAPER_COLUMN)
    s = P.Solver(P.MODEL_DISTILLATION_DAE, [T], N=N, Nf=Nf, **I.PAPER_COLUMN)
    st_or = None
    for k in range(4):
        s.set_params(x0=prob.x0.copy(), setpoint=sp, u_prev=np.array([I.U_REF]))
        st_or, info_or, _ = oracle.solve(prob, state=st_or, warm=k > 0)
        info = s.solve(warm=k > 0)[0]
        _compare(oracle, prob, s, 0, st_or, info_or, info, check_iters=False)
        assert abs(info["iters"] - info_or["iters"]) <= 3  # nested dissection: other pivots
        prob.set_params(x0=st_or.y[prob.off_x(1):prob.off_x(1) + N].copy())


def test_dae_and_substituted_columns_agree(P):
    wl = I.WORKLOADS["paper_distillation_N32_T90"]
    N, Nf, T = wl["N"], wl["Nf"], wl["T"]
    x0 = I.distillation_x0(N, Nf, wl["seed"])
    sp = np.full(T, I.PAPER_XBAR)
    out = {}
    for model in (P.MODEL_DISTILLATION, P.MODEL_DISTILLATION_DAE):
        s = P.Solver(model, [T], N=N, Nf=Nf, opts=P.options(tol=1e-11), **I.PAPER_COLUMN)
        s.set_params(x0=x0, setpoint=sp, u_prev=np.array([I.U_REF]))
        assert s.solve()[0]["status"] == 0
        y = s.get_solution(0)
        nu = 1 if model == P.MODEL_DISTILLATION else N + 4
        cu = 0 if model == P.MODEL_DISTILLATION else N
        xs = np.stack([y[N + k * (N + nu):][:N] for k in range(T)])
        us = np.array([y[N + k * (N + nu) + N + cu] for k in range(T)])
        out[model] = (xs, us)
    (xa, ua), (xb, ub) = out[P.MODEL_DISTILLATION], out[P.MODEL_DISTILLATION_DAE]
    assert np.max(np.abs(xa - xb)) <= 1e-6 and np.max(np.abs(ua - ub)) <= 1e-5 * np.max(np.abs(ua))
