"""The paper's nonlinear heated plate (Sec. 4.2, eq. pde-ocp) on the GPU
against the oracle.

Unlike the benchmark's linear plate, its Jacobian and Hessian change every
iteration: the control Q sets the Dirichlet data 4.1 Q^(1/3) and Q^(1/2) of
two sides.  Pins (the oracle's model is itself pinned by complex-step
derivatives, the discrete energy balance with the heat-loss term and the
region integral, tests/test_oracle_model.py):
  * cold solves on coarse grids in stage order: the solution (temperatures
    and controls, each within 1e-6 of its own scale), optimality by the
    oracle's evaluator (E_0 <= 1e-8), iteration counts inside the oracle's
    rounding spread;
  * three closed-loop re-solves as the setpoint schedule advances;
  * the full-size 21 x 21 plate under the library's defaults: the solution
    and optimality against the oracle's.
"""
import numpy as np
import pytest

import paper_2606_04725_gb300.inputs as I
from test_gpu_parity import _oracle_spread

pytestmark = pytest.mark.gpu

TOL_KKT = 1e-8


@pytest.fixture(scope="module")
def P():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2606_04725_gb300 as P
    P.build()
    return P


def _state(O, s, n, m):
    y, du = s.get_solution(0, duals=True)
    st = O.State(n, m)
    st.y[:] = y
    for k in ("zL", "zU", "s_p", "s_m", "w_p", "w_m", "b_p", "b_m"):
        getattr(st, k)[:] = du[k]
    return st


def _check(O, prob, s, info, st_or, info_or, spread=None):
    assert info_or["status"] == 0, info_or
    assert info["status"] == 0, info
    st = _state(O, s, prob.n, prob.m)
    ix = np.concatenate([np.arange(prob.off_x(k), prob.off_x(k) + prob.nx) for k in range(prob.T + 1)])
    iu = np.array([prob.off_u(k) for k in range(1, prob.T + 1)])
    eT = np.max(np.abs(st.y[ix] - st_or.y[ix])) / np.max(np.abs(st_or.y[ix]))
    eQ = np.max(np.abs(st.y[iu] - st_or.y[iu])) / np.max(np.abs(st_or.y[iu]))
    es, _ = O.kkt_error(prob, st)
    msg = f"T err {eT:.2e}, Q err {eQ:.2e}, E0 {es:.2e}, iters gpu {info['iters']} oracle {info_or['iters']}"
    assert eT <= 1e-6 and eQ <= 1e-6, msg
    assert es <= TOL_KKT, msg
    if spread is not None:
        assert min(spread) <= info["iters"] <= max(spread), msg + f", oracle spread {sorted(spread)}"


@pytest.mark.parametrize("n", [7, 11])
def test_paper_plate_cold_solve_and_closed_loop(P, oracle, n):
    T, dt = 12, 0.08
    x0 = np.full((n - 2) ** 2, 50.0)
    s = P.Solver(P.MODEL_PAPER_PLATE, [T], g=n, opts=P.options(ordering=1))
    prob = oracle.paper_plate(n, T, x0.copy(), I.paper_plate_setpoints(0.0, T), 50.0)
    st_or = None
    for k in range(4):
        sp = I.paper_plate_setpoints(k * dt, T)
        prob.set_params(sp=sp)
        s.set_params(x0=prob.x0.copy(), setpoint=sp, u_prev=np.array([50.0]))
        spread = _oracle_spread(oracle, prob) if k == 0 else None
        st_or, info_or, _ = oracle.solve(prob, state=None if st_or is None else st_or, warm=k > 0)
        info = s.solve(warm=k > 0)[0]
        _check(oracle, prob, s, info, st_or, info_or, spread)
        prob.set_params(x0=st_or.y[prob.off_x(1):prob.off_x(1) + prob.nx].copy())


def test_paper_plate_full_size_defaults(P, oracle):
    n, T = 21, 12
    x0 = np.full((n - 2) ** 2, 50.0)
    sp = I.paper_plate_setpoints(0.0, T)
    s = P.Solver(P.MODEL_PAPER_PLATE, [T])
    assert s.stats()["n_total"] == 361 + 12 * 362
    s.set_params(x0=x0, setpoint=sp, u_prev=np.array([50.0]))
    info = s.solve()[0]
    prob = oracle.paper_plate(n, T, x0.copy(), sp, 50.0)
    st_or, info_or, _ = oracle.solve(prob)
    _check(oracle, prob, s, info, st_or, info_or)
    assert abs(info["iters"] - info_or["iters"]) <= 3  # nested dissection: other pivots
