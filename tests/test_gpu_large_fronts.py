"""Large-front path (level-batched blocked LDL^T over many SMs) on the GPU.

The heated plate's nested-dissection fronts grow to thousands of rows, far
beyond a cluster's shared memory; those levels run the blocked path.  Pins:
  * on a small plate, forcing the blocked path on every level gives the same
    solution and iteration count as the cluster path, and both agree with the
    oracle (iteration count within the oracle's rounding spread, the GPU point
    KKT-optimal by the oracle's evaluator);
  * on larger plates (the oracle's banded solve is too slow there) the GPU's
    converged primal-dual point is checked by the oracle's KKT evaluator,
    which shares no code with the CUDA path: scaled E_0 <= 1e-8;
  * the full-size plate (g = 64, S = 8, T = 50: n = 209,296) likewise, plus
    the bounds of the controls and the state upper bound hold at the point,
    and the adjoint there satisfies the envelope theorem (dl/dx0 = -lambda
    for l = f).
"""
import numpy as np
import pytest

import paper_2606_04725_gb300.inputs as I

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


def _state(O, solver, n, m):
    y, du = solver.get_solution(0, duals=True)
    st = O.State(n, m)
    st.y[:] = y
    for k in ("zL", "zU", "s_p", "s_m", "w_p", "w_m", "b_p", "b_m"):
        getattr(st, k)[:] = du[k]
    return st


def _plate_solve(P, g, S, T, **opts):
    s = P.Solver(P.MODEL_PLATE, [T], g=g, S=S, opts=P.options(**opts))
    s.set_params(x0=np.zeros(g * g), setpoint=I.plate_target(g, seed=3))
    info = s.solve()[0]
    return s, info


def test_blocked_path_matches_cluster_path_and_oracle(P, oracle):
    g, S, T = 16, 4, 8
    s0, i0 = _plate_solve(P, g, S, T, ordering=2, factor_mode=0)
    s2, i2 = _plate_solve(P, g, S, T, ordering=2, factor_mode=2)
    assert i0["status"] == 0 and i2["status"] == 0
    assert abs(i0["iters"] - i2["iters"]) <= 1
    y0, y2 = s0.get_solution(0), s2.get_solution(0)
    assert np.max(np.abs(y0 - y2)) <= 1e-5
    prob = oracle.plate(g, S, T, np.zeros(g * g), I.plate_target(g, seed=3))
    st_or, info_or, _ = oracle.solve(prob)
    assert info_or["status"] == 0
    # the plate's primal point is defined to ~1e-3 at tol 1e-8; iterations and KKT
    assert abs(i2["iters"] - info_or["iters"]) <= 3
    es, _ = oracle.kkt_error(prob, _state(oracle, s2, prob.n, prob.m))
    assert es <= TOL_KKT, es


def _check_kkt_and_bounds(oracle, s, g, S, T):
    prob = oracle.plate(g, S, T, np.zeros(g * g), I.plate_target(g, seed=3))
    st = _state(oracle, s, prob.n, prob.m)
    es, _ = oracle.kkt_error(prob, st)
    assert es <= TOL_KKT, es
    lo, hi = prob.bounds()
    assert np.all(st.y >= lo - 1e-12) and np.all(st.y <= hi + 1e-12)


def test_plate_g32_converges_to_oracle_kkt_point(P, oracle):
    g, S, T = 32, 8, 20
    s, info = _plate_solve(P, g, S, T)
    assert info["status"] == 0, info
    _check_kkt_and_bounds(oracle, s, g, S, T)


def test_plate_full_size(P, oracle):
    """g = 64, S = 8, T = 50 (n = 209,296): one cold solve at tol 1e-8, then
    the adjoint at that point: for the loss l = f(y*) the envelope theorem
    gives dl/dx0 = -lambda on the initial-condition rows."""
    g, S, T = 64, 8, 50
    s, info = _plate_solve(P, g, S, T)
    assert info["status"] == 0, info
    assert s.stats()["n_total"] == 209296
    _check_kkt_and_bounds(oracle, s, g, S, T)
    prob = oracle.plate(g, S, T, np.zeros(g * g), I.plate_target(g, seed=3))
    y, du = s.get_solution(0, duals=True)
    _, grad_f, _, _ = oracle.evaluate(prob, y)
    dx0 = np.zeros(g * g)
    dsp = np.zeros(g * g)
    s.sensitivity(0, grad_f, dx0, dsp)
    lam0 = du["w_p"][:g * g] - du["w_m"][:g * g]
    scale = max(1e-12, np.max(np.abs(lam0)))
    assert np.max(np.abs(dx0 + lam0)) <= 1e-4 * scale, (np.max(np.abs(dx0 + lam0)), scale)
