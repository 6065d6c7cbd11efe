"""The heated plate of the 128 x 128, 16-actuator, 100-interval configuration
at the reduced grid g = 32 (S = 16, T = 100, n = 105,024), on the GPU under
the library's defaults (nested dissection, large-front path) against the
oracle's sparse Cholesky with its own nested dissection.

The oracle needs three and a half hours of one host core for its cold solve
here, so its results were written once by tests/golden/make_plate_g32_S16_T100.py (oracle
only) to tests/golden/plate_g32_S16_T100.json.  Pins:
  * the converged primal point at tol 1e-12 equals the oracle's at 4096 seeded
    positions within 1e-6 relative, with the same objective and tracking loss;
    the two sides eliminate in different orders, so their pivot sequences and
    inertia decisions differ and the iteration counts agree within 15%;
  * the GPU point is optimal by the oracle's own KKT evaluator;
  * the adjoint gradient of the state-tracking loss with respect to the
    initial field and the target field agrees with central differences of GPU
    re-solves at tol 1e-13 along 20 seeded unit directions (seed 5),
    h = 1e-6, within 1e-5 of the gradient's scale, and with the oracle's
    central differences along the first three of them.
"""
import json
import os

import numpy as np
import pytest

import paper_2606_04725_gb300.inputs as I
from test_gpu_plate_reduced import _loss_and_grad_y

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module")
def gold():
    with open(os.path.join(HERE, "golden", "plate_g32_S16_T100.json")) as f:
        return json.load(f)


@pytest.fixture(scope="module")
def P():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2606_04725_gb300 as P
    P.build()
    return P


@pytest.fixture(scope="module")
def solved(P, gold):
    g, S, T = gold["g"], gold["S"], gold["T"]
    target = I.plate_target(g, seed=gold["target_seed"])
    s = P.Solver(P.MODEL_PLATE, [T], g=g, S=S, opts=P.options(tol=gold["tol"]))
    s.set_params(x0=np.zeros(g * g), setpoint=target)
    info = s.solve()[0]
    assert info["status"] == 0, info
    return s, info, target


def test_primal_solution_matches_the_oracle(solved, gold):
    s, info, target = solved
    y = s.get_solution(0)
    idx = np.array(gold["sample_index"])
    ref = np.array(gold["sample_y"])
    err = np.max(np.abs(y[idx] - ref)) / max(1.0, np.max(np.abs(ref)))
    assert err <= 1e-6, err
    assert abs(info["objective"] - gold["objective"]) <= 1e-8 * max(1.0, abs(gold["objective"]))
    loss, _, _ = _loss_and_grad_y(y, target, gold["g"], gold["S"], gold["T"])
    assert abs(loss - gold["loss"]) <= 1e-8 * max(1.0, gold["loss"])
    # different elimination orders part at inertia-correction decisions (both
    # take about 20 corrections here): the counts agree within 15%
    assert abs(info["iters"] - gold["iters"]) <= max(3, (15 * gold["iters"]) // 100), (info["iters"], gold["iters"])


def test_gpu_point_is_optimal_by_the_oracle_evaluator(solved, gold, oracle):
    s, _, target = solved
    g, S, T = gold["g"], gold["S"], gold["T"]
    prob = oracle.plate(g, S, T, np.zeros(g * g), target.copy())
    y, du = s.get_solution(0, duals=True)
    st = oracle.State(prob.n, prob.m)
    st.y[:] = y
    for k in ("zL", "zU", "s_p", "s_m", "w_p", "w_m", "b_p", "b_m"):
        getattr(st, k)[:] = du[k]
    es, _ = oracle.kkt_error(prob, st, tol=gold["tol"], linsolve=oracle.LINSOLVE_SPARSE)
    assert es <= 10 * gold["tol"], es


def test_adjoint_matches_central_differences_on_20_directions(P, solved, gold):
    s, _, target = solved
    g, S, T = gold["g"], gold["S"], gold["T"]
    g2 = g * g
    y0, du0 = s.get_solution(0, duals=True)
    duals0 = np.concatenate([du0[k] for k in ("zL", "zU", "s_p", "s_m", "w_p", "w_m", "b_p", "b_m")])
    _, gy, gt = _loss_and_grad_y(y0, target, g, S, T)
    dx0, dtg = np.zeros(g2), np.zeros(g2)
    s.sensitivity(0, gy, dx0, dtg)
    grad = np.concatenate([dx0, dtg + gt])
    dirs = I.unit_directions(2 * g2, gold["directions"], seed=gold["direction_seed"])
    ad = dirs @ grad
    scale = np.max(np.abs(ad))
    h = gold["fd_h"]
    fd_solver = P.Solver(P.MODEL_PLATE, [T], g=g, S=S, opts=P.options(tol=gold["fd_tol"]))
    fd = []
    for q in range(dirs.shape[0]):
        dx, dt = dirs[q, :g2], dirs[q, g2:]
        vals = []
        for sgn in (+1, -1):
            fd_solver.set_start(0, y0, duals0)
            fd_solver.set_params(x0=sgn * h * dx, setpoint=target + sgn * h * dt)
            info = fd_solver.solve(warm=True)[0]
            assert info["status"] == 0, (q, sgn, info)
            vals.append(_loss_and_grad_y(fd_solver.get_solution(0), target + sgn * h * dt, g, S, T)[0])
        fd.append((vals[0] - vals[1]) / (2 * h))
    fd = np.array(fd)
    assert np.max(np.abs(fd - ad)) <= 1e-5 * scale, (np.max(np.abs(fd - ad)), scale)
    for q, v in zip(gold["fd_directions"], gold["fd"]):
        assert abs(ad[q] - v) <= 1e-5 * scale, (q, ad[q], v, scale)
