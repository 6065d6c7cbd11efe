"""Failure statuses of the interior-point loop on the GPU, each produced on
the host (bad parameters, tiny limits), never by a GPU fault.

  * NaN in the initial-state parameter: the residuals are not finite, so the
    solve stops with NMPC_NONFINITE, as the oracle does;
  * an iteration limit of 2: NMPC_MAX_ITER after exactly 2 iterations;
  * a regularization ceiling dw_max below the second trial value of the
    inertia correction (W&B Algorithm IC: 1e-4, then x100): the first
    factorization that needs a raised delta_w ends the solve with
    NMPC_INERTIA_FAIL, at the same iteration as the oracle with the same
    ceiling (stage order on both sides, so the same pivot sequence);
  * spin_limit = 1 makes the bounded waits between the CTAs of a cluster
    factorization and between the blocks of the persistent solves give up
    almost at once: the solve returns NMPC_TIMEOUT (host loop and graph),
    every kernel exits, and the context stays usable for the next solve.
"""
import numpy as np
import pytest

import paper_2606_04725_gb300.inputs as I

pytestmark = pytest.mark.gpu

NONFINITE, MAX_ITER, INERTIA_FAIL, TIMEOUT = 13, 10, 12, 14


@pytest.fixture(scope="module")
def P():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2606_04725_gb300 as P
    P.build()
    return P


def _column12(P, x0, T=20, **opts):
    s = P.Solver(P.MODEL_DISTILLATION, [T], N=12, Nf=5, opts=P.options(**opts))
    sp, _ = I.distillation_setpoints(12, seed=1)
    s.set_params(x0=x0, setpoint=np.full(T, sp), u_prev=np.array([I.U_REF]))
    return s, sp


@pytest.mark.parametrize("use_graph", [1, 0])
def test_nan_parameter_gives_nonfinite(P, oracle, use_graph):
    x0 = I.distillation_x0(12, 5, seed=1)
    x0[3] = np.nan
    s, sp = _column12(P, x0, use_graph=use_graph)
    info = s.solve()[0]
    assert info["status"] == NONFINITE, info
    _, oinfo, _ = oracle.solve(oracle.distillation(12, 5, 20, x0, np.full(20, sp), I.U_REF))
    assert oinfo["status"] == NONFINITE


@pytest.mark.parametrize("use_graph", [1, 0])
def test_iteration_limit_gives_max_iter(P, use_graph):
    s, _ = _column12(P, I.distillation_x0(12, 5, seed=1), max_iter=2, use_graph=use_graph)
    info = s.solve()[0]
    assert info["status"] == MAX_ITER and info["iters"] == 2, info


@pytest.mark.parametrize("use_graph", [1, 0])
def test_regularization_ceiling_gives_inertia_fail_at_the_oracles_iteration(P, oracle, use_graph):
    x0 = I.distillation_x0(12, 5, seed=1)
    sp, _ = I.distillation_setpoints(12, seed=1)
    prob = oracle.distillation(12, 5, 20, x0, np.full(20, sp), I.U_REF)
    _, full, _ = oracle.solve(prob)
    assert full["status"] == 0 and full["inertia_retries"] > 0  # the cold solve needs delta_w > 0
    _, oinfo, _ = oracle.solve(prob, dw_max=1e-3)
    assert oinfo["status"] == INERTIA_FAIL
    s, _ = _column12(P, x0, ordering=1, dw_max=1e-3, use_graph=use_graph)
    info = s.solve()[0]
    assert info["status"] == INERTIA_FAIL, info
    assert info["iters"] == oinfo["iters"], (info["iters"], oinfo["iters"])


@pytest.mark.parametrize("use_graph", [1, 0])
def test_tiny_spin_limit_gives_timeout_and_leaves_the_context_usable(P, use_graph):
    # N = 34, T = 200 under nested dissection: cluster-factored separator
    # fronts (waits between CTAs) and persistent solves (waits between blocks)
    wl = I.WORKLOADS["distillation_N34_T200"]
    x0 = I.distillation_x0(34, 17, wl["seed"])
    a, _ = I.distillation_setpoints(34, wl["seed"])
    s = P.Solver(P.MODEL_DISTILLATION, [200], N=34, Nf=17,
                 opts=P.options(ordering=2, spin_limit=1, use_graph=use_graph))
    s.set_params(x0=x0, setpoint=np.full(200, a), u_prev=np.array([I.U_REF]))
    with pytest.raises(P.NmpcError) as e:
        s.solve(raise_on_fail=True)
    assert e.value.status == TIMEOUT
    s.close()
    ok = P.Solver(P.MODEL_DISTILLATION, [200], N=34, Nf=17, opts=P.options(ordering=2, use_graph=use_graph))
    ok.set_params(x0=x0, setpoint=np.full(200, a), u_prev=np.array([I.U_REF]))
    assert ok.solve()[0]["status"] == 0
