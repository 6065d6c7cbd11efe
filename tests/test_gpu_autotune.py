"""The autotuner (nmpc_autotune) on the GPU.

It times one cold solve per candidate option set (ordering and nested-
dissection leaf size, supernode amalgamation, factorization schedule, solve
form) and keeps the fastest per interior-point iteration.  Pins: every candidate converges on these problems; the chosen
options are one of the candidates; a solver built with them reaches the
default options' solution (1e-6 relative) and iteration count (within 3:
another ordering meets the inertia test with other pivots);
a repeated call is answered from the cache with the same choice.
"""
import numpy as np
import pytest

import paper_2606_04725_gb300.inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2606_04725_gb300 as P
    P.build()
    return P


def _solve(P, hz, x0s, sps, opts):
    s = P.Solver(P.MODEL_DISTILLATION, hz, N=12, Nf=5, opts=opts)
    for i, T in enumerate(hz):
        s.set_params(instance=i, x0=x0s[i], setpoint=np.full(T, sps[i]), u_prev=np.array([I.U_REF]))
    infos = s.solve()
    return [s.get_solution(i) for i in range(len(hz))], infos


@pytest.mark.parametrize("hz", [[20], [50, 80, 120]])
def test_autotune_picks_a_converging_candidate_and_caches_it(P, hz):
    x0s = [I.distillation_x0(12, 5, seed=60 + i) for i in range(len(hz))]
    sps = [0.8 + 0.03 * i for i in range(len(hz))]
    x0 = np.concatenate(x0s)
    sp = np.concatenate([np.full(T, v) for T, v in zip(hz, sps)])
    up = np.full(len(hz), I.U_REF)
    o, rep = P.autotune(P.MODEL_DISTILLATION, hz, x0=x0, setpoint=sp, u_prev=up, N=12, Nf=5)
    assert not rep["cached"]
    cands = rep["candidates"]
    # per solve form: ND leaves 1 and 2 in two amalgamation modes with level
    # launches, the dataflow launch under ND (two amalgamation modes) and the
    # two-sided order (horizons >= 8), and stage order (horizons < 32)
    assert len(cands) == (16 if max(hz) < 32 else 14)
    assert all(c["status"] == 0 and c["iters"] > 0 and c["ms_per_iter"] > 0 and c["ms_resolve"] > 0 for c in cands), cands
    b = cands[rep["best"]]
    assert b["ms_resolve"] == min(c["ms_resolve"] for c in cands) and b["ms_resolve"] > 0
    assert (o.ordering, o.nd_leaf, o.panel_scale, o.amalgamation, o.factor_mode) == \
        (b["ordering"], b["nd_leaf"], b["panel_scale"], b["amalgamation"], b["factor_mode"])
    y_t, inf_t = _solve(P, hz, x0s, sps, o)
    y_d, inf_d = _solve(P, hz, x0s, sps, P.options())
    for i in range(len(hz)):
        assert inf_t[i]["status"] == 0 and inf_d[i]["status"] == 0
        assert abs(inf_t[i]["iters"] - inf_d[i]["iters"]) <= 3  # other orderings: other pivot sequences
        assert np.max(np.abs(y_t[i] - y_d[i])) / max(1.0, np.max(np.abs(y_d[i]))) <= 1e-6
    o2, rep2 = P.autotune(P.MODEL_DISTILLATION, hz, x0=x0, setpoint=sp, u_prev=up, N=12, Nf=5)
    assert rep2["cached"]
    assert (o2.ordering, o2.nd_leaf, o2.panel_scale, o2.amalgamation) == \
        (o.ordering, o.nd_leaf, o.panel_scale, o.amalgamation)
