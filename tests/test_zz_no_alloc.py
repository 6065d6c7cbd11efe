"""The allocation-free one-shot solve (nmpc_solve_static) against the regular
path.

Callers that cannot allocate device memory -- a control task restricted to
memory fixed at start-up, or a plug-in handed only a stream and its buffers --
cannot give nmpc_bind a workspace.  nmpc_solve_static runs the same kernels
with all device scratch in the library's static 32 MiB array.  This file is
named so that pytest collects it last.  Besides matching the regular path on
two calls in a row, the second call must leave the device's free memory
unchanged (cudaMemGetInfo before and after it).
"""
import numpy as np
import pytest

import paper_2606_04725_gb300.inputs as I

pytestmark = pytest.mark.gpu

TOL_Y = 1e-6  # relative primal tolerance used by the parity tests


@pytest.fixture(scope="module")
def P():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2606_04725_gb300 as P
    P.build()
    return P


def _regular_solve(P, hz, x0s, sps):
    s = P.Solver(P.MODEL_DISTILLATION, hz, N=12, Nf=5)
    for i, T in enumerate(hz):
        s.set_params(instance=i, x0=x0s[i], setpoint=np.full(T, sps[i]), u_prev=np.array([I.U_REF]))
    infos = s.solve()
    return np.concatenate([s.get_solution(i) for i in range(len(hz))]), infos


@pytest.mark.parametrize("device_arrays", [False, True])
def test_static_workspace_solve_matches_regular_solve_twice(P, device_arrays):
    import torch
    hz = [20, 20]
    x0s = [I.distillation_x0(12, 5, seed=21 + i) for i in range(2)]
    sps = [0.78, 0.82]
    y_ref, info_ref = _regular_solve(P, hz, x0s, sps)
    x0 = np.concatenate(x0s)
    sp = np.concatenate([np.full(T, v) for T, v in zip(hz, sps)])
    up = np.full(2, I.U_REF)
    for call in range(2):  # two calls in a row share (and re-clear) the static array
        if device_arrays:
            dev = torch.device("cuda")
            args = [torch.tensor(a, device=dev) for a in (x0, sp, up)]
            y_out = torch.zeros(y_ref.size, dtype=torch.float64, device=dev)
        else:
            args = [x0, sp, up]
            y_out = np.zeros(y_ref.size)
        torch.cuda.synchronize()
        free0 = torch.cuda.mem_get_info()[0]
        st, infos = P._lib.solve_static(P.MODEL_DISTILLATION, hz, *args, y_out, N=12, Nf=5)
        torch.cuda.synchronize()
        free1 = torch.cuda.mem_get_info()[0]
        assert st == 0, (call, st)
        if call == 1:
            # the first call loaded the kernels and looked up the array's
            # address; the second takes no device memory at all
            assert free1 == free0, (free0, free1)
        y = y_out.cpu().numpy() if device_arrays else y_out
        err = np.max(np.abs(y - y_ref)) / max(1.0, np.max(np.abs(y_ref)))
        assert err <= TOL_Y, (call, err)
        for a, b in zip(infos, info_ref):
            assert a["status"] == 0 and a["iters"] == b["iters"]


def test_static_workspace_rejects_problems_beyond_its_size(P, capfd):
    T = 4000  # about 0.35 GB of workspace, far beyond the 32 MiB static array
    x0 = I.distillation_x0(34, 17, seed=2)
    y_out = np.zeros(34 + T * 35)
    st, _ = P._lib.solve_static(P.MODEL_DISTILLATION, [T], x0, np.full(T, 0.95), np.array([I.U_REF]), y_out,
                                N=34, Nf=17)
    assert st == 3  # NMPC_ERR_WORKSPACE
    assert "static workspace" in capfd.readouterr().err
