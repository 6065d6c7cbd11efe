"""Adjoint sensitivity (nmpc_sensitivity, torch.autograd) on the GPU.

Pins, none of which uses the adjoint's own arithmetic:
  * envelope theorem: for l = f(y*), dl/dp_x0 equals minus the multipliers of
    the initial-condition rows, lambda = w+ - w- (closed form at the solution);
  * central finite differences of full re-solves (tol 1e-12, h = 1e-5) along
    seeded unit directions, on the GPU and on the oracle.
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


def test_envelope_theorem_initial_state(P, oracle):
    T = 20
    x0 = I.distillation_x0(12, 5, seed=1)
    sp = np.full(T, 0.8)
    s = P.Solver(P.MODEL_DISTILLATION, [T], N=12, Nf=5, opts=P.options(tol=1e-10))
    s.set_params(x0=x0, setpoint=sp, u_prev=np.array([I.U_REF]))
    assert s.solve()[0]["status"] == 0
    y, du = s.get_solution(0, duals=True)
    prob = oracle.distillation(12, 5, T, x0, sp, I.U_REF)
    _, grad_f, _, _ = oracle.evaluate(prob, y)            # dl/dy for l = f(y*)
    dx0 = np.zeros(12)
    dsp = np.zeros(T)
    s.sensitivity(0, grad_f, dx0, dsp)
    lam0 = du["w_p"][:12] - du["w_m"][:12]
    np.testing.assert_allclose(dx0, -lam0, rtol=1e-5, atol=1e-7)


@pytest.mark.parametrize("model", ["distill", "plate"])
def test_adjoint_matches_central_differences(P, oracle, model):
    rng = np.random.default_rng(5)
    if model == "distill":
        N, T = 12, 20
        x0 = I.distillation_x0(12, 5, seed=4)
        sp = np.full(T, 0.79)
        mk = lambda: P.Solver(P.MODEL_DISTILLATION, [T], N=12, Nf=5, opts=P.options(tol=1e-12))
        up = np.array([I.U_REF])
        nx, nsp = 12, T
        idx = np.array([N + (k - 1) * (N + 1) for k in range(1, T + 1)])
        def loss(y, spv):
            e = y[idx] - spv
            return np.sum(e * e)
        def dloss(y, spv):
            gy = np.zeros(y.size); gy[idx] = 2 * (y[idx] - spv)
            return gy, -2 * (y[idx] - spv)   # explicit dl/dsp part
    else:
        g, S, T = 6, 4, 4
        x0 = np.zeros(g * g)
        sp = I.plate_target(g, seed=3)
        mk = lambda: P.Solver(P.MODEL_PLATE, [T], g=g, S=S, opts=P.options(tol=1e-12))
        up = None
        nx, nsp = g * g, g * g
        def loss(y, spv):
            xs = np.stack([y[g * g + (k - 1) * (g * g + S):][:g * g] for k in range(1, T + 1)])
            return np.sum((xs - spv) ** 2)
        def dloss(y, spv):
            gy = np.zeros(y.size)
            acc = np.zeros(g * g)
            for k in range(1, T + 1):
                o = g * g + (k - 1) * (g * g + S)
                gy[o:o + g * g] = 2 * (y[o:o + g * g] - spv)
                acc -= 2 * (y[o:o + g * g] - spv)
            return gy, acc
    s = mk()
    s.set_params(x0=x0, setpoint=sp, u_prev=up)
    assert s.solve()[0]["status"] == 0
    y = s.get_solution(0)
    gy, dsp_explicit = dloss(y, sp)
    dx0 = np.zeros(nx)
    dsp = np.zeros(nsp)
    s.sensitivity(0, gy, dx0, dsp)
    grad_x0, grad_sp = dx0, dsp + dsp_explicit
    hstep = 1e-5
    for _ in range(4):
        u = rng.normal(size=nx + nsp)
        u /= np.linalg.norm(u)
        ux, us = u[:nx], u[nx:]
        vals = []
        for sgn in (+1, -1):
            s2 = mk()
            s2.set_params(x0=x0 + sgn * hstep * ux, setpoint=sp + sgn * hstep * us, u_prev=up)
            assert s2.solve()[0]["status"] == 0
            vals.append(loss(s2.get_solution(0), sp + sgn * hstep * us))
        fd = (vals[0] - vals[1]) / (2 * hstep)
        ad = grad_x0 @ ux + grad_sp @ us
        assert abs(fd - ad) <= 1e-4 * max(1.0, abs(fd)), (model, fd, ad)


def test_adjoint_matches_oracle_finite_differences(P, oracle):
    """The oracle's gradient of the tracking loss w.r.t. x0 (central
    differences of oracle re-solves at tol 1e-12) equals the GPU adjoint."""
    N, T = 12, 20
    x0 = I.distillation_x0(12, 5, seed=6)
    sp = np.full(T, 0.8)
    idx = np.array([N + (k - 1) * (N + 1) for k in range(1, T + 1)])
    s = P.Solver(P.MODEL_DISTILLATION, [T], N=12, Nf=5, opts=P.options(tol=1e-12))
    s.set_params(x0=x0, setpoint=sp, u_prev=np.array([I.U_REF]))
    assert s.solve()[0]["status"] == 0
    y = s.get_solution(0)
    gy = np.zeros(y.size)
    gy[idx] = 2 * (y[idx] - sp)
    dx0 = np.zeros(N)
    s.sensitivity(0, gy, dx0, np.zeros(T))
    hstep = 1e-5
    for i in (0, 4, 11):
        vals = []
        for sgn in (+1, -1):
            xp = x0.copy()
            xp[i] += sgn * hstep
            prob = oracle.distillation(12, 5, T, xp, sp, I.U_REF)
            st, info, _ = oracle.solve(prob, tol=1e-12)
            assert info["status"] == 0
            vals.append(np.sum((st.y[idx] - sp) ** 2))
        fd = (vals[0] - vals[1]) / (2 * hstep)
        assert abs(fd - dx0[i]) <= 1e-4 * max(1.0, abs(fd)), (i, fd, dx0[i])


def test_autograd_function(P):
    import torch
    from paper_2606_04725_gb300.autograd import nmpc_solve
    T = 20
    dev = torch.device("cuda")
    s = P.Solver(P.MODEL_DISTILLATION, [T], N=12, Nf=5, opts=P.options(tol=1e-10))
    x0 = torch.tensor(I.distillation_x0(12, 5, seed=1), device=dev, requires_grad=True)
    sp = torch.full((T,), 0.8, dtype=torch.float64, device=dev, requires_grad=True)
    up = torch.tensor([I.U_REF], dtype=torch.float64, device=dev)
    y = nmpc_solve(s, x0, sp, up)
    idx = torch.tensor([12 + (k - 1) * 13 for k in range(1, T + 1)], device=dev)
    loss = ((y[idx] - sp) ** 2).sum()
    gx, gs = torch.autograd.grad(loss, (x0, sp))
    # same numbers through the C ABI directly
    gy = torch.zeros_like(y)
    gy[idx] = 2 * (y.detach()[idx] - sp.detach())
    dx0 = torch.empty(12, dtype=torch.float64, device=dev)
    dsp = torch.empty(T, dtype=torch.float64, device=dev)
    s.sensitivity(0, gy, dx0, dsp)
    torch.testing.assert_close(gx, dx0, rtol=1e-12, atol=1e-14)
    torch.testing.assert_close(gs, dsp - 2 * (y.detach()[idx] - sp.detach()), rtol=1e-12, atol=1e-14)


def test_envelope_theorem_in_a_batch(P, oracle):
    """In a batch of three columns with uneven horizons (the batch's solves run
    over front lists), the adjoint of each instance satisfies the envelope
    theorem on its own initial-condition rows, as the single column does."""
    hz = [14, 20, 26]
    s = P.Solver(P.MODEL_DISTILLATION, hz, N=12, Nf=5, opts=P.options(tol=1e-10))
    x0s = [I.distillation_x0(12, 5, seed=11 + i) for i in range(3)]
    sps = [np.full(T, 0.78 + 0.02 * i) for i, T in enumerate(hz)]
    for i in range(3):
        s.set_params(x0=x0s[i], setpoint=sps[i], u_prev=np.array([I.U_REF]), instance=i)
    assert all(info["status"] == 0 for info in s.solve())
    for i, T in enumerate(hz):
        y, du = s.get_solution(i, duals=True)
        prob = oracle.distillation(12, 5, T, x0s[i], sps[i], I.U_REF)
        _, grad_f, _, _ = oracle.evaluate(prob, y)
        dx0 = np.zeros(12)
        s.sensitivity(i, grad_f, dx0, np.zeros(T))
        lam0 = du["w_p"][:12] - du["w_m"][:12]
        np.testing.assert_allclose(dx0, -lam0, rtol=1e-5, atol=1e-7, err_msg=f"instance {i}")
