"""Pins of the oracle's model code (CPU only).

Derivatives are pinned by complex-step differentiation of the oracle's own
residual code (same source compiled for complex numbers), which is exact to
rounding.  The residuals themselves are pinned by conservation laws that hold
for any state and control, by the paper's steady state (Sec. 4.1, Table
distill-params) and by exactness of the 5-point stencil on quadratics.  The
paper's heated plate (Sec. 4.2) is pinned by the discrete energy balance
with its heat-loss term, by a uniform field that is stationary when the
boundary data agree, and by the region integral of its tracking cost.
"""
import numpy as np
import pytest

EPS = 1e-30


def _distill(O, N=6, Nf=3, T=3, **kw):
    rng = np.random.default_rng(11)
    return O.distillation(N, Nf, T, rng.uniform(0.1, 0.9, N), rng.uniform(0.3, 0.9, T), 2.2, dt=0.7, **kw)


def _plate(O, g=4, S=8, T=2):
    rng = np.random.default_rng(12)
    return O.plate(g, S, T, rng.uniform(0, 1, g * g), rng.uniform(0, 1, g * g), dt=0.9, cq=0.3)


def _pplate(O, n=6, T=3, **kw):
    """The paper's heated plate (Sec. 4.2) on a coarse grid, arbitrary data."""
    rng = np.random.default_rng(13)
    return O.paper_plate(n, T, rng.uniform(40, 70, (n - 2) ** 2), rng.uniform(50, 60, T), 3000.0, dt=0.08, **kw)


def _ddae(O, N=7, Nf=4, T=3, **kw):
    """The column with its algebraic variables (eq. distill-ocp as printed)."""
    rng = np.random.default_rng(14)
    return O.distillation_dae(N, Nf, T, rng.uniform(0.1, 0.9, N), rng.uniform(0.3, 0.9, T), 2.2, dt=0.7, **kw)


def _toy(O, T=4):
    return O.toy(T, 1.0, np.sin(np.arange(1, T + 1) * 0.7), dt=0.7)


def _interior_point(prob, seed=5):
    rng = np.random.default_rng(seed)
    yL, yU = prob.bounds()
    lo = np.where(np.isfinite(yL), yL, -1.0)
    hi = np.where(np.isfinite(yU), yU, 2.0)
    return lo + (hi - lo) * rng.uniform(0.1, 0.9, prob.n)


def _models(O):
    return [("distill", _distill(O)), ("distill_paper_holdups", _distill(O, Ac=0.5, At=0.25, Ar=1.0)),
            ("distill_paper_cost", _distill(O, Ac=0.5, At=0.25, Ar=1.0, wdu=0.0, wu=0.1, ubar=2.51459)),
            ("plate", _plate(O)), ("paper_plate", _pplate(O)), ("distill_dae", _ddae(O)),
            ("distill_dae_paper", _ddae(O, Ac=0.5, At=0.25, Ar=1.0, wdu=0.0, wu=0.1, ubar=2.51459)), ("toy", _toy(O))]


def test_jacobian_complex_step(oracle):
    O = oracle
    for name, p in _models(O):
        y = _interior_point(p)
        J = O.jacobian_dense(p, y)
        for j in range(p.n):
            im = np.zeros(p.n)
            im[j] = EPS
            _, _, h, _ = O.evaluate_complex(p, y, im)
            col = h.imag / EPS
            np.testing.assert_allclose(J[:, j], col, rtol=1e-13, atol=1e-13, err_msg=f"{name} col {j}")


def test_gradient_complex_step(oracle):
    O = oracle
    for name, p in _models(O):
        y = _interior_point(p)
        _, g, _, _ = O.evaluate(p, y)
        for j in range(p.n):
            im = np.zeros(p.n)
            im[j] = EPS
            f, _, _, _ = O.evaluate_complex(p, y, im)
            assert abs(g[j] - f.imag / EPS) <= 1e-13 * max(1.0, abs(g[j])), (name, j)


def test_hessian_complex_step(oracle):
    """W = d/dy (grad f + H^T lam), differentiated through the complex code."""
    O = oracle
    for name, p in _models(O):
        y = _interior_point(p)
        lam = np.random.default_rng(3).normal(size=p.m)
        W = O.hessian_dense(p, y, lam)
        nnz = p.jac_nnz()
        _, _, _, (rp, ci, _) = O.evaluate(p, y)
        rows = np.repeat(np.arange(p.m), np.diff(rp))
        for j in range(p.n):
            im = np.zeros(p.n)
            im[j] = EPS
            _, g, _, Hv = O.evaluate_complex(p, y, im)
            assert Hv.size == nnz
            grad_l = g.imag / EPS + np.bincount(ci, weights=(Hv.imag / EPS) * lam[rows], minlength=p.n)
            np.testing.assert_allclose(W[:, j], grad_l, rtol=1e-12, atol=1e-12, err_msg=f"{name} col {j}")


def _rhs_from_h(p, y, k):
    """f(x_{k+1}, u_{k+1}) recovered from the backward-Euler row of stage k."""
    _, _, h, _ = __import__("oracle").evaluate(p, y)
    xk = y[p.off_x(k):p.off_x(k) + p.nx]
    xn = y[p.off_x(k + 1):p.off_x(k + 1) + p.nx]
    hk = h[p.nx * (k + 1):p.nx * (k + 2)]
    return (xn - xk - hk) / p._p.dt


@pytest.mark.parametrize("holdups", [(1.0, 1.0, 1.0), (0.5, 0.25, 1.0)])
def test_distillation_component_balance(oracle, holdups):
    """Summed over the column, internal flows cancel: for every x and u,
    A_c f_1 + A_t sum f_2..f_{N-1} + A_r f_N = F x_F - D x_1 - (F - D) x_N.
    A dropped term, a wrong sign, a shifted tray index or an overlapping
    stripping/reboiler range breaks this identity."""
    Ac, At, Ar = holdups
    for N, Nf in [(12, 5), (34, 17), (6, 2), (5, 4)]:
        p = oracle.distillation(N, Nf, 2, np.zeros(N), np.zeros(2), 1.0, Ac=Ac, At=At, Ar=Ar)
        rng = np.random.default_rng(N)
        for _ in range(5):
            y = rng.uniform(0, 1, p.n)
            y[p.off_u(1)] = rng.uniform(1, 5)
            y[p.off_u(2)] = rng.uniform(1, 5)
            f = _rhs_from_h(p, y, 0)
            A = np.full(N, At)
            A[0], A[-1] = Ac, Ar
            x = y[p.off_x(1):p.off_x(1) + N]
            lhs = np.dot(A, f)
            rhs = 0.4 * 0.5 - 0.2 * x[0] - (0.4 - 0.2) * x[-1]
            assert abs(lhs - rhs) < 1e-14, (N, Nf, lhs, rhs)


def test_distillation_steady_state_matches_paper(oracle):
    """Table distill-params: xbar = 0.8958 at ubar = 2.51459 for N = 32,
    N_f = 17.  The printed value has four digits and our reading of the
    stripping range gives 0.89551, so the pin holds at 3e-4."""
    p = oracle.distillation(32, 17, 1, np.zeros(32), np.zeros(1), 2.51459)
    x = oracle.steady_state(p, 2.51459)
    assert abs(x[0] - 0.8958) < 3e-4
    assert np.all((x > 0) & (x < 1))
    assert np.all(np.diff(x) < 0)  # light component decreases down the column
    # steady state: the stage residual of a constant trajectory vanishes
    q = oracle.distillation(32, 17, 1, x, np.zeros(1), 2.51459)
    y = np.concatenate([x, x, [2.51459]])
    _, _, h, _ = oracle.evaluate(q, y)
    assert np.max(np.abs(h)) < 1e-14


def test_plate_energy_balance(oracle):
    """Interior fluxes cancel and insulated faces carry none: the total heat
    rate is h^2 sum_c f_c = (4/S) c_q sum_s v_s (each segment spans 4/S)."""
    for g, S in [(4, 4), (4, 8), (8, 16), (6, 12)]:
        p = oracle.plate(g, S, 1, np.zeros(g * g), np.zeros(g * g), dt=0.5, cq=0.3)
        rng = np.random.default_rng(g * S)
        y = rng.uniform(-1, 1, p.n)
        f = _rhs_from_h(p, y, 0)
        v = y[p.off_u(1):p.off_u(1) + S]
        assert abs(np.sum(f) / g**2 - 4.0 / S * 0.3 * v.sum()) < 1e-12


def test_plate_stencil_exact_on_quadratics(oracle):
    """The 5-point Laplacian is exact on quadratics at interior cells and
    symmetric (the operator is self-adjoint with zero-flux boundaries)."""
    g = 8
    p = oracle.plate(g, 4, 1, np.zeros(g * g), np.zeros(g * g), dt=0.5, kappa=0.01)
    h = 1.0 / g
    ii, jj = np.meshgrid(np.arange(g), np.arange(g))
    X, Y = (ii.ravel() + 0.5) * h, (jj.ravel() + 0.5) * h
    y = np.zeros(p.n)
    y[p.off_x(1):p.off_x(1) + g * g] = X**2 + 3 * Y**2 + X * Y + 2 * X
    f = _rhs_from_h(p, y, 0)
    interior = (ii.ravel() > 0) & (ii.ravel() < g - 1) & (jj.ravel() > 0) & (jj.ravel() < g - 1)
    np.testing.assert_allclose(f[interior], 0.01 * (2 + 6), rtol=1e-10)
    J = oracle.jacobian_dense(p, np.zeros(p.n))
    A = J[g * g:, p.off_x(1):p.off_x(1) + g * g]
    np.testing.assert_allclose(A, A.T, atol=1e-14)
    assert np.allclose(A.sum(axis=1), 1.0)  # (I - dt kappa Lap) preserves constants


def test_objective_closed_forms(oracle):
    """Tracking cost vanishes on the setpoint; a constant offset c gives
    T dt c^2; a control ramp gives the Delta-u penalty in closed form."""
    N, T = 5, 4
    sp = np.array([0.2, 0.4, 0.6, 0.8])
    p = oracle.distillation(N, 2, T, np.zeros(N), sp, uprev=1.5, dt=0.5)
    y = np.zeros(p.n)
    for k in range(1, T + 1):
        y[p.off_x(k)] = sp[k - 1] + 0.1
        y[p.off_u(k)] = 1.5 + 0.25 * k
    f, _, _, _ = oracle.evaluate(p, y)
    assert abs(f - (T * 0.5 * 0.01 + T * 0.01 * 0.25**2)) < 1e-15
    g = 4
    tgt = np.linspace(0, 1, g * g)
    q = oracle.plate(g, 4, 2, np.zeros(g * g), tgt, dt=0.5)
    y = np.zeros(q.n)
    for k in (1, 2):
        y[q.off_x(k):q.off_x(k) + g * g] = tgt + 0.5
        y[q.off_u(k):q.off_u(k) + 4] = 2.0
    f, _, _, _ = oracle.evaluate(q, y)
    assert abs(f - (2 * 0.5 * 0.25 + 2 * 1e-3 * 0.5 * 4 * 4.0)) < 1e-14


def test_paper_control_cost_is_the_integral_for_a_constant_control(oracle):
    """Eq. (distill-ocp) integrates 0.1 (u - ubar)^2 over the prediction
    horizon: for a constant control c and states on the setpoint the cost is
    0.1 (c - ubar)^2 t_p, with t_p = T dt (Sec. 4.1: t_p = 180 s, dt = 2 s)."""
    N, T, dt, ubar = 5, 90, 2.0, 2.51459
    sp = np.linspace(0.5, 0.9, T)
    p = oracle.distillation(N, 2, T, np.zeros(N), sp, uprev=3.0, dt=dt, wdu=0.0, wu=0.1, ubar=ubar)
    for c in (1.0, 2.51459, 4.2):
        y = np.zeros(p.n)
        for k in range(1, T + 1):
            y[p.off_x(k)] = sp[k - 1]
            y[p.off_u(k)] = c
        f, _, _, _ = oracle.evaluate(p, y)
        assert abs(f - 0.1 * (c - ubar) ** 2 * 180.0) < 1e-12 * max(1.0, f), (c, f)


def _pplate_f(O, p, x, Q):
    """f_c(x, Q) of every interior node, from the residual of one step with
    x_1 = x, x_0 = 0: the step rows are s (x - 0 - dt f), scaled by
    s = 1 / (1 + 4 dt alpha / h^2) to a unit diagonal."""
    y = np.zeros(p.n)
    y[p.off_x(1):p.off_x(1) + p.nx] = x
    y[p.off_u(1)] = Q
    p.set_params(x0=np.zeros(p.nx))
    _, _, h, _ = O.evaluate(p, y)
    hh = 2.0 / (p._p.g - 1)
    s = 1.0 / (1.0 + 4.0 * p._p.dt * p._p.kappa / hh ** 2)
    return (x - h[p.nx:2 * p.nx] / s) / p._p.dt


def test_paper_plate_step_rows_have_a_unit_diagonal(oracle):
    """The scaled step row of node c has coefficient 1 on T_{k+1,c} and -s on
    T_{k,c}, s = 1 / (1 + 4 dt alpha / h^2)."""
    O = oracle
    p = _pplate(O, n=7, T=2)
    y = _interior_point(p)
    J = O.jacobian_dense(p, y)
    hh = 2.0 / 6
    s = 1.0 / (1.0 + 4.0 * 0.08 * 230.0 / hh ** 2)
    for c in range(p.nx):
        r = p.nx + p.nx + c  # step 1 -> 2
        assert abs(J[r, p.off_x(2) + c] - 1.0) <= 1e-14
        assert abs(J[r, p.off_x(1) + c] + s) <= 1e-16


def test_paper_plate_energy_balance(oracle):
    """Discrete divergence theorem of the 5-point Laplacian: summed over the
    interior nodes the interior edges cancel, so sum_c f_c = alpha (sum over
    the edges to the boundary of (T_boundary - T_c) / h^2 - 5 q_loss^2 nx),
    with the boundary data of eq. (pde-ocp): 4.1 Q^(1/3) at x1 = -1, Q^(1/2)
    at x2 = -1, T_b at x1 = 1 and x2 = 1."""
    O = oracle
    rng = np.random.default_rng(21)
    for n in (5, 9, 21):
        p = O.paper_plate(n, 1, np.zeros((n - 2) ** 2), np.zeros(1), 100.0, Tb=47.0, qloss=3.0)
        m = n - 2
        h = 2.0 / (n - 1)
        for _ in range(3):
            x = rng.uniform(-100, 300, m * m)
            Q = rng.uniform(50, 1e5)
            f = _pplate_f(O, p, x, Q)
            T = x.reshape(m, m)  # T[j, i] for node (i + 1, j + 1)
            edges = (4.1 * np.cbrt(Q) - T[:, 0]).sum() + (47.0 - T[:, -1]).sum() \
                + (np.sqrt(Q) - T[0, :]).sum() + (47.0 - T[-1, :]).sum()
            want = 230.0 * (edges / h ** 2 - 5.0 * 3.0 ** 2 * m * m)
            assert abs(f.sum() - want) <= 1e-11 * max(abs(want), 230.0 * np.abs(x).sum() / h ** 2), (n, f.sum(), want)


def test_paper_plate_uniform_field_is_stationary_when_boundaries_agree(oracle):
    """Without heat loss, a uniform field equal to all four boundary values is
    stationary: 4.1 Q^(1/3) = Q^(1/2) at Q = 4.1^6, where both equal 4.1^3,
    and T_b is set to that value."""
    O = oracle
    Q = 4.1 ** 6
    Tb = 4.1 ** 3
    for n in (4, 7, 12):
        p = O.paper_plate(n, 1, np.zeros((n - 2) ** 2), np.zeros(1), 100.0, Tb=Tb, qloss=0.0)
        f = _pplate_f(O, p, np.full((n - 2) ** 2, Tb), Q)
        assert np.max(np.abs(f)) <= 1e-9 * 230.0 * Tb * (n - 1) ** 2, (n, np.max(np.abs(f)))
        # and a perturbation of one boundary breaks it only next to that boundary
        f2 = _pplate_f(O, p, np.full((n - 2) ** 2, Tb), Q * 1.1)
        m = n - 2
        F = f2.reshape(m, m)
        assert np.all(F[1:, 1:] == 0) or m == 1
        assert np.all(F[:, 0] > 0) and np.all(F[0, :] > 0)
        # the x1 = -1 side (node column i = 1) carries 4.1 Q^(1/3), the x2 = -1
        # side (node row j = 1) Q^(1/2): they move by different amounts
        a = 230.0 * (n - 1) ** 2 / 4.0
        left, bottom = a * (4.1 * np.cbrt(Q * 1.1) - Tb), a * (np.sqrt(Q * 1.1) - Tb)
        assert np.allclose(F[1:, 0], left, rtol=1e-9) and np.allclose(F[0, 1:], bottom, rtol=1e-9)
        assert np.isclose(F[0, 0], left + bottom, rtol=1e-9) and not np.isclose(left, bottom, rtol=1e-3)


def test_paper_plate_tracking_cost_is_the_region_integral(oracle):
    """The stage cost's region term integrates a constant deviation d over
    [-0.5, 0.5]^2 exactly (area 1): with x_k = sp_k + d on every interior node
    and Q_k = Q, f = T dt (d^2 + rho Q^2), for grids whose nodes fall on the
    region's edges (n - 1 a multiple of 4)."""
    O = oracle
    for n in (5, 9, 21):
        T = 3
        sp = np.array([58.0, 55.0, 63.0])
        p = O.paper_plate(n, T, np.zeros((n - 2) ** 2), sp, 100.0)
        d, Q = 1.7, 2500.0
        y = np.zeros(p.n)
        for k in range(1, T + 1):
            y[p.off_x(k):p.off_x(k) + p.nx] = sp[k - 1] + d
            y[p.off_u(k)] = Q
        f, _, _, _ = O.evaluate(p, y)
        want = T * 0.08 * (d * d + 1e-8 * Q * Q)
        assert abs(f - want) <= 1e-12 * want, (n, f, want)


def test_jacobian_pattern_size_and_row_layout(oracle):
    """The CSR Jacobian fills exactly or_jac_nnz entries, rows ascending in
    columns; the DAE column has 2N + 3 rows per step (N balances, N
    equilibria, 3 flow equations)."""
    O = oracle
    for name, p in _models(O):
        y = _interior_point(p)
        _, _, _, (rp, ci, _) = O.evaluate(p, y)
        assert rp[-1] == p.jac_nnz() and rp.size == p.m + 1, name
        for r in range(p.m):
            assert np.all(np.diff(ci[rp[r]:rp[r + 1]]) > 0), (name, r)
    p = _ddae(O, N=7, T=3)
    assert p.m == 7 + 3 * (2 * 7 + 3) and p.n == 7 + 3 * (7 + 7 + 4)


def test_distillation_dae_residual_vanishes_on_the_substituted_trajectory(oracle):
    """Given any x, u trajectory, setting y = vle(x), L = u D, V = L + D,
    S = L + F makes the algebraic rows zero and the balance rows equal to the
    substituted model's rows (eq. distill-ocp with y, L, V, S eliminated)."""
    O = oracle
    N, Nf, T = 9, 5, 4
    rng = np.random.default_rng(31)
    x0 = rng.uniform(0.1, 0.9, N)
    sp = rng.uniform(0.3, 0.9, T)
    pd = O.distillation_dae(N, Nf, T, x0, sp, 2.2, dt=0.7, Ac=0.5, At=0.25)
    ps = O.distillation(N, Nf, T, x0, sp, 2.2, dt=0.7, Ac=0.5, At=0.25)
    ys = rng.uniform(0.1, 0.9, ps.n)
    for k in range(1, T + 1):
        ys[ps.off_u(k)] = rng.uniform(1, 5)
    yd = np.zeros(pd.n)
    yd[:N] = ys[:N]
    a = 1.6
    for k in range(1, T + 1):
        x = ys[ps.off_x(k):ps.off_x(k) + N]
        u = ys[ps.off_u(k)]
        yd[pd.off_x(k):pd.off_x(k) + N] = x
        o = pd.off_u(k)
        yd[o:o + N] = a * x / (1 + (a - 1) * x)
        yd[o + N:o + N + 4] = [u, u * 0.2, u * 0.2 + 0.2, u * 0.2 + 0.4]
    fd, _, hd, _ = O.evaluate(pd, yd)
    fs, _, hs, _ = O.evaluate(ps, ys)
    assert abs(fd - fs) <= 1e-13 * max(1.0, abs(fs))
    nr = 2 * N + 3
    for k in range(T):
        blk = hd[N + nr * k:N + nr * (k + 1)]
        np.testing.assert_allclose(blk[:N], hs[N * (k + 1):N * (k + 2)], rtol=1e-13, atol=1e-14)
        assert np.max(np.abs(blk[N:])) <= 1e-15
