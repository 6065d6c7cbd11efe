"""Pins of the oracle's interior-point method (CPU only).

* Optimality error: E_mu and E_0 equal the norms of the lifted KKT residual
  built from the dense Jacobian.
* Line search: each step of cold solves against the Newton direction, the
  fraction to the boundary and the filter tests with recomputed merits.
* Newton step: the condensed Lifted-KKT solve plus recovery (eqs.
  liftedkkt-pd, cholesky-lower/upper/delta, infiniteOCP-augmented) equals the
  solution of the full primal-dual Newton system of the barrier KKT
  conditions, assembled here densely and solved with numpy.
* Sylvester relation (eq. infiniteOCP-inertia): Cholesky of K_c succeeds
  exactly when K_aug has inertia (n + m_g, 0, m_g).
* Converged solutions: linear-quadratic cases against the exact solution of
  the equality-constrained QP; tiny box-constrained QPs against brute-force
  active-set enumeration; nonlinear cases by finite-difference stationarity.
"""
import itertools

import numpy as np
import pytest

GAMMA = 1e-9


def _random_state(O, p, seed):
    rng = np.random.default_rng(seed)
    st = O.State(p.n, p.m)
    yL, yU = p.bounds()
    lo = np.where(np.isfinite(yL), yL, -1.0)
    hi = np.where(np.isfinite(yU), yU, 2.0)
    st.y[:] = lo + (hi - lo) * rng.uniform(0.2, 0.8, p.n)
    st.zL[:] = np.where(np.isfinite(yL), rng.uniform(0.1, 2, p.n), 0.0)
    st.zU[:] = np.where(np.isfinite(yU), rng.uniform(0.1, 2, p.n), 0.0)
    for k in ("s_p", "s_m", "b_p", "b_m"):
        getattr(st, k)[:] = rng.uniform(0.1, 2, p.m)
    for k in ("w_p", "w_m"):
        getattr(st, k)[:] = rng.uniform(-1, 2, p.m)
    return st


def _full_newton(O, p, st, mu, dw):
    """Dense primal-dual Newton system of the lifted barrier KKT conditions
    in (dy, ds+, ds-, dw+, dw-, db+, db-, dzL, dzU)."""
    n, m = p.n, p.m
    yL, yU = p.bounds()
    L_idx = np.nonzero(np.isfinite(yL))[0]
    U_idx = np.nonzero(np.isfinite(yU))[0]
    _, g, h, _ = O.evaluate(p, st.y)
    H = O.jacobian_dense(p, st.y)
    W = O.hessian_dense(p, st.y, st.w_p - st.w_m) + dw * np.eye(n)
    nL, nU = len(L_idx), len(U_idx)
    sizes = [n, m, m, m, m, m, m, nL, nU]
    off = np.cumsum([0] + sizes)
    N = off[-1]
    J = np.zeros((N, N))
    F = np.zeros(N)
    EL = np.zeros((n, nL)); EL[L_idx, np.arange(nL)] = 1
    EU = np.zeros((n, nU)); EU[U_idx, np.arange(nU)] = 1
    I = np.eye(m)
    zL, zU = st.zL[L_idx], st.zU[U_idx]
    B = lambda r, c, M: J.__setitem__((slice(off[r], off[r + 1]), slice(off[c], off[c + 1])), M)
    # stationarity in y
    B(0, 0, W); B(0, 3, H.T); B(0, 4, -H.T); B(0, 7, -EL); B(0, 8, EU)
    F[off[0]:off[1]] = g + H.T @ (st.w_p - st.w_m) - EL @ zL + EU @ zU
    # stationarity in s+, s-
    B(1, 3, I); B(1, 5, -I); F[off[1]:off[2]] = st.w_p - st.b_p
    B(2, 4, I); B(2, 6, -I); F[off[2]:off[3]] = st.w_m - st.b_m
    # lifted constraints
    B(3, 0, H); B(3, 1, I); F[off[3]:off[4]] = h - GAMMA + st.s_p
    B(4, 0, -H); B(4, 2, I); F[off[4]:off[5]] = -h - GAMMA + st.s_m
    # complementarity
    B(5, 1, np.diag(st.b_p)); B(5, 5, np.diag(st.s_p)); F[off[5]:off[6]] = st.s_p * st.b_p - mu
    B(6, 2, np.diag(st.b_m)); B(6, 6, np.diag(st.s_m)); F[off[6]:off[7]] = st.s_m * st.b_m - mu
    gl = st.y[L_idx] - yL[L_idx]
    gu = yU[U_idx] - st.y[U_idx]
    B(7, 0, np.diag(zL) @ EL.T); B(7, 7, np.diag(gl)); F[off[7]:off[8]] = gl * zL - mu
    B(8, 0, -np.diag(zU) @ EU.T); B(8, 8, np.diag(gu)); F[off[8]:off[9]] = gu * zU - mu
    d = np.linalg.solve(J, -F)
    parts = [d[off[i]:off[i + 1]] for i in range(9)]
    dzL = np.zeros(n); dzL[L_idx] = parts[7]
    dzU = np.zeros(n); dzU[U_idx] = parts[8]
    return dict(y=parts[0], s_p=parts[1], s_m=parts[2], w_p=parts[3], w_m=parts[4],
                b_p=parts[5], b_m=parts[6], zL=dzL, zU=dzU)


def _small_problem(O, model):
    if model == "distill":
        return O.distillation(5, 3, 3, np.full(5, 0.5), np.full(3, 0.6), 2.0, dt=0.5)
    if model == "plate":
        return O.plate(4, 8, 2, np.zeros(16), np.full(16, 0.3), dt=0.5)
    return O.toy(4, 1.0, np.sin(np.arange(4)), dt=0.7)


def _residual_norms(O, p, st, mu):
    """Max-norms of the lifted barrier KKT conditions at st, from the dense
    Jacobian and the evaluated gradient and constraints: stationarity in y and
    in the slacks (dual), the lifted constraints (primal), complementarity;
    and the multiplier sums of the scaling of W&B eq. (5)."""
    yL, yU = p.bounds()
    L, U = np.isfinite(yL), np.isfinite(yU)
    _, g, h, _ = O.evaluate(p, st.y)
    H = O.jacobian_dense(p, st.y)
    ry = g + H.T @ (st.w_p - st.w_m) - np.where(L, st.zL, 0.0) + np.where(U, st.zU, 0.0)
    dual = max(np.abs(ry).max(), np.abs(st.w_p - st.b_p).max(), np.abs(st.w_m - st.b_m).max())
    prim = max(np.abs(h - GAMMA + st.s_p).max(), np.abs(-h - GAMMA + st.s_m).max())
    comp = max(np.abs(st.s_p * st.b_p - mu).max(), np.abs(st.s_m * st.b_m - mu).max(),
               np.abs((st.y - yL)[L] * st.zL[L] - mu).max(initial=0.0),
               np.abs((yU - st.y)[U] * st.zU[U] - mu).max(initial=0.0))
    sum_w = np.abs(st.w_p).sum() + np.abs(st.w_m).sum()
    sum_z = np.abs(st.zL[L]).sum() + np.abs(st.zU[U]).sum() + np.abs(st.b_p).sum() + np.abs(st.b_m).sum()
    n_z = L.sum() + U.sum() + 2 * p.m
    return dual, prim, comp, sum_w, sum_z, n_z


@pytest.mark.parametrize("model", ["distill", "plate", "toy"])
def test_optimality_error_is_the_kkt_residual(oracle, model):
    """The oracle's optimality error (the termination test of eqs.
    infiniteOCP-innerTol/outerTol, W&B eq. (5)) against the lifted KKT
    residual built from the dense Jacobian: unscaled, it is the largest of the
    dual, primal and complementarity residuals; scaled, the dual part is
    divided by s_d and the complementarity by s_c, each max(100, mean
    multiplier)/100.  States with small multipliers (s_d = s_c = 1, E scaled =
    unscaled) and with multipliers 1e3 times larger (scaling active)."""
    O = oracle
    p = _small_problem(O, model)
    for seed, mu, big in [(1, 0.0, 1.0), (2, 0.05, 1.0), (3, 0.0, 1e3), (4, 0.3, 1e3)]:
        st = _random_state(O, p, seed)
        for k in ("zL", "zU", "w_p", "w_m", "b_p", "b_m"):
            getattr(st, k)[:] *= big
        dual, prim, comp, sum_w, sum_z, n_z = _residual_norms(O, p, st, mu)
        es, eu = O.kkt_error(p, st, mu=mu, gamma=GAMMA)
        assert eu == pytest.approx(max(dual, prim, comp), rel=1e-12), (model, seed)
        sd = max(100.0, (sum_w + sum_z) / (2 * p.m + n_z)) / 100.0
        sc = max(100.0, sum_z / n_z) / 100.0
        assert es == pytest.approx(max(dual / sd, prim, comp / sc), rel=1e-12), (model, seed)
        if big == 1.0:
            assert es == eu
        else:
            assert sd > 1.0 and sc > 1.0


@pytest.mark.parametrize("model", ["distill", "plate", "toy"])
def test_newton_step_equals_uncondensed_solve(oracle, model):
    O = oracle
    p = _small_problem(O, model)
    for seed, mu, dw in [(1, 0.1, 0.0), (2, 1e-3, 0.5), (3, 1.0, 2.0)]:
        st = _random_state(O, p, seed)
        rc, d = O.newton_step(p, st, mu, dw, gamma=GAMMA)
        if rc != 0:
            continue  # K_c not PD at this point: covered by the Sylvester test
        ref = _full_newton(O, p, st, mu, dw)
        for k, v in ref.items():
            np.testing.assert_allclose(getattr(d, k), v, rtol=1e-8, atol=1e-9 * (1 + np.abs(v).max()),
                                       err_msg=f"{model} seed {seed} {k}")


def test_sylvester_inertia_relation(oracle):
    """eq. infiniteOCP-inertia for the lifted system (m_h = 0, m_g = 2m):
    inertia(K_aug) = (n + 2m, 0, 2m)  <=>  K_c positive definite, where
    K_aug = [[W + Sigma, 0, G^T], [0, Q, I], [G, I, 0]], G = [H; -H]."""
    O = oracle
    p = O.toy(5, 1.0, np.sin(np.arange(5)), dt=0.8)
    agree = {True: 0, False: 0}
    for seed in range(40):
        st = _random_state(O, p, seed)
        rng = np.random.default_rng(100 + seed)
        st.w_p[:] = rng.uniform(-6, 6, p.m)  # large multipliers make W indefinite
        dw = float(rng.choice([-3.0, -1.0, 0.0, 1.0, 5.0, 20.0]))
        n, m = p.n, p.m
        yL, yU = p.bounds()
        H = O.jacobian_dense(p, st.y)
        W = O.hessian_dense(p, st.y, st.w_p - st.w_m) + dw * np.eye(n)
        sig = np.where(np.isfinite(yL), st.zL / (st.y - np.where(np.isfinite(yL), yL, 0)), 0.0)
        sig += np.where(np.isfinite(yU), st.zU / (np.where(np.isfinite(yU), yU, 0) - st.y), 0.0)
        Q = np.concatenate([st.b_p / st.s_p, st.b_m / st.s_m])
        G = np.vstack([H, -H])
        Kaug = np.block([[W + np.diag(sig), np.zeros((n, 2 * m)), G.T],
                         [np.zeros((2 * m, n)), np.diag(Q), np.eye(2 * m)],
                         [G, np.eye(2 * m), np.zeros((2 * m, 2 * m))]])
        ev = np.linalg.eigvalsh(Kaug)
        right_inertia = (np.sum(ev > 1e-10) == n + 2 * m) and (np.sum(ev < -1e-10) == 2 * m)
        Kc = W + np.diag(sig) + G.T @ np.diag(Q) @ G
        pd = bool(np.all(np.linalg.eigvalsh(Kc) > 0))
        assert right_inertia == pd
        rc, _ = O.newton_step(p, st, 0.1, dw, gamma=GAMMA)
        assert (rc == 0) == pd
        agree[pd] += 1
    assert agree[True] > 3 and agree[False] > 3  # both branches exercised


def _quadratic_model(O, p):
    """f = 1/2 y'Qy + c'y + f0 and h = A y + h0 (exact for linear-quadratic
    models), read off the oracle's gradient and constraint values."""
    n = p.n
    f0, c, h0, _ = O.evaluate(p, np.zeros(n))
    Q = np.zeros((n, n))
    A = O.jacobian_dense(p, np.zeros(n))
    for j in range(n):
        e = np.zeros(n); e[j] = 1.0
        Q[:, j] = O.evaluate(p, e)[1] - c
    return Q, c, A, h0


def test_lq_plate_matches_equality_qp(oracle):
    """With bounds far away the plate OCP is an equality-constrained QP whose
    exact solution solves [[Q, A^T], [A, 0]] [y; lam] = [-c; -h0]."""
    O = oracle
    g, S, T = 3, 4, 4
    rng = np.random.default_rng(4)
    p = O.plate(g, S, T, rng.uniform(0, 0.5, g * g), rng.uniform(0, 1, g * g), dt=0.5,
                xhi=1e3, ulo=-1e3, uhi=1e3, cq=0.5, rho_u=1e-2)
    Q, c, A, h0 = _quadratic_model(O, p)
    n, m = p.n, p.m
    K = np.block([[Q, A.T], [A, np.zeros((m, m))]])
    sol = np.linalg.solve(K, np.concatenate([-c, -h0]))
    st, info, _ = O.solve(p)
    assert info["status"] == 0
    y_ref = sol[:n]
    assert np.max(np.abs(st.y - y_ref)) / max(1.0, np.max(np.abs(y_ref))) < 1e-6
    lam_ref = sol[n:]
    np.testing.assert_allclose(st.w_p - st.w_m, lam_ref, rtol=1e-4, atol=1e-5)


def test_box_qp_matches_bruteforce_active_set(oracle):
    """Tiny plate QP (g=2, S=4, T=1) with state upper bounds and control
    boxes: enumerate every active set (2^4 * 3^4), keep the one whose
    equality-QP solution is primal feasible with correctly signed bound
    multipliers; it is the unique optimum of the strictly convex QP."""
    O = oracle
    g, S, T = 2, 4, 1
    tgt = np.array([1.0, 0.2, 1.0, 0.0])
    p = O.plate(g, S, T, np.zeros(4), tgt, dt=1.0, xhi=0.6, cq=0.4, rho_u=0.05)
    Q, c, A, h0 = _quadratic_model(O, p)
    n, m = p.n, p.m
    yL, yU = p.bounds()
    xs = list(range(p.off_x(1), p.off_x(1) + 4))
    us = list(range(p.off_u(1), p.off_u(1) + 4))
    found = []
    for xa in itertools.product([0, 1], repeat=4):
        for ua in itertools.product([0, 1, 2], repeat=4):
            act = [(i, yU[i], +1) for i, a in zip(xs, xa) if a] + \
                  [(i, yL[i], -1) for i, a in zip(us, ua) if a == 1] + \
                  [(i, yU[i], +1) for i, a in zip(us, ua) if a == 2]
            E = np.zeros((len(act), n))
            for r, (i, _, _) in enumerate(act):
                E[r, i] = 1.0
            Aall = np.vstack([A, E])
            b = np.concatenate([-h0, [v for _, v, _ in act]])
            k = Aall.shape[0]
            K = np.block([[Q, Aall.T], [Aall, np.zeros((k, k))]])
            try:
                sol = np.linalg.solve(K, np.concatenate([-c, b]))
            except np.linalg.LinAlgError:
                continue
            y, nu = sol[:n], sol[n + m:]
            feas = np.all(y <= yU + 1e-12) and np.all(y >= yL - 1e-12)
            signs = all(s * v >= -1e-12 for (_, _, s), v in zip(act, nu))
            if feas and signs:
                found.append((y, len(act)))
    assert len(found) == 1
    y_ref, nact = found[0]
    assert 0 < nact < 8  # a genuine mix of active and inactive bounds
    st, info, _ = O.solve(p)
    assert info["status"] == 0
    assert np.max(np.abs(st.y - y_ref)) < 1e-6


def _fd_stationarity(O, p, st, step=1e-6):
    """grad f + H^T lam - zL + zU with grad f and H from central differences
    of the oracle's objective and constraint values only."""
    n = p.n
    lam = st.w_p - st.w_m
    r = -st.zL + st.zU
    for j in range(n):
        e = np.zeros(n); e[j] = step
        fp, _, hp, _ = O.evaluate(p, st.y + e)
        fm, _, hm, _ = O.evaluate(p, st.y - e)
        r[j] += (fp - fm) / (2 * step) + np.dot((hp - hm) / (2 * step), lam)
    return r


def test_toy_code_listing_problem_converges(oracle):
    """The code listing's problem: dy/dt = 4 sin u - y^3, y(0) = 1, 1 <= u <= 3,
    y >= 0, 15 supports on [0, 10] (14 intervals), setpoint sin(t + t_k)."""
    O = oracle
    T = 14
    dt = 10.0 / T
    t = dt * np.arange(1, T + 1)
    p = O.toy(T, 1.0, np.sin(t), dt=dt)
    st, info, _ = O.solve(p)
    assert info["status"] == 0 and info["E0_scaled"] <= 1e-8
    r = _fd_stationarity(O, p, st)
    assert np.max(np.abs(r)) < 1e-6
    _, _, h, _ = O.evaluate(p, st.y)
    assert np.max(np.abs(h)) <= 2 * GAMMA + 1e-8
    yL, yU = p.bounds()
    assert np.all(st.y >= yL) and np.all(st.y <= yU)
    # a second NMPC step from the measured state, warm-started
    y1 = st.y[p.off_x(1)]
    p.set_params(x0=[y1], sp=np.sin(t + 1.0))
    st, info, _ = O.solve(p, state=st, warm=True)
    assert info["status"] == 0


def test_distillation_closed_loop_small(oracle):
    """A small column (N=12, feed tray 5, T=20): a cold solve and four
    warm re-solves, each converged with FD-stationary primal-dual point."""
    O = oracle
    N, Nf, T = 12, 5, 20
    xs = np.loadtxt(__import__("os").path.join(__import__("os").path.dirname(__file__), "..",
                                                "paper_2606_04725_gb300", "data", "steady_state_N12_Nf5.txt"))
    rng = np.random.default_rng(1)
    x0 = np.clip(xs + rng.normal(0, 0.02, N), 0, 1)
    p = O.distillation(N, Nf, T, x0, np.full(T, 0.8), 2.51459)
    st, info, _ = O.solve(p)
    assert info["status"] == 0
    for k in range(4):
        p.set_params(x0=st.y[p.off_x(1):p.off_x(1) + N].copy(), uprev=st.y[p.off_u(1)])
        st, info, _ = O.solve(p, state=st, warm=True)
        assert info["status"] == 0 and info["iters"] < 20
    r = _fd_stationarity(O, p, st)
    assert np.max(np.abs(r)) < 1e-5


def test_paper_distillation_at_steady_state_stays_there(oracle):
    """The paper's column and cost (Sec. 4.1: N = 32, N_f = 17, holdups
    0.5 / 0.25 / 1.0, dt = 2, 90 intervals, cost (x_1 - xbar)^2 + 0.1 (u - ubar)^2).
    Started at the steady state of ubar with xbar its tray-1 value, the
    constant trajectory has zero cost and is feasible, so it is the optimum:
    the solver must return u = ubar and x = the steady state at every stage."""
    O = oracle
    N, Nf, T, ubar = 32, 17, 90, 2.51459
    kw = dict(dt=2.0, Ac=0.5, At=0.25, Ar=1.0, wdu=0.0, wu=0.1, ubar=ubar)
    xs = O.steady_state(O.distillation(N, Nf, 1, np.zeros(N), np.zeros(1), ubar), ubar)
    p = O.distillation(N, Nf, T, xs, np.full(T, xs[0]), ubar, **kw)
    st, info, _ = O.solve(p)
    assert info["status"] == 0
    u = np.array([st.y[p.off_u(k)] for k in range(1, T + 1)])
    X = np.stack([st.y[p.off_x(k):p.off_x(k) + N] for k in range(1, T + 1)])
    assert np.max(np.abs(u - ubar)) < 1e-6
    assert np.max(np.abs(X - xs)) < 1e-6


def _kc_extremes(O, p, st):
    """Smallest eigenvalue and largest diagonal entry of the condensed matrix
    K_c = W + Sigma_y + H^T (Q+ + Q-) H at st (eq. liftedkkt-pd), dense."""
    yL, yU = p.bounds()
    L, U = np.isfinite(yL), np.isfinite(yU)
    H = O.jacobian_dense(p, st.y)
    W = O.hessian_dense(p, st.y, st.w_p - st.w_m)
    sig = np.where(L, st.zL / np.where(L, st.y - yL, 1.0), 0.0) + np.where(U, st.zU / np.where(U, yU - st.y, 1.0), 0.0)
    Kc = W + np.diag(sig) + H.T @ np.diag(st.b_p / st.s_p + st.b_m / st.s_m) @ H
    return np.linalg.eigvalsh(Kc)[0], np.abs(np.diag(Kc)).max()


LS_PROBLEMS = {
    "distill": lambda O: O.distillation(5, 3, 6, np.full(5, 0.5), np.full(6, 0.6), 2.0, dt=0.5),
    "distill_long_dt": lambda O: O.distillation(5, 3, 6, np.full(5, 0.2), np.full(6, 0.9), 1.0, dt=2.0),
    "toy": lambda O: O.toy(14, 1.0, np.sin(np.arange(1, 15) * 10 / 14), dt=10 / 14),
    "toy_far": lambda O: O.toy(6, 2.0, np.full(6, -1.0), dt=0.5),
    "plate": lambda O: O.plate(4, 8, 3, np.zeros(16), np.full(16, 1.5), dt=0.5),
}


@pytest.mark.parametrize("name", list(LS_PROBLEMS))
def test_line_search_steps_follow_the_filter_method(oracle, name):
    """The oracle's steps against the filter line search of W&B Sec. 2 as the
    paper's step z += alpha delta (eq. infiniteOCP-lineSearch) is read:
    iterates after k and k + 1 iterations (max_iter = k, k + 1), the Newton
    direction at the k-th iterate (pinned above) and the merit functions
    recomputed here from the evaluated objective and constraints.  Per step:
    the traced phi_mu, theta and E_mu are those of the iterate, E_mu exceeds
    kappa_eps mu unless mu is at its floor (the barrier loop's exit); the dual
    step is the fraction-to-the-boundary step with tau = max(0.99, 1 - mu);
    the primal step is the primal fraction-to-the-boundary step halved
    (trials - 1) times; y, s and the constraint multipliers take the primal
    step, the bound and slack multipliers the dual step and then the kappa_Sigma
    safeguard; the accepted trial point is not blocked by the filter and
    decreases theta or phi_mu enough (or meets the Armijo condition); every
    longer trial step failed those tests, or was blocked by the filter, which is rebuilt here
    from the traced (theta, phi_mu) of the steps that were not Armijo steps
    and emptied at every barrier update; delta_w is the first value of the
    inertia-correction sequence (0, then 1e-4 or delta_last / 3, raised by 100
    until a first success, by 8 after) at which K_c + delta_w I, from dense
    matrices, is positive definite.  Every iteration of cold solves that
    backtrack (up to 9 trials), correct the inertia and lower mu."""
    O = oracle
    p = LS_PROBLEMS[name](O)
    yL, yU = p.bounds()
    L, U = np.isfinite(yL), np.isfinite(yU)
    gam, tol, ks = 1e-8, 1e-8, 1e10

    def merit(y, sp, sm, mu):
        f, g, h, _ = O.evaluate(p, y)
        lg = np.log((y - yL)[L]).sum() + np.log((yU - y)[U]).sum() + np.log(sp).sum() + np.log(sm).sum()
        return f - mu * lg, (np.abs(h - gam + sp) + np.abs(-h - gam + sm)).sum(), g

    def ftb(v, dv, tau):
        neg = dv < 0
        return min(1.0, np.min(tau * v[neg] / -dv[neg], initial=np.inf))

    def armijo_case(th, alpha, gphi, th_min):
        return th <= th_min and gphi < 0 and alpha * (-gphi) ** 2.3 > th ** 1.1

    def accepted(phi_t, th_t, phi, th, alpha, gphi, th_min):
        if armijo_case(th, alpha, gphi, th_min):
            return phi_t <= phi + 1e-4 * alpha * gphi
        return th_t <= (1 - 1e-5) * th or phi_t <= phi - 1e-5 * th

    def acceptable(phi_t, th_t, phi, th, alpha, gphi, filt):
        return (np.isfinite(phi_t) and th_t <= th_max and not any(th_t >= a and phi_t >= b for a, b in filt)
                and accepted(phi_t, th_t, phi, th, alpha, gphi, th_min))

    _, info, trace = O.solve(p)
    assert info["status"] == 0
    trace = np.asarray(trace)
    assert trace[:, 7].max() >= 2 and (np.diff(trace[:, 0]) != 0).any()
    th_min = th_max = None
    filt = []
    checked = corrected = decided = mu_updates = 0
    dw_last = 0.0
    z1, _, _ = O.solve(p, max_iter=0)
    for k in range(info["iters"]):
        zk = z1
        z1, _, tr = O.solve(p, max_iter=k + 1)
        np.testing.assert_array_equal(tr[k], trace[k])
        mu, alpha, ad, dw, theta, phi, emu, trials = tr[k]
        tau = max(0.99, 1.0 - mu)
        phi_k, th_k, g = merit(zk.y, zk.s_p, zk.s_m, mu)
        if k == 0:
            th_min, th_max = 1e-4 * max(1.0, th_k), 1e4 * max(1.0, th_k)
        if k == 0 or trace[k, 0] != trace[k - 1, 0]:
            filt = []                                   # reset with every barrier update
        assert phi == pytest.approx(phi_k, rel=1e-12) and theta == pytest.approx(th_k, rel=1e-12, abs=1e-300)
        assert emu == pytest.approx(O.kkt_error(p, zk, mu=mu)[0], rel=1e-12)
        assert emu > 10.0 * mu or mu == pytest.approx(tol / 10.0)
        # barrier update (eq. infiniteOCP-innerTol): from the previous mu, the
        # update max(tol/10, min(0.2 mu, mu^1.5)) repeats while E_mu <= 10 mu
        m_prev = 0.1 if k == 0 else trace[k - 1, 0]
        while m_prev != mu:
            assert O.kkt_error(p, zk, mu=m_prev)[0] <= 10.0 * m_prev, (k, m_prev, mu)
            assert m_prev > tol / 10.0
            m_prev = max(tol / 10.0, min(0.2 * m_prev, m_prev ** 1.5))
            assert m_prev >= mu * (1 - 1e-12), (k, m_prev, mu)
        mu_updates += k > 0 and trace[k - 1, 0] != mu
        # inertia correction (W&B Algorithm IC): delta_w is a value of the
        # sequence 0, first, first * kappa, ... and the first at which K_c +
        # delta_w I is positive definite (pivots above 1e-12 |K_jj|).  The
        # eigenvalues of the dense K_c decide definiteness where their rounding
        # error (about 1e-14 n max|K_jj|) is far below the 1e-4 scale of delta_w;
        # near convergence the slack weights b/s reach 1e15 and they cannot.
        lam_min, kdiag = _kc_extremes(O, p, zk)
        err = 1e-14 * p.n * kdiag
        decide = err < 1e-6
        cands = [0.0]
        if dw > 0.0:
            c = 1e-4 if dw_last == 0.0 else max(1e-20, dw_last / 3.0)
            while c < dw * (1 - 1e-14):
                cands.append(c)
                c *= 100.0 if dw_last == 0.0 else 8.0
            assert c == pytest.approx(dw, rel=1e-14), (k, c, dw)
            dw_last = dw
            corrected += 1
        if decide:
            assert lam_min + dw > -err, (k, dw)
            for c in cands if dw > 0.0 else []:
                assert lam_min + c <= err + 1e-11 * kdiag, (k, c, dw)
            decided += dw > 0.0
        rc, d = O.newton_step(p, zk, mu, dw)
        assert rc == 0
        a_max = min(ftb((zk.y - yL)[L], d.y[L], tau), ftb((yU - zk.y)[U], -d.y[U], tau),
                    ftb(zk.s_p, d.s_p, tau), ftb(zk.s_m, d.s_m, tau))
        d_max = min(ftb(zk.zL[L], d.zL[L], tau), ftb(zk.zU[U], d.zU[U], tau),
                    ftb(zk.b_p, d.b_p, tau), ftb(zk.b_m, d.b_m, tau))
        assert ad == pytest.approx(d_max, rel=1e-12)
        assert alpha == pytest.approx(a_max * 0.5 ** (trials - 1), rel=1e-12)
        close = dict(rtol=1e-12, atol=1e-14)
        np.testing.assert_allclose(z1.y, zk.y + alpha * d.y, **close)
        for a in ("s_p", "s_m", "w_p", "w_m"):
            np.testing.assert_allclose(getattr(z1, a), getattr(zk, a) + alpha * getattr(d, a), **close)

        def guard(v, gap):
            return np.maximum(np.minimum(v, ks * mu / gap), mu / (ks * gap))
        np.testing.assert_allclose(z1.zL[L], guard(zk.zL[L] + ad * d.zL[L], (z1.y - yL)[L]), **close)
        np.testing.assert_allclose(z1.zU[U], guard(zk.zU[U] + ad * d.zU[U], (yU - z1.y)[U]), **close)
        np.testing.assert_allclose(z1.b_p, guard(zk.b_p + ad * d.b_p, z1.s_p), **close)
        np.testing.assert_allclose(z1.b_m, guard(zk.b_m + ad * d.b_m, z1.s_m), **close)
        gb = g - np.where(L, mu / np.where(L, zk.y - yL, 1.0), 0.0) + np.where(U, mu / np.where(U, yU - zk.y, 1.0), 0.0)
        gphi = gb @ d.y - mu * (d.s_p / zk.s_p + d.s_m / zk.s_m).sum()
        phi_t, th_t, _ = merit(z1.y, z1.s_p, z1.s_m, mu)
        assert acceptable(phi_t, th_t, phi_k, th_k, alpha, gphi, filt), k
        with np.errstate(invalid="ignore", divide="ignore"):
            for j in range(int(trials) - 1):           # every longer step was rejected
                a = a_max * 0.5 ** j
                ph, th, _ = merit(zk.y + a * d.y, zk.s_p + a * d.s_p, zk.s_m + a * d.s_m, mu)
                assert not acceptable(ph, th, phi_k, th_k, a, gphi, filt), (k, j)
        if not armijo_case(th_k, alpha, gphi, th_min):
            filt.append(((1 - 1e-5) * th_k, phi_k - 1e-5 * th_k))
        checked += 1
    assert checked == info["iters"] and corrected > 0 and mu_updates > 0
    assert decided >= (2 if name.startswith("toy") else 0)


def test_paper_distillation_closed_loop(oracle):
    """The paper's column and cost (Sec. 4.1: N = 32, feed tray 17, holdups
    0.5 / 0.25 / 1.0, dt = 2, 90 intervals, (x_1 - 0.8958)^2 + 0.1 (u - ubar)^2)
    from a perturbed steady state: a cold solve and three warm re-solves of
    the closed loop, each converged; the last point stationary by central
    differences of the objective and constraints."""
    O = oracle
    N, Nf, T, ubar = 32, 17, 90, 2.51459
    kw = dict(dt=2.0, Ac=0.5, At=0.25, Ar=1.0, wdu=0.0, wu=0.1, ubar=ubar)
    xs = np.loadtxt(__import__("os").path.join(__import__("os").path.dirname(__file__), "..",
                                                "paper_2606_04725_gb300", "data", "steady_state_N32_Nf17.txt"))
    x0 = np.clip(xs + np.random.default_rng(6).normal(0, 0.02, N), 0, 1)
    p = O.distillation(N, Nf, T, x0, np.full(T, 0.8958), ubar, **kw)
    st, info, _ = O.solve(p)
    assert info["status"] == 0 and info["E0_scaled"] <= 1e-8
    for k in range(3):
        p.set_params(x0=st.y[p.off_x(1):p.off_x(1) + N].copy(), uprev=st.y[p.off_u(1)])
        st, info, _ = O.solve(p, state=st, warm=True)
        assert info["status"] == 0 and info["iters"] < 10
    r = _fd_stationarity(O, p, st)
    assert np.max(np.abs(r)) < 1e-5
