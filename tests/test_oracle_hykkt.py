"""Pins of the oracle's HyKKT form (CPU only).

HyKKT is the alternative to Lifted-KKT that Sec. 3.2.2 names: the
equalities h = 0 keep their multipliers lambda, the Newton system
[[Wh, H^T], [H, 0]] is solved through the augmented-Lagrangian matrix
K_gamma = Wh + gamma H^T H (sparse Cholesky) and conjugate gradients on the
Schur complement H K_gamma^-1 H^T (Regev et al. 2023; Golub & Greif 2003).

* Newton step: equals the solution of the full primal-dual Newton system of
  the barrier KKT conditions (y, lambda, zL, zU), assembled densely and
  solved with numpy, for any augmentation weight gamma.
* Optimality error: E_mu and E_0 are the norms of that KKT residual, with the
  scaling of W&B eq. (5) over lambda and the bound multipliers.
* Converged solutions: the LQ plate against the equality-constrained QP,
  multipliers included (no relaxation: exact); a box-constrained QP against
  brute-force active sets; the toy problem by finite-difference
  stationarity; the distillation column against the Lifted-KKT solution.
"""
import itertools

import numpy as np
import pytest

from test_oracle_ipm import _small_problem, _quadratic_model, _random_state

HY = dict(kkt=1)


def _full_newton_hy(O, p, st, mu, dw):
    """Dense primal-dual Newton system of the barrier problem with the
    equalities kept, in (dy, dlam, dzL, dzU)."""
    n, m = p.n, p.m
    yL, yU = p.bounds()
    L_idx = np.nonzero(np.isfinite(yL))[0]
    U_idx = np.nonzero(np.isfinite(yU))[0]
    _, g, h, _ = O.evaluate(p, st.y)
    H = O.jacobian_dense(p, st.y)
    W = O.hessian_dense(p, st.y, st.w_p) + dw * np.eye(n)
    nL, nU = len(L_idx), len(U_idx)
    off = np.cumsum([0, n, m, nL, nU])
    J = np.zeros((off[-1], off[-1]))
    F = np.zeros(off[-1])
    EL = np.zeros((n, nL)); EL[L_idx, np.arange(nL)] = 1
    EU = np.zeros((n, nU)); EU[U_idx, np.arange(nU)] = 1
    zL, zU = st.zL[L_idx], st.zU[U_idx]
    B = lambda r, c, M: J.__setitem__((slice(off[r], off[r + 1]), slice(off[c], off[c + 1])), M)
    B(0, 0, W); B(0, 1, H.T); B(0, 2, -EL); B(0, 3, EU)
    F[off[0]:off[1]] = g + H.T @ st.w_p - EL @ zL + EU @ zU
    B(1, 0, H); F[off[1]:off[2]] = h
    gl = st.y[L_idx] - yL[L_idx]
    gu = yU[U_idx] - st.y[U_idx]
    B(2, 0, np.diag(zL) @ EL.T); B(2, 2, np.diag(gl)); F[off[2]:off[3]] = gl * zL - mu
    B(3, 0, -np.diag(zU) @ EU.T); B(3, 3, np.diag(gu)); F[off[3]:off[4]] = gu * zU - mu
    d = np.linalg.solve(J, -F)
    dzL = np.zeros(n); dzL[L_idx] = d[off[2]:off[3]]
    dzU = np.zeros(n); dzU[U_idx] = d[off[3]:off[4]]
    return dict(y=d[:n], w_p=d[off[1]:off[2]], zL=dzL, zU=dzU)


@pytest.mark.parametrize("model", ["distill", "plate", "toy"])
@pytest.mark.parametrize("gamma", [1e2, 1e4, 1e6])
def test_hykkt_newton_step_equals_uncondensed_solve(oracle, model, gamma):
    """Augmentation, CG on the Schur complement and the final solve give the
    Newton step of the unaugmented system, whatever gamma is."""
    O = oracle
    p = _small_problem(O, model)
    done = 0
    for seed, mu, dw in [(1, 0.1, 0.0), (2, 1e-3, 0.5), (3, 1.0, 2.0), (4, 0.05, 5.0)]:
        st = _random_state(O, p, seed)
        rc, d = O.newton_step(p, st, mu, dw, hy_gamma=gamma, cg_tol=1e-15, **HY)
        if rc != 0:
            continue  # K_gamma not positive definite at this point
        ref = _full_newton_hy(O, p, st, mu, dw)
        for k, v in ref.items():
            np.testing.assert_allclose(getattr(d, k), v, rtol=1e-7, atol=1e-8 * (1 + np.abs(v).max()),
                                       err_msg=f"{model} seed {seed} {k} gamma {gamma}")
        done += 1
    assert done >= 2


def test_hykkt_cg_tolerance_controls_the_schur_residual(oracle):
    """A loose CG tolerance leaves a Schur residual that a tight one removes:
    the second block row H dy + h of the returned step is small only for the
    tight tolerance (the first block row holds exactly by the final solve)."""
    O = oracle
    p = _small_problem(O, "distill")
    st = _random_state(O, p, 5)
    _, _, h, _ = O.evaluate(p, st.y)
    H = O.jacobian_dense(p, st.y)
    res = {}
    for tol in (1e-1, 1e-14):
        rc, d = O.newton_step(p, st, 0.1, 1.0, hy_gamma=1.0, cg_tol=tol, cg_max_iter=200, **HY)
        assert rc == 0
        res[tol] = np.abs(H @ d.y + h).max()
    assert res[1e-14] < 1e-10 * max(1.0, np.abs(h).max())
    assert res[1e-1] > 1e3 * res[1e-14]


@pytest.mark.parametrize("model", ["distill", "plate", "toy"])
def test_hykkt_optimality_error_is_the_kkt_residual(oracle, model):
    O = oracle
    p = _small_problem(O, model)
    yL, yU = p.bounds()
    L, U = np.isfinite(yL), np.isfinite(yU)
    for seed, mu, big in [(1, 0.0, 1.0), (2, 0.05, 1.0), (3, 0.0, 1e3), (4, 0.3, 1e3)]:
        st = _random_state(O, p, seed)
        for k in ("zL", "zU", "w_p"):
            getattr(st, k)[:] *= big
        _, g, h, _ = O.evaluate(p, st.y)
        H = O.jacobian_dense(p, st.y)
        ry = g + H.T @ st.w_p - np.where(L, st.zL, 0.0) + np.where(U, st.zU, 0.0)
        dual, prim = np.abs(ry).max(), np.abs(h).max()
        comp = max(np.abs((st.y - yL)[L] * st.zL[L] - mu).max(initial=0.0),
                   np.abs((yU - st.y)[U] * st.zU[U] - mu).max(initial=0.0))
        sum_z = np.abs(st.zL[L]).sum() + np.abs(st.zU[U]).sum()
        n_z = L.sum() + U.sum()
        sd = max(100.0, (np.abs(st.w_p).sum() + sum_z) / (p.m + n_z)) / 100.0
        sc = max(100.0, sum_z / n_z) / 100.0
        es, eu = O.kkt_error(p, st, mu=mu, **HY)
        assert eu == pytest.approx(max(dual, prim, comp), rel=1e-12), (model, seed)
        assert es == pytest.approx(max(dual / sd, prim, comp / sc), rel=1e-12), (model, seed)


def test_hykkt_lq_plate_matches_equality_qp(oracle):
    """No relaxation of the equalities: primal and multipliers of the
    equality-constrained QP are met to the solver's tolerance."""
    O = oracle
    g, S, T = 3, 4, 4
    rng = np.random.default_rng(4)
    p = O.plate(g, S, T, rng.uniform(0, 0.5, g * g), rng.uniform(0, 1, g * g), dt=0.5,
                xhi=1e3, ulo=-1e3, uhi=1e3, cq=0.5, rho_u=1e-2)
    Q, c, A, h0 = _quadratic_model(O, p)
    n, m = p.n, p.m
    sol = np.linalg.solve(np.block([[Q, A.T], [A, np.zeros((m, m))]]), np.concatenate([-c, -h0]))
    st, info, _ = O.solve(p, tol=1e-10, **HY)
    assert info["status"] == 0
    assert np.max(np.abs(st.y - sol[:n])) / max(1.0, np.max(np.abs(sol[:n]))) < 1e-8
    np.testing.assert_allclose(st.w_p, sol[n:], rtol=1e-6, atol=1e-8)


def test_hykkt_box_qp_matches_bruteforce_active_set(oracle):
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
            k = Aall.shape[0]
            K = np.block([[Q, Aall.T], [Aall, np.zeros((k, k))]])
            try:
                sol = np.linalg.solve(K, np.concatenate([-c, -h0, [v for _, v, _ in act]]))
            except np.linalg.LinAlgError:
                continue
            y, nu = sol[:n], sol[n + m:]
            if np.all(y <= yU + 1e-12) and np.all(y >= yL - 1e-12) and \
                    all(s * v >= -1e-12 for (_, _, s), v in zip(act, nu)):
                found.append(y)
    assert len(found) == 1
    st, info, _ = O.solve(p, **HY)
    assert info["status"] == 0
    assert np.max(np.abs(st.y - found[0])) < 1e-6


def test_hykkt_toy_converges_to_a_stationary_point(oracle):
    O = oracle
    T = 14
    dt = 10.0 / T
    t = dt * np.arange(1, T + 1)
    p = O.toy(T, 1.0, np.sin(t), dt=dt)
    st, info, _ = O.solve(p, **HY)
    assert info["status"] == 0 and info["E0_scaled"] <= 1e-8
    n = p.n
    r = -st.zL + st.zU
    for j in range(n):
        e = np.zeros(n); e[j] = 1e-6
        fp, _, hp, _ = O.evaluate(p, st.y + e)
        fm, _, hm, _ = O.evaluate(p, st.y - e)
        r[j] += (fp - fm) / 2e-6 + np.dot((hp - hm) / 2e-6, st.w_p)
    assert np.max(np.abs(r)) < 1e-6
    _, _, h, _ = O.evaluate(p, st.y)
    assert np.max(np.abs(h)) <= 1e-8


def test_lifted_solution_tends_to_the_hykkt_solution(oracle):
    """Both forms solve the same NLP, Lifted-KKT with the equalities relaxed
    to |h| <= gamma: on the 12-tray column the lifted primal solution and its
    multipliers omega+ - omega- approach the HyKKT solution and lambda
    linearly as gamma goes to 0."""
    import paper_2606_04725_gb300.inputs as I
    O = oracle
    T = 20
    x0 = I.distillation_x0(12, 5, seed=1)
    sp, _ = I.distillation_setpoints(12, seed=1)
    p = O.distillation(12, 5, T, x0.copy(), np.full(T, sp), I.U_REF)
    sh, ih, _ = O.solve(p, kkt=1, tol=1e-12)
    assert ih["status"] == 0
    dy, dl = [], []
    for g in (1e-8, 1e-10):
        p = O.distillation(12, 5, T, x0.copy(), np.full(T, sp), I.U_REF)
        sl, il, _ = O.solve(p, kkt=0, tol=1e-11, gamma=g)
        assert il["status"] == 0
        dy.append(np.abs(sl.y - sh.y).max())
        dl.append(np.abs((sl.w_p - sl.w_m) - sh.w_p).max() / np.abs(sh.w_p).max())
    assert dy[0] < 1e-5 and dl[0] < 1e-4
    assert dy[1] < dy[0] / 50 and dl[1] < dl[0] / 50


def _kg_extremes(O, p, st, gamma):
    """Smallest eigenvalue and largest diagonal entry of the dense
    K_gamma = W + Sigma_y + gamma H^T H at st."""
    yL, yU = p.bounds()
    L, U = np.isfinite(yL), np.isfinite(yU)
    H = O.jacobian_dense(p, st.y)
    W = O.hessian_dense(p, st.y, st.w_p)
    sig = np.where(L, st.zL / np.where(L, st.y - yL, 1.0), 0.0) + np.where(U, st.zU / np.where(U, yU - st.y, 1.0), 0.0)
    K = W + np.diag(sig) + gamma * H.T @ H
    return np.linalg.eigvalsh(K)[0], np.abs(np.diag(K)).max()


@pytest.mark.parametrize("name", ["distill", "distill_long_dt", "toy", "toy_far", "plate"])
def test_hykkt_line_search_steps_follow_the_filter_method(oracle, name):
    """The HyKKT form's steps against W&B's filter line search, as the lifted
    form's are pinned: iterates after k and k + 1 iterations, the HyKKT
    Newton step at the k-th iterate (pinned above against the dense system),
    the merits phi_mu = f - mu sum log(gaps) and theta = ||h||_1 recomputed
    here.  Per step: traced phi_mu, theta and E_mu are the iterate's; the dual
    step is the bound multipliers' fraction to the boundary; the primal step
    the primal one halved (trials - 1) times; y and lambda take the primal
    step, zL and zU the dual step and the kappa_Sigma safeguard; the accepted
    trial passes the filter tests and every longer trial failed them; delta_w
    belongs to the inertia-correction sequence and makes K_gamma positive
    definite where dense eigenvalues can decide it."""
    from test_oracle_ipm import LS_PROBLEMS
    O = oracle
    p = LS_PROBLEMS[name](O)
    yL, yU = p.bounds()
    L, U = np.isfinite(yL), np.isfinite(yU)
    tol, ks, hg = 1e-8, 1e10, O.HY_GAMMA

    def merit(y, mu):
        f, g, h, _ = O.evaluate(p, y)
        lg = np.log((y - yL)[L]).sum() + np.log((yU - y)[U]).sum()
        return f - mu * lg, np.abs(h).sum(), g

    def ftb(v, dv, tau):
        neg = dv < 0
        return min(1.0, np.min(tau * v[neg] / -dv[neg], initial=np.inf))

    def armijo_case(th, alpha, gphi):
        return th <= th_min and gphi < 0 and alpha * (-gphi) ** 2.3 > th ** 1.1

    def acceptable(phi_t, th_t, phi, th, alpha, gphi, filt):
        if not (np.isfinite(phi_t) and th_t <= th_max) or any(th_t >= a and phi_t >= b for a, b in filt):
            return False
        if armijo_case(th, alpha, gphi):
            return phi_t <= phi + 1e-4 * alpha * gphi
        return th_t <= (1 - 1e-5) * th or phi_t <= phi - 1e-5 * th

    _, info, trace = O.solve(p, **HY)
    assert info["status"] == 0
    trace = np.asarray(trace)
    th_min = th_max = None
    filt = []
    dw_last = 0.0
    z1, _, _ = O.solve(p, max_iter=0, **HY)
    for k in range(info["iters"]):
        zk = z1
        z1, _, tr = O.solve(p, max_iter=k + 1, **HY)
        np.testing.assert_array_equal(tr[k], trace[k])
        mu, alpha, ad, dw, theta, phi, emu, trials = tr[k]
        tau = max(0.99, 1.0 - mu)
        phi_k, th_k, g = merit(zk.y, mu)
        if k == 0:
            th_min, th_max = 1e-4 * max(1.0, th_k), 1e4 * max(1.0, th_k)
        if k == 0 or trace[k, 0] != trace[k - 1, 0]:
            filt = []
        assert phi == pytest.approx(phi_k, rel=1e-12) and theta == pytest.approx(th_k, rel=1e-12, abs=1e-300)
        assert emu == pytest.approx(O.kkt_error(p, zk, mu=mu, **HY)[0], rel=1e-12)
        assert emu > 10.0 * mu or mu == pytest.approx(tol / 10.0)
        if dw > 0.0:
            c = 1e-4 if dw_last == 0.0 else max(1e-20, dw_last / 3.0)
            while c < dw * (1 - 1e-14):
                c *= 100.0 if dw_last == 0.0 else 8.0
            assert c == pytest.approx(dw, rel=1e-14)
            dw_last = dw
        lam_min, kdiag = _kg_extremes(O, p, zk, hg)
        err = 1e-14 * p.n * kdiag
        if err < 1e-6:
            assert lam_min + dw > -err, (k, dw)
        rc, d = O.newton_step(p, zk, mu, dw, **HY)
        assert rc == 0
        a_max = min(ftb((zk.y - yL)[L], d.y[L], tau), ftb((yU - zk.y)[U], -d.y[U], tau))
        d_max = min(ftb(zk.zL[L], d.zL[L], tau), ftb(zk.zU[U], d.zU[U], tau))
        assert ad == pytest.approx(d_max, rel=1e-12)
        assert alpha == pytest.approx(a_max * 0.5 ** (trials - 1), rel=1e-12)
        close = dict(rtol=1e-12, atol=1e-14)
        np.testing.assert_allclose(z1.y, zk.y + alpha * d.y, **close)
        np.testing.assert_allclose(z1.w_p, zk.w_p + alpha * d.w_p, **close)

        def guard(v, gap):
            return np.maximum(np.minimum(v, ks * mu / gap), mu / (ks * gap))
        np.testing.assert_allclose(z1.zL[L], guard(zk.zL[L] + ad * d.zL[L], (z1.y - yL)[L]), **close)
        np.testing.assert_allclose(z1.zU[U], guard(zk.zU[U] + ad * d.zU[U], (yU - z1.y)[U]), **close)
        gb = g - np.where(L, mu / np.where(L, zk.y - yL, 1.0), 0.0) + np.where(U, mu / np.where(U, yU - zk.y, 1.0), 0.0)
        gphi = gb @ d.y
        phi_t, th_t, _ = merit(z1.y, mu)
        assert acceptable(phi_t, th_t, phi_k, th_k, alpha, gphi, filt), k
        with np.errstate(invalid="ignore", divide="ignore"):
            for j in range(int(trials) - 1):
                a = a_max * 0.5 ** j
                ph, th, _ = merit(zk.y + a * d.y, mu)
                assert not acceptable(ph, th, phi_k, th_k, a, gphi, filt), (k, j)
        if not armijo_case(th_k, alpha, gphi):
            filt.append(((1 - 1e-5) * th_k, phi_k - 1e-5 * th_k))
