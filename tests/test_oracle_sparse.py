"""Pins of the oracle's sparse Cholesky (eq. cholesky-numeric on the pattern of
Sec. 3.2.3's SymCholesky) and of its nested-dissection ordering (CPU only).

The factorization must be exact for any symmetric ordering, so it is checked
against numpy on the permuted matrix; the ordering only has to be a
permutation that cuts fill, which is checked on grid graphs; and the
interior-point method run on it must reach the same points as on the band
Cholesky, which is pinned separately."""
import numpy as np
import pytest

import paper_2606_04725_gb300.inputs as I


def _random_spd(rng, n, dens):
    M = np.tril(rng.uniform(size=(n, n)) < dens, -1)
    A = np.where(M | M.T, rng.uniform(-1.0, 1.0, (n, n)), 0.0)
    A = (A + A.T) / 2
    return A + np.diag(np.abs(A).sum(axis=1) + rng.uniform(0.1, 1.0, n))


def _grid_graph(k):
    """5-point grid graph on k x k vertices as (xadj, adj)."""
    nb = [[] for _ in range(k * k)]
    for i in range(k):
        for j in range(k):
            v = i * k + j
            for di, dj in ((1, 0), (-1, 0), (0, 1), (0, -1)):
                if 0 <= i + di < k and 0 <= j + dj < k:
                    nb[v].append((i + di) * k + j + dj)
    xadj = np.cumsum([0] + [len(a) for a in nb])
    return xadj, np.array([u for a in nb for u in a])


def _permuted_pattern(n, xadj, adj, perm):
    """Lower CSC pattern (diagonal included) of the graph's matrix after the
    symmetric permutation perm."""
    inv = np.empty(n, dtype=int)
    inv[perm] = np.arange(n)
    cols = [[j] for j in range(n)]
    for v in range(n):
        for e in range(xadj[v], xadj[v + 1]):
            a, b = inv[v], inv[adj[e]]
            if a > b:
                cols[b].append(a)
    rowidx = np.array([r for c in cols for r in sorted(set(c))], dtype=np.int32)
    colptr = np.cumsum([0] + [len(set(c)) for c in cols]).astype(np.int32)
    return colptr, rowidx


def test_sparse_cholesky_solves_and_fill_match_numpy(oracle):
    """K x = b to rounding, and nnz(L) equals the nonzeros of numpy's Cholesky
    factor of P K P^T (random values: exact cancellation has probability 0),
    in nested-dissection and natural order."""
    rng = np.random.default_rng(11)
    for trial in range(12):
        n = int(rng.integers(1, 90))
        K = _random_spd(rng, n, rng.uniform(0.02, 0.2))
        b = rng.normal(size=n)
        for nd in (True, False):
            rc, perm, x, nnz = oracle.sparse_cholesky(K, use_nd=nd, b=b)
            assert rc == 0
            assert sorted(perm.tolist()) == list(range(n))
            if not nd:
                assert perm.tolist() == list(range(n))
            np.testing.assert_allclose(K @ x, b, rtol=0, atol=1e-12 * (1 + np.abs(b).max()))
            Lp = np.linalg.cholesky(K[np.ix_(perm, perm)])
            assert nnz == int(np.count_nonzero(np.abs(Lp) > 1e-300))


def test_sparse_cholesky_first_failing_pivot(oracle):
    """The column where the factorization stops is the first j (in the
    permuted order) whose Schur-complement pivot
        K_jj - K_j,<j K_<j,<j^-1 K_<j,j
    fails the test: not above tol |K_jj| (or not positive with tol = 0)."""
    rng = np.random.default_rng(12)
    decided = []
    for trial in range(30):
        n = int(rng.integers(2, 40))
        K = _random_spd(rng, n, 0.15)
        # make it indefinite or nearly singular in a random direction
        v = np.zeros(n)
        idx = rng.choice(n, size=min(n, 3), replace=False)
        v[idx] = rng.normal(size=len(idx))
        # Rayleigh quotient along v times U(0.6, 2.5): indefinite when above 1
        K = K - (v @ K @ v) / (v @ v) * rng.uniform(0.6, 2.5) * np.outer(v, v) / (v @ v)
        tol = [0.0, 1e-3, 1e-1][trial % 3]
        rc, perm, _, _ = oracle.sparse_cholesky(K, use_nd=True, tol=tol)
        Kp = K[np.ix_(perm, perm)]
        want = 0
        for j in range(n):
            piv = Kp[j, j] - (Kp[j, :j] @ np.linalg.solve(Kp[:j, :j], Kp[:j, j]) if j else 0.0)
            ok = piv > tol * abs(Kp[j, j]) if tol > 0 else piv > 0
            if not ok:
                want = j + 1
                break
        if want and abs(piv - (tol * abs(Kp[want - 1, want - 1]) if tol > 0 else 0.0)) < 1e-10 * np.abs(K).max():
            continue  # too close to the threshold to decide in rounding
        assert rc == want, (trial, rc, want)
        decided.append(want)
    assert len(decided) >= 25 and sum(1 for w in decided if w > 0) >= 15


def test_nested_dissection_cuts_fill_on_grids(oracle):
    """A permutation of the vertices whose factor fill on a k x k grid is well
    below the natural (row-by-row, banded) order's, and grows like
    k^2 log k rather than k^3."""
    fills = {}
    for k in (16, 32, 64):
        xadj, adj = _grid_graph(k)
        n = k * k
        perm = oracle.nd_order(xadj, adj, leaf=8)
        assert sorted(perm.tolist()) == list(range(n))
        nat = np.arange(n)
        nnz = {}
        for name, p in (("nd", perm), ("nat", nat)):
            colptr, rowidx = _permuted_pattern(n, xadj, adj, p)
            _, Lp, _ = oracle.symbolic(n, colptr, rowidx)
            nnz[name] = int(Lp[-1])
        fills[k] = nnz
        assert nnz["nd"] < (0.75 if k == 16 else 0.5) * nnz["nat"], (k, nnz)
    # natural order grows 8x per doubling of k (k^3); nested dissection about 4-5x
    assert fills[64]["nd"] / fills[32]["nd"] < 6.0


def test_nested_dissection_handles_disconnected_graphs(oracle):
    """Isolated vertices and several components: still a permutation."""
    rng = np.random.default_rng(3)
    n = 500
    nb = [set() for _ in range(n)]
    for _ in range(300):
        a, b = rng.integers(0, 250, size=2)  # vertices 250.. stay isolated
        if a != b:
            nb[a].add(b); nb[b].add(a)
    xadj = np.cumsum([0] + [len(s) for s in nb])
    adj = np.array([u for s in nb for u in sorted(s)])
    perm = oracle.nd_order(xadj, adj, leaf=4)
    assert sorted(perm.tolist()) == list(range(n))


def _solve_both(oracle, make, **kw):
    out = []
    for ls in (oracle.LINSOLVE_BAND, oracle.LINSOLVE_SPARSE):
        prob = make()
        st, info, _ = oracle.solve(prob, linsolve=ls, **kw)
        assert info["status"] == 0, info
        E, _ = oracle.kkt_error(prob, st)
        assert E <= kw.get("tol", 1e-8) * 1.0001
        out.append((st, info))
    return out


def test_interior_point_on_sparse_factor_equals_band(oracle):
    """The IPM on the sparse factor reaches the band path's solutions: the
    N = 12 column (seed 1) and a 6 x 6 plate with 4 actuators, at tol 1e-10,
    primal within 1e-7 (scaled by the variable's size)."""
    N, Nf, T = 12, 5, 20
    x0 = I.distillation_x0(N, Nf, seed=1)
    (a, ia), (b, ib) = _solve_both(
        oracle, lambda: oracle.distillation(N, Nf, T, x0.copy(), np.full(T, 0.8), I.U_REF), tol=1e-10)
    np.testing.assert_allclose(b.y, a.y, rtol=0, atol=1e-7 * max(1.0, np.abs(a.y).max()))
    g = 6
    tg = I.plate_target(g, seed=3)
    (a, ia), (b, ib) = _solve_both(
        oracle, lambda: oracle.plate(g, 4, 8, np.zeros(g * g), tg.copy()), tol=1e-10)
    np.testing.assert_allclose(b.y, a.y, rtol=0, atol=1e-7 * max(1.0, np.abs(a.y).max()))


def test_newton_step_on_sparse_factor_equals_band(oracle):
    """One Newton direction at a cold start, both factorizations: equal to
    rounding (the pinned band direction solves the same condensed system)."""
    g = 5
    prob = oracle.plate(g, 4, 6, np.zeros(g * g), I.plate_target(g, seed=2))
    st = oracle.State(prob.n, prob.m)
    st.y[:] = oracle.initial_guess(prob)
    st.zL[:] = 1.0; st.zU[:] = 1.0
    st.s_p[:] = st.s_m[:] = 0.1; st.w_p[:] = st.w_m[:] = 1.0; st.b_p[:] = st.b_m[:] = 1.0
    rc0, d0 = oracle.newton_step(prob, st, 0.1, linsolve=oracle.LINSOLVE_BAND)
    rc1, d1 = oracle.newton_step(prob, st, 0.1, linsolve=oracle.LINSOLVE_SPARSE)
    assert rc0 == 0 and rc1 == 0
    for f in oracle.State.FIELDS:
        a, b = getattr(d0, f), getattr(d1, f)
        np.testing.assert_allclose(b, a, rtol=0, atol=1e-10 * max(1.0, np.abs(a).max()))
