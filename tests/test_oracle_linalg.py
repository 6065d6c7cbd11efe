"""Pins of the oracle's linear algebra: banded Cholesky (eq. cholesky-numeric)
and the symbolic analysis of Sec. 3.2.3 (CPU only)."""
import os

import numpy as np

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _band_of(K, b):
    n = K.shape[0]
    band = np.zeros((n, b + 1))
    for j in range(n):
        for d in range(b + 1):
            if j + d < n:
                band[j, d] = K[j + d, j]
    return band


def _dense_of_band(band):
    n, w = band.shape
    L = np.zeros((n, n))
    for j in range(n):
        for d in range(w):
            if j + d < n:
                L[j + d, j] = band[j, d]
    return L


def test_band_cholesky_matches_library(oracle):
    rng = np.random.default_rng(0)
    for n, b in [(1, 0), (7, 2), (40, 5), (33, 32), (60, 11)]:
        A = rng.normal(size=(n, n))
        mask = np.abs(np.subtract.outer(np.arange(n), np.arange(n))) <= b
        K = (A @ A.T) * mask + n * np.eye(n)
        rc, band = oracle.band_cholesky(_band_of(K, b))
        assert rc == 0
        L = _dense_of_band(band)
        np.testing.assert_allclose(L, np.linalg.cholesky(K), rtol=1e-12, atol=1e-12)


def test_band_cholesky_laplacian_closed_form(oracle):
    """The 1-D Dirichlet Laplacian tridiag(-1, 2, -1) has the bidiagonal
    factor L_jj = sqrt((j+2)/(j+1)), L_{j+1,j} = -sqrt((j+1)/(j+2))."""
    n = 50
    band = np.zeros((n, 2))
    band[:, 0] = 2.0
    band[:-1, 1] = -1.0
    rc, band = oracle.band_cholesky(band)
    assert rc == 0
    j = np.arange(n)
    np.testing.assert_allclose(band[:, 0], np.sqrt((j + 2) / (j + 1)), rtol=1e-14)
    np.testing.assert_allclose(band[:-1, 1], -np.sqrt((j[:-1] + 1) / (j[:-1] + 2)), rtol=1e-14)


def test_band_cholesky_reports_first_bad_pivot(oracle):
    """Cholesky succeeds exactly for positive-definite input (the inertia test
    of eq. infiniteOCP-inertia); the failing column is the first one whose
    Schur complement pivot is not positive."""
    rng = np.random.default_rng(1)
    n = 12
    Q, _ = np.linalg.qr(rng.normal(size=(n, n)))
    ev = np.linspace(1, 3, n)
    ev[7] = -0.5
    K = Q @ np.diag(ev) @ Q.T
    rc, _ = oracle.band_cholesky(_band_of(K, n - 1))
    # pivot j is det(K[:j+1,:j+1]) / det(K[:j,:j])
    dets = [1.0] + [np.linalg.det(K[:j + 1, :j + 1]) for j in range(n)]
    first_bad = next(j for j in range(n) if dets[j + 1] / dets[j] <= 0)
    assert rc == first_bad + 1


def _read_fig():
    K, etree, L = {}, [], {}
    with open(os.path.join(GOLDEN, "fig_cholesky_symexample.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            t = line.split()
            if t[0] == "n":
                n = int(t[1])
            elif t[0] == "K":
                K[int(t[1][:-1])] = [int(v) for v in t[2:]]
            elif t[0] == "L":
                L[int(t[1][:-1])] = [int(v) for v in t[2:]]
            elif t[0] == "etree":
                etree.append((int(t[1]), int(t[2])))
    return n, K, etree, L


def _lower_csc(n, rows_of):
    """rows_of[i] = list of columns j with K_ij != 0 (1-based)."""
    cols = [[] for _ in range(n)]
    for i, js in rows_of.items():
        for j in js:
            if i >= j:
                cols[j - 1].append(i - 1)
    colptr = np.cumsum([0] + [len(c) for c in cols]).astype(np.int32)
    rowidx = np.array([r for c in cols for r in sorted(c)], dtype=np.int32)
    return colptr, rowidx


def test_symbolic_paper_figure(oracle):
    """Fig. cholesky-symExample: exact elimination tree and fill (4,3), (6,3), (6,4)."""
    n, K, etree, L = _read_fig()
    colptr, rowidx = _lower_csc(n, K)
    parent, Lp, Li = oracle.symbolic(n, colptr, rowidx)
    want_parent = np.full(n, -1)
    for c, p in etree:
        want_parent[c - 1] = p - 1
    np.testing.assert_array_equal(parent, want_parent)
    got = {}
    for j in range(n):
        for i in Li[Lp[j]:Lp[j + 1]]:
            got.setdefault(i + 1, []).append(j + 1)
    assert {i: sorted(v) for i, v in got.items()} == {i: sorted(v) for i, v in L.items()}


def test_symbolic_matches_numeric_elimination(oracle):
    """On random symmetric patterns the structure of L equals the nonzeros of a
    numeric Cholesky factor with random values (exact cancellation has
    probability zero), and parent[j] is the first subdiagonal row of L."""
    rng = np.random.default_rng(7)
    for trial in range(20):
        n = int(rng.integers(2, 30))
        dens = rng.uniform(0.05, 0.3)
        M = np.tril(rng.uniform(size=(n, n)) < dens, -1)
        S = M | M.T
        A = np.where(S, rng.uniform(0.1, 1.0, (n, n)), 0.0)
        A = (A + A.T) / 2
        K = A + np.diag(np.abs(A).sum(axis=1) + 1.0)
        colptr, rowidx = _lower_csc(n, {i + 1: list(np.nonzero(K[i])[0] + 1) for i in range(n)})
        parent, Lp, Li = oracle.symbolic(n, colptr, rowidx)
        Lnum = np.linalg.cholesky(K)
        for j in range(n):
            rows = np.nonzero(np.abs(Lnum[j:, j]) > 1e-300)[0] + j
            np.testing.assert_array_equal(Li[Lp[j]:Lp[j + 1]], rows)
            sub = rows[rows > j]
            assert parent[j] == (sub[0] if sub.size else -1)
