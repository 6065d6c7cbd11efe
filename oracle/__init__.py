"""Python access to the C oracle -- TEST INFRASTRUCTURE ONLY.

The oracle is a plain FP64 CPU implementation of the paper's lifted
interior-point method (arXiv 2606.04725, Sec. 3.2, Algorithm 2), used to check
the CUDA library.  Only ``tests/``, ``__graft_entry__.smoke()`` and
``bench.py``'s CPU-baseline leg may import this package.  It shares no code
with the CUDA library.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_SOURCES = [os.path.join(_HERE, f) for f in ("nmpc_oracle.c", "nmpc_oracle.h", "or_model.inc", "or_sparse.inc")]
_lock = threading.Lock()
_lib = None

OR_DISTILL, OR_PLATE, OR_TOY, OR_PPLATE, OR_DDAE = 0, 1, 2, 3, 4
STATUS = {0: "converged", 10: "max_iter", 11: "linesearch_fail", 12: "inertia_fail", 13: "nonfinite", 2: "alloc"}


def build(force: bool = False) -> str:
    """Compile the oracle with gcc into oracle/_build/liboracle.so."""
    os.makedirs(_BUILD, exist_ok=True)
    newest = max(os.path.getmtime(s) for s in _SOURCES)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < newest:
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-o", tmp,
                               os.path.join(_HERE, "nmpc_oracle.c"), "-lm"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class _Problem(C.Structure):
    _fields_ = [("model", C.c_int), ("nx", C.c_int), ("nu", C.c_int), ("T", C.c_int),
                ("n", C.c_int), ("m", C.c_int), ("N", C.c_int), ("Nf", C.c_int),
                ("g", C.c_int), ("S", C.c_int), ("dt", C.c_double),
                ("alpha", C.c_double), ("D", C.c_double), ("F", C.c_double), ("xF", C.c_double),
                ("Ac", C.c_double), ("At", C.c_double), ("Ar", C.c_double), ("wdu", C.c_double),
                ("wu", C.c_double), ("ubar", C.c_double),
                ("kappa", C.c_double), ("cq", C.c_double), ("rho_u", C.c_double),
                ("xlo", C.c_double), ("xhi", C.c_double), ("ulo", C.c_double), ("uhi", C.c_double),
                ("x0", C.POINTER(C.c_double)), ("sp", C.POINTER(C.c_double)), ("uprev", C.c_double),
                ("Tb", C.c_double), ("qloss", C.c_double), ("nr", C.c_int)]


class _Options(C.Structure):
    _fields_ = [("tol", C.c_double), ("gamma", C.c_double), ("mu0_cold", C.c_double),
                ("mu0_warm", C.c_double), ("push_cold", C.c_double), ("push_warm", C.c_double),
                ("max_iter", C.c_int), ("pivtol", C.c_double), ("dw_max", C.c_double),
                ("kkt", C.c_int), ("hy_gamma", C.c_double), ("cg_tol", C.c_double), ("cg_max_iter", C.c_int),
                ("linsolve", C.c_int)]


class _Info(C.Structure):
    _fields_ = [("status", C.c_int), ("iters", C.c_int), ("inertia_retries", C.c_int),
                ("ls_trials", C.c_int), ("mu_final", C.c_double), ("E0_scaled", C.c_double),
                ("E0_unscaled", C.c_double), ("objective", C.c_double), ("delta_w_last", C.c_double),
                ("cg_iters", C.c_int)]


class _State(C.Structure):
    _fields_ = [(k, C.POINTER(C.c_double)) for k in ("y", "zL", "zU", "s_p", "s_m", "w_p", "w_m", "b_p", "b_m")]


_D = C.POINTER(C.c_double)
_I = C.POINTER(C.c_int)


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = C.CDLL(build())
            L.or_setup.argtypes = [C.POINTER(_Problem)]
            L.or_jac_nnz.argtypes = [C.POINTER(_Problem)]
            L.or_bounds.argtypes = [C.POINTER(_Problem), _D, _D]
            L.or_eval.argtypes = [C.POINTER(_Problem), _D, _D, _D, _D, _I, _I, _D]
            L.or_eval_complex.argtypes = [C.POINTER(_Problem), _D, _D, _D, _D, _D, _D]
            L.or_hessian.argtypes = [C.POINTER(_Problem), _D, _D, _I, _I, _D, C.c_int]
            L.or_steady_state.argtypes = [C.POINTER(_Problem), C.c_double, _D]
            L.or_solve.argtypes = [C.POINTER(_Problem), C.POINTER(_Options), C.POINTER(_State), C.c_int,
                                   C.POINTER(_Info), _D, C.c_int]
            L.or_kkt_error.argtypes = [C.POINTER(_Problem), C.POINTER(_Options), C.POINTER(_State),
                                       C.c_double, _D, _D]
            L.or_newton_step.argtypes = [C.POINTER(_Problem), C.POINTER(_Options), C.POINTER(_State),
                                         C.c_double, C.c_double, C.POINTER(_State)]
            L.or_band_cholesky.argtypes = [C.c_int, C.c_int, _D]
            L.or_symbolic.argtypes = [C.c_int, _I, _I, _I, _I, _I, C.c_int]
            L.or_nd_order.argtypes = [C.c_int, _I, _I, C.c_int, _I]
            L.or_sparse_cholesky.argtypes = [C.c_int, _I, _I, _D, C.c_int, C.c_double, _I, _D,
                                             C.POINTER(C.c_long)]
            _lib = L
    return _lib


def _dp(a):
    return a.ctypes.data_as(_D)


def _ip(a):
    return a.ctypes.data_as(_I)


INF = float("inf")

# Newton-system forms: Lifted-KKT (eq. liftedkkt-pd) and HyKKT (Sec. 3.2.2's
# alternative: equalities kept, augmented-Lagrangian Cholesky plus CG).
KKT_LIFTED, KKT_HYKKT = 0, 1
# Factorization of the condensed matrix: band Cholesky in stage order, or the
# sparse Cholesky after the oracle's own nested-dissection ordering.
LINSOLVE_BAND, LINSOLVE_SPARSE = 0, 1
HY_GAMMA, CG_TOL, CG_MAX_ITER = 1e4, 1e-12, 200


class Problem:
    """One transcribed OCP instance (keeps its parameter arrays alive)."""

    def __init__(self, model, T, dt, x0, sp, *, N=0, Nf=0, g=0, S=0, uprev=0.0,
                 alpha=1.6, D=0.2, F=0.4, xF=0.5, Ac=1.0, At=1.0, Ar=1.0, wdu=0.01, wu=0.0, ubar=0.0,
                 kappa=0.01, cq=0.01, rho_u=1e-3, xlo=0.0, xhi=1.0, ulo=1.0, uhi=5.0, Tb=50.0, qloss=10.0):
        self.x0 = np.ascontiguousarray(x0, dtype=np.float64)
        self.sp = np.ascontiguousarray(sp, dtype=np.float64)
        p = _Problem()
        p.model, p.T, p.dt, p.N, p.Nf, p.g, p.S = model, T, dt, N, Nf, g, S
        p.alpha, p.D, p.F, p.xF, p.Ac, p.At, p.Ar, p.wdu = alpha, D, F, xF, Ac, At, Ar, wdu
        p.wu, p.ubar = wu, ubar
        p.kappa, p.cq, p.rho_u = kappa, cq, rho_u
        p.xlo, p.xhi, p.ulo, p.uhi = xlo, xhi, ulo, uhi
        p.uprev = uprev
        p.Tb, p.qloss = Tb, qloss
        self._p = p
        if lib().or_setup(C.byref(p)) != 0:
            raise ValueError("invalid problem dimensions")
        p.x0 = _dp(self.x0)
        p.sp = _dp(self.sp)
        self.n, self.m, self.nx, self.nu, self.T = p.n, p.m, p.nx, p.nu, p.T
        if self.x0.size != self.nx:
            raise ValueError("x0 has wrong length")
        self.model = model

    @property
    def ref(self):
        return C.byref(self._p)

    def set_params(self, x0=None, sp=None, uprev=None):
        if x0 is not None:
            self.x0[:] = x0
        if sp is not None:
            self.sp[:] = sp
        if uprev is not None:
            self._p.uprev = float(uprev)

    def off_x(self, k):
        return 0 if k == 0 else self.nx + (k - 1) * (self.nx + self.nu)

    def off_u(self, k):
        return self.off_x(k) + self.nx

    def jac_nnz(self):
        return lib().or_jac_nnz(self.ref)

    def bounds(self):
        yL = np.empty(self.n)
        yU = np.empty(self.n)
        lib().or_bounds(self.ref, _dp(yL), _dp(yU))
        return yL, yU


def distillation(N, Nf, T, x0, sp, uprev, dt=1.0, **kw):
    return Problem(OR_DISTILL, T, dt, x0, sp, N=N, Nf=Nf, uprev=uprev, **kw)


def plate(g, S, T, x0, target, dt=1.0, xhi=1.2, **kw):
    kw.setdefault("xlo", -INF)
    kw.setdefault("ulo", 0.0)
    kw.setdefault("uhi", 1.0)
    return Problem(OR_PLATE, T, dt, x0, target, g=g, S=S, xhi=xhi, **kw)


def distillation_dae(N, Nf, T, x0, sp, uprev, dt=1.0, **kw):
    """The column of eq. (distill-ocp) with its algebraic variables: per stage
    [x (N) | y (N) u L V S], the equilibria and flow equations as rows,
    y in [0, 1], L, V, S in [0, 10]."""
    return Problem(OR_DDAE, T, dt, x0, sp, N=N, Nf=Nf, uprev=uprev, **kw)


def paper_plate(n, T, x0, sp, uprev, dt=0.08, **kw):
    """The paper's heated plate (Sec. 4.2, eq. (pde-ocp), table pde-params):
    n x n nodes on [-1, 1]^2, alpha = 230, T_b = 50, q_loss = 10, rho = 1e-8,
    Q >= 50, dt = 0.08; sp holds the T stage setpoints T_sp(t_k); uprev is the
    control of the cold start."""
    kw.setdefault("kappa", 230.0)
    kw.setdefault("rho_u", 1e-8)
    kw.setdefault("xlo", -INF)
    kw.setdefault("xhi", INF)
    kw.setdefault("ulo", 50.0)
    kw.setdefault("uhi", INF)
    return Problem(OR_PPLATE, T, dt, x0, sp, g=n, S=1, uprev=uprev, **kw)


def toy(T, y0, sp, dt, **kw):
    kw.setdefault("xlo", 0.0)
    kw.setdefault("xhi", INF)
    kw.setdefault("ulo", 1.0)
    kw.setdefault("uhi", 3.0)
    return Problem(OR_TOY, T, dt, np.atleast_1d(y0), sp, **kw)


def evaluate(prob, y):
    y = np.ascontiguousarray(y, dtype=np.float64)
    f = np.zeros(1)
    grad = np.empty(prob.n)
    h = np.empty(prob.m)
    nnz = prob.jac_nnz()
    rp = np.empty(prob.m + 1, dtype=np.int32)
    ci = np.empty(nnz, dtype=np.int32)
    hv = np.empty(nnz)
    lib().or_eval(prob.ref, _dp(y), _dp(f), _dp(grad), _dp(h), _ip(rp), _ip(ci), _dp(hv))
    return f[0], grad, h, (rp, ci, hv)


def jacobian_dense(prob, y):
    _, _, _, (rp, ci, hv) = evaluate(prob, y)
    J = np.zeros((prob.m, prob.n))
    for r in range(prob.m):
        J[r, ci[rp[r]:rp[r + 1]]] += hv[rp[r]:rp[r + 1]]
    return J


def evaluate_complex(prob, y_re, y_im):
    y_re = np.ascontiguousarray(y_re, dtype=np.float64)
    y_im = np.ascontiguousarray(y_im, dtype=np.float64)
    nnz = prob.jac_nnz()
    f = np.empty(2)
    g = np.empty(2 * prob.n)
    h = np.empty(2 * prob.m)
    H = np.empty(2 * nnz)
    lib().or_eval_complex(prob.ref, _dp(y_re), _dp(y_im), _dp(f), _dp(g), _dp(h), _dp(H))
    return (f[0] + 1j * f[1], g[:prob.n] + 1j * g[prob.n:], h[:prob.m] + 1j * h[prob.m:],
            H[:nnz] + 1j * H[nnz:])


def hessian_dense(prob, y, lam):
    y = np.ascontiguousarray(y, dtype=np.float64)
    lam = np.ascontiguousarray(lam, dtype=np.float64)
    cnt = lib().or_hessian(prob.ref, _dp(y), _dp(lam), None, None, None, 0)
    r = np.empty(cnt, dtype=np.int32)
    c = np.empty(cnt, dtype=np.int32)
    v = np.empty(cnt)
    lib().or_hessian(prob.ref, _dp(y), _dp(lam), _ip(r), _ip(c), _dp(v), cnt)
    W = np.zeros((prob.n, prob.n))
    np.add.at(W, (r, c), v)
    return W + np.tril(W, -1).T


def steady_state(prob, u):
    x = np.empty(prob.nx)
    it = lib().or_steady_state(prob.ref, float(u), _dp(x))
    if it < 0:
        raise RuntimeError("steady-state Newton did not converge")
    return x


def default_options(**kw):
    o = dict(tol=1e-8, gamma=1e-8, mu0_cold=0.1, mu0_warm=1e-8, push_cold=1e-2, push_warm=1e-9,
             max_iter=200, pivtol=1e-12, dw_max=1e40, kkt=KKT_LIFTED, hy_gamma=HY_GAMMA, cg_tol=CG_TOL,
             cg_max_iter=CG_MAX_ITER, linsolve=LINSOLVE_BAND)
    o.update(kw)
    return o


def _opts(o):
    s = _Options()
    for k, v in o.items():
        setattr(s, k, v)
    return s


class State:
    """Primal-dual iterate: y, zL, zU (n) and s/w/b for both lifted sides (m)."""
    FIELDS = ("y", "zL", "zU", "s_p", "s_m", "w_p", "w_m", "b_p", "b_m")

    def __init__(self, n, m):
        for k in self.FIELDS:
            setattr(self, k, np.zeros(n if k in ("y", "zL", "zU") else m))

    def copy(self):
        s = State.__new__(State)
        for k in self.FIELDS:
            setattr(s, k, getattr(self, k).copy())
        return s

    def _c(self):
        st = _State()
        for k in self.FIELDS:
            setattr(st, k, _dp(getattr(self, k)))
        return st


def initial_guess(prob):
    """Constant-in-time initial guess: x_k = x0, u_k = u_prev (distillation) or
    the midpoint of the control bounds."""
    y = np.zeros(prob.n)
    yL, yU = prob.bounds()
    for k in range(prob.T + 1):
        y[prob.off_x(k):prob.off_x(k) + prob.nx] = prob.x0
        if k >= 1:
            ou = prob.off_u(k)
            lo, hi = yL[ou:ou + prob.nu], yU[ou:ou + prob.nu]
            if prob.model in (OR_DISTILL, OR_PPLATE):
                y[ou] = prob._p.uprev
            elif prob.model == OR_DDAE:
                # the algebraic variables consistent with x0 and u_prev
                p, u = prob._p, prob._p.uprev
                y[ou:ou + prob.nx] = p.alpha * prob.x0 / (1.0 + (p.alpha - 1.0) * prob.x0)
                y[ou + prob.nx:ou + prob.nx + 4] = [u, u * p.D, u * p.D + p.D, u * p.D + p.F]
            else:
                y[ou:ou + prob.nu] = np.where(np.isfinite(lo) & np.isfinite(hi), 0.5 * (lo + hi), 0.0)
    return y


def solve(prob, state=None, warm=False, trace_cap=400, **opts):
    o = default_options(**opts)
    if state is None:
        state = State(prob.n, prob.m)
        state.y[:] = initial_guess(prob)
    info = _Info()
    trace = np.zeros(8 * trace_cap)
    st = state._c()
    lib().or_solve(prob.ref, C.byref(_opts(o)), C.byref(st), int(warm), C.byref(info), _dp(trace), trace_cap)
    res = {k: getattr(info, k) for k, _ in _Info._fields_}
    res["status_name"] = STATUS.get(info.status, str(info.status))
    tr = trace.reshape(trace_cap, 8)[:info.iters]
    return state, res, tr


def kkt_error(prob, state, mu=0.0, **opts):
    o = default_options(**opts)
    es = C.c_double()
    eu = C.c_double()
    st = state._c()
    lib().or_kkt_error(prob.ref, C.byref(_opts(o)), C.byref(st), float(mu), C.byref(es), C.byref(eu))
    return es.value, eu.value


def newton_step(prob, state, mu, delta_w=0.0, **opts):
    o = default_options(**opts)
    d = State(prob.n, prob.m)
    st = state._c()
    dc = d._c()
    rc = lib().or_newton_step(prob.ref, C.byref(_opts(o)), C.byref(st), float(mu), float(delta_w), C.byref(dc))
    return rc, d


def band_cholesky(band):
    """band: (n, b+1) array with band[j, d] = K(j+d, j); factored in place."""
    band = np.ascontiguousarray(band, dtype=np.float64)
    n, w = band.shape
    rc = lib().or_band_cholesky(n, w - 1, _dp(band))
    return rc, band


def symbolic(n, colptr, rowidx):
    colptr = np.ascontiguousarray(colptr, dtype=np.int32)
    rowidx = np.ascontiguousarray(rowidx, dtype=np.int32)
    parent = np.empty(n, dtype=np.int32)
    Lp = np.empty(n + 1, dtype=np.int32)
    cap = n * (n + 1) // 2
    Li = np.empty(cap, dtype=np.int32)
    nnz = lib().or_symbolic(n, _ip(colptr), _ip(rowidx), _ip(parent), _ip(Lp), _ip(Li), cap)
    return parent, Lp, Li[:nnz]


def nd_order(xadj, adj, leaf=64):
    """Nested-dissection order of a symmetric graph (adjacency without self
    loops): perm[k] = the vertex numbered k."""
    xadj = np.ascontiguousarray(xadj, dtype=np.int32)
    adj = np.ascontiguousarray(adj, dtype=np.int32)
    n = len(xadj) - 1
    perm = np.empty(n, dtype=np.int32)
    lib().or_nd_order(n, _ip(xadj), _ip(adj), int(leaf), _ip(perm))
    return perm


def sparse_cholesky(K, use_nd=True, tol=0.0, b=None):
    """Sparse Cholesky of the symmetric dense matrix K (its lower triangle's
    nonzeros form the pattern), after nested dissection or in natural order.
    Returns (rc, perm, x, nnzL): rc 0 on success or j+1 for the first failing
    pivot j in the permuted order, x = K^-1 b when b is given and rc == 0."""
    K = np.asarray(K, dtype=np.float64)
    n = K.shape[0]
    cols, rows, vals = [], [], []
    colptr = np.zeros(n + 1, dtype=np.int32)
    for j in range(n):
        r = np.nonzero(K[j:, j])[0] + j
        rows.append(r); vals.append(K[r, j])
        colptr[j + 1] = colptr[j] + len(r)
    rowidx = np.ascontiguousarray(np.concatenate(rows) if rows else np.zeros(0), dtype=np.int32)
    v = np.ascontiguousarray(np.concatenate(vals) if vals else np.zeros(0), dtype=np.float64)
    perm = np.empty(n, dtype=np.int32)
    x = None if b is None else np.array(b, dtype=np.float64)
    nnz = C.c_long()
    rc = lib().or_sparse_cholesky(n, _ip(colptr), _ip(rowidx), _dp(v), int(bool(use_nd)), float(tol),
                                   _ip(perm), None if x is None else _dp(x), C.byref(nnz))
    return rc, perm, x, nnz.value
