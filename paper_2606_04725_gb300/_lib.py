"""ctypes binding of libnmpc.so (include/nmpc.h).

Argument marshalling only: every numeric step runs in the library's CUDA
kernels.  PyTorch supplies the device workspace and the CUDA stream.  If the
compiled library is missing, loading raises instead of falling back to any
other implementation.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libnmpc.so")
_lock = threading.Lock()
_lib = None

MODEL_DISTILLATION, MODEL_PLATE, MODEL_TOY, MODEL_PAPER_PLATE, MODEL_DISTILLATION_DAE = 0, 1, 2, 3, 4
ORDER_AUTO, ORDER_NATURAL, ORDER_ND = 0, 1, 2
KKT_LIFTED, KKT_HYKKT = 0, 1
STATUS = {0: "ok", 1: "invalid", 2: "cuda_error", 3: "workspace", 10: "max_iter", 11: "linesearch_fail",
          12: "inertia_fail", 13: "nonfinite", 14: "timeout", 15: "not_solved"}

EXPORTED = ["nmpc_problem_defaults", "nmpc_options_defaults", "nmpc_build", "nmpc_workspace_bytes",
            "nmpc_bind", "nmpc_set_params", "nmpc_solve", "nmpc_get_solution", "nmpc_set_start",
            "nmpc_sensitivity", "nmpc_get_trace", "nmpc_time_phases", "nmpc_get_stats", "nmpc_instance_dims", "nmpc_structure_export",
            "nmpc_autotune_workspace_bytes", "nmpc_autotune",
            "nmpc_solve_static", "nmpc_debug_recip", "nmpc_probe_fp64",
            "nmpc_destroy", "nmpc_status_string", "nmpc_last_error"]

STATIC_WORKSPACE_BYTES = 32 * 1024 * 1024


class Problem(C.Structure):
    _fields_ = [("model", C.c_int), ("n_instances", C.c_int), ("horizons", C.POINTER(C.c_int)),
                ("N", C.c_int), ("Nf", C.c_int), ("g", C.c_int), ("S", C.c_int), ("dt", C.c_double),
                ("alpha", C.c_double), ("D", C.c_double), ("F", C.c_double), ("xF", C.c_double),
                ("Ac", C.c_double), ("At", C.c_double), ("Ar", C.c_double), ("wdu", C.c_double),
                ("kappa", C.c_double), ("cq", C.c_double), ("rho_u", C.c_double),
                ("xlo", C.c_double), ("xhi", C.c_double), ("ulo", C.c_double), ("uhi", C.c_double),
                ("wu", C.c_double), ("ubar", C.c_double), ("Tb", C.c_double), ("qloss", C.c_double)]


class Options(C.Structure):
    _fields_ = [("tol", C.c_double), ("gamma", C.c_double), ("mu0_cold", C.c_double), ("mu0_warm", C.c_double),
                ("push_cold", C.c_double), ("push_warm", C.c_double), ("max_iter", C.c_int),
                ("ordering", C.c_int), ("nd_leaf", C.c_int), ("use_graph", C.c_int), ("spin_limit", C.c_longlong),
                ("pivtol", C.c_double), ("factor_mode", C.c_int), ("solve_mode", C.c_int),
                ("panel_scale", C.c_int), ("amalgamation", C.c_int), ("dw_max", C.c_double),
                ("kkt", C.c_int), ("hykkt_gamma", C.c_double), ("cg_tol", C.c_double), ("cg_max_iter", C.c_int)]


class Info(C.Structure):
    _fields_ = [("status", C.c_int), ("iters", C.c_int), ("inertia_retries", C.c_int), ("ls_trials", C.c_int),
                ("mu_final", C.c_double), ("kkt_scaled", C.c_double), ("kkt_unscaled", C.c_double),
                ("objective", C.c_double), ("ms_total", C.c_double), ("cg_iters", C.c_int)]


class Stats(C.Structure):
    _fields_ = [("n_total", C.c_int), ("m_total", C.c_int), ("n_supernodes", C.c_int), ("n_levels", C.c_int),
                ("nnz_L", C.c_longlong), ("factor_flops", C.c_double), ("solve_flops", C.c_double),
                ("workspace_bytes", C.c_longlong), ("analysis_ms", C.c_double), ("max_front", C.c_int),
                ("ordering_used", C.c_int), ("kernel_launches", C.c_longlong), ("amalgamation_used", C.c_int)]


class PhaseTimes(C.Structure):
    _fields_ = [("ms_eval", C.c_double), ("ms_assemble", C.c_double), ("ms_factor", C.c_double),
                ("ms_solve", C.c_double), ("reps", C.c_int)]


class TuneCandidate(C.Structure):
    _fields_ = [("ordering", C.c_int), ("nd_leaf", C.c_int), ("panel_scale", C.c_int), ("status", C.c_int),
                ("iters", C.c_int), ("ms_per_iter", C.c_double), ("amalgamation", C.c_int),
                ("factor_mode", C.c_int), ("ms_resolve", C.c_double)]


TUNE_MAX = 16


class TuneReport(C.Structure):
    _fields_ = [("n_candidates", C.c_int), ("best", C.c_int), ("cached", C.c_int),
                ("cand", TuneCandidate * TUNE_MAX)]


_P = C.c_void_p
_D = C.POINTER(C.c_double)


def lib():
    """Load libnmpc.so (built by paper_2606_04725_gb300.build)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError(f"{LIB_PATH} is missing: run paper_2606_04725_gb300.build.build() "
                                   "(the CUDA library is required; there is no fallback)")
            try:  # share the CUDA runtime PyTorch has loaded
                import torch  # noqa: F401
            except Exception:
                pass
            L = C.CDLL(LIB_PATH)
            L.nmpc_problem_defaults.argtypes = [C.c_int, C.POINTER(Problem)]
            L.nmpc_problem_defaults.restype = None
            L.nmpc_options_defaults.argtypes = [C.POINTER(Options)]
            L.nmpc_options_defaults.restype = None
            L.nmpc_build.argtypes = [C.POINTER(Problem), C.POINTER(Options), _P, C.POINTER(_P)]
            L.nmpc_workspace_bytes.argtypes = [_P, C.POINTER(C.c_size_t)]
            L.nmpc_bind.argtypes = [_P, _P, C.c_size_t]
            L.nmpc_set_params.argtypes = [_P, C.c_int, _P, _P, _P, C.c_int]
            L.nmpc_solve.argtypes = [_P, C.c_int, C.POINTER(Info)]
            L.nmpc_get_solution.argtypes = [_P, C.c_int, _P, _P, C.c_int]
            L.nmpc_set_start.argtypes = [_P, C.c_int, _P, _P, C.c_int]
            L.nmpc_sensitivity.argtypes = [_P, C.c_int, _P, _P, _P, C.c_int]
            L.nmpc_get_stats.argtypes = [_P, C.POINTER(Stats)]
            L.nmpc_get_trace.argtypes = [_P, C.c_int, _P, C.c_int]
            L.nmpc_time_phases.argtypes = [_P, C.c_int, C.POINTER(PhaseTimes)]
            L.nmpc_instance_dims.argtypes = [_P, C.c_int, C.POINTER(C.c_int), C.POINTER(C.c_int), C.POINTER(C.c_int)]
            L.nmpc_structure_export.argtypes = [_P, C.c_int, _P, C.c_longlong]
            L.nmpc_structure_export.restype = C.c_longlong
            L.nmpc_solve_static.argtypes = [C.POINTER(Problem), C.POINTER(Options), _P, _P, _P, _P, _P,
                                            C.POINTER(Info), C.c_int]
            L.nmpc_autotune_workspace_bytes.argtypes = [C.POINTER(Problem), C.POINTER(Options),
                                                        C.POINTER(C.c_size_t)]
            L.nmpc_autotune.argtypes = [C.POINTER(Problem), C.POINTER(Options), _P, _P, C.c_size_t, _P, _P, _P,
                                        C.c_int, C.POINTER(TuneReport)]
            L.nmpc_debug_recip.argtypes = [_P, _P, C.c_longlong, _P]
            L.nmpc_probe_fp64.argtypes = [C.c_int, C.c_int, C.c_int, _P, C.POINTER(C.c_double)]
            L.nmpc_destroy.argtypes = [_P]
            L.nmpc_destroy.restype = None
            L.nmpc_status_string.argtypes = [C.c_int]
            L.nmpc_status_string.restype = C.c_char_p
            L.nmpc_last_error.argtypes = [_P]
            L.nmpc_last_error.restype = C.c_char_p
            _lib = L
    return _lib


class NmpcError(RuntimeError):
    def __init__(self, status, msg=""):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


def autotune(model, horizons, x0=None, setpoint=None, u_prev=None, opts=None, device="cuda", stream=None,
             **prob_kw):
    """nmpc_autotune: the options (ordering, nd_leaf, panel_scale) with the
    least time per interior-point iteration for this problem and these
    parameters, found by timing one cold solve per candidate in a scratch
    workspace.  Parameters are packed instance after instance (setpoints of
    T_i values each for the distillation).  Returns (options, report)."""
    import torch
    dev = torch.device(device)
    p, hz = problem(model, horizons, **prob_kw)
    p.horizons = hz.ctypes.data_as(C.POINTER(C.c_int))
    o = Options()
    C.memmove(C.byref(o), C.byref(opts if opts is not None else options()), C.sizeof(Options))
    L = lib()
    b = C.c_size_t()
    st = L.nmpc_autotune_workspace_bytes(C.byref(p), C.byref(o), C.byref(b))
    if st != 0:
        raise NmpcError(st, "nmpc_autotune_workspace_bytes failed")
    with torch.cuda.device(dev):
        strm = stream if stream is not None else torch.cuda.current_stream(dev)
        ws = torch.empty(b.value + 256, dtype=torch.uint8, device=dev)
        aligned = (ws.data_ptr() + 255) & ~255
        ptrs = [_ptr(a) for a in (x0, setpoint, u_prev)]
        flags = {q[1] for q in ptrs if q[0] is not None}
        if len(flags) > 1:
            raise ValueError("mix of host and device parameter arrays")
        on_dev = flags.pop() if flags else 0
        rep = TuneReport()
        st = L.nmpc_autotune(C.byref(p), C.byref(o), C.c_void_p(strm.cuda_stream), C.c_void_p(aligned), b.value,
                             ptrs[0][0], ptrs[1][0], ptrs[2][0], on_dev, C.byref(rep))
        torch.cuda.synchronize(dev)
    if st != 0:
        raise NmpcError(st, "nmpc_autotune found no converging candidate")
    cands = [{k: getattr(rep.cand[i], k) for k, _ in TuneCandidate._fields_} for i in range(rep.n_candidates)]
    return o, {"cached": bool(rep.cached), "best": rep.best, "candidates": cands}


def problem(model, horizons, **kw):
    """nmpc_problem with library defaults for `model`, overridden by kw."""
    p = Problem()
    lib().nmpc_problem_defaults(int(model), C.byref(p))
    hz = np.ascontiguousarray(np.atleast_1d(horizons), dtype=np.int32)
    p.n_instances = int(hz.size)
    for k, v in kw.items():
        if not hasattr(p, k):
            raise KeyError(k)
        setattr(p, k, v)
    return p, hz


def options(**kw):
    o = Options()
    lib().nmpc_options_defaults(C.byref(o))
    for k, v in kw.items():
        if not hasattr(o, k):
            raise KeyError(k)
        setattr(o, k, v)
    return o


def _ptr(a):
    """(address, on_device) of a numpy array or a torch tensor."""
    if a is None:
        return None, None
    if isinstance(a, np.ndarray):
        if a.dtype != np.float64 or not a.flags.c_contiguous:
            raise TypeError("host arrays must be contiguous float64")
        return a.ctypes.data, 0
    import torch
    if isinstance(a, torch.Tensor):
        if a.dtype != torch.float64 or not a.is_contiguous():
            raise TypeError("tensors must be contiguous float64")
        return a.data_ptr(), (1 if a.is_cuda else 0)
    raise TypeError(type(a))


class Structure:
    """Host-only analysis (nmpc_build without bind): sizes and patterns."""

    def __init__(self, model, horizons, opts=None, **prob_kw):
        self._p, self._hz = problem(model, horizons, **prob_kw)
        self._p.horizons = self._hz.ctypes.data_as(C.POINTER(C.c_int))
        self._o = opts if opts is not None else options()
        h = _P()
        st = lib().nmpc_build(C.byref(self._p), C.byref(self._o), None, C.byref(h))
        if st != 0:
            raise NmpcError(st, "nmpc_build failed")
        self._h = h

    def stats(self):
        s = Stats()
        lib().nmpc_get_stats(self._h, C.byref(s))
        return {k: getattr(s, k) for k, _ in Stats._fields_}

    def export(self, what):
        L = lib()
        cnt = L.nmpc_structure_export(self._h, what, None, 0)
        if cnt < 0:
            raise ValueError(what)
        width = {8: 2, 9: 4}.get(what, 1)
        out = np.empty(cnt * width, dtype=np.int32)
        L.nmpc_structure_export(self._h, what, out.ctypes.data, cnt)
        return out.reshape(-1, width) if width > 1 else out

    def workspace_bytes(self):
        b = C.c_size_t()
        lib().nmpc_workspace_bytes(self._h, C.byref(b))
        return b.value

    def close(self):
        if getattr(self, "_h", None):
            lib().nmpc_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Solver(Structure):
    """A bound NMPC problem on one GPU: workspace and stream from PyTorch."""

    def __init__(self, model, horizons, opts=None, device="cuda", stream=None, **prob_kw):
        import torch
        self._torch = torch
        dev = torch.device(device)
        if dev.type != "cuda":
            raise ValueError("the NMPC library runs on a CUDA device only")
        self.device = dev
        with torch.cuda.device(dev):
            self.stream = stream if stream is not None else torch.cuda.current_stream(dev)
            self._p, self._hz = problem(model, horizons, **prob_kw)
            self._p.horizons = self._hz.ctypes.data_as(C.POINTER(C.c_int))
            self._o = opts if opts is not None else options()
            h = _P()
            st = lib().nmpc_build(C.byref(self._p), C.byref(self._o), C.c_void_p(self.stream.cuda_stream), C.byref(h))
            if st != 0:
                raise NmpcError(st, "nmpc_build failed")
            self._h = h
            nbytes = self.workspace_bytes()
            self.workspace = torch.empty(nbytes + 256, dtype=torch.uint8, device=dev)
            base = self.workspace.data_ptr()
            aligned = (base + 255) & ~255
            self._check(lib().nmpc_bind(self._h, C.c_void_p(aligned), C.c_size_t(nbytes)))
        self.n_instances = int(self._hz.size)
        self.dims = [self.instance_dims(i) for i in range(self.n_instances)]

    def _check(self, st):
        if st != 0:
            raise NmpcError(st, lib().nmpc_last_error(self._h).decode())
        return st

    def instance_dims(self, i):
        n, m, T = C.c_int(), C.c_int(), C.c_int()
        lib().nmpc_instance_dims(self._h, i, C.byref(n), C.byref(m), C.byref(T))
        return n.value, m.value, T.value

    def set_params(self, x0=None, setpoint=None, u_prev=None, instance=-1):
        if not (-1 <= instance < self.n_instances):
            raise NmpcError(1, "instance out of range")
        cnt = self.n_instances if instance < 0 else 1
        model = self._p.model
        nx = {0: self._p.N, 1: self._p.g * self._p.g, 2: 1, 3: (self._p.g - 2) ** 2, 4: self._p.N}[model]
        if model == 1:
            sp_total = cnt * nx
        else:
            # all instances: T_i setpoints each, one instance after another
            sp_total = sum(self.dims[i][2] for i in (range(self.n_instances) if instance < 0 else [instance]))
        for a, want, name in ((x0, cnt * nx, "x0"), (setpoint, sp_total, "setpoint"), (u_prev, cnt, "u_prev")):
            if a is not None and _numel(a) != want:
                raise ValueError(f"{name} has {_numel(a)} values, expected {want}")
        ptrs = [_ptr(a) for a in (x0, setpoint, u_prev)]
        flags = {p[1] for p in ptrs if p[0] is not None}
        if len(flags) > 1:
            raise ValueError("mix of host and device parameter arrays")
        on_dev = flags.pop() if flags else 0
        self._check(lib().nmpc_set_params(self._h, instance, ptrs[0][0], ptrs[1][0], ptrs[2][0], on_dev))

    def solve(self, warm=False, raise_on_fail=False):
        infos = (Info * self.n_instances)()
        st = lib().nmpc_solve(self._h, int(bool(warm)), infos)
        if st in (1, 2, 3):
            self._check(st)
        if raise_on_fail and st != 0:
            self._check(st)
        return [{k: getattr(infos[i], k) for k, _ in Info._fields_} for i in range(self.n_instances)]

    def get_solution(self, instance=0, duals=False, out=None):
        """Primal solution (and duals) of one instance, or of all instances
        packed one after another for instance = -1."""
        if instance < 0:
            n, m = sum(d[0] for d in self.dims), sum(d[1] for d in self.dims)
        else:
            n, m, _ = self.dims[instance]
        if out is None:
            y = np.empty(n)
            dv = np.empty(2 * n + 6 * m) if duals else None
        else:
            y, dv = out
            if _numel(y) != n or (dv is not None and _numel(dv) != 2 * n + 6 * m):
                raise ValueError("output buffers have the wrong size")
        py, dy_ = _ptr(y)
        pd = _ptr(dv)[0] if dv is not None else None
        self._check(lib().nmpc_get_solution(self._h, instance, py, pd, dy_))
        if dv is None:
            return y
        return y, unpack_duals(dv, n, m)

    def set_start(self, instance, y, duals=None):
        if instance < 0:
            n, m = sum(d[0] for d in self.dims), sum(d[1] for d in self.dims)
        else:
            n, m, _ = self.dims[instance]
        if _numel(y) != n or (duals is not None and _numel(duals) != 2 * n + 6 * m):
            raise ValueError("start point has the wrong size")
        py, on_dev = _ptr(y)
        pd = _ptr(duals)[0] if duals is not None else None
        self._check(lib().nmpc_set_start(self._h, instance, py, pd, on_dev))

    def trace(self, instance=0):
        cap = self._o.max_iter + 2
        buf = np.zeros(cap * 8)
        k = lib().nmpc_get_trace(self._h, instance, buf.ctypes.data, cap)
        if k < 0:
            raise NmpcError(15, "no trace")
        return buf.reshape(cap, 8)[:k]

    def time_phases(self, reps=10):
        t = PhaseTimes()
        self._check(lib().nmpc_time_phases(self._h, reps, C.byref(t)))
        return {k: getattr(t, k) for k, _ in PhaseTimes._fields_}

    def sensitivity(self, instance, dloss_dy, dx0=None, dsp=None):
        n, m, T = self.dims[instance]
        if _numel(dloss_dy) != n:
            raise ValueError("dloss_dy has the wrong size")
        py, on_dev = _ptr(dloss_dy)
        self._check(lib().nmpc_sensitivity(self._h, instance, py, _ptr(dx0)[0], _ptr(dsp)[0], on_dev))
        return dx0, dsp


def solve_static(model, horizons, x0, setpoint, u_prev, y_out, opts=None, stream=None, **prob_kw):
    """nmpc_solve_static: a one-shot cold solve whose device scratch is the
    library's static workspace (no allocation by the library or the caller
    beyond the given arrays).  Returns (status, infos)."""
    p, hz = problem(model, horizons, **prob_kw)
    p.horizons = hz.ctypes.data_as(C.POINTER(C.c_int))
    o = opts if opts is not None else options()
    infos = (Info * int(hz.size))()
    ptrs = [_ptr(a) for a in (x0, setpoint, u_prev, y_out)]
    flags = {q[1] for q in ptrs if q[0] is not None}
    if len(flags) > 1:
        raise ValueError("mix of host and device arrays")
    on_dev = flags.pop() if flags else 0
    st = lib().nmpc_solve_static(C.byref(p), C.byref(o), stream, ptrs[0][0], ptrs[1][0], ptrs[2][0],
                                 ptrs[3][0], infos, on_dev)
    return st, [{k: getattr(infos[i], k) for k, _ in Info._fields_} for i in range(int(hz.size))]


def debug_recip(x):
    """nmpc_debug_recip: the pivot reciprocal of the factorization applied to a
    float64 CUDA tensor (returns a new tensor)."""
    import torch
    if not (isinstance(x, torch.Tensor) and x.is_cuda and x.dtype == torch.float64 and x.is_contiguous()):
        raise TypeError("a contiguous float64 CUDA tensor is required")
    out = torch.empty_like(x)
    strm = torch.cuda.current_stream(x.device)
    st = lib().nmpc_debug_recip(C.c_void_p(x.data_ptr()), C.c_void_p(out.data_ptr()), x.numel(),
                                C.c_void_p(strm.cuda_stream))
    if st != 0:
        raise NmpcError(st, "nmpc_debug_recip failed")
    return out


def probe_fp64(kind=0, blocks_per_sm=4, iters=20000):
    """nmpc_probe_fp64: measured FP64 TFLOP/s (kind 0: FMA, 1: f64 mma.sync)."""
    import torch
    v = C.c_double()
    st = lib().nmpc_probe_fp64(int(kind), int(blocks_per_sm), int(iters),
                               C.c_void_p(torch.cuda.current_stream().cuda_stream), C.byref(v))
    if st != 0:
        raise NmpcError(st, "nmpc_probe_fp64 failed")
    return v.value


def _numel(a):
    return int(a.size) if isinstance(a, np.ndarray) else int(a.numel())


def unpack_duals(dv, n, m):
    keys = ("zL", "zU", "s_p", "s_m", "w_p", "w_m", "b_p", "b_m")
    lens = (n, n, m, m, m, m, m, m)
    out, o = {}, 0
    for k, ln in zip(keys, lens):
        out[k] = dv[o:o + ln]
        o += ln
    return out
