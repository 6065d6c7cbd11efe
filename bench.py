"""Benchmark: NMPC re-solves per second and ms per interior-point iteration at
KKT tolerance 1e-8, parametric vs rebuild, on the batched workload: 256
independent distillation columns (34 trays, feed tray 17) with horizons drawn
from U{50..200}, solved together as one block-diagonal system.

One step = one closed-loop re-solve of the whole batch: the parameter update
of every instance (new initial state = the predicted state x_1 of its
previous solution, its setpoint, u_prev = its previous u_1) in one call, a
warm-started solve of all instances to E_0 <= 1e-8, and the read of all
solutions, through the C ABI.  `value` is instance re-solves per second.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

Multi-GPU: one process per GPU (torchrun).  The batch is split into
contiguous instance ranges balanced by each instance's factorization flops;
each rank builds and solves its range with no exchange (the only collectives
are the barrier and the max/sum of the timings): the total work is fixed.
The reference arm (--impl reference) is the reference CPU implementation of
the method, timed on the same closed loop on all host cores.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD = "batch256_distillation_N34_T50_200"
SINGLE = "distillation_N34_T200"
METRIC = "NMPC re-solves/sec and ms per IPM iteration at 1e-8 KKT tol, parametric vs rebuild"
UNIT = "re-solves/s"
FP64_DFMA_PER_CLK_PER_SM = 2.0   # GB300: FP64 FMA per clock and SM (the probe measures about 1.9)
N_SM = 152


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except Exception:
        return {}


def fp64_nominal_tflops(sm_max_mhz):
    """Nominal FP64 rate: 152 SMs x 2 FMA per clock x 2 flops x the maximum SM clock."""
    return N_SM * FP64_DFMA_PER_CLK_PER_SM * 2 * (sm_max_mhz or 2070.0) * 1e6 / 1e12


def hbm_rooflines(st, ph, latency_bound=False):
    """Achieved bandwidth of the HBM-bound phases against the measured copy
    bandwidth, with algorithmic bytes per iteration: evaluation + assembly move
    8 (n + 5m) (iterate, slacks, multipliers) + 8 nnz(L) (the panels written,
    fill included) + 8 n (right-hand side); the two solves read the factor
    twice, 16 nnz(L).  Times from the phase timing (host-launched, warm)."""
    peak = _peaks().get("hbm_gbs")
    n, m, nnz = st["n_total"], st["m_total"], st["nnz_L"]
    out = {}
    for name, b, ms in (("eval_assembly", 8.0 * (n + 5 * m) + 8.0 * nnz + 8.0 * n, ph["ms_eval"] + ph["ms_assemble"]),
                        ("solves", 16.0 * nnz, ph["ms_solve"])):
        gbs = b / (ms * 1e-3) / 1e9
        out[name] = {"bound": "hbm", "algorithmic_bytes": b, "ms": ms, "achieved": gbs, "unit": "GB/s",
                     "peak": peak, "frac": gbs / peak if peak else None,
                     "peak_basis": "measured copy bandwidth (MEASURED_PEAKS.json hbm_gbs)"}
        if latency_bound:
            out[name]["note"] = "working set L2-resident; latency-bound, not bandwidth-bound"
    # the solves' FP64 work: one multiply-add per factor entry each way (4 nnz(L)
    # flops); on this GPU their bound is FP64 issue and latency rather than HBM
    tf = 4.0 * nnz / (ph["ms_solve"] * 1e-3) / 1e12
    out["solves"]["fp64_tflops"] = tf
    out["solves"]["fp64_frac_of_nominal"] = tf / fp64_nominal_tflops(_peaks().get("sm_max_mhz"))
    return out


class ClockSampler:
    """nvidia-smi samples (every 200 ms) during the timed region; entering waits
    (up to 2 s) for the first sample so that the sampling covers the region."""

    def __init__(self, index=0):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
            t0 = time.perf_counter()
            while not self.lines and time.perf_counter() - t0 < 2.0 and self.proc.poll() is None:
                time.sleep(0.01)
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            p = [x.strip() for x in ln.split(",")]
            if len(p) < 9:
                continue
            try:
                sm.append(float(p[1]))
                mx = float(p[2])
            except ValueError:
                continue
            for nm, v in zip(names, p[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx,
                "reasons": sorted(reasons), "samples": len(sm)}


def _dist():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def _reduce(x, world, op, device=None):
    if world <= 1:
        return float(x)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=op)
    return float(t.item())


def max_over_ranks(x, world, device=None):
    """Largest value of x over the ranks (the job takes as long as its slowest
    rank); x itself when there is one rank."""
    if world <= 1:
        return float(x)
    import torch.distributed as dist
    return _reduce(x, world, dist.ReduceOp.MAX, device)


def sum_over_ranks(x, world, device=None):
    if world <= 1:
        return float(x)
    import torch.distributed as dist
    return _reduce(x, world, dist.ReduceOp.SUM, device)


def whole_job_rate(units_this_rank, seconds, world, device=None):
    """Units all ranks processed over the slowest rank's time."""
    return sum_over_ranks(units_this_rank, world, device) / max_over_ranks(seconds, world, device)


def batch_inputs(wl):
    """Horizons, initial states and setpoints of the batch (seeded)."""
    import paper_2606_04725_gb300.inputs as I
    hz = I.batch_horizons(wl["n_instances"], wl["T_lo"], wl["T_hi"], wl["seed"])
    x0s, sps = I.batch_distillation(wl["n_instances"], wl["N"], wl["Nf"], wl["seed"])
    return hz, x0s, sps


def packed_setpoints(hz, sps):
    return np.concatenate([np.full(int(T), float(v)) for T, v in zip(hz, sps)])


def closed_loop_index(hz, N):
    """Positions of x_1 (N per instance) and u_1 in the packed solutions of
    instances with horizons hz (y_i = [x_0 | x_1 u_1 | ...], n_i = N + T_i (N + 1))."""
    offs = np.concatenate([[0], np.cumsum([N + int(T) * (N + 1) for T in hz])[:-1]])
    ix = (offs[:, None] + N + np.arange(N)[None, :]).ravel()
    iu = offs + 2 * N
    return ix, iu


# --------------------------------------------------------------- CPU legs
def run_oracle_loop(wl, budget_s, max_steps=None, skip_cold=True):
    """The oracle's closed loop on one column (single thread)."""
    import oracle as O
    import paper_2606_04725_gb300.inputs as I
    N, Nf, T, seed = wl["N"], wl["Nf"], wl["T"], wl["seed"]
    x0 = I.distillation_x0(N, Nf, seed)
    a, b = I.distillation_setpoints(N, seed)
    prob = O.distillation(N, Nf, T, x0, np.full(T, a), I.U_REF)
    st, info, _ = O.solve(prob)
    times, iters = [], []
    t_start = time.perf_counter()
    k = 1
    while True:
        if max_steps is not None and len(times) >= max_steps:
            break
        if time.perf_counter() - t_start > budget_s or k >= wl["resolves"] * 4:
            break
        prob.set_params(x0=st.y[prob.off_x(1):prob.off_x(1) + N].copy(), uprev=st.y[prob.off_u(1)],
                        sp=np.full(T, I.setpoint_schedule(a, b, k)))
        t0 = time.perf_counter()
        st, info, _ = O.solve(prob, state=st, warm=True)
        times.append(time.perf_counter() - t0)
        iters.append(info["iters"])
        k += 1
    return times, iters


def host_cores():
    """Cores this process may run on (affinity) and the machine's count."""
    try:
        aff = len(os.sched_getaffinity(0))
    except AttributeError:
        aff = os.cpu_count() or 1
    return aff, os.cpu_count() or aff


def oracle_batch_loop(hz, x0s, sps, N, Nf, steps, threads, instances=None, budget_s=None):
    """The oracle's closed loop on a batch: every instance solved cold, then
    `steps` warm re-solves of all instances, each instance restarted from its
    own previous solution (x0 <- x_1, u_prev <- u_1), as the GPU batch does.
    The instances of a step run on `threads` host threads (the oracle's C
    solver releases the interpreter lock).  Returns per-step seconds, the
    iterations of every re-solve and the cold solves' seconds."""
    from concurrent.futures import ThreadPoolExecutor

    import oracle as O
    import paper_2606_04725_gb300.inputs as I
    idx = list(range(len(hz))) if instances is None else list(instances)
    probs = {i: O.distillation(N, Nf, int(hz[i]), x0s[i].copy(), np.full(int(hz[i]), sps[i]), I.U_REF) for i in idx}
    states = {}

    def cold(i):
        st, info, _ = O.solve(probs[i])
        states[i] = st
        return info["iters"]

    def warm(i):
        p, st = probs[i], states[i]
        p.set_params(x0=st.y[p.off_x(1):p.off_x(1) + N].copy(), uprev=st.y[p.off_u(1)])
        st, info, _ = O.solve(p, state=st, warm=True)
        states[i] = st
        return info["iters"]

    with ThreadPoolExecutor(max_workers=threads) as ex:
        t0 = time.perf_counter()
        list(ex.map(cold, idx))
        cold_s = time.perf_counter() - t0
        times, iters = [], []
        for _ in range(steps):
            if budget_s is not None and times and sum(times) > budget_s:
                break
            t0 = time.perf_counter()
            its = list(ex.map(warm, idx))
            times.append(time.perf_counter() - t0)
            iters.append(its)
    return times, iters, cold_s


def reference_arm(args):
    """--impl reference: the reference CPU implementation on the same batch
    and closed loop, all host cores (rank 0 only under torchrun)."""
    rank, world, _ = _dist()
    if rank != 0:
        return
    import paper_2606_04725_gb300.inputs as I
    wl = I.WORKLOADS[WORKLOAD]
    hz, x0s, sps = batch_inputs(wl)
    cores, ncpu = host_cores()
    times, iters, cold_s = oracle_batch_loop(hz, x0s, sps, wl["N"], wl["Nf"], args.warmup + args.steps, cores)
    t = times[args.warmup:] or times
    its = [i for step in (iters[args.warmup:] or iters) for i in step]
    ni = len(hz)
    v = ni * len(t) / sum(t)
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
            "steps": len(t), "warmup": args.warmup, "ms_per_step": 1e3 * sum(t) / len(t),
            "higher_is_better": True, "scaling": "strong", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": WORKLOAD, "instances": ni, "N": wl["N"], "Nf": wl["Nf"],
                                            "T_range": [wl["T_lo"], wl["T_hi"]], "tol": 1e-8},
            "cpu_ms_per_instance_ipm_iter": 1e3 * sum(t) * cores / max(1, sum(its)),
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": f"the whole batch ({ni} instances), {len(t)} warm closed-loop re-solves after "
                                       f"{args.warmup} untimed ones, instances spread over {cores} threads "
                                       f"(affinity {cores} of {ncpu} cores)",
                             "cold_solve_s": cold_s},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


# --------------------------------------------------------------- GPU legs
def single_column(P, dev, steps=30, warmup=3, rank=0):
    """The N = 34, T = 200 column alone (its closed loop of warm re-solves,
    setpoint switching every 10): re-solves per second with inputs on the
    device, per-phase times and the roofline of its factorization."""
    import torch
    import paper_2606_04725_gb300.inputs as I
    wl = I.WORKLOADS[SINGLE]
    N, Nf, T = wl["N"], wl["Nf"], wl["T"]
    x0 = I.distillation_x0(N, Nf, wl["seed"] + 1000 * rank)
    a, b = I.distillation_setpoints(N, wl["seed"])
    s = P.Solver(P.MODEL_DISTILLATION, [T], N=N, Nf=Nf, device=dev)
    n = s.dims[0][0]
    sp = torch.tensor(np.stack([np.full(T, I.setpoint_schedule(a, b, k)) for k in range(warmup + steps + 1)]),
                      dtype=torch.float64, device=dev)
    y = torch.empty(n, dtype=torch.float64, device=dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    s.set_params(x0=x0, setpoint=np.full(T, a), u_prev=np.array([I.U_REF]))
    first = s.solve(warm=False)[0]
    s.get_solution(0, out=(y, None))
    ms, iters, ok = [], [], first["status"] == 0
    for q in range(warmup + steps):
        flush.fill_(float(q))
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(s.stream)
        s.set_params(x0=y[N:2 * N], setpoint=sp[q + 1], u_prev=y[2 * N:2 * N + 1])
        inf = s.solve(warm=True)[0]
        s.get_solution(0, out=(y, None))
        e1.record(s.stream)
        torch.cuda.synchronize()
        ok = ok and inf["status"] == 0
        if q >= warmup:
            ms.append(e0.elapsed_time(e1))
            iters.append(inf["iters"])
    # rebuild every re-solve (the paper's Base: cold; its WS: warm) on the same GPU
    rb = {}
    y_prev, du_prev = s.get_solution(0, duals=True)
    for mode in ("cold", "warm"):
        tt = []
        for _ in range(3):
            torch.cuda.synchronize()
            t1 = time.perf_counter()
            s2 = P.Solver(P.MODEL_DISTILLATION, [T], N=N, Nf=Nf, device=dev)
            s2.set_params(x0=y_prev[N:2 * N].copy(), setpoint=np.full(T, a), u_prev=y_prev[2 * N:2 * N + 1].copy())
            if mode == "warm":
                s2.set_start(0, y_prev, np.concatenate([du_prev[k] for k in ("zL", "zU", "s_p", "s_m", "w_p", "w_m", "b_p", "b_m")]))
            s2.solve(warm=(mode == "warm"))
            torch.cuda.synchronize()
            tt.append(time.perf_counter() - t1)
            s2.close()
        rb[mode] = len(tt) / sum(tt)
    ph = s.time_phases(reps=20)
    st = s.stats()
    v = len(ms) / (sum(ms) * 1e-3)
    out = {"workload": SINGLE, "n": n, "resolves_per_s": v, "ms_per_resolve": sum(ms) / len(ms),
           "ms_per_ipm_iter": sum(ms) / max(1, sum(iters)), "ipm_iters_per_resolve": sum(iters) / len(iters),
           "cold_solve_iters": first["iters"], "statuses_ok": ok,
           "ordering": ["auto", "natural", "nested_dissection", "two_sided"][st["ordering_used"]],
           "phases_ms": {k: ph[k] for k in ("ms_eval", "ms_assemble", "ms_factor", "ms_solve")},
           "factor_flops": st["factor_flops"], "factor_tflops": st["factor_flops"] / (ph["ms_factor"] * 1e-3) / 1e12,
           "hbm": hbm_rooflines(st, ph, latency_bound=True),
           "rebuild": {"cold_resolves_per_s": rb["cold"], "warm_resolves_per_s": rb["warm"],
                       "parametric_over_rebuild_cold": v / rb["cold"]}}
    s.close()
    return out


def plate_factorization(P, dev, peak):
    """Heated plate at full size (g = 64, S = 8, T = 50; n = 209,296): the
    large-front path.  Two interior-point iterations give an iterate, then one
    numeric factorization and one pair of solves are timed with CUDA events."""
    import paper_2606_04725_gb300.inputs as I
    g, S, T = 64, 8, 50
    s = P.Solver(P.MODEL_PLATE, [T], g=g, S=S, device=dev, opts=P.options(max_iter=2))
    s.set_params(x0=np.zeros(g * g), setpoint=I.plate_target(g, seed=3))
    s.solve()
    ph = s.time_phases(reps=2)
    st = s.stats()
    tf = st["factor_flops"] / (ph["ms_factor"] * 1e-3) / 1e12
    out = {"workload": "plate_g64_S8_T50", "n": st["n_total"], "max_front": st["max_front"],
           "factor_flops": st["factor_flops"], "factor_ms": ph["ms_factor"], "solve_ms": ph["ms_solve"],
           "factor_tflops": tf, "factor_frac_of_peak": tf / peak,
           "workspace_bytes": st["workspace_bytes"],
           "kernels": "k_big_diag, k_big_trsm, k_big_update (levels of large fronts); small fronts below them",
           "hbm": hbm_rooflines(st, ph)}
    s.close()
    return out


def plate_closed_loop(P, dev, resolves):
    """Heated plate at full size (g = 64, S = 8, T = 50; n = 209,296) in
    closed loop: a cold solve from the zero field (target of seed 3), then
    `resolves` warm re-solves, each from the previous solution's x_1 (the
    state one interval later) with the same target.  Re-solves/s and ms per
    interior-point iteration from CUDA events around each re-solve."""
    import torch
    import paper_2606_04725_gb300.inputs as I
    g, S, T = 64, 8, 50
    g2 = g * g
    s = P.Solver(P.MODEL_PLATE, [T], g=g, S=S, device=dev)
    target = I.plate_target(g, seed=3)
    s.set_params(x0=np.zeros(g2), setpoint=target)
    t0 = time.perf_counter()
    cold = s.solve()[0]
    torch.cuda.synchronize()
    cold_s = time.perf_counter() - t0
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ms, iters, ok = [], [], cold["status"] == 0
    for _ in range(resolves):
        y = s.get_solution(0)
        s.set_params(x0=y[g2:2 * g2].copy(), setpoint=target)  # x_1: the first stage after x_0
        ev0.record(torch.cuda.current_stream())
        info = s.solve(warm=True)[0]
        ev1.record(torch.cuda.current_stream())
        torch.cuda.synchronize()
        ms.append(ev0.elapsed_time(ev1))
        iters.append(info["iters"])
        ok = ok and info["status"] == 0
    s.close()
    tot = sum(ms)
    return {"workload": "plate_g64_S8_T50_closed_loop", "resolves": resolves,
            "resolves_per_s": resolves / (tot * 1e-3), "ms_per_resolve": tot / resolves,
            "ms_per_ipm_iter": tot / max(1, sum(iters)), "ipm_iters_per_resolve": sum(iters) / resolves,
            "cold_solve_s": cold_s, "cold_solve_iters": cold["iters"], "statuses_ok": ok,
            "note": "x0 <- x_1 of the previous solution, target fixed; CUDA events around each warm re-solve"}


def plate_g128_iteration(P, dev, peak):
    """The 128 x 128 plate with 16 actuators and 100 intervals (n = 1,656,384):
    analysis and binding, then one interior-point iteration from the cold
    start, with its factorization and solves timed by the phase timer.  A
    whole cold solve takes 50 to 60 such iterations."""
    import torch
    import paper_2606_04725_gb300.inputs as I
    g, S, T = 128, 16, 100
    t0 = time.perf_counter()
    s = P.Solver(P.MODEL_PLATE, [T], g=g, S=S, device=dev, opts=P.options(max_iter=1))
    build_s = time.perf_counter() - t0
    s.set_params(x0=np.zeros(g * g), setpoint=I.plate_target(g, seed=5))
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    info = s.solve()[0]
    torch.cuda.synchronize()
    it_s = time.perf_counter() - t0
    ph = s.time_phases(reps=1)
    st = s.stats()
    tf = st["factor_flops"] / (ph["ms_factor"] * 1e-3) / 1e12
    out = {"workload": "plate_g128_S16_T100", "n": st["n_total"], "max_front": st["max_front"],
           "nnz_L": st["nnz_L"], "factor_flops": st["factor_flops"], "workspace_bytes": st["workspace_bytes"],
           "build_and_bind_s": build_s, "first_iteration_s": it_s, "iters": info["iters"],
           "factor_ms": ph["ms_factor"], "solve_ms": ph["ms_solve"], "eval_ms": ph["ms_eval"],
           "assemble_ms": ph["ms_assemble"], "factor_tflops": tf, "factor_frac_of_peak": tf / peak}
    s.close()
    return out


def paper_column_resolves(P, dev, resolves=40, warmup=3, model=None, kkt=0):
    """The paper's own column and cost (N = 32, feed tray 17, holdups 0.5 /
    0.25 / 1.0, dt = 2, 90 intervals, (x_1 - xbar)^2 + 0.1 (u - ubar)^2):
    warm re-solves of its closed loop with inputs resident on the device,
    each timed with CUDA events on the library stream.  The paper's figure
    for this workload is its per-step GPU solve time with warm start and
    parameter update, on other hardware (context, not a target)."""
    import torch
    import paper_2606_04725_gb300.inputs as I
    wl = I.WORKLOADS["paper_distillation_N32_T90"]
    N, Nf, T = wl["N"], wl["Nf"], wl["T"]
    model = P.MODEL_DISTILLATION if model is None else model
    cu = N if model == P.MODEL_DISTILLATION_DAE else 0  # u within a stage's control block
    s = P.Solver(model, [T], N=N, Nf=Nf, device=dev, opts=P.options(kkt=kkt), **I.PAPER_COLUMN)
    n = s.dims[0][0]
    sp = torch.full((T,), I.PAPER_XBAR, dtype=torch.float64, device=dev)
    y = torch.empty(n, dtype=torch.float64, device=dev)
    s.set_params(x0=I.distillation_x0(N, Nf, wl["seed"]), setpoint=np.full(T, I.PAPER_XBAR),
                 u_prev=np.array([I.U_REF]))
    first = s.solve(warm=False)[0]
    s.get_solution(0, out=(y, None))
    ms, iters, cgs, ok = [], [], [], first["status"] == 0
    for q in range(warmup + resolves):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(s.stream)
        s.set_params(x0=y[N:2 * N], setpoint=sp, u_prev=y[2 * N + cu:2 * N + cu + 1])
        inf = s.solve(warm=True)[0]
        s.get_solution(0, out=(y, None))
        e1.record(s.stream)
        torch.cuda.synchronize()
        ok = ok and inf["status"] == 0
        if q >= warmup:
            ms.append(e0.elapsed_time(e1))
            iters.append(inf["iters"])
            cgs.append(inf["cg_iters"])
    name = "paper_distillation_N32_T90" + ("_dae" if cu else "") + ("_hykkt" if kkt else "")
    out = {"workload": name, "n": n, "resolves_per_s": len(ms) / (sum(ms) * 1e-3),
           "ms_per_resolve": sum(ms) / len(ms), "ms_per_ipm_iter": sum(ms) / max(1, sum(iters)),
           "ipm_iters_per_resolve": sum(iters) / len(iters), "cold_solve_iters": first["iters"],
           "statuses_ok": ok,
           "paper_gpu_ws_pu_s_per_step": {"value": 0.02, "hardware": "RTX 6000 Ada (MadNLP + cuDSS)",
                                          "note": "context only: other hardware and software"}}
    if kkt:
        out["kkt"] = "hykkt"
        out["cg_iters_per_resolve"] = sum(cgs) / len(cgs)
        out["cold_solve_cg_iters"] = first["cg_iters"]
    s.close()
    return out


def paper_plate_resolves(P, dev, warmup=3, kkt=0):
    """The paper's nonlinear heated plate (Sec. 4.2: 21 x 21 nodes, dt =
    0.08, 12 intervals) over its 3.0 s closed loop (37 warm re-solves after
    the cold one, the region setpoint stepping 58 / 55 / 63), each re-solve
    timed with CUDA events on the library stream with its inputs on the
    device; and one rebuild-every-solve re-solve (the paper's Base) for
    comparison.  The paper's per-step figures are on other hardware (context)."""
    import torch
    import paper_2606_04725_gb300.inputs as I
    wl = I.WORKLOADS["paper_plate_n21_T12"]
    n, T, dt = wl["g"], wl["T"], wl["dt"]
    nx = (n - 2) ** 2
    s = P.Solver(P.MODEL_PAPER_PLATE, [T], g=n, device=dev, opts=P.options(kkt=kkt))
    nv = s.dims[0][0]
    y = torch.empty(nv, dtype=torch.float64, device=dev)
    u0 = torch.full((1,), 50.0, dtype=torch.float64, device=dev)
    steps = int(round(wl["t_final"] / dt))
    sps = torch.tensor(np.stack([I.paper_plate_setpoints(k * dt, T, dt) for k in range(steps + warmup + 1)]),
                       dtype=torch.float64, device=dev)
    s.set_params(x0=np.full(nx, 50.0), setpoint=I.paper_plate_setpoints(0.0, T, dt), u_prev=np.array([50.0]))
    t0 = time.perf_counter()
    first = s.solve(warm=False)[0]
    cold_s = time.perf_counter() - t0
    s.get_solution(0, out=(y, None))
    ms, iters, cgs, ok = [], [], [], first["status"] == 0
    for k in range(1, steps + 1):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(s.stream)
        s.set_params(x0=y[nx:2 * nx], setpoint=sps[k], u_prev=u0)
        inf = s.solve(warm=True)[0]
        s.get_solution(0, out=(y, None))
        e1.record(s.stream)
        torch.cuda.synchronize()
        ok = ok and inf["status"] == 0
        ms.append(e0.elapsed_time(e1))
        iters.append(inf["iters"])
        cgs.append(inf["cg_iters"])
    yh = y.cpu().numpy()
    torch.cuda.synchronize()
    t1 = time.perf_counter()
    s2 = P.Solver(P.MODEL_PAPER_PLATE, [T], g=n, device=dev, opts=P.options(kkt=kkt))
    s2.set_params(x0=yh[nx:2 * nx].copy(), setpoint=I.paper_plate_setpoints(steps * dt, T, dt), u_prev=np.array([50.0]))
    rb = s2.solve(warm=False)[0]
    torch.cuda.synchronize()
    rebuild_s = time.perf_counter() - t1
    s2.close()
    ph = s.time_phases(reps=5)
    out = {"workload": "paper_plate_n21_T12" + ("_hykkt" if kkt else ""), "n": nv, "resolves": len(ms),
           "resolves_per_s": len(ms) / (sum(ms) * 1e-3), "ms_per_resolve": sum(ms) / len(ms),
           "ms_per_ipm_iter": sum(ms) / max(1, sum(iters)), "ipm_iters_per_resolve": sum(iters) / len(iters),
           "cold_solve_iters": first["iters"], "cold_solve_s": cold_s, "statuses_ok": ok and rb["status"] == 0,
           "rebuild_cold_s_per_resolve": rebuild_s, "phases_ms": {k: ph[k] for k in ("ms_eval", "ms_assemble",
                                                                                      "ms_factor", "ms_solve")},
           "paper_gpu_s_per_step": {"ws_pu": 0.06, "base": 0.97, "hardware": "RTX 6000 Ada (MadNLP + cuDSS)",
                                    "note": "context only: other hardware and software"}}
    if kkt:
        out["kkt"] = "hykkt"
        out["cg_iters_per_resolve"] = sum(cgs) / len(cgs)
        out["cold_solve_cg_iters"] = first["cg_iters"]
    s.close()
    return out


# DRAM bytes (read + write) of one k_factor_flow launch measured by ncu on the
# first 64 instances of the batch (profiles/k_factor_flow_batch64_distillation_N34_T50_200.md),
# with the flops of that case; the traffic grows with the instances as the flops do.
FLOW64_DRAM_BYTES, FLOW64_FLOPS = 494.803712e6 + 368.445184e6, 1971262569.0


def flow_traffic(opts, st):
    """DRAM bytes per factorization for the schedule the capture was taken
    with (nested dissection, leaves of one stage, sibling-limited supernodes,
    the dataflow factorization), scaled to this batch by its flops; None for
    any other schedule."""
    same = (st["ordering_used"] == 2 and opts.nd_leaf == 1 and st["amalgamation_used"] == 2
            and opts.factor_mode == 3)
    return FLOW64_DRAM_BYTES * st["factor_flops"] / FLOW64_FLOPS if same else None


def fp64_probe(P):
    """Measured FP64 rates of this GPU (library probe kernels): FMA chains and
    the f64 tensor-core mma.sync, four 256-thread blocks per SM."""
    return {"dfma_tflops": P._lib.probe_fp64(0, 4, 20000), "dmma_tflops": P._lib.probe_fp64(1, 4, 4000),
            "note": "independent accumulators on every thread (FMA) or warp (mma.sync m8n8k4); one timed launch"}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the single column, the full-size plate, the paper's column and plate, and the "
                         "rebuild variants")
    ap.add_argument("--schedule", default="",
                    help="fixed options instead of the autotuner's, e.g. ordering=2,nd_leaf=1,amalgamation=2,"
                         "panel_scale=3,factor_mode=3 (for profiling runs)")
    ap.add_argument("--instances", type=int, default=0,
                    help="solve only the first K instances of the batch (smaller profiling cases)")
    ap.add_argument("--no-probe", action="store_true", help="skip the FP64 throughput probe")
    ap.add_argument("--plate-closed-loop", type=int, default=0,
                    help="also run the 64x64 plate's closed loop with this many warm re-solves")
    ap.add_argument("--plate-g128", action="store_true",
                    help="also time one interior-point iteration of the 128 x 128 plate (S = 16, T = 100)")
    ap.add_argument("--host-loop", action="store_true",
                    help="drive the interior-point loop from the host instead of the conditional graph "
                         "(same kernels; for profilers that cannot see into conditional graphs)")
    args = ap.parse_args()
    if args.impl == "reference":
        reference_arm(args)
        return
    rank, world, local = _dist()
    import torch
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    import paper_2606_04725_gb300 as P
    import paper_2606_04725_gb300.inputs as I
    from paper_2606_04725_gb300.partition import instance_weights, rank_slice
    P.build()
    wl = I.WORKLOADS[WORKLOAD]
    N, Nf = wl["N"], wl["Nf"]
    hz_all, x0s_all, sps_all = batch_inputs(wl)
    if args.instances > 0:
        hz_all, x0s_all, sps_all = hz_all[:args.instances], x0s_all[:args.instances], sps_all[:args.instances]
    # contiguous instance ranges balanced by factorization flops (one range per rank)
    weights = instance_weights(P.MODEL_DISTILLATION, hz_all, N=N, Nf=Nf)
    i0, i1 = rank_slice(weights, rank, world)
    hz, x0s, sps = hz_all[i0:i1], x0s_all[i0:i1], sps_all[i0:i1]
    ni = len(hz)
    sp_host = packed_setpoints(hz, sps)
    # the schedule (ordering, amalgamation, solve form) chosen by the library's autotuner
    t0 = time.perf_counter()
    if args.schedule:
        opts = P.options(**{k: int(v) for k, v in (kv.split("=") for kv in args.schedule.split(","))})
        rep = {"candidates": []}
    else:
        opts, rep = P.autotune(P.MODEL_DISTILLATION, hz, x0=x0s.ravel().copy(), setpoint=sp_host,
                               u_prev=np.full(ni, I.U_REF), device=dev, N=N, Nf=Nf)
    tune_s = time.perf_counter() - t0
    if args.host_loop:
        opts.use_graph = 0
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    s = P.Solver(P.MODEL_DISTILLATION, hz, N=N, Nf=Nf, device=dev, opts=opts)
    build_s = time.perf_counter() - t0
    n_tot = sum(d[0] for d in s.dims)
    ix_h, iu_h = closed_loop_index(hz, N)
    ix, iu = torch.tensor(ix_h, device=dev), torch.tensor(iu_h, device=dev)
    SP = torch.tensor(sp_host, dtype=torch.float64, device=dev)
    X0 = torch.tensor(x0s.ravel(), dtype=torch.float64, device=dev)
    U = torch.full((ni,), I.U_REF, dtype=torch.float64, device=dev)
    Y = torch.empty(n_tot, dtype=torch.float64, device=dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    s.set_params(x0=X0, setpoint=SP, u_prev=U)
    infos = s.solve(warm=False)
    s.get_solution(-1, out=(Y, None))
    torch.cuda.synchronize()
    cold_s = time.perf_counter() - t0
    cold_ok = all(f["status"] == 0 for f in infos)
    cold_iters = max(f["iters"] for f in infos)

    def step():
        # closed loop on the device: x0 <- x_1, u_prev <- u_1 of every instance
        torch.index_select(Y, 0, ix, out=X0)
        torch.index_select(Y, 0, iu, out=U)
        s.set_params(x0=X0, setpoint=SP, u_prev=U)
        inf = s.solve(warm=True)
        s.get_solution(-1, out=(Y, None))
        return inf

    for _ in range(args.warmup):
        step()
    # the primal-dual point the timed steps start from: the end-to-end steps
    # below restart from it, so that both time the same closed-loop re-solves
    m_tot = sum(d[1] for d in s.dims)
    Y0 = Y.clone()
    D0 = torch.empty(2 * n_tot + 6 * m_tot, dtype=torch.float64, device=dev)
    s.get_solution(-1, out=(torch.empty_like(Y), D0))
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    batch_iters, mean_iters, ok = [], [], cold_ok
    launches0 = s.stats()["kernel_launches"]
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    wall0 = time.perf_counter()
    with ClockSampler(local) as clk:
        for q in range(args.steps):
            flush.fill_(float(q))                      # L2 flush outside the timed events
            ev[q][0].record(s.stream)
            inf = step()
            ev[q][1].record(s.stream)
            batch_iters.append(max(f["iters"] for f in inf))
            mean_iters.append(sum(f["iters"] for f in inf) / ni)
            ok = ok and all(f["status"] == 0 for f in inf)
        torch.cuda.synchronize()
    wall = time.perf_counter() - wall0
    launches = s.stats()["kernel_launches"] - launches0
    ms = [e0.elapsed_time(e1) for e0, e1 in ev]
    tot_ms = max_over_ranks(sum(ms), world, dev)
    value = whole_job_rate(ni * args.steps, tot_ms * 1e-3, world, dev)

    # end to end through the C ABI with host buffers: the parameters of every
    # instance copied in and every solution copied out inside the timed region;
    # the same closed-loop steps as the timed ones, from the same point
    X0h = torch.empty(ni * N, dtype=torch.float64).pin_memory()
    Uh = torch.empty(ni, dtype=torch.float64).pin_memory()
    SPh = torch.tensor(sp_host, dtype=torch.float64).pin_memory()
    Yh = torch.empty(n_tot, dtype=torch.float64).pin_memory()
    s.set_start(-1, Y0, D0)
    Yh.copy_(Y0)
    e2e_steps = args.steps
    e2e_s = 0.0
    if world > 1:
        torch.distributed.barrier()
    for q in range(e2e_steps):
        flush.fill_(float(q))
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        yh = Yh.numpy()
        np.take(yh, ix_h, out=X0h.numpy())
        np.take(yh, iu_h, out=Uh.numpy())
        s.set_params(x0=X0h.numpy(), setpoint=SPh.numpy(), u_prev=Uh.numpy())
        s.solve(warm=True)
        s.get_solution(-1, out=(yh, None))
        e2e_s += time.perf_counter() - t0
    e2e = whole_job_rate(ni * e2e_steps, e2e_s, world, dev)

    # roofline of the dominant kernel: the numeric factorization, FP64-bound
    ph = s.time_phases(reps=5)
    st = s.stats()
    clk = clk.summary()
    peak = fp64_nominal_tflops(clk["sm_max_mhz"])
    achieved = st["factor_flops"] / (ph["ms_factor"] * 1e-3) / 1e12
    probe = fp64_probe(P) if not args.no_probe else {}
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": tot_ms / args.steps, "higher_is_better": True,
            "scaling": "strong", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "instances": len(hz_all), "instances_this_rank": ni,
                       "N": N, "Nf": Nf, "T_range": [wl["T_lo"], wl["T_hi"]], "n": n_tot, "tol": 1e-8,
                       "ordering": ["auto", "natural", "nested_dissection", "two_sided"][st["ordering_used"]],
                       "nd_leaf": opts.nd_leaf, "amalgamation": opts.amalgamation, "panel_scale": opts.panel_scale,
                       "factor_mode": opts.factor_mode,
                       "l2": "flushed between re-solves (256 MB write); the batch's workspace is larger than L2"},
            "ms_per_ipm_iter": sum(ms) / max(1, sum(batch_iters)),
            "ipm_iters_per_resolve": {"batch": sum(batch_iters) / len(batch_iters),
                                      "instance_mean": sum(mean_iters) / len(mean_iters)},
            "statuses_ok": ok,
            "step_ms": {"median": statistics.median(ms), "min": min(ms), "max": max(ms)},
            "closed_loop": {"autotune_s": tune_s, "build_s": build_s, "cold_solve_s": cold_s,
                            "cold_solve_iters": cold_iters, "resolves": args.warmup + args.steps,
                            "instance_resolves_per_s_incl_build":
                                ni * (args.warmup + args.steps + 1) / (build_s + cold_s + tot_ms * 1e-3 * (args.warmup + args.steps) / args.steps)},
            "wall_s_timed": wall,
            "e2e": {"value": e2e, "unit": UNIT, "h2d_bytes_per_step": 8 * (ni * N + sp_host.size + ni),
                    "d2h_bytes_per_step": 8 * n_tot},
            "gpu_launches": int(launches),
            "phases_ms": {k: ph[k] for k in ("ms_eval", "ms_assemble", "ms_factor", "ms_solve")},
            "hbm": hbm_rooflines(st, ph),
            "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                         "frac": achieved / peak, "traffic": flow_traffic(opts, st),
                         "kernel": "numeric factorization of the whole batch (the launches of one factorization)",
                         "flops_per_launch_set": st["factor_flops"],
                         "peak_basis": "152 SMs x 2 FP64 FMA/clock x max SM clock (nominal FP64 rate)",
                         "frac_of_measured_dfma": achieved / probe["dfma_tflops"] if probe else None},
            "fp64_probe": probe,
            "autotune": {"seconds": tune_s,
                         "columns": ["ordering", "nd_leaf", "panel_scale", "amalgamation", "factor_mode",
                                     "ms_per_full_iteration", "ms_per_closed_loop_resolve"],
                         "candidates": [[c["ordering"], c["nd_leaf"], c["panel_scale"], c["amalgamation"],
                                         c["factor_mode"], round(c["ms_per_iter"], 3), round(c["ms_resolve"], 3)]
                                        for c in rep["candidates"]]},
            "clocks": clk}
    if not args.no_extras:
        t0 = time.perf_counter()
        rb = {}
        y_prev, du_prev = s.get_solution(-1, duals=True)
        for mode in ("cold", "warm"):
            torch.cuda.synchronize()
            t1 = time.perf_counter()
            s2 = P.Solver(P.MODEL_DISTILLATION, hz, N=N, Nf=Nf, device=dev, opts=opts)
            s2.set_params(x0=np.ascontiguousarray(y_prev[ix_h]), setpoint=sp_host,
                          u_prev=np.ascontiguousarray(y_prev[iu_h]))
            if mode == "warm":
                s2.set_start(-1, y_prev, np.concatenate([du_prev[k] for k in ("zL", "zU", "s_p", "s_m", "w_p",
                                                                                 "w_m", "b_p", "b_m")]))
            s2.solve(warm=(mode == "warm"))
            torch.cuda.synchronize()
            rb[mode] = ni / (time.perf_counter() - t1)
            s2.close()
        line["rebuild"] = {"cold_resolves_per_s": rb["cold"], "warm_resolves_per_s": rb["warm"],
                           "parametric_over_rebuild_cold": value / rb["cold"] if world == 1 else None,
                           "note": "destroy + analysis + bind + solve of the whole batch per re-solve, one each"}
    s.close()
    del flush
    if args.plate_g128:
        line["plate_g128"] = plate_g128_iteration(P, dev, peak)
    if args.plate_closed_loop > 0:
        line["plate_closed_loop"] = plate_closed_loop(P, dev, args.plate_closed_loop)
    if not args.no_extras:
        line["single_column"] = single_column(P, dev, rank=rank)
        line["plate_full_size"] = plate_factorization(P, dev, peak)
        line["paper_column"] = paper_column_resolves(P, dev)
        line["paper_column_dae"] = paper_column_resolves(P, dev, model=P.MODEL_DISTILLATION_DAE)
        line["paper_plate"] = paper_plate_resolves(P, dev)
        # the HyKKT form of the Newton system on the paper's two workloads
        line["hykkt"] = {"paper_column": paper_column_resolves(P, dev, kkt=1),
                         "paper_plate": paper_plate_resolves(P, dev, kkt=1)}
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cores, ncpu = host_cores()
        t_all, it_all, cold_all = oracle_batch_loop(hz, x0s, sps, N, Nf, 3, cores)
        sample = list(range(0, ni, 32))
        t_one, it_one, _ = oracle_batch_loop(hz, x0s, sps, N, Nf, 3, 1, instances=sample)
        line["cpu_baseline"] = {"value": ni * len(t_all) / sum(t_all), "unit": UNIT, "cores": cores, "kind": "oracle",
                                "sample": f"the whole batch ({ni} instances): cold solves ({cold_all:.1f} s), then "
                                          f"{len(t_all)} warm closed-loop re-solves, instances over {cores} threads "
                                          f"(affinity {cores} of {ncpu} cores)",
                                "single_thread": {"value": len(sample) * len(t_one) / sum(t_one), "unit": UNIT,
                                                  "cores": 1,
                                                  "sample": f"{len(sample)} instances (every 32nd), {len(t_one)} "
                                                            f"warm closed-loop re-solves each"}}
    if rank == 0:
        print(json.dumps(line))
    if world > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
