"""Benchmark: NMPC re-solves per second and ms per interior-point iteration at
KKT tolerance 1e-8, parametric (one build, warm start + parameter update)
versus rebuild-every-solve, on the distillation workload of 34 trays,
200 intervals (the closed loop of 50 re-solves switching setpoint every 10).

One step = one NMPC re-solve: parameter update (new initial state = the
predicted state x_1 of the previous solution, new setpoint, u_prev) plus a
warm-started solve to E_0 <= 1e-8, all on the GPU through the C ABI.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

Multi-GPU: one process per GPU (torchrun); each rank solves its own
independently seeded column (instances shard with no exchange): weak scaling.
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

WORKLOAD = "distillation_N34_T200"
METRIC = "NMPC re-solves/sec and ms per IPM iteration at 1e-8 KKT tol, parametric vs rebuild"
UNIT = "re-solves/s"
FP64_DFMA_PER_CLK_PER_SM = 2.0   # GB300: FP64 FMA rate 1/64 of FP32; probe measured 1.9
N_SM = 152
# DRAM bytes (read + write) of one numeric factorization of the workload above:
# the 11 level launches of k_factor_cluster, one ncu capture of the current kernel
# and supernode partition (profiles/k_factor_cluster_distillation_N34_T200.md)
FACTOR_DRAM_BYTES = 17.51e6


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except Exception:
        return {}


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
    return out


class ClockSampler:
    """nvidia-smi samples (every 50 ms) during the timed region; entering waits
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
                                          "--format=csv,noheader,nounits", "-lms", "50"],
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


def rank_seed(wl, rank):
    """Seed of the column a rank solves: every rank gets its own initial state
    (instances shard across ranks with no exchange)."""
    return wl["seed"] + 1000 * rank


def max_over_ranks(x, world, device=None):
    """Largest value of x over the ranks (the job takes as long as its slowest
    rank); x itself when there is one rank."""
    if world <= 1:
        return float(x)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank, seconds, world, device=None):
    """Units all ranks processed over the slowest rank's time."""
    return world * units_per_rank / max_over_ranks(seconds, world, device)


def run_oracle_loop(wl, budget_s, max_steps=None, skip_cold=True):
    """The oracle's closed loop on the same workload (CPU baseline)."""
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


def reference_arm(args):
    rank, world, _ = _dist()
    if rank != 0:
        return
    import paper_2606_04725_gb300.inputs as I
    wl = I.WORKLOADS[WORKLOAD]
    # each step: one warm oracle re-solve (bounded so the run ends in minutes)
    times, iters = run_oracle_loop(wl, budget_s=240.0, max_steps=args.warmup + args.steps)
    t = times[args.warmup:] or times
    v = len(t) / sum(t)
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
            "steps": len(t), "warmup": args.warmup, "ms_per_step": 1e3 * sum(t) / len(t),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": WORKLOAD, "N": wl["N"], "T": wl["T"], "tol": 1e-8},
            "ms_per_ipm_iter": 1e3 * sum(t) / max(1, sum(iters[args.warmup:] or iters)),
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": f"{len(t)} warm re-solves of the closed loop"},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


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
           "kernels": "k_big_diag, k_big_trsm, k_big_update (levels of large fronts); k_factor_cluster (small)",
           "hbm": hbm_rooflines(st, ph)}
    s.close()
    return out


def batch_resolves(P, dev, peak, n_inst=256, resolves=3):
    """Batch of 256 distillation columns (N = 34, T_i ~ U{50..200}) in one
    block-diagonal system: instance re-solves per second over warm re-solves
    of the whole batch (each instance restarted from its measured state), and
    the factorization rate."""
    import torch
    import paper_2606_04725_gb300.inputs as I
    wl = I.WORKLOADS["batch256_distillation_N34_T50_200"]
    hz = I.batch_horizons(n_inst, wl["T_lo"], wl["T_hi"], wl["seed"])
    x0s, sps = I.batch_distillation(n_inst, 34, 17, wl["seed"])
    # schedule chosen by the library's autotuner: one cold batch solve per candidate
    t0 = time.perf_counter()
    opts, rep = P.autotune(P.MODEL_DISTILLATION, hz, x0=np.concatenate(x0s),
                           setpoint=np.concatenate([np.full(T, v) for T, v in zip(hz, sps)]),
                           u_prev=np.full(n_inst, I.U_REF), device=dev, N=34, Nf=17)
    tune_s = time.perf_counter() - t0
    s = P.Solver(P.MODEL_DISTILLATION, hz, N=34, Nf=17, device=dev, opts=opts)
    for i, T in enumerate(hz):
        s.set_params(instance=i, x0=x0s[i], setpoint=np.full(T, sps[i]), u_prev=np.array([I.U_REF]))
    infos = s.solve()
    ok = all(f["status"] == 0 for f in infos)
    ms, iters = [], []
    stream = s.stream
    for _ in range(resolves):
        for i, T in enumerate(hz):
            y = s.get_solution(i)
            s.set_params(instance=i, x0=y[34:68].copy(), setpoint=np.full(T, sps[i]), u_prev=y[68:69].copy())
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        infos = s.solve(warm=True)
        e1.record(stream)
        torch.cuda.synchronize()
        ms.append(e0.elapsed_time(e1))
        iters.append(max(f["iters"] for f in infos))
        ok = ok and all(f["status"] == 0 for f in infos)
    ph = s.time_phases(reps=2)
    st = s.stats()
    tf = st["factor_flops"] / (ph["ms_factor"] * 1e-3) / 1e12
    out = {"workload": "batch256_distillation_N34_T50_200", "instances": n_inst, "n": st["n_total"],
           "instance_resolves_per_s": n_inst * len(ms) / (sum(ms) * 1e-3), "ms_per_batch_resolve": sum(ms) / len(ms),
           "max_ipm_iters_per_batch_resolve": max(iters), "statuses_ok": ok,
           "factor_ms": ph["ms_factor"], "factor_tflops": tf, "factor_frac_of_peak": tf / peak,
           "hbm": hbm_rooflines(st, ph),
           "autotune": {"seconds": tune_s,
                        "chosen": {"ordering": opts.ordering, "nd_leaf": opts.nd_leaf, "panel_scale": opts.panel_scale,
                                   "amalgamation": opts.amalgamation},
                        "ms_per_ipm_iter_by_candidate": [
                            [c["ordering"], c["nd_leaf"], c["panel_scale"], c["amalgamation"], round(c["ms_per_iter"], 3)]
                            for c in rep["candidates"]]}}
    s.close()
    return out


def paper_column_resolves(P, dev, resolves=40, warmup=3):
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
    s = P.Solver(P.MODEL_DISTILLATION, [T], N=N, Nf=Nf, device=dev, **I.PAPER_COLUMN)
    n = s.dims[0][0]
    ox1, ou1 = N, 2 * N
    sp = torch.full((T,), I.PAPER_XBAR, dtype=torch.float64, device=dev)
    y = torch.empty(n, dtype=torch.float64, device=dev)
    s.set_params(x0=I.distillation_x0(N, Nf, wl["seed"]), setpoint=np.full(T, I.PAPER_XBAR),
                 u_prev=np.array([I.U_REF]))
    first = s.solve(warm=False)[0]
    s.get_solution(0, out=(y, None))
    stream = s.stream
    ms, iters, ok = [], [], first["status"] == 0
    for q in range(warmup + resolves):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        s.set_params(x0=y[ox1:ox1 + N], setpoint=sp, u_prev=y[ou1:ou1 + 1])
        inf = s.solve(warm=True)[0]
        s.get_solution(0, out=(y, None))
        e1.record(stream)
        torch.cuda.synchronize()
        ok = ok and inf["status"] == 0
        if q >= warmup:
            ms.append(e0.elapsed_time(e1))
            iters.append(inf["iters"])
    out = {"workload": "paper_distillation_N32_T90", "n": n, "resolves_per_s": len(ms) / (sum(ms) * 1e-3),
           "ms_per_resolve": sum(ms) / len(ms), "ms_per_ipm_iter": sum(ms) / max(1, sum(iters)),
           "ipm_iters_per_resolve": sum(iters) / len(iters), "cold_solve_iters": first["iters"],
           "statuses_ok": ok,
           "paper_gpu_ws_pu_s_per_step": {"value": 0.02, "hardware": "RTX 6000 Ada (MadNLP + cuDSS)",
                                          "note": "context only: other hardware and software"}}
    s.close()
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=47)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--rebuild-steps", type=int, default=3)
    ap.add_argument("--no-plate", action="store_true", help="skip the full-size heated-plate factorization")
    ap.add_argument("--no-batch", action="store_true", help="skip the 256-instance batch")
    ap.add_argument("--no-paper-column", action="store_true", help="skip the paper's own column (N=32, T=90)")
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
    P.build()
    wl = I.WORKLOADS[WORKLOAD]
    N, Nf, T = wl["N"], wl["Nf"], wl["T"]
    seed = rank_seed(wl, rank)
    x0 = I.distillation_x0(N, Nf, seed)
    a, b = I.distillation_setpoints(N, wl["seed"])
    opts = P.options(use_graph=0) if args.host_loop else None
    torch.cuda.synchronize()
    t_build = time.perf_counter()
    s = P.Solver(P.MODEL_DISTILLATION, [T], N=N, Nf=Nf, device=dev, opts=opts)
    build_s = time.perf_counter() - t_build
    n, m, _ = s.dims[0]
    ox1, ou1 = N, 2 * N  # offsets of x_1 and u_1 in y = [x_0 | x_1 u_1 | ...]
    stream = s.stream
    # device-resident inputs: setpoint trajectories and the previous solution
    total = args.warmup + args.steps
    sp_dev = torch.tensor(np.stack([np.full(T, I.setpoint_schedule(a, b, k)) for k in range(total + 1)]),
                          dtype=torch.float64, device=dev)
    y_dev = torch.empty(n, dtype=torch.float64, device=dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    torch.cuda.synchronize()
    t_cold = time.perf_counter()
    s.set_params(x0=x0, setpoint=np.full(T, a), u_prev=np.array([I.U_REF]))
    info0 = s.solve(warm=False)[0]
    assert info0["status"] == 0, info0
    s.get_solution(0, out=(y_dev, None))
    torch.cuda.synchronize()
    cold_s = time.perf_counter() - t_cold

    def step(k, warm=True):
        s.set_params(x0=y_dev[ox1:ox1 + N], setpoint=sp_dev[k], u_prev=y_dev[ou1:ou1 + 1])
        inf = s.solve(warm=warm)[0]
        s.get_solution(0, out=(y_dev, None))
        return inf

    for k in range(1, args.warmup):
        step(k)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    iters, stats_ = [], []
    launches0 = s.stats()["kernel_launches"]
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    wall0 = time.perf_counter()
    with ClockSampler(local) as clk:
        for q in range(args.steps):
            flush.fill_(float(q))                      # L2 flush outside the timed events
            ev[q][0].record(stream)
            inf = step(args.warmup + q)
            ev[q][1].record(stream)
            iters.append(inf["iters"])
            stats_.append(inf["status"])
        torch.cuda.synchronize()
    wall = time.perf_counter() - wall0
    launches = s.stats()["kernel_launches"] - launches0
    ms = [e0.elapsed_time(e1) for e0, e1 in ev]
    tot_ms = max_over_ranks(sum(ms), world, dev)
    value = whole_job_rate(args.steps, tot_ms * 1e-3, world, dev)
    ms_iter = tot_ms / max(1, sum(iters))

    # end to end: host inputs (pinned), host result, copies inside the timed region
    hx = torch.empty(N, dtype=torch.float64).pin_memory()
    hsp = torch.empty(T, dtype=torch.float64).pin_memory()
    hu = torch.empty(1, dtype=torch.float64).pin_memory()
    hy = torch.empty(n, dtype=torch.float64).pin_memory()
    s.get_solution(0, out=(hy, None))
    e2e_steps = min(args.steps, 20)
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for q in range(e2e_steps):
        hx.copy_(hy[ox1:ox1 + N])
        hu[0] = hy[ou1]
        hsp.fill_(I.setpoint_schedule(a, b, args.warmup + args.steps + q))
        s.set_params(x0=hx.numpy(), setpoint=hsp.numpy(), u_prev=hu.numpy())
        s.solve(warm=True)
        s.get_solution(0, out=(hy.numpy(), None))
    torch.cuda.synchronize()
    e2e = whole_job_rate(e2e_steps, time.perf_counter() - t0, world, dev)

    # rebuild-every-solve comparison (paper Base / WS): destroy + build + bind + solve
    rb = {}
    y_prev, du_prev = s.get_solution(0, duals=True)
    for mode in ("cold", "warm"):
        tt = []
        for q in range(args.rebuild_steps):
            torch.cuda.synchronize()
            t1 = time.perf_counter()
            s2 = P.Solver(P.MODEL_DISTILLATION, [T], N=N, Nf=Nf, device=dev)
            s2.set_params(x0=y_prev[ox1:ox1 + N].copy(), setpoint=np.full(T, a), u_prev=y_prev[ou1:ou1 + 1].copy())
            if mode == "warm":
                s2.set_start(0, y_prev, np.concatenate([du_prev[k] for k in ("zL", "zU", "s_p", "s_m", "w_p", "w_m", "b_p", "b_m")]))
            s2.solve(warm=(mode == "warm"))
            torch.cuda.synchronize()
            tt.append(time.perf_counter() - t1)
            s2.close()
            del s2
        rb[mode] = len(tt) / sum(tt)

    # roofline of the dominant kernel (numeric factorization, FP64 FMA bound)
    ph = s.time_phases(reps=20)
    st = s.stats()
    achieved = st["factor_flops"] / (ph["ms_factor"] * 1e-3) / 1e12
    clk = clk.summary()
    peak = N_SM * FP64_DFMA_PER_CLK_PER_SM * 2 * (clk["sm_max_mhz"] or 2070.0) * 1e6 / 1e12
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": tot_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "N": N, "Nf": Nf, "T": T, "n": n, "m": m, "tol": 1e-8,
                       "ordering": ["auto", "natural", "nested_dissection"][st["ordering_used"]],
                       "amalgamation": ["auto", "relaxed", "sibling_limited"][st["amalgamation_used"]],
                       "l2": "flushed between re-solves (256 MB write)"},
            "ms_per_ipm_iter": ms_iter, "ipm_iters_per_resolve": sum(iters) / len(iters),
            "statuses_ok": all(x == 0 for x in stats_),
            "step_ms": {"median": statistics.median(ms), "min": min(ms), "max": max(ms)},
            "closed_loop": {"build_s": build_s, "cold_solve_s": cold_s, "cold_solve_iters": info0["iters"],
                            "resolves": args.steps + 1,
                            "resolves_per_s_incl_build": (args.steps + 1) / (build_s + cold_s + tot_ms * 1e-3)},
            "rebuild": {"cold_resolves_per_s": rb["cold"], "warm_resolves_per_s": rb["warm"],
                        "parametric_over_rebuild_cold": value / rb["cold"]},
            "wall_s_timed": wall,
            "e2e": {"value": e2e, "unit": UNIT, "h2d_bytes_per_step": 8 * (N + T + 1), "d2h_bytes_per_step": 8 * n},
            "gpu_launches": int(launches),
            "phases_ms": {k: ph[k] for k in ("ms_eval", "ms_assemble", "ms_factor", "ms_solve")},
            "hbm": hbm_rooflines(st, ph, latency_bound=True),
            "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                         "frac": achieved / peak, "traffic": FACTOR_DRAM_BYTES,
                         "traffic_basis": "dram__bytes_read.sum + dram__bytes_write.sum of the 11 level launches "
                                          "of one factorization, one ncu capture",
                         "kernel": "k_factor_cluster (the level launches of one numeric factorization)",
                         "flops_per_launch_set": st["factor_flops"],
                         "peak_basis": "152 SMs x 2 FP64 FMA/clock x max SM clock (nominal FP64 rate)"},
            "clocks": clk}
    if not args.no_plate:
        line["plate_full_size"] = plate_factorization(P, dev, peak)
    if not args.no_batch:
        line["batch_256"] = batch_resolves(P, dev, peak)
    if not args.no_paper_column:
        line["paper_column"] = paper_column_resolves(P, dev)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        times, its = run_oracle_loop(wl, budget_s=20.0)
        line["cpu_baseline"] = {"value": len(times) / sum(times), "unit": UNIT, "cores": 1, "kind": "oracle",
                                "sample": f"{len(times)} warm re-solves of the same closed loop (single thread)",
                                "ms_per_ipm_iter": 1e3 * sum(times) / max(1, sum(its))}
    if rank == 0:
        print(json.dumps(line))
    if world > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
