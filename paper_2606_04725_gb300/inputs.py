"""Seeded synthetic inputs shaped like the paper's workloads.

Only random numbers and fixed recipes live here; none of the method's
arithmetic.  The distillation initial states start from steady states stored
as package data (data/steady_state_N*_Nf*.txt), written once by a committed
script of the test suite that runs the reference CPU implementation.

Recipes (one per workload):
  distillation  x0 = steady state at u_ref = 2.51459 plus N(0, 0.02) noise,
                clipped to [0, 1]; setpoint of x_{k,1} constant over the
                horizon.  N = 12 (feed tray 5, T = 20): setpoint U[0.75, 0.85]
                (the reachable range of x_1 for this column).  N = 34 (feed
                tray 17, T = 200): two setpoints a, b ~ U[0.90, 0.99], the
                closed loop switching between them every 10 re-solves.
  batched       256 columns with N = 34, horizons U{50..200}, per-instance
                seeds for noise and setpoint U[0.90, 0.99].
  paper column  the paper's own column (Sec. 4.1, table distill-params):
                N = 32, feed tray 17, holdups 0.5 / 0.25 / 1.0, dt = 2,
                90 intervals (180 s prediction horizon), stage cost
                (x_1 - 0.8958)^2 + 0.1 (u - 2.51459)^2 per unit time;
                x0 as for the other columns (steady state plus noise).
  plate         target field = sum of 3 Gaussian bumps with amplitude
                U[0.3, 0.8], centre U[0.2, 0.8]^2, width U[0.08, 0.2];
                initial field 0.
  paper plate   the paper's nonlinear plate (Sec. 4.2, table pde-params):
                21 x 21 nodes, dt = 0.08, a 1.0 s prediction horizon
                (12 intervals), the piecewise region setpoint 58 / 55 / 63
                switching at t = 0.5 and 1.5 s of a 3.0 s run; initial field
                T_b = 50 everywhere, cold-start control Q = 50 (its bound).
"""
from __future__ import annotations

import os

import numpy as np

DATA = os.path.join(os.path.dirname(os.path.abspath(__file__)), "data")
U_REF = 2.51459


def steady_state(N: int, Nf: int) -> np.ndarray:
    return np.loadtxt(os.path.join(DATA, f"steady_state_N{N}_Nf{Nf}.txt"))


def distillation_x0(N: int, Nf: int, seed: int) -> np.ndarray:
    rng = np.random.default_rng(seed)
    return np.clip(steady_state(N, Nf) + rng.normal(0.0, 0.02, N), 0.0, 1.0)


def distillation_setpoints(N: int, seed: int) -> tuple[float, float]:
    rng = np.random.default_rng(seed + 1000)
    if N <= 12:
        a = float(rng.uniform(0.75, 0.85))
        return a, a
    a, b = rng.uniform(0.90, 0.99, 2)
    return float(a), float(b)


def setpoint_schedule(a: float, b: float, k: int, switch_every: int = 10) -> float:
    """Setpoint of re-solve k (0-based): a, then b, alternating every block."""
    return a if (k // switch_every) % 2 == 0 else b


def batch_horizons(n: int, lo: int, hi: int, seed: int) -> np.ndarray:
    return np.random.default_rng(seed).integers(lo, hi + 1, n).astype(np.int32)


def batch_distillation(n: int, N: int, Nf: int, seed: int):
    """Per-instance (x0, setpoint) for a batch of columns."""
    x0 = np.stack([distillation_x0(N, Nf, seed * 100003 + i) for i in range(n)])
    sp = np.random.default_rng(seed + 7).uniform(0.90, 0.99, n)
    return x0, sp


def plate_target(g: int, seed: int) -> np.ndarray:
    rng = np.random.default_rng(seed)
    h = 1.0 / g
    c = (np.arange(g) + 0.5) * h
    X, Y = np.meshgrid(c, c)  # X varies along i (fast index), Y along j
    field = np.zeros((g, g))
    for _ in range(3):
        a = rng.uniform(0.3, 0.8)
        cx, cy = rng.uniform(0.2, 0.8, 2)
        s = rng.uniform(0.08, 0.2)
        field += a * np.exp(-((X - cx) ** 2 + (Y - cy) ** 2) / (2 * s * s))
    return field.ravel()


def unit_directions(dim: int, count: int, seed: int) -> np.ndarray:
    d = np.random.default_rng(seed).normal(size=(count, dim))
    return d / np.linalg.norm(d, axis=1, keepdims=True)


def paper_plate_setpoints(t0: float, T: int, dt: float = 0.08) -> np.ndarray:
    """The region setpoint T_sp(t) of eq. (pde-ocp) at the stages
    t0 + k dt, k = 1..T: 58 before 0.5 s, 55 before 1.5 s, 63 after."""
    t = t0 + dt * np.arange(1, T + 1)
    return np.where(t < 0.5, 58.0, np.where(t < 1.5, 55.0, 63.0))


# Workloads by name: sizes as the paper's distillation and heated-plate
# studies scaled per the benchmark configurations.
WORKLOADS = {
    "distillation_N12_T20": dict(model=0, N=12, Nf=5, T=20, resolves=5, seed=1),
    "distillation_N34_T200": dict(model=0, N=34, Nf=17, T=200, resolves=50, seed=2),
    "plate_g64_S8_T50": dict(model=1, g=64, S=8, T=50, resolves=20, seed=3),
    "batch256_distillation_N34_T50_200": dict(model=0, N=34, Nf=17, n_instances=256, T_lo=50, T_hi=200,
                                              resolves=50, seed=4),
    "plate_g128_S16_T100": dict(model=1, g=128, S=16, T=100, resolves=20, seed=5),
    "paper_distillation_N32_T90": dict(model=0, N=32, Nf=17, T=90, resolves=150, seed=6),
    "paper_plate_n21_T12": dict(model=3, g=21, T=12, dt=0.08, resolves=37, t_final=3.0),
}

# The paper's column: problem constants (keyword names of nmpc_problem and
# of the oracle's problem) and the tray-1 setpoint of its parameter table.
PAPER_COLUMN = dict(dt=2.0, Ac=0.5, At=0.25, Ar=1.0, wdu=0.0, wu=0.1, ubar=U_REF)
PAPER_XBAR = 0.8958
