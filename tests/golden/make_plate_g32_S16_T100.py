"""Oracle reference values for the heated plate of the 128 x 128, 16-actuator,
100-interval configuration at the reduced grid g = 32 (S = 16, T = 100,
n = 105,024).  The oracle's band Cholesky is out of reach here (4.5e11 flops
per factorization), so the oracle runs its sparse Cholesky after its own
nested-dissection ordering (linsolve = 1, 1.8e11 flops per factorization,
about three minutes each on one host core: 3.5 hours for the cold solve, about
an hour more for the six re-solves); its results are stored once.

Calls only the oracle (and the seeded input recipes):
  * a cold solve at tol 1e-12 from the zero initial field, target field of
    seed 5: iteration count, objective, scaled optimality error and the primal
    solution at 4096 seeded sample positions;
  * the state-tracking loss l = sum_{k=1..T} dt h^2 |x_k - target|^2 at it;
  * central differences of l along the first three of the 20 seeded unit
    directions (seed 5) in (x0, target), h = 1e-6, from re-solves at tol
    1e-13 warm-started from the tol-1e-12 point (the six re-solves run in
    parallel processes).
Run:  python tests/golden/make_plate_g32_S16_T100.py
"""
import json
import multiprocessing as mp
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(HERE))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))
import oracle as O  # noqa: E402
import paper_2606_04725_gb300.inputs as I  # noqa: E402

G, S, T, SEED = 32, 16, 100, 5
DT = 1.0
H_FD, TOL, TOL_FD = 1e-6, 1e-12, 1e-13
LS = O.LINSOLVE_SPARSE
OUT = os.path.join(HERE, "plate_g32_S16_T100.json")


def tracking_loss(prob, y, target):
    g2 = G * G
    xs = np.stack([y[prob.off_x(k):prob.off_x(k) + g2] for k in range(1, T + 1)])
    return float(np.sum((xs - target) ** 2) * DT / g2)


def fd_leg(args):
    q, sgn, start = args
    x0 = np.zeros(G * G)
    target = I.plate_target(G, seed=SEED)
    dirs = I.unit_directions(2 * G * G, 20, seed=SEED)
    dx, dt = dirs[q, :G * G], dirs[q, G * G:]
    p2 = O.plate(G, S, T, x0 + sgn * H_FD * dx, target + sgn * H_FD * dt, dt=DT)
    st = O.State(p2.n, p2.m)
    for k in O.State.FIELDS:
        getattr(st, k)[:] = start[k]
    s2, i2, _ = O.solve(p2, state=st, warm=True, tol=TOL_FD, linsolve=LS)
    assert i2["status"] == 0, i2
    return q, sgn, tracking_loss(p2, s2.y, target + sgn * H_FD * dt), i2["iters"]


if __name__ == "__main__":
    O.build()
    x0 = np.zeros(G * G)
    target = I.plate_target(G, seed=SEED)
    prob = O.plate(G, S, T, x0.copy(), target.copy(), dt=DT)
    t0 = time.time()
    st, info, _ = O.solve(prob, tol=TOL, linsolve=LS)
    assert info["status"] == 0, info
    print("base solve", info, f"{time.time() - t0:.0f} s", flush=True)
    idx = np.sort(np.random.default_rng(SEED).choice(prob.n, 4096, replace=False))
    start = {k: getattr(st, k).copy() for k in O.State.FIELDS}
    legs = [(q, sgn, start) for q in range(3) for sgn in (+1, -1)]
    with mp.get_context("spawn").Pool(len(legs)) as pool:
        res = pool.map(fd_leg, legs)
    vals = {(q, sgn): v for q, sgn, v, _ in res}
    fd = [(vals[(q, 1)] - vals[(q, -1)]) / (2 * H_FD) for q in range(3)]
    print("fd", fd, "iters", [r[3] for r in res], f"{time.time() - t0:.0f} s", flush=True)
    rec = {"g": G, "S": S, "T": T, "target_seed": SEED, "x0": "zero field", "tol": TOL,
           "oracle_linsolve": "sparse Cholesky, the oracle's nested dissection",
           "iters": info["iters"], "inertia_retries": info["inertia_retries"],
           "objective": info["objective"], "E0_scaled": info["E0_scaled"],
           "loss": tracking_loss(prob, st.y, target),
           "sample_index": idx.tolist(), "sample_y": [float(v) for v in st.y[idx]],
           "fd_h": H_FD, "fd_tol": TOL_FD, "direction_seed": SEED, "directions": 20, "fd_directions": [0, 1, 2],
           "fd": fd, "fd_iters": [r[3] for r in sorted(res)],
           "written_by": "tests/golden/make_plate_g32_S16_T100.py (oracle only)"}
    with open(OUT, "w") as f:
        json.dump(rec, f, indent=0)
    print("wrote", OUT)
