"""Write the distillation steady states used as the base of the seeded initial
states (x0 = steady state + N(0, 0.02) noise, clipped to [0, 1]) into the
package's input data (paper_2606_04725_gb300/data), where the seeded input
generators read them.

Calls only the oracle: the steady state solves f(x, u_ref) = 0 of the column
model of Sec. 4.1 (eq. distill-ocp) by Newton's method, with the reference
reflux u_ref = 2.51459 of Table distill-params.  Holdups do not enter a
steady state.  Run:  python tests/golden/make_steady_states.py
"""
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))
import oracle as O  # noqa: E402

DATA = os.path.join(os.path.dirname(os.path.dirname(HERE)), "paper_2606_04725_gb300", "data")

U_REF = 2.51459
CASES = [(12, 5), (34, 17), (32, 17)]

if __name__ == "__main__":
    for N, Nf in CASES:
        p = O.distillation(N, Nf, 1, np.zeros(N), np.zeros(1), U_REF)
        x = O.steady_state(p, U_REF)
        path = os.path.join(DATA, f"steady_state_N{N}_Nf{Nf}.txt")
        with open(path, "w") as f:
            f.write(f"# steady state of the column model, N={N}, feed tray {Nf}, u_ref={U_REF}\n")
            f.write("# written by tests/golden/make_steady_states.py (oracle only)\n")
            for v in x:
                f.write(f"{v:.17e}\n")
        print(path, x[0])
