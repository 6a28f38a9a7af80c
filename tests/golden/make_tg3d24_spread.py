"""Write tests/golden/tg3d24_q2_oracle_spread.txt: how far the oracle's own end state
of the configured 3D Taylor-Green run (24^3 Q2, CFL 0.5 to t = 0.1) moves under
perturbations at the rounding and solver-tolerance level.

Reads the oracle outputs of tests/golden/make_tg3d24_end_state.py (the plain run,
the run with the initial velocity scaled by 1 + 1e-13, and the run with mass solves
to 1e-12 instead of 1e-14) and writes, per perturbation, the relative 2-norm
differences of x, v and e from the plain run's end state and the step counts.

    python tests/golden/make_tg3d24_end_state.py
    python tests/golden/make_tg3d24_end_state.py --perturb 1e-13
    python tests/golden/make_tg3d24_end_state.py --cg-tol 1e-12
    python tests/golden/make_tg3d24_spread.py
"""
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
BASE = "tg3d24_q2_t0.1_end_state"


def main():
    g = np.load(os.path.join(HERE, BASE + ".npz"))
    lines = ["# relative 2-norm differences of the end states x, v, e from the plain oracle run",
             "# (3D Taylor-Green 24^3 Q2/Q1, CFL 0.5, t = 0.1), then the step counts (plain, perturbed)"]
    for tag in ("perturbed1e-13", "cgtol1e-12"):
        h = np.load(os.path.join(HERE, f"{BASE}_{tag}.npz"))
        d = [float(np.linalg.norm(h[k].reshape(-1) - g[k].reshape(-1)) / np.linalg.norm(g[k])) for k in "xve"]
        lines.append(f"{tag} {d[0]:.6e} {d[1]:.6e} {d[2]:.6e}")
        lines.append(f"# {tag}: {int(g['steps'])} and {int(h['steps'])} steps")
    with open(os.path.join(HERE, "tg3d24_q2_oracle_spread.txt"), "w") as f:
        f.write("\n".join(lines) + "\n")
    print("\n".join(lines))


if __name__ == "__main__":
    main()
