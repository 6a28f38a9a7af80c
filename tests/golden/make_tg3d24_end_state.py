"""Write the oracle's state of the 3D Taylor-Green run at 24^3 (Q2/Q1, 4^3 Gauss
points, gamma = 5/3, CFL 0.5 from t = 0 to t = 0.1) to tests/golden/.

Calls only the oracle (oracle.hydro: full global assembly, sparse CG to 1e-14
relative per mass solve) and the seeded input generator. The RK2-average step,
the time-step rule dt_n = min(dt_est(S_n), t_end - t_n) and the problem are the
ones of Section 3.3, Eqs. 14-18, as the oracle reads them.

    python tests/golden/make_tg3d24_end_state.py                      # end state (t = 0.1)
    python tests/golden/make_tg3d24_end_state.py --stop-after 20      # state after 20 steps
    python tests/golden/make_tg3d24_end_state.py --perturb 1e-13      # initial v scaled by 1 + 1e-13
    python tests/golden/make_tg3d24_end_state.py --cg-tol 1e-12       # mass solves to 1e-12 only
    python tests/golden/make_tg3d24_end_state.py --no-viscosity       # the same run without viscosity

The whole run takes about two hours of one host core; it saves a checkpoint every
25 steps beside the output and resumes from it when restarted. The perturbed run
and the run with looser mass solves measure how far the oracle's own trajectory moves
under perturbations at the rounding and solver-tolerance level: the configured run
is sensitive to them (the linear artificial-viscosity term switches on the sign of
the smallest strain-rate eigenvalue).
"""
from __future__ import annotations

import argparse
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from oracle.hydro import Hydro, Params  # noqa: E402
from paper_2112_07075_b300 import inputs  # noqa: E402

N, P, Q1, T_END, CFL = 24, 2, 4, 0.1, 0.5


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--stop-after", type=int, default=0, help="stop after this many steps (0: run to t_end)")
    ap.add_argument("--perturb", type=float, default=0.0, help="scale the initial velocity by 1 + this")
    ap.add_argument("--cg-tol", type=float, default=0.0, help="relative tolerance of the mass solves (default 1e-14)")
    ap.add_argument("--no-viscosity", action="store_true", help="switch the artificial viscosity off")
    a = ap.parse_args()
    name = "tg3d24_q2_t0.1_end_state"
    if a.stop_after:
        name = f"tg3d24_q2_step{a.stop_after}_state"
    if a.perturb:
        name += f"_perturbed{a.perturb:g}"
    if a.cg_tol:
        name += f"_cgtol{a.cg_tol:g}"
    if a.no_viscosity:
        name += "_noviscosity"
    out = os.path.join(HERE, name + ".npz")
    ckpt = out + ".ckpt.npz"
    hy = Hydro(Params(dim=3, n=N, order=P, q1=Q1, vertices=inputs.box_vertices(3, N), cfl=CFL,
                      use_viscosity=not a.no_viscosity))
    if a.cg_tol:
        solve = hy.mass_solve
        hy.mass_solve = lambda b, tol=a.cg_tol: solve(b, tol)
    if os.path.exists(ckpt):
        c = np.load(ckpt)
        x, v, e, t, steps = c["x"], c["v"], c["e"], float(c["t"]), int(c["steps"])
        dts = list(c["dts"])
    else:
        x, v, e = hy.initial_state("taylor_green")
        v = v * (1.0 + a.perturb)
        t, steps, dts = 0.0, 0, []
    t0 = time.time()
    while t < T_END and (a.stop_after == 0 or steps < a.stop_after):
        x, v, e, info = hy.rk2avg_step(x, v, e, dt=None, t=t, t_end=T_END)
        t += info.dt
        steps += 1
        dts.append(info.dt)
        if steps % 25 == 0:
            np.savez(ckpt, x=x, v=v, e=e, t=t, steps=steps, dts=np.array(dts))
            print(f"step {steps} t={t:.6f} dt={info.dt:.3e} {time.time() - t0:.0f}s", flush=True)
    np.savez_compressed(out, x=x, v=v, e=e, t=t, steps=steps, dts=np.array(dts), perturb=a.perturb, cg_tol=a.cg_tol,
                        viscosity=not a.no_viscosity,
                        config=np.array("3D Taylor-Green 24^3 Q2/Q1 q4 gamma 5/3 CFL 0.5 t_end 0.1"))
    if os.path.exists(ckpt):
        os.remove(ckpt)
    print(f"done: {steps} steps, t = {t!r} -> {os.path.basename(out)}", flush=True)


if __name__ == "__main__":
    main()
