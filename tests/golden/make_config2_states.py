"""Writes tests/golden/config2_states.npz: the oracle's states after each of
the first 5 implicit Euler steps of the 128x128x32 box (the paper's
524,288-cell, 1,098,306-DoF mesh of Section 2.1), one deterministic sample
with phi = 0.1 and K = 4.845e-13 (Table 1), dt = 1/12 yr, benchmark boundary
sets, from the initial state.

Calls only the oracle.  Its Newton iteration runs to the oracle's default
tolerances; the linear solves use the oracle's vertical-line multigrid
smoother to a relative residual of 1e-10 (the converged step does not depend
on the solver: with the point smoother the first step at 64x64x16 agrees to
3e-15, but at this size the point smoother needs hundreds of Krylov
iterations per Newton step).  Command (from the repository root, about
30 min on one core):

    python tests/golden/make_config2_states.py

Stored per step n (1..5):
  c{n}_idx, c{n}_val: at the last step every node with |c| > C_FLOOR (every
      other node has |c| <= C_FLOOR); at steps 1-4 C_NODES of those nodes
      drawn at random (int32 index, FP64 value), with c{n}_count the number
      of nodes above the floor;
  p{n}_val: FP64 p at the P_NODES sampled node indices (p_idx);
  info{n}: Newton iterations, linear iterations, ||R|| before and after.
"""
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle as O  # noqa: E402

C_FLOOR = 1e-13
C_NODES = 16384
P_NODES = 4096
STEPS = 5
OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "config2_states.npz")


def main():
    P = O.Problem(128, 128, 32)
    phi = np.full(P.C, 0.1)
    K = np.full(P.C, 4.845e-13)
    p, c = O.initial_state(P)
    dt = O.SECONDS_PER_YEAR / 12
    rng = np.random.default_rng(2024)
    p_idx = np.sort(rng.choice(P.N, P_NODES, replace=False)).astype(np.int32)
    out = {"p_idx": p_idx, "c_floor": np.array(C_FLOOR), "dt": np.array(dt),
           "grid": np.array([P.nx, P.ny, P.nz], np.int32)}
    for n in range(1, STEPS + 1):
        t = time.time()
        p, c, info = O.newton_step(P, phi, K, p, c, dt, O.NewtonOpts(smoother=1, lin_rtol=1e-10))
        assert info["status"] == 0, info
        keep = np.nonzero(np.abs(c) > C_FLOOR)[0].astype(np.int32)
        out[f"c{n}_count"] = np.array(keep.size)
        if n < STEPS:
            keep = np.sort(rng.choice(keep, min(C_NODES, keep.size), replace=False))
        out[f"c{n}_idx"] = keep
        out[f"c{n}_val"] = c[keep]
        out[f"p{n}_val"] = p[p_idx]
        out[f"info{n}"] = np.array([info["newton_iters"], info["lin_iters"], info["res0"],
                                    info["res"]])
        print(f"step {n}: {time.time() - t:.1f} s, {keep.size} nodes above the floor, {info}",
              flush=True)
    np.savez_compressed(OUT, **out)
    print("wrote", OUT, os.path.getsize(OUT), "bytes")


if __name__ == "__main__":
    main()
