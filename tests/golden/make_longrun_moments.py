"""Writes tests/golden/longrun_moments_<case>.npz: the oracle's sample mean,
variance and exceedance probability P(c > 0.5) per node (Section 3, eqs.
pdestat and numer_var with w_i = 1/S, and the exceedance estimate) after a
long run from the initial state.

Cases:
  32 -- 32 samples at 32x32x8, 60 steps of dt = 1/12 yr, the first scrambled-
        Sobol samples of the qMC ensemble (porosity phi = 0.1 (1 + 0.3 (xi1
        cos(pi x/600) + xi2 cos(pi y/600) + xi3 sin(2 pi z/150))/3), normalised
        Kozeny-Carman K), benchmark boundary sets; file longrun_moments_32x32x8;
  64 -- the same at 64x64x16 with 16 samples (the first 16 points of the
        256-point ensemble); file longrun_moments_64x64x16;
  f3 -- the paper's own ensemble (Section 5.3): the parallelepiped field of
        eq. poro-paral3RVS at the first 16 Halton points (bases 2, 3, 5, the
        first point skipped), the paper's boundary sets (bc_mode 1), 300 steps
        of dt = 0.005 yr (1.5 yr) at 32x32x8; file
        longrun_moments_paper3rv_32x32x8.

Calls only the oracle (and the seeded sample points), with its vertical-line
multigrid smoother; one sample per spawned worker process.  Command (from the
repository root; about 2 h of CPU on 6 cores for 32 and 64, minutes for f3):

    python tests/golden/make_longrun_moments.py [--workers 6] [--case 32 64 f3]

Stored: xi [S][3]; mean, var, pexc [N]; amb [N] uint8, the number of samples
whose c lies within AMB_BAND of the threshold (there the decision c > 0.5 is
not fixed by the oracle's accuracy and may flip); c_idx and c_smp [S][len]:
c of every sample at a few sampled nodes (diagnostics of per-sample drift);
steps, dt_yr, bc_mode, fields.
"""
import argparse
import multiprocessing as mp
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

THRESH = 0.5
AMB_BAND = 1e-6
N_SAMPLED = 512
# case: (nx, ny, nz, samples, steps, dt in years, fields, bc_mode, file tag)
CASES = {"32": (32, 32, 8, 32, 60, 1.0 / 12.0, "sobol", 0, "32x32x8"),
         "64": (64, 64, 16, 16, 60, 1.0 / 12.0, "sobol", 0, "64x64x16"),
         "f3": (32, 32, 8, 16, 300, 0.005, "paper3rv", 1, "paper3rv_32x32x8")}


def _run(args):
    nx, ny, nz, xi, steps, dt_yr, fields, bc_mode = args
    import oracle as O
    P = O.Problem(nx, ny, nz, bc_mode=bc_mode)
    phi, K = (O.fields_sobol(P, xi) if fields == "sobol" else O.fields_paper3rv(P, xi))
    p, c = O.initial_state(P)
    dt = O.SECONDS_PER_YEAR * dt_yr
    t = time.time()
    # the oracle's vertical-line multigrid smoother: with the point smoother a
    # late step of a 64x64x16 sample stagnated at round-off (its BiCGStab did
    # not reach the Newton correction's accuracy); the converged step does
    # not depend on the smoother
    opts = O.NewtonOpts(smoother=1, lin_rtol=1e-10)
    for n in range(steps):
        p, c, info = O.newton_step(P, phi, K, p, c, dt, opts)
        if info["status"] != 0:
            raise RuntimeError(f"oracle step {n + 1} failed: {info}")
    return c, time.time() - t


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--workers", type=int, default=6)
    ap.add_argument("--case", choices=sorted(CASES), nargs="*", default=sorted(CASES))
    a = ap.parse_args()
    import oracle as O
    from paper_1906_01632_gb300 import inputs as I
    O.build()
    for case in a.case:
        nx, ny, nz, S, steps, dt_yr, fields, bc_mode, tag = CASES[case]
        xi = (I.sobol_xi(256, seed=0) if fields == "sobol" else I.halton_xi(256))[:S]
        t0 = time.time()
        with mp.get_context("spawn").Pool(a.workers) as pool:
            res = pool.map(_run, [(nx, ny, nz, xi[s], steps, dt_yr, fields, bc_mode)
                                  for s in range(S)], chunksize=1)
        cs = np.stack([r[0] for r in res])
        mean, var, pexc = O.moments(cs, threshold=THRESH)
        amb = (np.abs(cs - THRESH) <= AMB_BAND).sum(0).astype(np.uint8)
        rng = np.random.default_rng(7)
        c_idx = np.sort(rng.choice(cs.shape[1], N_SAMPLED, replace=False)).astype(np.int32)
        out = os.path.join(os.path.dirname(os.path.abspath(__file__)),
                           f"longrun_moments_{tag}.npz")
        np.savez_compressed(out, xi=xi, mean=mean, var=var, pexc=pexc, amb=amb,
                            c_idx=c_idx, c_smp=cs[:, c_idx], steps=np.array(steps),
                            threshold=np.array(THRESH), amb_band=np.array(AMB_BAND),
                            dt_yr=np.array(dt_yr), bc_mode=np.array(bc_mode),
                            fields=np.array(fields))
        print(f"{case}: {S} samples x {steps} steps in {time.time() - t0:.0f} s "
              f"(per sample {[round(r[1]) for r in res]}); wrote {out} "
              f"({os.path.getsize(out)} bytes); max var {var.max():.4f}, "
              f"nodes with an ambiguous sample {(amb > 0).sum()}", flush=True)


if __name__ == "__main__":
    main()
