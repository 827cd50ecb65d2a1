"""Write fit_reference_240sn.txt: reference minima of the 240-supernova fit
fixture, for the batched-fit parity test (tests/test_gpu_fit_golden.py).

Calls only the oracle (oracle/, oracle/fit.py) and the seeded input
generators (workloads/). The minimiser is the algorithm the paper names for
fitting (L-BFGS-B, Implementation, first paragraph) as a library routine:
scipy's L-BFGS-B on the FP64 oracle chi^2 and its analytic gradient, one
supernova at a time, gtol 1e-10 / ftol 1e-15.

    python tests/golden/make_fit_reference.py      # about 7 min on 8 cores
"""
from __future__ import annotations

import multiprocessing as mp
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
OUT = os.path.join(HERE, "fit_reference_240sn.txt")
N_SN, SEED = 240, 77
Z_BOX = 0.05  # mode 1: z free within its start +- Z_BOX
if ROOT not in sys.path:  # the oracle and the input generators live at the repository root
    sys.path.insert(0, ROOT)


def fixture():
    """(workload, oracle, starting batch, lower, upper): config 2 shapes with
    240 supernovae; observed fluxes = oracle bandfluxes at the truth + 5 %
    Gaussian noise; starts = the truth perturbed in t0, x0, x1, c."""
    import oracle
    import workloads as W
    wl = W.config2(seed=SEED, n_sn=N_SN)
    o = oracle.Oracle(wl.model, wl.bands)
    W.add_noise(wl.batch, o.bandflux(W.truth_batch(wl.batch)), np.random.default_rng(SEED + 1))
    start = W.fit_start(wl.batch, np.random.default_rng(SEED + 2))
    lower = np.full((N_SN, 5), -np.inf)
    upper = np.full((N_SN, 5), np.inf)
    lower[:, 0] = start.z - Z_BOX
    upper[:, 0] = start.z + Z_BOX
    return wl, o, start, lower, upper


def mode_args(mode, lower, upper, s):
    """fit_one's (lower, upper, mask) of supernova s: mode 0 fits t0, x0, x1, c;
    mode 1 fits z too, inside its box."""
    import oracle.fit as OF
    if mode == 0:
        return None, None, OF.DEFAULT_MASK
    return lower[s], upper[s], OF.DEFAULT_MASK | OF.MASK_Z


def _work(job):
    import oracle.fit as OF
    mode, sns = job
    wl, o, start, lower, upper = fixture()
    out = []
    for s in sns:
        lo, hi, mask = mode_args(mode, lower, upper, s)
        th, f, _ = OF.fit_one(o, start, s, lo, hi, mask)
        out.append((mode, s, th, f))
    return out


def main():
    jobs = [(m, list(range(i, N_SN, 16))) for m in (0, 1) for i in range(16)]
    rows = []
    with mp.get_context("spawn").Pool(min(8, os.cpu_count() or 1)) as pool:
        for out in pool.imap_unordered(_work, jobs):
            rows.extend(out)
    rows.sort(key=lambda r: (r[0], r[1]))
    with open(OUT, "w") as fh:
        fh.write("# Reference minima of the 240-supernova fit fixture (tests/golden/make_fit_reference.py):\n")
        fh.write("# scipy L-BFGS-B on the FP64 oracle chi^2, the paper's fitting algorithm (Implementation,\n")
        fh.write(f"# first paragraph). Fixture: workloads.config2(seed={SEED}, n_sn={N_SN}); fluxes = oracle\n")
        fh.write(f"# bandfluxes at the truth + 5 % noise (seed {SEED + 1}); starts = fit_start (seed {SEED + 2}).\n")
        fh.write(f"# mode 0: t0, x0, x1, c free; mode 1: z free too, within its start +- {Z_BOX}.\n")
        fh.write("# mode sn z t0 x0 x1 c chi2\n")
        for mode, s, th, f in rows:
            fh.write(f"{mode} {s} " + " ".join(repr(float(v)) for v in th) + f" {float(f)!r}\n")
    print(f"wrote {len(rows)} rows to {OUT}")


if __name__ == "__main__":
    main()
