"""Writes the oracle's values for the complex octo double workload (n = 128,
d = 63, 32 monomials per equation of 2..16 variables, unit-circle data) and
for a reduced analogue of the same recipe at n = 16, into
tests/golden/od_complex_golden.npz.  Calls only the oracle (oracle/); the
inputs come from the seeded generators of paper_2301_12659_gb300.workloads.

  cst128      the planted constant term of the full workload (octo double
              evaluation of -f(x*) with cst = 0), [8][2][128][64]
  cst16       the same for the reduced analogue, [8][2][16][64]
  x16_8, x16_9   the oracle's Newton series of the reduced analogue after 8
              and 9 steps from its start series, [8][2][16][64]
  hist16      the oracle's history of those 9 steps, [9][3]

Run:  python tests/golden/make_od_complex_golden.py   (about an hour on 8
host cores: the full workload's constant term takes ~5 minutes, the nine
oracle Newton steps on full-width octo double series the rest)."""
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle import oracle  # noqa: E402
from paper_2301_12659_gb300 import workloads as wl  # noqa: E402

OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "od_complex_golden.npz")


def reduced_config():
    """The complex octo double recipe at n = 16 (k in 2..16 of 16 variables)."""
    full = wl.CONFIGS["od-complex-n128-d63"]
    return wl.PlantedConfig("od-complex-n16-d63", 8, 2, 16, 63, full.mono_per_eq, full.kmin, 16, 16.0, 9,
                            full.tol, 20, unit_circle=True)


def main():
    t0 = time.time()
    s16, xs16, x016 = wl.planted_system(reduced_config())
    s16.cst = oracle.planted_constant(s16, xs16)
    x8, h8 = oracle.newton(s16, x016, 8)
    x9, h9 = oracle.newton(s16, x8, 1)
    print(f"reduced analogue: {time.time() - t0:.0f} s", flush=True)
    s, xs, _ = wl.planted_system(wl.CONFIGS["od-complex-n128-d63"])
    cst = oracle.planted_constant(s, xs)
    print(f"total: {time.time() - t0:.0f} s", flush=True)
    np.savez_compressed(OUT, cst128=cst, cst16=s16.cst, x16_8=x8, x16_9=x9, hist16=np.vstack([h8, h9]))


if __name__ == "__main__":
    main()
