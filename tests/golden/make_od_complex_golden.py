"""Writes the oracle's values for the complex octo double workload (n = 128,
d = 63, 32 monomials per equation of 2..16 variables, unit-circle data,
diagonal 128 x_i) and for reduced analogues of the same recipe at n = 16,
into tests/golden/od_complex_golden.npz.  Calls only the oracle (oracle/);
the inputs come from the seeded generators of paper_2301_12659_gb300.workloads.

  cst128        the planted constant term of the full workload (octo double
                evaluation of -f(x*) with cst = 0), [8][2][128][64]
  cst16         the reduced analogue with the diagonal n x_i = 16 x_i:
                its planted constant term, [8][2][16][64]
  x16_8, x16_9  its oracle Newton series after 8 and 9 steps from its
                start series, [8][2][16][64]; hist16 the history [9][3]
  cst16d128, x16d128_8, x16d128_9, hist16d128   the same for the reduced
                analogue with the full workload's diagonal 128 x_i (the
                same distribution of every equation, only n reduced)

Run:  python tests/golden/make_od_complex_golden.py   (about an hour per
reduced analogue on 8 host cores, five minutes for the full workload's
constant term; values already in the file are kept)."""
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle import oracle  # noqa: E402
from paper_2301_12659_gb300 import workloads as wl  # noqa: E402

OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "od_complex_golden.npz")


def reduced_config(diag: float = 16.0):
    """The complex octo double recipe at n = 16 (k in 2..16 of 16 variables)."""
    full = wl.CONFIGS["od-complex-n128-d63"]
    name = "od-complex-n16-d63" if diag == 16.0 else f"od-complex-n16-d63-diag{int(diag)}"
    return wl.PlantedConfig(name, 8, 2, 16, 63, full.mono_per_eq, full.kmin, 16, diag, 9, full.tol, 20,
                            unit_circle=True)


def reduced_run(diag):
    s, xs, x0 = wl.planted_system(reduced_config(diag))
    s.cst = oracle.planted_constant(s, xs)
    x8, h8 = oracle.newton(s, x0, 8)
    x9, h9 = oracle.newton(s, x8, 1)
    return s.cst, x8, x9, np.vstack([h8, h9])


def main():
    out = dict(np.load(OUT)) if os.path.exists(OUT) else {}
    t0 = time.time()
    for diag, tag in ((16.0, "16"), (128.0, "16d128")):
        if f"x{tag}_9" not in out:
            cst, x8, x9, hist = reduced_run(diag)
            out.update({f"cst{tag}": cst, f"x{tag}_8": x8, f"x{tag}_9": x9, f"hist{tag}": hist})
            print(f"reduced analogue, diagonal {diag:g}: {time.time() - t0:.0f} s", flush=True)
            np.savez_compressed(OUT, **out)
    if "cst128" not in out:
        s, xs, _ = wl.planted_system(wl.CONFIGS["od-complex-n128-d63"])
        out["cst128"] = oracle.planted_constant(s, xs)
        np.savez_compressed(OUT, **out)
    print(f"total: {time.time() - t0:.0f} s", flush=True)


if __name__ == "__main__":
    main()
