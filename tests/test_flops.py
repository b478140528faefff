"""Operation counts behind the roofline figures (paper_2301_12659_gb300/flops.py):
the paper's convention against its Table 2, the product count of the
evaluation against the product table the kernel runs, and the work of the
quad double workload that the per-unit figure of the integer pipe divides."""
import os

import numpy as np
import pytest

from paper_2301_12659_gb300 import flops
from paper_2301_12659_gb300 import workloads as wl

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def test_paper_multiplication_cost_is_table_2():
    rows = [l.split() for l in open(os.path.join(GOLDEN, "table2_md_mul_cost.txt")) if not l.startswith("#")]
    for name, limbs, adds, subs, muls, total, per_double in rows:
        K = int(limbs)
        assert int(adds) + int(subs) + int(muls) == int(total)
        assert flops.PAPER_MUL_COST[K] == int(total)
        assert float(per_double) == int(total) / K


def test_products_per_monomial_match_the_kernel_table():
    """The roofline counts 3k-3 truncated products per monomial of k >= 2
    variables (one for k = 1); the table the evaluation runs has exactly
    that many products."""
    from paper_2301_12659_gb300 import build
    from paper_2301_12659_gb300 import mdnewton as md
    build.build()
    md.load()
    for k in list(range(1, 40)) + [64, 128, 300]:
        ops = md.mdn_ed_schedule(k, 2)
        assert int(np.sum(ops[..., 0] == 1)) == flops.products_per_monomial(k), k


def test_quad_double_workload_counts():
    """n = 64, d = 31 with 16 monomials of 2..8 variables per equation plus
    the diagonal term: the products and md multiply-adds per evaluation that
    the integer-pipe figure (integer instructions per multiply-add, from the
    evaluation kernel's counters) is taken over."""
    cfg = wl.CONFIGS["qd-real-n64-d31"]
    s, _, _ = wl.planted_system(cfg)
    sizes = np.diff(s.vptr)
    assert s.M == 64 * 17 and sizes.min() == 1 and sizes.max() == 8
    e = flops.ed_counts(sizes, s.D, s.K, s.C)
    assert e["products"] == 12070
    assert e["md_fma"] == 12070 * 32 * 33 // 2
    # the paper's convention pads each product to (d+1)^2 multiplications
    assert e["paper_flops"] == 12070 * 32 * 32 * 336
    sc = flops.solve_counts(64, 32, 4, 1)
    assert sc["qr_md_fma"] == (4 * 64 ** 3) // 3 + 2 * 64 ** 3 + 64 ** 3 // 2
    assert sc["forward_md_fma"] == 64 * 64 * (32 * 31 // 2) + 2 * 64 * 64 * 32


@pytest.mark.parametrize("K", [1, 2, 4, 8])
def test_complex_counts_are_four_real_products(K):
    r, c = flops.cmd_ops(K, 1), flops.cmd_ops(K, 2)
    assert c["acc_fma"] == 4 * r["acc_fma"]
    assert c["acc_add"] == 2 * r["acc_add"]
