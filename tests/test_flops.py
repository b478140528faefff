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


def _householder_count(n):
    """Multiply-adds of a plain Householder QR of an n x n matrix, counted
    while it runs (pure Python, no formula): the pivot norm over rows j..n-1,
    then for every later column the dot product v^H y and the update
    y -= tau w v over the same rows."""
    import random
    rnd = random.Random(n)
    a = [[rnd.uniform(-1, 1) + (n if i == j else 0) for j in range(n)] for i in range(n)]
    count = 0
    for j in range(n):
        norm2 = 0.0
        for i in range(j, n):
            norm2 += a[i][j] * a[i][j]
            count += 1
        alpha = -norm2 ** 0.5 if a[j][j] >= 0 else norm2 ** 0.5
        v = [0.0] * n
        for i in range(j, n):
            v[i] = a[i][j]
        v[j] -= alpha
        vv = sum(v[i] * v[i] for i in range(j, n))
        for c in range(j + 1, n):
            w = 0.0
            for i in range(j, n):
                w += v[i] * a[i][c]
                count += 1
            for i in range(j, n):
                a[i][c] -= 2.0 * w / vv * v[i]
                count += 1
        a[j][j] = alpha
        for i in range(j + 1, n):
            a[i][j] = 0.0
    return count


@pytest.mark.parametrize("n", [1, 2, 5, 16, 64])
def test_method_qr_count_is_a_householder_qr(n):
    """The QR's method work is the multiply-adds a Householder QR performs,
    (2/3) n^3 + O(n^2) of them ((4/3) n^3 md operations, multiplications and
    additions), counted by running one."""
    assert flops.method_counts([1], n, 4, 1)["qr"] == _householder_count(n)
    if n == 64:
        assert abs(flops.method_counts([1], n, 4, 1)["qr"] / n ** 3 - 2 / 3) < 0.03


def test_method_forward_counts_by_enumeration():
    """Updates, Q^H b, back substitution and the block Toeplitz residual,
    counted by enumerating the products of each stage."""
    n, D = 5, 7
    upd = sum(n * n for k in range(D) for j in range(1, k + 1))
    res = sum(n * n for k in range(D) for j in range(k + 1))
    qhb = sum(2 * (n - j) for _ in range(D) for j in range(n))  # v^H b, then b -= tau w v
    bs = sum(sum(n - i for i in range(n)) for _ in range(D))
    m = flops.method_counts([2, 3], n, D, 1)
    assert m["updates"] == upd and m["residual"] == res and m["bs"] == bs
    assert m["qhb"] == qhb
    assert m["evaluate"] == (1 + 1) * 0 + (3 + 6) * D * (D + 1) // 2
