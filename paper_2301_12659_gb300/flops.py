"""Operation counts of the multiple double kernels (for the roofline report).

Two conventions:

* FP64 pipe operations of this library's algorithms (csrc/md.cuh): every
  DADD, DMUL and DFMA counts one (they occupy the FP64 pipe alike on this
  GPU); comparisons and selects run on the integer pipe and are not counted.
  ``md_ops(K)`` gives the count per primitive, mirroring md.cuh exactly.
* the paper's convention (Table 2, Section 5.1): a multiple double
  multiplication costs 23 (dd), 336 (qd) or 1742 (od) double operations and
  additions are not counted; a truncated series product of d+1 coefficients
  is counted with the zero padding, (d+1)^2 multiplications.

Algorithmic work of a phase = the number of md operations the method needs
(triangular convolution counts, n^2 per matrix-vector product, ...) times the
per-operation FP64 count.
"""
from __future__ import annotations

from functools import lru_cache

import numpy as np

#: Table 2: double operations in one md multiplication, per limb count
PAPER_MUL_COST = {1: 1, 2: 23, 4: 336, 8: 1742}


@lru_cache(maxsize=None)
def md_ops(K: int) -> dict:
    """FP64 pipe operations of the md.cuh primitives for K limbs."""
    two_sum, two_prod = 3, 2

    def cascade(L):  # term entering level L
        L = min(L, K - 1)
        return two_sum * (K - 1 - L) + 1

    renorm = 2 * two_sum * (K - 1)
    if K == 1:
        acc_fma, acc_mul, acc_add, acc_get = 1, 1, 1, 0
    else:
        acc_add = sum(cascade(L) for L in range(K))
        acc_fma = 0
        for L in range(K + 1):
            for I in range(L + 1):
                J = L - I
                if I >= K or J >= K:
                    continue
                acc_fma += (two_prod + cascade(L) + cascade(L + 1)) if L <= K - 2 else 1
        acc_mul = two_prod * (K - 1) + 1  # seeds: (0, L) products
        for L in range(K + 1):
            if 1 <= L and L - 1 <= K - 2:
                acc_mul += cascade(L)
            for I in range(1, L + 1):
                J = L - I
                if I >= K or J >= K:
                    continue
                acc_mul += (two_prod + cascade(L) + cascade(L + 1)) if L <= K - 2 else 1
        acc_get = renorm
    return {"acc_fma": acc_fma, "acc_mul": acc_mul, "acc_add": acc_add, "acc_get": acc_get,
            "md_fma": acc_fma + acc_get, "md_mul": acc_mul + acc_get, "md_add": acc_add + acc_get}


def cmd_ops(K: int, C: int) -> dict:
    """Per complex (C = 2, 4M products) or real (C = 1) md operation."""
    o = md_ops(K)
    if C == 1:
        return dict(o)
    return {"acc_fma": 4 * o["acc_fma"], "acc_mul": 2 * o["acc_mul"] + 2 * o["acc_fma"],
            "acc_add": 2 * o["acc_add"], "acc_get": 2 * o["acc_get"],
            "md_fma": 4 * o["acc_fma"] + 2 * o["acc_get"], "md_mul": 2 * o["acc_mul"] + 2 * o["acc_fma"] + 2 * o["acc_get"],
            "md_add": 2 * (o["acc_add"] + o["acc_get"])}


def products_per_monomial(k: int) -> int:
    """Truncated series products of the forward/backward/cross scheme."""
    return 1 if k == 1 else 3 * k - 3


def ed_counts(sizes, D: int, K: int, C: int) -> dict:
    """Evaluation and differentiation of monomials with `sizes` variables."""
    sizes = np.asarray(sizes)
    nprod = int(sum(products_per_monomial(int(k)) for k in sizes))
    o = cmd_ops(K, C)
    tri = D * (D + 1) // 2  # multiply-adds of one truncated product
    return {
        "products": nprod,
        "md_fma": nprod * tri,
        "fp64_ops": nprod * (tri * o["acc_fma"] + D * o["acc_get"]),
        "paper_flops": nprod * D * D * PAPER_MUL_COST[K] * (4 if C == 2 else 1),
    }


def solve_counts(n: int, D: int, K: int, C: int) -> dict:
    """Householder QR of A0 and its inverse, then the forward substitution."""
    o = cmd_ops(K, C)
    qr_fma = (4 * n ** 3) // 3 + 2 * n ** 3 + n ** 3 // 2  # QR, Q^H I, back substitution
    upd_fma = n * n * (D * (D - 1) // 2)                   # sum_{j>=1} A_j dx_{k-j}
    solve_fma = n * n * D                                   # dx_k = W r_k
    res_fma = n * n * D                                     # r_k - A_0 dx_k
    paper_mul = PAPER_MUL_COST[K] * (4 if C == 2 else 1)
    return {
        "qr_md_fma": qr_fma,
        "qr_fp64_ops": qr_fma * o["md_fma"],
        "forward_md_fma": upd_fma + solve_fma + res_fma,
        "forward_fp64_ops": (upd_fma + solve_fma + res_fma) * o["acc_fma"] + 3 * n * D * o["acc_get"],
        "paper_flops": (qr_fma + upd_fma + solve_fma + res_fma) * paper_mul,
    }


def method_counts(sizes, n: int, D: int, C: int) -> dict:
    """The method's md multiply-adds per Newton step, phase by phase, as the
    paper structures the step (independent of how this library forms them):

    * evaluation and differentiation (Section 5.1): 3k-3 truncated products
      per monomial of k >= 2 variables, D(D+1)/2 multiply-adds each;
    * Householder QR of A0 (Section 5.3): sum over the columns j of
      (n-j) for the pivot norm and 2(n-j) per later column (w = v^H y and
      y -= tau w v), (2/3) n^3 + O(n^2) multiply-adds, i.e. (4/3) n^3 md
      operations;
    * per stage k, Q^H b (n(n+1): per reflector j a dot product and an
      update over rows j..n-1) and the back substitution with R (n(n+1)/2);
    * the right hand side updates sum_{j>=1} A_j dx_{k-j} (n^2 per block,
      D(D-1)/2 blocks in all);
    * the residual b - A dx of the full block Toeplitz system
      (n^2 D(D+1)/2).
    Complex data count complex multiply-adds (four real ones each)."""
    sizes = np.asarray(sizes)
    nprod = int(sum(products_per_monomial(int(k)) for k in sizes))
    qr = sum((n - j) + 2 * (n - j) * (n - j - 1) for j in range(n))
    out = {
        "evaluate": nprod * (D * (D + 1) // 2),
        "qr": qr,
        "qhb": D * n * (n + 1),
        "bs": D * (n * (n + 1) // 2),
        "updates": n * n * (D * (D - 1) // 2),
        "residual": n * n * (D * (D + 1) // 2),
    }
    out["real_factor"] = 4 if C == 2 else 1
    return out


def step_counts(sizes, n: int, D: int, K: int, C: int) -> dict:
    e = ed_counts(sizes, D, K, C)
    s = solve_counts(n, D, K, C)
    return {"evaluate": e, "solve": s,
            "fp64_ops": e["fp64_ops"] + s["qr_fp64_ops"] + s["forward_fp64_ops"],
            "paper_flops": e["paper_flops"] + s["paper_flops"]}


def adjoint_counts(sizes, n: int, D: int, K: int, C: int) -> dict:
    """One gradient: the evaluation of A(t), the QR and inverse of A_0, the
    transposed forward substitution, and per monomial of k variables k-1
    products of its variables plus one correlation (D(D+1)/2 multiply-adds)."""
    s = step_counts(sizes, n, D, K, C)
    o = cmd_ops(K, C)
    tri = D * (D + 1) // 2
    sizes = np.asarray(sizes)
    corr = int(sum(max(0, int(k) - 1) + 1 for k in sizes))
    adj = corr * (tri * o["acc_fma"] + D * o["acc_get"])
    return {"fp64_ops": s["fp64_ops"] + adj, "qr_fp64_ops": s["solve"]["qr_fp64_ops"], "correlation_fp64_ops": adj}
