"""Error metrics on multiple double arrays (test infrastructure).

``md_diff`` forms x - y entry by entry with ``math.fsum`` (the correctly
rounded sum of the limbs of both), so a difference far below the leading
limbs is measured accurately.  The per-coefficient relative error follows
the normalisation |x - y| <= tol * max(|y_{v,k}|, s_v), s_v = max_k |y_{v,k}|
(series scale of variable v): a pure relative test is meaningless for
coefficients that are (nearly) zero.
"""
from __future__ import annotations

import math

import numpy as np


def md_value(x: np.ndarray) -> np.ndarray:
    """Leading-double value of md arrays [K, C, *S] -> [C, *S] (fsum of limbs)."""
    K = x.shape[0]
    flat = x.reshape(K, -1)
    out = np.array([math.fsum(flat[:, i]) for i in range(flat.shape[1])])
    return out.reshape(x.shape[1:])


def md_diff(x: np.ndarray, y: np.ndarray) -> np.ndarray:
    """Correctly rounded x - y for md arrays [K, C, *S] -> [C, *S]."""
    assert x.shape == y.shape
    K = x.shape[0]
    fx = x.reshape(K, -1)
    fy = y.reshape(K, -1)
    out = np.array([math.fsum(list(fx[:, i]) + list(-fy[:, i])) for i in range(fx.shape[1])])
    return out.reshape(x.shape[1:])


def magnitude(c_axis_arr: np.ndarray) -> np.ndarray:
    """|z| over the C axis (axis 0): abs for real, hypot for complex."""
    if c_axis_arr.shape[0] == 1:
        return np.abs(c_axis_arr[0])
    return np.hypot(c_axis_arr[0], c_axis_arr[1])


def series_rel_error(x: np.ndarray, ref: np.ndarray) -> np.ndarray:
    """Per-coefficient normalised error [n, D] of series arrays [K, C, n, D]."""
    err = magnitude(md_diff(x, ref))
    val = magnitude(md_value(ref))
    scale = np.max(val, axis=-1, keepdims=True)
    den = np.maximum(val, scale)
    den = np.where(den == 0.0, 1.0, den)
    return err / den


def correct_leading(x: np.ndarray, ref: np.ndarray, tol: float) -> int:
    """Number of leading coefficients within tol, minimum over the variables."""
    ok = series_rel_error(x, ref) <= tol
    counts = []
    for row in ok:
        c = 0
        while c < row.size and row[c]:
            c += 1
        counts.append(c)
    return int(min(counts))


def matrix_rel_error(a: np.ndarray, ref: np.ndarray, floor: float = 1.0) -> float:
    """max |a - ref| / max(|ref|, floor) over all entries of md arrays [K, C, ...]."""
    err = magnitude(md_diff(a, ref))
    val = magnitude(md_value(ref))
    return float(np.max(err / np.maximum(val, floor))) if err.size else 0.0
