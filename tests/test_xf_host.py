"""The integer-limb extended floats (csrc/xf.cuh), compiled for the host and
checked against exact rationals: conversions from and to multiple doubles,
add, sub, mul, reciprocal and reciprocal square root, zero and cancellation.

An xf of W 64-bit words carries 64W bits; each operation must be correct to
a few units of 2^(-64W) (far below the 2^(-53K) of the K-limb md values it
serves), and its md output must be K nonoverlapping limbs rounded to
nearest."""
import ctypes
import math
import os
import subprocess
from fractions import Fraction as Fr

import numpy as np
import pytest

from paper_2301_12659_gb300 import workloads as wl
from tests import exact as ex

HERE = os.path.dirname(os.path.abspath(__file__))
WORDS = {1: 1, 2: 2, 4: 4, 8: 7}
OPS = {"copy": 0, "add": 1, "sub": 2, "mul": 3, "recip": 4, "rsqrt": 5}


@pytest.fixture(scope="module")
def lib(tmp_path_factory):
    so = str(tmp_path_factory.mktemp("xf") / "xf_host.so")
    src = os.path.join(HERE, "native", "xf_host.cpp")
    subprocess.run(["g++", "-O2", "-std=c++17", "-shared", "-fPIC", "-o", so, src], check=True)
    h = ctypes.CDLL(so)
    h.xf_host_op.restype = ctypes.c_int
    return h


def _op(lib, K, op, a, b=None, extra=False):
    a = np.ascontiguousarray(a, dtype=np.float64)
    b = np.ascontiguousarray(a if b is None else b, dtype=np.float64)
    out = np.zeros(K + (1 if extra else 0))
    p = ctypes.POINTER(ctypes.c_double)
    rc = lib.xf_host_op(K, int(extra), OPS[op], a.ctypes.data_as(p), b.ctypes.data_as(p), out.ctypes.data_as(p))
    assert rc == 0
    return out


def _values(K, count, seed, spread=40):
    """md values [count][K] of full width with magnitudes 2^-spread..2^spread."""
    v = wl.random_md((count,), K, 1, seed)[:, 0].T.copy()
    rng = np.random.default_rng(seed)
    v *= np.exp2(rng.integers(-spread, spread + 1, size=count))[:, None]
    return v


def _nonoverlapping(limbs):
    for l in range(len(limbs) - 1):
        if limbs[l] == 0.0:
            assert np.all(np.asarray(limbs[l:]) == 0.0)
            return
        assert abs(limbs[l + 1]) <= np.spacing(abs(limbs[l])) / 2


@pytest.mark.parametrize("K", [1, 2, 4, 8])
def test_round_trip(lib, K):
    """md -> xf -> md is exact when the limbs span at most 64W bits (most
    values: the limbs of a full-width value lie 53 bits apart, with a gap
    where a limb is small) and otherwise loses only bits below 2^(1-64W)."""
    W = WORDS[K]
    exact = 0
    for a in _values(K, 200, 900 + K):
        out = _op(lib, K, "copy", a)
        A = ex.md_to_fr(a)
        assert abs(ex.md_to_fr(out) - A) <= Fr(2) ** (1 - 64 * W) * abs(A)
        _nonoverlapping(out)
        exact += ex.md_to_fr(out) == A
    assert exact >= 150


@pytest.mark.parametrize("K", [1, 2, 4, 8])
@pytest.mark.parametrize("op", ["add", "sub", "mul"])
def test_arithmetic_to_xf_precision(lib, K, op):
    W = WORDS[K]
    va, vb = _values(K, 150, 910 + K), _values(K, 150, 920 + K, spread=3)
    for a, b in zip(va, vb):
        A, B = ex.md_to_fr(a), ex.md_to_fr(b)
        want = A + B if op == "add" else A - B if op == "sub" else A * B
        got = _op(lib, K, op, a, b, extra=True)
        _nonoverlapping(got)
        err = abs(ex.md_to_fr(got) - want)
        bound = Fr(2) ** (3 - 64 * W) * abs(want)
        if op != "mul":
            bound += Fr(2) ** (-64 * W - 60) * max(abs(A), abs(B))
        assert err <= bound, (op, float(err), float(want))
        # rounded to K limbs: nearest, to the md precision
        gk = _op(lib, K, op, a, b)
        _nonoverlapping(gk)
        assert abs(ex.md_to_fr(gk) - want) <= Fr(2) ** (1 - 53 * K) * abs(want) + bound


@pytest.mark.parametrize("K", [1, 2, 4, 8])
def test_cancellation_is_exact(lib, K):
    """a - b for b a few units of the last limb away from a: the difference
    is formed exactly (the guard word), whatever the exponents."""
    rng = np.random.default_rng(930 + K)
    for a in _values(K, 60, 931 + K):
        A = ex.md_to_fr(a)
        tiny = Fr(int(rng.integers(-9, 10))) * Fr(2) ** (math.frexp(a[0])[1] - 53 * K - 3)
        b = np.array(ex.fr_to_md(A + tiny, K))
        if ex.md_to_fr(b) == A:
            continue
        got = _op(lib, K, "sub", a, b, extra=True)
        assert ex.md_to_fr(got) == A - ex.md_to_fr(b)
    one = np.zeros(K)
    one[0] = 1.0
    below = np.zeros(K)
    below[0] = 1.0 - 2.0 ** -53
    got = _op(lib, K, "sub", one, below, extra=True)
    assert ex.md_to_fr(got) == Fr(2) ** -53


@pytest.mark.parametrize("K", [1, 2, 4, 8])
def test_zero(lib, K):
    z = np.zeros(K)
    a = _values(K, 1, 940 + K)[0]
    assert ex.md_to_fr(_op(lib, K, "add", z, a)) == ex.md_to_fr(a)
    assert ex.md_to_fr(_op(lib, K, "add", a, z)) == ex.md_to_fr(a)
    assert np.all(_op(lib, K, "mul", z, a) == 0.0)
    assert np.all(_op(lib, K, "sub", a, a) == 0.0)
    assert np.all(_op(lib, K, "add", z, z) == 0.0)
    na = -a
    assert np.all(_op(lib, K, "add", a, na) == 0.0)


@pytest.mark.parametrize("K", [1, 2, 4, 8])
def test_reciprocal_and_rsqrt(lib, K):
    """1/a and 1/sqrt(a) to the xf precision (2^(8-64W), below the md
    precision 2^(-53K) by 11 bits or more); rounded to K limbs, within the
    per-operation contract 2^(-52K) of an md operation (in fact 2^(2-53K));
    exact where the result is a short dyadic number."""
    W = WORDS[K]
    tol = Fr(2) ** (8 - 64 * W)
    for a in _values(K, 100, 950 + K, spread=60):
        A = ex.md_to_fr(a)
        y = ex.md_to_fr(_op(lib, K, "recip", a, extra=True))
        assert abs(y * A - 1) <= tol
        yk = _op(lib, K, "recip", a)
        _nonoverlapping(yk)
        assert abs(ex.md_to_fr(yk) * A - 1) <= Fr(2) ** (2 - 53 * K)
        if a[0] < 0:  # a positive value
            a, A = -a, -A
        r = ex.md_to_fr(_op(lib, K, "rsqrt", a, extra=True))
        assert abs(r * r * A - 1) <= tol
        rk = _op(lib, K, "rsqrt", a)
        assert abs(ex.md_to_fr(rk) ** 2 * A - 1) <= Fr(2) ** (3 - 53 * K)
    # exact cases
    for v, r in ((1.0, 1), (4.0, Fr(1, 2)), (0.25, 2), (2.0 ** 40, Fr(1, 2 ** 20)), (2.0 ** -42, 2 ** 21)):
        a = np.zeros(K)
        a[0] = v
        assert ex.md_to_fr(_op(lib, K, "rsqrt", a)) == r
        assert ex.md_to_fr(_op(lib, K, "recip", a)) == 1 / Fr(v)
        assert ex.md_to_fr(_op(lib, K, "recip", -a)) == -1 / Fr(v)


@pytest.mark.parametrize("K", [1, 2, 4, 8])
def test_reciprocal_and_rsqrt_near_powers_of_two(lib, K):
    """1/a and 1/sqrt(a) for a just above and below powers of two (1 + 2^-k,
    2 - 2^-k, 4 (1 - 2^-k) and their multiples by 2^j): mantissas whose
    leading words are exactly those of a power of two, where the iteration
    heads for 1 (or 1/2) itself; same bounds as above."""
    W = WORDS[K]
    tol = Fr(2) ** (8 - 64 * W)
    ks = [k for k in (1, 2, 30, 52, 53, 60, 63, 64, 65, 100, 127, 128, 129, 150, 200, 255, 256, 257, 300, 400)
          if k <= 53 * K - 1]
    for k in ks:
        for base in (1 + Fr(1, 2 ** k), 2 - Fr(1, 2 ** k), 4 * (1 - Fr(1, 2 ** k)), 1 - Fr(1, 2 ** k)):
            for j in (-7, 0, 3):
                A = base * Fr(2) ** j
                a = np.array(ex.fr_to_md(A, K))
                if ex.md_to_fr(a) != A:
                    continue
                y = ex.md_to_fr(_op(lib, K, "recip", a, extra=True))
                assert abs(y * A - 1) <= tol, (k, base, j)
                assert abs(ex.md_to_fr(_op(lib, K, "recip", a)) * A - 1) <= Fr(2) ** (2 - 53 * K)
                r = ex.md_to_fr(_op(lib, K, "rsqrt", a, extra=True))
                assert abs(r * r * A - 1) <= tol, (k, base, j)
                assert abs(ex.md_to_fr(_op(lib, K, "rsqrt", a)) ** 2 * A - 1) <= Fr(2) ** (3 - 53 * K)


@pytest.mark.parametrize("K", [1, 2, 4, 8])
@pytest.mark.parametrize("D", [1, 7, 32, 64])
def test_fixed_point_convolution(lib, K, D):
    """c = a b mod t^D, one fixed-point accumulator per coefficient: error
    below 2^(12-64W) times the sum of the magnitudes of its terms (the md
    dot-product bound, with the accumulator's headroom), the last
    coefficient with alternating signs.  Coefficients of both series span
    2^-30..2^30 and include exact zeros."""
    W = WORDS[K]
    a = _values(K, D, 960 + K + D, spread=30)
    b = _values(K, D, 970 + K + D, spread=30)
    if D > 3:
        a[2] = 0.0
        b[D - 2] = 0.0
    out = np.zeros((D, K + 1))
    p = ctypes.POINTER(ctypes.c_double)
    ac, bc = np.ascontiguousarray(a), np.ascontiguousarray(b)
    assert lib.xf_host_conv(K, D, ac.ctypes.data_as(p), bc.ctypes.data_as(p), out.ctypes.data_as(p)) == 0
    A = [ex.md_to_fr(v) for v in a]
    B = [ex.md_to_fr(v) for v in b]
    for k in range(D):
        terms = [A[i] * B[k - i] * (-1 if (i % 2 and k == D - 1) else 1) for i in range(k + 1)]
        want = sum(terms, Fr(0))
        mag = sum((abs(t) for t in terms), Fr(0))
        got = ex.md_to_fr(out[k])
        _nonoverlapping(out[k])
        assert abs(got - want) <= Fr(2) ** (12 - 64 * W) * mag, (k, float(got - want), float(mag))


def _words(v, N):
    return np.array([(v >> (64 * i)) & (2**64 - 1) for i in range(N)], dtype=np.uint64)


def _value(w):
    return sum(int(x) << (64 * i) for i, x in enumerate(w))


@pytest.mark.parametrize("N", range(1, 10))
def test_multiword_carry_chain(lib, N):
    """add_words: a + b + cin modulo 2^(64N) with the carry out, against
    Python integers, on carries that run through every word (all-ones
    operands, a carry-in into 2^(64N) - 1) and on random words."""
    P = ctypes.POINTER(ctypes.c_uint64)
    lib.xf_host_add_words.restype = ctypes.c_int
    lib.xf_host_add_words.argtypes = [ctypes.c_int, P, P, ctypes.c_uint64, P]
    M = 2**(64 * N)
    rng = np.random.default_rng(700 + N)
    cases = [(M - 1, 0, 1), (M - 1, M - 1, 1), (M - 1, M - 1, 0), (0, 0, 1), (M - 1, 1, 0),
             (2**63, 2**63, 0), (M // 2, M // 2, 1)]
    for _ in range(200):
        a = int.from_bytes(rng.bytes(8 * N), "little")
        b = int.from_bytes(rng.bytes(8 * N), "little")
        # words that are all ones or zero in places make long carry runs
        if rng.random() < 0.5:
            a |= sum((2**64 - 1) << (64 * i) for i in range(N) if rng.random() < 0.5)
        cases.append((a, b, int(rng.integers(0, 2))))
    for a, b, cin in cases:
        wa, wb = _words(a, N), _words(b, N)
        out = np.zeros(N, dtype=np.uint64)
        c = lib.xf_host_add_words(N, wa.ctypes.data_as(P), wb.ctypes.data_as(P), cin, out.ctypes.data_as(P))
        total = a + b + cin
        assert _value(out) == total % M and c == total // M, (hex(a), hex(b), cin)


def test_column_sum_with_counted_carries(lib):
    """add_count: s plus many words, the carries counted in c, equals the
    exact sum as the two-word number c:s."""
    P = ctypes.POINTER(ctypes.c_uint64)
    lib.xf_host_add_count.restype = None
    lib.xf_host_add_count.argtypes = [ctypes.c_int, P, ctypes.c_uint64, ctypes.c_uint64, P]
    rng = np.random.default_rng(731)
    for count in (0, 1, 2, 15, 16, 17):
        for s0 in (0, 2**64 - 1, int(rng.integers(0, 2**63))):
            vals = np.array([2**64 - 1] * (count // 2) + [int(x) for x in rng.integers(0, 2**63, count - count // 2)],
                            dtype=np.uint64)
            out = np.zeros(2, dtype=np.uint64)
            lib.xf_host_add_count(count, vals.ctypes.data_as(P), s0, 5, out.ctypes.data_as(P))
            total = s0 + 5 * 2**64 + sum(int(v) for v in vals)
            assert int(out[0]) + (int(out[1]) << 64) == total


# the shapes the fixed-point Newton steps use at widths V = 1, 2, 3, 4, 7:
# (V, V, V-1), (V, V, V) and (V, V+1, V)
MUL_TOP_SHAPES = [(1, 1, 0), (1, 2, 1), (2, 2, 1), (2, 2, 2), (2, 3, 2), (3, 3, 2), (3, 3, 3), (3, 4, 3),
                  (4, 4, 3), (4, 4, 4), (4, 5, 4), (7, 7, 6), (7, 7, 7), (7, 8, 7)]


@pytest.mark.parametrize("shape", MUL_TOP_SHAPES)
def test_mul_top_against_integer_products(lib, shape):
    """mul_top (the truncated word product of the fixed-point reciprocal and
    reciprocal square root) against the exact product of Python integers:
    the columns from LO up, the lowest short by fewer than NA + NB units
    (only column LO-1's products enter below it) and never above the exact
    value.  Operands: random words, all-ones words (every carry runs) and
    sparse words."""
    NA, NB, LO = shape
    nout = NA + NB - LO
    rng = np.random.default_rng(1200 + 100 * NA + 10 * NB + LO)
    full = (1 << 64) - 1
    cases = [(rng.integers(0, 2 ** 63, size=NA, dtype=np.uint64) * np.uint64(2) + np.uint64(1),
              rng.integers(0, 2 ** 63, size=NB, dtype=np.uint64) * np.uint64(2) + np.uint64(1)) for _ in range(60)]
    cases.append((np.full(NA, full, dtype=np.uint64), np.full(NB, full, dtype=np.uint64)))
    cases.append((np.array([0] * (NA - 1) + [1 << 63], dtype=np.uint64), np.full(NB, full, dtype=np.uint64)))
    cases.append((np.array([1] + [0] * (NA - 1), dtype=np.uint64), np.array([0] * (NB - 1) + [1], dtype=np.uint64)))
    fn = lib.xf_host_mul_top
    fn.restype = ctypes.c_int
    pu = ctypes.POINTER(ctypes.c_uint64)
    for a, b in cases:
        a = np.ascontiguousarray(a, dtype=np.uint64)
        b = np.ascontiguousarray(b, dtype=np.uint64)
        out = np.zeros(nout, dtype=np.uint64)
        assert fn(NA, NB, LO, a.ctypes.data_as(pu), b.ctypes.data_as(pu), out.ctypes.data_as(pu)) == 0
        A = sum(int(w) << (64 * i) for i, w in enumerate(a))
        B = sum(int(w) << (64 * i) for i, w in enumerate(b))
        exact = (A * B) >> (64 * LO)
        got = sum(int(w) << (64 * i) for i, w in enumerate(out))
        assert 0 <= exact - got < NA + NB, (shape, exact - got)

