"""The library's multiple double primitives (csrc/md.cuh: TwoSum/TwoProd
based add, sub, mul, fma, division, reciprocal, square root and reciprocal
square root, the complex product) and its integer-limb extended floats
(csrc/xf.cuh, device build with the inline-PTX carry chains) run on the GPU
through a test-only probe (tests/native/md_probe.cu) and are checked against
exact rationals (Section 1.2: an md value is the exact sum of its limbs).

Bounds: the md operations are of the sloppy kind, |md_add(a, b) - (a + b)|
<= 2K^2 2^(-53K) (|a| + |b|) and |md_mul(a, b) - ab| <= 2K^2 2^(-53K) |ab|;
division, reciprocal and square roots to 2K^2 2^(-53K) relative (8K^2 for
the root of a root); the extended floats to a few units of 2^(-64W), W
mantissa words (64W >= 53K + 11)."""
import ctypes
import os
import platform
import subprocess
from fractions import Fraction as Fr

import numpy as np
import pytest

from paper_2301_12659_gb300 import workloads as wl
from tests import exact as ex
from tests.gpu_util import need_gpu

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
SRC = os.path.join(HERE, "native", "md_probe.cu")
SO = os.path.join(HERE, "native", "_build", f"md_probe-{platform.machine()}.so")
WORDS = {1: 1, 2: 2, 4: 4, 8: 7}


@pytest.fixture(scope="module")
def probe():
    need_gpu()
    os.makedirs(os.path.dirname(SO), exist_ok=True)
    inc = os.path.join(ROOT, "paper_2301_12659_gb300", "csrc")
    if not os.path.exists(SO) or os.path.getmtime(SO) < max(os.path.getmtime(SRC), os.path.getmtime(
            os.path.join(inc, "md.cuh")), os.path.getmtime(os.path.join(inc, "xf.cuh"))):
        subprocess.run([os.environ.get("NVCC", "nvcc"), "-gencode", "arch=compute_103a,code=sm_103a", "-O3",
                        "-std=c++17", "-fmad=false", "-shared", "-Xcompiler", "-fPIC", "-I", inc, "-o", SO, SRC],
                       check=True)
    lib = ctypes.CDLL(SO)
    P = ctypes.c_void_p
    lib.md_probe.argtypes = [ctypes.c_int] * 5 + [P, P, P]
    lib.md_probe.restype = ctypes.c_int
    return lib


def run(lib, K, op, a, b):
    a = np.ascontiguousarray(a, dtype=np.float64)
    b = np.ascontiguousarray(b, dtype=np.float64)
    N = a.shape[0]
    width = 2 * K if (op == 8 or op >= 10) else K
    r = np.zeros((N, width))
    rc = lib.md_probe(K, op, N, a.size, r.size, a.ctypes.data_as(ctypes.c_void_p), b.ctypes.data_as(ctypes.c_void_p),
                      r.ctypes.data_as(ctypes.c_void_p))
    assert rc == 0
    return r


def values(K, count, seed, spread=30, positive=False):
    v = wl.random_md((count,), K, 1, seed)[:, 0].T.copy()
    rng = np.random.default_rng(seed)
    v *= np.exp2(rng.integers(-spread, spread + 1, size=count))[:, None]
    if positive:
        v = np.where(v[:, :1] < 0, -v, v)
    return v


def operands(K, seed):
    """Pairs with random magnitudes, near-cancellation (b = -a + small) and zeros."""
    a = values(K, 96, seed)
    b = values(K, 96, seed + 1)
    c = values(K, 32, seed + 2)
    small = values(K, 32, seed + 3, spread=0) * 2.0 ** -60
    b_cancel = -c + 0.0
    b_cancel[:, -1] += small[:, 0] * np.spacing(np.abs(c[:, -1]))  # differs in the last limb
    za = np.zeros((4, K))
    zb = values(K, 4, seed + 4)
    return np.vstack([a, c, za, zb]), np.vstack([b, b_cancel, zb, za])


def rows_fr(m):
    return [ex.md_to_fr(row) for row in m]


@pytest.mark.parametrize("K", [2, 4, 8])
def test_md_add_sub_mul_fma(probe, K):
    a, b = operands(K, 60 + K)
    A, B = rows_fr(a), rows_fr(b)
    bound = Fr(2 * K * K) * Fr(2) ** (-53 * K)
    for op, f, size in ((0, lambda x, y: x + y, lambda x, y: abs(x) + abs(y)),
                        (1, lambda x, y: x - y, lambda x, y: abs(x) + abs(y)),
                        (2, lambda x, y: x * y, lambda x, y: abs(x * y)),
                        (3, lambda x, y: x + x * y, lambda x, y: abs(x) + abs(x * y))):
        r = run(probe, K, op, a, b)
        for i, (x, y) in enumerate(zip(A, B)):
            assert abs(ex.md_to_fr(r[i]) - f(x, y)) <= bound * size(x, y), (op, i)


@pytest.mark.parametrize("K", [2, 4, 8])
def test_md_division_and_roots(probe, K):
    a = values(K, 64, 80 + K)
    b = values(K, 64, 81 + K)
    bound = Fr(2 * K * K) * Fr(2) ** (-53 * K)
    r = run(probe, K, 4, a, b)
    for i, (x, y) in enumerate(zip(rows_fr(a), rows_fr(b))):
        assert abs(ex.md_to_fr(r[i]) * y - x) <= bound * abs(x), i
    r = run(probe, K, 5, a, b)
    for i, x in enumerate(rows_fr(a)):
        assert abs(ex.md_to_fr(r[i]) * x - 1) <= bound, i
    p = values(K, 64, 82 + K, positive=True)
    P = rows_fr(p)
    r = run(probe, K, 6, p, p)
    for i, x in enumerate(P):
        s = ex.md_to_fr(r[i])
        assert abs(s * s - x) <= 4 * bound * x, i
    r = run(probe, K, 7, p, p)
    for i, x in enumerate(P):
        y = ex.md_to_fr(r[i])
        assert abs(y * y * x - 1) <= 4 * bound, i
    # exact cases and zero
    z = np.zeros((3, K))
    z[0, 0], z[1, 0], z[2, 0] = 4.0, 0.25, 0.0
    r = run(probe, K, 6, z, z)
    assert [ex.md_to_fr(v) for v in r] == [2, Fr(1, 2), 0]


@pytest.mark.parametrize("K", [2, 4, 8])
def test_md_complex_product(probe, K):
    re_a, im_a = values(K, 48, 90 + K), values(K, 48, 91 + K)
    re_b, im_b = values(K, 48, 92 + K), values(K, 48, 93 + K)
    r = run(probe, K, 8, np.hstack([re_a, im_a]), np.hstack([re_b, im_b]))
    bound = Fr(4 * K * K) * Fr(2) ** (-53 * K)
    for i in range(48):
        a = (ex.md_to_fr(re_a[i]), ex.md_to_fr(im_a[i]))
        b = (ex.md_to_fr(re_b[i]), ex.md_to_fr(im_b[i]))
        exact = ex.mul(a, b)
        size = (abs(a[0]) + abs(a[1])) * (abs(b[0]) + abs(b[1]))
        assert abs(ex.md_to_fr(r[i, :K]) - exact[0]) <= bound * size
        assert abs(ex.md_to_fr(r[i, K:]) - exact[1]) <= bound * size


@pytest.mark.parametrize("K", [1, 2, 4, 8])
def test_xf_device_operations(probe, K):
    """The device build of xf.cuh (carry chains in the PTX condition code)
    against exact rationals: add/sub with cancellation, mul, 1/a, 1/sqrt(a)
    and the md -> xf -> md round trip, each to a few units of 2^(-64W)."""
    W = WORDS[K]
    a, b = operands(K, 100 + K)
    A, B = rows_fr(a), rows_fr(b)
    tol = Fr(2) ** (8 - 64 * W)
    r = run(probe, K, 10, a, b)
    for i, (x, y) in enumerate(zip(A, B)):
        assert abs(ex.md_to_fr(r[i]) - (x + y)) <= tol * (abs(x) + abs(y)), i
    r = run(probe, K, 11, a, b)
    for i, (x, y) in enumerate(zip(A, B)):
        assert abs(ex.md_to_fr(r[i]) - (x - y)) <= tol * (abs(x) + abs(y)), i
    r = run(probe, K, 12, a, b)
    for i, (x, y) in enumerate(zip(A, B)):
        assert abs(ex.md_to_fr(r[i]) - x * y) <= tol * abs(x * y), i
    nz = [i for i, x in enumerate(A) if x != 0]
    r = run(probe, K, 13, a, b)
    for i in nz:
        assert abs(ex.md_to_fr(r[i]) * A[i] - 1) <= tol, i
    p = values(K, 64, 110 + K, positive=True)
    r = run(probe, K, 14, p, p)
    for i, x in enumerate(rows_fr(p)):
        y = ex.md_to_fr(r[i])
        assert abs(y * y * x - 1) <= tol, i
    r = run(probe, K, 15, a, b)
    for i, x in enumerate(A):
        assert abs(ex.md_to_fr(r[i]) - x) <= Fr(2) ** (1 - 64 * W) * abs(x), i
