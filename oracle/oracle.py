"""ctypes binding of the CPU oracle (mdoracle.c).

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` use it.  The product package never imports
this module.  The oracle is a plain multiple double implementation written
from the paper (arXiv 2301.12659) that rounds the exact value of every
defining expression once; see the header comment of mdoracle.c.

All arrays are float64 numpy arrays with leading axes [K][C] (limbs, then
real/imaginary part), the layout of the product library.
"""
from __future__ import annotations

import ctypes
import os
import platform
import subprocess
import threading

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "mdoracle.c")
HDR = os.path.join(HERE, "mdoracle.h")
LIBPATH = os.path.join(HERE, "_build", f"libmdoracle-{platform.machine()}.so")

CFLAGS = ["-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared", "-fopenmp"]

_lock = threading.Lock()
_lib = None

ERRORS = {0: "ok", 1: "invalid argument", 2: "zero pivot in QR of A0", 3: "non-finite value",
          4: "expansion capacity exceeded"}


class OracleError(RuntimeError):
    pass


def build(force: bool = False) -> str:
    """Compile mdoracle.c into oracle/_build (gcc, no FMA contraction)."""
    os.makedirs(os.path.dirname(LIBPATH), exist_ok=True)
    newest = max(os.path.getmtime(SRC), os.path.getmtime(HDR))
    if force or not os.path.exists(LIBPATH) or os.path.getmtime(LIBPATH) < newest:
        tmp = LIBPATH + f".tmp{os.getpid()}"
        cmd = ["gcc", *CFLAGS, "-o", tmp, SRC, "-lm"]
        subprocess.run(cmd, check=True, capture_output=True, text=True)
        os.replace(tmp, LIBPATH)
    return LIBPATH


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = ctypes.CDLL(build())
            P = ctypes.c_void_p
            i = ctypes.c_int
            L.orc_set_threads.argtypes = [i]
            L.orc_get_threads.restype = i
            L.orc_md_binary.argtypes = [i, i, i, i, P, P, P]
            L.orc_md_sqrt.argtypes = [i, i, P, P]
            L.orc_series_mul.argtypes = [i, i, i, P, P, P]
            L.orc_evaluate.argtypes = [i, i, i, i, i, P, P, P, P, P, P, P, P]
            L.orc_planted_constant.argtypes = [i, i, i, i, i, P, P, P, P, P, P]
            L.orc_qr.argtypes = [i, i, i, P, P, P]
            L.orc_solve.argtypes = [i, i, i, i, P, P, P]
            L.orc_newton.argtypes = [i, i, i, i, i, P, P, P, P, P, P, i, P, P]
            L.orc_solve_late.argtypes = [i, i, i, i, P, P, i, i, P]
            L.orc_newton_late.argtypes = [i, i, i, i, i, P, P, P, P, P, P, i, i, i, P, P]
            L.orc_fabry_loss.argtypes = [i, i, i, P, P, P]
            L.orc_newton_staggered.argtypes = [i, i, i, i, i, P, P, P, P, P, P, i, i, P, P, P]
            L.orc_adjoint.argtypes = [i, i, i, i, i, P, P, P, P, P, P, P]
            L.orc_toeplitz_residual.argtypes = [i, i, i, i, P, P, P, P, i, P, P]
            for name in ("orc_md_binary", "orc_md_sqrt", "orc_series_mul", "orc_evaluate",
                         "orc_planted_constant", "orc_qr", "orc_solve", "orc_newton", "orc_solve_late",
                         "orc_newton_late", "orc_fabry_loss", "orc_adjoint",
                         "orc_newton_staggered", "orc_toeplitz_residual"):
                getattr(L, name).restype = i
            _lib = L
    return _lib


def set_threads(n: int) -> None:
    lib().orc_set_threads(int(n))


def get_threads() -> int:
    return int(lib().orc_get_threads())


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


def _i32(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.int32)


def _p(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _check(rc: int, what: str) -> None:
    if rc != 0:
        raise OracleError(f"{what}: {ERRORS.get(rc, rc)}")


OPS = {"add": 0, "sub": 1, "mul": 2, "div": 3}


def md_binary(op: str, a, b) -> np.ndarray:
    """Elementwise md op on arrays [K, C, N]."""
    a, b = _f64(a), _f64(b)
    K, C, N = a.shape
    r = np.zeros_like(a)
    _check(lib().orc_md_binary(OPS[op], K, C, N, _p(a), _p(b), _p(r)), f"md {op}")
    return r


def md_sqrt(a) -> np.ndarray:
    """Square roots of real md values [K, N]."""
    a = _f64(a)
    K, N = a.shape
    r = np.zeros_like(a)
    _check(lib().orc_md_sqrt(K, N, _p(a), _p(r)), "md sqrt")
    return r


def series_mul(a, b) -> np.ndarray:
    """Truncated product of two series [K, C, d+1]."""
    a, b = _f64(a), _f64(b)
    K, C, D = a.shape
    c = np.zeros_like(a)
    _check(lib().orc_series_mul(K, C, D - 1, _p(a), _p(b), _p(c)), "series mul")
    return c


def _sysargs(sysm):
    return (sysm.K, sysm.C, sysm.n, sysm.d, sysm.M, _i32(sysm.eq), _i32(sysm.vptr), _i32(sysm.vidx),
            _f64(sysm.coeff))


def evaluate(sysm, x, want_A: bool = True):
    """f(x(t)) [K,C,n,d+1] and, if asked, the Jacobian series A [K,C,d+1,n,n]."""
    K, C, n, d, M, eq, vptr, vidx, coeff = _sysargs(sysm)
    cst = None if sysm.cst is None else _f64(sysm.cst)
    x = _f64(x)
    f = np.zeros((K, C, n, d + 1))
    A = np.zeros((K, C, d + 1, n, n)) if want_A else None
    _check(lib().orc_evaluate(K, C, n, d, M, _p(eq), _p(vptr), _p(vidx), _p(coeff), _p(cst), _p(x),
                              _p(f), _p(A)), "evaluate")
    return (f, A) if want_A else f


def planted_constant(sysm, xstar) -> np.ndarray:
    """cst with f(x*) = 0: minus the system at x* without constant term, in
    octo double, rounded to K limbs."""
    K, C, n, d, M, eq, vptr, vidx, coeff = _sysargs(sysm)
    xstar = _f64(xstar)
    cst = np.zeros((K, C, n, d + 1))
    _check(lib().orc_planted_constant(K, C, n, d, M, _p(eq), _p(vptr), _p(vidx), _p(coeff), _p(xstar),
                                      _p(cst)), "planted constant")
    return cst


def qr(A0):
    """Householder QR of [K, C, n, n]: returns explicit (Q, R)."""
    A0 = _f64(A0)
    K, C, n, _ = A0.shape
    Q = np.zeros_like(A0)
    R = np.zeros_like(A0)
    _check(lib().orc_qr(K, C, n, _p(A0), _p(Q), _p(R)), "qr")
    return Q, R


def solve(A, b, late=None) -> np.ndarray:
    """Block lower triangular Toeplitz solve: A [K,C,d+1,n,n], b [K,C,n,d+1].
    late = (first_stage, limbs): the stated-accuracy variant whose stages
    k >= first_stage form their updates in `limbs` limbs."""
    A, b = _f64(A), _f64(b)
    K, C, D, n, _ = A.shape
    dx = np.zeros_like(b)
    if late is None:
        _check(lib().orc_solve(K, C, n, D - 1, _p(A), _p(b), _p(dx)), "solve")
    else:
        _check(lib().orc_solve_late(K, C, n, D - 1, _p(A), _p(b), int(late[0]), int(late[1]), _p(dx)), "solve")
    return dx


def toeplitz_residual(A, b, dx, rows=None):
    """Residual r_k = b_k - sum_{j<=k} A_j dx_{k-j} of the block Toeplitz
    system (md values [K,C,n,d+1]) and its 1-norm of leading doubles; with
    `rows`, the norm over those rows scaled by n / len(rows)."""
    A, b, dx = _f64(A), _f64(b), _f64(dx)
    K, C, D, n, _ = A.shape
    r = np.zeros_like(b)
    norm = np.zeros(1)
    rr = None if rows is None else _i32(rows)
    _check(lib().orc_toeplitz_residual(K, C, n, D - 1, _p(A), _p(b), _p(dx), _p(rr),
                                       0 if rr is None else int(rr.size), _p(r), _p(norm)), "toeplitz_residual")
    return r, float(norm[0])


def newton(sysm, x0, steps: int, late=None):
    """`steps` Newton iterations from x0; returns (x, hist[steps, 3]).
    late = (first_stage, limbs) as in solve()."""
    K, C, n, d, M, eq, vptr, vidx, coeff = _sysargs(sysm)
    cst = _f64(sysm.cst)
    x0 = _f64(x0)
    x = np.zeros_like(x0)
    hist = np.zeros((max(steps, 1), 3))
    ls, lk = (d + 1, K) if late is None else (int(late[0]), int(late[1]))
    _check(lib().orc_newton_late(K, C, n, d, M, _p(eq), _p(vptr), _p(vidx), _p(coeff), _p(cst), _p(x0),
                                 int(steps), ls, lk, _p(x), _p(hist)), "newton")
    return x, hist[:steps]


def fabry_loss(x):
    """L = sum_i x_{i,d}^2 + x_{0,d-1}/x_{0,d} of a real series x [K,1,n,d+1]:
    returns (L as [K] limbs, g = dL/dx like x)."""
    x = _f64(x)
    K, C, n, D = x.shape
    assert C == 1
    loss = np.zeros(K)
    g = np.zeros_like(x)
    _check(lib().orc_fabry_loss(K, n, D - 1, _p(x), _p(loss), _p(g)), "fabry_loss")
    return loss, g


def adjoint(sysm, x, g) -> np.ndarray:
    """Gradient [K,1,M,d+1] of a loss with dL/dx = g with respect to the
    coefficient series of a real system, at the converged series x."""
    K, C, n, d, M, eq, vptr, vidx, coeff = _sysargs(sysm)
    x, g = _f64(x), _f64(g)
    grad = np.zeros_like(coeff)
    _check(lib().orc_adjoint(K, C, n, d, M, _p(eq), _p(vptr), _p(vidx), _p(coeff), _p(x), _p(g), _p(grad)),
           "adjoint")
    return grad


def newton_staggered(sysm, x0, steps: int, first_steps: int):
    """Staggered Newton with the QR once: returns (x, hist[steps, 3], orders[steps])."""
    K, C, n, d, M, eq, vptr, vidx, coeff = _sysargs(sysm)
    cst = _f64(sysm.cst)
    x0 = _f64(x0)
    x = np.zeros_like(x0)
    hist = np.zeros((max(steps, 1), 3))
    orders = np.zeros(max(steps, 1), dtype=np.int32)
    _check(lib().orc_newton_staggered(K, C, n, d, M, _p(eq), _p(vptr), _p(vidx), _p(coeff), _p(cst), _p(x0),
                                      int(steps), int(first_steps), _p(x), _p(hist), _p(orders)), "newton_staggered")
    return x, hist[:steps], orders[:steps]
