"""Python binding of libmdnewton (include/mdnewton.h): argument marshalling only.

Every function keeps the name and argument order of its C entry point;
device buffers are passed as torch CUDA tensors (float64, contiguous, the
[K][C][...] structure-of-arrays layout of the header) and host structure
arrays as numpy int32 arrays.  All arithmetic runs in the CUDA kernels; there
is no CPU path: loading fails loudly when the library has not been built.

``Newton`` bundles the buffers a user needs (workspace, system, series) on
top of these calls.
"""
from __future__ import annotations

import ctypes
import os
import platform

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIBPATH = os.path.join(HERE, "_build", f"libmdnewton-{platform.machine()}.so")

STATUS = {0: "MDN_OK", 1: "MDN_EINVAL", 2: "MDN_ECUDA", 3: "MDN_ESINGULAR", 4: "MDN_ENONFINITE",
          5: "MDN_ENOTCONVERGED", 6: "MDN_ETIMEOUT", 7: "MDN_ESTATE", 8: "MDN_EWORKSPACE", 9: "MDN_ETOOLARGE"}
MDN_OK, MDN_EINVAL, MDN_ECUDA, MDN_ESINGULAR, MDN_ENONFINITE, MDN_ENOTCONVERGED, MDN_ETIMEOUT, \
    MDN_ESTATE, MDN_EWORKSPACE, MDN_ETOOLARGE = range(10)
MDN_STATIC_SCRATCH_BYTES = 2 << 20
MDN_MAX_STEPS = 64
MDN_MAX_DEGREE = 63

EXPORTS = ("mdn_create", "mdn_workspace_bytes", "mdn_load_system", "mdn_set_series", "mdn_newton",
           "mdn_get_series", "mdn_get_residual", "mdn_evaluate", "mdn_solve", "mdn_profile",
           "mdn_status_word", "mdn_last_error", "mdn_destroy", "mdn_evaluate_static", "mdn_set_late_updates", "mdn_adjoint", "mdn_fabry_loss", "mdn_set_residual_rows", "mdn_set_stagger",
           "mdn_ed_schedule", "mdn_batch_create", "mdn_batch_workspace_bytes", "mdn_batch_load", "mdn_batch_evaluate",
           "mdn_batch_solve", "mdn_batch_tiles", "mdn_batch_last_error", "mdn_batch_destroy", "mdn_residual",
           "mdn_md_scale", "mdn_set_wait_limit_ns")
BATCH_CONVERGED, BATCH_SINGULAR, BATCH_NONFINITE = 1, 2, 4
MDN_NUM_PHASES = 5
PHASES = ("evaluate", "assemble", "qr", "forward", "update")

_lib = None


class MdnError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


def load(path: str = None) -> ctypes.CDLL:
    """Load the shared library (built by paper_2301_12659_gb300.build)."""
    global _lib
    if _lib is not None:
        return _lib
    path = path or LIBPATH
    if not os.path.exists(path):
        raise RuntimeError(f"libmdnewton is not built ({path} missing): run paper_2301_12659_gb300.build.build()")
    L = ctypes.CDLL(path)
    P, I, D = ctypes.c_void_p, ctypes.c_int, ctypes.c_double
    L.mdn_create.argtypes = [ctypes.POINTER(P), I, I, I, I]
    L.mdn_workspace_bytes.argtypes = [P, I, P]
    L.mdn_workspace_bytes.restype = ctypes.c_size_t
    L.mdn_load_system.argtypes = [P, I, P, P, P, P, P, P, ctypes.c_size_t, P]
    L.mdn_set_series.argtypes = [P, P]
    L.mdn_newton.argtypes = [P, I, D, ctypes.POINTER(I), P]
    L.mdn_get_series.argtypes = [P, P]
    L.mdn_get_residual.argtypes = [P, P]
    L.mdn_evaluate.argtypes = [P, P, P, P]
    L.mdn_solve.argtypes = [P, P, P, P]
    L.mdn_profile.argtypes = [P, I, P, P]
    L.mdn_status_word.argtypes = [P]
    L.mdn_set_late_updates.argtypes = [P, I, I]
    L.mdn_adjoint.argtypes = [P, P, P, P]
    L.mdn_set_residual_rows.argtypes = [P, P, I]
    L.mdn_set_stagger.argtypes = [P, I]
    L.mdn_fabry_loss.argtypes = [P, P, P, P]
    L.mdn_residual.argtypes = [P, P, P, P, P, ctypes.POINTER(D)]
    L.mdn_md_scale.argtypes = [P, P, P, ctypes.c_int64, P]
    L.mdn_set_wait_limit_ns.argtypes = [P, ctypes.c_int64]
    L.mdn_batch_create.argtypes = [ctypes.POINTER(P), I, I, I, P, P, P, I, I]
    L.mdn_batch_workspace_bytes.argtypes = [P, P]
    L.mdn_batch_workspace_bytes.restype = ctypes.c_size_t
    L.mdn_batch_load.argtypes = [P, P, P, P, P, P, P, ctypes.c_size_t, P]
    L.mdn_batch_evaluate.argtypes = [P, P, P]
    L.mdn_batch_solve.argtypes = [P, P, P, I, D, P, P]
    L.mdn_batch_tiles.argtypes = [P, ctypes.POINTER(I), ctypes.POINTER(I)]
    L.mdn_batch_last_error.argtypes = [P]
    L.mdn_batch_last_error.restype = ctypes.c_char_p
    L.mdn_batch_destroy.argtypes = [P]
    L.mdn_evaluate_static.argtypes = [I, I, I, I, I, I, P, P, P, P, P, P, P, P]
    L.mdn_ed_schedule.argtypes = [I, I, P, I, ctypes.POINTER(I)]
    L.mdn_last_error.argtypes = [P]
    L.mdn_last_error.restype = ctypes.c_char_p
    L.mdn_destroy.argtypes = [P]
    for name in EXPORTS:
        if name not in ("mdn_workspace_bytes", "mdn_last_error", "mdn_destroy", "mdn_batch_workspace_bytes",
                        "mdn_batch_last_error", "mdn_batch_destroy"):
            getattr(L, name).restype = I
    _lib = L
    return L


def _ptr(t):
    """Device pointer of a tensor (or None)."""
    if t is None:
        return None
    if not t.is_cuda or t.dtype.is_floating_point and str(t.dtype) != "torch.float64":
        raise TypeError("expected a float64 CUDA tensor")
    if not t.is_contiguous():
        raise ValueError("expected a contiguous tensor")
    return ctypes.c_void_p(t.data_ptr())


def _host_i32(a):
    a = np.ascontiguousarray(a, dtype=np.int32)
    return a, a.ctypes.data_as(ctypes.c_void_p)


def _check(ctx, status: int):
    if status != MDN_OK:
        raise MdnError(status, mdn_last_error(ctx))


# ---- the C entry points -----------------------------------------------------

def mdn_create(limbs: int, is_complex: int, n: int, degree: int):
    h = ctypes.c_void_p()
    st = load().mdn_create(ctypes.byref(h), int(limbs), int(is_complex), int(n), int(degree))
    if st != MDN_OK:
        raise MdnError(st, f"mdn_create(limbs={limbs}, is_complex={is_complex}, n={n}, degree={degree})")
    return h


def mdn_workspace_bytes(ctx, n_monomials: int, var_ptr) -> int:
    arr, p = _host_i32(var_ptr)
    return int(load().mdn_workspace_bytes(ctx, int(n_monomials), p))


def mdn_load_system(ctx, n_monomials, eq_of_monomial, var_ptr, var_idx, coeff, const_term, workspace,
                    ws_bytes, cuda_stream) -> int:
    eq, peq = _host_i32(eq_of_monomial)
    vp, pvp = _host_i32(var_ptr)
    vi, pvi = _host_i32(var_idx)
    return load().mdn_load_system(ctx, int(n_monomials), peq, pvp, pvi, _ptr(coeff), _ptr(const_term),
                                  ctypes.c_void_p(workspace.data_ptr()), int(ws_bytes),
                                  ctypes.c_void_p(int(cuda_stream)))


def mdn_set_series(ctx, x) -> int:
    return load().mdn_set_series(ctx, _ptr(x))


def mdn_newton(ctx, max_steps: int, tol: float = 0.0):
    """Returns (status, steps_done, hist[steps_done, 3])."""
    done = ctypes.c_int(0)
    hist = np.zeros((max(int(max_steps), 1), 3))
    st = load().mdn_newton(ctx, int(max_steps), float(tol), ctypes.byref(done), hist.ctypes.data_as(ctypes.c_void_p))
    return st, done.value, hist[:done.value]


def mdn_get_series(ctx, x_out) -> int:
    return load().mdn_get_series(ctx, _ptr(x_out))


def mdn_get_residual(ctx, f_out) -> int:
    return load().mdn_get_residual(ctx, _ptr(f_out))


def mdn_evaluate(ctx, x, f_out, A_out=None) -> int:
    return load().mdn_evaluate(ctx, _ptr(x), _ptr(f_out), _ptr(A_out))


def mdn_solve(ctx, A, b, dx) -> int:
    return load().mdn_solve(ctx, _ptr(A), _ptr(b), _ptr(dx))


def mdn_profile(ctx, enable: int):
    """enable=1 starts the phase timers; enable=0 stops them and returns
    (status, ms per phase, kernel launches per phase)."""
    ms = np.zeros(MDN_NUM_PHASES)
    launches = np.zeros(MDN_NUM_PHASES, dtype=np.int64)
    st = load().mdn_profile(ctx, int(enable), ms.ctypes.data_as(ctypes.c_void_p),
                            launches.ctypes.data_as(ctypes.c_void_p))
    return st, ms, launches


def mdn_ed_schedule(k, groups):
    """The evaluation's product schedule for a monomial of k variables with
    `groups` products per warp wave: an int32 array [waves][groups][4] of
    (op, destination, a, b) records (host only; see include/mdnewton.h)."""
    L = load()
    nw = ctypes.c_int(0)
    st = L.mdn_ed_schedule(int(k), int(groups), None, 0, ctypes.byref(nw))
    if st != MDN_OK:
        raise ValueError(f"mdn_ed_schedule({k}, {groups}) returned {st}")
    ops = np.zeros((nw.value, int(groups), 4), dtype=np.int32)
    st = L.mdn_ed_schedule(int(k), int(groups), ops.ctypes.data_as(ctypes.c_void_p), nw.value * int(groups),
                           ctypes.byref(nw))
    if st != MDN_OK:
        raise ValueError(f"mdn_ed_schedule({k}, {groups}) returned {st}")
    return ops


def mdn_evaluate_static(limbs, is_complex, n, degree, n_monomials, n_var_refs, eq_of_monomial, var_ptr, var_idx,
                        coeff, const_term, x, f_out, cuda_stream) -> int:
    """f(x(t)) with no context and no device allocation (device int32
    structure tensors, device float64 series); see include/mdnewton.h."""
    for t in (eq_of_monomial, var_ptr, var_idx):
        if not t.is_cuda or str(t.dtype) != "torch.int32" or not t.is_contiguous():
            raise TypeError("expected contiguous int32 CUDA tensors for the structure")
    return load().mdn_evaluate_static(int(limbs), int(is_complex), int(n), int(degree), int(n_monomials),
                                      int(n_var_refs), ctypes.c_void_p(eq_of_monomial.data_ptr()),
                                      ctypes.c_void_p(var_ptr.data_ptr()), ctypes.c_void_p(var_idx.data_ptr()),
                                      _ptr(coeff), _ptr(const_term), _ptr(x), _ptr(f_out),
                                      ctypes.c_void_p(int(cuda_stream)))


def mdn_set_late_updates(ctx, first_stage: int, limbs: int) -> int:
    return load().mdn_set_late_updates(ctx, first_stage, limbs)


def mdn_adjoint(ctx, x, g, grad_out) -> int:
    return load().mdn_adjoint(ctx, _ptr(x), _ptr(g), _ptr(grad_out))


def mdn_fabry_loss(ctx, x, loss_out, g_out) -> int:
    return load().mdn_fabry_loss(ctx, _ptr(x), _ptr(loss_out), _ptr(g_out))


def mdn_set_residual_rows(ctx, rows) -> int:
    a, p = _host_i32(rows if rows is not None else [])
    return load().mdn_set_residual_rows(ctx, p if a.size else None, int(a.size))


def mdn_residual(ctx, A, b, dx, r_out=None):
    """Returns (status, norm): the residual b_k - sum_{j<=k} A_j dx_{k-j}
    into r_out (device, may be None) and its 1-norm of leading doubles."""
    norm = ctypes.c_double(0.0)
    st = load().mdn_residual(ctx, _ptr(A), _ptr(b), _ptr(dx), _ptr(r_out), ctypes.byref(norm))
    return st, norm.value


def mdn_md_scale(ctx, s, a, count: int, out) -> int:
    return load().mdn_md_scale(ctx, _ptr(s), _ptr(a), int(count), _ptr(out))


def mdn_set_wait_limit_ns(ctx, limit_ns: int) -> int:
    return load().mdn_set_wait_limit_ns(ctx, int(limit_ns))


def mdn_set_stagger(ctx, first_steps: int) -> int:
    return load().mdn_set_stagger(ctx, int(first_steps))


def mdn_status_word(ctx) -> int:
    return load().mdn_status_word(ctx)


def mdn_last_error(ctx) -> str:
    return load().mdn_last_error(ctx).decode()


def mdn_destroy(ctx) -> None:
    load().mdn_destroy(ctx)


# ---- convenience -------------------------------------------------------------

class Newton:
    """A loaded system on the current CUDA device: owns the device buffers
    (workspace, coefficient and constant series) as torch tensors."""

    def __init__(self, system, stream=None):
        import torch

        self.torch = torch
        s = system
        self.K, self.C, self.n, self.d = s.K, s.C, s.n, s.d
        self.shape_series = (s.K, s.C, s.n, s.d + 1)
        self.shape_A = (s.K, s.C, s.d + 1, s.n, s.n)
        self.ctx = mdn_create(s.K, s.C - 1, s.n, s.d)
        dev = torch.device("cuda", torch.cuda.current_device())
        self.stream = stream or torch.cuda.current_stream()
        self.ws_bytes = mdn_workspace_bytes(self.ctx, s.M, s.vptr)
        if self.ws_bytes == 0:
            raise MdnError(MDN_EINVAL, "workspace size")
        self.workspace = torch.empty(self.ws_bytes + 256, dtype=torch.uint8, device=dev)
        off = (-self.workspace.data_ptr()) % 256
        self.workspace = self.workspace[off:off + self.ws_bytes]
        self.coeff = torch.as_tensor(np.ascontiguousarray(s.coeff), device=dev)
        cst = s.cst if s.cst is not None else np.zeros(self.shape_series)
        self.cst = torch.as_tensor(np.ascontiguousarray(cst), device=dev)
        _check(self.ctx, mdn_load_system(self.ctx, s.M, s.eq, s.vptr, s.vidx, self.coeff, self.cst,
                                         self.workspace, self.ws_bytes, self.stream.cuda_stream))

    def set_constant(self, cst):
        """Replace the constant term series (device copy, same shape)."""
        self.cst.copy_(cst if isinstance(cst, self.torch.Tensor) else self.torch.as_tensor(cst))

    def set_series(self, x):
        x = x if isinstance(x, self.torch.Tensor) else self.torch.as_tensor(np.ascontiguousarray(x), device=self.cst.device)
        self._x_in = x.contiguous()
        _check(self.ctx, mdn_set_series(self.ctx, self._x_in))

    def newton(self, steps: int, tol: float = 0.0):
        st, done, hist = mdn_newton(self.ctx, steps, tol)
        self.steps_done = done
        if st not in (MDN_OK,):
            raise MdnError(st, mdn_last_error(self.ctx))
        return hist

    def series(self):
        x = self.torch.empty(self.shape_series, dtype=self.torch.float64, device=self.cst.device)
        _check(self.ctx, mdn_get_series(self.ctx, x))
        return x

    def evaluate(self, x, want_A: bool = True):
        dev = self.cst.device
        x = x if isinstance(x, self.torch.Tensor) else self.torch.as_tensor(np.ascontiguousarray(x), device=dev)
        f = self.torch.empty(self.shape_series, dtype=self.torch.float64, device=dev)
        A = self.torch.empty(self.shape_A, dtype=self.torch.float64, device=dev) if want_A else None
        _check(self.ctx, mdn_evaluate(self.ctx, x.contiguous(), f, A))
        return (f, A) if want_A else f

    def solve(self, A, b):
        dev = self.cst.device
        A = A if isinstance(A, self.torch.Tensor) else self.torch.as_tensor(np.ascontiguousarray(A), device=dev)
        b = b if isinstance(b, self.torch.Tensor) else self.torch.as_tensor(np.ascontiguousarray(b), device=dev)
        dx = self.torch.empty(self.shape_series, dtype=self.torch.float64, device=dev)
        _check(self.ctx, mdn_solve(self.ctx, A.contiguous(), b.contiguous(), dx))
        return dx

    def adjoint(self, x, g):
        """Gradient [K, 1, M, d+1] (md) of a loss with dL/dx = g (md) with
        respect to the coefficient series, at the series x."""
        grad = self.torch.empty_like(self.coeff)
        _check(self.ctx, mdn_adjoint(self.ctx, x.contiguous(), g.contiguous(), grad))
        return grad

    def fabry_loss(self, x):
        """(L as [K] limbs, dL/dx) of L = sum_i x_{i,d}^2 + x_{0,d-1}/x_{0,d}."""
        loss = self.torch.empty(self.K, dtype=self.torch.float64, device=self.cst.device)
        g = self.torch.empty_like(x)
        _check(self.ctx, mdn_fabry_loss(self.ctx, x.contiguous(), loss, g))
        return loss, g

    def residual(self, A, b, dx, want_r: bool = True):
        """(r or None, ||r||_1) of r_k = b_k - sum_{j<=k} A_j dx_{k-j}."""
        dev = self.cst.device
        A, b, dx = (t if isinstance(t, self.torch.Tensor) else self.torch.as_tensor(np.ascontiguousarray(t), device=dev)
                    for t in (A, b, dx))
        r = self.torch.empty(self.shape_series, dtype=self.torch.float64, device=dev) if want_r else None
        st, norm = mdn_residual(self.ctx, A.contiguous(), b.contiguous(), dx.contiguous(), r)
        _check(self.ctx, st)
        return r, norm

    def md_scale(self, s, a):
        """s * a entry by entry (md multiplication) for one md value s
        ([K, C]) and an md array a ([K, C, ...])."""
        a = a.contiguous()
        out = self.torch.empty_like(a)
        count = a[0, 0].numel()
        _check(self.ctx, mdn_md_scale(self.ctx, s.contiguous(), a, count, out))
        return out

    def set_wait_limit_ns(self, limit_ns: int):
        """Bound of every device wait (nanoseconds; default 2e9)."""
        _check(self.ctx, mdn_set_wait_limit_ns(self.ctx, limit_ns))

    def set_residual_rows(self, rows):
        """Residual monitor on these rows only (scaled by n/len(rows)); an
        empty list restores all rows."""
        _check(self.ctx, mdn_set_residual_rows(self.ctx, rows))

    def set_stagger(self, first_steps: int):
        """Staggered orders with the QR once (0: plain Newton)."""
        _check(self.ctx, mdn_set_stagger(self.ctx, first_steps))

    def set_late_updates(self, first_stage: int, limbs: int):
        """Stages k >= first_stage form their right hand side updates in
        `limbs` (= K/2) limbs; limbs = K switches the variant off."""
        _check(self.ctx, mdn_set_late_updates(self.ctx, first_stage, limbs))

    def close(self):
        if self.ctx is not None:
            mdn_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ---- batched systems ----------------------------------------------------------

def _bcheck(b, status: int):
    if status != MDN_OK:
        raise MdnError(status, load().mdn_batch_last_error(b).decode())


def mdn_batch_create(limbs: int, is_complex: int, n, degree, n_monomials, threads_per_block: int = 0,
                     blocks_per_sm: int = 0):
    h = ctypes.c_void_p()
    an, pn = _host_i32(n)
    ad, pd = _host_i32(degree)
    am, pm = _host_i32(n_monomials)
    st = load().mdn_batch_create(ctypes.byref(h), int(limbs), int(is_complex), int(an.size), pn, pd, pm,
                                 int(threads_per_block), int(blocks_per_sm))
    if st != MDN_OK:
        raise MdnError(st, "mdn_batch_create")
    return h


def mdn_batch_workspace_bytes(b, var_ptr) -> int:
    a, p = _host_i32(var_ptr)
    return int(load().mdn_batch_workspace_bytes(b, p))


def mdn_batch_load(b, eq_of_monomial, var_ptr, var_idx, coeff, const_term, workspace, ws_bytes, cuda_stream) -> int:
    aeq, peq = _host_i32(eq_of_monomial)
    avp, pvp = _host_i32(var_ptr)
    avi, pvi = _host_i32(var_idx)
    return load().mdn_batch_load(b, peq, pvp, pvi, _ptr(coeff), _ptr(const_term),
                                 ctypes.c_void_p(workspace.data_ptr()), int(ws_bytes),
                                 ctypes.c_void_p(int(cuda_stream)))


def mdn_batch_evaluate(b, x, f_out) -> int:
    return load().mdn_batch_evaluate(b, _ptr(x), _ptr(f_out))


def mdn_batch_solve(b, x0, x, max_steps: int, tol: float, steps_out, flags_out) -> int:
    """steps_out, flags_out: host int32 arrays of the batch's count."""
    assert steps_out.dtype == np.int32 and flags_out.dtype == np.int32
    return load().mdn_batch_solve(b, _ptr(x0), _ptr(x), int(max_steps), float(tol),
                                  steps_out.ctypes.data_as(ctypes.c_void_p), flags_out.ctypes.data_as(ctypes.c_void_p))


def mdn_batch_tiles(b):
    t, k = ctypes.c_int(0), ctypes.c_int(0)
    st = load().mdn_batch_tiles(b, ctypes.byref(t), ctypes.byref(k))
    return st, t.value, k.value


def mdn_batch_last_error(b) -> str:
    return load().mdn_batch_last_error(b).decode()


def mdn_batch_destroy(b) -> None:
    load().mdn_batch_destroy(b)


class Batch:
    """Many independent systems (one K and C) solved in one persistent
    launch; see the mdn_batch_* calls of include/mdnewton.h.  Series of all
    systems travel packed: the concatenation of the [K][C][n_s][d_s+1]
    blocks."""

    def __init__(self, systems, threads_per_block: int = 0, blocks_per_sm: int = 0, stream=None):
        import torch

        self.torch = torch
        K, C = systems[0].K, systems[0].C
        if any(s.K != K or s.C != C for s in systems):
            raise ValueError("one K and C for the whole batch")
        self.K, self.C, self.count = K, C, len(systems)
        self.n = np.array([s.n for s in systems], dtype=np.int32)
        self.deg = np.array([s.d for s in systems], dtype=np.int32)
        self.M = np.array([s.M for s in systems], dtype=np.int32)
        sizes = K * C * self.n.astype(np.int64) * (self.deg.astype(np.int64) + 1)
        self.series_off = np.concatenate([[0], np.cumsum(sizes)])
        eq = np.concatenate([s.eq for s in systems]).astype(np.int32)
        nnz = np.array([s.vptr[-1] for s in systems], dtype=np.int64)
        base = np.concatenate([[0], np.cumsum(nnz)[:-1]])
        vptr = np.concatenate([s.vptr[:-1].astype(np.int64) + b0 for s, b0 in zip(systems, base)] +
                              [np.array([nnz.sum()])]).astype(np.int32)
        vidx = np.concatenate([s.vidx for s in systems]).astype(np.int32)
        dev = torch.device("cuda", torch.cuda.current_device())
        self.dev = dev
        self.stream = stream or torch.cuda.current_stream()
        self.b = mdn_batch_create(K, C - 1, self.n, self.deg, self.M, threads_per_block, blocks_per_sm)
        self.ws_bytes = mdn_batch_workspace_bytes(self.b, vptr)
        if self.ws_bytes == 0:
            raise MdnError(MDN_EINVAL, "mdn_batch_workspace_bytes")
        ws = torch.empty(self.ws_bytes + 256, dtype=torch.uint8, device=dev)
        off = (-ws.data_ptr()) % 256
        self.workspace = ws[off:off + self.ws_bytes]
        self.coeff = torch.as_tensor(np.concatenate([np.ascontiguousarray(s.coeff).reshape(-1) for s in systems]),
                                     device=dev)
        self.cst = self.pack([s.cst if s.cst is not None else np.zeros((K, C, s.n, s.D)) for s in systems])
        _bcheck(self.b, mdn_batch_load(self.b, eq, vptr, vidx, self.coeff, self.cst, self.workspace, self.ws_bytes,
                                       self.stream.cuda_stream))

    def pack(self, series):
        """List of [K, C, n_s, d_s+1] arrays -> packed device tensor."""
        flat = np.concatenate([np.ascontiguousarray(x, dtype=np.float64).reshape(-1) for x in series])
        return self.torch.as_tensor(flat, device=self.dev)

    def unpack(self, packed):
        """Packed tensor -> list of host arrays [K, C, n_s, d_s+1]."""
        h = packed.detach().cpu().numpy()
        return [h[self.series_off[s]:self.series_off[s + 1]].reshape(self.K, self.C, int(self.n[s]),
                                                                     int(self.deg[s]) + 1)
                for s in range(self.count)]

    def set_constant(self, packed):
        self.cst.copy_(packed)

    def tiles(self):
        st, t, k = mdn_batch_tiles(self.b)
        _bcheck(self.b, st)
        return t, k

    def evaluate(self, x):
        f = self.torch.empty_like(x)
        _bcheck(self.b, mdn_batch_evaluate(self.b, x, f))
        return f

    def solve(self, x0, max_steps: int, tol: float, x=None):
        """Returns (x packed, steps [count], flags [count])."""
        x = self.torch.empty_like(x0) if x is None else x
        steps = np.zeros(self.count, dtype=np.int32)
        flags = np.zeros(self.count, dtype=np.int32)
        _bcheck(self.b, mdn_batch_solve(self.b, x0, x, max_steps, tol, steps, flags))
        return x, steps, flags

    def close(self):
        if getattr(self, "b", None) is not None:
            mdn_batch_destroy(self.b)
            self.b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
