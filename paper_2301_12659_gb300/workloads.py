"""Seeded synthetic workloads: the inputs of Newton's method on power series.

This module only draws random numbers and lays out inputs; it holds none of
the arithmetic of the method (no series products, no multiple double
operations), so both the CUDA path and the CPU oracle can take their inputs
from it.

Random numbers come from SplitMix64 (G. Steele, D. Lea, C. Flood, "Fast
splittable pseudorandom number generators", OOPSLA 2014), used as a
counter-based generator: draw ``i`` of a stream with seed ``s`` is
``mix(s + (i+1) * 0x9E3779B97F4A7C15 mod 2^64)``.  A double in [-1, 1) is
``2 * (z >> 11) * 2^-53 - 1``.

Systems follow the "columns of monomials" format of Section 3 generalised to
several monomials per equation:

    f_i(x(t)) = sum_{m in eq i} c_m(t) prod_{v in vars(m)} x_v(t) + cst_i(t)

with c_m(t) and cst_i(t) power series truncated at degree d (d+1
coefficients).  A multiple double (md) value with K limbs is stored limb by
limb (Section 1.2): every array is float64 with leading axes [K][C], C = 1
for real and 2 for complex data (real part, imaginary part).

Full-width md values: limb 0 is uniform in [-1, 1); limb l+1 is uniform in
(-ulp(limb l)/2, ulp(limb l)/2), so the limbs are nonoverlapping without any
renormalisation and every limb of the arithmetic is exercised.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field
from typing import Optional

import numpy as np

GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)
MASK64 = (1 << 64) - 1

#: Base seed; the workload of index c uses BASE_SEED + c.
BASE_SEED = 2301126590


def _mix(z: np.ndarray) -> np.ndarray:
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        return z ^ (z >> np.uint64(31))


def splitmix_stream(seed: int, count: int, offset: int = 0) -> np.ndarray:
    """Draws offset .. offset+count-1 of the SplitMix64 stream of ``seed``."""
    i = np.arange(offset + 1, offset + count + 1, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = np.uint64(seed & MASK64) + i * GAMMA
    return _mix(z)


def uniform_pm1(seed: int, count: int, offset: int = 0) -> np.ndarray:
    """Doubles in [-1, 1) with 53 random bits each."""
    z = splitmix_stream(seed, count, offset)
    u = (z >> np.uint64(11)).astype(np.float64) * 2.0 ** -53
    return 2.0 * u - 1.0


def substream_seed(seed: int, tag: int) -> int:
    """Seed of an independent substream (first draw of the stream seed+tag)."""
    return int(splitmix_stream((seed + tag) & MASK64, 1)[0])


class SplitMix64:
    """Sequential SplitMix64 for small structural draws (monomial shapes)."""

    def __init__(self, seed: int):
        self.seed = seed & MASK64
        self.count = 0

    def next(self) -> int:
        z = int(splitmix_stream(self.seed, 1, self.count)[0])
        self.count += 1
        return z

    def randint(self, lo: int, hi: int) -> int:
        """Uniform integer in [lo, hi] by the multiply-shift map of a 64-bit draw."""
        span = hi - lo + 1
        return lo + ((self.next() * span) >> 64)


def md_full_width(first: np.ndarray, K: int, seed: int) -> np.ndarray:
    """K-limb values with leading limbs ``first`` (shape S) -> array [K, *S]."""
    first = np.asarray(first, dtype=np.float64)
    out = np.zeros((K,) + first.shape, dtype=np.float64)
    out[0] = first
    for l in range(1, K):
        u = uniform_pm1(seed, first.size, offset=(l - 1) * first.size).reshape(first.shape)
        u = np.where(u == -1.0, 0.0, u)
        out[l] = u * (np.spacing(np.abs(out[l - 1])) * 0.5)
    return out


def random_md(shape, K: int, C: int, seed: int, unit_circle: bool = False) -> np.ndarray:
    """Random md values [K, C, *shape]: real uniform in [-1, 1), or complex
    uniform on the unit circle (to double precision) with full-width low limbs."""
    shape = tuple(shape)
    size = int(np.prod(shape)) if shape else 1
    out = np.zeros((K, C) + shape, dtype=np.float64)
    if C == 1 or not unit_circle:
        for c in range(C):
            lead = uniform_pm1(substream_seed(seed, 10 + c), size).reshape(shape)
            out[:, c] = md_full_width(lead, K, substream_seed(seed, 20 + c))
    else:
        theta = math.pi * uniform_pm1(substream_seed(seed, 10), size).reshape(shape)
        out[:, 0] = md_full_width(np.cos(theta), K, substream_seed(seed, 20))
        out[:, 1] = md_full_width(np.sin(theta), K, substream_seed(seed, 21))
    return out


@dataclass
class System:
    """A polynomial system with power series coefficients (host arrays).

    eq[m]      equation of monomial m (int32, [M])
    vptr       CSR offsets into vidx (int32, [M+1]); a repeated index is a power
    vidx       variable indices (int32, [nnz])
    coeff      coefficient series, float64 [K, C, M, d+1]
    cst        constant term series, float64 [K, C, n, d+1] (None until planted)
    """

    K: int
    C: int
    n: int
    d: int
    eq: np.ndarray
    vptr: np.ndarray
    vidx: np.ndarray
    coeff: np.ndarray
    cst: Optional[np.ndarray] = None
    name: str = ""
    meta: dict = field(default_factory=dict)

    @property
    def M(self) -> int:
        return int(self.eq.shape[0])

    @property
    def D(self) -> int:
        return self.d + 1

    def monomial_sizes(self) -> np.ndarray:
        return np.diff(self.vptr)

    def check(self) -> None:
        M, D = self.M, self.D
        assert self.eq.dtype == np.int32 and self.vptr.dtype == np.int32 and self.vidx.dtype == np.int32
        assert self.vptr.shape == (M + 1,) and self.vptr[0] == 0 and self.vptr[-1] == self.vidx.shape[0]
        assert np.all(np.diff(self.vptr) >= 1)
        assert np.all((self.eq >= 0) & (self.eq < self.n))
        assert np.all((self.vidx >= 0) & (self.vidx < self.n))
        assert self.coeff.shape == (self.K, self.C, M, D) and self.coeff.dtype == np.float64
        if self.cst is not None:
            assert self.cst.shape == (self.K, self.C, self.n, D)


@dataclass(frozen=True)
class PlantedConfig:
    """Planted-solution workload: every equation has `mono_per_eq` monomials
    of k ~ U{kmin..kmax} distinct variables plus the diagonal term diag*x_i."""

    name: str
    K: int
    C: int
    n: int
    d: int
    mono_per_eq: int
    kmin: int
    kmax: int
    diag: float
    steps: int
    tol: float
    index: int = 0
    unit_circle: bool = False
    noise: float = 1e-3

    @property
    def seed(self) -> int:
        return BASE_SEED + self.index


#: The three plain Newton workloads: double double (n=8, d=15), quad double
#: (n=64, d=31) and complex octo double (n=128, d=63).
CONFIGS = {
    "dd-real-n8-d15": PlantedConfig("dd-real-n8-d15", 2, 1, 8, 15, 4, 3, 3, 8.0, 6, 1e-28, 0),
    "qd-real-n64-d31": PlantedConfig("qd-real-n64-d31", 4, 1, 64, 31, 16, 2, 8, 64.0, 7, 1e-58, 1),
    "od-complex-n128-d63": PlantedConfig("od-complex-n128-d63", 8, 2, 128, 63, 32, 2, 16, 128.0, 8,
                                         1e-118, 2, unit_circle=True),
}

#: The adjoint workload: double double, n=64, d=31, built like the quad
#: double one; the loss is the Fabry-ratio loss of the converged series and
#: the gradient is taken with respect to every coefficient series.
ADJOINT_CONFIG = PlantedConfig("dd-real-n64-d31-adjoint", 2, 1, 64, 31, 16, 2, 8, 64.0, 7, 1e-28, 4)

#: The quad double recipe in the other precisions (the same system sizes),
#: for per-precision measurements: double double and real octo double.
EXTRA_CONFIGS = {
    "dd-real-n64-d31": PlantedConfig("dd-real-n64-d31", 2, 1, 64, 31, 16, 2, 8, 64.0, 7, 1e-28, 4),
    "od-real-n64-d31": PlantedConfig("od-real-n64-d31", 8, 1, 64, 31, 16, 2, 8, 64.0, 8, 1e-118, 7),
}


def small_config(K: int, C: int, n: int, d: int, mono_per_eq: int = 3, kmin: int = 1, kmax: int = 3,
                 diag: float = None, steps: int = 6, tol: float = None, index: int = 100) -> PlantedConfig:
    """A small planted workload of the same recipe (tests, smoke check)."""
    diag = float(n) if diag is None else diag
    tol = {1: 1e-12, 2: 1e-28, 4: 1e-58, 8: 1e-118}[K] if tol is None else tol
    return PlantedConfig(f"planted-K{K}-C{C}-n{n}-d{d}", K, C, n, d, mono_per_eq, kmin, min(kmax, n),
                         diag, steps, tol, index, unit_circle=(C == 2))


def planted_system(cfg: PlantedConfig):
    """Returns (system without cst, planted solution x*, start series x0).

    Draw order (all from substreams of cfg.seed): monomial shapes and variable
    choices, then coefficient series, then x*, then the start noise.  The
    start series is x*_0 (leading double) plus noise on the constant
    coefficient, every higher coefficient zero.
    """
    K, C, n, d, D = cfg.K, cfg.C, cfg.n, cfg.d, cfg.d + 1
    rng = SplitMix64(substream_seed(cfg.seed, 1))
    eq, vptr, vidx = [], [0], []
    diag_monomials = []
    for i in range(n):
        for _ in range(cfg.mono_per_eq):
            k = rng.randint(cfg.kmin, cfg.kmax)
            pool = list(range(n))
            chosen = []
            for t in range(k):  # partial Fisher-Yates: k distinct variables
                j = rng.randint(t, n - 1)
                pool[t], pool[j] = pool[j], pool[t]
                chosen.append(pool[t])
            eq.append(i)
            vidx.extend(chosen)
            vptr.append(len(vidx))
        diag_monomials.append(len(eq))
        eq.append(i)
        vidx.append(i)
        vptr.append(len(vidx))
    M = len(eq)
    eq = np.asarray(eq, dtype=np.int32)
    vptr = np.asarray(vptr, dtype=np.int32)
    vidx = np.asarray(vidx, dtype=np.int32)
    coeff = random_md((M, D), K, C, substream_seed(cfg.seed, 2), unit_circle=cfg.unit_circle)
    for m in diag_monomials:
        coeff[:, :, m, :] = 0.0
        coeff[0, 0, m, 0] = cfg.diag
    xstar = random_md((n, D), K, C, substream_seed(cfg.seed, 3), unit_circle=cfg.unit_circle)
    x0 = np.zeros((K, C, n, D), dtype=np.float64)
    noise = cfg.noise * uniform_pm1(substream_seed(cfg.seed, 4), C * n).reshape(C, n)
    x0[0, :, :, 0] = xstar[0, :, :, 0] + noise
    sysm = System(K, C, n, d, eq, vptr, vidx, coeff, None, cfg.name,
                  meta={"diag_monomials": np.asarray(diag_monomials, dtype=np.int32)})
    sysm.check()
    return sysm, xstar, x0


# ---------------------------------------------------------------------------
# batched homotopies: many independent planted systems of mixed size
# ---------------------------------------------------------------------------
@dataclass(frozen=True)
class BatchConfig:
    """`count` independent planted systems built like the quad double
    workload (16 monomials per equation of U{2..8} distinct variables,
    coefficients uniform in [-1, 1], diagonal term n*x_i, planted solution,
    1e-3 noise on x_0), each with n drawn from `n_choices` and d from
    `d_choices`; Newton stops by the batch stop rule with tolerance `tol`
    or after `max_steps` updates."""

    name: str
    K: int
    C: int
    count: int
    n_choices: tuple
    d_choices: tuple
    mono_per_eq: int = 16
    kmin: int = 2
    kmax: int = 8
    max_steps: int = 12
    tol: float = 1e-58
    index: int = 3
    noise: float = 1e-3

    @property
    def seed(self) -> int:
        return BASE_SEED + self.index


BATCH_CONFIGS = {
    "qd-real-batch4096": BatchConfig("qd-real-batch4096", 4, 1, 4096, (8, 16, 32, 64), (7, 15, 31)),
}


def _uniform_int(u: np.ndarray, lo: int, hi: int) -> np.ndarray:
    """Integers uniform in [lo, hi] from doubles u in [0, 1)."""
    return lo + np.floor(u * (hi - lo + 1)).astype(np.int64)


def batch_planted_systems(cfg: BatchConfig, count: Optional[int] = None):
    """The systems of a batch (the first `count` of them): lists of
    (System without cst, x*, x0).  System s draws from substreams of
    substream_seed(cfg.seed, 1000 + s): its size class, then its monomials
    (k uniform, the k distinct variables as the k smallest of n uniform
    keys), coefficients, x* and the start noise; the diagonal monomial of
    equation i follows its regular ones."""
    count = cfg.count if count is None else count
    K, C = cfg.K, cfg.C
    out = []
    for s in range(count):
        seed = substream_seed(cfg.seed, 1000 + s)
        u = 0.5 * (uniform_pm1(substream_seed(seed, 1), 2) + 1.0)
        n = int(cfg.n_choices[int(u[0] * len(cfg.n_choices))])
        d = int(cfg.d_choices[int(u[1] * len(cfg.d_choices))])
        D = d + 1
        mpe = cfg.mono_per_eq
        kmax = min(cfg.kmax, n)
        Mr = n * mpe
        ku = 0.5 * (uniform_pm1(substream_seed(seed, 2), Mr) + 1.0)
        k = _uniform_int(ku, cfg.kmin, kmax)
        keys = uniform_pm1(substream_seed(seed, 3), Mr * n).reshape(Mr, n)
        ranked = np.argsort(keys, axis=1, kind="stable")
        sizes = np.empty(Mr + n, dtype=np.int64)
        eq = np.empty(Mr + n, dtype=np.int32)
        vlists = []
        diag = []
        mi = 0
        for i in range(n):
            for r in range(mpe):
                m = i * mpe + r
                sizes[mi] = k[m]
                eq[mi] = i
                vlists.append(ranked[m, :k[m]])
                mi += 1
            sizes[mi] = 1
            eq[mi] = i
            vlists.append(np.array([i]))
            diag.append(mi)
            mi += 1
        vptr = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int32)
        vidx = np.concatenate(vlists).astype(np.int32)
        M = Mr + n
        coeff = random_md((M, D), K, C, substream_seed(seed, 4))
        coeff[:, :, diag, :] = 0.0
        coeff[0, 0, diag, 0] = float(n)
        xstar = random_md((n, D), K, C, substream_seed(seed, 5))
        x0 = np.zeros((K, C, n, D))
        x0[0, :, :, 0] = xstar[0, :, :, 0] + cfg.noise * uniform_pm1(substream_seed(seed, 6), C * n).reshape(C, n)
        sysm = System(K, C, n, d, eq, vptr, vidx, coeff, None, f"{cfg.name}#{s}",
                      meta={"diag_monomials": np.asarray(diag, dtype=np.int32)})
        out.append((sysm, xstar, x0))
    return out


# ---------------------------------------------------------------------------
# the paper's one-column systems (evaluation-only context workload)
# ---------------------------------------------------------------------------
def one_column_system(n: int, d: int, K: int, C: int = 1, index: int = 5, delta: float = 0.1):
    """One column of monomials with a lower triangular exponent matrix of
    ones (Section 3): equation i is x_0 x_1 ... x_i = b_i(t), monomial i has
    the i+1 variables 0..i and the constant coefficient series 1.  Returns
    (System with a zero constant term, x) where x_v(t) = exp(alpha_v t)
    truncated at degree d, alpha_v uniform in [-1, -1+delta] or [1-delta, 1],
    held in the leading limb (the series the paper evaluates at; the
    products of such series stay of moderate size).  Used to time the
    evaluation and differentiation the way the paper's Table 5 does."""
    D = d + 1
    seed = BASE_SEED + index
    eq = np.arange(n, dtype=np.int32)
    vptr = np.concatenate([[0], np.cumsum(np.arange(1, n + 1))]).astype(np.int32)
    vidx = np.concatenate([np.arange(i + 1) for i in range(n)]).astype(np.int32)
    coeff = np.zeros((K, C, n, D))
    coeff[0, 0, :, 0] = 1.0
    u = 0.5 * (uniform_pm1(substream_seed(seed, 1), 2 * n) + 1.0)
    alpha = (1.0 - delta * u[:n]) * np.where(u[n:] < 0.5, -1.0, 1.0)
    x = np.zeros((K, C, n, D))
    for j in range(D):
        x[0, 0, :, j] = alpha ** j / math.factorial(j)
    sysm = System(K, C, n, d, eq, vptr, vidx, coeff, np.zeros((K, C, n, D)), f"one-column-n{n}-d{d}-K{K}")
    sysm.check()
    return sysm, x


def section3_system(n: int, d: int, K: int, columns: int = 1, index: int = 6, delta: float = 0.1,
                    noise: float = 1e-3):
    """The columns-of-monomials systems of Section 3 for Newton: one column,
    x_0 x_1 ... x_i = b_i(t), or two columns, c1_i x_0...x_i +
    c2_i x_0...x_{n-1-i} = b_i(t) (the second exponent matrix has the rows of
    the first in reverse order), with the solution x_v(t) = exp(alpha_v t),
    alpha_v uniform in [-1, -1+delta] u [1-delta, 1].  The right hand sides
    b_i are the exponential series of the partial sums of the alpha_v (times
    c1_i, c2_i), held in the leading limb (double precision inputs).
    Returns (System with the constant term -b, start series: 1 + noise in
    the leading limb of x_0, every higher coefficient 0)."""
    D = d + 1
    seed = BASE_SEED + index
    u = 0.5 * (uniform_pm1(substream_seed(seed, 1), 4 * n) + 1.0)
    alpha = (1.0 - delta * u[:n]) * np.where(u[n:2 * n] < 0.5, -1.0, 1.0)
    eq, vlists, cvals = [], [], []
    c1 = 0.5 + u[2 * n:3 * n] if columns == 2 else np.ones(n)
    c2 = u[3 * n:] - 1.5
    for i in range(n):
        eq.append(i)
        vlists.append(np.arange(i + 1))
        cvals.append(c1[i])
        if columns == 2:
            eq.append(i)
            vlists.append(np.arange(n - i))
            cvals.append(c2[i])
    M = len(eq)
    vptr = np.concatenate([[0], np.cumsum([len(v) for v in vlists])]).astype(np.int32)
    vidx = np.concatenate(vlists).astype(np.int32)
    coeff = np.zeros((K, 1, M, D))
    coeff[0, 0, :, 0] = cvals
    fact = np.array([float(math.factorial(j)) for j in range(D)])
    csum = np.cumsum(alpha)
    cst = np.zeros((K, 1, n, D))
    for i in range(n):
        s1 = csum[i]
        b = c1[i] * s1 ** np.arange(D) / fact
        if columns == 2:
            s2 = csum[n - 1 - i]
            b = b + c2[i] * s2 ** np.arange(D) / fact
        cst[0, 0, i] = -b
    x0 = np.zeros((K, 1, n, D))
    x0[0, 0, :, 0] = 1.0 + noise * uniform_pm1(substream_seed(seed, 2), n)
    sysm = System(K, 1, n, d, np.asarray(eq, np.int32), vptr, vidx, coeff, cst,
                  f"section3-{columns}col-n{n}-d{d}-K{K}", meta={"alpha": alpha})
    sysm.check()
    return sysm, x0
