"""Seeded synthetic workloads shared by the oracle, the tests and the benchmark.

This module holds only input definitions: problem parameters and seeded random
test polynomials.  It contains none of the usFFT arithmetic (no lattice, no
transform, no solve, no selection), so both the CPU oracle and the CUDA path may
import it without sharing method code.

The PDE workloads stand in for the paper's numerical examples (Sec. 4.2-4.4,
Table 4.1): the same stochastic dimensions, search domains, sparsities and
coefficient families, on uniform meshes instead of the paper's unstructured
mesh (which is not available).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field, replace
from typing import Optional

import numpy as np

# problem kinds
PDE_1D = 1
PDE_2D = 2
TRIGPOLY = 3

# coefficient models (periodic in y, so no periodization is needed; Sec. 3.2)
COEF_AFFINE_SIN = 1     # a = 1 + sum_j c j^-mu psi_j(x) sin(2 pi y_j)
COEF_LOGNORMAL_SIN = 2  # a = exp(sum_j c j^-mu psi_j(x) sin(2 pi y_j))

MAP_PERIODIC = 0        # Theta_j = sin(2 pi y_j), y on the torus
MAP_TENT = 1            # Theta_j = y_j uniform on [alpha, beta], tent periodization
MAP_NORMAL = 2          # Theta_j = y_j standard normal, tau_1 o tau_{2,Delta} periodization

PRECISION_FP64 = 0
PRECISION_MIXED = 1
PRECISION_MIXED_JACOBI = 2
PRECISION_FP64_DST = 3


@dataclass
class Problem:
    """The parametric elliptic problem -div(a(x,y) grad u) = f, u = 0 on the boundary (Eq. (1.1))."""
    kind: int
    n: int                      # interior nodes per side (PDE); G = n (1-D) or n*n (2-D)
    d: int                      # stochastic dimension
    coef_model: int = COEF_AFFINE_SIN
    coef_scale: float = 0.9 * 6.0 / math.pi ** 2   # c = 0.9/zeta(2) (Sec. 4.3)
    coef_decay: float = 2.0                        # mu
    f_const: float = 1.0
    # TRIGPOLY black box: per node g a list of (frequency, coefficient) terms
    tp_freqs: Optional[np.ndarray] = None   # int8 [G][nterms][d]
    tp_coefs: Optional[np.ndarray] = None   # complex128 [G][nterms] (0 pads unused slots)
    # parameter map (Sec. 3.2): periodic model (Theta_j = sin 2 pi y_j), affine model with the
    # tent periodization on [map_alpha, map_beta], lognormal model with tau_1 o tau_{2,Delta}
    theta_map: int = 0                      # MAP_PERIODIC | MAP_TENT | MAP_NORMAL
    map_alpha: float = -1.0
    map_beta: float = 1.0
    map_shift: float = 0.0                  # Delta of the lognormal periodization

    @property
    def G(self) -> int:
        if self.kind == PDE_1D:
            return self.n
        if self.kind == PDE_2D:
            return self.n * self.n
        return int(self.tp_freqs.shape[0])


@dataclass
class Params:
    """Detection parameters of Algorithm 1 (search domain [-N,N]^d, s, s_local, theta, r)."""
    N: int
    s: int
    s_local: int
    delta: float
    delta_is_relative: bool
    r: int
    seed: int
    precision: int = PRECISION_FP64
    hbm_budget_bytes: int = 0          # 0 = no budget
    max_cg_iters: int = 4000
    max_lattice_trials: int = 64
    cg_tol: float = 0.0                # 0 = library default
    rr_lattices: int = 0               # 0: one reconstructing lattice per coupled step; odd L >= 1:
                                       # L random rank-1 lattices (Algorithm A), median estimate
    rr_size_factor: float = 2.0        # random lattice size >= factor * max(|I^(1..t-1)|, |I^(t)|, s~)
    max_lattice_sizes: int = 400       # sizes the reconstructing-lattice search tries


@dataclass
class Workload:
    name: str
    problem: Problem
    params: Params
    note: str = ""


def c1(seed: int = 1) -> Workload:
    """1-D, 31 interior nodes, d=4, Gamma=[-16,16]^4, s=50, delta=1e-12 relative, r=1."""
    return Workload(
        "c1_1d_n31_d4",
        Problem(kind=PDE_1D, n=31, d=4),
        Params(N=16, s=50, s_local=50, delta=1e-12, delta_is_relative=True, r=1, seed=seed),
        "1-D P1 FE, f=1, a=1+sum_{j<=4} 0.5471 j^-2 sin(j pi x) sin(2 pi y_j)")


def c2(seed: int = 1) -> Workload:
    """2-D 63x63 interior (64x64 squares, 8192 triangles), d=10, Gamma=[-32,32]^10, s=500, delta=1e-10 rel, r=2."""
    return Workload(
        "c2_2d_n63_d10",
        Problem(kind=PDE_2D, n=63, d=10),
        Params(N=32, s=500, s_local=500, delta=1e-10, delta_is_relative=True, r=2, seed=seed),
        "2-D P1 FE on the unit square, f=1, affine periodic coefficient, modes ordered by j1+j2")


def c3(seed: int = 1) -> Workload:
    """2-D 127x127 interior, lognormal-type coefficient, d=20, Gamma=[-32,32]^20, s=1000."""
    return Workload(
        "c3_2d_n127_d20_lognormal",
        Problem(kind=PDE_2D, n=127, d=20, coef_model=COEF_LOGNORMAL_SIN, coef_scale=0.5, coef_decay=2.0),
        Params(N=32, s=1000, s_local=1000, delta=1e-10, delta_is_relative=True, r=2, seed=seed,
               precision=PRECISION_MIXED),
        "a = exp(sum_{j<=20} 0.5 j^-2 phi_j(x) sin(2 pi y_j))")


def small_2d(n: int = 15, d: int = 4, seed: int = 1, N: int = 8, s: int = 40, r: int = 1) -> Workload:
    """A 2-D instance small enough for the banded-Cholesky oracle to finish in seconds."""
    return Workload(
        f"small_2d_n{n}_d{d}",
        Problem(kind=PDE_2D, n=n, d=d),
        Params(N=N, s=s, s_local=s, delta=1e-10, delta_is_relative=True, r=r, seed=seed))


def trigpoly(G: int, d: int, N: int, seed: int, base_terms: int = 6, node_terms: int = 2,
             max_active: int = 3, kmax: int = 4, mag_lo: float = 1e-6, mag_hi: float = 1.0) -> Problem:
    """Seeded real trigonometric polynomials p^(g), g=1..G (the black box of Theorem 1.1).

    Each p^(g) is real: its support is closed under k -> -k and its coefficients are
    Hermitian (c_{-k} = conj(c_k)).  The supports overlap: a common base set plus a few
    per-node frequencies.  Frequencies have at most `max_active` nonzero components,
    each of size <= min(kmax, N); magnitudes are log-uniform in [mag_lo, mag_hi].
    """
    rng = np.random.default_rng(seed)
    kmax = min(kmax, N)

    def draw_freq():
        k = np.zeros(d, dtype=np.int64)
        na = int(rng.integers(1, max_active + 1))
        dims = rng.choice(d, size=min(na, d), replace=False)
        for j in dims:
            v = 0
            while v == 0:
                v = int(rng.integers(-kmax, kmax + 1))
            k[j] = v
        return k

    def draw_coef():
        mag = math.exp(rng.uniform(math.log(mag_lo), math.log(mag_hi)))
        ph = rng.uniform(0.0, 2.0 * math.pi)
        return mag * complex(math.cos(ph), math.sin(ph))

    base = []
    seen = set()
    while len(base) < base_terms:
        k = draw_freq()
        key = tuple(k)
        if key in seen or tuple(-k) in seen:
            continue
        seen.add(key)
        base.append(k)
    per_node = []
    width = 1 + 2 * (base_terms + node_terms)
    freqs = np.zeros((G, width, d), dtype=np.int8)
    coefs = np.zeros((G, width), dtype=np.complex128)
    for g in range(G):
        terms = {tuple([0] * d): complex(rng.uniform(0.5, 1.0), 0.0)}
        for k in base:
            c = draw_coef()
            terms[tuple(k)] = c
            terms[tuple(-k)] = c.conjugate()
        extra = 0
        while extra < node_terms:
            k = draw_freq()
            if tuple(k) in terms or tuple(-k) in terms:
                continue
            c = draw_coef()
            terms[tuple(k)] = c
            terms[tuple(-k)] = c.conjugate()
            extra += 1
        for slot, (k, c) in enumerate(sorted(terms.items())):
            freqs[g, slot] = np.array(k, dtype=np.int8)
            coefs[g, slot] = c
        per_node.append(len(terms))
    return Problem(kind=TRIGPOLY, n=0, d=d, tp_freqs=freqs, tp_coefs=coefs)


def with_precision(w: Workload, precision: int) -> Workload:
    return replace(w, params=replace(w.params, precision=precision))


def trigpoly_grid(G: int, d: int, K: int, seed: int, mag_lo: float = 1e-3) -> Problem:
    """Real trigonometric polynomials whose support is the full grid [-K,K]^d (every node
    shares it), with Hermitian log-uniform coefficients: a dense test black box whose
    candidate sets are large enough to need the two-pass lattice FFT."""
    rng = np.random.default_rng(seed)
    axes = [np.arange(-K, K + 1)] * d
    grid = np.stack(np.meshgrid(*axes, indexing="ij"), axis=-1).reshape(-1, d)
    T = grid.shape[0]
    freqs = np.broadcast_to(grid.astype(np.int8), (G, T, d)).copy()
    coefs = np.zeros((G, T), dtype=np.complex128)
    index = {tuple(k): n for n, k in enumerate(grid.tolist())}
    for g in range(G):
        for n, k in enumerate(grid.tolist()):
            m = index[tuple(-v for v in k)]
            if m < n:
                coefs[g, n] = np.conj(coefs[g, m])
                continue
            mag = math.exp(rng.uniform(math.log(mag_lo), 0.0))
            ph = 0.0 if m == n else rng.uniform(0.0, 2.0 * math.pi)
            coefs[g, n] = mag * complex(math.cos(ph), math.sin(ph))
    return Problem(kind=TRIGPOLY, n=0, d=d, tp_freqs=freqs, tp_coefs=coefs)


def test_points(n: int, d: int, seed: int) -> np.ndarray:
    """n test parameters y^(j) drawn uniformly from the torus [0,1)^d (the distribution of the
    periodic model's parameters; Section 4 uses such random test points): float64 [n, d]."""
    return np.random.default_rng(np.random.SeedSequence([seed, 7, d])).random((n, d))


def parameter_points(prob: "Problem", n: int, seed: int) -> np.ndarray:
    """n test parameters drawn from the model's own distribution (Section 4): uniform on the
    torus (periodic model), uniform on [alpha, beta] (affine), standard normal (lognormal)."""
    rng = np.random.default_rng(np.random.SeedSequence([seed, 11, prob.d, prob.theta_map]))
    if prob.theta_map == MAP_TENT:
        return prob.map_alpha + (prob.map_beta - prob.map_alpha) * rng.random((n, prob.d))
    if prob.theta_map == MAP_NORMAL:
        return rng.standard_normal((n, prob.d))
    return rng.random((n, prob.d))


def with_map(w: "Workload", theta_map: int, alpha: float = -1.0, beta: float = 1.0, shift: float = 0.0) -> "Workload":
    """The same workload with another parameter map (Sec. 3.2)."""
    p = replace(w.problem, theta_map=theta_map, map_alpha=alpha, map_beta=beta, map_shift=shift)
    return replace(w, problem=p)


def batch_instances(count: int = 64, seed: int = 42, N: int = 16):
    """Independent instances shaped like the batching configuration: d ~ U{5..30}, meshes
    n ~ U{31..127} per side (2-D), s ~ U{100..2000}, affine or lognormal-type coefficient with
    probability 1/2 each; the mixed precision mode (the only one for n > 63).  Returns
    [(Workload, increments)], three increments each."""
    rng = np.random.default_rng(np.random.SeedSequence([seed, 4]))
    out = []
    for k in range(count):
        d = int(rng.integers(5, 31))
        n = int(rng.integers(31, 128))
        s = int(rng.integers(100, 2001))
        logn = bool(rng.integers(0, 2))
        prob = Problem(kind=PDE_2D, n=n, d=d, coef_model=COEF_LOGNORMAL_SIN if logn else COEF_AFFINE_SIN,
                       coef_scale=0.5 if logn else 0.9 * 6.0 / math.pi ** 2)
        par = Params(N=N, s=s, s_local=s, delta=1e-10, delta_is_relative=True, r=2, seed=seed * 1000 + k,
                     precision=PRECISION_MIXED)
        out.append((Workload(f"batch_{k}_n{n}_d{d}", prob, par), 3))
    return out


def serving_requests(count: int, rate: float = 200.0, seed: int = 7):
    """A seeded Poisson stream shaped like the serving configuration: half 128x128-mesh
    lognormal instances (d = 20, s = 1000, two increments), half 1-D instances with 255 nodes
    (d ~ U{4..20}, all d increments).  Returns [(arrival_s, Workload, increments, reserve_bytes)]."""
    rng = np.random.default_rng(np.random.SeedSequence([seed, 5]))
    t = 0.0
    out = []
    for k in range(count):
        t += float(rng.exponential(1.0 / rate))
        if rng.random() < 0.5:
            w = c3(seed * 10000 + k)
            out.append((t, w, 2, 2 << 30))
        else:
            d = int(rng.integers(4, 21))
            prob = Problem(kind=PDE_1D, n=255, d=d)
            par = Params(N=16, s=50, s_local=50, delta=1e-12, delta_is_relative=True, r=1, seed=seed * 10000 + k,
                         precision=PRECISION_MIXED)
            out.append((t, Workload(f"serve_1d_{k}_d{d}", prob, par), d, 64 << 20))
    return out
