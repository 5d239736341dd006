"""The usFFT detection increments (oracle side), Algorithm 1 steps 1, 2a and 2.

Increment numbering follows the library: increment 1 runs the 1-D detections of
dimension 1 (r iterations) and sets I^(1..1) = I^(1); increment t >= 2 runs the 1-D
detections of dimension t and then the coupled step t.  All random draws are keyed
by (phase, t, i, j), so this order gives the same result as the paper's order
(all 1-D detections first).

1-D detection of dimension t, iteration i (steps 1 & 2a): tails y'_j (j != t) are
uniform(seed, PHASE_1D_TAIL, t, i, j); nodes y^(l) have y_t = l/K_t, l = 0..K_t-1,
K_t = 2N+1 (a lattice with z = 1, M = K_t on coordinate t); coefficients at
k_t = -N..N (m = k_t mod K_t); selection with s~ = s_local; union into I^(t).

Coupled step t, iteration i (steps 2b-2e): r~ = r, s~ = s_local for t < d and
r~ = 1, s~ = s for t = d; J_t from I^(1..t-1) x I^(t); lattice (z, M) from the search
rule of oracle.lattice; tails y'_j (j > t) are uniform(seed, PHASE_TAIL, t, i, j);
samples at the M lattice nodes; coefficients at m_k = k.z mod M; selection and union
of positions in J_t; I^(1..t) keeps J_t's order.

Sampling uses exact lattice integers: sin(2 pi y_j) = sin(2 pi n/M) with
n = i z_j mod M for lattice coordinates.

Step 3 (reconstruct): one reconstructing rank-1 lattice for I^(1..d) (the search rule
of oracle.lattice with draws keyed by PHASE_RECON; the paper uses multiple lattices
here, a single reconstructing lattice gives the same coefficients exactly for
polynomials supported in I), samples at its nodes, DFT at k.z mod M, no threshold.
"""
from dataclasses import dataclass, field

import numpy as np

from . import detect, dft, fe, lattice, periodization, rng

PDE_1D, PDE_2D, TRIGPOLY = 1, 2, 3


@dataclass
class NodeSet:
    """M nodes: coordinates `lat` (0-based) from the lattice (z, M), the rest fixed tails."""
    d: int
    lat: list
    z: np.ndarray
    M: int
    tails: dict       # coordinate (0-based) -> y'_j

    def lattice_ints(self) -> np.ndarray:
        """n_ij = i z_j mod M, shape [M, len(lat)]."""
        i = np.arange(self.M, dtype=np.int64)[:, None]
        return np.mod(i * self.z[None, :].astype(np.int64), self.M)


def sample(prob, nodes: NodeSet, mesh=None) -> np.ndarray:
    """Black-box samples U [M, G]: u(x_g, y_i) for every node y_i of the set."""
    n_int = nodes.lattice_ints()
    if prob.kind == TRIGPOLY:
        return _trigpoly_samples(prob, nodes, n_int)
    if mesh is None:
        mesh = fe.make_mesh(prob.kind, prob.n)
    U = np.zeros((nodes.M, mesh.G))
    theta = np.zeros(nodes.d)
    for j, yv in nodes.tails.items():
        theta[j] = periodization.theta_of_node(prob, yv)
    for i in range(nodes.M):
        for c, j in enumerate(nodes.lat):
            theta[j] = periodization.theta_of_node(prob, n_int[i, c] / nodes.M)
        U[i] = fe.solve(prob, mesh, theta)
    return U


def sample_rows(prob, nodes: NodeSet, rows, mesh=None) -> np.ndarray:
    """The PDE samples of the lattice nodes listed in `rows` only (a bounded subset of
    sample(); used to time the oracle on part of a large workload)."""
    if mesh is None:
        mesh = fe.make_mesh(prob.kind, prob.n)
    n_int = nodes.lattice_ints()
    U = np.zeros((len(rows), mesh.G))
    theta = np.zeros(nodes.d)
    for j, yv in nodes.tails.items():
        theta[j] = periodization.theta_of_node(prob, yv)
    for r, i in enumerate(rows):
        for c, j in enumerate(nodes.lat):
            theta[j] = periodization.theta_of_node(prob, n_int[i, c] / nodes.M)
        U[r] = fe.solve(prob, mesh, theta)
    return U


def _trigpoly_samples(prob, nodes: NodeSet, n_int: np.ndarray) -> np.ndarray:
    F = prob.tp_freqs.astype(np.int64)        # [G, T, d]
    Cf = prob.tp_coefs                        # [G, T]
    G, T, d = F.shape
    lat = nodes.lat
    tail_idx = sorted(nodes.tails)
    tail_y = np.array([nodes.tails[j] for j in tail_idx])
    U = np.zeros((nodes.M, G))
    for g in range(G):
        for tt in range(T):
            c = Cf[g, tt]
            if c == 0:
                continue
            h = F[g, tt]
            tail_phase = float(np.dot(h[tail_idx], tail_y)) if tail_idx else 0.0
            lat_int = np.mod(n_int @ h[lat], nodes.M) if lat else np.zeros(nodes.M, dtype=np.int64)
            ang = 2.0 * np.pi * (lat_int.astype(np.float64) / nodes.M + tail_phase)
            U[:, g] += (c * np.exp(1j * ang)).real
    return U


@dataclass
class Record:
    """What one detection iteration produced (for parity tests)."""
    t: int
    i: int
    coupled: bool
    z: np.ndarray
    M: int
    tails: dict
    m: np.ndarray           # DFT indices of the candidates
    U: np.ndarray = None    # samples [M, G]
    C: np.ndarray = None    # coefficients [G, |J|]
    selected: list = field(default_factory=list)   # per node: sorted indices


class OracleRun:
    def __init__(self, prob, params, keep=False, lattice_divisor=1):
        self.prob = prob
        self.p = params
        self.keep = keep
        self.divisor = lattice_divisor      # > 1: lattice sizes of the sharded form over that many ranks
        self.t = 0
        self.theta = None if params.delta_is_relative else params.delta
        self.A = None
        self.I1d = {}                               # t -> sorted list of k_t
        self.I_prefix = np.zeros((0, 0), dtype=np.int64)
        self.J = None
        self.z = None
        self.M = 0
        self.records = []
        self.samples_used = 0
        self.mesh = None if prob.kind == TRIGPOLY else fe.make_mesh(prob.kind, prob.n)

    # ---- Algorithm 1, steps 1 & 2a -------------------------------------------------
    def detect_1d(self, t: int):
        p = self.p
        K = 2 * p.N + 1
        ks = np.arange(-p.N, p.N + 1)
        m = np.mod(ks, K)
        found = set()
        for i in range(1, p.r + 1):
            tails = {j - 1: rng.uniform(p.seed, rng.PHASE_1D_TAIL, t, i, j)
                     for j in range(1, self.prob.d + 1) if j != t}
            nodes = NodeSet(self.prob.d, [t - 1], np.array([1]), K, tails)
            U = sample(self.prob, nodes, self.mesh)
            self.samples_used += K
            C = dft.coefficients(U, m, K)
            if self.theta is None:                  # relative delta: fix theta once
                self.A = float(np.max(np.abs(C[:, p.N])))
                self.theta = p.delta * self.A
            sel = [detect.select(C[g], self.theta, p.s_local) for g in range(C.shape[0])]
            for sg in sel:
                found.update(int(x) for x in sg)
            self.records.append(Record(t, i, False, np.array([1]), K, tails, m,
                                       U if self.keep else None, C if self.keep else None,
                                       sel if self.keep else []))
        self.I1d[t] = [int(ks[x]) for x in sorted(found)]

    # ---- Algorithm 1, step 2 ---------------------------------------------------------
    def coupled(self, t: int):
        p = self.p
        d = self.prob.d
        r_t = p.r if t < d else 1
        s_t = p.s_local if t < d else p.s
        J = lattice.candidate_set(self.I_prefix, np.array(self.I1d[t], dtype=np.int64), p.N)
        if getattr(p, "rr_lattices", 0) > 0:
            return self._coupled_random(t, J, r_t, s_t)
        z, M = lattice.search(J, t, p.seed, p.max_lattice_trials, getattr(p, "max_lattice_sizes", 400),
                              divisor=self.divisor)
        self.J, self.z, self.M = J, z, M
        found = set()
        if len(J) > 0:
            m = lattice.lattice_indices(J, z, M)
            for i in range(1, r_t + 1):
                tails = {j - 1: rng.uniform(p.seed, rng.PHASE_TAIL, t, i, j) for j in range(t + 1, d + 1)}
                nodes = NodeSet(d, list(range(t)), z, M, tails)
                U = sample(self.prob, nodes, self.mesh)
                self.samples_used += M
                C = dft.coefficients(U, m, M)
                sel = [detect.select(C[g], self.theta, s_t) for g in range(C.shape[0])]
                for sg in sel:
                    found.update(int(x) for x in sg)
                self.records.append(Record(t, i, True, z, M, tails, m,
                                           U if self.keep else None, C if self.keep else None,
                                           sel if self.keep else []))
        idx = sorted(found)
        self.I_prefix = J[idx] if len(idx) else np.zeros((0, t), dtype=np.int64)

    def _coupled_random(self, t: int, J: np.ndarray, r_t: int, s_t: int):
        """Coupled step t with random rank-1 lattices in the role of Algorithm A: per detection
        iteration the same t-variate projection (fixed tails) is sampled on L random lattices
        (oracle.lattice.random_lattices) and c_k is read from the lattice DFTs at k.z_l mod M_l:
        from the first lattice in which no other candidate of J_t shares k's index (there the
        value is what a reconstructing lattice gives), else as the median over the L lattices,
        separately for the real and the imaginary part (a lattice where k shares its index with
        a large coefficient gives an outlier; the median discards it while most lattices are
        free of such collisions)."""
        p = self.p
        d = self.prob.d
        L = p.rr_lattices
        assert L % 2 == 1, "an odd number of lattices (the median is one of the estimates)"
        self.J = J
        found = set()
        n_prev, n_t = len(self.I_prefix), len(self.I1d[t])
        for i in range(1, r_t + 1):
            if len(J) == 0:
                break
            tails = {j - 1: rng.uniform(p.seed, rng.PHASE_TAIL, t, i, j) for j in range(t + 1, d + 1)}
            lats = lattice.random_lattices(t, i, n_prev, n_t, s_t, L, p.rr_size_factor, p.seed)
            est, ms = [], []
            for z_l, M_l in lats:
                U = sample(self.prob, NodeSet(d, list(range(t)), z_l, M_l, tails), self.mesh)
                self.samples_used += M_l
                m_l = lattice.lattice_indices(J, z_l, M_l)
                est.append(dft.coefficients(U, m_l, M_l))
                ms.append(m_l)
            E = np.stack(est)                                  # [L, G, |J|]
            C = np.median(E.real, axis=0) + 1j * np.median(E.imag, axis=0)
            for k in range(len(J)):
                for l, m_l in enumerate(ms):
                    if np.count_nonzero(m_l == m_l[k]) == 1:     # k alone at its index
                        C[:, k] = E[l, :, k]
                        break
            sel = [detect.select(C[g], self.theta, s_t) for g in range(C.shape[0])]
            for sg in sel:
                found.update(int(x) for x in sg)
            self.z = [z for z, _ in lats]
            self.M = [M for _, M in lats]
            self.records.append(Record(t, i, True, self.z, self.M, tails, ms, None,
                                       C if self.keep else None, sel if self.keep else []))
        idx = sorted(found)
        self.I_prefix = J[idx] if len(idx) else np.zeros((0, t), dtype=np.int64)

    # ---- Algorithm 1, step 3 ----------------------------------------------------------
    def reconstruct(self):
        """Coefficients of every node on I = I^(1..d) from one reconstructing rank-1 lattice
        (draws keyed by PHASE_RECON), no tails, no threshold: (I, z, M, C [G, |I|])."""
        assert self.t == self.prob.d
        I = self.I_prefix
        d = self.prob.d
        z, M = lattice.search(I, d, self.p.seed, self.p.max_lattice_trials, getattr(self.p, "max_lattice_sizes", 400),
                              phase=rng.PHASE_RECON)
        if len(I) == 0:
            return I, z, M, np.zeros((0, 0), dtype=np.complex128)
        m = lattice.lattice_indices(I, z, M)
        nodes = NodeSet(d, list(range(d)), z, M, {})
        U = sample(self.prob, nodes, self.mesh)
        self.samples_used += M
        return I, z, M, dft.coefficients(U, m, M)

    def reconstruct_multiple(self):
        """Step 3 on multiple rank-1 lattices (oracle.lattice.multiple_lattices): the samples of
        every lattice (all d coordinates on the lattice, no tails), their DFTs read at k.z_l mod
        M_l, and c_k from the first lattice in which k is alone at its index, where the lattice
        DFT is exactly c_k for a trigonometric polynomial supported in I (the aliasing formula of
        Appendix A).  Returns (I, [(z_l, M_l)], C [G, |I|])."""
        assert self.t == self.prob.d
        I = self.I_prefix
        d = self.prob.d
        lats, first = lattice.multiple_lattices(I, d, self.p.seed)
        if len(I) == 0:
            return I, lats, np.zeros((0, 0), dtype=np.complex128)
        assert first is not None, "some frequency of I shares its index in every lattice"
        C = None
        for l, (z_l, M_l) in enumerate(lats):
            mine = np.nonzero(first == l)[0]
            U = sample(self.prob, NodeSet(d, list(range(d)), z_l, M_l, {}), self.mesh)
            self.samples_used += M_l
            c_l = dft.coefficients(U, lattice.lattice_indices(I[mine], z_l, M_l), M_l)
            if C is None:
                C = np.zeros((c_l.shape[0], len(I)), dtype=np.complex128)
            C[:, mine] = c_l
        return I, lats, C

    def resume(self, t: int, I_prefix: np.ndarray, theta: float):
        """Continue from the state after increment t: I^(1..t) and theta (checkpoint)."""
        self.t = t
        self.I_prefix = np.array(I_prefix, dtype=np.int64).reshape(-1, t) if t > 0 else np.zeros((0, 0), np.int64)
        if t > 0:
            self.theta = theta
        self.I1d = {}

    def increment(self):
        self.t += 1
        t = self.t
        assert t <= self.prob.d
        self.detect_1d(t)
        if t == 1:
            self.I_prefix = np.array(self.I1d[1], dtype=np.int64)[:, None]
        else:
            self.coupled(t)
        return self.I_prefix
