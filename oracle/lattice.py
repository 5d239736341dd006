"""Candidate sets, rank-1 lattices and the reconstructing-lattice search (oracle side).

- Candidate set of the coupled step t (Algorithm 1, step 2):
    J_t = (I^(1..t-1) x I^(t)) intersected with P_(1..t)(Gamma),
  kept as an ordered list: lexicographic in (position in I^(1..t-1), position in
  I^(t)).  For the cube Gamma = [-N,N]^d the intersection keeps every element.
- Rank-1 lattice Lambda(z, M) = { (i/M) z mod 1 : i = 0..M-1 } (Appendix A); its
  node i has coordinates y_ij = (i z_j mod M)/M (Eq. (3.4)), kept here as the exact
  integers n_ij = i z_j mod M.
- A lattice reconstructs J when k -> k.z mod M is injective on J; then the length-M
  DFT of the lattice samples returns the projected coefficient of every k in J at
  index k.z mod M (Appendix A; single rank-1 lattice approach).

The paper gives no construction of the generating vector for this step (it cites
other work) and states that its lattice sizes are prime (proof of Lemma 3.1).  The
reading used here (the same on both sides, so (z, M) are bit-exact):

- admissible sizes are the 7-smooth integers (radix-2/3/5/7 FFTs); the first size
  tried is the smallest admissible M >= |J|, every next one the smallest admissible
  M' >= ceil(1.05 M) = floor((105 M + 99)/100) (integer arithmetic);
- at every size, trials tr = 0..T-1 draw z_1 = 1 and z_j = uniform integer in
  [1, M-1] (j = 2..t) from key(seed, PHASE_LATTICE, t, M, tr, j); the first z that
  is injective on J is accepted;
- the search gives up on a repeated candidate, after 400 sizes, or beyond
  M = 4096^2 (a limit of the library's FFT, adopted here so both sides agree);
- for the sharded form over P ranks (the lattice nodes split by residue i mod P, which
  needs P | M) the admissible sizes are the 7-smooth multiples of P; P = 1 is the rule
  above.

Pins (tests/test_oracle_lattice.py): on tiny sets, the injectivity test agrees with
the definition through the lattice Fourier matrix (its columns for J are orthonormal
exactly when the lattice reconstructs J), enumerated over every z.
"""
import math

import numpy as np

from . import rng

MAX_LATTICE_SIZE = 4096 * 4096


def candidate_set(I_prev: np.ndarray, I_t: np.ndarray, N: int) -> np.ndarray:
    """J_t as int64 [|I_prev| * |I_t|, t]; I_prev is [n, t-1], I_t is a 1-D list of k_t."""
    rows = []
    for kp in I_prev:
        for kt in I_t:
            k = np.concatenate([kp, [kt]])
            if np.all(np.abs(k) <= N):           # P_(1..t)(Gamma) for Gamma = [-N,N]^d
                rows.append(k)
    t = I_prev.shape[1] + 1
    if not rows:
        return np.zeros((0, t), dtype=np.int64)
    return np.array(rows, dtype=np.int64)


def is_smooth7(m: int) -> bool:
    if m < 1:
        return False
    for p in (2, 3, 5, 7):
        while m % p == 0:
            m //= p
    return m == 1


def next_admissible(x: int) -> int:
    m = max(int(x), 1)
    while not is_smooth7(m):
        m += 1
    return m


def lattice_indices(J: np.ndarray, z: np.ndarray, M: int) -> np.ndarray:
    """m_k = (k . z) mod M in [0, M) for every k in J (exact integer arithmetic)."""
    return np.mod(J.astype(np.int64) @ z.astype(np.int64), M)


def is_reconstructing(J: np.ndarray, z: np.ndarray, M: int) -> bool:
    m = lattice_indices(J, z, M)
    return len(np.unique(m)) == len(m)


def next_admissible_multiple(x: int, divisor: int) -> int:
    """Smallest admissible size >= x that is a multiple of divisor (itself 7-smooth)."""
    k = max(1, -(-max(x, 1) // divisor))
    while not is_smooth7(k * divisor):
        k += 1
    return k * divisor


def search(J: np.ndarray, t: int, seed: int, trials: int = 64, max_sizes: int = 400, phase: int = rng.PHASE_LATTICE,
           divisor: int = 1):
    """(z, M) of the first reconstructing lattice under the rule in the module header; the
    draws are keyed by `phase` (PHASE_LATTICE in the coupled steps, PHASE_RECON in step 3).
    With divisor P > 1 only sizes that are multiples of P are admissible (the strided split of
    the lattice nodes over P ranks needs P | M); P = 1 is the plain rule."""
    if len(J) == 0:
        return np.zeros(t, dtype=np.int64), 0
    if len(np.unique(J, axis=0)) < len(J):
        raise RuntimeError("repeated candidate: no lattice can separate it")
    M = next_admissible_multiple(len(J), divisor)
    for _ in range(max_sizes):
        if M > MAX_LATTICE_SIZE:
            break
        for tr in range(trials):
            z = np.ones(t, dtype=np.int64)
            for j in range(2, t + 1):
                z[j - 1] = rng.uniform_int(1, M - 1, seed, phase, t, M, tr, j) if M > 1 else 0
            if is_reconstructing(J, z, M):
                return z, M
        M = next_admissible_multiple((105 * M + 99) // 100, divisor)
    raise RuntimeError("no reconstructing lattice found")


def random_lattices(t: int, i: int, n_prev: int, n_t: int, s_t: int, L: int, factor: float, seed: int):
    """The L random rank-1 lattices of detection iteration i of the coupled step t (the random
    R1L approach in the role of Algorithm A; sizes from the bound max(s, N_Gamma) of the proof
    of Theorem 1.1, the rule itself a reading): M_1 is the smallest admissible size >=
    ceil(factor * max(|I^(1..t-1)|, |I^(t)|, s~)), M_(l+1) the smallest admissible size > M_l;
    every component of z_l is a unit mod M_l (gcd 1, so that each coordinate alone takes all M_l
    values): the first of the draws uniform in [1, M_l - 1] keyed (seed, PHASE_RANDOM_R1L, t, i,
    l, j, a), a = 0, 1, ..., 63, that is coprime to M_l, else 1.  Returns [(z_l, M_l)], l = 1..L."""
    base = max(int(math.ceil(factor * max(n_prev, n_t, s_t, 1))), 2)
    M = next_admissible(base)
    out = []
    for l in range(1, L + 1):
        z = np.ones(t, dtype=np.int64)
        for j in range(1, t + 1):
            for a in range(64):
                v = rng.uniform_int(1, M - 1, seed, rng.PHASE_RANDOM_R1L, t, i, l, j, a)
                if math.gcd(v, M) == 1:
                    z[j - 1] = v
                    break
        out.append((z, M))
        M = next_admissible(M + 1)
    return out


def multiple_lattices(I: np.ndarray, d: int, seed: int, max_lattices: int = 64):
    """The multiple rank-1 lattices of step 3 (Algorithm 1, step 3 with the multiple R1L approach,
    Appendix A; the rule is a reading): sizes start at the smallest admissible size >=
    max(2 (|I| - 1), 2), the size of the bound ceil(2 ln(2|I|)) 4 (|I| - 1) on the total, and each next
    size is the smallest admissible one above the last; each component of z_l is a unit mod M_l, the
    first draw uniform in [1, M_l - 1] keyed (seed, PHASE_MULTI_R1L, l, j, a), a = 0, 1, ..., 63,
    coprime to M_l, else 1.  Lattices are drawn until every k in I is alone at its index k.z_l mod
    M_l (no other frequency of I maps there) in at least one of them.
    Returns ([(z_l, M_l)], first) with first[k] the first such lattice (0-based), or None in place
    of first if max_lattices lattices leave some k without one."""
    n = len(I)
    first = np.full(n, -1, dtype=np.int64)
    out = []
    if n == 0:
        return out, first
    M = next_admissible(max(2 * (n - 1), 2))
    for l in range(1, max_lattices + 1):
        z = np.ones(d, dtype=np.int64)
        for j in range(1, d + 1):
            for a in range(64):
                v = rng.uniform_int(1, M - 1, seed, rng.PHASE_MULTI_R1L, l, j, a)
                if math.gcd(v, M) == 1:
                    z[j - 1] = v
                    break
        out.append((z, M))
        m = lattice_indices(I, z, M)
        values, counts = np.unique(m, return_counts=True)
        alone = np.isin(m, values[counts == 1])
        first[(first < 0) & alone] = l - 1
        if np.all(first >= 0):
            return out, first
        M = next_admissible(M + 1)
    return out, None

