"""Counter-based random draws (oracle side).

Algorithm 1 draws the non-lattice coordinates y'_j "uniformly at random" (steps 1/2a
and 2b) and the lattice search needs random generating vectors.  To make the CPU
oracle and the CUDA library draw identical numbers without sharing code, each side
implements the same published generator independently:

SplitMix64 (G. L. Steele, D. Lea, C. H. Flood, "Fast splittable pseudorandom number
generators", OOPSLA 2014): one step adds the golden gamma 0x9E3779B97F4A7C15 to the
state and returns the state passed through the 64-bit finaliser
  z ^= z >> 30; z *= 0xBF58476D1CE4E5B9; z ^= z >> 27; z *= 0x94D049BB133111EB; z ^= z >> 31.

Counter-based use: key(seed, f1, f2, ...) folds the fields one SplitMix64 step at a
time, h <- step(h xor f).  A uniform double in [0,1) is (h >> 11) * 2^-53; a uniform
integer in [lo, hi] is lo + (((h >> 32) * (hi - lo + 1)) >> 32).

Pins (tests/test_oracle_rng.py): the finaliser is a bijection (checked against its
inverse, written from the inverse xorshift/multiply steps), and the draws pass
moment and chi-square uniformity checks.
"""
MASK64 = (1 << 64) - 1
GOLDEN_GAMMA = 0x9E3779B97F4A7C15

# phases of the counter key
PHASE_1D_TAIL = 1      # tails y'_j, j != t, of the 1-D detections (steps 1 & 2a)
PHASE_TAIL = 2         # tails y'_{t+1..d} of the coupled step t (step 2b)
PHASE_LATTICE = 3      # generating-vector components of the lattice search (coupled steps)
PHASE_RECON = 4        # generating-vector components of the step-3 lattice
PHASE_RANDOM_R1L = 5   # generating vectors of the random rank-1 lattices (coupled steps)
PHASE_MULTI_R1L = 6    # generating vectors of the multiple rank-1 lattices of step 3


def mix64(z: int) -> int:
    z &= MASK64
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK64
    return z ^ (z >> 31)


def key(seed: int, *fields: int) -> int:
    h = seed & MASK64
    for f in fields:
        h = mix64(((h ^ (f & MASK64)) + GOLDEN_GAMMA) & MASK64)
    return h


def uniform(seed: int, *fields: int) -> float:
    return (key(seed, *fields) >> 11) * (2.0 ** -53)


def uniform_int(lo: int, hi: int, seed: int, *fields: int) -> int:
    span = hi - lo + 1
    assert 0 < span < (1 << 32)
    return lo + (((key(seed, *fields) >> 32) * span) >> 32)
