// Host planner: counter-based draws, admissible lattice sizes, candidate sets and the
// reconstructing rank-1 lattice search (Algorithm 1, step 2; Appendix A).
//
// The paper leaves the construction of the generating vector to the cited works and
// uses prime sizes (proof of Lemma 3.1).  This library reads the step as follows (the
// CPU oracle implements the same rule independently, so (z, M) are bit-exact):
//   - admissible sizes are 7-smooth (radix 2/3/5/7 FFT passes);
//   - the first size is the smallest admissible M >= |J|, the next one the smallest
//     admissible M' >= ceil(1.05 M) = floor((105 M + 99) / 100);
//   - at each size trials tr = 0..T-1 set z_1 = 1 and draw z_j in [1, M-1], j = 2..t,
//     from key(seed, PHASE_LATTICE, t, M, tr, j); the first z for which
//     k -> k.z mod M is injective on J is taken;
//   - the search gives up on a repeated candidate, after 400 sizes or beyond
//     M = 4096^2 (the largest two-pass FFT).
// Step 3 (the final coefficients on I) uses the same rule with the draws keyed by
// PHASE_RECON instead of PHASE_LATTICE.  The random rank-1 lattices of the alternative
// detection (random_lattices) follow their own rule, stated at its declaration.
#include <math.h>
#include <stdint.h>

#include <algorithm>
#include <vector>

#include "usfft_internal.h"

namespace usfft {

static const uint64_t kGoldenGamma = 0x9E3779B97F4A7C15ULL;
// largest lattice the FFT passes handle (two on-chip passes of <= 4096)
static const int64_t kMaxLatticeSize = 4096LL * 4096LL;

static inline uint64_t splitmix_finalise(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

uint64_t rng_key(uint64_t seed, const uint64_t* fields, int nfields) {
    uint64_t h = seed;
    for (int i = 0; i < nfields; ++i) h = splitmix_finalise((h ^ fields[i]) + kGoldenGamma);
    return h;
}

double rng_uniform(uint64_t seed, const uint64_t* fields, int nfields) {
    return (double)(rng_key(seed, fields, nfields) >> 11) * (1.0 / 9007199254740992.0);
}

int64_t rng_uniform_int(int64_t lo, int64_t hi, uint64_t seed, const uint64_t* fields, int nfields) {
    uint64_t span = (uint64_t)(hi - lo + 1);
    uint64_t top = rng_key(seed, fields, nfields) >> 32;
    return lo + (int64_t)((top * span) >> 32);
}

bool is_smooth7(int64_t m) {
    if (m < 1) return false;
    const int64_t primes[4] = {2, 3, 5, 7};
    for (int64_t p : primes)
        while (m % p == 0) m /= p;
    return m == 1;
}

int64_t next_admissible(int64_t x) {
    int64_t m = x < 1 ? 1 : x;
    while (!is_smooth7(m)) ++m;
    return m;
}

static int64_t gcd64(int64_t a, int64_t b) {
    while (b) {
        const int64_t r = a % b;
        a = b;
        b = r;
    }
    return a;
}

void random_lattices(int t, int i, int64_t n_prev, int64_t n_t, int64_t s_t, int L, double factor, uint64_t seed,
                     std::vector<int64_t>& z, std::vector<int64_t>& M) {
    z.assign((size_t)L * t, 1);
    M.assign((size_t)L, 0);
    int64_t big = std::max<int64_t>(std::max<int64_t>(n_prev, n_t), std::max<int64_t>(s_t, 1));
    int64_t base = (int64_t)ceil(factor * (double)big);
    if (base < 2) base = 2;
    int64_t m = next_admissible(base);
    for (int l = 1; l <= L; ++l) {
        M[(size_t)(l - 1)] = m;
        for (int j = 1; j <= t; ++j) {
            for (int a = 0; a < 64; ++a) {
                const uint64_t f[6] = {PHASE_RANDOM_R1L, (uint64_t)t, (uint64_t)i, (uint64_t)l, (uint64_t)j, (uint64_t)a};
                const int64_t v = rng_uniform_int(1, m - 1, seed, f, 6);
                if (gcd64(v, m) == 1) {
                    z[(size_t)((l - 1) * t + (j - 1))] = v;
                    break;
                }
            }
        }
        m = next_admissible(m + 1);
    }
}

void candidate_set(const int8_t* I_prev, int64_t n_prev, int t_prev, const std::vector<int>& I_t, int N,
                   std::vector<int8_t>& J, int64_t& nJ) {
    const int t = t_prev + 1;
    J.clear();
    J.reserve((size_t)(n_prev * (int64_t)I_t.size() * t));
    nJ = 0;
    for (int64_t a = 0; a < n_prev; ++a) {
        bool inside = true;
        for (int j = 0; j < t_prev; ++j) {
            int v = I_prev[a * t_prev + j];
            if (v < -N || v > N) inside = false;
        }
        for (size_t b = 0; b < I_t.size(); ++b) {
            int kt = I_t[b];
            if (!inside || kt < -N || kt > N) continue;
            for (int j = 0; j < t_prev; ++j) J.push_back(I_prev[a * t_prev + j]);
            J.push_back((int8_t)kt);
            ++nJ;
        }
    }
}

// Injectivity of k -> k.z mod M on J with an M-bit bitmap; early exit on the first collision.
static bool injective(const int8_t* J, int64_t n, int t, const int64_t* z, int64_t M,
                      std::vector<uint64_t>& bits) {
    const size_t words = (size_t)((M + 63) / 64);
    if (bits.size() < words) bits.resize(words);
    std::fill(bits.begin(), bits.begin() + words, 0ULL);
    for (int64_t a = 0; a < n; ++a) {
        int64_t acc = 0;
        for (int j = 0; j < t; ++j) acc += (int64_t)J[a * t + j] * z[j];
        int64_t m = acc % M;
        if (m < 0) m += M;
        uint64_t bit = 1ULL << (m & 63);
        uint64_t& w = bits[(size_t)(m >> 6)];
        if (w & bit) return false;
        w |= bit;
    }
    return true;
}

bool lattice_search(const int8_t* J, int64_t n, int t, uint64_t seed, int trials, int max_sizes,
                    std::vector<int64_t>& z, int64_t& M, uint64_t phase) {
    z.assign((size_t)t, 0);
    if (n == 0) {
        M = 0;
        return true;
    }
    // a repeated candidate can never be separated: fail at once
    {
        std::vector<int8_t> rows(J, J + n * t);
        std::vector<int64_t> idx((size_t)n);
        for (int64_t a = 0; a < n; ++a) idx[(size_t)a] = a;
        std::sort(idx.begin(), idx.end(), [&](int64_t x, int64_t y) {
            return std::lexicographical_compare(rows.begin() + x * t, rows.begin() + (x + 1) * t,
                                                rows.begin() + y * t, rows.begin() + (y + 1) * t);
        });
        for (int64_t a = 1; a < n; ++a)
            if (std::equal(rows.begin() + idx[(size_t)a - 1] * t, rows.begin() + (idx[(size_t)a - 1] + 1) * t,
                           rows.begin() + idx[(size_t)a] * t))
                return false;
    }
    std::vector<uint64_t> bits;
    int64_t m = next_admissible(n);
    for (int size = 0; size < max_sizes && m <= kMaxLatticeSize; ++size) {
        for (int tr = 0; tr < trials; ++tr) {
            z[0] = 1;
            for (int j = 2; j <= t; ++j) {
                if (m > 1) {
                    uint64_t f[5] = {phase, (uint64_t)t, (uint64_t)m, (uint64_t)tr, (uint64_t)j};
                    z[(size_t)(j - 1)] = rng_uniform_int(1, m - 1, seed, f, 5);
                } else {
                    z[(size_t)(j - 1)] = 0;
                }
            }
            if (injective(J, n, t, z.data(), m, bits)) {
                M = m;
                return true;
            }
        }
        m = next_admissible((105 * m + 99) / 100);
    }
    return false;
}

}  // namespace usfft
