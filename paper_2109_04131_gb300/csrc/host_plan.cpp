// Host planner: counter-based draws, admissible lattice sizes, candidate sets and the
// reconstructing rank-1 lattice search (Algorithm 1, step 2; Appendix A).
//
// The paper leaves the construction of the generating vector to the cited works and
// uses prime sizes (proof of Lemma 3.1).  This library reads the step as follows (the
// CPU oracle implements the same rule independently, so (z, M) are bit-exact):
//   - admissible sizes are 7-smooth (radix 2/3/5/7 FFT passes);
//   - the first size is the smallest admissible M >= |J|, the next one the smallest
//     admissible M' >= ceil(1.05 M) = floor((105 M + 99) / 100);
//   - for the sharded form over P ranks (strided lattice partition) admissible sizes are
//     also multiples of P (P = 1: every 7-smooth size);
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
#include <unistd.h>

#include <algorithm>
#include <atomic>
#include <condition_variable>
#include <functional>
#include <mutex>
#include <thread>
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

int64_t next_admissible_multiple(int64_t x, int64_t divisor) {
    if (divisor <= 1) return next_admissible(x);
    int64_t k = ((x < 1 ? 1 : x) + divisor - 1) / divisor;
    while (!is_smooth7(k * divisor)) ++k;
    return k * divisor;
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

// Step 3 with multiple rank-1 lattices (Algorithm 1, step 3; Appendix A: the lattice sizes of the
// bound M <= ceil(2 ln(2|I|)) 4 (|I| - 1), i.e. sizes from 2 (|I| - 1) on).  Each lattice is kept
// only as long as some k of I is not yet alone at its index in an earlier one.
bool multiple_lattices(const int8_t* I, int64_t n, int d, uint64_t seed, int max_lattices, std::vector<int64_t>& z,
                       std::vector<int64_t>& M, std::vector<int>& first) {
    z.clear();
    M.clear();
    first.assign((size_t)std::max<int64_t>(n, 0), -1);
    if (n <= 0) return true;
    int64_t m = next_admissible(std::max<int64_t>(2 * (n - 1), 2));
    int64_t open = n;
    std::vector<int64_t> idx((size_t)n), sorted;
    for (int l = 1; l <= max_lattices && open > 0; ++l) {
        std::vector<int64_t> zl((size_t)d, 1);
        for (int j = 1; j <= d; ++j) {
            for (int a = 0; a < 64; ++a) {
                const uint64_t f[4] = {PHASE_MULTI_R1L, (uint64_t)l, (uint64_t)j, (uint64_t)a};
                const int64_t v = rng_uniform_int(1, m - 1, seed, f, 4);
                if (gcd64(v, m) == 1) {
                    zl[(size_t)(j - 1)] = v;
                    break;
                }
            }
        }
        for (int64_t k = 0; k < n; ++k) {
            int64_t acc = 0;
            for (int j = 0; j < d; ++j) acc += (int64_t)I[(size_t)(k * d + j)] * zl[(size_t)j];
            const int64_t r = acc % m;
            idx[(size_t)k] = r < 0 ? r + m : r;
        }
        sorted = idx;
        std::sort(sorted.begin(), sorted.end());
        for (int64_t k = 0; k < n; ++k) {
            if (first[(size_t)k] >= 0) continue;
            auto range = std::equal_range(sorted.begin(), sorted.end(), idx[(size_t)k]);
            if (range.second - range.first == 1) {
                first[(size_t)k] = l - 1;
                --open;
            }
        }
        z.insert(z.end(), zl.begin(), zl.end());
        M.push_back(m);
        m = next_admissible(m + 1);
    }
    return open == 0;
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
// The residue is formed with a floating-point quotient estimate: |k.z| < 2^45 (|k_j| <= 127,
// z_j < 2^31, t <= 64) is exact in a double, the estimate floor(k.z / M) is off by at most one,
// and one correction each way gives the exact residue (an integer division per candidate is
// the slowest step of the check otherwise).
static bool injective(const int8_t* J, int64_t n, int t, const int64_t* z, int64_t M,
                      std::vector<uint64_t>& bits) {
    const size_t words = (size_t)((M + 63) / 64);
    if (bits.size() < words) bits.resize(words);
    std::fill(bits.begin(), bits.begin() + words, 0ULL);
    const double inv = 1.0 / (double)M;
    for (int64_t a = 0; a < n; ++a) {
        int64_t acc = 0;
        for (int j = 0; j < t; ++j) acc += (int64_t)J[a * t + j] * z[j];
        int64_t m = acc - (int64_t)floor((double)acc * inv) * M;
        if (m < 0) m += M;
        if (m >= M) m -= M;
        uint64_t bit = 1ULL << (m & 63);
        uint64_t& w = bits[(size_t)(m >> 6)];
        if (w & bit) return false;
        w |= bit;
    }
    return true;
}

// true if two rows of J (n rows of t entries) are equal: rows folded into 64-bit keys (exact
// for t <= 8, a hash otherwise, with equal keys compared in full), sorted
static bool has_repeated_row(const int8_t* J, int64_t n, int t) {
    std::vector<std::pair<uint64_t, int64_t>> key((size_t)n);
    for (int64_t a = 0; a < n; ++a) {
        uint64_t k = 0;
        if (t <= 8) {
            for (int j = 0; j < t; ++j) k = (k << 8) | (uint8_t)J[a * t + j];
        } else {
            for (int j = 0; j < t; ++j) {
                k ^= (uint64_t)(uint8_t)J[a * t + j] + kGoldenGamma + (k << 6) + (k >> 2);
            }
        }
        key[(size_t)a] = {k, a};
    }
    std::sort(key.begin(), key.end());
    for (size_t a = 1; a < key.size(); ++a) {
        if (key[a].first != key[a - 1].first) continue;
        if (t <= 8) return true;
        // equal hashes: compare against every earlier row with the same key
        for (size_t b = a; b-- > 0 && key[b].first == key[a].first;)
            if (std::equal(J + key[b].second * t, J + (key[b].second + 1) * t, J + key[a].second * t)) return true;
    }
    return false;
}

// the generating vector of trial tr at size m
static void draw_z(int t, int64_t m, int tr, uint64_t seed, uint64_t phase, int64_t* z) {
    z[0] = 1;
    for (int j = 2; j <= t; ++j) {
        if (m > 1) {
            uint64_t f[5] = {phase, (uint64_t)t, (uint64_t)m, (uint64_t)tr, (uint64_t)j};
            z[j - 1] = rng_uniform_int(1, m - 1, seed, f, 5);
        } else {
            z[j - 1] = 0;
        }
    }
}

// A small persistent pool of host threads for the lattice search (thread creation costs more
// than a search step).  One job at a time: a search that finds the pool busy (another plan is
// searching concurrently) runs alone, so many instances planned at once never oversubscribe
// the host.  The workers are detached and live as long as the process; a process forked from
// it has no workers, so the pool serves only the process that created it.
class SearchPool {
  public:
    static SearchPool& get() {
        static SearchPool* pool = new SearchPool();   // never destroyed (detached workers)
        return *pool;
    }
    int workers() const { return (int)nworkers_; }
    // runs f(0..count-1) on the workers and the caller; false (nothing run) if the pool is busy
    bool try_run(int count, const std::function<void(int)>& f) {
        if (nworkers_ == 0 || getpid() != owner_) return false;
        std::unique_lock<std::mutex> job(job_mu_, std::try_to_lock);
        if (!job.owns_lock()) return false;
        {
            std::lock_guard<std::mutex> lk(mu_);
            fn_ = &f;
            count_ = count;
            next_.store(0);
            active_ = nworkers_;
            ++gen_;
        }
        cv_.notify_all();
        for (int i; (i = next_.fetch_add(1)) < count;) f(i);
        std::unique_lock<std::mutex> lk(mu_);
        done_.wait(lk, [&] { return active_ == 0; });
        fn_ = nullptr;
        return true;
    }

  private:
    SearchPool() : owner_(getpid()) {
        const unsigned hc = std::thread::hardware_concurrency();
        nworkers_ = hc > 1 ? std::min(hc, 16u) - 1 : 0;
        for (unsigned w = 0; w < nworkers_; ++w) std::thread([this] { loop(); }).detach();
    }
    void loop() {
        uint64_t seen = 0;
        for (;;) {
            const std::function<void(int)>* f;
            int count;
            {
                std::unique_lock<std::mutex> lk(mu_);
                cv_.wait(lk, [&] { return gen_ != seen; });
                seen = gen_;
                f = fn_;
                count = count_;
            }
            for (int i; (i = next_.fetch_add(1)) < count;) (*f)(i);
            std::lock_guard<std::mutex> lk(mu_);
            if (--active_ == 0) done_.notify_one();
        }
    }
    const pid_t owner_;
    std::mutex job_mu_, mu_;
    std::condition_variable cv_, done_;
    const std::function<void(int)>* fn_ = nullptr;
    int count_ = 0;
    std::atomic<int> next_{0};
    unsigned nworkers_ = 0, active_ = 0;
    uint64_t gen_ = 0;
};

bool lattice_search(const int8_t* J, int64_t n, int t, uint64_t seed, int trials, int max_sizes,
                    std::vector<int64_t>& z, int64_t& M, uint64_t phase, int64_t divisor) {
    z.assign((size_t)t, 0);
    if (n == 0) {
        M = 0;
        return true;
    }
    // a repeated candidate can never be separated: the search gives up at once after its first
    // unsuccessful batch of sizes (any success already proves the rows distinct, so the sort of
    // the check is skipped in the common case)
    bool checked_repeats = false;
    // The trials check the rows in a fixed pseudo-random order (Fisher-Yates with SplitMix64
    // draws of a constant key).  Injectivity does not depend on the order, so (z, M) are those of
    // the candidate order; but in that (lexicographic) order the first rows share their leading
    // coordinates and rarely collide, and a failing trial met its first collision after about
    // 1100 of the 2-D workload's 4667 rows at t = 3, against about 130 in the mixed order.
    std::vector<int8_t> Jmix;
    if (n >= 64) {
        std::vector<int64_t> order((size_t)n);
        for (int64_t a = 0; a < n; ++a) order[(size_t)a] = a;
        for (int64_t a = n - 1; a > 0; --a) {
            const int64_t b = (int64_t)(splitmix_finalise((uint64_t)a + kGoldenGamma) % (uint64_t)(a + 1));
            std::swap(order[(size_t)a], order[(size_t)b]);
        }
        Jmix.resize((size_t)n * t);
        for (int64_t a = 0; a < n; ++a)
            std::copy(J + order[(size_t)a] * t, J + (order[(size_t)a] + 1) * t, Jmix.data() + (size_t)a * t);
        J = Jmix.data();
    }
    // The sizes in order; the result is the first size with a successful trial and its first
    // such trial.  For large candidate sets the next few sizes are examined at once in borrowed
    // host threads (each size's trials in order in one thread) and the smallest size index with
    // a success is kept: the same (z, M) as the sequential scan, in less wall time.
    // Large sets: the (size, trial) pairs of the next sizes, in order, are shared out among the
    // pool's threads; each pair past the best success found so far is skipped, and the smallest
    // successful pair is kept -- the same (z, M) as the sequential scan.
    SearchPool& pool = SearchPool::get();
    const int batch = n >= 1024 ? 16 : 1;
    std::vector<uint64_t> bits;
    int64_t m = next_admissible_multiple(n, divisor);
    int size = 0;
    while (size < max_sizes && m <= kMaxLatticeSize) {
        std::vector<int64_t> ms;
        for (int b = 0; b < batch && size + b < max_sizes && m <= kMaxLatticeSize; ++b) {
            ms.push_back(m);
            m = next_admissible_multiple((105 * m + 99) / 100, divisor);
        }
        const int items = (int)ms.size() * trials;
        std::atomic<int> best{items};
        const std::function<void(int)> job = [&](int i) {
            if (i >= best.load()) return;
            thread_local std::vector<uint64_t> tbits;
            std::vector<int64_t> zz((size_t)t);
            const int64_t mi = ms[(size_t)(i / trials)];
            draw_z(t, mi, i % trials, seed, phase, zz.data());
            if (injective(J, n, t, zz.data(), mi, tbits)) {
                int cur = best.load();
                while (i < cur && !best.compare_exchange_weak(cur, i)) {
                }
            }
        };
        if (batch == 1 || !pool.try_run(items, job)) {
            for (int i = 0; i < items && best.load() == items; ++i) job(i);   // alone, in order
        }
        if (best.load() < items) {
            const int i = best.load();
            M = ms[(size_t)(i / trials)];
            draw_z(t, M, i % trials, seed, phase, z.data());
            return true;
        }
        size += (int)ms.size();
        if (!checked_repeats) {
            checked_repeats = true;
            if (has_repeated_row(J, n, t)) return false;
        }
    }
    return false;
}

}  // namespace usfft
