// Internal declarations of the usFFT GB300 library (not part of the C ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "usfft.h"

#define USFFT_MAX_D 64

// ---------------------------------------------------------------------------------
// Host planner (host_plan.cpp)
// ---------------------------------------------------------------------------------
namespace usfft {

// Counter-based SplitMix64 draws (Steele, Lea, Flood 2014): key(seed, f1, f2, ...)
// folds one SplitMix64 step per field, h <- mix64((h ^ f) + golden gamma).
enum Phase : uint64_t { PHASE_1D_TAIL = 1, PHASE_TAIL = 2, PHASE_LATTICE = 3, PHASE_RECON = 4, PHASE_RANDOM_R1L = 5,
                        PHASE_MULTI_R1L = 6 };
uint64_t rng_key(uint64_t seed, const uint64_t* fields, int nfields);
double rng_uniform(uint64_t seed, const uint64_t* fields, int nfields);                 // [0,1)
int64_t rng_uniform_int(int64_t lo, int64_t hi, uint64_t seed, const uint64_t* fields, int nfields);

bool is_smooth7(int64_t m);
int64_t next_admissible(int64_t x);
// smallest 7-smooth multiple of divisor that is >= x (divisor itself 7-smooth)
int64_t next_admissible_multiple(int64_t x, int64_t divisor);

// Reconstructing rank-1 lattice search: J is [n][t] int8 row-major.  Returns false if
// none is found within max_sizes sizes; z receives t entries.  `phase` keys the draws
// (PHASE_LATTICE for the coupled steps, PHASE_RECON for step 3).
// divisor: admissible sizes are multiples of it (the sharded form over that many ranks).
bool lattice_search(const int8_t* J, int64_t n, int t, uint64_t seed, int trials, int max_sizes,
                    std::vector<int64_t>& z, int64_t& M, uint64_t phase = PHASE_LATTICE, int64_t divisor = 1);

// The L random rank-1 lattices of detection iteration i of the coupled step t (random R1L
// approach in the role of Algorithm A): M_1 = smallest admissible size >= ceil(factor *
// max(n_prev, n_t, s_t)) (at least 2), M_(l+1) = smallest admissible size > M_l; z_l has t
// components, each the first draw in [1, M_l - 1] keyed (seed, PHASE_RANDOM_R1L, t, i, l, j, a),
// a = 0..63, that is coprime to M_l (else 1).  z receives L*t entries, M receives L sizes.
void random_lattices(int t, int i, int64_t n_prev, int64_t n_t, int64_t s_t, int L, double factor, uint64_t seed,
                     std::vector<int64_t>& z, std::vector<int64_t>& M);

// The multiple rank-1 lattices of step 3 for the frequency set I ([n][d] int8 rows): lattice l =
// 1, 2, ... has size M_1 = the smallest admissible size >= max(2 (n - 1), 2), M_(l+1) = the smallest
// admissible size > M_l, and d components, each the first draw in [1, M_l - 1] keyed (seed,
// PHASE_MULTI_R1L, l, j, a), a = 0..63, that is coprime to M_l (else 1).  Lattices are added until
// every k in I is alone at its index k.z_l mod M_l in at least one of them; first[k] receives the
// first such l (0-based).  false if max_lattices lattices do not get there.
bool multiple_lattices(const int8_t* I, int64_t n, int d, uint64_t seed, int max_lattices, std::vector<int64_t>& z,
                       std::vector<int64_t>& M, std::vector<int>& first);

// Candidate set J_t = I_prev x I_t within [-N,N]^t (lexicographic in the positions).
void candidate_set(const int8_t* I_prev, int64_t n_prev, int t_prev, const std::vector<int>& I_t, int N,
                   std::vector<int8_t>& J, int64_t& nJ);

// ---------------------------------------------------------------------------------
// Device-side descriptions passed to kernels by value
// ---------------------------------------------------------------------------------
struct NodeSpec {          // M sampling nodes: lattice coordinates and fixed tails
    int64_t M;
    int d;
    int64_t z[USFFT_MAX_D];      // >= 0: lattice coordinate with multiplier z_j; -1: tail
    double tail[USFFT_MAX_D];    // y'_j for tail coordinates
    const double* Y;             // non-NULL: explicit points, node i is Y[i*d .. i*d+d) (device;
                                 // parameters of the model's domain; z and tail unused)
    int map;                     // USFFT_MAP_*: Theta_j of a torus coordinate (Sec. 3.2)
    double map_alpha, map_beta, map_shift;
    // the k-th node of the set is lattice node first + max(stride, 1) k (a rank's strided part of
    // the lattice in the sharded form; first = stride = 0: node k is lattice node k)
    int64_t first, stride;
};

// number of nodes of a lattice node set (M, or the rank's strided share of it)
inline int64_t node_count(const NodeSpec& ns) {
    return ns.stride > 1 ? (ns.M - ns.first + ns.stride - 1) / ns.stride : ns.M;
}

// Theta_j and the inverse map on the device (k_theta.cuh) take these fields of a problem.
struct ParamMap {
    int map;
    double alpha, beta, shift;
};

struct FftPlan {           // M = L1 * L2 (L2 == 1: single pass of length L1)
    int64_t M;
    int L1, L2;
};

// ---------------------------------------------------------------------------------
// Kernel launchers (defined in the .cu files); all return cudaGetLastError()
// ---------------------------------------------------------------------------------
// psi[j][e] = c j^-mu psi_j(centroid_e), j < d, e < E (E = n+1 in 1-D, 2(n+1)^2 in 2-D)
cudaError_t launch_psi_table(int kind, int n, int d, double scale, double decay, double* psi,
                             cudaStream_t s);

// 1-D: fused coefficient assembly + cyclic reduction; U[i][g], i < M, g < n
cudaError_t launch_sample_1d(const NodeSpec& ns, int n, int coef_model, double f, const double* psi,
                             int64_t i0, int64_t count, double* U, cudaStream_t s, int* launches);

// 2-D: fused coefficient assembly + Jacobi-PCG (fp64) or fp32-PCG with fp64-residual
// refinement (mixed); iters_out[i] receives the CG iterations of system i (may be NULL);
// fail_count gets +1 for every system that hit max_iters; iters_sum[0] accumulates the CG
// iterations and, for the refinement kernels, iters_sum[1] the refinement steps.
struct CgConfig {
    int precision;
    int max_iters;
    double tol;
    int blocks;            // 0 = auto
    double coef_scale;     // c and mu of the coefficient (the MIXED kernel assembles from them
    double coef_decay;     // directly, in separable form, instead of reading the mode table)
};
cudaError_t launch_sample_2d(const NodeSpec& ns, int n, int coef_model, double f, const double* psi,
                             const CgConfig& cg, int64_t i0, int64_t count, double* U, int* iters_out,
                             unsigned int* fail_count, unsigned long long* iters_sum, double* scratch,
                             size_t scratch_bytes, cudaStream_t s, int* launches);
size_t sample_2d_scratch_bytes(int n, int precision, int blocks);
// shared memory of the large-mesh (n > 63) MIXED kernel; at most 232448 bytes can be launched
size_t big_smem_bytes(int n, int d);
int sample_2d_default_blocks(int n, int precision);

// TRIGPOLY black box: U[i][g] = Re sum_s c_{g,s} exp(2 pi i h_{g,s} . y_i)
cudaError_t launch_sample_trigpoly(const NodeSpec& ns, int G, int nterms, const int8_t* freqs,
                                   const double* coefs, double* aux /* [G*nterms*3] */, double* U,
                                   cudaStream_t s, int* launches);

// FFT along the lattice axis with the gather at the DFT indices of the candidates:
// C[g][k] = (1/M) sum_i U[i][g] exp(-2 pi i i m_k / M).
struct GatherPlan {        // buckets of candidates by m mod L1 (CSR), entries (k, m div L1)
    const int* offsets;    // [L1 + 1]
    const int* k;          // [nJ]
    const int* m2;         // [nJ]
    // the single in-place pass (optional): input row i at position pos_of[i] ([M]); the
    // candidates' DFT indices m_k ([nJ]); both NULL for the bucketed passes only
    const int* pos_of = nullptr;
    const int* mk = nullptr;
};
// pos_of of the single in-place pass for lattice size M (empty if M does not fit on chip)
std::vector<int> fft_inplace_positions(int64_t M);
FftPlan make_fft_plan(int64_t M);
size_t fft_scratch_bytes(const FftPlan& p, int G);
// W[j] = e^{-2 pi i j / M}: fp64 (double2) or double-float (float4 = re.hi, re.lo, im.hi, im.lo)
cudaError_t launch_twiddles(int64_t M, void* W, bool df, cudaStream_t s, int* launches);
// df selects double-float arithmetic for the transform (W must then be the float4 table);
// the scratch holds [M][ceil(G/2)] 16-byte complex values of the same arithmetic.
cudaError_t launch_fft_gather(const FftPlan& p, int G, const double* U, const void* W, bool df,
                              const GatherPlan& gp, int64_t nJ, void* scratch, double2* C,
                              cudaStream_t s, int* launches);

// Random-lattice estimate (Algorithm A): C[g][k] = Call[src[k]][g][k] where src[k] >= 0 (the
// first lattice with k alone at its index), else the median over the L lattices of the real
// and, separately, the imaginary parts (L odd, <= 31).  Call is [L][G][nJ].
// C[g][k] = Call[src[k]][g][k] (step 3 on multiple rank-1 lattices: src[k] in [0, L) for every k)
cudaError_t launch_lattice_pick(const double2* Call, int L, int G, int64_t nJ, const int* src, double2* C,
                                cudaStream_t s, int* launches);
cudaError_t launch_random_lattice_combine(const double2* Call, int L, int G, int64_t nJ, const int* src, double2* C,
                                          cudaStream_t s, int* launches);

// Per-node selection of the <= s~ largest |C[g][k]| >= theta and the union (bitmap OR).
cudaError_t launch_select_union(const double2* C, int G, int64_t nJ, double theta, int s_tilde,
                                uint32_t* bitmap, cudaStream_t s, int* launches);
// out = max_g |C[g][col]|
cudaError_t launch_absmax_column(const double2* C, int G, int64_t nJ, int64_t col, double* out,
                                 cudaStream_t s, int* launches);

// Sparse approximation at explicit points (Section 4): V[j][g] = sum_k C[g][k] e^{2 pi i k.y_j}
// (V may be NULL); with Uchk, per point tile r of 64 points and node g the partials
// part_sum[r][g] = sum_j |Uchk[j][g] - V[j][g]|^2 and part_max[r][g] = max_j |...|.
int64_t evaluate_max_points();
int evaluate_point_tile();
// Y holds parameters of the model's domain; the kernel maps them to the torus (phi^-1, Eq. (3.1)).
cudaError_t launch_evaluate(const double* Y, int64_t n, int d, const ParamMap& pm, const int8_t* I, int64_t nI,
                            const double2* C, int G, double2* V, const double* Uchk, double* part_sum,
                            double* part_max, cudaStream_t s, int* launches);
// tot_sum[g] += sum_r part_sum[r][g], tot_max[g] = max(tot_max[g], max_r part_max[r][g])
cudaError_t launch_error_accumulate(const double* part_sum, const double* part_max, int tiles, int G, double* tot_sum,
                                    double* tot_max, cudaStream_t s, int* launches);
// tot_sum[g] <- sqrt(tot_sum[g] / n)
cudaError_t launch_error_finalize(double* tot_sum, int G, int64_t n, cudaStream_t s, int* launches);

// Quantities of interest (Sec. 4, 4.1): dfac[k] = D_k of frequency row k (int8 [nI][d]) under
// the map; then per node g mean[g] = sum_k C[g][k] D_k, var[g] = sum_{k != 0} |C[g][k]|^2 and
// gsi[g][l-1] = sum_{k in J_l} |C[g][k]|^2 / var[g], with the rows grouped by order l through
// perm / offsets (order l = offsets[l] .. offsets[l+1]-1 of perm, l = 0..d).
cudaError_t launch_expectation_factors(const int8_t* I, int64_t nI, int d, const ParamMap& pm, double2* dfac,
                                       cudaStream_t s, int* launches);
cudaError_t launch_statistics(const double2* C, int G, int64_t nI, int d, const double2* dfac, const int* perm,
                              const int64_t* offsets, double2* mean, double* var, double* gsi, cudaStream_t s,
                              int* launches);

// Tuned launch parameters (tune.cpp; filled by usfft_autotune): tune_get returns the stored value
// or `fallback`.  Knobs that leave results bit-identical only.
enum TuneKnob { TUNE_SAMPLER_BLOCKS = 1, TUNE_FFT_TILE = 2 };
int tune_get(int knob, int64_t key, int fallback);
void tune_set(int knob, int64_t key, int value, double ms);
void tune_erase(int knob, int64_t key);
std::string tune_dump();
bool tune_parse(const char* text, std::string& err);
void tune_clear();
// keys of the knobs
inline int64_t tune_key_sampler(int precision, int n) { return (int64_t)precision * 64 + (n + 15) / 16; }
inline int64_t tune_key_fft(int L, bool final_pass) { return 2 * (int64_t)L + (final_pass ? 1 : 0); }
// the two-pass FFT's default column-pair tile, and whether a tile fits its shared memory
int fft_default_tile(int L, int Gp, int nb);
bool fft_tile_fits(int L, int Gt, int nb);

// Raises the kernel's dynamic shared-memory limit to at least `bytes` (never lowers it: plans
// launch from several host threads at once); smem_attr.cpp.
cudaError_t allow_dyn_smem(const void* func, size_t bytes);

// Sets the message usfft_last_error(NULL) returns on the calling thread (capi.cu).
void set_thread_error(const std::string& msg);

}  // namespace usfft
