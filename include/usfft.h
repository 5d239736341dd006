/*
 * usfft.h -- C ABI of the GB300 (sm_103a) usFFT sampling-and-detection library.
 *
 * The library runs the dimension-incremental detection of the uniform sparse FFT
 * (usFFT; Kaemmerer, Potts, Taubert, "The uniform sparse FFT with application to PDEs
 * with random coefficients", Algorithm 1, steps 1, 2a and 2) for the parametric
 * elliptic problem -div(a(x,y) grad u) = f, u = 0 on the boundary (Eq. (1.1)), with
 * the PDE solved on the GPU at every sampling node (the "black box" of Sec. 2.1).
 *
 * One increment t (see usfft_increment) runs, on one GPU:
 *   - the 1-D detections of dimension t (Algorithm 1, steps 1 & 2a);
 *   - for t >= 2 the coupled step t (Algorithm 1, step 2): candidate set J_t, a
 *     reconstructing rank-1 lattice (Appendix A), FE solves at its M nodes
 *     (fused coefficient assembly + cyclic reduction in 1-D / preconditioned CG in
 *     2-D), one length-M FFT per mesh node with the gather at k.z mod M, per-node
 *     selection of the <= s~ largest coefficients >= theta and the union over nodes.
 *
 * Conventions for every entry point:
 *   - Return value: usfft_status; USFFT_OK (0) on success.  No call aborts the process.
 *     On failure the plan's message is available through usfft_last_error(plan)
 *     (or usfft_last_error(NULL) for failures before a plan exists).
 *   - Pointers are host pointers unless the argument says "device".
 *   - A plan is not thread-safe: one host thread at a time per plan.
 *   - Device memory: the plan owns every buffer it allocates.  If params->alloc is
 *     non-NULL all device memory comes from that allocator (the Python binding passes
 *     PyTorch's caching allocator); otherwise cudaMalloc/cudaFree are used.
 *   - Stream: all device work of a plan is issued on the stream given to usfft_plan
 *     (NULL = the legacy default stream).  Calls that return host data synchronise
 *     that stream with a host-side deadline (USFFT_ETIMEOUT, never a device trap).
 */
#ifndef USFFT_H
#define USFFT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    USFFT_OK = 0,
    USFFT_EINVAL = 1,     /* invalid argument or problem (e.g. a_min <= 0, sizes out of range) */
    USFFT_ENOMEM = 2,     /* allocation failed or the hbm_budget_bytes would be exceeded */
    USFFT_ELATTICE = 3,   /* no reconstructing lattice within max_lattice_trials x max_lattice_sizes */
    USFFT_ENOCONV = 4,    /* a CG solve hit max_cg_iters before its tolerance */
    USFFT_ETIMEOUT = 5,   /* the device did not finish before the host-side deadline */
    USFFT_ECUDA = 6,      /* a CUDA runtime call failed (message holds the CUDA error string) */
    USFFT_ESTATE = 7,     /* call not valid in the plan's state (e.g. increment after t = d) */
    USFFT_ECOMM = 8       /* the collective hook of the sharded form reported a failure */
} usfft_status;

/* problem kinds */
#define USFFT_PDE_1D 1        /* (0,1), n interior nodes, P1 elements of width h = 1/(n+1)        */
#define USFFT_PDE_2D 2        /* unit square, n*n interior nodes, "/"-split squares of side 1/(n+1) */
#define USFFT_TRIGPOLY 3      /* test black box: G real trigonometric polynomials (Theorem 1.1)   */

/* coefficient models (Eq. (1.2) and the lognormal form of Sec. 1):
 *   AFFINE_SIN:    a(x,y) = 1 + sum_{j<=d} c j^-mu psi_j(x) Theta_j(y)
 *   LOGNORMAL_SIN: a(x,y) = exp(sum_{j<=d} c j^-mu psi_j(x) Theta_j(y))
 * with Theta_j chosen by the problem's theta_map (below): sin(2 pi y_j) for the periodic
 * model of Sec. 4.2, else the parameter y_j itself (affine / lognormal models).
 * psi_j(x) = sin(j pi x) in 1-D; sin(j1 pi x1) sin(j2 pi x2) in 2-D with (j1, j2) the
 * j-th pair of the diagonal enumeration of Sec. 4.3 / Table 4.2, shifted by one:
 * (1,1), (1,2), (2,1), (1,3), (2,2), (3,1), ...  The coefficient of an element is taken
 * at its centroid (midpoint in 1-D). */
#define USFFT_COEF_AFFINE_SIN 1
#define USFFT_COEF_LOGNORMAL_SIN 2

/* parameter maps (theta_map; Sec. 3.2).  The library samples on the torus: a sampling node
 * y~ in [0,1)^d gives Theta_j = sin(2 pi y~_j) (PERIODIC, no periodization), or Theta_j =
 * phi_j(y~_j) with
 *   TENT:   phi_j(y~) = beta - |(beta - alpha)(1 - 2 y~)|  (Eq. (3.2); y_j uniform on
 *           [alpha, beta], affine model), inverse (y - alpha) / (2 (beta - alpha));
 *   NORMAL: phi_{j,Delta} = tau_1 o tau_{2,Delta} (Eq. (3.3); y_j standard normal, lognormal
 *           model), tau_1(v) = sqrt(2) erfinv(2 v), tau_{2,Delta} the shifted tent with poles
 *           at y~ = Delta and 1/2 + Delta; inverse y~ = erf(y / sqrt 2) / 4 + Delta + 1/4.
 * The detected coefficients are those of u~(x, y~) = u(x, phi(y~)).  Explicit points (the
 * evaluation calls) are parameters y of the model's own domain. */
#define USFFT_MAP_PERIODIC 0
#define USFFT_MAP_TENT 1
#define USFFT_MAP_NORMAL 2

/* precision of the sampler */
#define USFFT_FP64 0          /* fp64 everywhere; 2-D solves by Jacobi-preconditioned CG */
#define USFFT_MIXED 1         /* 2-D: fp64-residual iterative refinement around fp32 flexible CG
                                 (one block reduction per iteration) preconditioned by the
                                 constant-coefficient operator (2-D sine transform as BF16
                                 tensor-core GEMMs); 1-D: fp64; the lattice FFT in double-float
                                 (pairs of fp32), its gathered output and the selection in fp64 */
#define USFFT_MIXED_JACOBI 2  /* 2-D: the same refinement around fp32 Jacobi-CG (for comparison) */
#define USFFT_FP64_DST 3      /* fp64 everywhere; 2-D solves by fp64 CG preconditioned by the same
                                 constant-coefficient operator as USFFT_MIXED, applied exactly (the
                                 sine transforms as fp64 matrix products): against USFFT_MIXED it
                                 differs in the arithmetic precision only; 1-D and TRIGPOLY as FP64 */

typedef struct {
    int kind;                 /* USFFT_PDE_1D | USFFT_PDE_2D | USFFT_TRIGPOLY */
    int n;                    /* PDE: interior nodes per side, 1 <= n <= 1023 (1-D); 2-D: 1 <= n <= 127
                                 with USFFT_MIXED and USFFT_FP64_DST, 1 <= n <= 63 with USFFT_FP64 and
                                 USFFT_MIXED_JACOBI */
    int d;                    /* stochastic dimension, 1 <= d <= 64 */
    int coef_model;           /* USFFT_COEF_* (PDE kinds) */
    double coef_scale;        /* c  */
    double coef_decay;        /* mu */
    double f_const;           /* constant right-hand side f */
    /* TRIGPOLY only (copied at plan time; the caller keeps ownership):
     * G = tp_nodes polynomials, each with tp_nterms slots; slot (g, s) holds the frequency
     * tp_freqs[(g*tp_nterms + s)*d + j] (j = 0..d-1) and the complex coefficient
     * (tp_coefs[2*(g*tp_nterms+s)], tp_coefs[2*(g*tp_nterms+s)+1]); a zero coefficient marks
     * an unused slot.  The sample is the real part of the sum, so supports should be closed
     * under k -> -k with conjugate coefficients. */
    int tp_nodes;
    int tp_nterms;
    const int8_t* tp_freqs;
    const double* tp_coefs;
    /* parameter map (PDE kinds; TRIGPOLY takes PERIODIC only) */
    int theta_map;            /* USFFT_MAP_PERIODIC | USFFT_MAP_TENT | USFFT_MAP_NORMAL */
    double map_alpha;         /* TENT: alpha < beta */
    double map_beta;
    double map_shift;         /* NORMAL: Delta in (0, 1/2); a lattice with a node at a pole is
                                 rejected (USFFT_EINVAL); Lemma 3.1 gives 1/(4M) as the best
                                 Delta for a single prime-size lattice */
} usfft_problem;

/* Device allocator hook: alloc(bytes, stream, ctx) returns device memory or NULL;
 * free(ptr, stream, ctx) releases it. */
typedef void* (*usfft_alloc_fn)(size_t bytes, void* stream, void* ctx);
typedef void (*usfft_free_fn)(void* ptr, void* stream, void* ctx);

typedef struct {
    int N;                    /* search domain Gamma = [-N, N]^d, 1 <= N <= 127 */
    int s;                    /* sparsity s (s~ of the last increment, t = d) */
    int s_local;              /* s_local (s~ of increments t < d and of the 1-D detections) */
    double delta;             /* threshold: theta = delta (absolute) or delta * A (relative) */
    int delta_is_relative;    /* relative: A = max_g |c~_{g,0}| of the 1-D detection t=1, i=1 */
    int r;                    /* detection iterations r (r~ = 1 at t = d) */
    uint64_t seed;            /* key of the counter-based SplitMix64 draws (tails, lattices) */
    int precision;            /* USFFT_FP64 | USFFT_MIXED | USFFT_MIXED_JACOBI | USFFT_FP64_DST */
    size_t hbm_budget_bytes;  /* 0 = unlimited; otherwise ENOMEM beyond this many plan bytes */
    int max_cg_iters;         /* per CG solve (inner solve in MIXED); 0 = 4000 */
    int max_lattice_trials;   /* generating vectors tried per lattice size; 0 = 64 */
    double cg_tol;            /* relative residual target of the FE solve; 0 = 1e-13 */
    usfft_alloc_fn alloc;     /* NULL = cudaMalloc */
    usfft_free_fn free;
    void* alloc_ctx;
    /* Sampling of the coupled steps (Algorithm A):
     *   rr_lattices = 0: one reconstructing rank-1 lattice per detection iteration (above);
     *   rr_lattices = L (odd, <= 31): L random rank-1 lattices per detection iteration, all
     *   sampling the same projection (the iteration's tails).  Sizes: M_1 = smallest 7-smooth
     *   size >= ceil(rr_size_factor * max(|I^(1..t-1)|, |I^(t)|, s~)) (at least 2), M_(l+1) the
     *   next 7-smooth size after M_l; every component of z_l a unit mod M_l drawn from the
     *   counter RNG (phase 5).  Estimate of c_k: the value of the first lattice in which no
     *   other candidate shares k's index, else the median over the L lattices of the real
     *   and, separately, the imaginary parts.  Fewer samples than one reconstructing lattice
     *   (sizes grow with max(s, N) instead of |J_t|) at the price of a failure probability
     *   (proof of Theorem 1.1, Appendix B).  Step 3 always uses one reconstructing lattice. */
    int rr_lattices;
    double rr_size_factor;    /* 0 = 2.0 */
    int max_lattice_sizes;    /* lattice sizes the reconstructing-lattice search tries; 0 = 400 */
} usfft_params;

typedef struct {
    int t;                    /* increment just completed (1-based) */
    int64_t M;                /* lattice size of the coupled step (0 for t = 1) */
    int64_t n_candidates;     /* |J_t| (K_t = 2N+1 for t = 1) */
    int64_t n_detected;       /* |I^(1..t)| */
    int64_t n_1d;             /* |I^(t)| */
    int64_t samples;          /* lattice samples (FE solves) this increment: r*K + r~*M */
    int64_t cg_iters_total;   /* summed over all solves (2-D); 0 for 1-D / TRIGPOLY */
    int32_t cg_iters_max;
    int32_t kernel_launches;  /* kernels this increment launched */
    double theta;             /* absolute threshold in use */
    double ms_device;         /* device time of the increment's kernels (CUDA events) */
    double ms_host_plan;      /* host time of J_t construction + lattice search */
    int64_t h2d_bytes;        /* host-to-device bytes copied by this increment */
    int64_t d2h_bytes;        /* device-to-host bytes copied by this increment */
} usfft_increment_info;

typedef struct usfft_plan_s usfft_plan_t;

/* Create a plan: validates the problem (uniform ellipticity, Eq. (2.1): a_min > 0 for the
 * affine model), copies it, precomputes the mode table psi_j(centroid_e) on the device.
 * stream: a cudaStream_t (NULL = default stream).  *out receives the plan or NULL. */
usfft_status usfft_plan(const usfft_problem* problem, const usfft_params* params,
                        void* stream, usfft_plan_t** out);

/* Run the next increment t = (previous t) + 1 <= d (semantics in the file header).
 * info may be NULL.  Synchronises the plan's stream before returning (the detected
 * set is host data). */
usfft_status usfft_increment(usfft_plan_t* plan, usfft_increment_info* info);

/* Re-run the device part of the last coupled step (sampling, FFT + gather, selection,
 * union for all r~ iterations) on the resident lattice, candidate indices and tails,
 * without any host planning or host<->device copies; the detected set is recomputed on
 * the device.  For timing; the result equals the last increment's.  If sync == 0 the call
 * returns after enqueueing (kernel count in *launches, may be NULL). */
usfft_status usfft_replay(usfft_plan_t* plan, int sync, int32_t* launches);

/* Go back to the state after increment t (0 <= t <= current); the plan keeps every
 * detected set, so a later usfft_increment recomputes increment t+1 exactly. */
usfft_status usfft_rewind(usfft_plan_t* plan, int t);

/* Resume from a checkpoint: set the state after increment t (0 <= t <= d) to the detected
 * set I^(1..t) ([n][t] int8 rows, host) and the absolute threshold theta (> 0; ignored
 * when t == 0).  The next usfft_increment runs increment t+1 from this state exactly as it
 * would have after the increments 1..t (Algorithm 1 needs only I^(1..t) and theta to
 * continue; every draw is keyed by (phase, t, i, j)); with t == d the next call is
 * usfft_reconstruct.  Earlier history is discarded. */
usfft_status usfft_resume(usfft_plan_t* plan, int t, const int8_t* I, int64_t n, double theta);

/* Stage timing for measurement.  usfft_set_timing(plan, on) resets the accumulators; with
 * timing on, every later increment or replay records a CUDA event pair (on the plan's
 * stream) around each stage launch.  usfft_get_stage_times synchronises the stream and
 * returns, accumulated since the reset, the device time and launch count per stage, the
 * total CG iterations and the total refinement steps of the 2-D solves. */
#define USFFT_STAGE_SAMPLE 0   /* coefficient assembly + FE solve (the black-box sampler) */
#define USFFT_STAGE_FFT 1      /* lattice FFT + gather at k.z mod M */
#define USFFT_STAGE_SELECT 2   /* threshold / top-s~ selection + union */
typedef struct {
    double ms[3];
    int32_t launches[3];
    int64_t cg_iters_total;       /* CG iterations (inner iterations in the refinement modes) */
    int64_t refine_steps_total;   /* fp64 refinement steps (USFFT_MIXED, USFFT_MIXED_JACOBI) */
} usfft_stage_times;
usfft_status usfft_set_timing(usfft_plan_t* plan, int on);
usfft_status usfft_get_stage_times(usfft_plan_t* plan, usfft_stage_times* out);

/* Current detected set I^(1..t): *n receives |I|; if freqs is non-NULL it receives
 * |I| rows of t int8 values (capacity *n_capacity rows; EINVAL if too small). */
usfft_status usfft_get_set(const usfft_plan_t* plan, int8_t* freqs, int64_t n_capacity,
                           int64_t* n, int32_t* t);

/* Final coefficients (Algorithm 1, step 3) on the detected set I = I^(1..d), after all d
 * increments (USFFT_ESTATE before): a reconstructing rank-1 lattice for I is searched with
 * the rule of usfft_search_lattice, its draws keyed by phase 4 instead of 3; the FE problem
 * is solved at its M nodes (all d coordinates on the lattice, no random tails) and each
 * node's length-M FFT is read at k.z mod M, without a threshold.  The paper uses multiple
 * rank-1 lattices here; one reconstructing lattice computes the same coefficients exactly
 * for trigonometric polynomials supported in I (Appendix A).
 * *n receives |I|; freqs (may be NULL) receives [|I|][d] int8; coefs (may be NULL: only the
 * sizes are returned) receives [G][|I|][2] (re, im) fp64 through a host pointer, or a device
 * pointer when coefs_on_device != 0.  The last-step inspection calls then describe this
 * step (lattice, candidates = I, samples, coefficients). */
usfft_status usfft_reconstruct(usfft_plan_t* plan, int64_t* n, int8_t* freqs, double* coefs,
                               int coefs_on_device);

/* Step 3 on multiple rank-1 lattices, the paper's choice there (Algorithm 1, step 3; Appendix A,
 * the sampling bound M <= ceil(2 ln(2|I|)) 4 (|I| - 1)).  Same arguments, outputs, errors and
 * stored reconstruction as usfft_reconstruct.  The lattices are those of usfft_multiple_lattices
 * for I and params.seed: sizes from the smallest 7-smooth size >= 2 (|I| - 1) upwards, each
 * generating vector drawn (draws keyed by phase 6), added until every k of I is alone at its index
 * k.z_l mod M_l in at least one lattice (USFFT_ELATTICE if 64 lattices do not get there).  The FE
 * problem is solved at the nodes of every lattice (all d coordinates on the lattice, no tails),
 * each node's length-M_l FFT is read at k.z_l mod M_l, and c_k is the value of the first lattice
 * in which k is alone: the exact coefficient for trigonometric polynomials supported in I.
 * Afterwards usfft_get_random_lattices returns these lattices (count L, t = d) and the
 * single-lattice inspection calls describe the last one. */
usfft_status usfft_reconstruct_multiple(usfft_plan_t* plan, int64_t* n, int8_t* freqs, double* coefs,
                                        int coefs_on_device);

/* Evaluation at explicit parameter points (Section 4).  y is [n][d] fp64 row-major (one
 * point y^(j) per row; coordinates on the torus, any real value is taken mod 1 by the
 * 1-periodic coefficient model).  With on_device != 0, y and the output are device pointers
 * (the calls then work in place, in one pass), else host pointers (staged through the plan
 * in chunks of 8192 points).  Outputs belong to the caller. */

/* The black box at the points: the FE solution u-check(x_g, y^(j)) of Eq. (1.1) for fixed
 * y^(j) (or the test polynomials' values), samples [n][G] fp64.  USFFT_ENOCONV if a 2-D
 * solve misses the CG tolerance. */
usfft_status usfft_sample_points(usfft_plan_t* plan, const double* y, int64_t n, double* samples,
                                 int on_device);

/* The approximation u^usFFT(x_g, y^(j)) = sum_{k in I} c_{g,k} e^{2 pi i k.y^(j)} with the set
 * and coefficients of the last usfft_reconstruct (USFFT_ESTATE before one): values
 * [n][G][2] (re, im) fp64.  The imaginary part is zero up to rounding when I is closed under
 * k -> -k (the coefficients of a real function are then conjugate pairs). */
usfft_status usfft_evaluate(usfft_plan_t* plan, const double* y, int64_t n, double* values,
                            int on_device);

/* The errors of Section 4 over n >= 1 test points, per mesh node g:
 *   err2[g]   = ( (1/n) sum_j |u-check(x_g, y^(j)) - u^usFFT(x_g, y^(j))|^2 )^(1/2)
 *   errinf[g] = max_j |u-check(x_g, y^(j)) - u^usFFT(x_g, y^(j))|
 * (|.| the complex modulus).  y is a host (y_on_device == 0) or device pointer; err2 and
 * errinf are host arrays of G doubles.  The FE solutions and the approximation are formed
 * chunk by chunk on the device and never leave it; the sums are reduced in a fixed order. */
usfft_status usfft_errors(usfft_plan_t* plan, const double* y, int64_t n, int y_on_device,
                          double* err2, double* errinf);

/* Quantities of interest of the last usfft_reconstruct (USFFT_ESTATE before one), per mesh
 * node g (host arrays, each may be NULL):
 *   mean[g][2]   E(u^usFFT(x_g, .)) = sum_{k in I} c_{g,k} D_k (Sec. 4.1): D_k = prod_j D_{k_j}
 *                with D_{k_j} = 1 for k_j = 0 and, for k_j != 0, 0 (PERIODIC: the mean is
 *                c_{g,0}), 2i/(pi k_j) for odd k_j and 0 for even k_j (TENT, Eq. (4.5)), the
 *                TENT factor times e^{2 pi i k_j Delta} (NORMAL);
 *   variance[g]  sigma^2 = sum_{k in I, k != 0} |c_{g,k}|^2 (Sec. 4);
 *   gsi[g][l-1]  the global sensitivity index rho(J_l) (Eq. (4.3)) of J_l = the k in I with
 *                exactly l non-zero components (Eq. (4.4)), l = 1..d (0 where sigma^2 = 0).
 * One warp per node reads the node's coefficients once; sums are reduced in a fixed order. */
usfft_status usfft_statistics(usfft_plan_t* plan, double* mean, double* variance, double* gsi);

/* Inspection of the last detection step (the coupled step of the last increment, or the
 * 1-D detection when t = 1): lattice, candidates J_t with their DFT indices k.z mod M,
 * and the samples U [M][G], coefficients C [G][|J|] and union bitmap of its LAST detection
 * iteration (the resident buffers).  Sizes are queried with NULL outputs.  The copies
 * synchronise the plan's stream. */
usfft_status usfft_get_lattice(const usfft_plan_t* plan, int64_t* z /* [t] or NULL */,
                               int64_t* M, int32_t* t);
usfft_status usfft_get_candidates(const usfft_plan_t* plan, int8_t* J /* [|J|][t] or NULL */,
                                  int64_t* n, int64_t* m /* [|J|] DFT indices or NULL */);
usfft_status usfft_get_samples(const usfft_plan_t* plan, double* U /* host [M][G] or NULL */,
                               int64_t* M, int64_t* G);
usfft_status usfft_get_coefficients(const usfft_plan_t* plan, double* C /* host [G][|J|][2] or NULL */,
                                    int64_t* G, int64_t* n);
usfft_status usfft_get_selection(const usfft_plan_t* plan, uint32_t* bitmap /* host, ceil(|J|/32) */,
                                 int64_t* n);

/* Per-iteration inspection of the last detection step (Algorithm 1, steps 2b-2e, repeated over
 * the r~ detection iterations; single reconstructing lattice only).  usfft_set_keep_iterations
 * (plan, 1) makes every later detection step copy, after each iteration i, its samples U [M][G],
 * coefficients C [G][|J|] and the union bitmap of iterations 1..i into plan-owned device buffers
 * (r~ copies of each; counted in usfft_plan_bytes); on = 0 frees them.  Off by default (the
 * copies cost device time and memory).  usfft_get_iteration: *count (may be NULL) receives the
 * number of kept iterations of the last detection step (0 after a random-lattice step or with
 * keeping off); if any of U, C, bitmap (host, sized as for usfft_get_samples,
 * usfft_get_coefficients and usfft_get_selection) is non-NULL, iteration i (1 <= i <= count,
 * else USFFT_EINVAL) is copied there.  Synchronises the plan's stream. */
usfft_status usfft_set_keep_iterations(usfft_plan_t* plan, int on);
usfft_status usfft_get_iteration(const usfft_plan_t* plan, int i, double* U, double* C, uint32_t* bitmap,
                                 int32_t* count);

/* The random rank-1 lattices of the last coupled step when params.rr_lattices > 0 (after
 * usfft_reconstruct_multiple: step 3's lattices, count L, t = d): *count
 * receives r~ * L (0 after a single-lattice step or a 1-D step), *t the number of lattice
 * coordinates; z (may be NULL) receives [count][t] generating vectors and M (may be NULL)
 * [count] sizes, lattice q = (i-1)*L + (l-1) of detection iteration i.  With random lattices
 * the single-lattice inspection calls (usfft_get_lattice, usfft_get_candidates' indices,
 * usfft_get_samples) describe the last lattice sampled; usfft_get_coefficients returns the
 * estimate of the last iteration. */
usfft_status usfft_get_random_lattices(const usfft_plan_t* plan, int64_t* z, int64_t* M, int32_t* count,
                                       int32_t* t);

/* Message of the last failure of this plan (plan == NULL: of the calling thread). */
const char* usfft_last_error(const usfft_plan_t* plan);

/* Device bytes the plan holds now (its buffers grow with the lattice sizes it meets).  The one
 * call that may run while another thread works on the same plan (it reads one counter). */
size_t usfft_plan_bytes(const usfft_plan_t* plan);

/* The batched form: one increment (usfft_increment) of each of `count` distinct plans at
 * once.  The host work of the plans runs in up to max_threads threads (0: one per hardware
 * thread) and their device work overlaps on the plans' streams, so the plans should have been
 * created on distinct streams.  statuses[k] and infos[k] (infos may be NULL) receive plan k's
 * result, which is the one the plan gives alone; the return value is the first non-OK status
 * in plan order (USFFT_EINVAL for a NULL or repeated plan, nothing run). */
usfft_status usfft_increment_many(usfft_plan_t* const* plans, int count, int max_threads,
                                  usfft_increment_info* infos, usfft_status* statuses);

/* ---- Sharded form: one instance over several GPUs (one process or thread per rank) ----
 *
 * The coupled step of increment t splits by lattice residue: with P ranks the lattice size M is
 * taken from the sizes that are also multiples of P (the rule of usfft_search_lattice_multiple),
 * rank p solves the FE problem at the nodes i = p + P i2 (i2 < M / P) only, runs the length-M/P
 * lattice FFT over them, reads it at k.z mod (M/P) and multiplies by e^{-2 pi i p (k.z mod M) / M}
 * / P: the sum of these partial coefficients over the ranks is the DFT of Algorithm 1, step 2d.
 * The exchange is an all-reduce through the caller's hook (below): a sum of the G x |J_t| complex
 * coefficients per detection iteration, then each rank selects the <= s~ largest >= theta at its
 * block of mesh nodes (g in [G p / P, G (p+1) / P)) and the union is a maximum-reduce of one byte
 * per candidate.  The 1-D detections (2N + 1 nodes) run in full on every rank.  Every rank ends
 * with the same detected set, which equals the unsharded result for the same lattice (the sums
 * are ordered differently, so coefficients agree to rounding).
 *
 * Hook: allreduce(buf, count, dtype, op, stream, ctx) must replace the `count` elements at the
 * device pointer buf by their sum (op USFFT_RED_SUM) or maximum (USFFT_RED_MAX) over all ranks,
 * ordered after the work already issued on `stream` (the plan's stream) and before the work issued
 * on it later; dtype USFFT_RED_F64 (double) or USFFT_RED_U8 (uint8_t).  It returns 0 on success;
 * anything else ends the call with USFFT_ECOMM.  Every rank must make the same sequence of calls.
 * The Python module paper_2109_04131_gb300/sharded.py provides one over torch.distributed (NCCL). */
#define USFFT_RED_SUM 0
#define USFFT_RED_MAX 1
#define USFFT_RED_F64 0
#define USFFT_RED_U8 1
typedef int (*usfft_allreduce_fn)(void* buf, size_t count, int dtype, int op, void* stream, void* ctx);

/* Increment t of the plan as rank `rank` of `nranks` (1 <= nranks <= 64, all prime factors <= 7;
 * nranks = 1 is usfft_increment).  Each rank holds its own plan of the same problem and
 * parameters (single-lattice detection: rr_lattices = 0).  info->samples counts this rank's
 * solves; info->M is the full lattice size.  Afterwards usfft_get_lattice and
 * usfft_get_candidates describe the full lattice, usfft_get_samples returns this rank's M / P
 * sample rows (node i = p + P row), usfft_get_coefficients the summed coefficients.
 * usfft_replay of a sharded step repeats its exchange through the same hook (every rank must
 * replay; hook and ctx must still be valid). */
usfft_status usfft_increment_sharded(usfft_plan_t* plan, int rank, int nranks, usfft_allreduce_fn allreduce,
                                     void* ctx, usfft_increment_info* info);

/* The lattice rule of usfft_search_lattice restricted to sizes that are multiples of `divisor`
 * (1 <= divisor <= 64, prime factors <= 7; 1 gives usfft_search_lattice): the sharded form's rule.
 * Host only. */
usfft_status usfft_search_lattice_multiple(const int8_t* J, int64_t n, int t, uint64_t seed, int trials,
                                           int max_sizes, int64_t divisor, int64_t* z, int64_t* M);

/* ---- Autotuning of launch parameters ----
 *
 * usfft_autotune times `reps` replays (usfft_replay) of the plan's last step (0: 3) for each
 * candidate of the launch parameters that leave every result bit-identical, keeps the fastest in a
 * process-wide table and applies it to the plan:
 *   - the persistent grid of the 2-D sampler (the resident CTAs, twice and four times that), keyed
 *     by precision and mesh-size bucket (n + 15) / 16; plans created later start from it;
 *   - the column-pair tile of each pass of the two-pass lattice FFT (1 .. 32 within shared memory),
 *     keyed by the pass's sub-transform length, used by every later launch of that length.
 * The plan needs a completed increment (USFFT_ESTATE otherwise); its detected set and state are
 * unchanged (the replays recompute the last step's result).  out (may be NULL) receives the times
 * per replay before and after and the chosen values (0 where a parameter did not apply).
 * The table as text ("<knob> <key> <value> <ms per replay>" per line, knob 1 = sampler grid,
 * 2 = FFT tile): usfft_tune_export (text may be NULL to query *length; capacity >= length + 1),
 * usfft_tune_import (adds or replaces the entries of the text; NULL clears the table; USFFT_EINVAL
 * and no change if a line does not parse).  The table is shared by all plans of the process and
 * guarded for concurrent use. */
typedef struct {
    double ms_before, ms_after;   /* ms per replay of the last step */
    int32_t sampler_blocks;       /* chosen persistent grid of the 2-D sampler (0: not tuned) */
    int32_t fft_pass1_tile;       /* chosen tiles of the two-pass FFT (0: not tuned) */
    int32_t fft_final_tile;
} usfft_tune_report;
usfft_status usfft_autotune(usfft_plan_t* plan, int reps, usfft_tune_report* out);
usfft_status usfft_tune_export(char* text, size_t capacity, size_t* length);
usfft_status usfft_tune_import(const char* text);

/* Free every device buffer and the plan.  NULL is ignored. */
void usfft_destroy(usfft_plan_t* plan);

/* Library build information, e.g. "usfft sm_103a cudart 13000". */
const char* usfft_version(void);

/* ---- Host-only planner utilities (no device work; usable without a GPU) ---- */

/* The random rank-1 lattice rule of params.rr_lattices on the host (no GPU needed): the L
 * lattices of detection iteration i of the coupled step t, given |I^(1..t-1)| = n_prev,
 * |I^(t)| = n_t and s~ = s_t; z receives [L][t], M receives [L].  USFFT_EINVAL for t outside
 * [1, 64], i < 1, L outside [1, 31] or factor outside (0, 1e6). */
usfft_status usfft_random_lattices(int t, int i, int64_t n_prev, int64_t n_t, int64_t s_t, int L, double factor,
                                   uint64_t seed, int64_t* z, int64_t* M);

/* The multiple rank-1 lattices of usfft_reconstruct_multiple on the host (no GPU needed), for
 * the frequency set freqs ([n][d] int8 rows, host): lattice l = 1, 2, ... has size M_1 = the
 * smallest 7-smooth size >= max(2 (n - 1), 2), M_(l+1) = the smallest 7-smooth size > M_l, and
 * generating vector components z_j, each the first draw in [1, M_l - 1] keyed (seed, 6, l, j, a),
 * a = 0..63, that is coprime to M_l (else 1).  Lattices are added until every k is alone at its
 * index k.z_l mod M_l in at least one of them.  *count receives the number of lattices, z (may be
 * NULL; capacity [max_lattices][d]) their generating vectors and M (may be NULL; capacity
 * [max_lattices]) their sizes.  USFFT_ELATTICE if max_lattices lattices (1..1024) are not enough
 * (the arrays then hold all of them); USFFT_EINVAL for bad arguments. */
usfft_status usfft_multiple_lattices(const int8_t* freqs, int64_t n, int d, uint64_t seed, int max_lattices,
                                     int64_t* z, int64_t* M, int32_t* count);

/* The reconstructing rank-1 lattice search used by usfft_increment for the candidate set
 * J ([n][t] int8, row-major): the smallest admissible (7-smooth) size M >= n, then
 * M' = smallest admissible >= ceil(1.05 M); at each size `trials` generating vectors
 * z = (1, z_2, ..., z_t), z_j uniform in [1, M-1] from the counter-based draws keyed by
 * (seed, 3, t, M, trial, j); the first z with k -> k.z mod M injective on J is returned
 * (Appendix A: a reconstructing lattice makes the single-lattice DFT exact on J).
 * z receives t entries.  USFFT_ELATTICE if none is found within max_sizes sizes.
 * Host only, thread-safe.  For n >= 1024 the (size, trial) pairs of the next sizes are shared out
 * over a small pool of host threads of the calling process (one search at a time; a concurrent
 * search runs in its own thread); the result is that of the sequential scan. */
usfft_status usfft_search_lattice(const int8_t* J, int64_t n, int t, uint64_t seed, int trials,
                                  int max_sizes, int64_t* z, int64_t* M);

/* Counter-based SplitMix64 draws (Steele, Lea, Flood 2014) used for the random tails
 * y' of Algorithm 1 (steps 1/2a and 2b) and the lattice search: the fields are folded one
 * SplitMix64 step each, h <- mix64((h ^ field) + 0x9E3779B97F4A7C15), starting from h = seed.
 * usfft_draw_key returns h; usfft_draw_uniform returns (h >> 11) * 2^-53 in [0, 1). */
uint64_t usfft_draw_key(uint64_t seed, const uint64_t* fields, int nfields);
double usfft_draw_uniform(uint64_t seed, const uint64_t* fields, int nfields);

/* ---- Sampling without device allocation ----
 *
 * usfft_sample_2d_static: the mixed-precision 2-D FE sampler (the USFFT_MIXED solver of
 * usfft_increment: fp64 refinement around fp32 flexible CG with the sine-transform
 * preconditioner) for callers that cannot allocate device memory, e.g. a plug-in inside a
 * framework that has already reserved HBM for its own pool, or a latency-critical loop that
 * must never enter the allocator.  It calls no cudaMalloc, cudaFree or other allocating
 * routine.  The paper has no counterpart: this is a deployment variant of the black-box
 * sampler, not a step of the method.
 *
 * The caller passes inputs and outputs: problem (USFFT_PDE_2D, 1 <= n <= 63, 1 <= d <= 64; host),
 * z[d] and tails[d] (host): coordinate j is a lattice coordinate with y_j = (i z_j mod M)/M
 * when 0 <= z_j < M, otherwise (z_j < 0) it is fixed to tails[j] in [0,1); the nodes
 * i = i0 .. i0+count-1 of that set are solved and their samples written to U (device,
 * [count][n*n] fp64 row-major, caller-owned).  tol (0 = 1e-13) and max_iters (0 = 4000) as in
 * usfft_params.  If unconverged is non-NULL the call synchronises `stream` and stores how many
 * solves missed tol; with NULL it returns after enqueueing the work on `stream`.
 *
 * Scratch: one fixed 40 MiB device array in the library (a counter of unconverged solves and
 * one slot of edge weights, diagonal and residual per resident CTA; the sampler assembles the
 * coefficient in separable form and needs no mode table).  Requests that would need more are
 * rejected with USFFT_EINVAL and a message in usfft_last_error(NULL).  CUDA loads modules lazily
 * by default, so a device first holds the array when the first call on it sets it up, and keeps
 * it until the process exits: a caller that reserves nearly all of HBM for its own pool should
 * make its first call on each device (count = 0 is enough: the set-up runs before that early
 * return) before reserving the pool.  The first call on a device looks up the array's device
 * address (cudaGetSymbolAddress) with that device current; make it before any stream capture.
 * All calls share the array and it keeps the last call's contents (the counter is cleared by
 * every call): calls whose work overlaps on the GPU (other streams, or other host threads) race
 * and corrupt each other's results; serialise them. */
usfft_status usfft_sample_2d_static(const usfft_problem* problem, const int64_t* z, const double* tails,
                                    int64_t M, int64_t i0, int64_t count, double tol, int max_iters,
                                    double* U, void* stream, uint32_t* unconverged);

#ifdef __cplusplus
}
#endif
#endif /* USFFT_H */
