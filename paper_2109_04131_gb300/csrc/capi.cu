// C ABI of the library: plans, increments (Algorithm 1, steps 1, 2a and 2), replay, rewind
// and inspection.  Host work here is planning and marshalling only (candidate sets, the
// lattice search, the counter-based draws of the tails, gather buckets); every numeric
// step of the path runs in the kernels of k_*.cu.
#include <cuda_runtime.h>
#include <stdint.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <cstdlib>
#include <string>
#include <thread>
#include <vector>

#include "usfft.h"
#include "usfft_internal.h"

using namespace usfft;

namespace usfft {
// k_shard.cu
cudaError_t launch_shard_twist(double2* C, int G, int64_t nJ, const int* mk, int64_t p, int64_t M, double scale,
                               cudaStream_t s, int* launches);
cudaError_t launch_bits_to_bytes(const uint32_t* bits, int64_t n, uint8_t* bytes, cudaStream_t s, int* launches);
cudaError_t launch_bytes_to_bits(const uint8_t* bytes, int64_t n, uint32_t* bits, cudaStream_t s, int* launches);
}  // namespace usfft

namespace {

struct Buf {
    void* p = nullptr;
    size_t bytes = 0;
};

struct Snapshot {
    int t = 0;
    std::vector<int8_t> Ipre;
    int64_t nIpre = 0;
    std::vector<std::vector<int>> I1d;
    double theta = 0.0, A = 0.0;
    bool theta_set = false;
};

thread_local std::string g_last_error;

}  // namespace

void usfft::set_thread_error(const std::string& msg) { g_last_error = msg; }

struct usfft_plan_s {
    usfft_problem prob;
    usfft_params par;
    std::vector<int8_t> tp_freqs;
    std::vector<double> tp_coefs;
    cudaStream_t stream = nullptr;
    int G = 0, E = 0, d = 0, N = 0, K = 0;
    int t = 0;
    double theta = 0.0, A = 0.0;
    bool theta_set = false;
    std::vector<std::vector<int>> I1d;
    std::vector<int8_t> Ipre;
    int64_t nIpre = 0;
    std::vector<Snapshot> hist;
    // last detection step (coupled, or the 1-D detection of t = 1)
    bool last_coupled = false;
    int last_t = 0;
    std::vector<int8_t> J;
    int64_t nJ = 0;
    std::vector<int64_t> z;
    int64_t M = 0;
    std::vector<int64_t> m;
    int s_tilde = 0;
    std::vector<NodeSpec> specs;
    FftPlan fp{};
    // device buffers
    Buf psi, U, C, bitmap, twid, goff, gk, gm2, fftscr, cgscr, iters, failc, scal, tpf, tpc, tpaux;
    Buf fpos, fmk;            // single in-place FFT pass: digit-reversed positions, candidates' m_k
    bool inplace = false;
    // step 3 result (usfft_reconstruct) and the buffers of point evaluation
    Buf Crec, Irec, Ypts, Upts, Vpts, epart, etot;
    int64_t nrec = -1;     // |I| of the stored reconstruction, -1: none
    std::vector<int8_t> Irec_h;
    // random rank-1 lattice detection of the last coupled step (params.rr_lattices > 0):
    // lattice q = i*L + l of iteration i, its FFT plan and its slices of the gather/twiddle buffers
    // (also step 3 on multiple rank-1 lattices, usfft_reconstruct_multiple: one iteration, every
    // estimate from its first alias-free lattice, rr_pick_only)
    bool rr_active = false, rr_pick_only = false;
    int rr_L = 0, rr_iters = 0;
    std::vector<int64_t> rr_M, rr_z;
    std::vector<FftPlan> rr_fp;
    std::vector<size_t> rr_goff_at, rr_gk_at, rr_twid_at;
    Buf rr_goff, rr_gk, rr_gm2, rr_src, rr_twid, rr_C;
    std::atomic<size_t> bytes{0};   // read by usfft_plan_bytes from other threads
    int cg_blocks = 0;
    int launches = 0;
    int64_t cg_iters_total = 0;
    int cg_iters_max = 0;
    int64_t h2d = 0, d2h = 0;
    bool replay_valid = false;
    // per-iteration copies of the last single-lattice detection step (usfft_set_keep_iterations):
    // samples, coefficients and the union bitmap after iteration i (cumulative over 1..i)
    bool keep_iters = false;
    int kept = 0;
    // sharded form (usfft_increment_sharded): this rank's share of the last coupled step
    bool step_sharded = false;                // the last detection step ran sharded
    int shard_rank = 0, shard_n = 1;
    usfft_allreduce_fn shard_fn = nullptr;
    void* shard_ctx = nullptr;
    int64_t shard_M = 0;                      // full lattice size (plan->M is the rank's M / P)
    std::vector<int64_t> shard_m;             // full DFT indices k.z mod M (plan->m: mod M / P)
    Buf smk, sflags;                          // the full indices (int32) and the union flags (bytes)
    std::vector<Buf> kU, kC, kB;
    // stage timing (usfft_set_timing): event pairs per stage launch
    bool timing = false;
    std::vector<std::pair<int, std::pair<cudaEvent_t, cudaEvent_t>>> tev;
    std::vector<cudaEvent_t> ev_pool;
    size_t ev_used = 0;
    double* pinned = nullptr;   // small pinned staging area
    cudaEvent_t ev0 = nullptr, ev1 = nullptr, evs = nullptr;
    std::string err;
};

namespace {

usfft_status fail(usfft_plan_t* p, usfft_status st, const std::string& msg) {
    if (p) p->err = msg;
    g_last_error = msg;
    return st;
}

#define CK(call)                                                                                     \
    do {                                                                                             \
        cudaError_t _e = (call);                                                                     \
        if (_e != cudaSuccess)                                                                       \
            return fail(plan, USFFT_ECUDA, std::string(#call) + ": " + cudaGetErrorString(_e));     \
    } while (0)

void buf_free(usfft_plan_t* plan, Buf& b) {
    if (!b.p) return;
    if (plan->par.alloc && plan->par.free)
        plan->par.free(b.p, plan->stream, plan->par.alloc_ctx);
    else
        cudaFree(b.p);
    plan->bytes -= b.bytes;
    b.p = nullptr;
    b.bytes = 0;
}

usfft_status ensure(usfft_plan_t* plan, Buf& b, size_t bytes, const char* what) {
    if (bytes == 0) bytes = 16;
    if (b.bytes >= bytes) return USFFT_OK;
    size_t want = bytes + bytes / 8;
    size_t after = plan->bytes - b.bytes + want;
    if (plan->par.hbm_budget_bytes && after > plan->par.hbm_budget_bytes) {
        want = bytes;
        after = plan->bytes - b.bytes + want;
        if (after > plan->par.hbm_budget_bytes) {
            char msg[256];
            snprintf(msg, sizeof msg, "%s: %zu bytes would exceed the budget of %zu bytes (plan holds %zu)", what,
                     bytes, plan->par.hbm_budget_bytes, plan->bytes.load());
            return fail(plan, USFFT_ENOMEM, msg);
        }
    }
    buf_free(plan, b);
    void* p = nullptr;
    if (plan->par.alloc) {
        p = plan->par.alloc(want, plan->stream, plan->par.alloc_ctx);
    } else if (cudaMalloc(&p, want) != cudaSuccess) {
        cudaGetLastError();
        p = nullptr;
    }
    if (!p) {
        char msg[256];
        snprintf(msg, sizeof msg, "%s: device allocation of %zu bytes failed", what, want);
        return fail(plan, USFFT_ENOMEM, msg);
    }
    b.p = p;
    b.bytes = want;
    plan->bytes += want;
    return USFFT_OK;
}

double timeout_seconds() {
    const char* e = getenv("USFFT_TIMEOUT_S");
    double v = e ? atof(e) : 0.0;
    return v > 0 ? v : 3600.0;
}

// Wait for the plan's stream with a host-side deadline (never a device-side trap).
usfft_status wait_stream(usfft_plan_t* plan) {
    cudaError_t e = cudaEventRecord(plan->evs, plan->stream);
    if (e != cudaSuccess) return fail(plan, USFFT_ECUDA, std::string("cudaEventRecord: ") + cudaGetErrorString(e));
    auto t0 = std::chrono::steady_clock::now();
    const double limit = timeout_seconds();
    int spins = 0;
    for (;;) {
        e = cudaEventQuery(plan->evs);
        if (e == cudaSuccess) return USFFT_OK;
        if (e != cudaErrorNotReady)
            return fail(plan, USFFT_ECUDA, std::string("device error: ") + cudaGetErrorString(e));
        double el = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
        if (el > limit) return fail(plan, USFFT_ETIMEOUT, "device work did not finish before the host deadline");
        if (++spins > 64) std::this_thread::sleep_for(std::chrono::microseconds(50));
    }
}

void set_map(NodeSpec& ns, const usfft_problem& pr) {
    ns.map = pr.kind == USFFT_TRIGPOLY ? USFFT_MAP_PERIODIC : pr.theta_map;
    ns.map_alpha = pr.map_alpha;
    ns.map_beta = pr.map_beta;
    ns.map_shift = pr.map_shift;
}

ParamMap param_map(const usfft_problem& pr) {
    ParamMap pm;
    pm.map = pr.kind == USFFT_TRIGPOLY ? USFFT_MAP_PERIODIC : pr.theta_map;
    pm.alpha = pr.map_alpha;
    pm.beta = pr.map_beta;
    pm.shift = pr.map_shift;
    return pm;
}

// tau_{2,Delta} of the lognormal map, evaluated as the kernels do (k_theta.cuh)
double tau2_host(double yt, double shift) {
    const double u = yt - shift;
    return yt < shift ? -0.5 - 2.0 * u : (yt < 0.5 + shift ? -0.5 + 2.0 * u : 1.5 - 2.0 * u);
}

// Lognormal map: true if a node i/M of a lattice of size M (as the kernels compute it) lands on
// a pole of tau_1 (tau_{2,Delta} = -1/2 or +1/2), i.e. at y~ = Delta or 1/2 + Delta.
bool lattice_hits_pole(int64_t M, double shift) {
    const double cands[2] = {shift, 0.5 + shift};
    for (double c : cands) {
        const int64_t base = (int64_t)floor(c * (double)M);
        for (int64_t nn = base - 1; nn <= base + 2; ++nn) {
            if (nn < 0 || nn >= M) continue;
            if (fabs(tau2_host((double)nn / (double)M, shift)) >= 0.5) return true;
        }
    }
    return false;
}

NodeSpec spec_1d(const usfft_plan_t* p, int t, int i) {
    NodeSpec ns;
    memset(&ns, 0, sizeof ns);
    ns.M = p->K;
    ns.d = p->d;
    set_map(ns, p->prob);
    for (int j = 1; j <= p->d; ++j) {
        if (j == t) {
            ns.z[j - 1] = 1;
        } else {
            ns.z[j - 1] = -1;
            uint64_t f[4] = {PHASE_1D_TAIL, (uint64_t)t, (uint64_t)i, (uint64_t)j};
            ns.tail[j - 1] = rng_uniform(p->par.seed, f, 4);
        }
    }
    return ns;
}

NodeSpec spec_coupled(const usfft_plan_t* p, int t, int i) {
    NodeSpec ns;
    memset(&ns, 0, sizeof ns);
    ns.M = p->M;
    ns.d = p->d;
    set_map(ns, p->prob);
    for (int j = 1; j <= p->d; ++j) {
        if (j <= t) {
            ns.z[j - 1] = p->z[(size_t)(j - 1)];
        } else {
            ns.z[j - 1] = -1;
            uint64_t f[4] = {PHASE_TAIL, (uint64_t)t, (uint64_t)i, (uint64_t)j};
            ns.tail[j - 1] = rng_uniform(p->par.seed, f, 4);
        }
    }
    return ns;
}

cudaEvent_t pool_event(usfft_plan_t* plan) {
    if (plan->ev_used == plan->ev_pool.size()) {
        cudaEvent_t e;
        if (cudaEventCreate(&e) != cudaSuccess) {
            cudaGetLastError();
            return nullptr;
        }
        plan->ev_pool.push_back(e);
    }
    return plan->ev_pool[plan->ev_used++];
}

// Records an event pair around one stage launch when timing is on.
struct StageTimer {
    usfft_plan_t* plan;
    int stage;
    cudaEvent_t a = nullptr, b = nullptr;
    StageTimer(usfft_plan_t* p, int st) : plan(p), stage(st) {
        if (!plan->timing) return;
        a = pool_event(plan);
        b = pool_event(plan);
        if (a && b) cudaEventRecord(a, plan->stream);
    }
    ~StageTimer() {
        if (!plan->timing || !a || !b) return;
        cudaEventRecord(b, plan->stream);
        plan->tev.push_back({stage, {a, b}});
    }
};

// the MIXED precision mode runs the lattice FFT in double-float arithmetic (16 bytes per complex
// value either way, so the twiddle and scratch buffers serve both)
bool fft_df(const usfft_plan_t* plan) { return plan->par.precision == USFFT_MIXED; }

// sampler dispatch: out[0..M)[G] for the node set (out = the plan's sample buffer by default)
usfft_status run_sampler(usfft_plan_t* plan, const NodeSpec& ns, double* out = nullptr) {
    const int kind = plan->prob.kind;
    double* U = out ? out : (double*)plan->U.p;
    StageTimer timer(plan, USFFT_STAGE_SAMPLE);
    const int64_t count = node_count(ns);
    if (kind == USFFT_PDE_1D) {
        CK(launch_sample_1d(ns, plan->prob.n, plan->prob.coef_model, plan->prob.f_const, (const double*)plan->psi.p,
                            0, count, U, plan->stream, &plan->launches));
    } else if (kind == USFFT_PDE_2D) {
        CgConfig cg;
        cg.precision = plan->par.precision;
        cg.max_iters = plan->par.max_cg_iters;
        cg.tol = plan->par.cg_tol;
        cg.blocks = plan->cg_blocks;
        cg.coef_scale = plan->prob.coef_scale;
        cg.coef_decay = plan->prob.coef_decay;
        CK(launch_sample_2d(ns, plan->prob.n, plan->prob.coef_model, plan->prob.f_const, (const double*)plan->psi.p, cg,
                            0, count, U, (int*)plan->iters.p, (unsigned int*)plan->failc.p,
                            (unsigned long long*)((char*)plan->failc.p + 8), (double*)plan->cgscr.p,
                            plan->cgscr.bytes, plan->stream, &plan->launches));
    } else {
        CK(launch_sample_trigpoly(ns, plan->G, plan->prob.tp_nterms, (const int8_t*)plan->tpf.p,
                                  (const double*)plan->tpc.p, (double*)plan->tpaux.p, U,
                                  plan->stream, &plan->launches));
    }
    return USFFT_OK;
}

// buffers and gather plan for a detection step with nJ candidates at indices m, lattice size M
usfft_status prepare_step(usfft_plan_t* plan, int64_t M, const std::vector<int64_t>& m, bool check_poles = true) {
    const int64_t nJ = (int64_t)m.size();
    usfft_status st;
    plan->step_sharded = false;
    plan->shard_M = 0;
    if (check_poles && plan->prob.kind != USFFT_TRIGPOLY && plan->prob.theta_map == USFFT_MAP_NORMAL &&
        lattice_hits_pole(M, plan->prob.map_shift)) {
        char msg[200];
        snprintf(msg, sizeof msg, "a node of the lattice of size %lld lies on a pole of the lognormal map "
                 "(Delta = %.17g): choose another map_shift", (long long)M, plan->prob.map_shift);
        return fail(plan, USFFT_EINVAL, msg);
    }
    plan->fp = make_fft_plan(M);
    if (plan->fp.L2 <= 0) return fail(plan, USFFT_EINVAL, "lattice size has no factorisation into FFT passes <= 4096");
    const int G = plan->G;
    if ((st = ensure(plan, plan->U, sizeof(double) * (size_t)M * G, "samples")) != USFFT_OK) return st;
    if ((st = ensure(plan, plan->C, sizeof(double2) * (size_t)nJ * G, "coefficients")) != USFFT_OK) return st;
    if ((st = ensure(plan, plan->twid, sizeof(double2) * (size_t)M, "twiddles")) != USFFT_OK) return st;
    if ((st = ensure(plan, plan->fftscr, fft_scratch_bytes(plan->fp, G), "fft scratch")) != USFFT_OK) return st;
    if ((st = ensure(plan, plan->bitmap, sizeof(uint32_t) * (size_t)((nJ + 31) / 32), "bitmap")) != USFFT_OK) return st;
    if ((st = ensure(plan, plan->iters, sizeof(int) * (size_t)M, "cg iterations")) != USFFT_OK) return st;
    const int L1 = plan->fp.L1;
    std::vector<int> off((size_t)L1 + 1, 0), bk((size_t)nJ), bm2((size_t)nJ);
    for (int64_t k = 0; k < nJ; ++k) off[(size_t)(m[(size_t)k] % L1) + 1]++;
    for (int b = 0; b < L1; ++b) off[(size_t)b + 1] += off[(size_t)b];
    std::vector<int> fill(off.begin(), off.end() - 1);
    for (int64_t k = 0; k < nJ; ++k) {
        const int b = (int)(m[(size_t)k] % L1);
        const int e = fill[(size_t)b]++;
        bk[(size_t)e] = (int)k;
        bm2[(size_t)e] = (int)(m[(size_t)k] / L1);
    }
    // the single in-place FFT pass when the lattice fits on chip
    const std::vector<int> pos = fft_inplace_positions(M);
    plan->inplace = !pos.empty();
    std::vector<int> mk32;
    if (plan->inplace) {
        mk32.resize((size_t)std::max<int64_t>(nJ, 1));
        for (int64_t k = 0; k < nJ; ++k) mk32[(size_t)k] = (int)m[(size_t)k];
        if ((st = ensure(plan, plan->fpos, sizeof(int) * pos.size(), "fft positions")) != USFFT_OK) return st;
        if ((st = ensure(plan, plan->fmk, sizeof(int) * mk32.size(), "candidate indices")) != USFFT_OK) return st;
        CK(cudaMemcpyAsync(plan->fpos.p, pos.data(), sizeof(int) * pos.size(), cudaMemcpyHostToDevice, plan->stream));
        CK(cudaMemcpyAsync(plan->fmk.p, mk32.data(), sizeof(int) * mk32.size(), cudaMemcpyHostToDevice, plan->stream));
        plan->h2d += (int64_t)(sizeof(int) * (pos.size() + mk32.size()));
    }
    if ((st = ensure(plan, plan->goff, sizeof(int) * off.size(), "gather offsets")) != USFFT_OK) return st;
    if ((st = ensure(plan, plan->gk, sizeof(int) * (size_t)std::max<int64_t>(nJ, 1), "gather k")) != USFFT_OK) return st;
    if ((st = ensure(plan, plan->gm2, sizeof(int) * (size_t)std::max<int64_t>(nJ, 1), "gather m2")) != USFFT_OK) return st;
    CK(cudaMemcpyAsync(plan->goff.p, off.data(), sizeof(int) * off.size(), cudaMemcpyHostToDevice, plan->stream));
    plan->h2d += (int64_t)(sizeof(int) * off.size());
    if (nJ) {
        CK(cudaMemcpyAsync(plan->gk.p, bk.data(), sizeof(int) * (size_t)nJ, cudaMemcpyHostToDevice, plan->stream));
        CK(cudaMemcpyAsync(plan->gm2.p, bm2.data(), sizeof(int) * (size_t)nJ, cudaMemcpyHostToDevice, plan->stream));
        plan->h2d += (int64_t)(2 * sizeof(int) * (size_t)nJ);
    }
    // host vectors must outlive the asynchronous copies
    CK(cudaStreamSynchronize(plan->stream));
    CK(launch_twiddles(M, plan->twid.p, fft_df(plan), plan->stream, &plan->launches));
    plan->M = M;
    plan->m = m;
    plan->nJ = nJ;
    return USFFT_OK;
}

// buffers, gather plans, twiddles and estimate sources of a step on several lattices: rt
// iterations of L lattices each over the nJ candidates J (t columns); lattice l of iteration i is
// zall[((i-1) L + l) t ...] with size Mall[(i-1) L + l].  The estimate of candidate k in iteration i
// comes from the first of its lattices in which no other candidate shares k's index.
usfft_status prepare_lattice_set(usfft_plan_t* plan, const std::vector<int8_t>& J, int64_t nJ, int t, int rt, int L,
                                 const std::vector<int64_t>& zall, const std::vector<int64_t>& Mall) {
    const int G = plan->G;
    plan->rr_L = L;
    plan->rr_iters = rt;
    plan->rr_M.clear();
    plan->rr_z.clear();
    plan->rr_fp.clear();
    plan->rr_goff_at.clear();
    plan->rr_gk_at.clear();
    plan->rr_twid_at.clear();
    std::vector<int> goff_h, gk_h, gm2_h, src_h((size_t)rt * nJ, -1);
    size_t twid_total = 0, scr_max = 0;
    int64_t Mmax = 0;
    std::vector<int64_t> m((size_t)nJ), sorted;
    for (int i = 1; i <= rt; ++i) {
        const int64_t* zi = zall.data() + (size_t)(i - 1) * L * t;
        const int64_t* Mi = Mall.data() + (size_t)(i - 1) * L;
        for (int l = 0; l < L; ++l) {
            const int64_t M = Mi[(size_t)l];
            if (M > (int64_t)1 << 24) return fail(plan, USFFT_EINVAL, "lattice larger than 4096^2");
            if (plan->prob.kind != USFFT_TRIGPOLY && plan->prob.theta_map == USFFT_MAP_NORMAL &&
                lattice_hits_pole(M, plan->prob.map_shift))
                return fail(plan, USFFT_EINVAL, "a lattice node lies on a pole of the lognormal map");
            const FftPlan fp = make_fft_plan(M);
            if (fp.L2 <= 0) return fail(plan, USFFT_EINVAL, "lattice size has no FFT factorisation");
            for (int64_t a = 0; a < nJ; ++a) {
                int64_t acc = 0;
                for (int j = 0; j < t; ++j) acc += (int64_t)J[(size_t)(a * t + j)] * zi[(size_t)(l * t + j)];
                const int64_t mm = acc % M;
                m[(size_t)a] = mm < 0 ? mm + M : mm;
            }
            // candidates alone at their index in this lattice
            sorted = m;
            std::sort(sorted.begin(), sorted.end());
            int* src_i = src_h.data() + (size_t)(i - 1) * nJ;
            for (int64_t a = 0; a < nJ; ++a) {
                if (src_i[a] >= 0) continue;
                auto range = std::equal_range(sorted.begin(), sorted.end(), m[(size_t)a]);
                if (range.second - range.first == 1) src_i[a] = l;
            }
            // gather buckets by m mod L1 (as in prepare_step)
            const int L1 = fp.L1;
            plan->rr_goff_at.push_back(goff_h.size());
            plan->rr_gk_at.push_back(gk_h.size());
            const size_t o0 = goff_h.size(), k0 = gk_h.size();
            goff_h.resize(o0 + L1 + 1, 0);
            gk_h.resize(k0 + nJ);
            gm2_h.resize(k0 + nJ);
            int* off = goff_h.data() + o0;
            for (int64_t a = 0; a < nJ; ++a) off[(size_t)(m[(size_t)a] % L1) + 1]++;
            for (int b = 0; b < L1; ++b) off[b + 1] += off[b];
            std::vector<int> fill(off, off + L1);
            for (int64_t a = 0; a < nJ; ++a) {
                const int b = (int)(m[(size_t)a] % L1);
                const int e = fill[(size_t)b]++;
                gk_h[k0 + e] = (int)a;
                gm2_h[k0 + e] = (int)(m[(size_t)a] / L1);
            }
            plan->rr_twid_at.push_back(twid_total);
            twid_total += (size_t)M;
            scr_max = std::max(scr_max, fft_scratch_bytes(fp, G));
            Mmax = std::max(Mmax, M);
            plan->rr_M.push_back(M);
            plan->rr_z.insert(plan->rr_z.end(), zi + (size_t)l * t, zi + (size_t)(l + 1) * t);
            plan->rr_fp.push_back(fp);
        }
    }
    usfft_status st;
    if ((st = ensure(plan, plan->U, sizeof(double) * (size_t)Mmax * G, "samples")) != USFFT_OK) return st;
    if ((st = ensure(plan, plan->C, sizeof(double2) * (size_t)nJ * G, "coefficients")) != USFFT_OK) return st;
    if ((st = ensure(plan, plan->rr_C, sizeof(double2) * (size_t)L * nJ * G, "lattice coefficients")) != USFFT_OK)
        return st;
    if ((st = ensure(plan, plan->rr_twid, sizeof(double2) * twid_total, "twiddles")) != USFFT_OK) return st;
    if ((st = ensure(plan, plan->fftscr, scr_max, "fft scratch")) != USFFT_OK) return st;
    if ((st = ensure(plan, plan->bitmap, sizeof(uint32_t) * (size_t)((nJ + 31) / 32), "bitmap")) != USFFT_OK) return st;
    if ((st = ensure(plan, plan->iters, sizeof(int) * (size_t)Mmax, "cg iterations")) != USFFT_OK) return st;
    if ((st = ensure(plan, plan->rr_goff, sizeof(int) * goff_h.size(), "gather offsets")) != USFFT_OK) return st;
    if ((st = ensure(plan, plan->rr_gk, sizeof(int) * gk_h.size(), "gather k")) != USFFT_OK) return st;
    if ((st = ensure(plan, plan->rr_gm2, sizeof(int) * gm2_h.size(), "gather m2")) != USFFT_OK) return st;
    if ((st = ensure(plan, plan->rr_src, sizeof(int) * src_h.size(), "estimate sources")) != USFFT_OK) return st;
    CK(cudaMemcpyAsync(plan->rr_goff.p, goff_h.data(), sizeof(int) * goff_h.size(), cudaMemcpyHostToDevice, plan->stream));
    CK(cudaMemcpyAsync(plan->rr_gk.p, gk_h.data(), sizeof(int) * gk_h.size(), cudaMemcpyHostToDevice, plan->stream));
    CK(cudaMemcpyAsync(plan->rr_gm2.p, gm2_h.data(), sizeof(int) * gm2_h.size(), cudaMemcpyHostToDevice, plan->stream));
    CK(cudaMemcpyAsync(plan->rr_src.p, src_h.data(), sizeof(int) * src_h.size(), cudaMemcpyHostToDevice, plan->stream));
    plan->h2d += (int64_t)(sizeof(int) * (goff_h.size() + gk_h.size() + gm2_h.size() + src_h.size()));
    CK(cudaStreamSynchronize(plan->stream));   // host vectors outlive the copies
    for (size_t q = 0; q < plan->rr_M.size(); ++q)
        CK(launch_twiddles(plan->rr_M[q], (double2*)plan->rr_twid.p + plan->rr_twid_at[q], fft_df(plan),
                           plan->stream, &plan->launches));
    // the last lattice stands for the step in the single-lattice inspection calls
    plan->M = plan->rr_M.back();
    plan->z.assign(plan->rr_z.end() - t, plan->rr_z.end());
    plan->m.assign((size_t)nJ, 0);
    for (int64_t a = 0; a < nJ; ++a) {
        int64_t acc = 0;
        for (int j = 0; j < t; ++j) acc += (int64_t)J[(size_t)(a * t + j)] * plan->z[(size_t)j];
        const int64_t mm = acc % plan->M;
        plan->m[(size_t)a] = mm < 0 ? mm + plan->M : mm;
    }
    plan->nJ = nJ;
    return USFFT_OK;
}

// the random rank-1 lattices of params.rr_lattices for the coupled step t (rt iterations)
usfft_status prepare_rr(usfft_plan_t* plan, const std::vector<int8_t>& J, int64_t nJ, int t, int rt, int s_t) {
    const int L = plan->par.rr_lattices;
    const double factor = plan->par.rr_size_factor > 0.0 ? plan->par.rr_size_factor : 2.0;
    std::vector<int64_t> zall, Mall, zi, Mi;
    plan->rr_pick_only = false;
    for (int i = 1; i <= rt; ++i) {
        random_lattices(t, i, plan->nIpre, (int64_t)plan->I1d[(size_t)t].size(), s_t, L, factor, plan->par.seed, zi, Mi);
        zall.insert(zall.end(), zi.begin(), zi.end());
        Mall.insert(Mall.end(), Mi.begin(), Mi.end());
    }
    return prepare_lattice_set(plan, J, nJ, t, rt, L, zall, Mall);
}

// device part of a random-lattice step: per iteration L x (sample -> FFT+gather), the
// estimate (alias-free lattice or median), select/union
usfft_status run_rr_device(usfft_plan_t* plan) {
    const int64_t nJ = plan->nJ;
    const int G = plan->G, L = plan->rr_L;
    CK(cudaMemsetAsync(plan->bitmap.p, 0, sizeof(uint32_t) * (size_t)((nJ + 31) / 32), plan->stream));
    if (nJ == 0) return USFFT_OK;
    for (int i = 0; i < plan->rr_iters; ++i) {
        for (int l = 0; l < L; ++l) {
            const size_t q = (size_t)i * L + l;
            usfft_status st = run_sampler(plan, plan->specs[q]);
            if (st != USFFT_OK) return st;
            StageTimer timer(plan, USFFT_STAGE_FFT);
            GatherPlan gp{(const int*)plan->rr_goff.p + plan->rr_goff_at[q], (const int*)plan->rr_gk.p + plan->rr_gk_at[q],
                          (const int*)plan->rr_gm2.p + plan->rr_gk_at[q]};
            CK(launch_fft_gather(plan->rr_fp[q], G, (const double*)plan->U.p,
                                 (const double2*)plan->rr_twid.p + plan->rr_twid_at[q], fft_df(plan), gp, nJ,
                                 plan->fftscr.p, (double2*)plan->rr_C.p + (size_t)l * G * nJ, plan->stream,
                                 &plan->launches));
        }
        {
            StageTimer timer(plan, USFFT_STAGE_FFT);
            const int* src = (const int*)plan->rr_src.p + (size_t)i * nJ;
            if (plan->rr_pick_only)
                CK(launch_lattice_pick((const double2*)plan->rr_C.p, L, G, nJ, src, (double2*)plan->C.p, plan->stream,
                                       &plan->launches));
            else
                CK(launch_random_lattice_combine((const double2*)plan->rr_C.p, L, G, nJ, src, (double2*)plan->C.p,
                                                 plan->stream, &plan->launches));
        }
        if (plan->s_tilde > 0) {
            StageTimer timer(plan, USFFT_STAGE_SELECT);
            CK(launch_select_union((const double2*)plan->C.p, G, nJ, plan->theta, plan->s_tilde, (uint32_t*)plan->bitmap.p,
                                   plan->stream, &plan->launches));
        }
    }
    return USFFT_OK;
}

// device part of a detection step: r~ iterations of sample -> FFT+gather -> select/union
// copies of iteration it's samples, coefficients and union bitmap (inspection only)
usfft_status keep_iteration(usfft_plan_t* plan, size_t it) {
    const size_t ub = sizeof(double) * (size_t)plan->M * plan->G, cb = sizeof(double2) * (size_t)plan->nJ * plan->G;
    const size_t bb = sizeof(uint32_t) * (size_t)((plan->nJ + 31) / 32);
    if (plan->kU.size() <= it) {
        plan->kU.resize(it + 1);
        plan->kC.resize(it + 1);
        plan->kB.resize(it + 1);
    }
    usfft_status st;
    if ((st = ensure(plan, plan->kU[it], ub, "kept samples")) != USFFT_OK) return st;
    if ((st = ensure(plan, plan->kC[it], cb, "kept coefficients")) != USFFT_OK) return st;
    if ((st = ensure(plan, plan->kB[it], bb, "kept bitmap")) != USFFT_OK) return st;
    CK(cudaMemcpyAsync(plan->kU[it].p, plan->U.p, ub, cudaMemcpyDeviceToDevice, plan->stream));
    CK(cudaMemcpyAsync(plan->kC[it].p, plan->C.p, cb, cudaMemcpyDeviceToDevice, plan->stream));
    CK(cudaMemcpyAsync(plan->kB[it].p, plan->bitmap.p, bb, cudaMemcpyDeviceToDevice, plan->stream));
    plan->kept = (int)it + 1;
    return USFFT_OK;
}

// the caller's all-reduce of the sharded form
usfft_status shard_allreduce(usfft_plan_t* plan, void* buf, size_t count, int dtype, int op) {
    if (count == 0) return USFFT_OK;
    const int rc = plan->shard_fn(buf, count, dtype, op, (void*)plan->stream, plan->shard_ctx);
    if (rc != 0) {
        char msg[160];
        snprintf(msg, sizeof msg, "the collective hook failed (%d) on an all-reduce of %zu elements", rc, count);
        return fail(plan, USFFT_ECOMM, msg);
    }
    return USFFT_OK;
}

// device part of a sharded coupled step on this rank: r~ iterations of (its M/P solves, its
// length-M/P FFT + gather, the twist, sum over ranks, selection at its node block, union of
// the flags over ranks)
usfft_status run_sharded_device(usfft_plan_t* plan) {
    const int64_t nJ = plan->nJ;
    const int G = plan->G, P = plan->shard_n, p = plan->shard_rank;
    CK(cudaMemsetAsync(plan->bitmap.p, 0, sizeof(uint32_t) * (size_t)((nJ + 31) / 32), plan->stream));
    if (nJ == 0) return USFFT_OK;
    GatherPlan gp{(const int*)plan->goff.p, (const int*)plan->gk.p, (const int*)plan->gm2.p};
    if (plan->inplace) {
        gp.pos_of = (const int*)plan->fpos.p;
        gp.mk = (const int*)plan->fmk.p;
    }
    const int g0 = (int)((int64_t)G * p / P), g1 = (int)((int64_t)G * (p + 1) / P);
    for (size_t it = 0; it < plan->specs.size(); ++it) {
        usfft_status st = run_sampler(plan, plan->specs[it]);
        if (st != USFFT_OK) return st;
        {
            StageTimer timer(plan, USFFT_STAGE_FFT);
            CK(launch_fft_gather(plan->fp, G, (const double*)plan->U.p, plan->twid.p, fft_df(plan), gp, nJ,
                                 plan->fftscr.p, (double2*)plan->C.p, plan->stream, &plan->launches));
            CK(launch_shard_twist((double2*)plan->C.p, G, nJ, (const int*)plan->smk.p, p, plan->shard_M,
                                  1.0 / (double)P, plan->stream, &plan->launches));
        }
        if ((st = shard_allreduce(plan, plan->C.p, 2 * (size_t)G * nJ, USFFT_RED_F64, USFFT_RED_SUM)) != USFFT_OK)
            return st;
        if (plan->s_tilde > 0) {
            StageTimer timer(plan, USFFT_STAGE_SELECT);
            if (g1 > g0)
                CK(launch_select_union((const double2*)plan->C.p + (size_t)g0 * nJ, g1 - g0, nJ, plan->theta,
                                       plan->s_tilde, (uint32_t*)plan->bitmap.p, plan->stream, &plan->launches));
            CK(launch_bits_to_bytes((const uint32_t*)plan->bitmap.p, nJ, (uint8_t*)plan->sflags.p, plan->stream,
                                    &plan->launches));
        }
        if (plan->s_tilde > 0) {
            if ((st = shard_allreduce(plan, plan->sflags.p, (size_t)nJ, USFFT_RED_U8, USFFT_RED_MAX)) != USFFT_OK)
                return st;
            CK(launch_bytes_to_bits((const uint8_t*)plan->sflags.p, nJ, (uint32_t*)plan->bitmap.p, plan->stream,
                                    &plan->launches));
        }
        if (plan->keep_iters) {
            usfft_status st2 = keep_iteration(plan, it);
            if (st2 != USFFT_OK) return st2;
        }
    }
    return USFFT_OK;
}

usfft_status run_step_device(usfft_plan_t* plan, bool first_1d_sets_theta) {
    plan->kept = 0;
    if (plan->rr_active) return run_rr_device(plan);
    if (plan->step_sharded) return run_sharded_device(plan);
    const int64_t nJ = plan->nJ;
    CK(cudaMemsetAsync(plan->bitmap.p, 0, sizeof(uint32_t) * (size_t)((nJ + 31) / 32), plan->stream));
    if (nJ == 0) return USFFT_OK;
    GatherPlan gp{(const int*)plan->goff.p, (const int*)plan->gk.p, (const int*)plan->gm2.p};
    if (plan->inplace) {
        gp.pos_of = (const int*)plan->fpos.p;
        gp.mk = (const int*)plan->fmk.p;
    }
    for (size_t it = 0; it < plan->specs.size(); ++it) {
        usfft_status st = run_sampler(plan, plan->specs[it]);
        if (st != USFFT_OK) return st;
        {
            StageTimer timer(plan, USFFT_STAGE_FFT);
            CK(launch_fft_gather(plan->fp, plan->G, (const double*)plan->U.p, plan->twid.p, fft_df(plan), gp, nJ,
                                 plan->fftscr.p, (double2*)plan->C.p, plan->stream, &plan->launches));
        }
        if (first_1d_sets_theta && it == 0 && !plan->theta_set) {
            // relative threshold: theta = delta * max_g |c_{g,0}| of the first 1-D detection
            CK(launch_absmax_column((const double2*)plan->C.p, plan->G, nJ, plan->N, (double*)plan->scal.p,
                                    plan->stream, &plan->launches));
            CK(cudaMemcpyAsync(plan->pinned, plan->scal.p, sizeof(double), cudaMemcpyDeviceToHost, plan->stream));
            plan->d2h += (int64_t)sizeof(double);
            usfft_status w = wait_stream(plan);
            if (w != USFFT_OK) return w;
            plan->A = plan->pinned[0];
            plan->theta = plan->par.delta * plan->A;
            plan->theta_set = true;
        }
        if (plan->s_tilde > 0) {
            StageTimer timer(plan, USFFT_STAGE_SELECT);
            CK(launch_select_union((const double2*)plan->C.p, plan->G, nJ, plan->theta, plan->s_tilde,
                                   (uint32_t*)plan->bitmap.p, plan->stream, &plan->launches));
        }
        if (plan->keep_iters) {
            usfft_status st2 = keep_iteration(plan, it);
            if (st2 != USFFT_OK) return st2;
        }
    }
    return USFFT_OK;
}

usfft_status read_bitmap(usfft_plan_t* plan, std::vector<uint32_t>& bits) {
    const size_t words = (size_t)((plan->nJ + 31) / 32);
    bits.assign(words, 0u);
    if (words) CK(cudaMemcpyAsync(bits.data(), plan->bitmap.p, 4 * words, cudaMemcpyDeviceToHost, plan->stream));
    plan->d2h += (int64_t)(4 * words);
    return wait_stream(plan);
}

usfft_status read_cg_stats(usfft_plan_t* plan, int64_t count) {
    if (plan->prob.kind != USFFT_PDE_2D || count <= 0) return USFFT_OK;
    std::vector<int> it((size_t)count);
    unsigned int fails = 0;
    CK(cudaMemcpyAsync(it.data(), plan->iters.p, sizeof(int) * (size_t)count, cudaMemcpyDeviceToHost, plan->stream));
    CK(cudaMemcpyAsync(&fails, plan->failc.p, sizeof(unsigned), cudaMemcpyDeviceToHost, plan->stream));
    plan->d2h += (int64_t)(sizeof(int) * (size_t)count + sizeof(unsigned));
    usfft_status st = wait_stream(plan);
    if (st != USFFT_OK) return st;
    for (int v : it) {
        plan->cg_iters_total += v;
        plan->cg_iters_max = std::max(plan->cg_iters_max, v);
    }
    if (fails) {
        char msg[160];
        snprintf(msg, sizeof msg, "%u FE solves did not reach the CG tolerance within max_cg_iters", fails);
        return fail(plan, USFFT_ENOCONV, msg);
    }
    return USFFT_OK;
}

void take_snapshot(usfft_plan_t* p) {
    Snapshot s;
    s.t = p->t;
    s.Ipre = p->Ipre;
    s.nIpre = p->nIpre;
    s.I1d = p->I1d;
    s.theta = p->theta;
    s.A = p->A;
    s.theta_set = p->theta_set;
    if ((int)p->hist.size() > p->t) p->hist.resize((size_t)p->t);
    p->hist.push_back(s);
}

}  // namespace

extern "C" {

#define USFFT_STR2(x) #x
#define USFFT_STR(x) USFFT_STR2(x)
const char* usfft_version(void) { return "usfft sm_103a cudart " USFFT_STR(CUDART_VERSION); }

const char* usfft_last_error(const usfft_plan_t* plan) {
    if (plan) return plan->err.c_str();
    return g_last_error.c_str();
}

usfft_status usfft_plan(const usfft_problem* problem, const usfft_params* params, void* stream, usfft_plan_t** out) {
    usfft_plan_t* plan = nullptr;
    if (!out) return fail(nullptr, USFFT_EINVAL, "out is NULL");
    *out = nullptr;
    if (!problem || !params) return fail(nullptr, USFFT_EINVAL, "problem or params is NULL");
    const usfft_problem& pr = *problem;
    const usfft_params& pa = *params;
    if (pr.d < 1 || pr.d > USFFT_MAX_D) return fail(nullptr, USFFT_EINVAL, "d must lie in [1, 64]");
    if (pa.N < 1 || pa.N > 127) return fail(nullptr, USFFT_EINVAL, "N must lie in [1, 127] (int8 frequencies)");
    if (pa.r < 1 || pa.s < 0 || pa.s_local < 0) return fail(nullptr, USFFT_EINVAL, "r >= 1, s >= 0, s_local >= 0");
    if (!(pa.delta >= 0.0)) return fail(nullptr, USFFT_EINVAL, "delta must be >= 0");
    if (pa.precision != USFFT_FP64 && pa.precision != USFFT_MIXED && pa.precision != USFFT_MIXED_JACOBI &&
        pa.precision != USFFT_FP64_DST)
        return fail(nullptr, USFFT_EINVAL, "precision");
    if (pa.rr_lattices < 0 || pa.rr_lattices > 31 || (pa.rr_lattices > 0 && pa.rr_lattices % 2 == 0))
        return fail(nullptr, USFFT_EINVAL, "rr_lattices must be 0 or odd in [1, 31]");
    if (pa.rr_size_factor < 0.0 || !(pa.rr_size_factor < 1e6))
        return fail(nullptr, USFFT_EINVAL, "rr_size_factor must lie in [0, 1e6)");
    int G = 0, E = 0;
    if (pr.kind == USFFT_PDE_1D) {
        if (pr.n < 1 || pr.n > 1023) return fail(nullptr, USFFT_EINVAL, "1-D: n must lie in [1, 1023]");
        G = pr.n;
        E = pr.n + 1;
    } else if (pr.kind == USFFT_PDE_2D) {
        if (pr.n < 1 || pr.n > 127) return fail(nullptr, USFFT_EINVAL, "2-D: n must lie in [1, 127]");
        if (pr.n > 63 && pa.precision != USFFT_MIXED && pa.precision != USFFT_FP64_DST)
            return fail(nullptr, USFFT_EINVAL, "2-D: n > 63 runs in the MIXED and FP64_DST precision modes only");
        if (pr.n > 63 && pa.precision == USFFT_MIXED && big_smem_bytes(pr.n, pr.d) > 232448)
            return fail(nullptr, USFFT_EINVAL, "2-D: d too large for the shared-memory tables at n > 63");
        if (pa.precision == USFFT_MIXED_JACOBI && pr.n < 4) return fail(nullptr, USFFT_EINVAL, "2-D mixed: n >= 4");
        G = pr.n * pr.n;
        E = 2 * (pr.n + 1) * (pr.n + 1);
    } else if (pr.kind == USFFT_TRIGPOLY) {
        if (pr.tp_nodes < 1 || pr.tp_nterms < 1 || !pr.tp_freqs || !pr.tp_coefs)
            return fail(nullptr, USFFT_EINVAL, "TRIGPOLY: tp_nodes, tp_nterms, tp_freqs, tp_coefs required");
        G = pr.tp_nodes;
    } else {
        return fail(nullptr, USFFT_EINVAL, "unknown problem kind");
    }
    if (pr.kind != USFFT_TRIGPOLY) {
        if (pr.coef_model != USFFT_COEF_AFFINE_SIN && pr.coef_model != USFFT_COEF_LOGNORMAL_SIN)
            return fail(nullptr, USFFT_EINVAL, "unknown coefficient model");
        if (pr.theta_map == USFFT_MAP_TENT) {
            if (!(pr.map_alpha < pr.map_beta)) return fail(nullptr, USFFT_EINVAL, "tent map: need alpha < beta");
        } else if (pr.theta_map == USFFT_MAP_NORMAL) {
            if (!(pr.map_shift > 0.0 && pr.map_shift < 0.5))
                return fail(nullptr, USFFT_EINVAL, "lognormal map: need 0 < map_shift < 1/2");
            if (pr.coef_model == USFFT_COEF_AFFINE_SIN)
                return fail(nullptr, USFFT_EINVAL, "lognormal map: Theta_j is unbounded, use the lognormal coefficient");
        } else if (pr.theta_map != USFFT_MAP_PERIODIC) {
            return fail(nullptr, USFFT_EINVAL, "unknown parameter map");
        }
        // uniform ellipticity (Eq. (2.1)) of the affine model: 1 - c max|Theta| sum_j j^-mu > 0
        if (pr.coef_model == USFFT_COEF_AFFINE_SIN) {
            double sum = 0.0;
            for (int j = 1; j <= pr.d; ++j) sum += pow((double)j, -pr.coef_decay);
            const double tmax = pr.theta_map == USFFT_MAP_TENT ? fmax(fabs(pr.map_alpha), fabs(pr.map_beta)) : 1.0;
            if (1.0 - fabs(pr.coef_scale) * tmax * sum <= 0.0)
                return fail(nullptr, USFFT_EINVAL, "coefficient violates uniform ellipticity: a_min <= 0");
        }
    } else if (pr.theta_map != USFFT_MAP_PERIODIC) {
        return fail(nullptr, USFFT_EINVAL, "TRIGPOLY: the test polynomials are periodic (theta_map 0)");
    }
    plan = new usfft_plan_s();
    plan->prob = pr;
    plan->par = pa;
    if (plan->par.max_cg_iters <= 0) plan->par.max_cg_iters = 4000;
    if (plan->par.max_lattice_trials <= 0) plan->par.max_lattice_trials = 64;
    if (plan->par.max_lattice_sizes <= 0) plan->par.max_lattice_sizes = 400;
    if (!(plan->par.cg_tol > 0.0)) plan->par.cg_tol = 1e-13;
    plan->stream = (cudaStream_t)stream;
    plan->G = G;
    plan->E = E;
    plan->d = pr.d;
    plan->N = pa.N;
    plan->K = 2 * pa.N + 1;
    plan->I1d.assign((size_t)pr.d + 1, std::vector<int>());
    if (!pa.delta_is_relative) {
        plan->theta = pa.delta;
        plan->theta_set = true;
    }
    usfft_status st;
    auto bail = [&](usfft_status s) {
        usfft_destroy(plan);
        return s;
    };
    if (cudaEventCreate(&plan->ev0) != cudaSuccess || cudaEventCreate(&plan->ev1) != cudaSuccess ||
        cudaEventCreateWithFlags(&plan->evs, cudaEventDisableTiming) != cudaSuccess) {
        cudaGetLastError();
        fail(plan, USFFT_ECUDA, "cudaEventCreate failed");
        return bail(USFFT_ECUDA);
    }
    if (cudaMallocHost(&plan->pinned, 64) != cudaSuccess) {
        cudaGetLastError();
        fail(plan, USFFT_ECUDA, "cudaMallocHost failed");
        return bail(USFFT_ECUDA);
    }
    if ((st = ensure(plan, plan->scal, 64, "scalars")) != USFFT_OK) return bail(st);
    if ((st = ensure(plan, plan->failc, 64, "fail counter")) != USFFT_OK) return bail(st);
    if (pr.kind == USFFT_TRIGPOLY) {
        const size_t nt = (size_t)G * pr.tp_nterms;
        plan->tp_freqs.assign(pr.tp_freqs, pr.tp_freqs + nt * pr.d);
        plan->tp_coefs.assign(pr.tp_coefs, pr.tp_coefs + nt * 2);
        if ((st = ensure(plan, plan->tpf, nt * pr.d, "trigpoly freqs")) != USFFT_OK) return bail(st);
        if ((st = ensure(plan, plan->tpc, nt * 2 * sizeof(double), "trigpoly coefs")) != USFFT_OK) return bail(st);
        if ((st = ensure(plan, plan->tpaux, nt * 3 * sizeof(double), "trigpoly aux")) != USFFT_OK) return bail(st);
        if (cudaMemcpyAsync(plan->tpf.p, plan->tp_freqs.data(), nt * pr.d, cudaMemcpyHostToDevice, plan->stream) !=
                cudaSuccess ||
            cudaMemcpyAsync(plan->tpc.p, plan->tp_coefs.data(), nt * 2 * sizeof(double), cudaMemcpyHostToDevice,
                            plan->stream) != cudaSuccess) {
            cudaGetLastError();
            fail(plan, USFFT_ECUDA, "copy of the trigonometric polynomials failed");
            return bail(USFFT_ECUDA);
        }
        plan->prob.tp_freqs = nullptr;
        plan->prob.tp_coefs = nullptr;
    } else {
        if ((st = ensure(plan, plan->psi, sizeof(double) * (size_t)E * pr.d, "mode table")) != USFFT_OK) return bail(st);
        if (launch_psi_table(pr.kind, pr.n, pr.d, pr.coef_scale, pr.coef_decay, (double*)plan->psi.p, plan->stream) !=
            cudaSuccess) {
            fail(plan, USFFT_ECUDA, "mode table kernel failed");
            return bail(USFFT_ECUDA);
        }
        if (pr.kind == USFFT_PDE_2D) {
            plan->cg_blocks = tune_get(TUNE_SAMPLER_BLOCKS, tune_key_sampler(pa.precision, pr.n),
                                       sample_2d_default_blocks(pr.n, pa.precision));
            size_t sb = sample_2d_scratch_bytes(pr.n, pa.precision, plan->cg_blocks);
            if ((st = ensure(plan, plan->cgscr, sb, "cg scratch")) != USFFT_OK) return bail(st);
        }
    }
    if ((st = wait_stream(plan)) != USFFT_OK) return bail(st);
    take_snapshot(plan);
    *out = plan;
    return USFFT_OK;
}

}  // extern "C"

namespace {

struct ShardCtx {
    int rank = 0, nranks = 1;
    usfft_allreduce_fn fn = nullptr;
    void* ctx = nullptr;
};

// usfft_increment (sh.nranks == 1) and usfft_increment_sharded
usfft_status increment_impl(usfft_plan_t* plan, usfft_increment_info* info, const ShardCtx& sh) {
    if (plan->t >= plan->d) return fail(plan, USFFT_ESTATE, "all d increments are done");
    const int t = plan->t + 1;
    const int N = plan->N, K = plan->K;
    plan->rr_active = false;
    plan->step_sharded = false;
    plan->launches = 0;
    plan->cg_iters_total = 0;
    plan->cg_iters_max = 0;
    plan->h2d = plan->d2h = 0;
    double ms_host = 0.0;
    usfft_status st;
    CK(cudaMemsetAsync(plan->failc.p, 0, sizeof(unsigned), plan->stream));
    CK(cudaEventRecord(plan->ev0, plan->stream));
    int64_t samples = 0;

    // ---- 1-D detections of dimension t (Algorithm 1, steps 1 & 2a) ----
    {
        std::vector<int64_t> m((size_t)K);
        for (int idx = 0; idx < K; ++idx) m[(size_t)idx] = ((idx - N) % K + K) % K;
        if ((st = prepare_step(plan, K, m)) != USFFT_OK) return st;
        plan->specs.clear();
        for (int i = 1; i <= plan->par.r; ++i) plan->specs.push_back(spec_1d(plan, t, i));
        plan->s_tilde = plan->par.s_local;
        if ((st = run_step_device(plan, true)) != USFFT_OK) return st;
        if ((st = read_cg_stats(plan, K)) != USFFT_OK) return st;
        std::vector<uint32_t> bits;
        if ((st = read_bitmap(plan, bits)) != USFFT_OK) return st;
        plan->I1d[(size_t)t].clear();
        for (int idx = 0; idx < K; ++idx)
            if (bits[(size_t)idx >> 5] >> (idx & 31) & 1u) plan->I1d[(size_t)t].push_back(idx - N);
        samples += (int64_t)K * plan->par.r;
        plan->last_coupled = false;
        plan->last_t = t;
        plan->z.assign(1, 1);
        plan->J.resize((size_t)K);
        for (int idx = 0; idx < K; ++idx) plan->J[(size_t)idx] = (int8_t)(idx - N);
    }
    if (t == 1) {
        plan->nIpre = (int64_t)plan->I1d[1].size();
        plan->Ipre.assign(plan->I1d[1].begin(), plan->I1d[1].end());
    } else {
        // ---- coupled step t (Algorithm 1, step 2) ----
        auto h0 = std::chrono::steady_clock::now();
        std::vector<int8_t> J;
        int64_t nJ = 0;
        candidate_set(plan->Ipre.data(), plan->nIpre, t - 1, plan->I1d[(size_t)t], N, J, nJ);
        const int rt = t < plan->d ? plan->par.r : 1;
        plan->s_tilde = t < plan->d ? plan->par.s_local : plan->par.s;
        plan->specs.clear();
        if (plan->par.rr_lattices > 0) {
            // random rank-1 lattices in the role of Algorithm A
            plan->J = J;
            plan->last_coupled = true;
            plan->last_t = t;
            plan->rr_active = true;
            if (nJ > 0) {
                if ((st = prepare_rr(plan, J, nJ, t, rt, plan->s_tilde)) != USFFT_OK) return st;
                for (int i = 1; i <= rt; ++i)
                    for (int l = 0; l < plan->rr_L; ++l) {
                        const size_t q = (size_t)(i - 1) * plan->rr_L + l;
                        NodeSpec ns = spec_coupled(plan, t, i);      // tails of iteration i
                        ns.M = plan->rr_M[q];
                        for (int j = 0; j < t; ++j) ns.z[j] = plan->rr_z[q * t + j];
                        plan->specs.push_back(ns);
                    }
            } else {
                plan->M = 0;
                plan->m.clear();
                plan->nJ = 0;
                plan->rr_iters = 0;
            }
            ms_host = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - h0).count();
        } else {
            std::vector<int64_t> z;
            int64_t M = 0;
            if (!lattice_search(J.data(), nJ, t, plan->par.seed, plan->par.max_lattice_trials, plan->par.max_lattice_sizes,
                                z, M, PHASE_LATTICE, sh.nranks))
                return fail(plan, USFFT_ELATTICE, "no reconstructing rank-1 lattice found");
            std::vector<int64_t> m((size_t)nJ);
            for (int64_t a = 0; a < nJ; ++a) {
                int64_t acc = 0;
                for (int j = 0; j < t; ++j) acc += (int64_t)J[(size_t)(a * t + j)] * z[(size_t)j];
                int64_t mm = acc % M;
                m[(size_t)a] = mm < 0 ? mm + M : mm;
            }
            ms_host = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - h0).count();
            plan->J = J;
            plan->z = z;
            plan->last_coupled = true;
            plan->last_t = t;
            if (nJ > 0 && sh.nranks > 1) {
                // this rank's share: nodes p + P i2, a length-M/P FFT read at m mod M/P
                const int64_t P = sh.nranks, L = M / P;
                if (plan->prob.kind != USFFT_TRIGPOLY && plan->prob.theta_map == USFFT_MAP_NORMAL &&
                    lattice_hits_pole(M, plan->prob.map_shift))
                    return fail(plan, USFFT_EINVAL, "a node of the lattice lies on a pole of the lognormal map");
                std::vector<int64_t> mr((size_t)nJ);
                std::vector<int> m32((size_t)nJ);
                for (int64_t a = 0; a < nJ; ++a) {
                    mr[(size_t)a] = m[(size_t)a] % L;
                    m32[(size_t)a] = (int)m[(size_t)a];
                }
                if ((st = prepare_step(plan, L, mr, false)) != USFFT_OK) return st;
                if ((st = ensure(plan, plan->smk, sizeof(int) * (size_t)nJ, "full lattice indices")) != USFFT_OK) return st;
                if ((st = ensure(plan, plan->sflags, (size_t)nJ, "union flags")) != USFFT_OK) return st;
                CK(cudaMemcpyAsync(plan->smk.p, m32.data(), sizeof(int) * (size_t)nJ, cudaMemcpyHostToDevice,
                                   plan->stream));
                plan->h2d += (int64_t)(sizeof(int) * (size_t)nJ);
                CK(cudaStreamSynchronize(plan->stream));   // m32 outlives the copy
                plan->step_sharded = true;
                plan->shard_rank = sh.rank;
                plan->shard_n = sh.nranks;
                plan->shard_fn = sh.fn;
                plan->shard_ctx = sh.ctx;
                plan->shard_M = M;
                plan->shard_m = m;
            } else if (nJ > 0) {
                if ((st = prepare_step(plan, M, m)) != USFFT_OK) return st;
            } else {
                plan->M = 0;
                plan->m.clear();
                plan->nJ = 0;
            }
            for (int i = 1; i <= rt && nJ > 0; ++i) {
                NodeSpec ns = spec_coupled(plan, t, i);
                if (plan->step_sharded) {
                    ns.M = plan->shard_M;
                    ns.first = sh.rank;
                    ns.stride = sh.nranks;
                }
                plan->specs.push_back(ns);
            }
        }
        if ((st = run_step_device(plan, false)) != USFFT_OK) return st;
        if ((st = read_cg_stats(plan, plan->M)) != USFFT_OK) return st;
        std::vector<uint32_t> bits;
        if ((st = read_bitmap(plan, bits)) != USFFT_OK) return st;
        std::vector<int8_t> I;
        int64_t nI = 0;
        for (int64_t a = 0; a < nJ; ++a)
            if (bits[(size_t)a >> 5] >> (a & 31) & 1u) {
                I.insert(I.end(), J.begin() + a * t, J.begin() + (a + 1) * t);
                ++nI;
            }
        plan->Ipre.swap(I);
        plan->nIpre = nI;
        for (const NodeSpec& ns : plan->specs) samples += node_count(ns);
    }
    CK(cudaEventRecord(plan->ev1, plan->stream));
    if ((st = wait_stream(plan)) != USFFT_OK) return st;
    plan->t = t;
    plan->replay_valid = true;
    take_snapshot(plan);
    if (info) {
        memset(info, 0, sizeof *info);
        info->t = t;
        info->M = plan->last_coupled ? (plan->step_sharded ? plan->shard_M : plan->M) : 0;
        info->n_candidates = plan->last_coupled ? plan->nJ : K;
        info->n_detected = plan->nIpre;
        info->n_1d = (int64_t)plan->I1d[(size_t)t].size();
        info->samples = samples;
        info->cg_iters_total = plan->cg_iters_total;
        info->cg_iters_max = plan->cg_iters_max;
        info->kernel_launches = plan->launches;
        info->theta = plan->theta;
        float ms = 0.f;
        cudaEventElapsedTime(&ms, plan->ev0, plan->ev1);
        info->ms_device = ms;
        info->ms_host_plan = ms_host;
        info->h2d_bytes = plan->h2d;
        info->d2h_bytes = plan->d2h;
    }
    return USFFT_OK;
}

// P is a valid rank count of the sharded form: 1 <= P <= 64 and 7-smooth (so that 7-smooth
// lattice sizes that are multiples of P exist)
bool valid_rank_count(int64_t P) { return P >= 1 && P <= 64 && is_smooth7(P); }

}  // namespace

extern "C" {

usfft_status usfft_increment(usfft_plan_t* plan, usfft_increment_info* info) {
    if (!plan) return fail(nullptr, USFFT_EINVAL, "plan is NULL");
    return increment_impl(plan, info, ShardCtx());
}

usfft_status usfft_increment_sharded(usfft_plan_t* plan, int rank, int nranks, usfft_allreduce_fn allreduce,
                                     void* ctx, usfft_increment_info* info) {
    if (!plan) return fail(nullptr, USFFT_EINVAL, "plan is NULL");
    if (!valid_rank_count(nranks) || rank < 0 || rank >= nranks)
        return fail(plan, USFFT_EINVAL, "usfft_increment_sharded: need 0 <= rank < nranks <= 64, nranks 7-smooth");
    if (nranks > 1 && !allreduce) return fail(plan, USFFT_EINVAL, "usfft_increment_sharded: allreduce hook is NULL");
    if (nranks > 1 && plan->par.rr_lattices > 0)
        return fail(plan, USFFT_EINVAL, "usfft_increment_sharded: single reconstructing lattices only (rr_lattices = 0)");
    ShardCtx sh;
    sh.rank = rank;
    sh.nranks = nranks;
    sh.fn = allreduce;
    sh.ctx = ctx;
    return increment_impl(plan, info, sh);
}

usfft_status usfft_search_lattice_multiple(const int8_t* J, int64_t n, int t, uint64_t seed, int trials, int max_sizes,
                                           int64_t divisor, int64_t* z, int64_t* M) {
    if (t < 1 || n < 0 || (n > 0 && !J) || !z || !M || trials < 1 || max_sizes < 1 || !valid_rank_count(divisor))
        return fail(nullptr, USFFT_EINVAL, "usfft_search_lattice_multiple: invalid argument");
    std::vector<int64_t> zz;
    int64_t mm = 0;
    if (!lattice_search(J, n, t, seed, trials, max_sizes, zz, mm, PHASE_LATTICE, divisor))
        return fail(nullptr, USFFT_ELATTICE, "no reconstructing rank-1 lattice found");
    for (int j = 0; j < t; ++j) z[j] = zz[(size_t)j];
    *M = mm;
    return USFFT_OK;
}

// ms per replay of the plan's last step: one untimed replay, then `reps` between two events
static usfft_status time_replays(usfft_plan_t* plan, int reps, double* ms) {
    usfft_status st = run_step_device(plan, false);
    if (st != USFFT_OK) return st;
    CK(cudaEventRecord(plan->ev0, plan->stream));
    for (int k = 0; k < reps; ++k)
        if ((st = run_step_device(plan, false)) != USFFT_OK) return st;
    CK(cudaEventRecord(plan->ev1, plan->stream));
    if ((st = wait_stream(plan)) != USFFT_OK) return st;
    float e = 0.f;
    CK(cudaEventElapsedTime(&e, plan->ev0, plan->ev1));
    *ms = (double)e / reps;
    return USFFT_OK;
}

usfft_status usfft_autotune(usfft_plan_t* plan, int reps, usfft_tune_report* out) {
    if (!plan) return fail(nullptr, USFFT_EINVAL, "plan is NULL");
    if (plan->t < 1 || !plan->replay_valid) return fail(plan, USFFT_ESTATE, "usfft_autotune needs a completed increment");
    if (reps < 1) reps = 3;
    const int saved_launches = plan->launches;
    const bool saved_keep = plan->keep_iters, saved_timing = plan->timing;
    plan->keep_iters = false;
    plan->timing = false;
    usfft_tune_report rep;
    memset(&rep, 0, sizeof rep);
    usfft_status st = time_replays(plan, reps, &rep.ms_before);
    double best_ms = rep.ms_before;
    // 1. persistent grid of the 2-D sampler: one, two or four CTAs per SM's worth of resident CTAs
    if (st == USFFT_OK && plan->prob.kind == USFFT_PDE_2D && plan->par.precision != USFFT_FP64) {
        const int def = sample_2d_default_blocks(plan->prob.n, plan->par.precision);
        const int cur = plan->cg_blocks;
        int best = cur;
        for (int mult : {1, 2, 4}) {
            const int cand = def * mult;
            if (cand == cur) continue;
            if ((st = ensure(plan, plan->cgscr, sample_2d_scratch_bytes(plan->prob.n, plan->par.precision, cand),
                             "cg scratch")) != USFFT_OK)
                break;
            plan->cg_blocks = cand;
            double ms = 0.0;
            if ((st = time_replays(plan, reps, &ms)) != USFFT_OK) break;
            if (ms < best_ms) {
                best_ms = ms;
                best = cand;
            }
        }
        plan->cg_blocks = best;
        if (st == USFFT_OK) tune_set(TUNE_SAMPLER_BLOCKS, tune_key_sampler(plan->par.precision, plan->prob.n), best, best_ms);
        rep.sampler_blocks = best;
    }
    // 2. column-pair tile of each pass of the two-pass lattice FFT (when the last step used it)
    if (st == USFFT_OK && !plan->rr_active && !plan->inplace && plan->nJ > 0 && plan->fp.L2 > 0) {
        const int Gp = (plan->G + 1) / 2;
        const bool two = plan->fp.L1 > 1;
        for (int pass = two ? 0 : 1; pass < 2 && st == USFFT_OK; ++pass) {
            const bool fin = pass == 1;
            const int L = fin ? plan->fp.L2 : plan->fp.L1;
            const int nb = fin ? (two && plan->fp.L1 > 2 ? 2 : 1) : 1;
            const int64_t key = tune_key_fft(L, fin);
            int best = tune_get(TUNE_FFT_TILE, key, fft_default_tile(L, Gp, nb));
            for (int cand : {1, 2, 4, 8, 16, 32}) {
                if (cand > Gp || !fft_tile_fits(L, cand, nb) || cand == best) continue;
                tune_set(TUNE_FFT_TILE, key, cand, 0.0);
                double ms = 0.0;
                if ((st = time_replays(plan, reps, &ms)) != USFFT_OK) break;
                if (ms < best_ms) {
                    best_ms = ms;
                    best = cand;
                }
            }
            tune_set(TUNE_FFT_TILE, key, best, best_ms);
            if (fin) rep.fft_final_tile = best; else rep.fft_pass1_tile = best;
        }
    }
    if (st == USFFT_OK) st = time_replays(plan, reps, &rep.ms_after);
    plan->keep_iters = saved_keep;
    plan->timing = saved_timing;
    plan->launches = saved_launches;
    if (out) *out = rep;
    return st;
}

usfft_status usfft_tune_export(char* text, size_t capacity, size_t* length) {
    const std::string t = tune_dump();
    if (length) *length = t.size();
    if (!text) return USFFT_OK;
    if (capacity < t.size() + 1) return fail(nullptr, USFFT_EINVAL, "usfft_tune_export: buffer too small");
    memcpy(text, t.c_str(), t.size() + 1);
    return USFFT_OK;
}

usfft_status usfft_tune_import(const char* text) {
    if (!text) {
        tune_clear();
        return USFFT_OK;
    }
    std::string err;
    if (!tune_parse(text, err)) return fail(nullptr, USFFT_EINVAL, err);
    return USFFT_OK;
}

usfft_status usfft_replay(usfft_plan_t* plan, int sync, int32_t* launches) {
    if (!plan) return fail(nullptr, USFFT_EINVAL, "plan is NULL");
    if (plan->t < 1 || !plan->replay_valid) return fail(plan, USFFT_ESTATE, "no increment to replay");
    plan->launches = 0;
    usfft_status st = run_step_device(plan, false);
    if (st != USFFT_OK) return st;
    if (launches) *launches = plan->launches;
    if (sync) return wait_stream(plan);
    return USFFT_OK;
}

usfft_status usfft_rewind(usfft_plan_t* plan, int t) {
    if (!plan) return fail(nullptr, USFFT_EINVAL, "plan is NULL");
    if (t < 0 || t > plan->t || (size_t)t >= plan->hist.size()) return fail(plan, USFFT_EINVAL, "t out of range");
    const Snapshot& s = plan->hist[(size_t)t];
    plan->t = s.t;
    plan->Ipre = s.Ipre;
    plan->nIpre = s.nIpre;
    plan->I1d = s.I1d;
    plan->theta = s.theta;
    plan->A = s.A;
    plan->theta_set = s.theta_set;
    plan->hist.resize((size_t)t + 1);
    plan->replay_valid = false;
    return USFFT_OK;
}

usfft_status usfft_resume(usfft_plan_t* plan, int t, const int8_t* I, int64_t n, double theta) {
    if (!plan) return fail(nullptr, USFFT_EINVAL, "plan is NULL");
    if (t < 0 || t > plan->d || n < 0 || (n > 0 && !I)) return fail(plan, USFFT_EINVAL, "usfft_resume: invalid argument");
    if (t > 0 && !(theta > 0.0)) return fail(plan, USFFT_EINVAL, "usfft_resume: theta must be > 0");
    plan->t = t;
    plan->nIpre = t > 0 ? n : 0;
    plan->Ipre.assign(I, I + (t > 0 ? n * t : 0));
    for (auto& v : plan->I1d) v.clear();
    if (t > 0) {
        plan->theta = theta;
        plan->theta_set = true;
    } else if (plan->par.delta_is_relative) {
        plan->theta_set = false;
    }
    plan->hist.clear();
    plan->replay_valid = false;
    Snapshot s;
    s.t = t;
    s.Ipre = plan->Ipre;
    s.nIpre = plan->nIpre;
    s.I1d = plan->I1d;
    s.theta = plan->theta;
    s.A = plan->A;
    s.theta_set = plan->theta_set;
    plan->hist.assign((size_t)t + 1, s);
    return USFFT_OK;
}

usfft_status usfft_set_timing(usfft_plan_t* plan, int on) {
    if (!plan) return fail(nullptr, USFFT_EINVAL, "plan is NULL");
    usfft_status st = wait_stream(plan);
    if (st != USFFT_OK) return st;
    plan->timing = on != 0;
    plan->tev.clear();
    plan->ev_used = 0;
    CK(cudaMemsetAsync((char*)plan->failc.p + 8, 0, 16, plan->stream));
    return USFFT_OK;
}

usfft_status usfft_get_stage_times(usfft_plan_t* plan, usfft_stage_times* out) {
    if (!plan || !out) return fail(plan, USFFT_EINVAL, "plan or out is NULL");
    usfft_status st = wait_stream(plan);
    if (st != USFFT_OK) return st;
    memset(out, 0, sizeof *out);
    for (auto& e : plan->tev) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, e.second.first, e.second.second) != cudaSuccess) {
            cudaGetLastError();
            continue;
        }
        if (e.first >= 0 && e.first < 3) {
            out->ms[e.first] += ms;
            out->launches[e.first] += 1;
        }
    }
    unsigned long long it[2] = {0, 0};
    CK(cudaMemcpy(it, (char*)plan->failc.p + 8, 16, cudaMemcpyDeviceToHost));
    out->cg_iters_total = (int64_t)it[0];
    out->refine_steps_total = (int64_t)it[1];
    return USFFT_OK;
}

usfft_status usfft_get_set(const usfft_plan_t* plan, int8_t* freqs, int64_t n_capacity, int64_t* n, int32_t* t) {
    if (!plan) return fail(nullptr, USFFT_EINVAL, "plan is NULL");
    if (n) *n = plan->nIpre;
    if (t) *t = plan->t;
    if (freqs) {
        if (n_capacity < plan->nIpre) return fail(const_cast<usfft_plan_t*>(plan), USFFT_EINVAL, "freqs too small");
        memcpy(freqs, plan->Ipre.data(), plan->Ipre.size());
    }
    return USFFT_OK;
}

usfft_status usfft_get_lattice(const usfft_plan_t* plan, int64_t* z, int64_t* M, int32_t* t) {
    if (!plan) return fail(nullptr, USFFT_EINVAL, "plan is NULL");
    const int tt = plan->last_coupled ? plan->last_t : 1;
    if (t) *t = tt;
    if (M) *M = plan->last_coupled ? (plan->step_sharded ? plan->shard_M : plan->M) : plan->K;
    if (z) for (int j = 0; j < tt; ++j) z[j] = plan->last_coupled ? plan->z[(size_t)j] : 1;
    return USFFT_OK;
}

usfft_status usfft_get_candidates(const usfft_plan_t* plan, int8_t* J, int64_t* n, int64_t* m) {
    if (!plan) return fail(nullptr, USFFT_EINVAL, "plan is NULL");
    if (n) *n = plan->nJ;
    if (J) memcpy(J, plan->J.data(), plan->J.size());
    const std::vector<int64_t>& mm = plan->step_sharded ? plan->shard_m : plan->m;
    if (m) for (int64_t k = 0; k < plan->nJ; ++k) m[k] = mm[(size_t)k];
    return USFFT_OK;
}

usfft_status usfft_get_samples(const usfft_plan_t* plan_c, double* U, int64_t* M, int64_t* G) {
    usfft_plan_t* plan = const_cast<usfft_plan_t*>(plan_c);
    if (!plan) return fail(nullptr, USFFT_EINVAL, "plan is NULL");
    if (M) *M = plan->M;
    if (G) *G = plan->G;
    if (U && plan->M > 0) {
        CK(cudaMemcpyAsync(U, plan->U.p, sizeof(double) * (size_t)plan->M * plan->G, cudaMemcpyDeviceToHost,
                           plan->stream));
        return wait_stream(plan);
    }
    return USFFT_OK;
}

usfft_status usfft_get_coefficients(const usfft_plan_t* plan_c, double* C, int64_t* G, int64_t* n) {
    usfft_plan_t* plan = const_cast<usfft_plan_t*>(plan_c);
    if (!plan) return fail(nullptr, USFFT_EINVAL, "plan is NULL");
    if (G) *G = plan->G;
    if (n) *n = plan->nJ;
    if (C && plan->nJ > 0) {
        CK(cudaMemcpyAsync(C, plan->C.p, sizeof(double2) * (size_t)plan->nJ * plan->G, cudaMemcpyDeviceToHost,
                           plan->stream));
        return wait_stream(plan);
    }
    return USFFT_OK;
}

usfft_status usfft_get_random_lattices(const usfft_plan_t* plan_c, int64_t* z, int64_t* M, int32_t* count,
                                       int32_t* t) {
    const usfft_plan_t* plan = plan_c;
    if (!plan) return fail(nullptr, USFFT_EINVAL, "plan is NULL");
    const bool on = plan->rr_active && plan->nJ > 0;
    const int32_t cnt = on ? (int32_t)plan->rr_M.size() : 0;
    const int32_t tt = on ? (int32_t)(plan->rr_z.size() / std::max<size_t>(plan->rr_M.size(), 1)) : 0;
    if (count) *count = cnt;
    if (t) *t = tt;
    if (cnt && z) memcpy(z, plan->rr_z.data(), sizeof(int64_t) * plan->rr_z.size());
    if (cnt && M) memcpy(M, plan->rr_M.data(), sizeof(int64_t) * plan->rr_M.size());
    return USFFT_OK;
}

usfft_status usfft_get_selection(const usfft_plan_t* plan_c, uint32_t* bitmap, int64_t* n) {
    usfft_plan_t* plan = const_cast<usfft_plan_t*>(plan_c);
    if (!plan) return fail(nullptr, USFFT_EINVAL, "plan is NULL");
    if (n) *n = plan->nJ;
    if (bitmap && plan->nJ > 0) {
        CK(cudaMemcpyAsync(bitmap, plan->bitmap.p, sizeof(uint32_t) * (size_t)((plan->nJ + 31) / 32),
                           cudaMemcpyDeviceToHost, plan->stream));
        return wait_stream(plan);
    }
    return USFFT_OK;
}

usfft_status usfft_set_keep_iterations(usfft_plan_t* plan, int on) {
    if (!plan) return fail(nullptr, USFFT_EINVAL, "plan is NULL");
    plan->keep_iters = on != 0;
    if (!plan->keep_iters) {
        usfft_status st = wait_stream(plan);
        if (st != USFFT_OK) return st;
        for (std::vector<Buf>* v : {&plan->kU, &plan->kC, &plan->kB})
            for (Buf& b : *v) buf_free(plan, b);
        plan->kU.clear();
        plan->kC.clear();
        plan->kB.clear();
        plan->kept = 0;
    }
    return USFFT_OK;
}

usfft_status usfft_get_iteration(const usfft_plan_t* plan_c, int i, double* U, double* C, uint32_t* bitmap,
                                 int32_t* count) {
    usfft_plan_t* plan = const_cast<usfft_plan_t*>(plan_c);
    if (!plan) return fail(nullptr, USFFT_EINVAL, "plan is NULL");
    if (count) *count = plan->kept;
    if (!U && !C && !bitmap) return USFFT_OK;
    if (i < 1 || i > plan->kept) return fail(plan, USFFT_EINVAL, "usfft_get_iteration: no such kept iteration");
    const size_t it = (size_t)(i - 1);
    if (U && plan->M > 0)
        CK(cudaMemcpyAsync(U, plan->kU[it].p, sizeof(double) * (size_t)plan->M * plan->G, cudaMemcpyDeviceToHost,
                           plan->stream));
    if (C && plan->nJ > 0)
        CK(cudaMemcpyAsync(C, plan->kC[it].p, sizeof(double2) * (size_t)plan->nJ * plan->G, cudaMemcpyDeviceToHost,
                           plan->stream));
    if (bitmap && plan->nJ > 0)
        CK(cudaMemcpyAsync(bitmap, plan->kB[it].p, sizeof(uint32_t) * (size_t)((plan->nJ + 31) / 32),
                           cudaMemcpyDeviceToHost, plan->stream));
    return wait_stream(plan);
}

// the coefficients of step 3 (in plan->C, on I = plan->Ipre) kept with I for usfft_evaluate /
// usfft_errors / usfft_statistics, and copied to the caller's host or device buffer
static usfft_status store_reconstruction(usfft_plan_t* plan, double* coefs, int coefs_on_device) {
    const int64_t nI = plan->nIpre;
    const int d = plan->d;
    const size_t bytes = sizeof(double2) * (size_t)nI * plan->G;
    usfft_status st;
    if ((st = ensure(plan, plan->Crec, bytes, "reconstruction coefficients")) != USFFT_OK) return st;
    if ((st = ensure(plan, plan->Irec, (size_t)nI * d, "reconstruction set")) != USFFT_OK) return st;
    CK(cudaMemcpyAsync(plan->Crec.p, plan->C.p, bytes, cudaMemcpyDeviceToDevice, plan->stream));
    CK(cudaMemcpyAsync(plan->Irec.p, plan->Ipre.data(), (size_t)nI * d, cudaMemcpyHostToDevice, plan->stream));
    plan->h2d += (int64_t)nI * d;
    CK(cudaMemcpyAsync(coefs, plan->C.p, bytes, coefs_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                       plan->stream));
    if ((st = wait_stream(plan)) != USFFT_OK) return st;
    plan->nrec = nI;
    plan->Irec_h = plan->Ipre;
    return USFFT_OK;
}

usfft_status usfft_reconstruct(usfft_plan_t* plan, int64_t* n, int8_t* freqs, double* coefs, int coefs_on_device) {
    if (!plan) return fail(nullptr, USFFT_EINVAL, "plan is NULL");
    if (plan->t != plan->d) return fail(plan, USFFT_ESTATE, "usfft_reconstruct needs all d increments done");
    if (n) *n = plan->nIpre;
    if (freqs) memcpy(freqs, plan->Ipre.data(), plan->Ipre.size());
    if (!coefs) return USFFT_OK;
    const int d = plan->d;
    const int64_t nI = plan->nIpre;
    if (nI == 0) {             // nothing detected: the approximation is zero
        plan->nrec = 0;
        plan->Irec_h.clear();
        return USFFT_OK;
    }
    // one reconstructing rank-1 lattice for I (Algorithm 1, step 3; single-lattice reading)
    std::vector<int64_t> z;
    int64_t M = 0;
    if (!lattice_search(plan->Ipre.data(), nI, d, plan->par.seed, plan->par.max_lattice_trials, plan->par.max_lattice_sizes, z, M,
                        PHASE_RECON))
        return fail(plan, USFFT_ELATTICE, "no reconstructing rank-1 lattice for the detected set");
    std::vector<int64_t> m((size_t)nI);
    for (int64_t a = 0; a < nI; ++a) {
        int64_t acc = 0;
        for (int j = 0; j < d; ++j) acc += (int64_t)plan->Ipre[(size_t)(a * d + j)] * z[(size_t)j];
        int64_t mm = acc % M;
        m[(size_t)a] = mm < 0 ? mm + M : mm;
    }
    plan->launches = 0;
    plan->cg_iters_total = 0;
    plan->cg_iters_max = 0;
    plan->nrec = -1;
    plan->rr_active = false;
    plan->rr_pick_only = false;
    CK(cudaMemsetAsync(plan->failc.p, 0, sizeof(unsigned), plan->stream));
    usfft_status st = prepare_step(plan, M, m);
    if (st != USFFT_OK) return st;
    plan->J = plan->Ipre;
    plan->z = z;
    plan->last_coupled = true;
    plan->last_t = d;
    plan->replay_valid = false;
    NodeSpec ns;
    memset(&ns, 0, sizeof ns);
    ns.M = M;
    ns.d = d;
    set_map(ns, plan->prob);
    for (int j = 0; j < d; ++j) ns.z[j] = z[(size_t)j];
    plan->specs.assign(1, ns);
    plan->s_tilde = 0;                       // no threshold in step 3
    if ((st = run_step_device(plan, false)) != USFFT_OK) return st;
    if ((st = read_cg_stats(plan, M)) != USFFT_OK) return st;
    return store_reconstruction(plan, coefs, coefs_on_device);
}

// most lattices step 3 may take on multiple rank-1 lattices before it reports USFFT_ELATTICE
static const int kMaxReconLattices = 64;

usfft_status usfft_reconstruct_multiple(usfft_plan_t* plan, int64_t* n, int8_t* freqs, double* coefs,
                                        int coefs_on_device) {
    if (!plan) return fail(nullptr, USFFT_EINVAL, "plan is NULL");
    if (plan->t != plan->d) return fail(plan, USFFT_ESTATE, "usfft_reconstruct_multiple needs all d increments done");
    if (n) *n = plan->nIpre;
    if (freqs) memcpy(freqs, plan->Ipre.data(), plan->Ipre.size());
    if (!coefs) return USFFT_OK;
    const int d = plan->d;
    const int64_t nI = plan->nIpre;
    if (nI == 0) {             // nothing detected: the approximation is zero
        plan->nrec = 0;
        plan->Irec_h.clear();
        return USFFT_OK;
    }
    // the lattices (Algorithm 1, step 3 on multiple rank-1 lattices): added until every k of I
    // is alone at its index in one of them
    std::vector<int64_t> z, M;
    std::vector<int> first;
    if (!multiple_lattices(plan->Ipre.data(), nI, d, plan->par.seed, kMaxReconLattices, z, M, first))
        return fail(plan, USFFT_ELATTICE, "multiple rank-1 lattices: a frequency of I shares its index in all 64 lattices");
    const int L = (int)M.size();
    plan->launches = 0;
    plan->cg_iters_total = 0;
    plan->cg_iters_max = 0;
    plan->nrec = -1;
    CK(cudaMemsetAsync(plan->failc.p, 0, sizeof(unsigned), plan->stream));
    plan->J = plan->Ipre;
    plan->last_coupled = true;
    plan->last_t = d;
    plan->replay_valid = false;
    plan->rr_active = true;
    plan->s_tilde = 0;                       // no threshold in step 3
    usfft_status st = prepare_lattice_set(plan, plan->Ipre, nI, d, 1, L, z, M);
    plan->rr_pick_only = true;
    if (st != USFFT_OK) {
        plan->rr_active = false;
        return st;
    }
    plan->specs.clear();
    for (int l = 0; l < L; ++l) {
        NodeSpec ns;
        memset(&ns, 0, sizeof ns);
        ns.M = M[(size_t)l];
        ns.d = d;
        set_map(ns, plan->prob);
        for (int j = 0; j < d; ++j) ns.z[j] = z[(size_t)l * d + j];
        plan->specs.push_back(ns);
    }
    if ((st = run_step_device(plan, false)) != USFFT_OK) return st;
    if ((st = read_cg_stats(plan, plan->M)) != USFFT_OK) return st;
    return store_reconstruction(plan, coefs, coefs_on_device);
}

// ---- evaluation at given points (Section 4) ----------------------------------------------
namespace {

const int64_t kPointChunk = 8192;

usfft_status check_points(usfft_plan_t* plan, const double* y, int64_t n, const char* who) {
    if (n < 0 || (n > 0 && !y)) return fail(plan, USFFT_EINVAL, std::string(who) + ": need n >= 0 and y");
    return USFFT_OK;
}

// points [cnt][d] on the device: the caller's (device input) or staged through Ypts
usfft_status stage_points(usfft_plan_t* plan, const double* y, int64_t off, int64_t cnt, int on_device,
                          const double** yd) {
    const int d = plan->d;
    if (on_device) {
        *yd = y + off * d;
        return USFFT_OK;
    }
    usfft_status st = ensure(plan, plan->Ypts, sizeof(double) * (size_t)kPointChunk * d, "points");
    if (st != USFFT_OK) return st;
    CK(cudaMemcpyAsync(plan->Ypts.p, y + off * d, sizeof(double) * (size_t)cnt * d, cudaMemcpyHostToDevice,
                       plan->stream));
    plan->h2d += (int64_t)(sizeof(double) * (size_t)cnt * d);
    *yd = (const double*)plan->Ypts.p;
    return USFFT_OK;
}

// FE solutions (or the test polynomials) at cnt explicit points into out [cnt][G] (device)
usfft_status sample_at(usfft_plan_t* plan, const double* yd, int64_t cnt, double* out) {
    usfft_status st = ensure(plan, plan->iters, sizeof(int) * (size_t)cnt, "cg iterations");
    if (st != USFFT_OK) return st;
    NodeSpec ns;
    memset(&ns, 0, sizeof ns);
    ns.M = cnt;
    ns.d = plan->d;
    set_map(ns, plan->prob);
    ns.Y = yd;
    if ((st = run_sampler(plan, ns, out)) != USFFT_OK) return st;
    return read_cg_stats(plan, cnt);
}

void reset_counters(usfft_plan_t* plan) {
    plan->launches = 0;
    plan->cg_iters_total = 0;
    plan->cg_iters_max = 0;
    plan->h2d = plan->d2h = 0;
}

}  // namespace

usfft_status usfft_sample_points(usfft_plan_t* plan, const double* y, int64_t n, double* samples, int on_device) {
    if (!plan) return fail(nullptr, USFFT_EINVAL, "plan is NULL");
    usfft_status st = check_points(plan, y, n, "usfft_sample_points");
    if (st != USFFT_OK) return st;
    if (n > 0 && !samples) return fail(plan, USFFT_EINVAL, "usfft_sample_points: samples is NULL");
    reset_counters(plan);
    CK(cudaMemsetAsync(plan->failc.p, 0, sizeof(unsigned), plan->stream));
    const int G = plan->G;
    for (int64_t off = 0; off < n; off += kPointChunk) {
        const int64_t cnt = std::min(kPointChunk, n - off);
        const double* yd = nullptr;
        if ((st = stage_points(plan, y, off, cnt, on_device, &yd)) != USFFT_OK) return st;
        double* out = samples + off * G;
        if (!on_device) {
            if ((st = ensure(plan, plan->Upts, sizeof(double) * (size_t)kPointChunk * G, "point samples")) != USFFT_OK)
                return st;
            out = (double*)plan->Upts.p;
        }
        if ((st = sample_at(plan, yd, cnt, out)) != USFFT_OK) return st;
        if (!on_device) {
            CK(cudaMemcpyAsync(samples + off * G, out, sizeof(double) * (size_t)cnt * G, cudaMemcpyDeviceToHost,
                               plan->stream));
            plan->d2h += (int64_t)(sizeof(double) * (size_t)cnt * G);
            if ((st = wait_stream(plan)) != USFFT_OK) return st;
        }
    }
    return wait_stream(plan);
}

usfft_status usfft_evaluate(usfft_plan_t* plan, const double* y, int64_t n, double* values, int on_device) {
    if (!plan) return fail(nullptr, USFFT_EINVAL, "plan is NULL");
    if (plan->nrec < 0) return fail(plan, USFFT_ESTATE, "usfft_evaluate needs a usfft_reconstruct first");
    usfft_status st = check_points(plan, y, n, "usfft_evaluate");
    if (st != USFFT_OK) return st;
    if (n > 0 && !values) return fail(plan, USFFT_EINVAL, "usfft_evaluate: values is NULL");
    reset_counters(plan);
    const int G = plan->G;
    for (int64_t off = 0; off < n; off += kPointChunk) {
        const int64_t cnt = std::min(kPointChunk, n - off);
        const double* yd = nullptr;
        if ((st = stage_points(plan, y, off, cnt, on_device, &yd)) != USFFT_OK) return st;
        double2* out = (double2*)values + off * G;
        if (!on_device) {
            if ((st = ensure(plan, plan->Vpts, sizeof(double2) * (size_t)kPointChunk * G, "point values")) != USFFT_OK)
                return st;
            out = (double2*)plan->Vpts.p;
        }
        CK(launch_evaluate(yd, cnt, plan->d, param_map(plan->prob), (const int8_t*)plan->Irec.p, plan->nrec, (const double2*)plan->Crec.p,
                           G, out, nullptr, nullptr, nullptr, plan->stream, &plan->launches));
        if (!on_device) {
            CK(cudaMemcpyAsync(values + 2 * off * G, out, sizeof(double2) * (size_t)cnt * G, cudaMemcpyDeviceToHost,
                               plan->stream));
            plan->d2h += (int64_t)(sizeof(double2) * (size_t)cnt * G);
            if ((st = wait_stream(plan)) != USFFT_OK) return st;
        }
    }
    return wait_stream(plan);
}

usfft_status usfft_errors(usfft_plan_t* plan, const double* y, int64_t n, int y_on_device, double* err2,
                          double* errinf) {
    if (!plan) return fail(nullptr, USFFT_EINVAL, "plan is NULL");
    if (plan->nrec < 0) return fail(plan, USFFT_ESTATE, "usfft_errors needs a usfft_reconstruct first");
    if (n < 1 || !y) return fail(plan, USFFT_EINVAL, "usfft_errors: need n >= 1 test points");
    if (!err2 || !errinf) return fail(plan, USFFT_EINVAL, "usfft_errors: err2 and errinf are required");
    reset_counters(plan);
    CK(cudaMemsetAsync(plan->failc.p, 0, sizeof(unsigned), plan->stream));
    const int G = plan->G;
    const int64_t tiles_max = (kPointChunk + evaluate_point_tile() - 1) / evaluate_point_tile();
    usfft_status st;
    if ((st = ensure(plan, plan->Upts, sizeof(double) * (size_t)kPointChunk * G, "point samples")) != USFFT_OK) return st;
    if ((st = ensure(plan, plan->epart, 2 * sizeof(double) * (size_t)tiles_max * G, "error partials")) != USFFT_OK)
        return st;
    if ((st = ensure(plan, plan->etot, 2 * sizeof(double) * (size_t)G, "errors")) != USFFT_OK) return st;
    double* psum = (double*)plan->epart.p;
    double* pmax = psum + (size_t)tiles_max * G;
    double* tsum = (double*)plan->etot.p;
    double* tmax = tsum + G;
    CK(cudaMemsetAsync(tsum, 0, 2 * sizeof(double) * (size_t)G, plan->stream));
    for (int64_t off = 0; off < n; off += kPointChunk) {
        const int64_t cnt = std::min(kPointChunk, n - off);
        const double* yd = nullptr;
        if ((st = stage_points(plan, y, off, cnt, y_on_device, &yd)) != USFFT_OK) return st;
        // the reference values: FE solutions at the test points
        if ((st = sample_at(plan, yd, cnt, (double*)plan->Upts.p)) != USFFT_OK) return st;
        CK(launch_evaluate(yd, cnt, plan->d, param_map(plan->prob), (const int8_t*)plan->Irec.p, plan->nrec, (const double2*)plan->Crec.p,
                           G, nullptr, (const double*)plan->Upts.p, psum, pmax, plan->stream, &plan->launches));
        const int tiles = (int)((cnt + evaluate_point_tile() - 1) / evaluate_point_tile());
        CK(launch_error_accumulate(psum, pmax, tiles, G, tsum, tmax, plan->stream, &plan->launches));
    }
    CK(launch_error_finalize(tsum, G, n, plan->stream, &plan->launches));
    CK(cudaMemcpyAsync(err2, tsum, sizeof(double) * (size_t)G, cudaMemcpyDeviceToHost, plan->stream));
    CK(cudaMemcpyAsync(errinf, tmax, sizeof(double) * (size_t)G, cudaMemcpyDeviceToHost, plan->stream));
    plan->d2h += (int64_t)(2 * sizeof(double) * (size_t)G);
    return wait_stream(plan);
}

usfft_status usfft_statistics(usfft_plan_t* plan, double* mean, double* variance, double* gsi) {
    if (!plan) return fail(nullptr, USFFT_EINVAL, "plan is NULL");
    if (plan->nrec < 0) return fail(plan, USFFT_ESTATE, "usfft_statistics needs a usfft_reconstruct first");
    reset_counters(plan);
    const int G = plan->G, d = plan->d;
    const int64_t nI = plan->nrec;
    // group the frequencies of I by their number of non-zero components (index bookkeeping)
    std::vector<int64_t> offsets((size_t)d + 2, 0);
    std::vector<int> order((size_t)nI), perm((size_t)nI);
    for (int64_t k = 0; k < nI; ++k) {
        int l = 0;
        for (int j = 0; j < d; ++j) l += plan->Irec_h[(size_t)(k * d + j)] != 0;
        order[(size_t)k] = l;
        offsets[(size_t)l + 1]++;
    }
    for (int l = 0; l <= d; ++l) offsets[(size_t)l + 1] += offsets[(size_t)l];
    {
        std::vector<int64_t> fill(offsets.begin(), offsets.end() - 1);
        for (int64_t k = 0; k < nI; ++k) perm[(size_t)fill[(size_t)order[(size_t)k]]++] = (int)k;
    }
    usfft_status st;
    const size_t stat_bytes = sizeof(double2) * (size_t)std::max<int64_t>(nI, 1) + sizeof(int) * (size_t)std::max<int64_t>(nI, 1) +
                              sizeof(int64_t) * offsets.size() + sizeof(double2) * G + sizeof(double) * G +
                              sizeof(double) * (size_t)G * d + 256 * 6;
    if ((st = ensure(plan, plan->epart, stat_bytes, "statistics")) != USFFT_OK) return st;
    char* base = (char*)plan->epart.p;
    auto carve = [&](size_t bytes) {
        char* p = base;
        base += (bytes + 255) & ~(size_t)255;
        return p;
    };
    double2* dfac = (double2*)carve(sizeof(double2) * (size_t)std::max<int64_t>(nI, 1));
    int* dperm = (int*)carve(sizeof(int) * (size_t)std::max<int64_t>(nI, 1));
    int64_t* doff = (int64_t*)carve(sizeof(int64_t) * offsets.size());
    double2* dmean = (double2*)carve(sizeof(double2) * G);
    double* dvar = (double*)carve(sizeof(double) * G);
    double* dgsi = (double*)carve(sizeof(double) * (size_t)G * d);
    if (nI) CK(cudaMemcpyAsync(dperm, perm.data(), sizeof(int) * (size_t)nI, cudaMemcpyHostToDevice, plan->stream));
    CK(cudaMemcpyAsync(doff, offsets.data(), sizeof(int64_t) * offsets.size(), cudaMemcpyHostToDevice, plan->stream));
    plan->h2d += (int64_t)(sizeof(int) * (size_t)nI + sizeof(int64_t) * offsets.size());
    CK(launch_expectation_factors((const int8_t*)plan->Irec.p, nI, d, param_map(plan->prob), dfac, plan->stream,
                                  &plan->launches));
    CK(launch_statistics((const double2*)plan->Crec.p, G, nI, d, dfac, dperm, doff, dmean, dvar, dgsi, plan->stream,
                         &plan->launches));
    if (mean) CK(cudaMemcpyAsync(mean, dmean, sizeof(double2) * G, cudaMemcpyDeviceToHost, plan->stream));
    if (variance) CK(cudaMemcpyAsync(variance, dvar, sizeof(double) * G, cudaMemcpyDeviceToHost, plan->stream));
    if (gsi) CK(cudaMemcpyAsync(gsi, dgsi, sizeof(double) * (size_t)G * d, cudaMemcpyDeviceToHost, plan->stream));
    plan->d2h += (int64_t)((mean ? 16 : 0) + (variance ? 8 : 0) + (gsi ? 8 * d : 0)) * G;
    return wait_stream(plan);   // the host vectors above outlive the copies
}

usfft_status usfft_search_lattice(const int8_t* J, int64_t n, int t, uint64_t seed, int trials, int max_sizes,
                                  int64_t* z, int64_t* M) {
    if (t < 1 || n < 0 || (n > 0 && !J) || !z || !M || trials < 1 || max_sizes < 1)
        return fail(nullptr, USFFT_EINVAL, "usfft_search_lattice: invalid argument");
    std::vector<int64_t> zz;
    int64_t mm = 0;
    if (!lattice_search(J, n, t, seed, trials, max_sizes, zz, mm))
        return fail(nullptr, USFFT_ELATTICE, "no reconstructing rank-1 lattice found");
    for (int j = 0; j < t; ++j) z[j] = zz[(size_t)j];
    *M = mm;
    return USFFT_OK;
}

usfft_status usfft_random_lattices(int t, int i, int64_t n_prev, int64_t n_t, int64_t s_t, int L, double factor,
                                   uint64_t seed, int64_t* z, int64_t* M) {
    if (t < 1 || t > USFFT_MAX_D || i < 1 || L < 1 || L > 31 || !(factor > 0.0 && factor < 1e6) || !z || !M ||
        n_prev < 0 || n_t < 0 || s_t < 0)
        return fail(nullptr, USFFT_EINVAL, "usfft_random_lattices: invalid argument");
    std::vector<int64_t> zz, mm;
    random_lattices(t, i, n_prev, n_t, s_t, L, factor, seed, zz, mm);
    memcpy(z, zz.data(), sizeof(int64_t) * zz.size());
    memcpy(M, mm.data(), sizeof(int64_t) * mm.size());
    return USFFT_OK;
}

usfft_status usfft_multiple_lattices(const int8_t* freqs, int64_t n, int d, uint64_t seed, int max_lattices, int64_t* z,
                                     int64_t* M, int32_t* count) {
    if (n < 0 || (n > 0 && !freqs) || d < 1 || d > USFFT_MAX_D || max_lattices < 1 || max_lattices > 1024 || !count)
        return fail(nullptr, USFFT_EINVAL, "usfft_multiple_lattices: invalid argument");
    std::vector<int64_t> zz, mm;
    std::vector<int> first;
    const bool ok = multiple_lattices(freqs, n, d, seed, max_lattices, zz, mm, first);
    *count = (int32_t)mm.size();
    if (z) memcpy(z, zz.data(), sizeof(int64_t) * zz.size());
    if (M) memcpy(M, mm.data(), sizeof(int64_t) * mm.size());
    return ok ? USFFT_OK : fail(nullptr, USFFT_ELATTICE, "usfft_multiple_lattices: max_lattices lattices leave a frequency shared");
}

uint64_t usfft_draw_key(uint64_t seed, const uint64_t* fields, int nfields) {
    return rng_key(seed, fields, nfields);
}

double usfft_draw_uniform(uint64_t seed, const uint64_t* fields, int nfields) {
    return rng_uniform(seed, fields, nfields);
}

size_t usfft_plan_bytes(const usfft_plan_t* plan) { return plan ? plan->bytes.load(std::memory_order_relaxed) : 0; }

void usfft_destroy(usfft_plan_t* plan) {
    if (!plan) return;
    cudaStreamSynchronize(plan->stream);
    Buf* bufs[] = {&plan->psi,   &plan->U,    &plan->C,    &plan->bitmap, &plan->twid, &plan->goff,
                   &plan->gk,    &plan->gm2,  &plan->fftscr, &plan->cgscr, &plan->iters, &plan->failc,
                   &plan->scal,  &plan->tpf,  &plan->tpc,  &plan->tpaux, &plan->Crec, &plan->Irec,
                   &plan->Ypts,  &plan->Upts, &plan->Vpts, &plan->epart, &plan->etot, &plan->rr_goff,
                   &plan->rr_gk, &plan->rr_gm2, &plan->rr_src, &plan->rr_twid, &plan->rr_C, &plan->fpos,
                   &plan->fmk};
    for (Buf* b : bufs) buf_free(plan, *b);
    for (std::vector<Buf>* v : {&plan->kU, &plan->kC, &plan->kB})
        for (Buf& b : *v) buf_free(plan, b);
    buf_free(plan, plan->smk);
    buf_free(plan, plan->sflags);
    if (plan->pinned) cudaFreeHost(plan->pinned);
    if (plan->ev0) cudaEventDestroy(plan->ev0);
    if (plan->ev1) cudaEventDestroy(plan->ev1);
    if (plan->evs) cudaEventDestroy(plan->evs);
    for (cudaEvent_t e : plan->ev_pool) cudaEventDestroy(e);
    delete plan;
}

}  // extern "C"
