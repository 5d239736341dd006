// usfft_sample_2d_static: the mixed-precision 2-D sampler with all of its scratch in one
// fixed, file-scope device array, for callers that cannot allocate device memory.
//
// Who needs it: code whose device memory is owned by someone else and that may not call
// cudaMalloc / cudaFree or an allocating library routine -- e.g. a plug-in running inside a
// framework that has already reserved (almost) all of HBM for its own pool, or a
// latency-critical loop that must never enter the allocator.  Such a caller passes its own
// input description and output buffer; the scratch the sampler needs (a counter of unconverged
// solves and one slot of edge weights, diagonal and residual per resident CTA) lives in g_static_scratch below.
//
// When the array is backed by device memory: CUDA loads a module lazily by default (CUDA 12.2
// and later), so the driver places g_static_scratch on a device when this file's module is
// first used there -- the set-up of the first call on that device -- not when the library is
// loaded.  From then on the device holds it until the process exits.  A caller that reserves
// nearly all of HBM for its own pool should therefore make its first call on each device (a
// call with count = 0 is enough) before it reserves the pool.
//
// Set-up: the first call on a device (with that device current) looks up the device
// address of g_static_scratch with cudaGetSymbolAddress -- the host-side symbol is only a
// stand-in and must never be passed to a kernel -- and caches it per device.  Make the first
// call on each device before any stream capture.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <string.h>

#include <mutex>
#include <string>

#include "usfft.h"
#include "usfft_internal.h"

namespace {

constexpr size_t kStaticScratchBytes = size_t(40) << 20;   // 40 MiB per device: a slot for each of 152 CTAs at n = 63
constexpr int kMaxDevices = 64;

__device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

std::mutex g_setup_mutex;
void* g_scratch_addr[kMaxDevices] = {};

// the message is what usfft_last_error(NULL) returns on this thread
usfft_status static_fail(usfft_status st, const std::string& msg) {
    usfft::set_thread_error(msg);
    return st;
}

// Device address of g_static_scratch on the current device (set up once per device).
usfft_status scratch_address(void** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return static_fail(USFFT_ECUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
    if (dev < 0 || dev >= kMaxDevices) return static_fail(USFFT_EINVAL, "device ordinal beyond 63");
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_scratch_addr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_static_scratch);
        if (e != cudaSuccess || !p) {
            cudaGetLastError();   // do not leave the error for the next launch check of any entry point
            return static_fail(USFFT_ECUDA, std::string("cudaGetSymbolAddress(g_static_scratch): ") +
                                                cudaGetErrorString(e));
        }
        g_scratch_addr[dev] = p;
    }
    *out = g_scratch_addr[dev];
    return USFFT_OK;
}

}  // namespace

extern "C" usfft_status usfft_sample_2d_static(const usfft_problem* problem, const int64_t* z, const double* tails,
                                               int64_t M, int64_t i0, int64_t count, double tol, int max_iters,
                                               double* U, void* stream, uint32_t* unconverged) {
    using namespace usfft;
    if (!problem || !z || !tails || !U) return static_fail(USFFT_EINVAL, "usfft_sample_2d_static: NULL argument");
    const usfft_problem& pr = *problem;
    if (pr.kind != USFFT_PDE_2D) return static_fail(USFFT_EINVAL, "usfft_sample_2d_static: 2-D problems only");
    if (pr.n < 1 || pr.n > 63) return static_fail(USFFT_EINVAL, "usfft_sample_2d_static: n must lie in [1, 63]");
    if (pr.d < 1 || pr.d > USFFT_MAX_D) return static_fail(USFFT_EINVAL, "usfft_sample_2d_static: d must lie in [1, 64]");
    if (pr.coef_model != USFFT_COEF_AFFINE_SIN && pr.coef_model != USFFT_COEF_LOGNORMAL_SIN)
        return static_fail(USFFT_EINVAL, "usfft_sample_2d_static: unknown coefficient model");
    if (pr.theta_map != USFFT_MAP_PERIODIC && pr.theta_map != USFFT_MAP_TENT && pr.theta_map != USFFT_MAP_NORMAL)
        return static_fail(USFFT_EINVAL, "usfft_sample_2d_static: unknown parameter map");
    if (M < 1 || M > (int64_t(1) << 31) || i0 < 0 || count < 0 || i0 + count > M)
        return static_fail(USFFT_EINVAL, "usfft_sample_2d_static: need 1 <= M <= 2^31 and 0 <= i0 <= i0+count <= M");
    NodeSpec ns;
    memset(&ns, 0, sizeof ns);
    ns.M = M;
    ns.d = pr.d;
    ns.map = pr.theta_map;
    ns.map_alpha = pr.map_alpha;
    ns.map_beta = pr.map_beta;
    ns.map_shift = pr.map_shift;
    for (int j = 0; j < pr.d; ++j) {
        if (z[j] >= M) return static_fail(USFFT_EINVAL, "usfft_sample_2d_static: z_j must be < M");
        ns.z[j] = z[j] < 0 ? -1 : z[j];
        ns.tail[j] = tails[j];
    }
    // scratch layout: [counters, 256 bytes][per-CTA slots of edge weights, diagonal and residual].
    // The mixed sampler assembles the coefficient in separable form from c and mu directly, so
    // it needs no mode table.
    const int n = pr.n;
    const size_t cnt_bytes = 256;
    const size_t slot_bytes = sample_2d_scratch_bytes(n, USFFT_MIXED, 1);
    if (cnt_bytes + slot_bytes > kStaticScratchBytes)
        return static_fail(USFFT_EINVAL, "usfft_sample_2d_static: the problem needs more than the 40 MiB static scratch");
    int blocks = sample_2d_default_blocks(n, USFFT_MIXED);
    const int fit = (int)((kStaticScratchBytes - cnt_bytes) / slot_bytes);
    if (blocks > fit) blocks = fit;

    // the per-device set-up comes before the count == 0 return, so that an empty call can
    // serve as the set-up call
    void* base = nullptr;
    usfft_status st = scratch_address(&base);
    if (st != USFFT_OK) return st;
    if (count == 0) {
        if (unconverged) *unconverged = 0;
        return USFFT_OK;
    }
    unsigned int* fails = reinterpret_cast<unsigned int*>(base);
    double* slots = reinterpret_cast<double*>(static_cast<unsigned char*>(base) + cnt_bytes);
    cudaStream_t s = (cudaStream_t)stream;

    cudaError_t e = cudaMemsetAsync(fails, 0, sizeof(unsigned int), s);   // the counter starts at zero
    if (e == cudaSuccess) {
        CgConfig cg;
        cg.precision = USFFT_MIXED;
        cg.max_iters = max_iters > 0 ? max_iters : 4000;
        cg.tol = tol > 0.0 ? tol : 1e-13;
        cg.blocks = blocks;
        cg.coef_scale = pr.coef_scale;
        cg.coef_decay = pr.coef_decay;
        e = launch_sample_2d(ns, n, pr.coef_model, pr.f_const, nullptr, cg, i0, count, U, nullptr, fails, nullptr, slots,
                             slot_bytes * (size_t)blocks, s, nullptr);
    }
    if (e != cudaSuccess) return static_fail(USFFT_ECUDA, std::string("usfft_sample_2d_static: ") + cudaGetErrorString(e));
    if (unconverged) {
        unsigned int h = 0;
        e = cudaMemcpyAsync(&h, fails, sizeof h, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess)
            return static_fail(USFFT_ECUDA, std::string("usfft_sample_2d_static: ") + cudaGetErrorString(e));
        *unconverged = h;
    }
    return USFFT_OK;
}
