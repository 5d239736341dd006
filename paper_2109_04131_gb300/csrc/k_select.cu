// Per-node thresholding and union of the detected sets (Algorithm 1, steps 1/2a and 2d-2e).
//
// Node g keeps the indices of the at most s~ largest |C[g][k]| that are >= theta; the
// union over nodes (and detection iterations) is an OR into one bitmap over the
// candidates.  Readings shared with the oracle: |c|^2 = re*re + im*im with every
// operation rounded separately (no FMA), compared with theta*theta; equal magnitudes
// are ordered by the smaller candidate index.
//
// One CTA per node.  If at most s~ candidates pass the threshold they are all taken.
// Otherwise the s~-th largest magnitude is found exactly by an MSB-first radix select
// over the bit patterns of |c|^2 (non-negative doubles order like their bits), eight
// 8-bit digits with a 256-bin shared histogram; then every key above it is taken and the
// remaining quota of keys equal to it goes to the smallest indices (warp ballots and
// prefix counts over index-ordered chunks).  The digit passes scan a compacted list instead of
// all candidates once the keys still in play fit it (at most kSelList: right after the keys are
// formed when few pass the threshold, else once the selected digit's bucket is that small).
#include <cuda_runtime.h>

#include "usfft_internal.h"

namespace usfft {

static const int kSelThreads = 256;
static const int kSelList = 1024;   // keys of the selected radix bucket compacted once it holds at most this many

__device__ __forceinline__ double mag2_rn(double2 c) {
    return __dadd_rn(__dmul_rn(c.x, c.x), __dmul_rn(c.y, c.y));
}

// key of a magnitude: 1 + its bit pattern if m2 >= theta^2, else 0.  The comparison is done
// on the bit patterns (non-negative doubles order like their bits; the bound at the pattern
// of +inf keeps a nan out, as the fp64 comparison would), on the integer pipe: on this GPU
// the fp64 comparison issues at the FP64 pipe's rate (1/64 of FP32).
__device__ __forceinline__ unsigned long long key_bits(double m2, unsigned long long tbits) {
    const unsigned long long mb = (unsigned long long)__double_as_longlong(m2);
    return (mb >= tbits && mb <= 0x7ff0000000000000ull) ? mb + 1ull : 0ull;
}

__device__ __forceinline__ void set_bit(uint32_t* bitmap, int64_t k) {
    atomicOr(bitmap + (k >> 5), 1u << (k & 31));
}

// Keys: 1 + bit pattern of |c|^2 for candidates >= theta, 0 for the others (the bit patterns
// of non-negative doubles are ordered like the values; +1 keeps a zero magnitude eligible
// when theta = 0).  With KEYS_IN_SMEM the keys of a node are computed once (three fp64
// operations per candidate) into shared memory and every radix pass is integer work;
// otherwise (more candidates than fit) they are recomputed from C in every pass.
// The union of a CTA's nodes is collected in a shared-memory bitmap (sbits, when it fits) and
// OR-ed into the global one once at the end: every node sets up to s~ bits, mostly the same
// frequencies, and one global atomic per bit would contend on a few words of L2.
template <bool KEYS_IN_SMEM>
__global__ void __launch_bounds__(kSelThreads) select_union_kernel(const double2* C, int G, int64_t nJ,
                                                                     double theta2, int s_tilde, uint32_t* bitmap,
                                                                     bool local_bits) {
    extern __shared__ unsigned long long skeys[];
    const int64_t nwords = (nJ + 31) / 32;
    uint32_t* sbits = reinterpret_cast<uint32_t*>(skeys + (KEYS_IN_SMEM ? nJ : 0));
    uint32_t* bits = local_bits ? sbits : bitmap;
    __shared__ unsigned int hist[256];
    __shared__ unsigned long long sh_prefix;
    __shared__ unsigned int sh_want;
    __shared__ unsigned int warp_cnt[kSelThreads / 32];
    __shared__ unsigned int sh_total;
    __shared__ unsigned int sh_bucket, sh_listn;
    __shared__ unsigned long long slist[kSelList];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int nw = blockDim.x >> 5;
    if (local_bits) {
        for (int64_t w = tid; w < nwords; w += blockDim.x) sbits[w] = 0u;
        __syncthreads();
    }

    const unsigned long long tbits = theta2 > 0.0 ? (unsigned long long)__double_as_longlong(theta2) : 0ull;
    for (int g = blockIdx.x; g < G; g += gridDim.x) {
        const double2* row = C + (int64_t)g * nJ;
        auto key_of = [&](int64_t k) -> unsigned long long {
            if (KEYS_IN_SMEM) return skeys[k];
            const double m2 = mag2_rn(row[k]);
            return key_bits(m2, tbits);
        };
        // pass 0: keys and the count of candidates above the threshold
        unsigned int cnt = 0;
        for (int64_t k = tid; k < nJ; k += blockDim.x) {
            const double m2 = mag2_rn(row[k]);
            const unsigned long long key = key_bits(m2, tbits);
            if (KEYS_IN_SMEM) skeys[k] = key;
            cnt += key ? 1u : 0u;
        }
        cnt = __reduce_add_sync(0xffffffffu, cnt);
        if (lane == 0) warp_cnt[warp] = cnt;
        __syncthreads();
        if (tid == 0) {
            unsigned int t = 0;
            for (int w = 0; w < nw; ++w) t += warp_cnt[w];
            sh_total = t;
            sh_prefix = 0ull;
            sh_want = (unsigned int)s_tilde;
        }
        __syncthreads();
        const unsigned int total = sh_total;
        if (total <= (unsigned int)s_tilde) {
            for (int64_t k = tid; k < nJ; k += blockDim.x)
                if (key_of(k)) set_bit(bits, k);
            __syncthreads();
            continue;
        }
        // exact s~-th largest key: MSB-first radix select, 8-bit digits.  Once the selected digit's bucket
        // holds at most kSelList keys they are copied to slist and the later passes scan only them
        // (every other key fails their prefix test anyway)
        int listn = -1;
        if (total <= (unsigned int)kSelList) {      // few keys above the threshold: compact them right away
            if (tid == 0) sh_listn = 0u;
            __syncthreads();
            for (int64_t k = tid; k < nJ; k += blockDim.x) {
                const unsigned long long key = key_of(k);
                if (key) slist[atomicAdd(&sh_listn, 1u)] = key;
            }
            __syncthreads();
            listn = (int)sh_listn;
        }
        for (int shift = 56; shift >= 0; shift -= 8) {
            hist[tid] = 0u;     // blockDim.x == 256
            __syncthreads();
            const unsigned long long prefix = sh_prefix;
            const unsigned long long himask = (shift == 56) ? 0ull : ~((1ull << (shift + 8)) - 1ull);
            if (listn < 0) {
                for (int64_t k = tid; k < nJ; k += blockDim.x) {
                    const unsigned long long key = key_of(k);
                    if (key && (key & himask) == prefix) atomicAdd(&hist[(key >> shift) & 255ull], 1u);
                }
            } else {
                for (int q = tid; q < listn; q += blockDim.x) {
                    const unsigned long long key = slist[q];
                    if ((key & himask) == prefix) atomicAdd(&hist[(key >> shift) & 255ull], 1u);
                }
            }
            __syncthreads();
            if (warp == 0) {
                // warp-parallel scan from the top digit: lane l owns digits 255-8l .. 248-8l
                const unsigned int want = sh_want;
                unsigned int c[8], own = 0;
#pragma unroll
                for (int q = 0; q < 8; ++q) {
                    c[q] = hist[255 - 8 * lane - q];
                    own += c[q];
                }
                unsigned int incl = own;             // inclusive prefix over lanes 0..lane
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const unsigned int v = __shfl_up_sync(0xffffffffu, incl, o);
                    if (lane >= o) incl += v;
                }
                const unsigned int excl = incl - own;   // keys with a larger digit than this lane's range
                const bool hit = excl < want && want <= incl;
                if (hit) {
                    unsigned int cum = excl;
                    int dsel = 255 - 8 * lane;
                    unsigned int cnt_sel = 0;
#pragma unroll
                    for (int q = 0; q < 8; ++q) {
                        if (cum + c[q] >= want) {
                            dsel = 255 - 8 * lane - q;
                            cnt_sel = c[q];
                            break;
                        }
                        cum += c[q];
                    }
                    sh_want = want - cum;
                    sh_prefix = prefix | ((unsigned long long)dsel << shift);
                    sh_bucket = cnt_sel;
                }
            }
            __syncthreads();
            if (listn < 0 && shift > 0 && sh_bucket <= (unsigned int)kSelList) {
                if (tid == 0) sh_listn = 0u;
                __syncthreads();
                const unsigned long long mask = ~((1ull << shift) - 1ull), pfx = sh_prefix;
                for (int64_t k = tid; k < nJ; k += blockDim.x) {
                    const unsigned long long key = key_of(k);
                    if (key && (key & mask) == pfx) slist[atomicAdd(&sh_listn, 1u)] = key;
                }
                __syncthreads();
                listn = (int)sh_listn;
            }
        }
        const unsigned long long tau = sh_prefix;
        const unsigned int take_eq = sh_want;        // how many keys == tau to take
        for (int64_t k = tid; k < nJ; k += blockDim.x)
            if (key_of(k) > tau) set_bit(bits, k);
        // keys equal to tau: the first take_eq in index order
        unsigned int taken = 0;
        for (int64_t base = 0; base < nJ && taken < take_eq; base += blockDim.x) {
            const int64_t k = base + tid;
            const bool eq = (k < nJ) && key_of(k) == tau;
            const unsigned int ball = __ballot_sync(0xffffffffu, eq);
            if (lane == 0) warp_cnt[warp] = __popc(ball);
            __syncthreads();
            unsigned int before = taken;
            for (int w = 0; w < warp; ++w) before += warp_cnt[w];
            before += __popc(ball & ((1u << lane) - 1u));
            if (eq && before < take_eq) set_bit(bits, k);
            unsigned int chunk = 0;
            for (int w = 0; w < nw; ++w) chunk += warp_cnt[w];
            __syncthreads();
            taken += chunk;
        }
        __syncthreads();
    }
    if (local_bits) {
        __syncthreads();
        for (int64_t w = tid; w < nwords; w += blockDim.x)
            if (sbits[w]) atomicOr(bitmap + w, sbits[w]);
    }
}

static const int64_t kMaxSmemKeys = 24576;   // 192 KB of keys (+ 3 KB of bitmap) per CTA

cudaError_t launch_select_union(const double2* C, int G, int64_t nJ, double theta, int s_tilde, uint32_t* bitmap,
                                cudaStream_t s, int* launches) {
    if (G <= 0 || nJ <= 0) return cudaSuccess;
    cudaError_t e;
    const size_t bits_bytes = sizeof(uint32_t) * (size_t)((nJ + 31) / 32);
    if (nJ <= kMaxSmemKeys) {
        const size_t smem = sizeof(unsigned long long) * (size_t)nJ + bits_bytes;
        e = allow_dyn_smem((const void*)select_union_kernel<true>, smem);
        if (e != cudaSuccess) return e;
        int per_sm = 0;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, select_union_kernel<true>, kSelThreads, smem);
        if (e != cudaSuccess || per_sm < 1) {
            cudaGetLastError();
            per_sm = 1;
        }
        int blocks = 152 * per_sm;
        if (blocks > G) blocks = G;
        select_union_kernel<true><<<blocks, kSelThreads, smem, s>>>(C, G, nJ, theta * theta, s_tilde, bitmap, true);
    } else {
        int blocks = G < 152 * 8 ? G : 152 * 8;
        const bool local = bits_bytes <= 32768;          // 1M candidates
        const size_t smem = local ? bits_bytes : 0;
        if (local) {
            e = allow_dyn_smem((const void*)select_union_kernel<false>, smem);
            if (e != cudaSuccess) return e;
        }
        select_union_kernel<false><<<blocks, kSelThreads, smem, s>>>(C, G, nJ, theta * theta, s_tilde, bitmap, local);
    }
    if (launches) ++*launches;
    return cudaGetLastError();
}

__global__ void absmax_column_kernel(const double2* C, int G, int64_t nJ, int64_t col, double* out) {
    __shared__ double red[32];
    double m = 0.0;
    for (int g = threadIdx.x; g < G; g += blockDim.x) {
        const double2 c = C[(int64_t)g * nJ + col];
        m = fmax(m, hypot(c.x, c.y));
    }
    for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t = fmax(t, red[w]);
        *out = t;
    }
}

cudaError_t launch_absmax_column(const double2* C, int G, int64_t nJ, int64_t col, double* out, cudaStream_t s,
                                 int* launches) {
    absmax_column_kernel<<<1, 1024, 0, s>>>(C, G, nJ, col, out);
    if (launches) ++*launches;
    return cudaGetLastError();
}

}  // namespace usfft
