// Coefficient estimate of the random rank-1 lattice detection (random R1L approach in the
// role of Algorithm A).  Every candidate k has L lattice values c_l(k) = (1/M_l) FFT_l at
// k.z_l mod M_l (gathered into Call[l][g][k] by the FFT passes).  Where k is alone at its
// index in some lattice (no other candidate of J_t shares it) the first such lattice's value
// is taken (it is what a reconstructing lattice gives); otherwise the median over the L
// values, separately for the real and the imaginary part (L odd, so the median is one of the
// values).  One thread per (g, k); consecutive threads take consecutive k (coalesced).  Step 3 on
// multiple rank-1 lattices uses the first half only (lattice_pick_kernel): there every k of I is
// alone in some lattice by construction.
#include <cuda_runtime.h>

#include "usfft_internal.h"

namespace usfft {

namespace {

constexpr int kMaxLattices = 31;

__device__ __forceinline__ double median_odd(double* v, int L) {
    // insertion sort of at most 31 values, then the middle one
    for (int a = 1; a < L; ++a) {
        const double x = v[a];
        int b = a - 1;
        while (b >= 0 && v[b] > x) {
            v[b + 1] = v[b];
            --b;
        }
        v[b + 1] = x;
    }
    return v[L / 2];
}

__global__ void random_lattice_combine_kernel(const double2* __restrict__ Call, int L, int G, int64_t nJ,
                                              const int* __restrict__ src, double2* C) {
    const int64_t total = (int64_t)G * nJ;
    const int64_t plane = total;
    for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
         idx += (int64_t)gridDim.x * blockDim.x) {
        const int64_t k = idx % nJ;
        const int s = src[k];
        if (s >= 0) {
            C[idx] = Call[(int64_t)s * plane + idx];
            continue;
        }
        double re[kMaxLattices], im[kMaxLattices];
        for (int l = 0; l < L; ++l) {
            const double2 v = Call[(int64_t)l * plane + idx];
            re[l] = v.x;
            im[l] = v.y;
        }
        C[idx] = make_double2(median_odd(re, L), median_odd(im, L));
    }
}

// Step 3 on multiple rank-1 lattices: every k of I is alone at its index in some lattice by
// construction, and its value is taken from the first such lattice src[k]; an index outside
// [0, L) (which the host never passes) gives NaN rather than a read outside Call.
__global__ void lattice_pick_kernel(const double2* __restrict__ Call, int L, int G, int64_t nJ,
                                    const int* __restrict__ src, double2* C) {
    const int64_t total = (int64_t)G * nJ;
    for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
         idx += (int64_t)gridDim.x * blockDim.x) {
        const int s = src[idx % nJ];
        C[idx] = (s >= 0 && s < L) ? Call[(int64_t)s * total + idx] : make_double2(__longlong_as_double(0x7ff8000000000000ll),
                                                                                 __longlong_as_double(0x7ff8000000000000ll));
    }
}

}  // namespace

cudaError_t launch_lattice_pick(const double2* Call, int L, int G, int64_t nJ, const int* src, double2* C,
                                cudaStream_t s, int* launches) {
    if (G <= 0 || nJ <= 0) return cudaSuccess;
    if (L < 1) return cudaErrorInvalidValue;
    int64_t blocks = ((int64_t)G * nJ + 255) / 256;
    if (blocks > 152 * 16) blocks = 152 * 16;
    lattice_pick_kernel<<<(unsigned)blocks, 256, 0, s>>>(Call, L, G, nJ, src, C);
    if (launches) ++*launches;
    return cudaGetLastError();
}

cudaError_t launch_random_lattice_combine(const double2* Call, int L, int G, int64_t nJ, const int* src, double2* C,
                                          cudaStream_t s, int* launches) {
    if (G <= 0 || nJ <= 0) return cudaSuccess;
    if (L < 1 || L > kMaxLattices || (L & 1) == 0) return cudaErrorInvalidValue;
    int64_t blocks = ((int64_t)G * nJ + 255) / 256;
    if (blocks > 152 * 16) blocks = 152 * 16;
    random_lattice_combine_kernel<<<(unsigned)blocks, 256, 0, s>>>(Call, L, G, nJ, src, C);
    if (launches) ++*launches;
    return cudaGetLastError();
}

}  // namespace usfft
