// Quantities of interest of the sparse approximation (Sec. 4 and 4.1): expectation,
// variance and the global sensitivity indices of the sets J_l (Eq. (4.3), (4.4)).
//
// E(u^usFFT(x_g, .)) = sum_k c_{g,k} D_k with D_k = prod_j D_{k_j}: 1 for k_j = 0; for k_j != 0
// zero in the periodic model, 2i/(pi k_j) for odd and 0 for even k_j under the tent map
// (Eq. (4.5)), and that times e^{2 pi i k_j Delta} under the lognormal map.  The variance is
// sum_{k != 0} |c_{g,k}|^2 and rho(J_l) its share carried by the k with l non-zero components.
//
// The D_k depend on k only (one small kernel); the per-node pass reads the node's row of C
// once (HBM-bound: 16 bytes per coefficient), one warp per node, the frequencies visited
// group by group (order l) through a permutation so that each group's sum is a plain warp
// reduction in a fixed order.
#include <cuda_runtime.h>
#include <math.h>

#include "usfft_internal.h"

namespace usfft {

namespace {

__global__ void expectation_factors_kernel(const int8_t* I, int64_t nI, int d, const ParamMap pm, double2* dfac) {
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < nI; k += (int64_t)gridDim.x * blockDim.x) {
        double re = 1.0, im = 0.0;
        for (int j = 0; j < d; ++j) {
            const int kj = I[k * d + j];
            if (kj == 0) continue;
            if (pm.map == USFFT_MAP_PERIODIC || (kj & 1) == 0) {
                re = 0.0;
                im = 0.0;
                break;
            }
            // factor 2i / (pi k_j), times e^{2 pi i k_j Delta} under the lognormal map
            double fr = 0.0, fi = 2.0 / (M_PI * (double)kj);
            if (pm.map == USFFT_MAP_NORMAL) {
                double sv, cv;
                sincospi(2.0 * (double)kj * pm.shift, &sv, &cv);
                const double gr = -fi * sv, gi = fi * cv;    // (i fi) (cv + i sv)
                fr = gr;
                fi = gi;
            }
            const double nr = re * fr - im * fi, ni = re * fi + im * fr;
            re = nr;
            im = ni;
        }
        dfac[k] = make_double2(re, im);
    }
}

__device__ __forceinline__ double warp_sum_d(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__global__ void statistics_kernel(const double2* __restrict__ C, int G, int64_t nI, int d,
                                  const double2* __restrict__ dfac, const int* __restrict__ perm,
                                  const int64_t* __restrict__ offsets, double2* mean, double* var, double* gsi) {
    const int lane = threadIdx.x & 31;
    const int warps = blockDim.x >> 5;
    for (int g = blockIdx.x * warps + (threadIdx.x >> 5); g < G; g += gridDim.x * warps) {
        const double2* row = C + (int64_t)g * nI;
        double mr = 0.0, mi = 0.0, v = 0.0;
        // order 0 (k = 0): the mean only
        for (int64_t a = offsets[0] + lane; a < offsets[1]; a += 32) {
            const int k = perm[a];
            const double2 c = row[k], f = dfac[k];
            mr += c.x * f.x - c.y * f.y;
            mi += c.x * f.y + c.y * f.x;
        }
        for (int l = 1; l <= d; ++l) {
            double part = 0.0;
            for (int64_t a = offsets[l] + lane; a < offsets[l + 1]; a += 32) {
                const int k = perm[a];
                const double2 c = row[k], f = dfac[k];
                mr += c.x * f.x - c.y * f.y;
                mi += c.x * f.y + c.y * f.x;
                part += c.x * c.x + c.y * c.y;
            }
            part = warp_sum_d(part);
            v += part;
            if (gsi && lane == 0) gsi[(int64_t)g * d + (l - 1)] = part;   // scaled below
        }
        mr = warp_sum_d(mr);
        mi = warp_sum_d(mi);
        if (lane == 0) {
            if (mean) mean[g] = make_double2(mr, mi);
            if (var) var[g] = v;
        }
        if (gsi) {
            __syncwarp();
            for (int l = lane; l < d; l += 32) {
                double* p = gsi + (int64_t)g * d + l;
                *p = v > 0.0 ? *p / v : 0.0;
            }
        }
    }
}

}  // namespace

cudaError_t launch_expectation_factors(const int8_t* I, int64_t nI, int d, const ParamMap& pm, double2* dfac,
                                       cudaStream_t s, int* launches) {
    if (nI <= 0) return cudaSuccess;
    int64_t blocks = (nI + 255) / 256;
    if (blocks > 152 * 8) blocks = 152 * 8;
    expectation_factors_kernel<<<(unsigned)blocks, 256, 0, s>>>(I, nI, d, pm, dfac);
    if (launches) ++*launches;
    return cudaGetLastError();
}

cudaError_t launch_statistics(const double2* C, int G, int64_t nI, int d, const double2* dfac, const int* perm,
                              const int64_t* offsets, double2* mean, double* var, double* gsi, cudaStream_t s,
                              int* launches) {
    if (G <= 0) return cudaSuccess;
    const int warps = 8;
    int blocks = (G + warps - 1) / warps;
    if (blocks > 152 * 16) blocks = 152 * 16;
    statistics_kernel<<<blocks, 32 * warps, 0, s>>>(C, G, nI, d, dfac, perm, offsets, mean, var, gsi);
    if (launches) ++*launches;
    return cudaGetLastError();
}

}  // namespace usfft
