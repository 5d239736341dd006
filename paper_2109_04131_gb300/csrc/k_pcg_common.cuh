// Device helpers shared by the 2-D sampler kernels (k_sample2d.cu, k_sample2d_dst.cu).
#pragma once
#include <cuda_runtime.h>
#include <math.h>

#include "k_theta.cuh"
#include "usfft_internal.h"

namespace usfft {

struct Pcg2dArgs {
    NodeSpec ns;
    int n, coef_model, max_iters;
    double rhs;            // h^2 f
    double tol;            // relative residual target (fp64 / refinement)
    double tol_inner;      // relative residual target of an fp32 inner solve
    const double* psi;     // [d][2(n+1)^2]
    int64_t i0, count;
    double* U;             // [count][n*n]
    int* iters_out;
    unsigned int* fail_count;
    unsigned long long* iters_sum;   // total CG iterations of the launch (may be NULL)
    unsigned long long* outer_sum;   // total refinement steps of the launch (mixed; may be NULL)
    double* scratch;       // refinement kernels: per-CTA fp64 weight slots
    double coef_scale;     // c, mu (separable assembly of the MIXED kernel)
    double coef_decay;
};

// Spatial mode of the 2-D coefficient: (j1, j2) = (m1(j-1)+1, m2(j-1)+1) with the diagonal
// enumeration of Sec. 4.2 / Table 4.2.
__host__ __device__ inline void mode_pair(int j, int& j1, int& j2) {
    const int jm = j - 1;
    int k = 0;
    while ((k + 1) * (k + 2) / 2 <= jm) ++k;
    const int m1 = jm - k * (k + 1) / 2;
    j1 = m1 + 1;
    j2 = (k - m1) + 1;
}

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Block-wide sum plus one scalar ratio, computed once by thread 0 and broadcast:
// ratio = num / sum (NUM_OVER_SUM) or sum / den (SUM_OVER_DEN).  `buf` holds 34 values.
// Every thread of the block must call it (two barriers).
enum { NUM_OVER_SUM = 0, SUM_OVER_DEN = 1 };
template <typename T, int MODE>
__device__ __forceinline__ void block_sum_ratio(T v, T other, T* buf, T& sum, T& ratio) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    v = warp_sum(v);
    if (lane == 0) buf[warp] = v;
    __syncthreads();
    if (warp == 0) {
        T w = lane < nw ? buf[lane] : (T)0;
        w = warp_sum(w);
        if (lane == 0) {
            buf[32] = w;
            buf[33] = (MODE == NUM_OVER_SUM) ? other / w : w / other;
        }
    }
    __syncthreads();
    sum = buf[32];
    ratio = buf[33];
}

// Block-wide sum; `buf` holds 33 doubles; the result is returned to every thread.
__device__ __forceinline__ double block_sum(double v, double* buf) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    v = warp_sum(v);
    if (lane == 0) buf[warp] = v;
    __syncthreads();
    if (warp == 0) {
        double w = lane < nw ? buf[lane] : 0.0;
        w = warp_sum(w);
        if (lane == 0) buf[32] = w;
    }
    __syncthreads();
    return buf[32];
}


}  // namespace usfft
