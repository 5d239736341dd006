// Black-box sampler, part 1: the mode table psi_j(centroid_e) (2-D and 1-D) and the 1-D
// sampler (fused coefficient assembly + cyclic reduction).
//
// Problem: Eq. (1.1) on (0,1), P1 elements of width h = 1/(n+1), coefficient of element
// e taken at its midpoint, f constant (the paper's FE black box, Sec. 2.1).  Scaled by h,
// the stiffness system of interior node p (1..n) reads
//   -a_{p-1} u_{p-1} + (a_{p-1} + a_p) u_p - a_p u_{p+1} = h^2 f,
// with a_e the coefficient of element e = [x_e, x_{e+1}] and u_0 = u_{n+1} = 0.
//
// One warp solves one system by cyclic reduction: the system is padded to
// NP = 2^q - 1 equations (identity rows), even positions are eliminated level by
// level (stride s = 1, 2, 4, ...), the middle equation is solved, and the eliminated
// unknowns are recovered in reverse order.  Equations of one level are independent and
// spread over the 32 lanes; levels are separated by __syncwarp().
#include <cuda_runtime.h>
#include <math.h>

#include "k_theta.cuh"
#include "usfft_internal.h"

namespace usfft {

// ---------------------------------------------------------------------------------
// psi[j][e] = c (j+1)^-mu psi_{j+1}(centroid_e)
// ---------------------------------------------------------------------------------
__device__ __forceinline__ void mode_2d(int j, int& j1, int& j2) {
    // diagonal enumeration of Sec. 4.2 / Table 4.2 applied to j-1, shifted by one
    int jm = j - 1;
    int k = 0;
    while ((k + 1) * (k + 2) / 2 <= jm) ++k;
    int m1 = jm - k * (k + 1) / 2;
    j1 = m1 + 1;
    j2 = (k - m1) + 1;
}

__global__ void psi_table_kernel(int kind, int n, int d, double scale, double decay, double* psi) {
    const double h = 1.0 / (double)(n + 1);
    const int64_t E = (kind == USFFT_PDE_1D) ? (int64_t)(n + 1) : 2LL * (n + 1) * (n + 1);
    const int64_t total = E * d;
    for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
         idx += (int64_t)gridDim.x * blockDim.x) {
        int j = (int)(idx / E) + 1;
        int64_t e = idx % E;
        double amp = scale * pow((double)j, -decay);
        double v;
        if (kind == USFFT_PDE_1D) {
            double x = ((double)e + 0.5) * h;
            v = sinpi((double)j * x);
        } else {
            int64_t sq = (n + 1) * (int64_t)(n + 1);
            bool upper = e >= sq;
            int64_t es = upper ? e - sq : e;
            int P = (int)(es % (n + 1)), Q = (int)(es / (n + 1));
            // lower triangle {(P,Q),(P+1,Q),(P+1,Q+1)}, upper {(P,Q),(P+1,Q+1),(P,Q+1)}
            double x1 = upper ? ((double)P + 1.0 / 3.0) * h : ((double)P + 2.0 / 3.0) * h;
            double x2 = upper ? ((double)Q + 2.0 / 3.0) * h : ((double)Q + 1.0 / 3.0) * h;
            int j1, j2;
            mode_2d(j, j1, j2);
            v = sinpi((double)j1 * x1) * sinpi((double)j2 * x2);
        }
        psi[idx] = amp * v;
    }
}

cudaError_t launch_psi_table(int kind, int n, int d, double scale, double decay, double* psi,
                             cudaStream_t s) {
    int64_t E = (kind == USFFT_PDE_1D) ? (int64_t)(n + 1) : 2LL * (n + 1) * (n + 1);
    int64_t total = E * d;
    int blocks = (int)((total + 255) / 256);
    if (blocks > 4096) blocks = 4096;
    if (blocks < 1) blocks = 1;
    psi_table_kernel<<<blocks, 256, 0, s>>>(kind, n, d, scale, decay, psi);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------------
// 1-D sampler
// ---------------------------------------------------------------------------------
struct Cr1dArgs {
    NodeSpec ns;
    int n, NP, coef_model;
    double rhs;                  // h^2 f
    const double* psi;           // [d][n+1]
    int64_t i0, count;
    double* U;                   // [count][n]
};

__global__ void __launch_bounds__(256) sample_1d_cr_kernel(const __grid_constant__ Cr1dArgs a) {
    extern __shared__ double smem[];
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int warps = blockDim.x >> 5;
    const int NP = a.NP;
    const int d = a.ns.d;
    const int n = a.n;
    // per warp: sub, diag, sup, rhs on positions 0..NP+1, coefficients (n+1), sines (d)
    const int W = NP + 2;
    double* base = smem + (size_t)warp * (4 * W + (n + 1) + d);
    double* sub = base;
    double* dia = sub + W;
    double* sup = dia + W;
    double* rhs = sup + W;
    double* ae = rhs + W;
    double* sj = ae + (n + 1);

    for (int64_t sys = (int64_t)blockIdx.x * warps + warp; sys < a.count; sys += (int64_t)gridDim.x * warps) {
        const int64_t i = lattice_node(a.ns, a.i0 + sys);
        for (int j = lane; j < d; j += 32) sj[j] = node_theta(a.ns, j, i);
        __syncwarp();
        // element coefficients (fused assembly; never stored in HBM)
        for (int e = lane; e <= n; e += 32) {
            double acc = 0.0;
            for (int j = 0; j < d; ++j) acc = fma(a.psi[(size_t)j * (n + 1) + e], sj[j], acc);
            ae[e] = (a.coef_model == USFFT_COEF_LOGNORMAL_SIN) ? exp(acc) : 1.0 + acc;
        }
        __syncwarp();
        for (int p = lane + 1; p <= NP; p += 32) {
            if (p <= n) {
                sub[p] = (p > 1) ? -ae[p - 1] : 0.0;
                dia[p] = ae[p - 1] + ae[p];
                sup[p] = (p < n) ? -ae[p] : 0.0;
                rhs[p] = a.rhs;
            } else {
                sub[p] = 0.0;
                dia[p] = 1.0;
                sup[p] = 0.0;
                rhs[p] = 0.0;
            }
        }
        __syncwarp();
        // forward reduction
        int s = 1;
        for (; 2 * s <= NP; s *= 2) {
            for (int p = 2 * s * (lane + 1); p <= NP; p += 2 * s * 32) {
                double al = -sub[p] / dia[p - s];
                double ga = -sup[p] / dia[p + s];
                dia[p] = dia[p] + al * sup[p - s] + ga * sub[p + s];
                rhs[p] = rhs[p] + al * rhs[p - s] + ga * rhs[p + s];
                sub[p] = al * sub[p - s];
                sup[p] = ga * sup[p + s];
            }
            __syncwarp();
        }
        // middle equation (position (NP+1)/2) couples to nothing inside
        if (lane == 0) {
            int mid = (NP + 1) / 2;
            rhs[mid] = rhs[mid] / dia[mid];
        }
        __syncwarp();
        // back substitution; rhs[p] is overwritten by u_p
        for (s = (NP + 1) / 4; s >= 1; s /= 2) {
            for (int p = s * (2 * lane + 1); p <= NP; p += 2 * s * 32) {
                double ul = (p - s >= 1) ? rhs[p - s] : 0.0;
                double ur = (p + s <= NP) ? rhs[p + s] : 0.0;
                rhs[p] = (rhs[p] - sub[p] * ul - sup[p] * ur) / dia[p];
            }
            __syncwarp();
        }
        double* out = a.U + (size_t)sys * n;
        for (int g = lane; g < n; g += 32) out[g] = rhs[g + 1];
        __syncwarp();
    }
}

cudaError_t launch_sample_1d(const NodeSpec& ns, int n, int coef_model, double f, const double* psi,
                             int64_t i0, int64_t count, double* U, cudaStream_t s, int* launches) {
    if (count <= 0) return cudaSuccess;
    Cr1dArgs a;
    a.ns = ns;
    a.n = n;
    int NP = 1;
    while (NP < n) NP = 2 * NP + 1;
    a.NP = NP;
    a.coef_model = coef_model;
    double h = 1.0 / (double)(n + 1);
    a.rhs = h * h * f;
    a.psi = psi;
    a.i0 = i0;
    a.count = count;
    a.U = U;
    size_t per_warp = sizeof(double) * (size_t)(4 * (NP + 2) + (n + 1) + ns.d);
    int warps = (int)(96 * 1024 / per_warp);
    if (warps > 8) warps = 8;
    if (warps < 1) warps = 1;
    size_t smem = per_warp * warps;
    if (smem > 48 * 1024) {
        cudaError_t e = allow_dyn_smem((const void*)sample_1d_cr_kernel, smem);
        if (e != cudaSuccess) return e;
    }
    int64_t blocks = (count + warps - 1) / warps;
    if (blocks > 152 * 16) blocks = 152 * 16;
    sample_1d_cr_kernel<<<(unsigned)blocks, warps * 32, smem, s>>>(a);
    if (launches) ++*launches;
    return cudaGetLastError();
}

}  // namespace usfft
