// Evaluation of the sparse approximation and its errors (Section 4).
//
// u^usFFT(x_g, y) = sum_{k in I} c_{g,k} e^{2 pi i k.phi^-1(y)} (Eq. (3.1); phi^-1 the inverse
// parameter map, the identity for the periodic model) is a dense complex contraction
// V[j][g] = sum_k E[j][k] C[g][k] with E[j][k] = e^{2 pi i k.y~_j}, y~_j = phi^-1(y_j); with the FE solutions
// U[j][g] at the same points the errors of Section 4 are, per mesh node g,
//   err_2(x_g)   = ( (1/n) sum_j |U[j][g] - V[j][g]|^2 )^(1/2),
//   err_inf(x_g) = max_j |U[j][g] - V[j][g]|.
//
// The contraction runs in fp64 on the CUDA cores (FP64 tensor rates are low on this part):
// a 64 x 64 (point x node) tile per CTA, 4 x 4 per thread, k in chunks of 16.  E is formed
// on chip from the points and the int8 frequency rows: each product k_l y_jl is reduced
// mod 1 with its rounding error kept (fma), so the phase is accurate to the rounding of
// numbers in [-1/2, 1/2] for any |k|, then sincospi.  The error reduction is fused into
// the epilogue: per (point tile, node) partial sums of |U - V|^2 and maxima of |U - V|,
// reduced afterwards in a fixed order (bitwise reproducible).
#include <cuda_runtime.h>
#include <math.h>

#include "k_theta.cuh"
#include "usfft_internal.h"

namespace usfft {

namespace {

constexpr int TJ = 64, TG = 64, TK = 16, NT = 256;

__global__ void __launch_bounds__(NT) evaluate_kernel(const double* __restrict__ Y, int64_t n, int d,
                                                      const ParamMap pm, const int8_t* __restrict__ I, int64_t nI,
                                                      const double2* __restrict__ C, int G, double2* V,
                                                      const double* __restrict__ Uchk, double* part_sum,
                                                      double* part_max) {
    extern __shared__ double smem_d[];
    double2* Es = reinterpret_cast<double2*>(smem_d);        // [TK][TJ]
    double2* Cs = Es + TK * TJ;                               // [TK][TG]
    double* Ys = reinterpret_cast<double*>(Cs + TK * TG);     // [TJ][d]
    int8_t* Is = reinterpret_cast<int8_t*>(Ys + TJ * d);      // [TK][d]
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    const int64_t j0 = (int64_t)blockIdx.y * TJ;
    const int g0 = blockIdx.x * TG;

    for (int e = tid; e < TJ * d; e += NT) {
        const int jj = e / d;
        Ys[e] = (j0 + jj < n) ? to_torus(pm, Y[(j0 + jj) * d + (e - jj * d)]) : 0.0;
    }
    double2 acc[4][4];
#pragma unroll
    for (int p = 0; p < 4; ++p)
#pragma unroll
        for (int q = 0; q < 4; ++q) acc[p][q] = make_double2(0.0, 0.0);

    for (int64_t k0 = 0; k0 < nI; k0 += TK) {
        __syncthreads();   // previous chunk consumed (and Ys written, first time)
        for (int e = tid; e < TK * d; e += NT) {
            const int kk = e / d;
            Is[e] = (k0 + kk < nI) ? I[(k0 + kk) * d + (e - kk * d)] : (int8_t)0;
        }
        for (int e = tid; e < TK * TG; e += NT) {
            const int kk = e & (TK - 1), g = e / TK;
            Cs[kk * TG + g] = (k0 + kk < nI && g0 + g < G) ? C[(int64_t)(g0 + g) * nI + k0 + kk]
                                                          : make_double2(0.0, 0.0);
        }
        __syncthreads();
        for (int e = tid; e < TK * TJ; e += NT) {
            const int kk = e / TJ, jj = e - kk * TJ;
            const int8_t* kr = Is + kk * d;
            const double* yr = Ys + jj * d;
            double ph = 0.0;
            for (int l = 0; l < d; ++l) {
                if (!kr[l]) continue;
                const double kl = (double)kr[l];
                const double pr = kl * yr[l];
                ph += (pr - rint(pr)) + fma(kl, yr[l], -pr);
            }
            ph -= rint(ph);
            double sv, cv;
            sincospi(2.0 * ph, &sv, &cv);
            Es[kk * TJ + jj] = make_double2(cv, sv);
        }
        __syncthreads();
#pragma unroll 4
        for (int kk = 0; kk < TK; ++kk) {
            double2 ev[4], cv[4];
#pragma unroll
            for (int p = 0; p < 4; ++p) ev[p] = Es[kk * TJ + ty + 16 * p];
#pragma unroll
            for (int q = 0; q < 4; ++q) cv[q] = Cs[kk * TG + tx + 16 * q];
#pragma unroll
            for (int p = 0; p < 4; ++p)
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    acc[p][q].x = fma(ev[p].x, cv[q].x, fma(-ev[p].y, cv[q].y, acc[p][q].x));
                    acc[p][q].y = fma(ev[p].x, cv[q].y, fma(ev[p].y, cv[q].x, acc[p][q].y));
                }
        }
    }

    if (V) {
#pragma unroll
        for (int p = 0; p < 4; ++p) {
            const int64_t j = j0 + ty + 16 * p;
            if (j >= n) continue;
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int g = g0 + tx + 16 * q;
                if (g < G) V[j * G + g] = acc[p][q];
            }
        }
    }
    if (!Uchk) return;
    double ssum[4], smax[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        ssum[q] = 0.0;
        smax[q] = 0.0;
        const int g = g0 + tx + 16 * q;
#pragma unroll
        for (int p = 0; p < 4; ++p) {
            const int64_t j = j0 + ty + 16 * p;
            if (j >= n || g >= G) continue;
            const double dx = Uchk[j * G + g] - acc[p][q].x, dy = acc[p][q].y;
            const double a2 = dx * dx + dy * dy;
            ssum[q] += a2;
            smax[q] = fmax(smax[q], sqrt(a2));
        }
    }
    // reduce over the 16 thread rows (ty) that share a node, in a fixed order
    __syncthreads();
    double* rs = smem_d;                  // [16][TG] sums, then [16][TG] maxima
    double* rm = smem_d + 16 * TG;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        rs[ty * TG + tx + 16 * q] = ssum[q];
        rm[ty * TG + tx + 16 * q] = smax[q];
    }
    __syncthreads();
    if (tid < TG && g0 + tid < G) {
        double s = 0.0, m = 0.0;
        for (int r = 0; r < 16; ++r) {
            s += rs[r * TG + tid];
            m = fmax(m, rm[r * TG + tid]);
        }
        part_sum[(int64_t)blockIdx.y * G + g0 + tid] = s;
        part_max[(int64_t)blockIdx.y * G + g0 + tid] = m;
    }
}

// tot_sum[g] += sum over point tiles (in order), tot_max[g] = max(...)
__global__ void error_accumulate_kernel(const double* part_sum, const double* part_max, int tiles, int G,
                                        double* tot_sum, double* tot_max) {
    for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < G; g += gridDim.x * blockDim.x) {
        double s = 0.0, m = 0.0;
        for (int r = 0; r < tiles; ++r) {
            s += part_sum[(int64_t)r * G + g];
            m = fmax(m, part_max[(int64_t)r * G + g]);
        }
        tot_sum[g] += s;
        tot_max[g] = fmax(tot_max[g], m);
    }
}

// err2[g] = sqrt(tot_sum[g] / n) (in place), tot_max is err_inf already
__global__ void error_finalize_kernel(double* tot_sum, int G, double inv_n) {
    for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < G; g += gridDim.x * blockDim.x)
        tot_sum[g] = sqrt(tot_sum[g] * inv_n);
}

size_t eval_smem_bytes(int d) {
    return sizeof(double2) * (size_t)(TK * TJ + TK * TG) + sizeof(double) * (size_t)TJ * d + (size_t)TK * d + 16;
}

}  // namespace

int64_t evaluate_max_points() { return (int64_t)65535 * TJ; }
int evaluate_point_tile() { return TJ; }

cudaError_t launch_evaluate(const double* Y, int64_t n, int d, const ParamMap& pm, const int8_t* I, int64_t nI,
                            const double2* C, int G, double2* V, const double* Uchk, double* part_sum,
                            double* part_max, cudaStream_t s, int* launches) {
    if (n <= 0 || G <= 0) return cudaSuccess;
    if (n > evaluate_max_points()) return cudaErrorInvalidValue;
    const size_t smem = eval_smem_bytes(d);
    cudaError_t e = allow_dyn_smem((const void*)evaluate_kernel, smem);
    if (e != cudaSuccess) return e;
    dim3 grid((unsigned)((G + TG - 1) / TG), (unsigned)((n + TJ - 1) / TJ));
    evaluate_kernel<<<grid, NT, smem, s>>>(Y, n, d, pm, I, nI, C, G, V, Uchk, part_sum, part_max);
    if (launches) ++*launches;
    return cudaGetLastError();
}

cudaError_t launch_error_accumulate(const double* part_sum, const double* part_max, int tiles, int G, double* tot_sum,
                                    double* tot_max, cudaStream_t s, int* launches) {
    if (G <= 0 || tiles <= 0) return cudaSuccess;
    const int blocks = (G + 255) / 256;
    error_accumulate_kernel<<<blocks, 256, 0, s>>>(part_sum, part_max, tiles, G, tot_sum, tot_max);
    if (launches) ++*launches;
    return cudaGetLastError();
}

cudaError_t launch_error_finalize(double* tot_sum, int G, int64_t n, cudaStream_t s, int* launches) {
    if (G <= 0 || n <= 0) return cudaSuccess;
    error_finalize_kernel<<<(G + 255) / 256, 256, 0, s>>>(tot_sum, G, 1.0 / (double)n);
    if (launches) ++*launches;
    return cudaGetLastError();
}

}  // namespace usfft
