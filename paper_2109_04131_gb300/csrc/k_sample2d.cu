// Black-box sampler, part 2: the 2-D FE solve at every lattice node (Eq. (1.1) on the
// unit square; the paper's FE black box, Sec. 2.1), fused with the coefficient assembly.
//
// Discretisation (the same reading as the oracle): n*n interior nodes, h = 1/(n+1), each
// square split along its "/" diagonal, P1 elements, element coefficient a_T at the
// centroid, f constant (load h^2 f per node).  On right isosceles triangles the P1
// coupling across the hypotenuse vanishes, so the stiffness matrix is the 5-point
// operator whose off-diagonal entry on an axis-parallel edge is -w_e,
// w_e = (a_T1 + a_T2)/2 over the two triangles sharing the edge, and whose diagonal is
// the sum of the four edge weights.  The matrix is never stored: one CTA assembles the
// edge weights of its system in shared memory (one pattern for all systems).
//
// Solver: conjugate gradients on the symmetrically Jacobi-scaled system
//   (D^-1/2 K D^-1/2) x~ = D^-1/2 b,  x = D^-1/2 x~,
// which produces the iterates of Jacobi-preconditioned CG with fewer fp64 operations
// per node and iteration (unit diagonal, z = r).  Stopping: ||r~|| <= tol ||b~||.
//   FP64:  the whole CG in fp64.
//   MIXED: fp32 CG inner solves on the scaled operator and fp64 iterative refinement:
//          r~ = b~ - K~ x~ is formed in fp64 with the fp64 edge weights, the correction
//          solves K~ d = r~ / ||r~|| in fp32, x~ += ||r~|| d in fp64.
// One CTA owns one system at a time (persistent grid); node g = tid + k*T, k < NPT.
#include <cuda_runtime.h>
#include <math.h>

#include "usfft_internal.h"
#include "k_pcg_common.cuh"

namespace usfft {

// DST-preconditioned mixed kernel (k_sample2d_dst.cu)
size_t dst_smem_bytes(int n, int d);
template <int NPT>
cudaError_t launch_dst_npt(const Pcg2dArgs& a, int blocks, int threads, cudaStream_t s);
cudaError_t launch_mixed_big(const Pcg2dArgs& a, int blocks, cudaStream_t s);
template <int NPT>
int dst_resident_blocks(int threads, int d, int n);
// fp64 sampler with the same preconditioner (k_sample2d_dst64.cu)
size_t fp64_dst_slot_bytes(int n, int d);
size_t mixed_slot_bytes(int n);
int fp64_dst_default_blocks(int n, int d);
cudaError_t launch_fp64_dst(const Pcg2dArgs& a, int blocks, cudaStream_t s);

// Shared-memory layout (doubles): ph[(n+2)^2] | wx[n(n+1)] | wy[(n+1)n] | sj[d] | red[2*34]
// wx[qq(n+1)+P]: edge (P,qq+1)-(P+1,qq+1) (global node coords), P = 0..n
// wy[Q n + pp]:  edge (pp+1,Q)-(pp+1,Q+1),                       Q = 0..n
__device__ void assemble_scaled(const Pcg2dArgs& a, int64_t i, double* ph, double* wx, double* wy, double* sj) {
    const int n = a.n, d = a.ns.d;
    const int n1 = n + 1, W = n + 2;
    const int sq = n1 * n1;
    for (int j = threadIdx.x; j < d; j += blockDim.x) sj[j] = node_theta(a.ns, j, i);
    __syncthreads();
    const bool logn = a.coef_model == USFFT_COEF_LOGNORMAL_SIN;
    // phase 1: lower-triangle coefficients of every square into ph (temporary)
    for (int e = threadIdx.x; e < sq; e += blockDim.x) {
        double acc = 0.0;
        for (int j = 0; j < d; ++j) acc = fma(__ldg(a.psi + (size_t)j * 2 * sq + e), sj[j], acc);
        ph[e] = logn ? exp(acc) : 1.0 + acc;
    }
    __syncthreads();
    // phase 2: upper-triangle coefficient of square (P,Q) closes the horizontal edge above
    // it and the vertical edge on its left
    for (int e = threadIdx.x; e < sq; e += blockDim.x) {
        const int P = e % n1, Q = e / n1;
        double acc = 0.0;
        for (int j = 0; j < d; ++j) acc = fma(__ldg(a.psi + (size_t)j * 2 * sq + sq + e), sj[j], acc);
        const double au = logn ? exp(acc) : 1.0 + acc;
        if (Q < n) wx[Q * n1 + P] = 0.5 * (ph[(Q + 1) * n1 + P] + au);
        if (P >= 1) wy[Q * n + (P - 1)] = 0.5 * (au + ph[Q * n1 + (P - 1)]);
    }
    __syncthreads();
    // D^-1/2 into the halo array (zero on the boundary), then scale every edge
    for (int e = threadIdx.x; e < W * W; e += blockDim.x) ph[e] = 0.0;
    __syncthreads();
    for (int g = threadIdx.x; g < n * n; g += blockDim.x) {
        const int pp = g % n, qq = g / n;
        const double dg = wx[qq * n1 + pp] + wx[qq * n1 + pp + 1] + wy[qq * n + pp] + wy[(qq + 1) * n + pp];
        ph[(qq + 1) * W + pp + 1] = 1.0 / sqrt(dg);
    }
    __syncthreads();
    for (int e = threadIdx.x; e < n * n1; e += blockDim.x) {
        const int qq = e / n1, P = e % n1;          // horizontal: (P,qq+1)-(P+1,qq+1)
        wx[e] *= ph[(qq + 1) * W + P] * ph[(qq + 1) * W + P + 1];
    }
    for (int e = threadIdx.x; e < n1 * n; e += blockDim.x) {
        const int Q = e / n, pp = e % n;            // vertical: (pp+1,Q)-(pp+1,Q+1)
        wy[e] *= ph[Q * W + pp + 1] * ph[(Q + 1) * W + pp + 1];
    }
    __syncthreads();
}

// y = K~ v at node (pp,qq) from a halo array vh (unit diagonal)
template <typename T, typename WT>
__device__ __forceinline__ T apply_scaled(const T* vh, const WT* wx, const WT* wy, int n, int pp, int qq) {
    const int n1 = n + 1, W = n + 2;
    const int h = (qq + 1) * W + pp + 1;
    T acc = (T)wx[qq * n1 + pp] * vh[h - 1];
    acc = fma((T)wx[qq * n1 + pp + 1], vh[h + 1], acc);
    acc = fma((T)wy[qq * n + pp], vh[h - W], acc);
    acc = fma((T)wy[(qq + 1) * n + pp], vh[h + W], acc);
    return vh[h] - acc;
}

template <int NPT>
__global__ void __launch_bounds__(1024) pcg2d_fp64_kernel(const __grid_constant__ Pcg2dArgs a) {
    extern __shared__ double sm[];
    const int n = a.n, G = n * n, W = n + 2, n1 = n + 1;
    double* ph = sm;
    double* wx = ph + W * W;
    double* wy = wx + n * n1;
    double* sj = wy + n1 * n;
    double* red = sj + a.ns.d;
    const int T = blockDim.x, tid = threadIdx.x;

    for (int64_t sys = blockIdx.x; sys < a.count; sys += gridDim.x) {
        const int64_t i = lattice_node(a.ns, a.i0 + sys);
        assemble_scaled(a, i, ph, wx, wy, sj);
        // D^-1/2 is parked in the output row until the solution is scaled back
        double* out = a.U + (size_t)sys * G;
        double x[NPT], r[NPT], p[NPT], q[NPT];
        double rr_l = 0.0;
#pragma unroll
        for (int k = 0; k < NPT; ++k) {
            const int g = tid + k * T;
            if (g < G) {
                const double dg = ph[((g / n) + 1) * W + (g % n) + 1];
                out[g] = dg;
                x[k] = 0.0;
                r[k] = a.rhs * dg;
                p[k] = r[k];
                rr_l = fma(r[k], r[k], rr_l);
            } else {
                x[k] = r[k] = p[k] = 0.0;
            }
        }
        __syncthreads();                     // every D^-1/2 read before ph is reused
#pragma unroll
        for (int k = 0; k < NPT; ++k) {
            const int g = tid + k * T;
            if (g < G) ph[((g / n) + 1) * W + (g % n) + 1] = p[k];
        }
        double rr = block_sum(rr_l, red);
        const double stop = a.tol * a.tol * rr;
        int it = 0;
        while (rr > stop && it < a.max_iters) {
            double pq_l = 0.0;
#pragma unroll
            for (int k = 0; k < NPT; ++k) {
                const int g = tid + k * T;
                q[k] = 0.0;
                if (g < G) {
                    q[k] = apply_scaled<double, double>(ph, wx, wy, n, g % n, g / n);
                    pq_l = fma(p[k], q[k], pq_l);
                }
            }
            double pq, alpha;
            block_sum_ratio<double, NUM_OVER_SUM>(pq_l, rr, red, pq, alpha);      // alpha = rr / (p, Kp)
            double rn_l = 0.0;
#pragma unroll
            for (int k = 0; k < NPT; ++k) {
                x[k] = fma(alpha, p[k], x[k]);
                r[k] = fma(-alpha, q[k], r[k]);
                rn_l = fma(r[k], r[k], rn_l);
            }
            double rn, beta;
            block_sum_ratio<double, SUM_OVER_DEN>(rn_l, rr, red + 34, rn, beta);  // beta = rn / rr
            rr = rn;
#pragma unroll
            for (int k = 0; k < NPT; ++k) {
                const int g = tid + k * T;
                p[k] = fma(beta, p[k], r[k]);
                if (g < G) ph[((g / n) + 1) * W + (g % n) + 1] = p[k];
            }
            __syncthreads();
            ++it;
        }
#pragma unroll
        for (int k = 0; k < NPT; ++k) {
            const int g = tid + k * T;
            if (g < G) out[g] = x[k] * out[g];
        }
        if (tid == 0) {
            if (a.iters_out) a.iters_out[sys] = it;
            if (a.iters_sum) atomicAdd(a.iters_sum, (unsigned long long)it);
            if (rr > stop && a.fail_count) atomicAdd(a.fail_count, 1u);
        }
        __syncthreads();
    }
}

// MIXED layout (bytes, inside the same dynamic allocation as the fp64 assembly arrays):
//   [0, 8 W^2)            fp64 halo xh (residual operator input)  -- aliases ph of assembly
//   [8 W^2, +4 n(n+1))    fp32 wx32                              -- aliases wx of assembly
//   [.., +4 n(n+1))       fp32 wy32
//   [.., +4 W^2)          fp32 halo ph32
//   sj and red as in the fp64 layout (after wy of the assembly layout)
template <int NPT>
__global__ void __launch_bounds__(1024) pcg2d_mixed_kernel(const __grid_constant__ Pcg2dArgs a) {
    extern __shared__ double sm[];
    const int n = a.n, G = n * n, W = n + 2, n1 = n + 1;
    double* ph = sm;
    double* wx = ph + W * W;
    double* wy = wx + n * n1;
    double* sj = wy + n1 * n;
    double* red = sj + a.ns.d;
    float* red32 = reinterpret_cast<float*>(red);               // fp32 reduction scratch (68 floats)
    double* xh = sm;                                            // fp64 halo
    float* wx32 = reinterpret_cast<float*>(wx);
    float* wy32 = wx32 + n * n1;
    float* ph32 = wy32 + n1 * n;
    const int T = blockDim.x, tid = threadIdx.x;
    double* w64x = a.scratch + (size_t)blockIdx.x * 2 * n * n1;
    double* w64y = w64x + n * n1;

    for (int64_t sys = blockIdx.x; sys < a.count; sys += gridDim.x) {
        const int64_t i = lattice_node(a.ns, a.i0 + sys);
        assemble_scaled(a, i, ph, wx, wy, sj);
        double* out = a.U + (size_t)sys * G;     // holds D^-1/2 until the end
        double x[NPT], bt[NPT];
#pragma unroll
        for (int k = 0; k < NPT; ++k) {
            const int g = tid + k * T;
            const double dg = (g < G) ? ph[((g / n) + 1) * W + (g % n) + 1] : 0.0;
            if (g < G) out[g] = dg;
            bt[k] = a.rhs * dg;
            x[k] = 0.0;
        }
        // fp64 scaled weights to this CTA's scratch slot, fp32 copies to shared memory
        for (int e = tid; e < n * n1; e += T) {
            w64x[e] = wx[e];
            w64y[e] = wy[e];
        }
        __syncthreads();
        for (int e = tid; e < n * n1; e += T) {
            wx32[e] = (float)__ldcg(w64x + e);
            wy32[e] = (float)__ldcg(w64y + e);
        }
        for (int e = tid; e < W * W; e += T) {
            ph32[e] = 0.0f;
            xh[e] = 0.0;
        }
        __syncthreads();
        double rr0_l = 0.0;
#pragma unroll
        for (int k = 0; k < NPT; ++k) rr0_l = fma(bt[k], bt[k], rr0_l);
        const double rr0 = block_sum(rr0_l, red);
        const double stop = a.tol * a.tol * rr0;
        double rr64 = rr0;
        double r64[NPT];
#pragma unroll
        for (int k = 0; k < NPT; ++k) r64[k] = bt[k];
        int total = 0, outer = 0;
        while (rr64 > stop && outer < 16) {
            // ---- fp32 inner solve of K~ d = r64 / ||r64|| ----
            const double nr = sqrt(rr64);
            const float inv = (float)(1.0 / nr);
            float d32[NPT], r32[NPT], p32[NPT], q32[NPT];
            float rr_l = 0.0f;
#pragma unroll
            for (int k = 0; k < NPT; ++k) {
                const int g = tid + k * T;
                d32[k] = 0.0f;
                r32[k] = (float)r64[k] * inv;
                p32[k] = r32[k];
                rr_l = fmaf(r32[k], r32[k], rr_l);
                if (g < G) ph32[((g / n) + 1) * W + (g % n) + 1] = p32[k];
            }
            float rr, unused;
            block_sum_ratio<float, SUM_OVER_DEN>(rr_l, 1.0f, red32, rr, unused);
            const float istop = (float)(a.tol_inner * a.tol_inner) * rr;
            int it = 0;
            while (rr > istop && it < a.max_iters) {
                float pq_l = 0.0f;
#pragma unroll
                for (int k = 0; k < NPT; ++k) {
                    const int g = tid + k * T;
                    q32[k] = 0.0f;
                    if (g < G) {
                        q32[k] = apply_scaled<float, float>(ph32, wx32, wy32, n, g % n, g / n);
                        pq_l = fmaf(p32[k], q32[k], pq_l);
                    }
                }
                float pq, alpha;
                block_sum_ratio<float, NUM_OVER_SUM>(pq_l, rr, red32, pq, alpha);
                float rn_l = 0.0f;
#pragma unroll
                for (int k = 0; k < NPT; ++k) {
                    d32[k] = fmaf(alpha, p32[k], d32[k]);
                    r32[k] = fmaf(-alpha, q32[k], r32[k]);
                    rn_l = fmaf(r32[k], r32[k], rn_l);
                }
                float rn, beta;
                block_sum_ratio<float, SUM_OVER_DEN>(rn_l, rr, red32 + 34, rn, beta);
                rr = rn;
#pragma unroll
                for (int k = 0; k < NPT; ++k) {
                    const int g = tid + k * T;
                    p32[k] = fmaf(beta, p32[k], r32[k]);
                    if (g < G) ph32[((g / n) + 1) * W + (g % n) + 1] = p32[k];
                }
                __syncthreads();
                ++it;
            }
            total += it;
            // ---- fp64 update and residual r64 = b~ - K~ x ----
#pragma unroll
            for (int k = 0; k < NPT; ++k) {
                const int g = tid + k * T;
                x[k] = fma(nr, (double)d32[k], x[k]);
                if (g < G) xh[((g / n) + 1) * W + (g % n) + 1] = x[k];
            }
            __syncthreads();
            double rl = 0.0;
#pragma unroll
            for (int k = 0; k < NPT; ++k) {
                const int g = tid + k * T;
                r64[k] = 0.0;
                if (g < G) {
                    const int pp = g % n, qq = g / n, h = (qq + 1) * W + pp + 1;
                    double acc = __ldcg(w64x + qq * n1 + pp) * xh[h - 1];
                    acc = fma(__ldcg(w64x + qq * n1 + pp + 1), xh[h + 1], acc);
                    acc = fma(__ldcg(w64y + qq * n + pp), xh[h - W], acc);
                    acc = fma(__ldcg(w64y + (qq + 1) * n + pp), xh[h + W], acc);
                    r64[k] = bt[k] - (xh[h] - acc);
                    rl = fma(r64[k], r64[k], rl);
                }
            }
            rr64 = block_sum(rl, red + 33);
            ++outer;
        }
#pragma unroll
        for (int k = 0; k < NPT; ++k) {
            const int g = tid + k * T;
            if (g < G) out[g] = x[k] * out[g];
        }
        if (tid == 0) {
            if (a.iters_out) a.iters_out[sys] = total;
            if (a.iters_sum) atomicAdd(a.iters_sum, (unsigned long long)total);
            if (a.outer_sum) atomicAdd(a.outer_sum, (unsigned long long)outer);
            if (rr64 > stop && a.fail_count) atomicAdd(a.fail_count, 1u);
        }
        __syncthreads();
    }
}

// smallest nodes-per-thread count that fits the system into one CTA of <= 1024 threads
// nodes per thread: the smallest power of two with at most 1024 threads per CTA (512 for the
// MIXED kernel, whose per-thread state then gets up to 128 registers)
static int pick_npt(int G, int precision) {
    const int max_threads = precision == USFFT_MIXED ? 512 : 1024;
    int npt = 1;
    while ((G + npt - 1) / npt > max_threads) npt *= 2;
    return npt;
}

static size_t smem_bytes(int n, int d) {
    const size_t W = (size_t)n + 2;
    return sizeof(double) * (W * W + 2 * (size_t)n * (n + 1) + (size_t)d + 68);
}

template <int NPT>
static int resident_blocks(int precision, int threads, int n) {
    if (precision == USFFT_MIXED) return dst_resident_blocks<NPT>(threads, USFFT_MAX_D, n);
    const size_t smem = smem_bytes(n, USFFT_MAX_D);
    int per_sm = 0;
    cudaError_t e;
    if (precision == USFFT_MIXED_JACOBI) {
        e = allow_dyn_smem((const void*)pcg2d_mixed_kernel<NPT>, smem);
        if (e == cudaSuccess)
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, pcg2d_mixed_kernel<NPT>, threads, smem);
    } else {
        e = allow_dyn_smem((const void*)pcg2d_fp64_kernel<NPT>, smem);
        if (e == cudaSuccess)
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, pcg2d_fp64_kernel<NPT>, threads, smem);
    }
    if (e != cudaSuccess) {
        cudaGetLastError();
        per_sm = 1;
    }
    return per_sm < 1 ? 1 : per_sm;
}

// persistent grid: one wave of resident CTAs on every SM
int sample_2d_default_blocks(int n, int precision) {
    if (precision == USFFT_FP64_DST) return fp64_dst_default_blocks(n, USFFT_MAX_D);
    if (n > 63) {                       // large-mesh MIXED kernel: one 1024-thread CTA per SM
        int dev = 0, sms = 0;
        if (cudaGetDevice(&dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
            cudaGetLastError();
            sms = 152;
        }
        return sms;
    }
    const int G = n * n;
    const int npt = pick_npt(G, precision);
    const int threads = ((G + npt - 1) / npt + 31) / 32 * 32;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
        cudaGetLastError();
        sms = 152;
    }
    int per_sm;
    switch (npt) {
        case 1: per_sm = resident_blocks<1>(precision, threads, n); break;
        case 2: per_sm = resident_blocks<2>(precision, threads, n); break;
        case 4: per_sm = resident_blocks<4>(precision, threads, n); break;
        default: per_sm = dst_resident_blocks<8>(threads, USFFT_MAX_D, n); break;   // MIXED only
    }
    return sms * per_sm;
}

size_t sample_2d_scratch_bytes(int n, int precision, int blocks) {
    if (precision == USFFT_FP64) return 0;
    if (precision == USFFT_FP64_DST) return fp64_dst_slot_bytes(n, USFFT_MAX_D) * (size_t)blocks;
    if (precision == USFFT_MIXED) return mixed_slot_bytes(n) * (size_t)blocks;
    return sizeof(double) * 2 * (size_t)n * (n + 1) * (size_t)blocks;
}

template <int NPT>
static cudaError_t launch_npt(const Pcg2dArgs& a, int precision, int blocks, int threads, cudaStream_t s) {
    if (precision == USFFT_MIXED) return launch_dst_npt<NPT>(a, blocks, threads, s);
    const size_t smem = smem_bytes(a.n, a.ns.d);
    cudaError_t e;
    if (precision == USFFT_MIXED_JACOBI) {
        e = allow_dyn_smem((const void*)pcg2d_mixed_kernel<NPT>, smem);
        if (e != cudaSuccess) return e;
        pcg2d_mixed_kernel<NPT><<<blocks, threads, smem, s>>>(a);
    } else {
        e = allow_dyn_smem((const void*)pcg2d_fp64_kernel<NPT>, smem);
        if (e != cudaSuccess) return e;
        pcg2d_fp64_kernel<NPT><<<blocks, threads, smem, s>>>(a);
    }
    return cudaGetLastError();
}

cudaError_t launch_sample_2d(const NodeSpec& ns, int n, int coef_model, double f, const double* psi,
                             const CgConfig& cg, int64_t i0, int64_t count, double* U, int* iters_out,
                             unsigned int* fail_count, unsigned long long* iters_sum, double* scratch,
                             size_t scratch_bytes, cudaStream_t s, int* launches) {
    if (count <= 0) return cudaSuccess;
    if (n < 1 || n > 127 || (n > 63 && cg.precision != USFFT_MIXED && cg.precision != USFFT_FP64_DST))
        return cudaErrorInvalidValue;
    Pcg2dArgs a;
    a.ns = ns;
    a.n = n;
    a.coef_model = coef_model;
    a.max_iters = cg.max_iters;
    const double h = 1.0 / (double)(n + 1);
    a.rhs = h * h * f;
    a.tol = cg.tol;
    a.tol_inner = cg.precision == USFFT_MIXED ? 5e-5 : 1e-4;
    a.psi = psi;
    a.i0 = i0;
    a.count = count;
    a.U = U;
    a.iters_out = iters_out;
    a.fail_count = fail_count;
    a.iters_sum = iters_sum;
    a.outer_sum = iters_sum ? iters_sum + 1 : nullptr;
    a.scratch = scratch;
    a.coef_scale = cg.coef_scale;
    a.coef_decay = cg.coef_decay;
    const int G = n * n;
    const int npt = pick_npt(G, cg.precision);
    const int threads = ((G + npt - 1) / npt + 31) / 32 * 32;
    int blocks = cg.blocks > 0 ? cg.blocks : sample_2d_default_blocks(n, cg.precision);
    if (blocks > count) blocks = (int)count;
    if (cg.precision != USFFT_FP64 && scratch_bytes < sample_2d_scratch_bytes(n, cg.precision, blocks))
        return cudaErrorInvalidValue;
    cudaError_t e;
    if (cg.precision == USFFT_FP64_DST) {
        e = launch_fp64_dst(a, blocks, s);
        if (launches) ++*launches;
        return e;
    }
    if (n > 63) {
        e = launch_mixed_big(a, blocks, s);
        if (launches) ++*launches;
        return e;
    }
    switch (npt) {
        case 1: e = launch_npt<1>(a, cg.precision, blocks, threads, s); break;
        case 2: e = launch_npt<2>(a, cg.precision, blocks, threads, s); break;
        case 4: e = launch_npt<4>(a, cg.precision, blocks, threads, s); break;
        default: e = launch_dst_npt<8>(a, blocks, threads, s); break;                 // MIXED only
    }
    if (launches) ++*launches;
    return e;
}

}  // namespace usfft
