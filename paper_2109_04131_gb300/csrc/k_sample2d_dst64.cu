// 2-D sampler in fp64 with the fast-Poisson preconditioner (the USFFT_FP64_DST precision mode).
//
// The same discretisation and preconditioner as the mixed sampler (k_sample2d_dst.cu), with
// every operation in fp64: coefficient assembly in separable form, the 5-point operator K with
// edge weights w_e = mean of the two adjacent triangle coefficients, and preconditioned CG on
// K u = b with the preconditioner
//   M^-1 = D^-1/2 K_0^-1 D^-1/2,  D = diag(K) / 4,
//   K_0^-1 r = c^2 S ((S R S) o L) S,  S_jk = sin(pi (j+1)(k+1)/(n+1)),  c = 2/(n+1),
//   L_pq = 1 / (mu_p + mu_q),  mu_k = 4 sin^2(pi (k+1) / (2(n+1))).
// The mixed mode applies this operator in BF16 on the tensor cores inside fp32 iterations
// refined in fp64; here it is applied exactly (to fp64 rounding), so CG is the plain
// (non-flexible) method and the comparison of the two modes isolates the arithmetic precision.
//
// The sine transforms are matrix products on the FP64 CUDA cores (the GPU's FP64 tensor rate
// is no higher).  Each 1-D transform of the n x n grid halves its multiply count with the
// symmetry S_j,n-1-k = (-1)^j S_jk: a butterfly stage forms X_k + X_n-1-k and X_k - X_n-1-k,
// the even outputs j take the sums (plus, for odd n, the middle row, S_j,(n-1)/2 =
// sin(pi (j+1)/2)) and the odd outputs the differences, so one transform costs n^2 ceil(n/2)
// fused multiply-adds.  Each thread computes 4 x 4 output tiles of one parity in registers and
// writes them back in place after a barrier, so one n x n buffer in shared memory suffices.
//
// Layout: shared memory holds the transform grid X[p][q] (row stride LDX = n | 1, odd, so
// column accesses spread over the banks) and the half sine table Sh[j][k], k < ceil(n/2)
// (194 KB at n = 127); the per-node vectors, edge weights and the table of L sit in the CTA's
// scratch slot in global memory (L2-resident for the smaller meshes; their traffic is small
// against the transforms' fp64 arithmetic either way).  Halo layout h = (p+1) W + (q+1),
// W = n + 2; output index g = q n + p, as in the other samplers.  One CTA owns one system at
// a time (persistent grid).
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "k_pcg_common.cuh"
#include "usfft_internal.h"

namespace usfft {

struct Dst64Layout {
    int n, W, LDX, H, J1, JA;
    size_t o_X, o_S, o_sj, o_md, o_red, total;      // shared memory (bytes)
    size_t s_L, s_x, s_r, s_q, s_p, s_wl, s_wd, s_dg, s_sc, s_lo, s_At, s_Tr, slot;   // scratch (doubles)
};

__host__ __device__ inline size_t a16(size_t x) { return (x + 15) & ~(size_t)15; }

__host__ __device__ inline Dst64Layout dst64_layout(int n, int d) {
    Dst64Layout L;
    L.n = n;
    L.W = n + 2;
    L.LDX = n | 1;
    L.H = (n + 1) / 2;
    L.J1 = 1;
    L.JA = 1;
    for (int j = 1; j <= d; ++j) {
        int j1, j2;
        mode_pair(j, j1, j2);
        if (j1 > L.J1) L.J1 = j1;
        if (j1 > L.JA) L.JA = j1;
        if (j2 > L.JA) L.JA = j2;
    }
    size_t o = 0;
    L.o_X = o;   o = a16(o + sizeof(double) * (size_t)n * L.LDX);
    L.o_S = o;   o = a16(o + sizeof(double) * (size_t)n * L.H);
    L.o_sj = o;  o = a16(o + sizeof(double) * (size_t)d);
    L.o_md = o;  o = a16(o + sizeof(double) * (size_t)d + sizeof(int) * 2 * (size_t)d);
    L.o_red = o; o = a16(o + sizeof(double) * 34);
    L.total = o;
    const size_t WW = (size_t)L.W * L.W, n1 = (size_t)n + 1;
    size_t s = 0;
    L.s_L = s;  s += (size_t)n * n;
    L.s_x = s;  s += WW;
    L.s_r = s;  s += WW;
    L.s_q = s;  s += WW;
    L.s_p = s;  s += WW;
    L.s_wl = s; s += WW;
    L.s_wd = s; s += WW;
    L.s_dg = s; s += WW;
    L.s_sc = s; s += WW;
    L.s_lo = s; s += n1 * n1;
    L.s_At = s; s += (size_t)L.JA * 2 * n1;
    L.s_Tr = s; s += (size_t)L.J1 * 2 * n1;
    L.slot = (s + 31) & ~(size_t)31;     // 256-byte aligned slots
    return L;
}

// One 1-D DST-I of the n x n grid X in place: along the first index (AXIS1 = false, X <- S X) or
// the second (AXIS1 = true, X <- X S).  Element (k, c) -- k along the transform axis -- lives
// at k LDX + c, or c LDX + k.  Every thread of the CTA must call it (four barriers).
template <int TPT, bool AXIS1>
__device__ __forceinline__ void dst_pass(double* X, const double* Sh, int n, int LDX, int H) {
    const int T = blockDim.x, tid = threadIdx.x;
    auto at = [&](int k, int c) -> int { return AXIS1 ? c * LDX + k : k * LDX + c; };
    // butterfly: rows k < n/2 get the sums, rows n-1-k the differences
    const int half = n / 2;
    for (int e = tid; e < half * n; e += T) {
        const int k = e / n, c = e % n;
        const double lo = X[at(k, c)], hi = X[at(n - 1 - k, c)];
        X[at(k, c)] = lo + hi;
        X[at(n - 1 - k, c)] = lo - hi;
    }
    __syncthreads();
    // 4 x 4 tiles: four outputs j of one parity (j = par + 2 (4 rg + a)) by four columns c
    const int NE = (n + 1) / 2, NO = n / 2;
    const int RG0 = (NE + 3) / 4, RG1 = (NO + 3) / 4, CG = (n + 3) / 4;
    const int tiles = (RG0 + RG1) * CG;
    double acc[TPT][4][4];
#pragma unroll
    for (int u = 0; u < TPT; ++u) {
        const int tile = tid + u * T;
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
            for (int b = 0; b < 4; ++b) acc[u][a][b] = 0.0;
        if (tile >= tiles) continue;
        const int rg = tile / CG, cg = tile % CG;
        const int par = rg < RG0 ? 0 : 1, rgi = par ? rg - RG0 : rg;
        int j[4], c[4];
#pragma unroll
        for (int a = 0; a < 4; ++a) {
            j[a] = min(par + 2 * (4 * rgi + a), n - 1);     // clamped rows are computed, not stored
            c[a] = min(4 * cg + a, n - 1);
        }
        const int kmax = par ? NO : NE;
        for (int k = 0; k < kmax; ++k) {
            const int src = par ? n - 1 - k : k;
            double xv[4], sv[4];
#pragma unroll
            for (int b = 0; b < 4; ++b) xv[b] = X[at(src, c[b])];
#pragma unroll
            for (int a = 0; a < 4; ++a) sv[a] = Sh[j[a] * H + k];
#pragma unroll
            for (int a = 0; a < 4; ++a)
#pragma unroll
                for (int b = 0; b < 4; ++b) acc[u][a][b] = fma(sv[a], xv[b], acc[u][a][b]);
        }
    }
    __syncthreads();
#pragma unroll
    for (int u = 0; u < TPT; ++u) {
        const int tile = tid + u * T;
        if (tile >= tiles) continue;
        const int rg = tile / CG, cg = tile % CG;
        const int par = rg < RG0 ? 0 : 1, rgi = par ? rg - RG0 : rg;
#pragma unroll
        for (int a = 0; a < 4; ++a) {
            const int jj = par + 2 * (4 * rgi + a);
            if (jj >= n) continue;
#pragma unroll
            for (int b = 0; b < 4; ++b) {
                const int cc = 4 * cg + b;
                if (cc < n) X[at(jj, cc)] = acc[u][a][b];
            }
        }
    }
    __syncthreads();
}

// z = D^-1/2 K_0^-1 D^-1/2 r: X <- sc o r on the grid, four transforms with the eigenvalue
// scaling (L, c^2 folded in) between the pairs; z is left in X (z at node (p, q) is
// sc[h] X[p][q]).
template <int TPT>
__device__ __forceinline__ void apply_precond64(double* X, const double* Sh, const double* Lt, const double* r,
                                                const double* sc, int n, int LDX, int H, int W) {
    const int T = blockDim.x, tid = threadIdx.x, G = n * n;
    for (int g = tid; g < G; g += T) {
        const int p = g / n, q = g % n, h = (p + 1) * W + q + 1;
        X[p * LDX + q] = sc[h] * r[h];
    }
    __syncthreads();
    dst_pass<TPT, false>(X, Sh, n, LDX, H);
    dst_pass<TPT, true>(X, Sh, n, LDX, H);
    for (int g = tid; g < G; g += T) {
        const int p = g / n, q = g % n;
        X[p * LDX + q] *= Lt[g];
    }
    __syncthreads();
    dst_pass<TPT, false>(X, Sh, n, LDX, H);
    dst_pass<TPT, true>(X, Sh, n, LDX, H);
}

template <int TPT>
__global__ void __launch_bounds__(TPT == 1 ? 256 : 512) pcg2d_fp64_dst_kernel(const __grid_constant__ Pcg2dArgs a) {
    extern __shared__ __align__(16) unsigned char smraw[];
    const int n = a.n, G = n * n, n1 = n + 1, d = a.ns.d;
    const Dst64Layout Lo = dst64_layout(n, d);
    const int W = Lo.W, WW = W * W, LDX = Lo.LDX, H = Lo.H, J1 = Lo.J1, JA = Lo.JA;
    double* X = reinterpret_cast<double*>(smraw + Lo.o_X);
    double* Sh = reinterpret_cast<double*>(smraw + Lo.o_S);
    double* sj = reinterpret_cast<double*>(smraw + Lo.o_sj);
    double* amp = reinterpret_cast<double*>(smraw + Lo.o_md);
    int* mj1 = reinterpret_cast<int*>(amp + d);
    int* mj2 = mj1 + d;
    double* red = reinterpret_cast<double*>(smraw + Lo.o_red);
    double* slot = a.scratch + (size_t)blockIdx.x * Lo.slot;
    double* Lt = slot + Lo.s_L;
    double* x = slot + Lo.s_x;
    double* r = slot + Lo.s_r;
    double* q = slot + Lo.s_q;
    double* p = slot + Lo.s_p;
    double* wl = slot + Lo.s_wl;
    double* wd = slot + Lo.s_wd;
    double* dg = slot + Lo.s_dg;
    double* sc = slot + Lo.s_sc;
    double* low = slot + Lo.s_lo;
    double* At = slot + Lo.s_At;
    double* Tr = slot + Lo.s_Tr;
    const int T = blockDim.x, tid = threadIdx.x;

    // per CTA: sine table, scaled inverse eigenvalues, separable mode factors, zero halos
    for (int e = tid; e < n * H; e += T) {
        const int jj = e / H, k = e % H;
        const int m = ((jj + 1) * (k + 1)) % (2 * n1);          // exact reduction of the argument
        Sh[e] = sinpi((double)m / (double)n1);
    }
    {
        const double c2 = 4.0 / ((double)n1 * (double)n1);
        for (int g = tid; g < G; g += T) {
            const int pp = g / n, qq = g % n;
            const double s1 = sinpi((double)(pp + 1) / (2.0 * n1)), s2 = sinpi((double)(qq + 1) / (2.0 * n1));
            Lt[g] = c2 / (4.0 * s1 * s1 + 4.0 * s2 * s2);
        }
    }
    for (int e = tid; e < WW; e += T) {
        p[e] = 0.0;
        wl[e] = 0.0;
        wd[e] = 0.0;
    }
    {
        const double hh = 1.0 / (double)n1;
        for (int e = tid; e < JA * 2 * n1; e += T) {
            const int jj = e / (2 * n1) + 1, o = (e / n1) % 2 + 1, Pp = e % n1;
            At[e] = sinpi((double)jj * (((double)Pp + (double)o / 3.0) * hh));
        }
        for (int j = tid; j < d; j += T) {
            int j1, j2;
            mode_pair(j + 1, j1, j2);
            mj1[j] = j1;
            mj2[j] = j2;
            amp[j] = a.coef_scale * pow((double)(j + 1), -a.coef_decay);
        }
    }
    const double b = a.rhs;
    const double rr0 = (double)G * b * b;
    const double stop = a.tol * a.tol * rr0;
    const bool logn = a.coef_model == USFFT_COEF_LOGNORMAL_SIN;
    __syncthreads();

    for (int64_t sys = blockIdx.x; sys < a.count; sys += gridDim.x) {
        const int64_t i = lattice_node(a.ns, a.i0 + sys);
        // ---- assembly (fp64, separable form of psi_j = sin(j1 pi x1) sin(j2 pi x2)) ----
        for (int j = tid; j < d; j += T) sj[j] = node_theta(a.ns, j, i);
        __syncthreads();
        for (int e = tid; e < J1 * 2 * n1; e += T) {
            const int j1 = e / (2 * n1) + 1, o = (e / n1) % 2, Q = e % n1;
            double acc = 0.0;
            for (int j = 0; j < d; ++j)
                if (mj1[j] == j1) acc = fma(amp[j] * sj[j], At[((mj2[j] - 1) * 2 + o) * n1 + Q], acc);
            Tr[e] = acc;
        }
        __syncthreads();
        // lower-triangle coefficients of square (P, Q), centroid ((P + 2/3) h, (Q + 1/3) h)
        for (int e = tid; e < n1 * n1; e += T) {
            const int Pp = e % n1, Q = e / n1;
            double acc = 0.0;
            for (int j1 = 0; j1 < J1; ++j1) acc = fma(At[(j1 * 2 + 1) * n1 + Pp], Tr[(j1 * 2 + 0) * n1 + Q], acc);
            low[e] = logn ? exp(acc) : 1.0 + acc;
        }
        __syncthreads();
        // upper-triangle coefficient (centroid ((P + 1/3) h, (Q + 2/3) h)) closes two edges
        for (int e = tid; e < n1 * n1; e += T) {
            const int Pp = e % n1, Q = e / n1;
            double acc = 0.0;
            for (int j1 = 0; j1 < J1; ++j1) acc = fma(At[(j1 * 2 + 0) * n1 + Pp], Tr[(j1 * 2 + 1) * n1 + Q], acc);
            const double au = logn ? exp(acc) : 1.0 + acc;
            if (Q < n) wl[(Pp + 1) * W + Q + 1] = 0.5 * (low[(Q + 1) * n1 + Pp] + au);   // edge (P,Q+1)-(P+1,Q+1)
            if (Pp >= 1) wd[Pp * W + Q + 1] = 0.5 * (au + low[Q * n1 + (Pp - 1)]);       // edge (P,Q)-(P,Q+1)
        }
        __syncthreads();
        // diagonal and preconditioner scaling; x = 0, r = b
        double rz_l = 0.0;
        for (int g = tid; g < G; g += T) {
            const int pp = g / n, qq = g % n, h = (pp + 1) * W + qq + 1;
            const double dgh = (wl[h] + wl[h + W]) + (wd[h] + wd[h + 1]);
            dg[h] = dgh;
            sc[h] = rsqrt(0.25 * dgh);
            x[h] = 0.0;
            r[h] = b;
        }
        __syncthreads();

        // ---- preconditioned CG in fp64 ----
        apply_precond64<TPT>(X, Sh, Lt, r, sc, n, LDX, H, W);
        for (int g = tid; g < G; g += T) {
            const int pp = g / n, qq = g % n, h = (pp + 1) * W + qq + 1;
            const double z = sc[h] * X[pp * LDX + qq];
            p[h] = z;
            rz_l = fma(r[h], z, rz_l);
        }
        double gamma = block_sum(rz_l, red);          // its barriers also publish p
        double rho = rr0;
        int it = 0;
        while (it < a.max_iters) {
            double pq_l = 0.0;
            for (int g = tid; g < G; g += T) {
                const int pp = g / n, qq = g % n, h = (pp + 1) * W + qq + 1;
                double acc = wl[h] * p[h - W];
                acc = fma(wl[h + W], p[h + W], acc);
                acc = fma(wd[h], p[h - 1], acc);
                acc = fma(wd[h + 1], p[h + 1], acc);
                const double qh = fma(dg[h], p[h], -acc);
                q[h] = qh;
                pq_l = fma(p[h], qh, pq_l);
            }
            const double alpha = gamma / block_sum(pq_l, red);
            double rr_l = 0.0;
            for (int g = tid; g < G; g += T) {
                const int pp = g / n, qq = g % n, h = (pp + 1) * W + qq + 1;
                x[h] = fma(alpha, p[h], x[h]);
                const double rh = fma(-alpha, q[h], r[h]);
                r[h] = rh;
                rr_l = fma(rh, rh, rr_l);
            }
            rho = block_sum(rr_l, red);
            ++it;
            if (rho <= stop) break;
            apply_precond64<TPT>(X, Sh, Lt, r, sc, n, LDX, H, W);
            rz_l = 0.0;
            for (int g = tid; g < G; g += T) {
                const int pp = g / n, qq = g % n, h = (pp + 1) * W + qq + 1;
                rz_l = fma(r[h], sc[h] * X[pp * LDX + qq], rz_l);
            }
            const double gamma_new = block_sum(rz_l, red);
            const double beta = gamma_new / gamma;
            gamma = gamma_new;
            for (int g = tid; g < G; g += T) {
                const int pp = g / n, qq = g % n, h = (pp + 1) * W + qq + 1;
                p[h] = fma(beta, p[h], sc[h] * X[pp * LDX + qq]);
            }
            __syncthreads();
        }
        double* out = a.U + (size_t)sys * G;
        for (int g = tid; g < G; g += T) out[g] = x[((g % n) + 1) * W + (g / n) + 1];   // g = q n + p
        if (tid == 0) {
            if (a.iters_out) a.iters_out[sys] = it;
            if (a.iters_sum) atomicAdd(a.iters_sum, (unsigned long long)it);
            if (rho > stop && a.fail_count) atomicAdd(a.fail_count, 1u);
        }
        __syncthreads();
    }
}

static const size_t kMaxDst64Smem = 232448;    // 227 KB of dynamic shared memory per CTA

size_t fp64_dst_smem_bytes(int n, int d) { return dst64_layout(n, d).total; }
size_t fp64_dst_slot_bytes(int n, int d) { return sizeof(double) * dst64_layout(n, d).slot; }

static void (*dst64_kernel_for(int n))(Pcg2dArgs) {
    return n <= 63 ? pcg2d_fp64_dst_kernel<1> : pcg2d_fp64_dst_kernel<2>;
}
static int dst64_threads(int n) { return n <= 63 ? 256 : 512; }

int fp64_dst_default_blocks(int n, int d) {
    int dev = 0, sms = 0, per_sm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
        cudaGetLastError();
        sms = 152;
    }
    void (*k)(Pcg2dArgs) = dst64_kernel_for(n);
    const size_t smem = fp64_dst_smem_bytes(n, d);
    cudaError_t e = allow_dyn_smem((const void*)k, smem);
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, dst64_threads(n), smem);
    if (e != cudaSuccess) {
        cudaGetLastError();
        per_sm = 1;
    }
    return sms * (per_sm < 1 ? 1 : per_sm);
}

cudaError_t launch_fp64_dst(const Pcg2dArgs& a, int blocks, cudaStream_t s) {
    if (a.n < 1 || a.n > 127) return cudaErrorInvalidValue;
    void (*k)(Pcg2dArgs) = dst64_kernel_for(a.n);
    const size_t smem = fp64_dst_smem_bytes(a.n, a.ns.d);
    if (smem > kMaxDst64Smem) return cudaErrorInvalidValue;
    cudaError_t e = allow_dyn_smem((const void*)k, smem);
    if (e != cudaSuccess) return e;
    k<<<blocks, dst64_threads(a.n), smem, s>>>(a);
    return cudaGetLastError();
}

}  // namespace usfft
