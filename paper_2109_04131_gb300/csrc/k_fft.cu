// Batched strided FFT along the lattice axis with the fused gather at k.z mod M.
//
// For every mesh node g the projected coefficients of Algorithm 1 (steps 1/2a, 2d) are
//   C[g][k] = (1/M) sum_{i<M} U[i][g] e^{-2 pi i i m_k / M},
// the length-M DFT of the g-th column of the sample matrix U[M][G] (one row per FE solve)
// read at the candidate indices m_k = k.z mod M (single rank-1 lattice, Appendix A).
//
// Layout and passes.  Columns are contiguous in g, so a CTA takes a tile of Gt adjacent
// columns and reads whole row segments.  M = L1 * L2 with L1, L2 <= 4096:
//   pass 1 (only if L2 > 1), for every i2 < L2:
//     Y[m1][i2][g] = e^{-2 pi i i2 m1 / M} sum_{i1<L1} U[i1 L2 + i2][g] e^{-2 pi i i1 m1 / L1}
//   final pass, for every m1 < L1 (or the single pass, L1 = 1 outer index):
//     X[m1 + L1 m2][g] = sum_{i2<L2} Y[m1][i2][g] e^{-2 pi i i2 m2 / L2},
//   and only the X entries of the candidates in bucket m1 (m_k mod L1 = m1) are written, to
//   C[g][k] / M.  The full spectrum is never stored.
// Each sub-transform of length L runs in shared memory as a mixed-radix Stockham
// autosort FFT (radices 8, 4, 2 in registers, every other prime factor by a direct
// length-R DFT per output), ping-ponging between two buffers.  Twiddles come from one
// fp64 table W[j] = e^{-2 pi i j / M}, j < M (W_L^j = W[j M / L]).
#include <cuda_runtime.h>
#include <math.h>

#include "usfft_internal.h"

namespace usfft {

static const int kLMax = 4096;        // longest on-chip sub-transform
static const int kTileElems = 2048;   // L * Gt complex elements per buffer (32 KB)
static const int kFftThreads = 256;

__global__ void twiddle_kernel(int64_t M, double2* W) {
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < M; j += (int64_t)gridDim.x * blockDim.x) {
        double sv, cv;
        // exact reduction to [0, 1/2]-symmetric arguments is not needed: 2j/M < 2
        sincospi(2.0 * (double)j / (double)M, &sv, &cv);
        W[j] = make_double2(cv, -sv);
    }
}

cudaError_t launch_twiddles(int64_t M, double2* W, cudaStream_t s, int* launches) {
    int64_t b = (M + 255) / 256;
    if (b > 4096) b = 4096;
    if (b < 1) b = 1;
    twiddle_kernel<<<(unsigned)b, 256, 0, s>>>(M, W);
    if (launches) ++*launches;
    return cudaGetLastError();
}

struct FftArgs {
    int L, Gt, G, nOuter;
    int64_t M;
    int64_t wstride;              // M / L
    // input rows: row(o, l) = o * in_outer + l * in_step
    const double* Ur;             // real input (or null)
    const double2* Yc;            // complex input (or null)
    int64_t in_outer, in_step;
    // intermediate output rows: row(o, m) = m * out_m + o * out_outer, times W[(o m) mod M]
    double2* Yo;
    int64_t out_m, out_outer;
    // final output: gather through the bucket of o
    const int* boff;
    const int* bk;
    const int* bm2;
    double2* C;
    int64_t nJ;
    double scale;
    int nst;
    int radix[32];
};

__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
    return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ double2 cadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ double2 csub(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ double2 mul_mi(double2 a) { return make_double2(a.y, -a.x); }   // * (-i)

__device__ __forceinline__ void dft2(double2* v) {
    double2 a = v[0], b = v[1];
    v[0] = cadd(a, b);
    v[1] = csub(a, b);
}
__device__ __forceinline__ void dft4(double2* v) {
    double2 s02 = cadd(v[0], v[2]), d02 = csub(v[0], v[2]);
    double2 s13 = cadd(v[1], v[3]), d13 = mul_mi(csub(v[1], v[3]));
    v[0] = cadd(s02, s13);
    v[2] = csub(s02, s13);
    v[1] = cadd(d02, d13);
    v[3] = csub(d02, d13);
}
__device__ __forceinline__ void dft8(double2* v) {
    const double s = 0.70710678118654752440;
    double2 e[4] = {v[0], v[2], v[4], v[6]};
    double2 o[4] = {v[1], v[3], v[5], v[7]};
    dft4(e);
    dft4(o);
    // o[k] *= w8^k, w8 = e^{-2 pi i / 8}
    double2 o1 = make_double2((o[1].x + o[1].y) * s, (o[1].y - o[1].x) * s);
    double2 o2 = mul_mi(o[2]);
    double2 o3 = make_double2((o[3].y - o[3].x) * s, -(o[3].x + o[3].y) * s);
    v[0] = cadd(e[0], o[0]);
    v[4] = csub(e[0], o[0]);
    v[1] = cadd(e[1], o1);
    v[5] = csub(e[1], o1);
    v[2] = cadd(e[2], o2);
    v[6] = csub(e[2], o2);
    v[3] = cadd(e[3], o3);
    v[7] = csub(e[3], o3);
}

template <int R>
__device__ __forceinline__ void stage_pow2(const double2* src, double2* dst, const double2* W, int L, int Gt, int Ns,
                                           int64_t wstride) {
    const int nb = L / R;
    const int tw_unit = L / (Ns * R);
    for (int item = threadIdx.x; item < nb * Gt; item += blockDim.x) {
        const int c = item % Gt, j = item / Gt;
        const int jm = j % Ns;
        double2 v[R];
#pragma unroll
        for (int r = 0; r < R; ++r) {
            v[r] = src[(j + r * nb) * Gt + c];
            if (r > 0 && jm != 0) v[r] = cmul(v[r], __ldg(W + (int64_t)(jm * r * tw_unit) * wstride));
        }
        if (R == 2) dft2(v);
        if (R == 4) dft4(v);
        if (R == 8) dft8(v);
        const int base = (j / Ns) * Ns * R + jm;
#pragma unroll
        for (int r = 0; r < R; ++r) dst[(base + r * Ns) * Gt + c] = v[r];
    }
}

// any radix R: one thread per output element, direct length-R DFT
__device__ __forceinline__ void stage_generic(const double2* src, double2* dst, const double2* W, int L, int Gt, int Ns,
                                              int R, int64_t wstride) {
    const int nb = L / R;
    const int tw_unit = L / (Ns * R);
    const int unit = L / R;                                   // W_R^1 = W_L^(L/R)
    for (int item = threadIdx.x; item < L * Gt; item += blockDim.x) {
        const int c = item % Gt;
        const int rest = item / Gt;
        const int k = rest % R, j = rest / R;
        const int jm = j % Ns;
        double2 acc = make_double2(0.0, 0.0);
        for (int r = 0; r < R; ++r) {
            double2 v = src[(j + r * nb) * Gt + c];
            const int e = (jm * r * tw_unit + ((r * k) % R) * unit) % L;
            acc = cadd(acc, cmul(v, __ldg(W + (int64_t)e * wstride)));
        }
        dst[((j / Ns) * Ns * R + jm + k * Ns) * Gt + c] = acc;
    }
}

__global__ void __launch_bounds__(kFftThreads) fft_pass_kernel(const __grid_constant__ FftArgs a, const double2* W) {
    extern __shared__ double2 fbuf[];
    const int L = a.L, Gt = a.Gt;
    const int ntile = (a.G + Gt - 1) / Gt;
    const int o = blockIdx.x / ntile;
    const int g0 = (blockIdx.x % ntile) * Gt;
    double2* b0 = fbuf;
    double2* b1 = fbuf + (size_t)L * Gt;
    // load the tile: L rows x Gt columns, columns fastest (row segments are contiguous)
    for (int idx = threadIdx.x; idx < L * Gt; idx += blockDim.x) {
        const int l = idx / Gt, c = idx % Gt, g = g0 + c;
        double2 v = make_double2(0.0, 0.0);
        if (g < a.G) {
            const int64_t row = (int64_t)o * a.in_outer + (int64_t)l * a.in_step;
            if (a.Ur) v.x = __ldcs(a.Ur + row * a.G + g);
            else v = __ldcs(a.Yc + row * a.G + g);
        }
        b0[idx] = v;
    }
    __syncthreads();
    int Ns = 1;
    for (int st = 0; st < a.nst; ++st) {
        const int R = a.radix[st];
        if (R == 8) stage_pow2<8>(b0, b1, W, L, Gt, Ns, a.wstride);
        else if (R == 4) stage_pow2<4>(b0, b1, W, L, Gt, Ns, a.wstride);
        else if (R == 2) stage_pow2<2>(b0, b1, W, L, Gt, Ns, a.wstride);
        else stage_generic(b0, b1, W, L, Gt, Ns, R, a.wstride);
        __syncthreads();
        double2* t = b0;
        b0 = b1;
        b1 = t;
        Ns *= R;
    }
    if (a.Yo) {
        // intermediate pass: twiddle by W[(o m) mod M] and store Y[m][o][g]
        for (int idx = threadIdx.x; idx < L * Gt; idx += blockDim.x) {
            const int m = idx / Gt, c = idx % Gt, g = g0 + c;
            if (g >= a.G) continue;
            double2 v = b0[idx];
            const int64_t e = ((int64_t)o * m) % a.M;
            if (e) v = cmul(v, __ldg(W + e));
            a.Yo[((int64_t)m * a.out_m + (int64_t)o * a.out_outer) * a.G + g] = v;
        }
    } else {
        // final pass: gather the candidates of bucket o
        const int e0 = a.boff[o], cnt = a.boff[o + 1] - e0;
        for (int idx = threadIdx.x; idx < cnt * Gt; idx += blockDim.x) {
            const int e = e0 + idx % cnt, c = idx / cnt, g = g0 + c;
            if (g >= a.G) continue;
            const double2 v = b0[a.bm2[e] * Gt + c];
            a.C[(int64_t)g * a.nJ + a.bk[e]] = make_double2(v.x * a.scale, v.y * a.scale);
        }
    }
}

FftPlan make_fft_plan(int64_t M) {
    FftPlan p;
    p.M = M;
    if (M <= kLMax) {
        p.L1 = 1;
        p.L2 = (int)M;     // single pass: the final pass over the whole length
        return p;
    }
    // most balanced divisor pair with both factors <= kLMax
    int best = 0;
    for (int64_t a = 1; a * a <= M; ++a)
        if (M % a == 0 && M / a <= kLMax) best = (int)a;
    if (best == 0) {
        p.L1 = p.L2 = 0;     // not supported
        return p;
    }
    p.L1 = (int)(M / best) >= best ? (int)(M / best) : best;   // L1 = the larger factor
    p.L2 = (int)(M / p.L1);
    return p;
}

size_t fft_scratch_bytes(const FftPlan& p, int G) {
    return (p.L1 > 1) ? sizeof(double2) * (size_t)p.M * (size_t)G : 0;
}

static int factorize(int L, int* radix) {
    int n = 0;
    while (L % 8 == 0) { radix[n++] = 8; L /= 8; }
    while (L % 4 == 0) { radix[n++] = 4; L /= 4; }
    while (L % 2 == 0) { radix[n++] = 2; L /= 2; }
    for (int p = 3; p <= L; p += 2)
        while (L % p == 0) { radix[n++] = p; L /= p; }
    return n;
}

static int pick_gt(int L, int G) {
    int gt = kTileElems / L;
    if (gt < 1) gt = 1;
    if (gt > 64) gt = 64;
    if (gt > G) gt = G;
    return gt;
}

static cudaError_t run_pass(FftArgs& a, const double2* W, cudaStream_t s) {
    size_t smem = 2 * sizeof(double2) * (size_t)a.L * a.Gt;
    cudaError_t e = cudaFuncSetAttribute(fft_pass_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int ntile = (a.G + a.Gt - 1) / a.Gt;
    int64_t blocks = (int64_t)a.nOuter * ntile;
    fft_pass_kernel<<<(unsigned)blocks, kFftThreads, smem, s>>>(a, W);
    return cudaGetLastError();
}

cudaError_t launch_fft_gather(const FftPlan& p, int G, const double* U, const double2* W, const GatherPlan& gp,
                              int64_t nJ, double2* scratch, double2* C, cudaStream_t s, int* launches) {
    if (p.M <= 0 || nJ <= 0) return cudaSuccess;
    if (p.L2 <= 0) return cudaErrorInvalidValue;
    FftArgs a;
    memset(&a, 0, sizeof(a));
    a.G = G;
    a.M = p.M;
    a.nJ = nJ;
    a.scale = 1.0 / (double)p.M;
    cudaError_t e;
    const bool two = p.L1 > 1;
    if (two) {
        // pass 1: length L1 over i1 (rows i1 L2 + i2), outer index i2
        a.L = p.L1;
        a.Gt = pick_gt(a.L, G);
        a.nOuter = p.L2;
        a.wstride = p.M / a.L;
        a.Ur = U;
        a.in_outer = 1;
        a.in_step = p.L2;
        a.Yo = scratch;
        a.out_m = p.L2;
        a.out_outer = 1;
        a.nst = factorize(a.L, a.radix);
        e = run_pass(a, W, s);
        if (launches) ++*launches;
        if (e != cudaSuccess) return e;
    }
    // final pass: length L2 over i2 (rows m1 L2 + i2), outer index m1, gather bucket m1
    FftArgs b = a;
    b.L = p.L2;
    b.Gt = pick_gt(b.L, G);
    b.nOuter = two ? p.L1 : 1;
    b.wstride = p.M / b.L;
    b.Ur = two ? nullptr : U;
    b.Yc = two ? scratch : nullptr;
    b.in_outer = p.L2;
    b.in_step = 1;
    b.Yo = nullptr;
    b.boff = gp.offsets;
    b.bk = gp.k;
    b.bm2 = gp.m2;
    b.C = C;
    b.nst = factorize(b.L, b.radix);
    e = run_pass(b, W, s);
    if (launches) ++*launches;
    return e;
}

}  // namespace usfft
