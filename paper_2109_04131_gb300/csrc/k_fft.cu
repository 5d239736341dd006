// Batched strided FFT along the lattice axis with the fused gather at k.z mod M.
//
// For every mesh node g the projected coefficients of Algorithm 1 (steps 1/2a, 2d) are
//   C[g][k] = (1/M) sum_{i<M} U[i][g] e^{-2 pi i i m_k / M},
// the length-M DFT of the g-th column of the sample matrix U[M][G] (one row per FE solve)
// read at the candidate indices m_k = k.z mod M (single rank-1 lattice, Appendix A).
//
// Real input, two columns per transform.  Columns 2c and 2c+1 are packed into one complex
// sequence z = u_2c + i u_2c+1; with Z = DFT(z), the two real transforms are
//   U_2c[m] = (Z[m] + conj Z[M-m]) / 2,   U_2c+1[m] = (Z[m] - conj Z[M-m]) / (2i),
// which halves the fp64 work (the kernels are bound by the fp64 pipe).
//
// Passes.  Columns are contiguous in g, so a CTA takes a tile of Gt adjacent column pairs
// and reads whole row segments.  M = L1 * L2 with L1, L2 <= 4096:
//   pass 1 (only if L1 > 1), for every i2 < L2:
//     Y[m1][i2][c] = e^{-2 pi i i2 m1 / M} sum_{i1<L1} z[i1 L2 + i2][c] e^{-2 pi i i1 m1 / L1}
//   final pass, for the bucket pair {m1, L1-m1 mod L1} (m1 <= L1/2; single pass: m1 = 0):
//     Z[m1 + L1 m2][c] = sum_{i2<L2} Y[m1][i2][c] e^{-2 pi i i2 m2 / L2}
//   and only the candidates of the two buckets (m_k mod L1 = m1 or L1-m1) are written, to
//   C[g][k] / M; M - (m1 + L1 m2) lies in the partner bucket at m2' = L2-1-m2 (m1 > 0) or
//   (L2-m2) mod L2 (m1 = 0).  The full spectrum is never stored.
// Each sub-transform of length L runs in shared memory as a mixed-radix Stockham autosort
// FFT (radices 8, 4, 2, 3 in registers, every other prime factor by a direct length-R DFT
// per output), ping-ponging between two buffers, with its twiddles W_L^j (L <= 1024) staged
// in shared memory from the fp64 table W[j] = e^{-2 pi i j / M} (W_L^j = W[j M / L]).
#include <cuda_runtime.h>
#include <math.h>
#include <string.h>

#include "usfft_internal.h"

namespace usfft {

static const int kLMax = 4096;        // longest on-chip sub-transform
static const int kTileElems = 2048;   // L * (columns per CTA) complex elements per buffer (32 KB)
static const int kTwSmem = 1024;      // sub-transform twiddles staged in shared memory up to this L
static const int kFftThreads = 256;

__global__ void twiddle_kernel(int64_t M, double2* W) {
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < M; j += (int64_t)gridDim.x * blockDim.x) {
        double sv, cv;
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
    int L;              // sub-transform length of this pass
    int Gt;             // column pairs per CTA
    int Gp;             // column pairs in total = ceil(G/2)
    int G;
    int nOuter;         // pass 1: L2 (i2); final pass: number of bucket pairs
    int L1;             // final pass: number of buckets
    int64_t M;
    int64_t wstride;    // M / L
    // input rows: row(o, l) = o * in_outer + l * in_step  (o = i2, or the bucket m1)
    const double* Ur;   // real samples [M][G] (pass 1, or the single pass)
    const double2* Yc;  // packed intermediate [M][Gp] (final pass of two)
    int64_t in_outer, in_step;
    // pass 1 output: Y row m1 * out_m + i2 * out_outer, times W[(i2 m1) mod M]
    double2* Yo;
    int64_t out_m, out_outer;
    // final pass: gather through the buckets
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
    return make_double2(fma(a.x, b.x, -a.y * b.y), fma(a.x, b.y, a.y * b.x));
}
__device__ __forceinline__ double2 cadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ double2 csub(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ double2 mul_mi(double2 a) { return make_double2(a.y, -a.x); }   // * (-i)

__device__ __forceinline__ void dft2(double2* v) {
    double2 a = v[0], b = v[1];
    v[0] = cadd(a, b);
    v[1] = csub(a, b);
}
__device__ __forceinline__ void dft3(double2* v) {
    // w = e^{-2 pi i/3} = -1/2 - i sqrt(3)/2
    const double s = 0.86602540378443864676;
    const double2 t1 = cadd(v[1], v[2]);
    const double2 t2 = make_double2(fma(-0.5, t1.x, v[0].x), fma(-0.5, t1.y, v[0].y));
    const double2 t3 = make_double2(s * (v[1].x - v[2].x), s * (v[1].y - v[2].y));
    v[0] = cadd(v[0], t1);
    v[1] = make_double2(t2.x + t3.y, t2.y - t3.x);     // t2 - i t3
    v[2] = make_double2(t2.x - t3.y, t2.y + t3.x);     // t2 + i t3
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

// twiddle W_L^e from shared memory (tw != null) or from the global table
__device__ __forceinline__ double2 twid(const double2* tw, const double2* W, int e, int64_t wstride) {
    return tw ? tw[e] : __ldg(W + (int64_t)e * wstride);
}

// one Stockham stage over `cols` columns (column c of the tile at buf[l * cols + c])
template <int R>
__device__ __forceinline__ void stage_reg(const double2* src, double2* dst, const double2* tw, const double2* W,
                                          int L, int cols, int Ns, int64_t wstride) {
    const int nb = L / R;
    const int tw_unit = L / (Ns * R);
    for (int item = threadIdx.x; item < nb * cols; item += blockDim.x) {
        const int c = item % cols, j = item / cols;
        const int jm = j % Ns;
        double2 v[R];
#pragma unroll
        for (int r = 0; r < R; ++r) {
            v[r] = src[(j + r * nb) * cols + c];
            if (r > 0 && jm != 0) v[r] = cmul(v[r], twid(tw, W, jm * r * tw_unit, wstride));
        }
        if (R == 2) dft2(v);
        if (R == 3) dft3(v);
        if (R == 4) dft4(v);
        if (R == 8) dft8(v);
        const int base = (j / Ns) * Ns * R + jm;
#pragma unroll
        for (int r = 0; r < R; ++r) dst[(base + r * Ns) * cols + c] = v[r];
    }
}

// any radix R: one thread per output element, direct length-R DFT
__device__ __forceinline__ void stage_generic(const double2* src, double2* dst, const double2* tw, const double2* W,
                                              int L, int cols, int Ns, int R, int64_t wstride) {
    const int nb = L / R;
    const int tw_unit = L / (Ns * R);
    const int unit = L / R;                                   // W_R^1 = W_L^(L/R)
    for (int item = threadIdx.x; item < L * cols; item += blockDim.x) {
        const int c = item % cols;
        const int rest = item / cols;
        const int k = rest % R, j = rest / R;
        const int jm = j % Ns;
        double2 acc = make_double2(0.0, 0.0);
        for (int r = 0; r < R; ++r) {
            const double2 v = src[(j + r * nb) * cols + c];
            const int e = (jm * r * tw_unit + ((r * k) % R) * unit) % L;
            acc = cadd(acc, cmul(v, twid(tw, W, e, wstride)));
        }
        dst[((j / Ns) * Ns * R + jm + k * Ns) * cols + c] = acc;
    }
}

// length-L FFT of `cols` columns held in b0; returns the buffer holding the result
__device__ double2* fft_tile(double2* b0, double2* b1, const double2* tw, const double2* W, const FftArgs& a,
                             int cols) {
    int Ns = 1;
    for (int st = 0; st < a.nst; ++st) {
        const int R = a.radix[st];
        if (R == 8) stage_reg<8>(b0, b1, tw, W, a.L, cols, Ns, a.wstride);
        else if (R == 4) stage_reg<4>(b0, b1, tw, W, a.L, cols, Ns, a.wstride);
        else if (R == 2) stage_reg<2>(b0, b1, tw, W, a.L, cols, Ns, a.wstride);
        else if (R == 3) stage_reg<3>(b0, b1, tw, W, a.L, cols, Ns, a.wstride);
        else stage_generic(b0, b1, tw, W, a.L, cols, Ns, R, a.wstride);
        __syncthreads();
        double2* t = b0;
        b0 = b1;
        b1 = t;
        Ns *= R;
    }
    return b0;
}

__device__ __forceinline__ void stage_twiddles(double2* tw, const double2* W, int L, int64_t wstride) {
    for (int j = threadIdx.x; j < L; j += blockDim.x) tw[j] = __ldg(W + (int64_t)j * wstride);
}

// ---- pass 1 (two-pass plans): length L1 over i1 for a fixed i2 = o, packed column pairs ----
__global__ void __launch_bounds__(kFftThreads) fft_pass1_kernel(const __grid_constant__ FftArgs a, const double2* W) {
    extern __shared__ double2 fbuf[];
    const int L = a.L, Gt = a.Gt;
    const int ntile = (a.Gp + Gt - 1) / Gt;
    const int o = blockIdx.x / ntile;
    const int c0 = (blockIdx.x % ntile) * Gt;
    double2* b0 = fbuf;
    double2* b1 = fbuf + (size_t)L * Gt;
    double2* tw = (L <= kTwSmem) ? b1 + (size_t)L * Gt : nullptr;      // W_L^j
    double2* ot = (L <= kTwSmem) ? tw + L : nullptr;                    // W[(o m) mod M], m < L
    if (tw) {
        stage_twiddles(tw, W, L, a.wstride);
        for (int m = threadIdx.x; m < L; m += blockDim.x) ot[m] = __ldg(W + ((int64_t)o * m) % a.M);
    }
    for (int idx = threadIdx.x; idx < L * Gt; idx += blockDim.x) {
        const int l = idx / Gt, c = idx % Gt, g = 2 * (c0 + c);
        double2 v = make_double2(0.0, 0.0);
        const int64_t row = (int64_t)o * a.in_outer + (int64_t)l * a.in_step;
        if (g < a.G) v.x = __ldcs(a.Ur + row * a.G + g);
        if (g + 1 < a.G) v.y = __ldcs(a.Ur + row * a.G + g + 1);
        b0[idx] = v;
    }
    __syncthreads();
    const double2* res = fft_tile(b0, b1, tw, W, a, Gt);
    for (int idx = threadIdx.x; idx < L * Gt; idx += blockDim.x) {
        const int m = idx / Gt, c = idx % Gt;
        if (c0 + c >= a.Gp) continue;
        double2 v = res[idx];
        if (m) v = cmul(v, ot ? ot[m] : __ldg(W + ((int64_t)o * m) % a.M));
        a.Yo[((int64_t)m * a.out_m + (int64_t)o * a.out_outer) * a.Gp + c0 + c] = v;
    }
}

// ---- final pass: buckets m1 and L1-m1 (length L2 over i2), unpack, gather ----
__global__ void __launch_bounds__(kFftThreads) fft_final_kernel(const __grid_constant__ FftArgs a, const double2* W) {
    extern __shared__ double2 fbuf[];
    const int L = a.L, Gt = a.Gt;
    const int ntile = (a.Gp + Gt - 1) / Gt;
    const int m1 = blockIdx.x / ntile;                  // 0 <= m1 <= L1/2
    const int c0 = (blockIdx.x % ntile) * Gt;
    const int L1 = a.L1;
    const int m1p = (L1 - m1) % L1;                     // partner bucket
    const int nb = (m1p == m1) ? 1 : 2;                 // transforms in this CTA
    const int cols = nb * Gt;                           // column c of bucket b at b * Gt + c
    double2* b0 = fbuf;
    double2* b1 = fbuf + (size_t)L * cols;
    double2* tw = (L <= kTwSmem) ? b1 + (size_t)L * cols : nullptr;
    if (tw) stage_twiddles(tw, W, L, a.wstride);
    for (int idx = threadIdx.x; idx < L * cols; idx += blockDim.x) {
        const int l = idx / cols, cc = idx % cols;
        const int b = cc / Gt, c = cc % Gt;
        const int bucket = b ? m1p : m1;
        double2 v = make_double2(0.0, 0.0);
        const int64_t row = (int64_t)bucket * a.in_outer + (int64_t)l * a.in_step;
        if (a.Yc) {
            if (c0 + c < a.Gp) v = __ldcs(a.Yc + row * a.Gp + c0 + c);
        } else {
            const int g = 2 * (c0 + c);
            if (g < a.G) v.x = __ldcs(a.Ur + row * a.G + g);
            if (g + 1 < a.G) v.y = __ldcs(a.Ur + row * a.G + g + 1);
        }
        b0[idx] = v;
    }
    __syncthreads();
    const double2* Z = fft_tile(b0, b1, tw, W, a, cols);
    // gather: candidates of bucket m1 (partner transform m1p) and, if distinct, of bucket m1p
    for (int b = 0; b < nb; ++b) {
        const int bucket = b ? m1p : m1;
        const int pb = (nb == 2) ? 1 - b : 0;           // column block of the partner transform
        const int e0 = a.boff[bucket], cnt = a.boff[bucket + 1] - e0;
        for (int idx = threadIdx.x; idx < cnt * Gt; idx += blockDim.x) {
            const int e = e0 + idx % cnt, c = idx / cnt;
            if (c0 + c >= a.Gp) continue;
            const int m2 = a.bm2[e];
            const int m2p = (bucket == 0) ? (L - m2) % L : L - 1 - m2;
            const double2 A = Z[m2 * cols + b * Gt + c];
            const double2 Bc = Z[m2p * cols + pb * Gt + c];      // Z[M - m], conjugated below
            const double s = 0.5 * a.scale;
            const double2 even = make_double2((A.x + Bc.x) * s, (A.y - Bc.y) * s);
            const double2 odd = make_double2((A.y + Bc.y) * s, (Bc.x - A.x) * s);
            const int g = 2 * (c0 + c);
            const int64_t k = a.bk[e];
            a.C[(int64_t)g * a.nJ + k] = even;
            if (g + 1 < a.G) a.C[(int64_t)(g + 1) * a.nJ + k] = odd;
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
    return (p.L1 > 1) ? sizeof(double2) * (size_t)p.M * (size_t)((G + 1) / 2) : 0;
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

// column pairs per CTA for a sub-transform of length L (nb transforms per column pair)
static int pick_gt(int L, int Gp, int nb) {
    int gt = kTileElems / (L * nb);
    if (gt < 1) gt = 1;
    if (gt > 32) gt = 32;
    if (gt > Gp) gt = Gp;
    return gt;
}

static size_t pass_smem(int L, int cols) {
    size_t s = 2 * sizeof(double2) * (size_t)L * cols;
    if (L <= kTwSmem) s += 2 * sizeof(double2) * (size_t)L;
    return s;
}

cudaError_t launch_fft_gather(const FftPlan& p, int G, const double* U, const double2* W, const GatherPlan& gp,
                              int64_t nJ, double2* scratch, double2* C, cudaStream_t s, int* launches) {
    if (p.M <= 0 || nJ <= 0) return cudaSuccess;
    if (p.L2 <= 0) return cudaErrorInvalidValue;
    FftArgs a;
    memset(&a, 0, sizeof(a));
    a.G = G;
    a.Gp = (G + 1) / 2;
    a.M = p.M;
    a.nJ = nJ;
    a.scale = 1.0 / (double)p.M;
    cudaError_t e;
    const bool two = p.L1 > 1;
    if (two) {
        // pass 1: length L1 over i1 (rows i1 L2 + i2), outer index i2
        a.L = p.L1;
        a.Gt = pick_gt(a.L, a.Gp, 1);
        a.nOuter = p.L2;
        a.wstride = p.M / a.L;
        a.Ur = U;
        a.in_outer = 1;
        a.in_step = p.L2;
        a.Yo = scratch;
        a.out_m = p.L2;
        a.out_outer = 1;
        a.nst = factorize(a.L, a.radix);
        const size_t smem = pass_smem(a.L, a.Gt);
        e = cudaFuncSetAttribute(fft_pass1_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        const int ntile = (a.Gp + a.Gt - 1) / a.Gt;
        fft_pass1_kernel<<<(unsigned)((int64_t)a.nOuter * ntile), kFftThreads, smem, s>>>(a, W);
        if (launches) ++*launches;
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    // final pass: length L2 over i2 (rows m1 L2 + i2), bucket pairs {m1, L1 - m1}
    FftArgs b = a;
    b.L = p.L2;
    b.L1 = two ? p.L1 : 1;
    b.Gt = pick_gt(b.L, b.Gp, b.L1 > 2 ? 2 : 1);
    b.nOuter = b.L1 / 2 + 1;
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
    const size_t smem = pass_smem(b.L, (b.L1 > 2 ? 2 : 1) * b.Gt);
    e = cudaFuncSetAttribute(fft_final_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const int ntile = (b.Gp + b.Gt - 1) / b.Gt;
    fft_final_kernel<<<(unsigned)((int64_t)b.nOuter * ntile), kFftThreads, smem, s>>>(b, W);
    if (launches) ++*launches;
    return cudaGetLastError();
}

}  // namespace usfft
