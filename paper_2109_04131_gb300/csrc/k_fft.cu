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
// in shared memory from the table W[j] = e^{-2 pi i j / M} (W_L^j = W[j M / L]).
//
// Arithmetic.  The kernels are templates over the complex arithmetic: fp64 (double2), or
// double-float (float4 = re.hi, re.lo, im.hi, im.lo; every real value a pair of floats with
// about 48 significant bits, from the error-free transformations TwoSum (Knuth) and the fma
// product (Dekker)).  The double-float transform runs on the FP32 pipe, 64x the FP64 rate of
// this part, at a rounding error of a few 1e-15 relative to the largest coefficient of a
// node; both arithmetic kinds store 16 bytes per complex value.
#include <cuda_runtime.h>
#include <math.h>
#include <string.h>

#include <vector>

#include "k_cvt.cuh"
#include "usfft_internal.h"

namespace usfft {

static const int kLMax = 4096;        // longest on-chip sub-transform
static const int kTileElems = 2048;   // L * (columns per CTA) complex elements per buffer (32 KB)
static const int kTwSmem = 1024;      // sub-transform twiddles staged in shared memory up to this L
static const int kFftThreads = 256;

// W[j] = e^{-2 pi i j / M} in fp64, or split into double-float (float4) when DFT_DF
template <bool DFT_DF>
__global__ void twiddle_kernel(int64_t M, void* Wv) {
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < M; j += (int64_t)gridDim.x * blockDim.x) {
        double sv, cv;
        sincospi(2.0 * (double)j / (double)M, &sv, &cv);
        if (DFT_DF) {
            const float ch = __double2float_rn(cv), sh = __double2float_rn(-sv);
            reinterpret_cast<float4*>(Wv)[j] =
                make_float4(ch, __double2float_rn(cv - (double)ch), sh, __double2float_rn(-sv - (double)sh));
        } else {
            reinterpret_cast<double2*>(Wv)[j] = make_double2(cv, -sv);
        }
    }
}

cudaError_t launch_twiddles(int64_t M, void* W, bool df, cudaStream_t s, int* launches) {
    int64_t b = (M + 255) / 256;
    if (b > 4096) b = 4096;
    if (b < 1) b = 1;
    if (df)
        twiddle_kernel<true><<<(unsigned)b, 256, 0, s>>>(M, W);
    else
        twiddle_kernel<false><<<(unsigned)b, 256, 0, s>>>(M, W);
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
    const void* Yc;     // packed intermediate [M][Gp] (final pass of two), the arithmetic's complex type
    int64_t in_outer, in_step;
    // pass 1 output: Y row m1 * out_m + i2 * out_outer, times W[(i2 m1) mod M]
    void* Yo;
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

// ---- complex arithmetic: fp64 -----------------------------------------------------------
struct F64 {
    typedef double2 C;
    static constexpr bool kFastDiv = false;   // index division by a multiply-high (measured slower here)
    static __device__ __forceinline__ C zero() { return make_double2(0.0, 0.0); }
    static __device__ __forceinline__ C pair(double x, double y) { return make_double2(x, y); }
    static __device__ __forceinline__ C pair_trunc(double x, double y) { return make_double2(x, y); }
    static __device__ __forceinline__ C add(C a, C b) { return make_double2(a.x + b.x, a.y + b.y); }
    static __device__ __forceinline__ C sub(C a, C b) { return make_double2(a.x - b.x, a.y - b.y); }
    static __device__ __forceinline__ C mul(C a, C b) {
        return make_double2(fma(a.x, b.x, -a.y * b.y), fma(a.x, b.y, a.y * b.x));
    }
    static __device__ __forceinline__ C mul_mi(C a) { return make_double2(a.y, -a.x); }   // * (-i)
    static __device__ __forceinline__ C mul_k(C a, double k) { return make_double2(a.x * k, a.y * k); }
    static __device__ __forceinline__ C half(C a) { return make_double2(0.5 * a.x, 0.5 * a.y); }
    static __device__ __forceinline__ C norm(C a) { return a; }
    // (A + conj B) s and (A - conj B) s / i, the unpacked transforms of the two real columns
    static __device__ __forceinline__ void unpack(C A, C B, double s, float, float, double2& even, double2& odd) {
        even = make_double2((A.x + B.x) * s, (A.y - B.y) * s);
        odd = make_double2((A.y + B.y) * s, (B.x - A.x) * s);
    }
};

// ---- complex arithmetic: double-float --------------------------------------------------
__device__ __forceinline__ float2 df_two_sum(float a, float b) {        // s + e = a + b exactly
    const float s = __fadd_rn(a, b);
    const float bb = __fadd_rn(s, -a);
    return make_float2(s, __fadd_rn(__fadd_rn(a, -__fadd_rn(s, -bb)), __fadd_rn(b, -bb)));
}
__device__ __forceinline__ float2 df_norm(float s, float t) {           // fast two-sum, |s| >= |t|
    const float h = __fadd_rn(s, t);
    return make_float2(h, __fadd_rn(t, -__fadd_rn(h, -s)));
}
__device__ __forceinline__ float2 dfr_add(float hi, float lo, float bhi, float blo) {
    const float2 se = df_two_sum(hi, bhi);
    return df_norm(se.x, __fadd_rn(se.y, __fadd_rn(lo, blo)));
}
__device__ __forceinline__ float2 dfr_mul(float ahi, float alo, float bhi, float blo) {
    const float p = __fmul_rn(ahi, bhi);
    float e = __fmaf_rn(ahi, bhi, -p);
    e = __fmaf_rn(ahi, blo, __fmaf_rn(alo, bhi, e));
    return df_norm(p, e);
}
// Unnormalised forms for the transform's inner arithmetic: the high parts' sum or product is
// still split exactly (TwoSum, fma), but the low word is left as it falls instead of being
// folded into a canonical pair after every operation; the value hi + lo carries the same
// information, and each stage renormalises once per value as it stores (DF::norm), so the low
// word never grows by more than the few operations of one butterfly.
__device__ __forceinline__ float2 dfl_add(float hi, float lo, float bhi, float blo) {
    const float2 se = df_two_sum(hi, bhi);
    return make_float2(se.x, __fadd_rn(se.y, __fadd_rn(lo, blo)));
}
__device__ __forceinline__ float2 dfl_mul(float ahi, float alo, float bhi, float blo) {
    const float p = __fmul_rn(ahi, bhi);
    const float e = __fmaf_rn(ahi, bhi, -p);
    return make_float2(p, __fmaf_rn(ahi, blo, __fmaf_rn(alo, bhi, e)));
}
struct DF {
    typedef float4 C;   // re.hi, re.lo, im.hi, im.lo
    static constexpr bool kFastDiv = true;    // index division by a multiply-high (measured faster here)
    static __device__ __forceinline__ float2 split(double x) { return d2df(x); }
    static __device__ __forceinline__ C zero() { return make_float4(0.f, 0.f, 0.f, 0.f); }
    static __device__ __forceinline__ C pair(double x, double y) {
        const float2 a = split(x), b = split(y);
        return make_float4(a.x, a.y, b.x, b.y);
    }
    // x as a pair without fp64 arithmetic: hi = x truncated to 24 significant bits (exact), lo = the
    // remaining 29 bits of the significand, rounded to float and scaled by a power of two (exact);
    // |lo| < ulp(hi), so the pair is unnormalised the way the butterflies' results are.  Magnitudes
    // outside [2^-74, 2^127) (and inf, nan) take the rounded split with one fp64 subtraction.  Used by
    // the two-pass kernels' loads (2.5% faster there; the in-place kernel measured 1% slower with it).
    static __device__ __forceinline__ float2 split_trunc(double x) {
        const uint32_t uh = (uint32_t)__double2hiint(x), ul = (uint32_t)__double2loint(x);
        const uint32_t e = (uh >> 20) & 0x7ffu;
        if (e < 949u || e > 1150u) return d2df(x);
        const uint32_t sign = uh & 0x80000000u;
        const float hi = __uint_as_float(sign | ((e - 896u) << 23) | ((uh & 0xfffffu) << 3) | (ul >> 29));
        const float lo = __fmul_rn(__uint2float_rn(ul & 0x1fffffffu), __uint_as_float((e - 948u) << 23));
        return make_float2(hi, sign ? -lo : lo);
    }
    static __device__ __forceinline__ C pair_trunc(double x, double y) {
        const float2 a = split_trunc(x), b = split_trunc(y);
        return make_float4(a.x, a.y, b.x, b.y);
    }
    static __device__ __forceinline__ C add(C a, C b) {
        const float2 r = dfl_add(a.x, a.y, b.x, b.y), i = dfl_add(a.z, a.w, b.z, b.w);
        return make_float4(r.x, r.y, i.x, i.y);
    }
    static __device__ __forceinline__ C sub(C a, C b) {
        const float2 r = dfl_add(a.x, a.y, -b.x, -b.y), i = dfl_add(a.z, a.w, -b.z, -b.w);
        return make_float4(r.x, r.y, i.x, i.y);
    }
    static __device__ __forceinline__ C mul(C a, C b) {
        const float2 rr = dfl_mul(a.x, a.y, b.x, b.y), ii = dfl_mul(a.z, a.w, b.z, b.w);
        const float2 ri = dfl_mul(a.x, a.y, b.z, b.w), ir = dfl_mul(a.z, a.w, b.x, b.y);
        const float2 r = dfl_add(rr.x, rr.y, -ii.x, -ii.y), i = dfl_add(ri.x, ri.y, ir.x, ir.y);
        return make_float4(r.x, r.y, i.x, i.y);
    }
    static __device__ __forceinline__ C norm(C a) {
        const float2 r = df_norm(a.x, a.y), i = df_norm(a.z, a.w);
        return make_float4(r.x, r.y, i.x, i.y);
    }
    static __device__ __forceinline__ C mul_mi(C a) { return make_float4(a.z, a.w, -a.x, -a.y); }
    static __device__ __forceinline__ C mul_k(C a, double k) {
        const float kh = (float)k, kl = (float)(k - (double)kh);   // folded at compile time for literals
        const float2 r = dfl_mul(a.x, a.y, kh, kl), i = dfl_mul(a.z, a.w, kh, kl);
        return make_float4(r.x, r.y, i.x, i.y);
    }
    static __device__ __forceinline__ C half(C a) { return make_float4(0.5f * a.x, 0.5f * a.y, 0.5f * a.z, 0.5f * a.w); }
    // s given as (sh, sl), the split of the fp64 scale (formed once per kernel)
    static __device__ __forceinline__ void unpack(C A, C B, double, float sh, float sl, double2& even, double2& odd) {
        const float2 es = dfr_add(A.x, A.y, B.x, B.y);
        const float2 er = dfr_mul(es.x, es.y, sh, sl);
        const float2 ad = dfr_add(A.z, A.w, -B.z, -B.w);
        const float2 ei = dfr_mul(ad.x, ad.y, sh, sl);
        const float2 os = dfr_add(A.z, A.w, B.z, B.w);
        const float2 orr = dfr_mul(os.x, os.y, sh, sl);
        const float2 od = dfr_add(B.x, B.y, -A.x, -A.y);
        const float2 oi = dfr_mul(od.x, od.y, sh, sl);
        even = make_double2(df2d(er.x, er.y), df2d(ei.x, ei.y));
        odd = make_double2(df2d(orr.x, orr.y), df2d(oi.x, oi.y));
    }
};

template <class A>
__device__ __forceinline__ void dft2(typename A::C* v) {
    const typename A::C a = v[0], b = v[1];
    v[0] = A::add(a, b);
    v[1] = A::sub(a, b);
}
template <class A>
__device__ __forceinline__ void dft3(typename A::C* v) {
    // w = e^{-2 pi i/3} = -1/2 - i sqrt(3)/2:  v1 = t2 - i t3, v2 = t2 + i t3
    typedef typename A::C C;
    const C t1 = A::add(v[1], v[2]);
    const C t2 = A::sub(v[0], A::half(t1));
    const C t3 = A::mul_k(A::sub(v[1], v[2]), 0.86602540378443864676);
    v[0] = A::add(v[0], t1);
    v[1] = A::add(t2, A::mul_mi(t3));
    v[2] = A::sub(t2, A::mul_mi(t3));
}
template <class A>
__device__ __forceinline__ void dft4(typename A::C* v) {
    typedef typename A::C C;
    const C s02 = A::add(v[0], v[2]), d02 = A::sub(v[0], v[2]);
    const C s13 = A::add(v[1], v[3]), d13 = A::mul_mi(A::sub(v[1], v[3]));
    v[0] = A::add(s02, s13);
    v[2] = A::sub(s02, s13);
    v[1] = A::add(d02, d13);
    v[3] = A::sub(d02, d13);
}
template <class A>
__device__ __forceinline__ void dft8(typename A::C* v) {
    typedef typename A::C C;
    const double s = 0.70710678118654752440;
    C e[4] = {v[0], v[2], v[4], v[6]};
    C o[4] = {v[1], v[3], v[5], v[7]};
    dft4<A>(e);
    dft4<A>(o);
    // o[k] *= w8^k, w8 = e^{-2 pi i / 8}:  w8 o = s (o - i o),  w8^3 o = s (-i o - o)
    const C o1 = A::mul_k(A::add(o[1], A::mul_mi(o[1])), s);
    const C o2 = A::mul_mi(o[2]);
    const C o3 = A::mul_k(A::sub(A::mul_mi(o[3]), o[3]), s);
    v[0] = A::add(e[0], o[0]);
    v[4] = A::sub(e[0], o[0]);
    v[1] = A::add(e[1], o1);
    v[5] = A::sub(e[1], o1);
    v[2] = A::add(e[2], o2);
    v[6] = A::sub(e[2], o2);
    v[3] = A::add(e[3], o3);
    v[7] = A::sub(e[3], o3);
}

// twiddle W_L^e from shared memory (tw != null) or from the global table
template <class CT>
__device__ __forceinline__ CT twid(const CT* tw, const CT* W, int e, int64_t wstride) {
    return tw ? tw[e] : __ldg(W + (int64_t)e * wstride);
}

// q = x / d from a multiply-high by ceil(2^32 / d): exact whenever x d < 2^32, which every index of the
// two-pass tiles satisfies (x < L cols <= 2^18, d <= 4096); a division by a value known only at run
// time would cost tens of integer instructions per butterfly
// (FAST; the fp64 instantiations keep the plain division, which measured faster there)
template <bool FAST>
struct Recip {
    unsigned m;
    int d;
    __device__ __forceinline__ explicit Recip(int dd)
        : m(FAST && dd > 1 ? (unsigned)((0x100000000ull + (unsigned)dd - 1) / (unsigned)dd) : 0u), d(dd) {}
    __device__ __forceinline__ int div(int x) const {
        if (!FAST) return x / d;
        return d > 1 ? (int)__umulhi((unsigned)x, m) : x;
    }
};

// one Stockham stage over `cols` columns (column c of the tile at buf[l * cols + c])
template <class A, int R>
__device__ __forceinline__ void stage_reg(const typename A::C* src, typename A::C* dst, const typename A::C* tw,
                                          const typename A::C* W, int L, int cols, int Ns, int64_t wstride) {
    const int nb = L / R;
    const int tw_unit = L / (Ns * R);
    const Recip<A::kFastDiv> rc(cols), rn(Ns);
    for (int item = threadIdx.x; item < nb * cols; item += blockDim.x) {
        const int j = rc.div(item), c = item - j * cols;
        const int jq = rn.div(j), jm = j - jq * Ns;
        typename A::C v[R];
#pragma unroll
        for (int r = 0; r < R; ++r) {
            v[r] = src[(j + r * nb) * cols + c];
            if (r > 0 && jm != 0) v[r] = A::mul(v[r], twid(tw, W, jm * r * tw_unit, wstride));
        }
        if (R == 2) dft2<A>(v);
        if (R == 3) dft3<A>(v);
        if (R == 4) dft4<A>(v);
        if (R == 8) dft8<A>(v);
        const int base = jq * Ns * R + jm;
#pragma unroll
        for (int r = 0; r < R; ++r) dst[(base + r * Ns) * cols + c] = A::norm(v[r]);
    }
}

// any radix R: one thread per output element, direct length-R DFT
template <class A>
__device__ __forceinline__ void stage_generic(const typename A::C* src, typename A::C* dst, const typename A::C* tw,
                                              const typename A::C* W, int L, int cols, int Ns, int R,
                                              int64_t wstride) {
    const int nb = L / R;
    const int tw_unit = L / (Ns * R);
    const int unit = L / R;                                   // W_R^1 = W_L^(L/R)
    const Recip<A::kFastDiv> rc(cols), rr(R), rn(Ns);
    for (int item = threadIdx.x; item < L * cols; item += blockDim.x) {
        const int rest = rc.div(item), c = item - rest * cols;
        const int j = rr.div(rest), k = rest - j * R;
        const int jq = rn.div(j), jm = j - jq * Ns;
        typename A::C acc = A::zero();
        for (int r = 0; r < R; ++r) {
            const typename A::C v = src[(j + r * nb) * cols + c];
            const int e = (jm * r * tw_unit + ((r * k) % R) * unit) % L;
            acc = A::add(acc, A::mul(v, twid(tw, W, e, wstride)));
        }
        dst[(jq * Ns * R + jm + k * Ns) * cols + c] = A::norm(acc);
    }
}

// length-L FFT of `cols` columns held in b0; returns the buffer holding the result
template <class A>
__device__ typename A::C* fft_tile(typename A::C* b0, typename A::C* b1, const typename A::C* tw,
                                   const typename A::C* W, const FftArgs& a, int cols) {
    int Ns = 1;
    for (int st = 0; st < a.nst; ++st) {
        const int R = a.radix[st];
        if (R == 8) stage_reg<A, 8>(b0, b1, tw, W, a.L, cols, Ns, a.wstride);
        else if (R == 4) stage_reg<A, 4>(b0, b1, tw, W, a.L, cols, Ns, a.wstride);
        else if (R == 2) stage_reg<A, 2>(b0, b1, tw, W, a.L, cols, Ns, a.wstride);
        else if (R == 3) stage_reg<A, 3>(b0, b1, tw, W, a.L, cols, Ns, a.wstride);
        else stage_generic<A>(b0, b1, tw, W, a.L, cols, Ns, R, a.wstride);
        __syncthreads();
        typename A::C* t = b0;
        b0 = b1;
        b1 = t;
        Ns *= R;
    }
    return b0;
}

template <class CT>
__device__ __forceinline__ void stage_twiddles(CT* tw, const CT* W, int L, int64_t wstride) {
    for (int j = threadIdx.x; j < L; j += blockDim.x) tw[j] = __ldg(W + (int64_t)j * wstride);
}

// ---- pass 1 (two-pass plans): length L1 over i1 for a fixed i2 = o, packed column pairs ----
template <class A>
__global__ void __launch_bounds__(kFftThreads) fft_pass1_kernel(const __grid_constant__ FftArgs a,
                                                                  const typename A::C* W) {
    typedef typename A::C C;
    extern __shared__ __align__(16) unsigned char fraw[];
    C* fbuf = reinterpret_cast<C*>(fraw);
    const int L = a.L, Gt = a.Gt;
    const int ntile = (a.Gp + Gt - 1) / Gt;
    const int o = blockIdx.x / ntile;
    const int c0 = (blockIdx.x % ntile) * Gt;
    C* b0 = fbuf;
    C* b1 = fbuf + (size_t)L * Gt;
    C* tw = (L <= kTwSmem) ? b1 + (size_t)L * Gt : nullptr;            // W_L^j
    C* ot = (L <= kTwSmem) ? tw + L : nullptr;                          // W[(o m) mod M], m < L
    if (tw) {
        stage_twiddles(tw, W, L, a.wstride);
        for (int m = threadIdx.x; m < L; m += blockDim.x) ot[m] = __ldg(W + ((int64_t)o * m) % a.M);
    }
    const Recip<A::kFastDiv> rg(Gt);
    for (int idx = threadIdx.x; idx < L * Gt; idx += blockDim.x) {
        const int l = rg.div(idx), c = idx - l * Gt, g = 2 * (c0 + c);
        const int64_t row = (int64_t)o * a.in_outer + (int64_t)l * a.in_step;
        const double x = g < a.G ? __ldcs(a.Ur + row * a.G + g) : 0.0;
        const double y = g + 1 < a.G ? __ldcs(a.Ur + row * a.G + g + 1) : 0.0;
        b0[idx] = A::pair_trunc(x, y);
    }
    __syncthreads();
    const C* res = fft_tile<A>(b0, b1, tw, W, a, Gt);
    C* Yo = reinterpret_cast<C*>(a.Yo);
    for (int idx = threadIdx.x; idx < L * Gt; idx += blockDim.x) {
        const int m = rg.div(idx), c = idx - m * Gt;
        if (c0 + c >= a.Gp) continue;
        C v = res[idx];
        if (m) v = A::mul(v, ot ? ot[m] : __ldg(W + ((int64_t)o * m) % a.M));
        Yo[((int64_t)m * a.out_m + (int64_t)o * a.out_outer) * a.Gp + c0 + c] = A::norm(v);
    }
}

// ---- final pass: buckets m1 and L1-m1 (length L2 over i2), unpack, gather ----
template <class A>
__global__ void __launch_bounds__(kFftThreads) fft_final_kernel(const __grid_constant__ FftArgs a,
                                                                  const typename A::C* W) {
    typedef typename A::C C;
    extern __shared__ __align__(16) unsigned char fraw[];
    C* fbuf = reinterpret_cast<C*>(fraw);
    const int L = a.L, Gt = a.Gt;
    const int ntile = (a.Gp + Gt - 1) / Gt;
    const int m1 = blockIdx.x / ntile;                  // 0 <= m1 <= L1/2
    const int c0 = (blockIdx.x % ntile) * Gt;
    const int L1 = a.L1;
    const int m1p = (L1 - m1) % L1;                     // partner bucket
    const int nb = (m1p == m1) ? 1 : 2;                 // transforms in this CTA
    const int cols = nb * Gt;                           // column c of bucket b at b * Gt + c
    C* b0 = fbuf;
    C* b1 = fbuf + (size_t)L * cols;
    C* tw = (L <= kTwSmem) ? b1 + (size_t)L * cols : nullptr;
    if (tw) stage_twiddles(tw, W, L, a.wstride);
    const C* Yc = reinterpret_cast<const C*>(a.Yc);
    const Recip<A::kFastDiv> rcol(cols), rg(Gt);
    for (int idx = threadIdx.x; idx < L * cols; idx += blockDim.x) {
        const int l = rcol.div(idx), cc = idx - l * cols;
        const int b = rg.div(cc), c = cc - b * Gt;
        const int bucket = b ? m1p : m1;
        const int64_t row = (int64_t)bucket * a.in_outer + (int64_t)l * a.in_step;
        C v = A::zero();
        if (Yc) {
            if (c0 + c < a.Gp) v = __ldcs(Yc + row * a.Gp + c0 + c);
        } else {
            const int g = 2 * (c0 + c);
            const double x = g < a.G ? __ldcs(a.Ur + row * a.G + g) : 0.0;
            const double y = g + 1 < a.G ? __ldcs(a.Ur + row * a.G + g + 1) : 0.0;
            v = A::pair_trunc(x, y);
        }
        b0[idx] = v;
    }
    __syncthreads();
    const C* Z = fft_tile<A>(b0, b1, tw, W, a, cols);
    // the output scale 1 / (2M): fp64, and its split for the double-float unpack
    const double s_half = 0.5 * a.scale;
    const float s_hi = __double2float_rn(s_half);
    const float s_lo = __double2float_rn(s_half - (double)s_hi);
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
            const C Za = Z[m2 * cols + b * Gt + c];
            const C Zb = Z[m2p * cols + pb * Gt + c];         // Z[M - m], conjugated in the unpack
            double2 even, odd;
            A::unpack(Za, Zb, s_half, s_hi, s_lo, even, odd);
            const int g = 2 * (c0 + c);
            const int64_t k = a.bk[e];
            a.C[(int64_t)g * a.nJ + k] = even;
            if (g + 1 < a.G) a.C[(int64_t)(g + 1) * a.nJ + k] = odd;
        }
    }
}

// ---- single pass, in place (lattices that fit on chip) ---------------------------------------
// The whole length-M transform of CP packed column pairs in shared memory, in place: the samples
// are loaded at their mixed-radix digit-reversed positions (pos_of[i], host-computed), then
// decimation-in-time stages of radix R (8, 4, 2, 3 in registers, others by a direct DFT)
// combine sub-transforms of length L into L R, leaving the spectrum in natural order; the
// gather then reads Z[m_k] and Z[M - m_k] per candidate and writes C[g][k] with consecutive
// threads on consecutive k (coalesced).  Twiddles W_M^e = T1[e mod B] T2[e div B] from two
// small shared tables.  No intermediate array in HBM: the samples are read once and the
// coefficients written once.
// Launch bound: two CTAs per SM (64 registers a thread; the radix-8 double-float butterfly
// spills a few values to L1), which measured 15% faster than one CTA at 106 registers.
static const int kInplaceThreads = 512;
static const int kTwB = 128;

// e < M < 2^31: 32-bit exponent arithmetic (kTwB is a power of two)
template <class A>
__device__ __forceinline__ typename A::C tw_pair(const typename A::C* T1, const typename A::C* T2, unsigned e) {
    const unsigned r = e & (kTwB - 1), q = e / kTwB;
    if (q == 0) return T1[r];
    if (r == 0) return T2[q];
    return A::mul(T1[r], T2[q]);
}

// one radix-R decimation-in-time butterfly of the in-place pass (compile-time R: registers)
template <class A, int R>
__device__ __forceinline__ void inplace_butterfly(typename A::C* buf, int base, int L, int j, unsigned estep, int M,
                                                  const typename A::C* T1, const typename A::C* T2) {
    typedef typename A::C C;
    C v[R];
#pragma unroll
    for (int r = 0; r < R; ++r) {
        v[r] = buf[base + r * L];
        if (r > 0 && j > 0) v[r] = A::mul(v[r], tw_pair<A>(T1, T2, (unsigned)j * (unsigned)r * estep));
    }
    if (R == 8) dft8<A>(v);
    else if (R == 4) dft4<A>(v);
    else if (R == 2) dft2<A>(v);
    else if (R == 3) dft3<A>(v);
    else {   // direct DFT of length R: out[k] = sum_r v[r] W_R^{rk}, W_R = W_M^(M/R)
        C out[R];
        const unsigned unit = (unsigned)(M / R);
#pragma unroll
        for (int k = 0; k < R; ++k) {
            C acc = v[0];
#pragma unroll
            for (int r = 1; r < R; ++r) acc = A::add(acc, A::mul(v[r], tw_pair<A>(T1, T2, (unsigned)((r * k) % R) * unit)));
            out[k] = acc;
        }
#pragma unroll
        for (int k = 0; k < R; ++k) v[k] = out[k];
    }
#pragma unroll
    for (int r = 0; r < R; ++r) buf[base + r * L] = A::norm(v[r]);
}

// One column pair per CTA.  Per butterfly the group index q = bt / L comes from a multiply-high by
// the stage's reciprocal ceil(2^32 / L) in the double-float instantiation (Recip: exact while
// bt L < 2^32, bt < M / R, L <= M <= 14528).
template <class A>
__global__ void __launch_bounds__(kInplaceThreads, 2) fft_inplace_kernel(const __grid_constant__ FftArgs a,
                                                                        const typename A::C* W, const int* pos_of,
                                                                        const int* mk) {
    typedef typename A::C C;
    extern __shared__ __align__(16) unsigned char fraw[];
    const int M = (int)a.M;
    const int nT2 = (M + kTwB - 1) / kTwB;
    C* buf = reinterpret_cast<C*>(fraw);
    C* T1 = buf + M;
    C* T2 = T1 + kTwB;
    const int cp = blockIdx.x;                             // the column pair of this CTA
    const int tid = threadIdx.x, T = blockDim.x;
    for (int r = tid; r < kTwB; r += T) T1[r] = r < M ? __ldg(W + r) : A::zero();
    for (int q = tid; q < nT2; q += T) T2[q] = __ldg(W + (int64_t)q * kTwB);
    // load at the digit-reversed positions
    const int g = 2 * cp;
    const bool hx = g < a.G, hy = g + 1 < a.G;
    for (int i = tid; i < M; i += T) {
        const double* u = a.Ur + (int64_t)i * a.G + g;
        buf[pos_of[i]] = A::pair(hx ? __ldcs(u) : 0.0, hy ? __ldcs(u + 1) : 0.0);
    }
    __syncthreads();
    int L = 1;
    for (int st = 0; st < a.nst; ++st) {
        const int R = a.radix[st];
        const int LR = L * R;
        const unsigned estep = (unsigned)(M / LR);         // W_{LR}^1 = W_M^(M / LR)
        const int nb = M / R;                               // butterflies of the column pair
        const Recip<A::kFastDiv> rl(L);
        for (int bt = tid; bt < nb; bt += T) {
            const int q = rl.div(bt);
            const int j = bt - q * L, base = q * LR + j;
            switch (R) {
                case 8: inplace_butterfly<A, 8>(buf, base, L, j, estep, M, T1, T2); break;
                case 4: inplace_butterfly<A, 4>(buf, base, L, j, estep, M, T1, T2); break;
                case 2: inplace_butterfly<A, 2>(buf, base, L, j, estep, M, T1, T2); break;
                case 3: inplace_butterfly<A, 3>(buf, base, L, j, estep, M, T1, T2); break;
                case 5: inplace_butterfly<A, 5>(buf, base, L, j, estep, M, T1, T2); break;
                default: inplace_butterfly<A, 7>(buf, base, L, j, estep, M, T1, T2); break;
            }
        }
        __syncthreads();
        L = LR;
    }
    // gather and unpack: C[g][k] for the candidates, consecutive threads on consecutive k
    const double s_half = 0.5 * a.scale;
    const float s_hi = __double2float_rn(s_half);
    const float s_lo = __double2float_rn(s_half - (double)s_hi);
    const int nJ = (int)a.nJ;
    double2* Ce = a.C + (int64_t)g * a.nJ;
    for (int k = tid; k < nJ; k += T) {
        const int m = mk[k];
        const int mp = m == 0 ? 0 : M - m;
        double2 even, odd;
        A::unpack(buf[m], buf[mp], s_half, s_hi, s_lo, even, odd);
        Ce[k] = even;
        if (hy) Ce[a.nJ + k] = odd;
    }
}

// one column pair per CTA (110 KB at M = 6912: two CTAs per SM, which the kernel's launch
// bound of two 512-thread CTAs, 64 registers a thread, also lets the register file hold) measured
// faster than two; the second resident CTA hides the shared-memory latency of the stages
static int inplace_cp(int64_t M) {
    const size_t tables = sizeof(double2) * (size_t)(kTwB + (M + kTwB - 1) / kTwB);
    return sizeof(double2) * (size_t)M + tables <= 232448 ? 1 : 0;
}

static int factorize(int L, int* radix);

// positions of the single in-place pass: input row i goes to pos_of[i] (mixed-radix digit
// reversal for the stage radices); empty when M does not fit on chip
std::vector<int> fft_inplace_positions(int64_t M) {
    std::vector<int> pos;
    if (M < 1 || inplace_cp(M) == 0) return pos;
    int radix[32];
    const int S = factorize((int)M, radix);
    for (int st = 0; st < S; ++st)            // the butterflies exist for these radices only
        if (radix[st] != 2 && radix[st] != 3 && radix[st] != 4 && radix[st] != 5 && radix[st] != 7 && radix[st] != 8)
            return pos;
    // position p holds input index perm[p]: the input splits by i mod R_last, recursively
    std::vector<int> perm((size_t)M), tmp((size_t)M);
    for (int64_t i = 0; i < M; ++i) perm[(size_t)i] = (int)i;
    // build perm by repeatedly splitting blocks (outermost split uses the last radix)
    int64_t blocks = 1, len = M;
    for (int s = S - 1; s >= 0; --s) {
        const int R = radix[s];
        const int64_t sub = len / R;
        for (int64_t b = 0; b < blocks; ++b) {
            const int* src = perm.data() + b * len;
            int* dst = tmp.data() + b * len;
            for (int r = 0; r < R; ++r)
                for (int64_t q = 0; q < sub; ++q) dst[r * sub + q] = src[r + q * R];
        }
        perm.swap(tmp);
        blocks *= R;
        len = sub;
    }
    pos.assign((size_t)M, 0);
    for (int64_t p = 0; p < M; ++p) pos[(size_t)perm[(size_t)p]] = (int)p;
    return pos;
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

int fft_default_tile(int L, int Gp, int nb) { return pick_gt(L, Gp, nb); }
bool fft_tile_fits(int L, int Gt, int nb) { return Gt >= 1 && pass_smem(L, nb * Gt) <= 232448; }

// the tuned tile of a pass (usfft_autotune), else the default; clamped to the columns and the
// shared memory
static int pass_tile(int L, int Gp, int nb, bool final_pass) {
    const int def = pick_gt(L, Gp, nb);
    int gt = tune_get(TUNE_FFT_TILE, tune_key_fft(L, final_pass), def);
    if (gt > Gp) gt = Gp;
    return fft_tile_fits(L, gt, nb) ? gt : def;
}

template <class A>
static cudaError_t launch_fft_impl(const FftPlan& p, int G, const double* U, const typename A::C* W,
                                   const GatherPlan& gp, int64_t nJ, void* scratch, double2* C, cudaStream_t s,
                                   int* launches) {
    if (p.M <= 0 || nJ <= 0) return cudaSuccess;
    FftArgs a;
    memset(&a, 0, sizeof(a));
    a.G = G;
    a.Gp = (G + 1) / 2;
    a.M = p.M;
    a.nJ = nJ;
    a.scale = 1.0 / (double)p.M;
    cudaError_t e;
    const int cp = (gp.pos_of && gp.mk) ? inplace_cp(p.M) : 0;
    if (cp > 0) {
        a.Ur = U;
        a.C = C;
        a.nst = factorize((int)p.M, a.radix);
        const size_t smem = sizeof(typename A::C) * ((size_t)p.M + kTwB + (p.M + kTwB - 1) / kTwB);
        e = allow_dyn_smem((const void*)fft_inplace_kernel<A>, smem);
        if (e != cudaSuccess) return e;
        fft_inplace_kernel<A><<<a.Gp, kInplaceThreads, smem, s>>>(a, W, gp.pos_of, gp.mk);
        if (launches) ++*launches;
        return cudaGetLastError();
    }
    if (p.L2 <= 0) return cudaErrorInvalidValue;
    const bool two = p.L1 > 1;
    if (two) {
        // pass 1: length L1 over i1 (rows i1 L2 + i2), outer index i2
        a.L = p.L1;
        a.Gt = pass_tile(a.L, a.Gp, 1, false);
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
        e = allow_dyn_smem((const void*)fft_pass1_kernel<A>, smem);
        if (e != cudaSuccess) return e;
        const int ntile = (a.Gp + a.Gt - 1) / a.Gt;
        fft_pass1_kernel<A><<<(unsigned)((int64_t)a.nOuter * ntile), kFftThreads, smem, s>>>(a, W);
        if (launches) ++*launches;
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    // final pass: length L2 over i2 (rows m1 L2 + i2), bucket pairs {m1, L1 - m1}
    FftArgs b = a;
    b.L = p.L2;
    b.L1 = two ? p.L1 : 1;
    b.Gt = pass_tile(b.L, b.Gp, b.L1 > 2 ? 2 : 1, true);
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
    e = allow_dyn_smem((const void*)fft_final_kernel<A>, smem);
    if (e != cudaSuccess) return e;
    const int ntile = (b.Gp + b.Gt - 1) / b.Gt;
    fft_final_kernel<A><<<(unsigned)((int64_t)b.nOuter * ntile), kFftThreads, smem, s>>>(b, W);
    if (launches) ++*launches;
    return cudaGetLastError();
}

cudaError_t launch_fft_gather(const FftPlan& p, int G, const double* U, const void* W, bool df, const GatherPlan& gp,
                              int64_t nJ, void* scratch, double2* C, cudaStream_t s, int* launches) {
    if (df)
        return launch_fft_impl<DF>(p, G, U, reinterpret_cast<const float4*>(W), gp, nJ, scratch, C, s, launches);
    return launch_fft_impl<F64>(p, G, U, reinterpret_cast<const double2*>(W), gp, nJ, scratch, C, s, launches);
}

}  // namespace usfft
