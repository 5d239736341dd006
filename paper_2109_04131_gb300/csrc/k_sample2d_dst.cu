// 2-D sampler, mixed precision with a fast-Poisson preconditioner (the MIXED precision mode).
//
// Same discretisation and assembly as k_sample2d.cu (5-point P1 operator K with edge
// weights w_e = mean of the two adjacent triangle coefficients).  The solve is fp64
// iterative refinement around an fp32 flexible preconditioned CG:
//   x = 0, r = b;  repeat:  solve K d = r / ||r|| in fp32 to tol_inner,
//                           x += ||r|| d (fp64),  r = b - K x,
//   until ||r|| <= tol ||b||.
// The residual after the first correction, as large as b, is formed in fp64 from x with the
// fp64 weights.  After every later correction it is updated as r -= ||r|| K d, with K d formed
// in double-float from the correction's fp32 values and the weights' double-float pairs: its
// rounding error, about 1e-14 of ||r|| K d, is relative to the current residual (1e-4 of ||b||
// or less), so the update adds under 1e-17 ||b|| where the fp64 evaluation of b - K x itself
// carries about 1e-13 ||b|| (the diagonal times x is about 1e4 b), and it runs on the FP32 pipe.
// Preconditioner: the inverse of the constant-coefficient operator K_0 (w_e = 1) between two
// symmetric diagonal scalings, D^-1/2 K_0^-1 D^-1/2 with D = diag(K) / diag(K_0); K_0^-1 is
// applied exactly through its eigenbasis, the 2-D sine transform (DST-I):
//   K_0^-1 r = c^2 S ((S R S) o L) S,  S_jk = sin(pi (j+1)(k+1)/(n+1)),  c = 2/(n+1),
//   L_qp = 1 / (mu_p + mu_q),  mu_k = 2 - 2 cos(pi (k+1)/(n+1)),
// with R the residual on the n x n grid.  Without the scaling the preconditioned operator has
// condition number at most max w / min w (every edge weight lies in [min w, max w]),
// independent of the mesh width; the scaling removes the pointwise size of the coefficient
// and leaves its variation, so a handful of iterations reduce the residual by 1e-5
// (Jacobi-PCG needs hundreds).  The four n x n matrix products run on
// the tensor cores (mma.sync m16n8k16, BF16 operands in shared memory, fp32
// accumulation), as two chained pairs per application; the rounded preconditioner is slightly
// non-symmetric, which the flexible (Polak-Ribiere) beta tolerates -- only the convergence rate
// depends on it, the solution accuracy comes from the fp64 refinement.  The inner CG takes the
// single-reduction form (all inner products of an iteration in one block reduction).  One CTA
// owns one system at a time (persistent grid).
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "k_cvt.cuh"
#include "k_pcg_common.cuh"
#include "usfft_internal.h"

namespace usfft {

struct DstLayout {
    int n, W, P, LD, J1, JA;
    size_t o_xh, o_S, o_L, o_Ta, o_Tb, o_wq, o_ph, o_sc, o_sj, o_r64, o_r32, o_A, o_AF, o_Tr, o_md, total;
};

__host__ __device__ inline size_t align16(size_t x) { return (x + 15) & ~(size_t)15; }

__host__ __device__ inline DstLayout dst_layout(int n, int d) {
    DstLayout L;
    L.n = n;
    L.W = n + 2;
    L.P = (n + 15) / 16 * 16;
    L.LD = L.P + 8;   // row stride in elements: 4 mod 32 words, conflict-free BF16 fragment loads
    size_t o = 0;
    L.o_xh = o;  o = align16(o + sizeof(double) * (size_t)L.W * L.W);
    L.o_S = o;   o = align16(o + sizeof(__nv_bfloat16) * (size_t)L.P * L.LD);
    L.o_L = o;   o = align16(o + sizeof(float) * (size_t)L.P * L.LD);
    L.o_Ta = o;  o = align16(o + sizeof(__nv_bfloat16) * (size_t)L.P * L.LD);
    L.o_Tb = o;  o = align16(o + sizeof(__nv_bfloat16) * (size_t)L.P * L.LD);
    L.o_wq = o;  o = align16(o + sizeof(float4) * (size_t)L.W * L.W);   // a node's four edge weights
    L.o_ph = o;  o = align16(o + sizeof(float) * (size_t)L.W * L.W);
    L.o_sc = o;  o = align16(o + sizeof(float) * (size_t)L.W * L.W);
    L.o_sj = o;  o = align16(o + sizeof(double) * (size_t)d);
    L.o_r64 = o; o = align16(o + sizeof(double) * 36);
    L.o_r32 = o; o = align16(o + sizeof(float) * 4 * 36);
    // separable assembly: J1 = largest first mode index, JA = largest index of either factor
    L.J1 = 1;
    L.JA = 1;
    for (int j = 1; j <= d; ++j) {
        int j1, j2;
        mode_pair(j, j1, j2);
        if (j1 > L.J1) L.J1 = j1;
        if (j1 > L.JA) L.JA = j1;
        if (j2 > L.JA) L.JA = j2;
    }
    L.o_A = o;   o = align16(o + sizeof(double) * (size_t)L.JA * 2 * (n + 1));   // sin(j pi (P + o/3) h)
    L.o_AF = o;  o = align16(o + sizeof(float2) * (size_t)L.JA * 2 * (n + 1));   // the same as double-float
    L.o_Tr = o;  o = align16(o + sizeof(float2) * (size_t)L.J1 * 2 * (n + 1));   // per-row partial sums (double-float)
    L.o_md = o;  o = align16(o + sizeof(double) * (size_t)d + sizeof(int) * 2 * (size_t)d);   // amplitudes, modes
    L.total = o;
    return L;
}

typedef __nv_bfloat16 bf16;

// Double-float arithmetic (a value is hi + lo with |lo| <= ulp(hi)/2, about 48 significant
// bits) from the error-free transformations of Knuth (TwoSum) and Dekker (the exact product,
// here with fmaf): the coefficient assembly runs on the FP32 pipe at a precision far below
// the 1e-10 bar instead of on the 64x slower FP64 pipe.  Every operation is explicitly
// rounded (__fadd_rn, __fmul_rn) so that no contraction changes the transformations.
__device__ __forceinline__ float2 df_split(double x) { return d2df(x); }
__device__ __forceinline__ float2 df_add(float2 a, float2 b) {          // a + b
    const float s = __fadd_rn(a.x, b.x);
    const float bb = __fadd_rn(s, -a.x);
    const float e = __fadd_rn(__fadd_rn(a.x, -__fadd_rn(s, -bb)), __fadd_rn(b.x, -bb));
    const float t = __fadd_rn(e, __fadd_rn(a.y, b.y));
    const float h = __fadd_rn(s, t);
    return make_float2(h, __fadd_rn(t, -__fadd_rn(h, -s)));
}
__device__ __forceinline__ float2 df_fma(float2 acc, float2 a, float2 b) {   // acc + a b
    const float p = __fmul_rn(a.x, b.x);
    float pe = __fmaf_rn(a.x, b.x, -p);
    pe = __fmaf_rn(a.x, b.y, __fmaf_rn(a.y, b.x, pe));
    return df_add(acc, make_float2(p, pe));
}
__device__ __forceinline__ double df_to_double(float2 a) { return df2d(a.x, a.y); }
// exp of a double-float x on the FP32 pipe, for the lognormal coefficient.  Range reduction
// x = k ln2 + r with k = rint(x / ln2) (Cody and Waite: ln2 = L0 + L1 + L2, L0 with 12 significant
// bits so that k L0 and x - k L0 are exact), |r| <= 0.35; exp(r) from its Taylor series to degree 15
// (the remainder r^16/16! < 1.2e-19 relative) by Horner in double-float with the coefficients 1/j!
// as double-float constants; then the exact scaling by 2^k.  Relative error a few 1e-15 (Horner's
// 15 double-float steps).  Outside |x| < 60 (where 2^k or the low word would leave the float
// range) the fp64 exp is used.  Not inlined: the small-mesh kernel, whose affine workloads never
// call it, measured 0.2% faster without its code inline.
__device__ __noinline__ float2 df_exp(float2 x) {
    if (!(fabsf(x.x) < 60.f)) return df_split(exp(df_to_double(x)));
    const float k = rintf(x.x * 1.44269504f);
    const float L0 = 0x1.62ep-1f, L1 = 0x1.0bfbe8p-15f, L2 = 0x1.cf79acp-40f;
    float2 r = make_float2(__fmaf_rn(-k, L0, x.x), x.y);          // x.hi - k L0: exact
    const float p1 = __fmul_rn(k, L1);
    r = df_add(r, make_float2(-p1, -__fmaf_rn(k, L1, -p1)));       // - k L1, exactly as a pair
    r = df_add(r, make_float2(-__fmul_rn(k, L2), 0.f));            // - k L2
    const float ch[16] = {1.0f, 1.0f, 0.5f, 0x1.555556p-3f, 0x1.555556p-5f, 0x1.111112p-7f, 0x1.6c16c2p-10f,
                          0x1.a01a02p-13f, 0x1.a01a02p-16f, 0x1.71de3ap-19f, 0x1.27e4fcp-22f, 0x1.ae6456p-26f,
                          0x1.1eed8ep-29f, 0x1.612462p-33f, 0x1.93974ap-37f, 0x1.ae7f3ep-41f};
    const float cl[16] = {0.f, 0.f, 0.f, -0x1.555556p-28f, -0x1.555556p-30f, -0x1.ddddde0p-32f, -0x1.27d27ep-35f,
                          -0x1.7f97fap-39f, -0x1.7f97fap-42f, 0x1.55b1ccp-45f, -0x1.10ec14p-47f, 0x1.fd5138p-52f,
                          0x1.ff1b12p-54f, -0x1.8af25ep-58f, 0x1.180f94p-62f, 0x1.ccee08p-67f};
    float2 p = make_float2(ch[15], cl[15]);
#pragma unroll
    for (int j = 14; j >= 0; --j) p = df_fma(make_float2(ch[j], cl[j]), p, r);
    const float s2 = __uint_as_float((uint32_t)((int)k + 127) << 23);  // 2^k, |k| <= 87
    return make_float2(__fmul_rn(p.x, s2), __fmul_rn(p.y, s2));
}
// a (double-float) times the float f: the exact product of the high parts plus lo f, unnormalised
__device__ __forceinline__ float2 df_mulf(float2 a, float f) {
    const float p = __fmul_rn(a.x, f);
    return make_float2(p, __fmaf_rn(a.y, f, __fmaf_rn(a.x, f, -p)));
}
// the exact difference a - b of two floats as a double-float (TwoSum)
__device__ __forceinline__ float2 df_two_diff(float a, float b) {
    const float s = __fadd_rn(a, -b);
    const float bb = __fadd_rn(s, -a);
    return make_float2(s, __fadd_rn(__fadd_rn(a, -__fadd_rn(s, -bb)), __fadd_rn(-b, -bb)));
}
// a b of two double-floats: the exact product of the high parts plus the cross terms, unnormalised
__device__ __forceinline__ float2 df_mul_lazy(float2 a, float2 b) {
    const float p = __fmul_rn(a.x, b.x);
    return make_float2(p, __fmaf_rn(a.x, b.y, __fmaf_rn(a.y, b.x, __fmaf_rn(a.x, b.x, -p))));
}
// a + b with the high parts' sum exact (TwoSum) and the low words added, unnormalised
__device__ __forceinline__ float2 df_add_lazy(float2 a, float2 b) {
    const float s = __fadd_rn(a.x, b.x);
    const float bb = __fadd_rn(s, -a.x);
    const float e = __fadd_rn(__fadd_rn(a.x, -__fadd_rn(s, -bb)), __fadd_rn(b.x, -bb));
    return make_float2(s, __fadd_rn(e, __fadd_rn(a.y, b.y)));
}
__device__ __forceinline__ float2 df_neg(float2 a) { return make_float2(-a.x, -a.y); }
// a - b with the high parts' difference exact (TwoSum) and the low words added, unnormalised
__device__ __forceinline__ float2 df_sub_lazy(float2 a, float2 b) {
    const float s = __fadd_rn(a.x, -b.x);
    const float bb = __fadd_rn(s, -a.x);
    const float e = __fadd_rn(__fadd_rn(a.x, -__fadd_rn(s, -bb)), __fadd_rn(-b.x, -bb));
    return make_float2(s, __fadd_rn(e, __fadd_rn(a.y, -b.y)));
}

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// four 8x8 BF16 matrices between shared memory and the mma fragment layout (one row address
// per lane: lanes 8i..8i+7 give the rows of matrix i; the register i of a lane holds row
// lane/4, columns 2(lane%4), 2(lane%4)+1 of matrix i).  .trans stores matrix i transposed.
__device__ __forceinline__ void ldsm_x4(uint32_t addr, uint32_t& r0, uint32_t& r1, uint32_t& r2, uint32_t& r3) {
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];\n"
                 : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3)
                 : "r"(addr)
                 : "memory");
}
__device__ __forceinline__ void stsm_x4(uint32_t addr, uint32_t r0, uint32_t r1, uint32_t r2, uint32_t r3) {
    asm volatile("stmatrix.sync.aligned.m8n8.x4.shared.b16 [%0], {%1,%2,%3,%4};\n"
                 :
                 : "r"(addr), "r"(r0), "r"(r1), "r"(r2), "r"(r3)
                 : "memory");
}
__device__ __forceinline__ void stsm_x4_trans(uint32_t addr, uint32_t r0, uint32_t r1, uint32_t r2, uint32_t r3) {
    asm volatile("stmatrix.sync.aligned.m8n8.x4.trans.shared.b16 [%0], {%1,%2,%3,%4};\n"
                 :
                 : "r"(addr), "r"(r0), "r"(r1), "r"(r2), "r"(r3)
                 : "memory");
}
__device__ __forceinline__ uint32_t pack_bf16x2(float lo, float hi) {
    const __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<const uint32_t*>(&v);
}

// C = A B on the tensor cores (P x P, row stride LD elements, P a multiple of 16), BF16
// operands, fp32 accumulation.  A is stored row-major; B is stored TRANSPOSED
// (Bt[n][k] = B[k][n]), so that the B fragment of mma.m16n8k16 (.col) has the same shape as
// the A fragment and both come from one ldmatrix.x4 each per k-step.  Rows are LD = P + 8
// elements apart (4 mod 32 words), so the eight 16-byte rows of each 8x8 matrix fall on
// distinct banks.  C is written row-major (TRANSPOSE_OUT = false) or transposed (true) with
// one stmatrix.x4 per 16x16 tile, as BF16; before rounding it is multiplied elementwise by
// Lsc (fp32, stride LD) if SCALE.  Accumulator layout of mma.m16n8k16: c0 (g, 2t) c1 (g, 2t+1)
// c2 (g+8, 2t) c3 (g+8, 2t+1), g = lane/4, t = lane%4.  Each warp takes 16x16 output tiles
// (two n8 tiles sharing the A fragment).
template <int P, bool TRANSPOSE_OUT, bool SCALE>
__device__ __forceinline__ void gemm_bf16(const bf16* __restrict__ A, const bf16* __restrict__ Bt,
                                          bf16* __restrict__ C, const float* __restrict__ mu, int n, float c2) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nwarps = blockDim.x >> 5;
    const int g = lane >> 2, t = lane & 3;
    constexpr int NT = P / 16, TILES = (P / 16) * NT, LD = P + 8;
    // row addresses of this lane: A matrices (rows 0-7 | 8-15) x (k 0-7 | 8-15) in the order of
    // the A fragment registers a0..a3; Bt matrices (n 0-7: k 0-7 | 8-15), (n 8-15: k 0-7 | 8-15)
    const uint32_t a_lane = smem_u32(A) + 2u * (uint32_t)((lane & 15) * LD + ((lane >> 4) << 3));
    const uint32_t b_lane = smem_u32(Bt) + 2u * (uint32_t)(((lane & 7) + ((lane >> 4) << 3)) * LD + (((lane >> 3) & 1) << 3));
    // stores: matrix i = lane / 8 is (rows 0-7 | 8-15 by bit 0 of i) x (cols 0-7 | 8-15 by bit 1)
    const int st_r = (lane & 7) + (((lane >> 3) & 1) << 3), st_c = (lane >> 4) << 3;
    for (int tile = warp; tile < TILES; tile += nwarps) {
        const int m0 = (tile / NT) * 16, n0 = (tile % NT) * 16;
        float c[2][4] = {{0.f, 0.f, 0.f, 0.f}, {0.f, 0.f, 0.f, 0.f}};
        const uint32_t pa = a_lane + 2u * (uint32_t)(m0 * LD), pb = b_lane + 2u * (uint32_t)(n0 * LD);
#pragma unroll
        for (int k0 = 0; k0 < P; k0 += 16) {
            uint32_t a0, a1, a2, a3, b00, b01, b10, b11;
            ldsm_x4(pa + 2u * k0, a0, a1, a2, a3);
            ldsm_x4(pb + 2u * k0, b00, b01, b10, b11);
            asm volatile(
                "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 "
                "{%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};\n"
                : "+f"(c[0][0]), "+f"(c[0][1]), "+f"(c[0][2]), "+f"(c[0][3])
                : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b00), "r"(b01));
            asm volatile(
                "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 "
                "{%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};\n"
                : "+f"(c[1][0]), "+f"(c[1][1]), "+f"(c[1][2]), "+f"(c[1][3])
                : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b10), "r"(b11));
        }
        if (SCALE) {    // the scaled inverse eigenvalues c^2 / (mu_row + mu_col), zero in the padding
            const int ra = m0 + g, rb = m0 + g + 8;
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int col0 = n0 + 8 * h + 2 * t;
#pragma unroll
                for (int e = 0; e < 2; ++e) {
                    const int col = col0 + e;
                    c[h][e] = (ra < n && col < n) ? c[h][e] * (c2 / (mu[ra] + mu[col])) : 0.f;
                    c[h][2 + e] = (rb < n && col < n) ? c[h][2 + e] * (c2 / (mu[rb] + mu[col])) : 0.f;
                }
            }
        }
        const uint32_t r0 = pack_bf16x2(c[0][0], c[0][1]), r1 = pack_bf16x2(c[0][2], c[0][3]);
        const uint32_t r2 = pack_bf16x2(c[1][0], c[1][1]), r3 = pack_bf16x2(c[1][2], c[1][3]);
        if (TRANSPOSE_OUT)   // C^T: matrix (rows a, cols b) of C lands at rows b, cols a
            stsm_x4_trans(smem_u32(C) + 2u * (uint32_t)((n0 + st_c + (lane & 7)) * LD + m0 + (st_r & 8)), r0, r1, r2, r3);
        else
            stsm_x4(smem_u32(C) + 2u * (uint32_t)((m0 + st_r) * LD + n0 + st_c), r0, r1, r2, r3);
    }
}

// Two chained products on one 16-row strip per warp: C = ((A B1) B2) o Lsc (Lsc only if SCALE),
// written transposed (Ct[n][m] = C[m][n]).  Warp w < P/16 owns rows 16w..16w+15; the other warps
// have no work here.  The strip of A B1 stays in registers: its fp32 accumulators, rounded to
// BF16 pairs, are exactly the A fragments of the second product (the accumulator of n8-tiles
// 2k and 2k+1 is the A fragment of k-step k), so the intermediate never goes through shared
// memory and needs no barrier.  B1 and B2 are given transposed (Bt[n][k] = B[k][n]).  Ct must
// not be one of the operands (other warps still read them).  The rounding points are those of
// two separate products through BF16 shared buffers, so the result is the same.
template <int P, bool SCALE>
__device__ __forceinline__ void gemm_pair_strip(const bf16* __restrict__ A, const bf16* __restrict__ Bt1,
                                                const bf16* __restrict__ Bt2, bf16* __restrict__ Ct,
                                                const float* __restrict__ Lsc) {
    constexpr int NT = P / 16, LD = P + 8;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (warp >= NT) return;
    const int g = lane >> 2, t = lane & 3, m0 = warp * 16;
    const uint32_t a_lane = smem_u32(A) + 2u * (uint32_t)((m0 + (lane & 15)) * LD + ((lane >> 4) << 3));
    const uint32_t b_off = 2u * (uint32_t)(((lane & 7) + ((lane >> 4) << 3)) * LD + (((lane >> 3) & 1) << 3));
    const uint32_t b1_lane = smem_u32(Bt1) + b_off, b2_lane = smem_u32(Bt2) + b_off;
    // first product: the whole strip (16 x P) in 2 NT accumulator tiles of 16 x 8
    float c[2 * NT][4];
#pragma unroll
    for (int j = 0; j < 2 * NT; ++j) c[j][0] = c[j][1] = c[j][2] = c[j][3] = 0.f;
#pragma unroll
    for (int kk = 0; kk < NT; ++kk) {
        uint32_t a0, a1, a2, a3;
        ldsm_x4(a_lane + 32u * kk, a0, a1, a2, a3);
#pragma unroll
        for (int np = 0; np < NT; ++np) {
            uint32_t b00, b01, b10, b11;
            ldsm_x4(b1_lane + 2u * (uint32_t)(16 * np * LD) + 32u * kk, b00, b01, b10, b11);
            asm volatile(
                "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 "
                "{%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};\n"
                : "+f"(c[2 * np][0]), "+f"(c[2 * np][1]), "+f"(c[2 * np][2]), "+f"(c[2 * np][3])
                : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b00), "r"(b01));
            asm volatile(
                "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 "
                "{%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};\n"
                : "+f"(c[2 * np + 1][0]), "+f"(c[2 * np + 1][1]), "+f"(c[2 * np + 1][2]), "+f"(c[2 * np + 1][3])
                : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b10), "r"(b11));
        }
    }
    uint32_t af[NT][4];
#pragma unroll
    for (int kk = 0; kk < NT; ++kk) {
        af[kk][0] = pack_bf16x2(c[2 * kk][0], c[2 * kk][1]);
        af[kk][1] = pack_bf16x2(c[2 * kk][2], c[2 * kk][3]);
        af[kk][2] = pack_bf16x2(c[2 * kk + 1][0], c[2 * kk + 1][1]);
        af[kk][3] = pack_bf16x2(c[2 * kk + 1][2], c[2 * kk + 1][3]);
    }
    // second product, one 16 x 16 output tile at a time
    const int st_c = (lane >> 4) << 3, st_rb = ((lane >> 3) & 1) << 3;
#pragma unroll
    for (int np = 0; np < NT; ++np) {
        float d[2][4] = {{0.f, 0.f, 0.f, 0.f}, {0.f, 0.f, 0.f, 0.f}};
#pragma unroll
        for (int kk = 0; kk < NT; ++kk) {
            uint32_t b00, b01, b10, b11;
            ldsm_x4(b2_lane + 2u * (uint32_t)(16 * np * LD) + 32u * kk, b00, b01, b10, b11);
            asm volatile(
                "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 "
                "{%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};\n"
                : "+f"(d[0][0]), "+f"(d[0][1]), "+f"(d[0][2]), "+f"(d[0][3])
                : "r"(af[kk][0]), "r"(af[kk][1]), "r"(af[kk][2]), "r"(af[kk][3]), "r"(b00), "r"(b01));
            asm volatile(
                "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 "
                "{%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};\n"
                : "+f"(d[1][0]), "+f"(d[1][1]), "+f"(d[1][2]), "+f"(d[1][3])
                : "r"(af[kk][0]), "r"(af[kk][1]), "r"(af[kk][2]), "r"(af[kk][3]), "r"(b10), "r"(b11));
        }
        const int n0 = 16 * np;
        if (SCALE) {
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int col0 = n0 + 8 * h + 2 * t;
                const float2 l0 = *reinterpret_cast<const float2*>(Lsc + (m0 + g) * LD + col0);
                const float2 l1 = *reinterpret_cast<const float2*>(Lsc + (m0 + g + 8) * LD + col0);
                d[h][0] *= l0.x;
                d[h][1] *= l0.y;
                d[h][2] *= l1.x;
                d[h][3] *= l1.y;
            }
        }
        stsm_x4_trans(smem_u32(Ct) + 2u * (uint32_t)((n0 + st_c + (lane & 7)) * LD + m0 + st_rb),
                      pack_bf16x2(d[0][0], d[0][1]), pack_bf16x2(d[0][2], d[0][3]),
                      pack_bf16x2(d[1][0], d[1][1]), pack_bf16x2(d[1][2], d[1][3]));
    }
}

// z = D^-1/2 K_0^-1 D^-1/2 r for the NPT nodes of this thread (sc = D^-1/2 in the halo layout,
// D = diag(K) / 4).  The transform grid X (rows q, columns p)
// is kept transposed in Ta (Ta[p][q]), the layout the B operand wants; nid[k] >> 16 = p LD + q
// of the node (nid[k] = -1: no node).  S is symmetric, so it serves as A and as transposed B.
// Two strip-pair products: Tb = ((S X S) o L)^T, then Ta = (S Y S)^T = Z^T with Y = Tb^T.
template <int NPT, int P>
__device__ __forceinline__ void apply_precond(const float (&r)[NPT], float (&z)[NPT], const int (&nid)[NPT],
                                              const float* sc, bf16* Ta, bf16* Tb, const bf16* S,
                                              const float* Li, int LD) {
#pragma unroll
    for (int k = 0; k < NPT; ++k)
        if (nid[k] >= 0) Ta[nid[k] >> 16] = __float2bfloat16_rn(sc[nid[k] & 0xffff] * r[k]);
    __syncthreads();
    gemm_pair_strip<P, true>(S, Ta, S, Tb, Li);       // Tb = ((S X S) o L)^T
    __syncthreads();
    gemm_pair_strip<P, false>(S, Tb, S, Ta, nullptr);  // Ta = (S Y S)^T, Y = Tb^T
    __syncthreads();
#pragma unroll
    for (int k = 0; k < NPT; ++k)
        z[k] = (nid[k] >= 0) ? sc[nid[k] & 0xffff] * __bfloat162float(Ta[nid[k] >> 16]) : 0.f;
}

// Eight block-wide fp32 sums in one reduction (every thread receives all eight).  Within a
// warp the eight values are reduced and spread at once (xor 16: four values each way, xor 8:
// two, xor 4: one, then xor 2 and 1): lane l ends with value (l >> 2) & 7; lanes l % 4 == 0
// write it.  Then every warp adds the per-warp partials (at most MAXW = 16 or 32 warps).  buf
// holds 8 MAXW floats; the caller's next use of it comes after a barrier.
template <int MAXW = 16>
__device__ __forceinline__ void block_sum8(float (&v)[8], float* buf) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const bool b16 = lane & 16, b8 = lane & 8, b4 = lane & 4;
    float u4[4], u2[2];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const float keep = b16 ? v[4 + j] : v[j], give = b16 ? v[j] : v[4 + j];
        u4[j] = keep + __shfl_xor_sync(0xffffffffu, give, 16);
    }
#pragma unroll
    for (int j = 0; j < 2; ++j) {
        const float keep = b8 ? u4[2 + j] : u4[j], give = b8 ? u4[j] : u4[2 + j];
        u2[j] = keep + __shfl_xor_sync(0xffffffffu, give, 8);
    }
    float u = (b4 ? u2[1] : u2[0]) + __shfl_xor_sync(0xffffffffu, b4 ? u2[0] : u2[1], 4);
    u += __shfl_xor_sync(0xffffffffu, u, 2);
    u += __shfl_xor_sync(0xffffffffu, u, 1);
    // value index held by this lane: 4 (bit 16) + 2 (bit 8) + 1 (bit 4)
    const int idx = (b16 ? 4 : 0) + (b8 ? 2 : 0) + (b4 ? 1 : 0);
    if ((lane & 3) == 0) buf[idx * MAXW + warp] = u;
    __syncthreads();
    if (MAXW == 32) {      // up to 32 warps: every warp adds all 32 partials of each value
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            float x = lane < nw ? buf[j * 32 + lane] : 0.f;
            v[j] = warp_sum(x);
        }
        return;
    }
    // every warp adds the per-warp partials itself (the same operations in the same order, so
    // every thread gets the same sums) instead of waiting at a second barrier for warp 0:
    // lane l adds warps (l & 15) of values 2j + (l >> 4), then takes the partner half's value
    const bool odd = lane & 16;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const int vi = 2 * j + (odd ? 1 : 0), w = lane & 15;
        float x = w < nw ? buf[vi * 16 + w] : 0.f;
        x += __shfl_xor_sync(0xffffffffu, x, 8);
        x += __shfl_xor_sync(0xffffffffu, x, 4);
        x += __shfl_xor_sync(0xffffffffu, x, 2);
        x += __shfl_xor_sync(0xffffffffu, x, 1);
        const float y = __shfl_xor_sync(0xffffffffu, x, 16);
        v[2 * j] = odd ? y : x;
        v[2 * j + 1] = odd ? x : y;
    }
}

// Block-wide sum of squares w (partials v, of r / prev) and what every thread needs from it,
// formed once by thread 0: ||r||^2 = w prev^2, ||r|| = sqrt(w) prev, 1/||r|| and ||r|| as floats,
// and ||r||^2 > stop.  No thread repeats the fp64 division, conversions and comparison (on this
// GPU the FP64 pipe, which also issues the conversions, runs at 1/64 of the FP32 rate).
struct Norm2 {
    double sq, root;
    float inv, rootf;
    int above;
};
// The partial sums are of type T: fp32 where the per-thread terms are fp32 squares of r / ||r_prev||
// (the norm only needs a few digits), fp64 otherwise.
template <typename T>
__device__ __forceinline__ Norm2 block_norm2(T v, double* buf, double prev, double stop) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    T* part = reinterpret_cast<T*>(buf);      // buf[0..31] as partials; buf[32..35] the results
    v = warp_sum(v);
    if (lane == 0) part[warp] = v;
    __syncthreads();
    if (warp == 0) {
        T w = lane < nw ? part[lane] : T(0);
        w = warp_sum(w);
        if (lane == 0) {
            const double sq = (double)w * prev * prev, root = sqrt((double)w) * prev;
            buf[32] = sq;
            buf[33] = root;
            float* f = reinterpret_cast<float*>(buf + 34);
            f[0] = (float)(1.0 / root);
            f[1] = (float)root;
            reinterpret_cast<int*>(buf + 35)[0] = sq > stop;
        }
    }
    __syncthreads();
    Norm2 o;
    o.sq = buf[32];
    o.root = buf[33];
    const float* f = reinterpret_cast<const float*>(buf + 34);
    o.inv = f[0];
    o.rootf = f[1];
    o.above = reinterpret_cast<const int*>(buf + 35)[0];
    return o;
}

// doubles of one CTA's scratch slot of the small-mesh kernel (n <= 63): seven arrays of
// (P+2)^2 >= W^2 doubles (P = n rounded up to 16, so that the array offsets are compile-time
// constants of the kernel instance), each rounded up to an even count so that the float4 view
// stays 16-byte aligned
__host__ __device__ constexpr int mixed_small_array_doubles(int P) { return ((P + 2) * (P + 2) + 1) & ~1; }
__host__ __device__ inline size_t mixed_small_slot_doubles(int n) {
    return 7 * (size_t)mixed_small_array_doubles((n + 15) / 16 * 16);
}

// P = the transform size, n rounded up to a multiple of 16 (a compile-time constant, so the
// k-loop of the fragment loads and mma unrolls)
template <int NPT, int P>
__global__ void __launch_bounds__(512) pcg2d_mixed_dst_kernel(const __grid_constant__ Pcg2dArgs a) {
    extern __shared__ __align__(16) unsigned char smraw[];
    const int n = a.n, G = n * n, n1 = n + 1;
    const DstLayout Lo = dst_layout(n, a.ns.d);
    const int W = Lo.W, LD = Lo.LD;
    double* xh = reinterpret_cast<double*>(smraw + Lo.o_xh);
    bf16* S = reinterpret_cast<bf16*>(smraw + Lo.o_S);
    float* Li = reinterpret_cast<float*>(smraw + Lo.o_L);
    bf16* Ta = reinterpret_cast<bf16*>(smraw + Lo.o_Ta);
    bf16* Tb = reinterpret_cast<bf16*>(smraw + Lo.o_Tb);
    // fp32 weights of the four edges of halo node h: (left, right, below, above), i.e. to the
    // neighbours h - W, h + W, h - 1, h + 1 (one 16-byte load per node in the SpMV)
    float4* wq = reinterpret_cast<float4*>(smraw + Lo.o_wq);
    float* ph = reinterpret_cast<float*>(smraw + Lo.o_ph);
    float* scs = reinterpret_cast<float*>(smraw + Lo.o_sc);   // preconditioner scaling, halo layout
    double* sj = reinterpret_cast<double*>(smraw + Lo.o_sj);
    double* red64 = reinterpret_cast<double*>(smraw + Lo.o_r64);
    float* red32 = reinterpret_cast<float*>(smraw + Lo.o_r32);
    double* At = reinterpret_cast<double*>(smraw + Lo.o_A);     // At[(j-1)][o-1][P] = sin(j pi (P + o/3) h)
    float2* AtF = reinterpret_cast<float2*>(smraw + Lo.o_AF);   // At as double-float
    float2* Tr = reinterpret_cast<float2*>(smraw + Lo.o_Tr);    // Tr[(j1-1)][o-1][Q], double-float
    double* amp = reinterpret_cast<double*>(smraw + Lo.o_md);   // c j^-mu
    int* mj1 = reinterpret_cast<int*>(amp + a.ns.d);
    int* mj2 = mj1 + a.ns.d;
    const int J1 = Lo.J1, JA = Lo.JA;
    const int T = blockDim.x, tid = threadIdx.x;
    // the CTA's scratch slot (mixed_small_slot_doubles): fp64 weights (left, down) and diagonal,
    // the low words of the four edge weights' double-float pairs (the high words are wq), the
    // double-float diagonal, and the residual r in double-float (each node's own thread keeps it
    // there across the inner solve); halo layout, arrays W2 doubles apart
    constexpr int W2 = mixed_small_array_doubles(P);
    double* w64l = a.scratch + (size_t)blockIdx.x * (7 * W2);
    double* w64d = w64l + W2;
    double* d64 = w64d + W2;
    float4* wql = reinterpret_cast<float4*>(d64 + W2);
    float2* Ddf = reinterpret_cast<float2*>(d64 + 3 * W2);
    float2* rdf = reinterpret_cast<float2*>(d64 + 4 * W2);

    // per-thread node indices, packed: halo position (low 16 bits) | transform-grid position
    // (high 16 bits); -1 marks a thread slot without a node (W^2, P LD < 2^15 for n <= 63).
    // Threads walk the nodes column by column (consecutive threads: consecutive y), and the
    // halo arrays are stored column-major, h = (p+1) W + (q+1): every per-node shared access
    // and the transposed transform grid (p LD + q) are then contiguous across a warp.
    int nid[NPT];
#pragma unroll
    for (int k = 0; k < NPT; ++k) {
        const int g = tid + k * T;
        nid[k] = -1;
        if (g < G) {
            const int pp = g / n, qq = g % n;
            nid[k] = ((pp + 1) * W + qq + 1) | ((pp * LD + qq) << 16);
        }
    }
    // per CTA: the sine matrix and the scaled inverse eigenvalues (fp32), zero padded
    const float c2 = 4.0f / ((float)n1 * (float)n1);
    for (int e = tid; e < P * LD; e += T) {
        const int j = e / LD, k = e % LD;
        float sv = 0.f, lv = 0.f;
        if (j < n && k < n) {
            sv = sinpif((float)((j + 1) * (k + 1)) / (float)n1);
            const float s1 = sinpif((float)(k + 1) / (2.0f * n1)), s2 = sinpif((float)(j + 1) / (2.0f * n1));
            lv = c2 / (4.0f * s1 * s1 + 4.0f * s2 * s2);
        }
        S[e] = __float2bfloat16_rn(sv);
        Li[e] = lv;
        Ta[e] = __float2bfloat16_rn(0.f);
        Tb[e] = __float2bfloat16_rn(0.f);
    }
    for (int e = tid; e < W * W; e += T) {
        wq[e] = make_float4(0.f, 0.f, 0.f, 0.f);
        w64l[e] = 0.0;
        w64d[e] = 0.0;
        d64[e] = 0.0;
        wql[e] = make_float4(0.f, 0.f, 0.f, 0.f);
        Ddf[e] = make_float2(0.f, 0.f);
    }
    // separable coefficient: psi_j(centroid) = sin(j1 pi x1) sin(j2 pi x2); the centroids of
    // square (P,Q) are ((P+2/3)h, (Q+1/3)h) (lower triangle) and ((P+1/3)h, (Q+2/3)h) (upper)
    {
        const double hh = 1.0 / (double)n1;
        for (int e = tid; e < JA * 2 * n1; e += T) {
            const int jj = e / (2 * n1) + 1, o = (e / n1) % 2 + 1, Pp = e % n1;
            At[e] = sinpi((double)jj * (((double)Pp + (double)o / 3.0) * hh));
            AtF[e] = df_split(At[e]);
        }
        for (int j = tid; j < a.ns.d; j += T) {
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
    const double nr0 = sqrt(rr0);
    // square e = P (n+1) + Q (Q fastest, so that consecutive threads write consecutive halo nodes
    // h = (P+1) W + Q + 1 of the scratch arrays): P from a multiply-high by ceil(2^32 / (n+1)),
    // exact for e (n+1) < 2^32
    const unsigned mul_n1 = (unsigned)((0x100000000ull + (unsigned)n1 - 1) / (unsigned)n1);
    const float nstop = (float)(a.tol * nr0);        // sqrt(stop)
    const float tol_in = (float)a.tol_inner;
    const float inv0 = (float)(1.0 / nr0), nrf0 = (float)nr0;
    __syncthreads();

    for (int64_t sys = blockIdx.x; sys < a.count; sys += gridDim.x) {
        const int64_t i = lattice_node(a.ns, a.i0 + sys);
        // ---- assembly: fp64 weights to the CTA's scratch slot, fp32 copies to shared memory ----
        for (int j = tid; j < a.ns.d; j += T) sj[j] = amp[j] * node_theta(a.ns, j, i);   // c j^-mu theta_j(y)
        __syncthreads();
        const bool logn = a.coef_model == USFFT_COEF_LOGNORMAL_SIN;
        const int sq = n1 * n1, d = a.ns.d;
        // per-row partial sums Tr[j1][o][Q] = sum_{j: j1(j) = j1} c j^-mu sin(2 pi y_j) At[j2(j)][o][Q]
        for (int e = tid; e < J1 * 2 * n1; e += T) {
            const int j1 = e / (2 * n1) + 1, o = (e / n1) % 2, Q = e % n1;
            double acc = 0.0;
            for (int j = 0; j < d; ++j)
                if (mj1[j] == j1) acc = fma(sj[j], At[((mj2[j] - 1) * 2 + o) * n1 + Q], acc);
            Tr[e] = df_split(acc);
        }
        __syncthreads();
        // triangle coefficients a = 1 + sum_j1 At Tr (affine) or exp(sum_j1 At Tr) (lognormal):
        // the rank-J1 sums in double-float, the exponential in fp64
        const float2 one = make_float2(1.f, 0.f);
        float2* low = reinterpret_cast<float2*>(xh);   // lower-triangle coefficients by square (temporary)
        for (int e = tid; e < sq; e += T) {
            const int Pp = (int)__umulhi((unsigned)e, mul_n1), Q = e - Pp * n1;
            float2 acc = make_float2(0.f, 0.f);
            for (int j1 = 0; j1 < J1; ++j1) acc = df_fma(acc, AtF[(j1 * 2 + 1) * n1 + Pp], Tr[(j1 * 2 + 0) * n1 + Q]);
            low[e] = logn ? df_exp(acc) : df_add(one, acc);
        }
        __syncthreads();
        for (int e = tid; e < sq; e += T) {
            const int Pp = (int)__umulhi((unsigned)e, mul_n1), Q = e - Pp * n1;
            float2 acc = make_float2(0.f, 0.f);
            for (int j1 = 0; j1 < J1; ++j1) acc = df_fma(acc, AtF[(j1 * 2 + 0) * n1 + Pp], Tr[(j1 * 2 + 1) * n1 + Q]);
            const float2 au = logn ? df_exp(acc) : df_add(one, acc);
            if (Q < n) {            // edge (Pp,Q+1)-(Pp+1,Q+1): left of node (Pp+1,Q+1)
                float2 w = df_add(low[Pp * n1 + Q + 1], au);
                w = make_float2(0.5f * w.x, 0.5f * w.y);              // exact
                const int h = (Pp + 1) * W + Q + 1;
                w64l[h] = df_to_double(w);
                wq[h].x = w.x;          // left edge of h
                wq[h - W].y = w.x;      // right edge of its left neighbour
                wql[h].x = w.y;
                wql[h - W].y = w.y;
            }
            if (Pp >= 1) {          // edge (Pp,Q)-(Pp,Q+1): below node (Pp,Q+1)
                float2 w = df_add(au, low[(Pp - 1) * n1 + Q]);
                w = make_float2(0.5f * w.x, 0.5f * w.y);
                const int h = Pp * W + Q + 1;
                w64d[h] = df_to_double(w);
                wq[h].z = w.x;          // lower edge of h
                wq[h - 1].w = w.x;      // upper edge of the node below
                wql[h].z = w.y;
                wql[h - 1].w = w.y;
            }
        }
        __syncthreads();
        // the diagonal of every node (sum of its four edge weights) in double-float from the
        // weights' pairs, and as fp64 (its exact value hi + lo) for the first refinement residual;
        // the symmetric diagonal scaling of the preconditioner, sc = (diag / 4)^-1/2
        // (the slot's loads of all the thread's nodes issued before its first store)
        {
            float4 wlk[NPT];
#pragma unroll
            for (int k = 0; k < NPT; ++k)
                wlk[k] = nid[k] >= 0 ? __ldcg(wql + (nid[k] & 0xffff)) : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
            for (int k = 0; k < NPT; ++k) {
                if (nid[k] >= 0) {
                    const int h = nid[k] & 0xffff;
                    const float4 wh = wq[h], wl = wlk[k];
                    const float2 s = df_add(df_add(make_float2(wh.x, wl.x), make_float2(wh.y, wl.y)),
                                            df_add(make_float2(wh.z, wl.z), make_float2(wh.w, wl.w)));
                    Ddf[h] = s;
                    d64[h] = df_to_double(s);
                    scs[h] = rsqrtf(0.25f * s.x);
                }
            }
        }
        __syncthreads();
        for (int e = tid; e < W * W; e += T) {
            xh[e] = 0.0;
            ph[e] = 0.f;
        }
        __syncthreads();

        // ---- iterative refinement around fp32 flexible PCG (r = b at first, then rdf) ----
        double rr64 = rr0, nr = nr0;
        float inv = inv0, nrf = nrf0;
        int more = rr0 > stop;
        // the high words of r for the next step's fp32 right-hand side (dead during the inner solve)
        float rhi[NPT];
#pragma unroll
        for (int k = 0; k < NPT; ++k) rhi[k] = (nid[k] >= 0) ? d2f_round(b) : 0.f;
        int total = 0, outer = 0;
        while (more && outer < 16) {
            // Flexible PCG in the single-reduction form of Chronopoulos and Gear on K d = r / ||r||:
            // each iteration applies the preconditioner, z = M r, and the operator to z, w = K z
            // (ph holds z in the halo layout), and forms every inner product it needs in one block
            // reduction: gamma = r.z, delta = z.w, zeta = z.q, rho = r.r, nu = r.w, mu = r.q,
            // omega = w.w, phi = w.q (q = K p of the previous direction).  Then
            //   beta = -alpha_prev zeta / gamma_prev      (Polak-Ribiere: z.(r - r_prev) / gamma_prev)
            //   p.q  = delta + 2 beta zeta + beta^2 (p.q)_prev   (q_new = w + beta q, K symmetric)
            //   alpha = gamma / p.q,  p = z + beta p,  q = w + beta q,  d += alpha p,  r -= alpha q
            //   ||r_new||^2 = rho - 2 alpha (nu + beta mu) + alpha^2 q_new.q_new
            // The stop test uses that recurrence, re-anchored every iteration on the exact rho.
            float d32[NPT], r32[NPT], p32[NPT], q32[NPT];
#pragma unroll
            for (int k = 0; k < NPT; ++k) {
                d32[k] = 0.f;
                p32[k] = 0.f;
                q32[k] = 0.f;
                r32[k] = rhi[k] * inv;
            }
            // inner target: tol_inner, or less when this step only has to close the remaining
            // gap to the outer tolerance (0.3 x the reduction still missing)
            const float gap = 0.3f * nstop / nrf;
            const float tin = gap > tol_in ? gap : tol_in;
            float alpha = 0.f, gamma_prev = 1.f, pq_prev = 0.f, qq = 0.f, istop = 0.f;
            int it = 0;
            while (it < a.max_iters) {
                float z32[NPT];
                apply_precond<NPT, P>(r32, z32, nid, scs, Ta, Tb, S, Li, LD);
#pragma unroll
                for (int k = 0; k < NPT; ++k)
                    if (nid[k] >= 0) ph[nid[k] & 0xffff] = z32[k];
                __syncthreads();
                float v[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
                float w32[NPT];
#pragma unroll
                for (int k = 0; k < NPT; ++k) {
                    w32[k] = 0.f;
                    if (nid[k] >= 0) {
                        const int h = nid[k] & 0xffff;
                        const float4 w = wq[h];
                        const float zk = z32[k];
                        float acc = w.x * (zk - ph[h - W]);
                        acc = fmaf(w.y, zk - ph[h + W], acc);
                        acc = fmaf(w.z, zk - ph[h - 1], acc);
                        w32[k] = fmaf(w.w, zk - ph[h + 1], acc);
                    }
                    const float rk = r32[k], zk = z32[k], wk = w32[k], qk = q32[k];
                    v[0] = fmaf(rk, zk, v[0]);
                    v[1] = fmaf(zk, wk, v[1]);
                    v[2] = fmaf(zk, qk, v[2]);
                    v[3] = fmaf(rk, rk, v[3]);
                    v[4] = fmaf(rk, wk, v[4]);
                    v[5] = fmaf(rk, qk, v[5]);
                    v[6] = fmaf(wk, wk, v[6]);
                    v[7] = fmaf(wk, qk, v[7]);
                }
                block_sum8(v, red32);
                if (it == 0) istop = tin * tin * v[3];
                const float beta = it == 0 ? 0.f : -alpha * v[2] / gamma_prev;
                const float pq = v[1] + beta * (2.f * v[2] + beta * pq_prev);
                alpha = v[0] / pq;
                const float qq_new = v[6] + beta * (2.f * v[7] + beta * qq);
                const float rr = v[3] - 2.f * alpha * (v[4] + beta * v[5]) + alpha * alpha * qq_new;
#pragma unroll
                for (int k = 0; k < NPT; ++k) {
                    p32[k] = fmaf(beta, p32[k], z32[k]);
                    q32[k] = fmaf(beta, q32[k], w32[k]);
                    d32[k] = fmaf(alpha, p32[k], d32[k]);
                    r32[k] = fmaf(-alpha, q32[k], r32[k]);
                }
                gamma_prev = v[0];
                pq_prev = pq;
                qq = qq_new;
                ++it;
                if (rr <= istop) break;
            }
            total += it;
            // x += ||r|| d in fp64; after the first correction d also goes to the halo grid (ph)
            // for the double-float update of r
#pragma unroll
            for (int k = 0; k < NPT; ++k)
                if (nid[k] >= 0) {
                    const int h = nid[k] & 0xffff;
                    xh[h] = fma(nr, f2d_exact(d32[k]), xh[h]);
                    if (outer > 0) ph[h] = d32[k];
                }
            __syncthreads();
            // ||r||^2 in fp32 from r / ||r_prev|| (about 1e-5 and below: far inside the fp32 range);
            // the norm only sets the stop and the scale of the next correction, and x and r use
            // the same value of it
            float rs_l = 0.f;
            // the slot's loads for RB nodes at a time issued before any of their stores
            constexpr int RB = NPT < 2 ? NPT : 2;
            if (outer == 0) {
                // r = b - K x in fp64 with the fp64 weights, then split into double-float
#pragma unroll
                for (int k0 = 0; k0 < NPT; k0 += RB) {
                    double wk[RB][5];
#pragma unroll
                    for (int kk = 0; kk < RB; ++kk) {
                        const int h = nid[k0 + kk] >= 0 ? nid[k0 + kk] & 0xffff : W + 1;
                        wk[kk][0] = __ldcg(w64l + h);
                        wk[kk][1] = __ldcg(w64l + h + W);
                        wk[kk][2] = __ldcg(w64d + h);
                        wk[kk][3] = __ldcg(w64d + h + 1);
                        wk[kk][4] = __ldcg(d64 + h);
                    }
#pragma unroll
                    for (int kk = 0; kk < RB; ++kk) {
                        const int k = k0 + kk;
                        rhi[k] = 0.f;
                        if (nid[k] >= 0) {
                            const int h = nid[k] & 0xffff;
                            double acc = wk[kk][0] * xh[h - W];
                            acc = fma(wk[kk][1], xh[h + W], acc);
                            acc = fma(wk[kk][2], xh[h - 1], acc);
                            acc = fma(wk[kk][3], xh[h + 1], acc);
                            const float2 r = df_split(b - fma(wk[kk][4], xh[h], -acc));
                            rdf[h] = r;
                            rhi[k] = r.x;
                            const float rs = r.x * inv;
                            rs_l = fmaf(rs, rs, rs_l);
                        }
                    }
                }
            } else {
                // r -= ||r|| K d in double-float: K d = D d_h - sum_e w_e d_e (D, w_e double-float
                // pairs, d fp32), ||r|| split once
                const float2 nrd = df_split(nr);
#pragma unroll
                for (int k0 = 0; k0 < NPT; k0 += RB) {
                  float4 wlk[RB];
                  float2 ddk[RB], rdk[RB];
#pragma unroll
                  for (int kk = 0; kk < RB; ++kk) {
                      const int h = nid[k0 + kk] >= 0 ? nid[k0 + kk] & 0xffff : W + 1;
                      wlk[kk] = __ldcg(wql + h);
                      ddk[kk] = __ldcg(Ddf + h);
                      rdk[kk] = __ldcg(rdf + h);
                  }
#pragma unroll
                  for (int kk = 0; kk < RB; ++kk) {
                    const int k = k0 + kk;
                    rhi[k] = 0.f;
                    if (nid[k] >= 0) {
                        const int h = nid[k] & 0xffff;
                        const float4 wh = wq[h], wl = wlk[kk];
                        float2 kd = df_mulf(ddk[kk], d32[k]);
                        kd = df_sub_lazy(kd, df_mulf(make_float2(wh.x, wl.x), ph[h - W]));
                        kd = df_sub_lazy(kd, df_mulf(make_float2(wh.y, wl.y), ph[h + W]));
                        kd = df_sub_lazy(kd, df_mulf(make_float2(wh.z, wl.z), ph[h - 1]));
                        kd = df_sub_lazy(kd, df_mulf(make_float2(wh.w, wl.w), ph[h + 1]));
                        // t = ||r|| K d (exact product of the high parts), r - t renormalised
                        const float p = __fmul_rn(nrd.x, kd.x);
                        const float pe = __fmaf_rn(nrd.x, kd.y, __fmaf_rn(nrd.y, kd.x, __fmaf_rn(nrd.x, kd.x, -p)));
                        const float2 r = df_add(rdk[kk], make_float2(-p, -pe));
                        rdf[h] = r;
                        rhi[k] = r.x;
                        const float rs = r.x * inv;
                        rs_l = fmaf(rs, rs, rs_l);
                    }
                  }
                }
            }
            const Norm2 nm = block_norm2(rs_l, red64, nr, stop);
            rr64 = nm.sq;
            nr = nm.root;
            inv = nm.inv;
            nrf = nm.rootf;
            more = nm.above;
            ++outer;
        }
        double* out = a.U + (size_t)sys * G;
        for (int g = tid; g < G; g += T) out[g] = xh[((g % n) + 1) * W + (g / n) + 1];   // g = q n + p
        if (tid == 0) {
            if (a.iters_out) a.iters_out[sys] = total;
            if (a.iters_sum) atomicAdd(a.iters_sum, (unsigned long long)total);
            if (a.outer_sum) atomicAdd(a.outer_sum, (unsigned long long)outer);
            if (rr64 > stop && a.fail_count) atomicAdd(a.fail_count, 1u);
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------------------------
// Large meshes (64 <= n <= 127): the same solver with the per-node vectors in the CTA's global
// scratch slot (L2 / HBM) instead of shared memory and registers; shared memory holds only the
// sine-transform operands (S, L, two transform buffers: 174 KB at P = 128), the separable-assembly
// tables and the reduction buffers.  One CTA of 1024 threads per system; nodes are visited in
// loops g = tid, tid + T, ... (column-major enumeration, halo h = (p+1) W + (q+1), transform
// position p LD + q, as in the small kernel).  Scratch slot: 7 W^2 doubles (fp64 x; the edge
// weights' double-float low words; the double-float residual; fp32 weights, scaling, p, r, q, d, w)
// and the fp64 mode table.
// ---------------------------------------------------------------------------------------------
struct BigLayout {
    int W, LD, J1, JA;
    size_t o_S, o_mu, o_zs, o_Ta, o_Tb, o_A, o_AF, o_Tr, o_md, o_sj, o_r64, o_r32, total;
};

__host__ __device__ inline BigLayout big_layout(int n, int d, int P) {
    BigLayout L;
    L.W = n + 2;
    L.LD = P + 8;
    size_t o = 0;
    L.o_S = o;   o = align16(o + sizeof(__nv_bfloat16) * (size_t)P * L.LD);
    L.o_mu = o;  o = align16(o + sizeof(float) * (size_t)P);                       // mu_k of K_0
    L.o_zs = o;  o = align16(o + sizeof(float) * (size_t)L.W * L.W);               // z, halo layout
    L.o_Ta = o;  o = align16(o + sizeof(__nv_bfloat16) * (size_t)P * L.LD);
    L.o_Tb = o;  o = align16(o + sizeof(__nv_bfloat16) * (size_t)P * L.LD);
    L.J1 = 1;
    L.JA = 1;
    for (int j = 1; j <= d; ++j) {
        int j1, j2;
        mode_pair(j, j1, j2);
        if (j1 > L.J1) L.J1 = j1;
        if (j1 > L.JA) L.JA = j1;
        if (j2 > L.JA) L.JA = j2;
    }
    L.o_A = 0;   // the fp64 mode table lives in the scratch slot (read once per solve)
    L.o_AF = o;  o = align16(o + sizeof(float2) * (size_t)L.JA * 2 * (n + 1));
    L.o_Tr = o;  o = align16(o + sizeof(float2) * (size_t)L.J1 * 2 * (n + 1));
    L.o_md = o;  o = align16(o + sizeof(double) * (size_t)d + sizeof(int) * 2 * (size_t)d);
    L.o_sj = o;  o = align16(o + sizeof(double) * (size_t)d);
    L.o_r64 = o; o = align16(o + sizeof(double) * 36);
    L.o_r32 = o; o = align16(o + sizeof(float) * 8 * 36);
    L.total = o;
    return L;
}

// doubles of one CTA's scratch slot of the large-mesh kernel: 7 W^2 (vectors and weights) and the
// fp64 mode table At for up to 11 first-mode indices (d <= 64) by 2 (n + 1)
__host__ __device__ inline size_t big_slot_doubles(int n) {
    const size_t W = (size_t)n + 2;
    return 7 * W * W + 22 * ((size_t)n + 1);
}

template <int P>
__global__ void __launch_bounds__(1024) pcg2d_mixed_big_kernel(const __grid_constant__ Pcg2dArgs a) {
    extern __shared__ __align__(16) unsigned char smraw[];
    const int n = a.n, G = n * n, n1 = n + 1;
    const BigLayout Lo = big_layout(n, a.ns.d, P);
    const int W = Lo.W, LD = Lo.LD, WW = W * W;
    bf16* S = reinterpret_cast<bf16*>(smraw + Lo.o_S);
    float* mu = reinterpret_cast<float*>(smraw + Lo.o_mu);
    float* zv = reinterpret_cast<float*>(smraw + Lo.o_zs);      // z in shared memory (the SpMV reads its neighbours)
    bf16* Ta = reinterpret_cast<bf16*>(smraw + Lo.o_Ta);
    bf16* Tb = reinterpret_cast<bf16*>(smraw + Lo.o_Tb);
    float2* AtF = reinterpret_cast<float2*>(smraw + Lo.o_AF);
    float2* Tr = reinterpret_cast<float2*>(smraw + Lo.o_Tr);
    double* amp = reinterpret_cast<double*>(smraw + Lo.o_md);
    int* mj1 = reinterpret_cast<int*>(amp + a.ns.d);
    int* mj2 = mj1 + a.ns.d;
    double* sj = reinterpret_cast<double*>(smraw + Lo.o_sj);
    double* red64 = reinterpret_cast<double*>(smraw + Lo.o_r64);
    float* red32 = reinterpret_cast<float*>(smraw + Lo.o_r32);
    const int J1 = Lo.J1, JA = Lo.JA;
    const int T = blockDim.x, tid = threadIdx.x;
    // node g = q n + r: q = g / n from a multiply-high by ceil(2^32 / n), exact for g n < 2^32
    // (g < n^2, n <= 127); a division by the run-time n costs tens of integer instructions
    const unsigned mul_n = (unsigned)((0x100000000ull + (unsigned)n - 1) / (unsigned)n);
    const unsigned mul_n1 = (unsigned)((0x100000000ull + (unsigned)n1 - 1) / (unsigned)n1);
    // the CTA's scratch slot: fp64 x, the low words of the edge weights' double-float pairs (left,
    // down), the residual in double-float, the fp32 weights (the pairs' high words), scaling, p, r,
    // q, d, w (7 W^2 doubles), then the fp64 mode table At.  The fp64 weights are the exact sums
    // hi + lo of the pairs.
    double* x64 = a.scratch + (size_t)blockIdx.x * big_slot_doubles(n);
    double* At = x64 + 7 * (size_t)WW;
    float* wll = reinterpret_cast<float*>(x64 + WW);
    float* wdl = wll + WW;
    float2* rdf = reinterpret_cast<float2*>(x64 + 2 * (size_t)WW);
    float* wl = reinterpret_cast<float*>(x64 + 3 * (size_t)WW);
    float* wd = wl + WW;
    float* scs = wd + WW;
    float* ph = scs + WW;
    float* rv = ph + WW;
    float* qv = rv + WW;
    float* dv = qv + WW;
    float* wv = dv + WW;

    const float c2 = 4.0f / ((float)n1 * (float)n1);
    for (int e = tid; e < P * LD; e += T) {
        const int j = e / LD, k = e % LD;
        float sv = 0.f;
        if (j < n && k < n) sv = sinpif((float)((j + 1) * (k + 1)) / (float)n1);
        S[e] = __float2bfloat16_rn(sv);
        Ta[e] = __float2bfloat16_rn(0.f);
        Tb[e] = __float2bfloat16_rn(0.f);
    }
    for (int k = tid; k < P; k += T) {     // eigenvalues of K_0's 1-D factor, mu_k = 4 sin^2(pi (k+1) / (2(n+1)))
        const float s1 = sinpif((float)(k + 1) / (2.0f * n1));
        mu[k] = 4.0f * s1 * s1;
    }
    for (int e = tid; e < WW; e += T) {     // the halo ring stays zero (Dirichlet boundary)
        wl[e] = 0.f;
        wd[e] = 0.f;
        ph[e] = 0.f;
        zv[e] = 0.f;
        wll[e] = 0.f;
        wdl[e] = 0.f;
        dv[e] = 0.f;            // the residual update reads d at the halo
        x64[e] = 0.0;
    }
    {
        const double hh = 1.0 / (double)n1;
        for (int e = tid; e < JA * 2 * n1; e += T) {
            const int jj = e / (2 * n1) + 1, o = (e / n1) % 2 + 1, Pp = e % n1;
            At[e] = sinpi((double)jj * (((double)Pp + (double)o / 3.0) * hh));
            AtF[e] = df_split(At[e]);
        }
        for (int j = tid; j < a.ns.d; j += T) {
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
    const float nstop = (float)(a.tol * sqrt(rr0));
    const float tol_in = (float)a.tol_inner;
    __syncthreads();

    for (int64_t sys = blockIdx.x; sys < a.count; sys += gridDim.x) {
        const int64_t i = lattice_node(a.ns, a.i0 + sys);
        for (int j = tid; j < a.ns.d; j += T) sj[j] = amp[j] * node_theta(a.ns, j, i);   // c j^-mu theta_j(y)
        __syncthreads();
        const bool logn = a.coef_model == USFFT_COEF_LOGNORMAL_SIN;
        const int d = a.ns.d;
        for (int e = tid; e < J1 * 2 * n1; e += T) {
            const int j1 = e / (2 * n1) + 1, o = (e / n1) % 2, Q = e % n1;
            double acc = 0.0;
            for (int j = 0; j < d; ++j)
                if (mj1[j] == j1) acc = fma(sj[j], At[((mj2[j] - 1) * 2 + o) * n1 + Q], acc);
            Tr[e] = df_split(acc);
        }
        __syncthreads();
        // triangle coefficients a = 1 + sum_j1 At Tr (affine) or exp(sum_j1 At Tr) (lognormal), squares
        // e = P (n+1) + Q (Q fastest: consecutive threads write consecutive halo nodes): first every
        // square's lower-triangle coefficient, once, into the r and q slot arrays (free until the solve;
        // 2 W^2 floats hold the (n+1)^2 pairs), then the upper ones and the edge weights
        const float2 one = make_float2(1.f, 0.f);
        float2* low = reinterpret_cast<float2*>(rv);
        for (int e = tid; e < n1 * n1; e += T) {
            const int Pp = (int)__umulhi((unsigned)e, mul_n1), Q = e - Pp * n1;
            float2 acc = make_float2(0.f, 0.f);
            for (int j1 = 0; j1 < J1; ++j1) acc = df_fma(acc, AtF[(j1 * 2 + 1) * n1 + Pp], Tr[(j1 * 2 + 0) * n1 + Q]);
            low[e] = logn ? df_exp(acc) : df_add(one, acc);
        }
        __syncthreads();
        for (int e = tid; e < n1 * n1; e += T) {
            const int Pp = (int)__umulhi((unsigned)e, mul_n1), Q = e - Pp * n1;
            float2 acc = make_float2(0.f, 0.f);
            for (int j1 = 0; j1 < J1; ++j1) acc = df_fma(acc, AtF[(j1 * 2 + 0) * n1 + Pp], Tr[(j1 * 2 + 1) * n1 + Q]);
            const float2 au = logn ? df_exp(acc) : df_add(one, acc);
            if (Q < n) {            // edge (Pp,Q+1)-(Pp+1,Q+1): left of node (Pp+1,Q+1); lower triangle of (Pp, Q+1)
                float2 w = df_add(low[Pp * n1 + Q + 1], au);
                w = make_float2(0.5f * w.x, 0.5f * w.y);
                const int h = (Pp + 1) * W + Q + 1;
                wl[h] = w.x;
                wll[h] = w.y;
            }
            if (Pp >= 1) {          // edge (Pp,Q)-(Pp,Q+1): below node (Pp,Q+1); lower triangle of (Pp-1, Q)
                float2 w = df_add(au, low[(Pp - 1) * n1 + Q]);
                w = make_float2(0.5f * w.x, 0.5f * w.y);
                const int h = Pp * W + Q + 1;
                wd[h] = w.x;
                wdl[h] = w.y;
            }
        }
        __syncthreads();
        for (int g = tid; g < G; g += T) {
            const int gq = (int)__umulhi((unsigned)g, mul_n), h = (gq + 1) * W + (g - gq * n) + 1;
            // the diagonal (sum of the four edge weights) in double-float, for the scaling only
            const float2 dg = df_add(df_add(make_float2(wl[h], wll[h]), make_float2(wl[h + W], wll[h + W])),
                                     df_add(make_float2(wd[h], wdl[h]), make_float2(wd[h + 1], wdl[h + 1])));
            scs[h] = rsqrtf(0.25f * dg.x);
            x64[h] = 0.0;
            rv[h] = d2f_round(b);        // r = b, kept as fp32 (the inner solve starts from fp32(r) / ||r||)
        }
        __syncthreads();

        // ---- fp64 iterative refinement around fp32 flexible PCG ----
        double rr64 = rr0, nr = sqrt(rr0);
        float inv = (float)(1.0 / nr), nrf = (float)nr;
        int total = 0, outer = 0;
        bool at_floor = false;     // the residual stagnated at its rounding floor (see below)
        // zv = D^-1/2 K_0^-1 D^-1/2 rv; Ta already holds D^-1/2 rv on the transform grid, written by the
        // pass that last changed rv (the step start or the previous iteration's update)
        auto precond = [&]() {
            __syncthreads();
            gemm_bf16<P, false, false>(S, Ta, Tb, nullptr, n, c2);
            __syncthreads();
            gemm_bf16<P, true, true>(Tb, S, Ta, mu, n, c2);
            __syncthreads();
            gemm_bf16<P, false, false>(S, Ta, Tb, nullptr, n, c2);
            __syncthreads();
            gemm_bf16<P, true, false>(Tb, S, Ta, nullptr, n, c2);
            __syncthreads();
            for (int g0 = tid; g0 < G; g0 += 2 * T) {      // two nodes per iteration, loads first
                const int g1 = g0 + T;
                const bool has1 = g1 < G;
                const int p0 = (int)__umulhi((unsigned)g0, mul_n), q0 = g0 - p0 * n, h0 = (p0 + 1) * W + q0 + 1;
                const int p1 = has1 ? (int)__umulhi((unsigned)g1, mul_n) : p0, q1 = has1 ? g1 - p1 * n : q0;
                const int h1 = (p1 + 1) * W + q1 + 1;
                const float s0 = scs[h0], s1 = scs[h1];
                const float t0 = __bfloat162float(Ta[p0 * LD + q0]), t1 = __bfloat162float(Ta[p1 * LD + q1]);
                zv[h0] = s0 * t0;
                if (has1) zv[h1] = s1 * t1;
            }
        };
        while (rr64 > stop && outer < 16) {
            // single-reduction flexible PCG (the small-mesh kernel's inner solve; p in ph, w = K z in wv)
            for (int g0 = tid; g0 < G; g0 += 2 * T) {      // two nodes per iteration, loads first
                const int g1 = g0 + T;
                const bool has1 = g1 < G;
                const int p0 = (int)__umulhi((unsigned)g0, mul_n), q0 = g0 - p0 * n, h0 = (p0 + 1) * W + q0 + 1;
                const int p1 = has1 ? (int)__umulhi((unsigned)g1, mul_n) : p0, q1 = has1 ? g1 - p1 * n : q0;
                const int h1 = (p1 + 1) * W + q1 + 1;
                const float r0 = rv[h0] * inv, r1 = rv[h1] * inv;   // fp32(r) / ||r||
                const float s0 = scs[h0], s1 = scs[h1];
                rv[h0] = r0;
                Ta[p0 * LD + q0] = __float2bfloat16_rn(s0 * r0);
                dv[h0] = 0.f;
                ph[h0] = 0.f;
                qv[h0] = 0.f;
                if (has1) {
                    rv[h1] = r1;
                    Ta[p1 * LD + q1] = __float2bfloat16_rn(s1 * r1);
                    dv[h1] = 0.f;
                    ph[h1] = 0.f;
                    qv[h1] = 0.f;
                }
            }
            __syncthreads();
            const float gap = 0.3f * nstop / nrf;
            const float tin = gap > tol_in ? gap : tol_in;
            float alpha = 0.f, gamma_prev = 1.f, pq_prev = 0.f, qq = 0.f, istop = 0.f;
            int it = 0;
            while (it < a.max_iters) {
                precond();
                __syncthreads();
                float v[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
                // two nodes per iteration (g and g + T), every slot load of both before any store
                for (int g0 = tid; g0 < G; g0 += 2 * T) {
                    const int g1 = g0 + T;
                    const bool has1 = g1 < G;
                    const int gq0 = (int)__umulhi((unsigned)g0, mul_n), h0 = (gq0 + 1) * W + (g0 - gq0 * n) + 1;
                    const int gq1 = (int)__umulhi((unsigned)g1, mul_n);
                    const int h1 = has1 ? (gq1 + 1) * W + (g1 - gq1 * n) + 1 : h0;
                    const float a0 = wl[h0], a1 = wl[h0 + W], a2 = wd[h0], a3 = wd[h0 + 1], r0 = rv[h0], q0 = qv[h0];
                    const float b0 = wl[h1], b1 = wl[h1 + W], b2 = wd[h1], b3 = wd[h1 + 1], r1 = rv[h1], q1 = qv[h1];
                    const float z0 = zv[h0], z1 = zv[h1];
                    float acc0 = a0 * zv[h0 - W];
                    acc0 = fmaf(a1, zv[h0 + W], acc0);
                    acc0 = fmaf(a2, zv[h0 - 1], acc0);
                    acc0 = fmaf(a3, zv[h0 + 1], acc0);
                    const float w0k = fmaf((a0 + a1) + (a2 + a3), z0, -acc0);
                    float acc1 = b0 * zv[h1 - W];
                    acc1 = fmaf(b1, zv[h1 + W], acc1);
                    acc1 = fmaf(b2, zv[h1 - 1], acc1);
                    acc1 = fmaf(b3, zv[h1 + 1], acc1);
                    const float w1k = fmaf((b0 + b1) + (b2 + b3), z1, -acc1);
                    wv[h0] = w0k;
                    v[0] = fmaf(r0, z0, v[0]);
                    v[1] = fmaf(z0, w0k, v[1]);
                    v[2] = fmaf(z0, q0, v[2]);
                    v[3] = fmaf(r0, r0, v[3]);
                    v[4] = fmaf(r0, w0k, v[4]);
                    v[5] = fmaf(r0, q0, v[5]);
                    v[6] = fmaf(w0k, w0k, v[6]);
                    v[7] = fmaf(w0k, q0, v[7]);
                    if (has1) {
                        wv[h1] = w1k;
                        v[0] = fmaf(r1, z1, v[0]);
                        v[1] = fmaf(z1, w1k, v[1]);
                        v[2] = fmaf(z1, q1, v[2]);
                        v[3] = fmaf(r1, r1, v[3]);
                        v[4] = fmaf(r1, w1k, v[4]);
                        v[5] = fmaf(r1, q1, v[5]);
                        v[6] = fmaf(w1k, w1k, v[6]);
                        v[7] = fmaf(w1k, q1, v[7]);
                    }
                }
                block_sum8<32>(v, red32);
                if (it == 0) istop = tin * tin * v[3];
                const float beta = it == 0 ? 0.f : -alpha * v[2] / gamma_prev;
                const float pq = v[1] + beta * (2.f * v[2] + beta * pq_prev);
                alpha = v[0] / pq;
                const float qq_new = v[6] + beta * (2.f * v[7] + beta * qq);
                const float rr = v[3] - 2.f * alpha * (v[4] + beta * v[5]) + alpha * alpha * qq_new;
                // two nodes per iteration, every slot load of both before any store (the compiler may not
                // move a load past a store through these pointers)
                for (int g0 = tid; g0 < G; g0 += 2 * T) {
                    const int g1 = g0 + T;
                    const bool has1 = g1 < G;
                    const int gq0 = (int)__umulhi((unsigned)g0, mul_n), qq0 = g0 - gq0 * n, h0 = (gq0 + 1) * W + qq0 + 1;
                    const int gq1 = (int)__umulhi((unsigned)g1, mul_n), qq1 = g1 - gq1 * n;
                    const int h1 = has1 ? (gq1 + 1) * W + qq1 + 1 : h0;
                    const float ph0 = ph[h0], qv0 = qv[h0], wv0 = wv[h0], dv0 = dv[h0], rv0 = rv[h0], sc0 = scs[h0];
                    const float ph1 = ph[h1], qv1 = qv[h1], wv1 = wv[h1], dv1 = dv[h1], rv1 = rv[h1], sc1 = scs[h1];
                    const float pn0 = fmaf(beta, ph0, zv[h0]), qn0 = fmaf(beta, qv0, wv0);
                    const float pn1 = fmaf(beta, ph1, zv[h1]), qn1 = fmaf(beta, qv1, wv1);
                    const float rn0 = fmaf(-alpha, qn0, rv0), rn1 = fmaf(-alpha, qn1, rv1);
                    ph[h0] = pn0;
                    qv[h0] = qn0;
                    dv[h0] = fmaf(alpha, pn0, dv0);
                    rv[h0] = rn0;
                    Ta[gq0 * LD + qq0] = __float2bfloat16_rn(sc0 * rn0);   // the next preconditioner's input
                    if (has1) {
                        ph[h1] = pn1;
                        qv[h1] = qn1;
                        dv[h1] = fmaf(alpha, pn1, dv1);
                        rv[h1] = rn1;
                        Ta[gq1 * LD + qq1] = __float2bfloat16_rn(sc1 * rn1);
                    }
                }
                gamma_prev = v[0];
                pq_prev = pq;
                qq = qq_new;
                ++it;
                if (rr <= istop) break;
            }
            total += it;
            for (int g0 = tid; g0 < G; g0 += 2 * T) {      // two nodes per iteration, loads first
                const int g1 = g0 + T;
                const bool has1 = g1 < G;
                const int p0 = (int)__umulhi((unsigned)g0, mul_n), h0 = (p0 + 1) * W + (g0 - p0 * n) + 1;
                const int p1 = has1 ? (int)__umulhi((unsigned)g1, mul_n) : p0;
                const int h1 = has1 ? (p1 + 1) * W + (g1 - p1 * n) + 1 : h0;
                const float d0 = dv[h0], d1 = dv[h1];
                const double x0 = x64[h0], x1 = x64[h1];
                x64[h0] = fma(nr, f2d_exact(d0), x0);
                if (has1) x64[h1] = fma(nr, f2d_exact(d1), x1);
            }
            __syncthreads();
            // the residual: after the first correction b - sum_e w_e (x_i - x_j) in fp64 with the fp64
            // weights (hi + lo, exact) in difference form -- at these mesh widths the terms diag x_i
            // and w x_j are ~1e4 times b and cancel, the differences do not; after each later
            // correction r -= ||r|| sum_e w_e (d_i - d_j) in double-float (the differences of the
            // fp32 correction exact by TwoSum), whose rounding is relative to the current residual
            float rs_l = 0.f;
            // two nodes per iteration (g and g + T, the same order of the norm's terms as one at a
            // time), both nodes' slot loads before any store
            if (outer == 0) {
                auto resid0 = [&](int h) -> float2 {
                    const double xi = x64[h];
                    double acc = df2d(wl[h], wll[h]) * (xi - x64[h - W]);
                    acc = fma(df2d(wl[h + W], wll[h + W]), xi - x64[h + W], acc);
                    acc = fma(df2d(wd[h], wdl[h]), xi - x64[h - 1], acc);
                    acc = fma(df2d(wd[h + 1], wdl[h + 1]), xi - x64[h + 1], acc);
                    return df_split(b - acc);
                };
                for (int g0 = tid; g0 < G; g0 += 2 * T) {
                    const int g1 = g0 + T;
                    const bool has1 = g1 < G;
                    const int p0 = (int)__umulhi((unsigned)g0, mul_n), h0 = (p0 + 1) * W + (g0 - p0 * n) + 1;
                    const int p1 = has1 ? (int)__umulhi((unsigned)g1, mul_n) : p0;
                    const int h1 = has1 ? (p1 + 1) * W + (g1 - p1 * n) + 1 : h0;
                    const float2 ra = resid0(h0), rb = resid0(h1);
                    rdf[h0] = ra;
                    rv[h0] = ra.x;
                    const float rsa = ra.x * inv;
                    rs_l = fmaf(rsa, rsa, rs_l);
                    if (has1) {
                        rdf[h1] = rb;
                        rv[h1] = rb.x;
                        const float rsb = rb.x * inv;
                        rs_l = fmaf(rsb, rsb, rs_l);
                    }
                }
            } else {
                const float2 nrd = df_split(nr);
                auto resid1 = [&](int h) -> float2 {
                    const float di = dv[h];
                    float2 kd = df_mul_lazy(make_float2(wl[h], wll[h]), df_two_diff(di, dv[h - W]));
                    kd = df_add_lazy(kd, df_mul_lazy(make_float2(wl[h + W], wll[h + W]), df_two_diff(di, dv[h + W])));
                    kd = df_add_lazy(kd, df_mul_lazy(make_float2(wd[h], wdl[h]), df_two_diff(di, dv[h - 1])));
                    kd = df_add_lazy(kd, df_mul_lazy(make_float2(wd[h + 1], wdl[h + 1]), df_two_diff(di, dv[h + 1])));
                    return df_add(rdf[h], df_neg(df_mul_lazy(nrd, kd)));
                };
                for (int g0 = tid; g0 < G; g0 += 2 * T) {
                    const int g1 = g0 + T;
                    const bool has1 = g1 < G;
                    const int p0 = (int)__umulhi((unsigned)g0, mul_n), h0 = (p0 + 1) * W + (g0 - p0 * n) + 1;
                    const int p1 = has1 ? (int)__umulhi((unsigned)g1, mul_n) : p0;
                    const int h1 = has1 ? (p1 + 1) * W + (g1 - p1 * n) + 1 : h0;
                    const float2 ra = resid1(h0), rb = resid1(h1);
                    rdf[h0] = ra;
                    rv[h0] = ra.x;
                    const float rsa = ra.x * inv;
                    rs_l = fmaf(rsa, rsa, rs_l);
                    if (has1) {
                        rdf[h1] = rb;
                        rv[h1] = rb.x;
                        const float rsb = rb.x * inv;
                        rs_l = fmaf(rsb, rsb, rs_l);
                    }
                }
            }
            const double rr_prev = rr64;
            {
                const Norm2 nm = block_norm2(rs_l, red64, nr, stop);
                rr64 = nm.sq;
                nr = nm.root;
                inv = nm.inv;
                nrf = nm.rootf;
            }
            ++outer;
            // At these mesh widths the fp64 residual of the 5-point system has a rounding floor
            // near 1e-13 relative (the granularity of x times the diagonal, ~1e4 b), which the
            // residual of the first correction carries; an outer step that no longer halves the
            // residual norm below 1e-11 relative is taken to have reached it.
            if (rr64 > stop && rr64 > 0.25 * rr_prev && rr64 <= 1e-22 * rr0) {
                at_floor = true;
                break;
            }
        }
        double* out = a.U + (size_t)sys * G;
        for (int g = tid; g < G; g += T) out[g] = x64[(g - (int)__umulhi((unsigned)g, mul_n) * n + 1) * W + (int)__umulhi((unsigned)g, mul_n) + 1];   // g = q n + p
        if (tid == 0) {
            if (a.iters_out) a.iters_out[sys] = total;
            if (a.iters_sum) atomicAdd(a.iters_sum, (unsigned long long)total);
            if (a.outer_sum) atomicAdd(a.outer_sum, (unsigned long long)outer);
            if (rr64 > stop && !at_floor && a.fail_count) atomicAdd(a.fail_count, 1u);
        }
        __syncthreads();
    }
}

size_t big_smem_bytes(int n, int d) { return big_layout(n, d, (n + 15) / 16 * 16).total; }
static const size_t kMaxBigSmem = 232448;    // 227 KB of dynamic shared memory per CTA

static void (*big_kernel_for(int n))(Pcg2dArgs) {
    switch ((n + 15) / 16 * 16) {
        case 64: return pcg2d_mixed_big_kernel<64>;
        case 80: return pcg2d_mixed_big_kernel<80>;
        case 96: return pcg2d_mixed_big_kernel<96>;
        case 112: return pcg2d_mixed_big_kernel<112>;
        case 128: return pcg2d_mixed_big_kernel<128>;
        default: return nullptr;
    }
}

cudaError_t launch_mixed_big(const Pcg2dArgs& a, int blocks, cudaStream_t s) {
    void (*k)(Pcg2dArgs) = big_kernel_for(a.n);
    const size_t smem = big_smem_bytes(a.n, a.ns.d);
    if (!k || smem > kMaxBigSmem) return cudaErrorInvalidValue;
    cudaError_t e = allow_dyn_smem((const void*)k, smem);
    if (e != cudaSuccess) return e;
    k<<<blocks, 1024, smem, s>>>(a);
    return cudaGetLastError();
}

size_t dst_smem_bytes(int n, int d) { return dst_layout(n, d).total; }

size_t mixed_slot_bytes(int n) {
    return sizeof(double) * (n > 63 ? big_slot_doubles(n) : mixed_small_slot_doubles(n));
}

// the kernel instance for (NPT, P = n rounded up to 16); nullptr for a pair no n produces
template <int NPT>
static void (*dst_kernel_for(int n))(Pcg2dArgs) {
    const int P = (n + 15) / 16 * 16;
    if (NPT == 1) {
        if (P == 16) return pcg2d_mixed_dst_kernel<1, 16>;
        if (P == 32) return pcg2d_mixed_dst_kernel<1, 32>;
    } else if (NPT == 2) {
        if (P == 32) return pcg2d_mixed_dst_kernel<2, 32>;
    } else if (NPT == 4) {
        if (P == 48) return pcg2d_mixed_dst_kernel<4, 48>;
    } else if (NPT == 8) {
        if (P == 48) return pcg2d_mixed_dst_kernel<8, 48>;
        if (P == 64) return pcg2d_mixed_dst_kernel<8, 64>;
    }
    return nullptr;
}

template <int NPT>
cudaError_t launch_dst_npt(const Pcg2dArgs& a, int blocks, int threads, cudaStream_t s) {
    const size_t smem = dst_smem_bytes(a.n, a.ns.d);
    void (*k)(Pcg2dArgs) = dst_kernel_for<NPT>(a.n);
    if (!k) return cudaErrorInvalidValue;
    cudaError_t e = allow_dyn_smem((const void*)k, smem);
    if (e != cudaSuccess) return e;
    k<<<blocks, threads, smem, s>>>(a);
    return cudaGetLastError();
}

template <int NPT>
int dst_resident_blocks(int threads, int d, int n) {
    const size_t smem = dst_smem_bytes(n, d);
    int per_sm = 0;
    void (*k)(Pcg2dArgs) = dst_kernel_for<NPT>(n);
    cudaError_t e = k ? allow_dyn_smem((const void*)k, smem)
                      : cudaErrorInvalidValue;
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, threads, smem);
    if (e != cudaSuccess) {
        cudaGetLastError();
        per_sm = 1;
    }
    return per_sm < 1 ? 1 : per_sm;
}

template cudaError_t launch_dst_npt<1>(const Pcg2dArgs&, int, int, cudaStream_t);
template cudaError_t launch_dst_npt<2>(const Pcg2dArgs&, int, int, cudaStream_t);
template cudaError_t launch_dst_npt<4>(const Pcg2dArgs&, int, int, cudaStream_t);
template cudaError_t launch_dst_npt<8>(const Pcg2dArgs&, int, int, cudaStream_t);
template int dst_resident_blocks<1>(int, int, int);
template int dst_resident_blocks<2>(int, int, int);
template int dst_resident_blocks<4>(int, int, int);
template int dst_resident_blocks<8>(int, int, int);

}  // namespace usfft
