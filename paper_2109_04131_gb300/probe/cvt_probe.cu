// Throughput of float <-> double conversions on the GPU: the conversion instructions against the
// bit-field conversions of k_cvt.cuh (integer pipe) and against DFMA, thread-ops per clock per
// SM; plus an exactness check of the bit-field versions against the conversion instructions on
// 4M sampled values (normal range).  Each thread runs 8 independent chains; every result feeds
// an XOR sink.  Grid: 2 CTAs of 512 threads per SM, one 8-byte sink store per thread.
// Build and run: nvcc -gencode arch=compute_103a,code=sm_103a -O3 -I paper_2109_04131_gb300/csrc
//                     -o cvt_probe paper_2109_04131_gb300/probe/cvt_probe.cu && ./cvt_probe
#include <cstdio>
#include <cstdint>
#include <cuda_runtime.h>

#include "k_cvt.cuh"

using usfft::d2f_round;
using usfft::f2d_exact;

template <int MODE>
__global__ void __launch_bounds__(512) probe(int iters, unsigned long long* sink, long long* cyc) {
    float f[8];
    double d[8];
    unsigned long long acc = 0;
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        f[j] = 1.0f + 1e-3f * (threadIdx.x + j);
        d[j] = 1.0 + 1e-6 * (threadIdx.x + 3 * j);
    }
    __syncthreads();
    const long long c0 = clock64();
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            if (MODE == 0) {            // DFMA chain
                d[j] = fma(d[j], 0.999999999, 1e-9);
            } else if (MODE == 1) {     // float -> double by the conversion instruction, f advanced on the FP32 pipe
                f[j] = fmaf(f[j], 0.9999999f, 1e-7f);
                acc ^= (unsigned long long)__double_as_longlong((double)f[j]);
            } else if (MODE == 2) {     // same with the bit-field conversion
                f[j] = fmaf(f[j], 0.9999999f, 1e-7f);
                acc ^= (unsigned long long)__double_as_longlong(f2d_exact(f[j]));
            } else if (MODE == 3) {     // no conversion (cost of the surrounding work)
                f[j] = fmaf(f[j], 0.9999999f, 1e-7f);
                acc ^= (unsigned long long)__float_as_uint(f[j]);
            } else if (MODE == 4) {     // double -> float by the conversion instruction; d advanced by an integer add
                d[j] = __longlong_as_double(__double_as_longlong(d[j]) + 12345);
                acc ^= __float_as_uint(__double2float_rn(d[j]));
            } else if (MODE == 5) {     // same with the bit-field conversion
                d[j] = __longlong_as_double(__double_as_longlong(d[j]) + 12345);
                acc ^= __float_as_uint(d2f_round(d[j]));
            } else {                    // no conversion
                d[j] = __longlong_as_double(__double_as_longlong(d[j]) + 12345);
                acc ^= (unsigned long long)__double_as_longlong(d[j]);
            }
        }
    }
    const long long c1 = clock64();
#pragma unroll
    for (int j = 0; j < 8; ++j) acc ^= (unsigned long long)__double_as_longlong(d[j]) ^ __float_as_uint(f[j]);
    const int gid = blockIdx.x * blockDim.x + threadIdx.x;
    sink[gid] = acc;
    if (threadIdx.x == 0) cyc[blockIdx.x] = c1 - c0;
}

// exactness check: f2d_exact == (double)f for every sampled normal float; d2f_round vs round-to-nearest
__global__ void check(unsigned int* bad) {
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;       // 2^22 samples
    const uint32_t fb = (i * 2654435761u) ^ (i << 7);
    const float f = __uint_as_float(fb);
    if (f == f) {
        const double a = (double)f, b = f2d_exact(f);
        const uint32_t fe = (fb >> 23) & 0xff; if (fe != 0 && fe != 255 && __double_as_longlong(a) != __double_as_longlong(b)) atomicAdd(bad, 1u);
    }
    const unsigned long long db = ((unsigned long long)(i * 2246822519u) << 32) | (i * 3266489917u);
    const double x = __longlong_as_double((long long)db);
    if (x == x) {
        const float r0 = __double2float_rn(x), r1 = d2f_round(x);
        const uint32_t xe = (uint32_t)(db >> 52) & 0x7ff; if (xe >= 897 && xe <= 1150 && __float_as_uint(r0) != __float_as_uint(r1)) atomicAdd(bad + 1, 1u);
    }
}

template <int MODE>
static void run(const char* name, int iters, unsigned long long* sink, long long* cyc, int blocks) {
    probe<MODE><<<blocks, 512>>>(iters, sink, cyc);
    cudaDeviceSynchronize();
    probe<MODE><<<blocks, 512>>>(iters, sink, cyc);
    cudaError_t e = cudaDeviceSynchronize();
    long long h[1024];
    cudaMemcpy(h, cyc, sizeof(long long) * blocks, cudaMemcpyDeviceToHost);
    double mean = 0;
    for (int b = 0; b < blocks; ++b) mean += h[b];
    mean /= blocks;
    // thread-ops per SM per clock: blocks/152 resident blocks per SM (all resident at once)
    const double ops = (double)iters * 8 * 512 * ((double)blocks / 152.0);
    printf("%-34s %8.2f thread-ops/clk/SM  (%s)\n", name, ops / mean, cudaGetErrorString(e));
}

int main() {
    const int blocks = 152 * 2, iters = 4096;
    unsigned long long* sink;
    long long* cyc;
    cudaMalloc(&sink, sizeof(unsigned long long) * blocks * 512);
    cudaMalloc(&cyc, sizeof(long long) * blocks);
    unsigned int* bad;
    cudaMalloc(&bad, 8);
    cudaMemset(bad, 0, 8);
    check<<<(1 << 22) / 256, 256>>>(bad);
    unsigned int hb[2] = {0, 0};
    cudaMemcpy(hb, bad, 8, cudaMemcpyDeviceToHost);
    printf("mismatches: float->double %u, double->float %u of %d\n", hb[0], hb[1], 1 << 22);
    cudaFree(bad);
    run<0>("DFMA", iters, sink, cyc, blocks);
    run<1>("cvt float->double (+FFMA,XOR)", iters, sink, cyc, blocks);
    run<2>("bits float->double (+FFMA,XOR)", iters, sink, cyc, blocks);
    run<3>("no conversion (FFMA,XOR)", iters, sink, cyc, blocks);
    run<4>("cvt double->float (+IADD,XOR)", iters, sink, cyc, blocks);
    run<5>("bits double->float (+IADD,XOR)", iters, sink, cyc, blocks);
    run<6>("no conversion (IADD,XOR)", iters, sink, cyc, blocks);
    cudaFree(sink);
    cudaFree(cyc);
    return 0;
}
