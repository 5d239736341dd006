// FP64 and FP32 FMA throughput of the GPU: 8 independent FMA chains per thread, 8 CTAs of
// 256 threads per SM, timed with CUDA events.  Used for the ALU peaks of the roofline.
// Build and run: bench.py --alu-probe (nvcc -gencode arch=compute_103a,code=sm_103a).
#include <cstdio>
#include <cuda_runtime.h>

template <typename T>
__global__ void fma_chains(T* out, int iters, T a, T b) {
    T x[8];
    for (int k = 0; k < 8; ++k) x[k] = (T)(threadIdx.x + k);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int k = 0; k < 8; ++k) x[k] = fma(x[k], a, b);
    }
    T s = 0;
    for (int k = 0; k < 8; ++k) s += x[k];
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

template <typename T>
static double run(int iters) {
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, 0);
    const int blocks = sms * 8, threads = 256;
    T* out = nullptr;
    if (cudaMalloc(&out, sizeof(T) * blocks * threads) != cudaSuccess) return -1.0;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    fma_chains<T><<<blocks, threads>>>(out, 100, (T)0.999, (T)0.001);
    cudaEventRecord(e0);
    fma_chains<T><<<blocks, threads>>>(out, iters, (T)0.999, (T)0.001);
    cudaEventRecord(e1);
    cudaEventSynchronize(e1);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    cudaFree(out);
    return 2.0 * 8 * (double)iters * blocks * threads / (ms * 1e-3) / 1e12;
}

int main() {
    const double f64 = run<double>(20000);
    const double f32 = run<float>(200000);
    int sms = 0, clk = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, 0);
    cudaDeviceGetAttribute(&clk, cudaDevAttrClockRate, 0);
    printf("{\"fp64_fma_tflops\": %.4f, \"fp32_fma_tflops\": %.3f, \"sms\": %d, \"max_clock_khz\": %d, \"status\": \"%s\"}\n",
           f64, f32, sms, clk, cudaGetErrorString(cudaGetLastError()));
    return 0;
}
