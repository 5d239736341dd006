// Kernels of the sharded form of a coupled step (one instance over P ranks).
//
// The lattice is split by residue: rank p owns the nodes i = p + P i2, i2 < L = M / P (P | M).
// The DFT of Algorithm 1, step 2d then splits into P partial sums,
//   c_{g,k} = (1/M) sum_i u_g(y_i) e^{-2 pi i i m_k / M}
//           = sum_p (1/P) e^{-2 pi i p m_k / M} [ (1/L) sum_{i2} u_g(y_{p + P i2}) e^{-2 pi i i2 (m_k mod L) / L} ],
// and the bracket is the rank's own length-L lattice FFT read at m_k mod L.  shard_twist applies
// the factor in front; a sum over the ranks (an all-reduce) then gives every rank the full
// coefficients.  The phase index (p m_k) mod M is reduced exactly in integers.
#include <cuda_runtime.h>
#include <stdint.h>

#include "usfft_internal.h"

namespace usfft {

__global__ void shard_twist_kernel(double2* C, int G, int64_t nJ, const int* mk, int64_t p, int64_t M, double scale) {
    const int64_t total = (int64_t)G * nJ;
    for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
         idx += (int64_t)gridDim.x * blockDim.x) {
        const int64_t k = idx % nJ;
        const int64_t a = (p * (int64_t)mk[k]) % M;
        double sv, cv;
        sincospi(2.0 * (double)a / (double)M, &sv, &cv);
        const double2 c = C[idx];
        // c (cos - i sin) * scale
        C[idx] = make_double2(scale * (c.x * cv + c.y * sv), scale * (c.y * cv - c.x * sv));
    }
}

__global__ void bits_to_bytes_kernel(const uint32_t* bits, int64_t n, uint8_t* bytes) {
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x)
        bytes[k] = (uint8_t)((bits[k >> 5] >> (k & 31)) & 1u);
}

// one thread per 32-bit word
__global__ void bytes_to_bits_kernel(const uint8_t* bytes, int64_t n, uint32_t* bits) {
    const int64_t words = (n + 31) / 32;
    for (int64_t w = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; w < words; w += (int64_t)gridDim.x * blockDim.x) {
        uint32_t v = 0;
        for (int b = 0; b < 32; ++b) {
            const int64_t k = w * 32 + b;
            if (k < n && bytes[k]) v |= 1u << b;
        }
        bits[w] = v;
    }
}

static unsigned grid_for(int64_t n, int threads) {
    int64_t b = (n + threads - 1) / threads;
    if (b > 152 * 32) b = 152 * 32;
    return (unsigned)(b < 1 ? 1 : b);
}

cudaError_t launch_shard_twist(double2* C, int G, int64_t nJ, const int* mk, int64_t p, int64_t M, double scale,
                               cudaStream_t s, int* launches) {
    if ((int64_t)G * nJ == 0) return cudaSuccess;
    shard_twist_kernel<<<grid_for((int64_t)G * nJ, 256), 256, 0, s>>>(C, G, nJ, mk, p, M, scale);
    if (launches) ++*launches;
    return cudaGetLastError();
}

cudaError_t launch_bits_to_bytes(const uint32_t* bits, int64_t n, uint8_t* bytes, cudaStream_t s, int* launches) {
    if (n == 0) return cudaSuccess;
    bits_to_bytes_kernel<<<grid_for(n, 256), 256, 0, s>>>(bits, n, bytes);
    if (launches) ++*launches;
    return cudaGetLastError();
}

cudaError_t launch_bytes_to_bits(const uint8_t* bytes, int64_t n, uint32_t* bits, cudaStream_t s, int* launches) {
    if (n == 0) return cudaSuccess;
    bytes_to_bits_kernel<<<grid_for((n + 31) / 32, 128), 128, 0, s>>>(bytes, n, bits);
    if (launches) ++*launches;
    return cudaGetLastError();
}

}  // namespace usfft
