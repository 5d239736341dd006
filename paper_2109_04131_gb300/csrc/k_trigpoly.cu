// Test black box: G real trigonometric polynomials p^(g)(y) = Re sum_s c_{g,s} e^{2 pi i h_{g,s}.y}
// sampled at the nodes of a lattice with fixed tails (the setting of Theorem 1.1), or at
// explicit points.
//
// For lattice coordinates the phase of node i is exact in integers:
// sum_j h_j (i z_j mod M) = i (h.z) mod M, so each term keeps m_s = (h_lat . z) mod M and the
// fixed tail rotation e^{2 pi i h_tail . y'}; the sample is
// Re sum_s c_s e^{2 pi i ((i m_s) mod M)/M} e^{2 pi i h_tail . y'}.
#include <cuda_runtime.h>
#include <math.h>

#include "usfft_internal.h"

namespace usfft {

__global__ void trigpoly_setup_kernel(const __grid_constant__ NodeSpec ns, int G, int nterms, const int8_t* freqs,
                                      double* aux) {
    const int64_t total = (int64_t)G * nterms;
    for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
         idx += (int64_t)gridDim.x * blockDim.x) {
        const int8_t* h = freqs + idx * ns.d;
        int64_t m = 0;
        double ph = 0.0;
        for (int j = 0; j < ns.d; ++j) {
            if (ns.z[j] >= 0) {
                int64_t term = ((int64_t)h[j] * ns.z[j]) % ns.M;
                m = (m + term) % ns.M;
            } else {
                ph += (double)h[j] * ns.tail[j];
            }
        }
        if (m < 0) m += ns.M;
        double sv, cv;
        sincospi(2.0 * ph, &sv, &cv);
        aux[3 * idx + 0] = (double)m;
        aux[3 * idx + 1] = cv;
        aux[3 * idx + 2] = sv;
    }
}

// rows k < count: lattice node i = first + stride k (stride >= 1) of the lattice of size M
__global__ void trigpoly_sample_kernel(int64_t M, int64_t count, int64_t first, int64_t stride, int G, int nterms,
                                       const double* coefs, const double* aux, double* U) {
    const int64_t total = count * G;
    for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
         idx += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = first + stride * (idx / G);
        const int g = (int)(idx % G);
        double acc = 0.0;
        for (int s = 0; s < nterms; ++s) {
            const int64_t t = (int64_t)g * nterms + s;
            const double cr = coefs[2 * t], ci = coefs[2 * t + 1];
            if (cr == 0.0 && ci == 0.0) continue;
            const int64_t m = (int64_t)aux[3 * t];
            const int64_t a = (i * m) % M;
            double sv, cv;
            sincospi(2.0 * (double)a / (double)M, &sv, &cv);
            // rotation by the tail phase
            const double rr = cv * aux[3 * t + 1] - sv * aux[3 * t + 2];
            const double ri = cv * aux[3 * t + 2] + sv * aux[3 * t + 1];
            acc += cr * rr - ci * ri;
        }
        U[idx] = acc;
    }
}

// Explicit points y_i (rows of Y): the phase h.y_i is summed term by term, each product
// h_j y_ij reduced mod 1 with its rounding error kept (fma), so the phase error stays at the
// rounding level of numbers in [-1/2, 1/2] whatever |h|.
__global__ void trigpoly_points_kernel(const double* Y, int64_t count, int d, int G, int nterms,
                                       const int8_t* freqs, const double* coefs, double* U) {
    const int64_t total = count * G;
    for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
         idx += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = idx / G;
        const int g = (int)(idx % G);
        const double* y = Y + i * d;
        double acc = 0.0;
        for (int s = 0; s < nterms; ++s) {
            const int64_t t = (int64_t)g * nterms + s;
            const double cr = coefs[2 * t], ci = coefs[2 * t + 1];
            if (cr == 0.0 && ci == 0.0) continue;
            const int8_t* h = freqs + t * d;
            double ph = 0.0;
            for (int j = 0; j < d; ++j) {
                if (!h[j]) continue;
                const double hj = (double)h[j];
                const double p = hj * y[j];
                const double e = fma(hj, y[j], -p);
                ph += (p - rint(p)) + e;
            }
            ph -= rint(ph);
            double sv, cv;
            sincospi(2.0 * ph, &sv, &cv);
            acc += cr * cv - ci * sv;
        }
        U[idx] = acc;
    }
}

cudaError_t launch_sample_trigpoly(const NodeSpec& ns, int G, int nterms, const int8_t* freqs,
                                   const double* coefs, double* aux, double* U, cudaStream_t s, int* launches) {
    if (ns.M <= 0) return cudaSuccess;
    if (ns.Y) {
        int64_t b = (ns.M * G + 255) / 256;
        if (b > 152 * 64) b = 152 * 64;
        trigpoly_points_kernel<<<(unsigned)b, 256, 0, s>>>(ns.Y, ns.M, ns.d, G, nterms, freqs, coefs, U);
        if (launches) ++*launches;
        return cudaGetLastError();
    }
    int64_t tot = (int64_t)G * nterms;
    int b1 = (int)((tot + 255) / 256);
    trigpoly_setup_kernel<<<b1 > 0 ? b1 : 1, 256, 0, s>>>(ns, G, nterms, freqs, aux);
    const int64_t count = node_count(ns);
    int64_t tot2 = count * G;
    int64_t b2 = (tot2 + 255) / 256;
    if (b2 > 152 * 64) b2 = 152 * 64;
    if (b2 < 1) b2 = 1;
    trigpoly_sample_kernel<<<(unsigned)b2, 256, 0, s>>>(ns.M, count, ns.first, ns.stride > 1 ? ns.stride : 1, G, nterms,
                                                        coefs, aux, U);
    if (launches) *launches += 2;
    return cudaGetLastError();
}

}  // namespace usfft
