// Theta_j of a sampling node and the inverse parameter map on the device (Sec. 3.2).
//
// Sampling nodes live on the torus.  The periodic model takes Theta_j = sin(2 pi y~_j); the
// affine and lognormal models take Theta_j = phi_j(y~_j), the tent transformation (Eq. (3.2))
// or tau_1 o tau_{2,Delta} (Eq. (3.3)).  Explicit points are parameters of the model's own
// domain: Theta_j = sin(2 pi y_j) (periodic) or y_j itself.
#pragma once
#include <cuda_runtime.h>
#include <math.h>

#include "usfft_internal.h"

namespace usfft {

// phi_j(y~) of the non-periodic maps
__device__ __forceinline__ double theta_of_torus(int map, double a, double b, double shift, double yt) {
    if (map == USFFT_MAP_TENT) return b - fabs((b - a) * (1.0 - 2.0 * yt));
    const double u = yt - shift;
    const double v = yt < shift ? -0.5 - 2.0 * u : (yt < 0.5 + shift ? -0.5 + 2.0 * u : 1.5 - 2.0 * u);
    return M_SQRT2 * erfinv(2.0 * v);
}

// the lattice node index of the k-th node of a node set
__host__ __device__ __forceinline__ int64_t lattice_node(const NodeSpec& ns, int64_t k) {
    return ns.stride > 1 ? ns.first + ns.stride * k : ns.first + k;
}

// Theta_j of node i of a node set: explicit point, lattice coordinate (exact integer
// reduction n = i z_j mod M, Eq. (3.4)) or fixed tail
__device__ __forceinline__ double node_theta(const NodeSpec& ns, int j, int64_t i) {
    if (ns.Y) {
        const double y = ns.Y[i * ns.d + j];
        return ns.map == USFFT_MAP_PERIODIC ? sinpi(2.0 * y) : y;
    }
    const int64_t zj = ns.z[j];
    if (zj >= 0) {
        const int64_t nn = (i * zj) % ns.M;
        if (ns.map == USFFT_MAP_PERIODIC) return sinpi(2.0 * (double)nn / (double)ns.M);
        return theta_of_torus(ns.map, ns.map_alpha, ns.map_beta, ns.map_shift, (double)nn / (double)ns.M);
    }
    if (ns.map == USFFT_MAP_PERIODIC) return sinpi(2.0 * ns.tail[j]);
    return theta_of_torus(ns.map, ns.map_alpha, ns.map_beta, ns.map_shift, ns.tail[j]);
}

// phi^-1(y): the torus point of a parameter (identity for the periodic model)
__device__ __forceinline__ double to_torus(const ParamMap& pm, double y) {
    if (pm.map == USFFT_MAP_TENT) return (y - pm.alpha) / (2.0 * (pm.beta - pm.alpha));
    if (pm.map == USFFT_MAP_NORMAL) return 0.5 * erf(y / M_SQRT2) / 2.0 + pm.shift + 0.25;
    return y;
}

}  // namespace usfft
