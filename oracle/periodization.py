"""Parameter maps and periodizations (Section 3.2) and the quantities of interest of
Sections 4 and 4.1 (oracle side; test infrastructure).

The usFFT needs a function that is 1-periodic in every parameter.  Three models:

- periodic (MAP_PERIODIC): Theta_j = sin(2 pi y_j), y on the torus; nothing to periodize.
- affine (MAP_TENT): Theta_j = y_j with y_j uniform on [alpha, beta]; the usFFT works on
  u~(x, y~) = u(x, phi(y~)) with the tent transformation (Eq. (3.2))
      phi_j(y~) = beta - |(beta - alpha)(1 - 2 y~)|,  phi_j^-1(y) = (y - alpha) / (2 (beta - alpha)).
- lognormal (MAP_NORMAL): Theta_j = y_j with y_j standard normal; phi_{j,Delta} =
  tau_1 o tau_{2,Delta} (Eq. (3.3)) with
      tau_1(v) = sqrt(2) erfinv(2 v),                        tau_1^-1(y) = erf(y / sqrt 2) / 2,
      tau_{2,Delta}(y~) = -1/2 - 2 (y~ - Delta)   for 0 <= y~ < Delta,
                          -1/2 + 2 (y~ - Delta)   for Delta <= y~ < 1/2 + Delta,
                          +3/2 - 2 (y~ - Delta)   for 1/2 + Delta <= y~ < 1,
      tau_{2,Delta}^-1(v) = v / 2 + Delta + 1/4.

The approximation in the original parameters is u^usFFT(y) = sum_k c_k e^{2 pi i k.phi^-1(y)}
(Eq. (3.1)), and its expectation (Section 4.1; Eq. (4.5) for the tent map) is sum_k c_k D_k
with D_k = prod_j D_{k_j}:
      periodic:   D_{k_j} = 1 if k_j = 0, else 0            (the mean is c_0)
      tent:       D_{k_j} = 2i / (pi k_j) for odd k_j, 1 for k_j = 0, 0 otherwise
      lognormal:  D_{k_j,Delta} = the tent factor times e^{2 pi i k_j Delta}.
The variance of the approximation is sum_{k != 0} |c_k|^2 and the global sensitivity index
of a subset J of I is sum_{k in J, k != 0} |c_k|^2 / variance (Eq. (4.3)); J_l collects the
k with exactly l non-zero components (Eq. (4.4)).

Pins (tests/test_oracle_periodization.py): points of the three curves of Figure 3.1
(tests/golden/fig_3_1_periodization.txt, Delta = 0.1); (A1)-(A4) of the tent map and the
round trip phi(phi^-1(y)) = y; tau_1^-1(y) + 1/2 equals the normal distribution function
(scipy.stats.norm.cdf, a different library routine); every D factor against adaptive
quadrature of its defining integral; Sum_l GSI(J_l) = 1 and the variance against Parseval
on a reconstructing lattice.
"""
import math

import numpy as np
from scipy.special import erf, erfinv

MAP_PERIODIC = 0
MAP_TENT = 1
MAP_NORMAL = 2


def tent(yt, alpha, beta):
    return beta - np.abs((beta - alpha) * (1.0 - 2.0 * np.asarray(yt, dtype=np.float64)))


def tent_inv(y, alpha, beta):
    return (np.asarray(y, dtype=np.float64) - alpha) / (2.0 * (beta - alpha))


def tau1(v):
    return math.sqrt(2.0) * erfinv(2.0 * np.asarray(v, dtype=np.float64))


def tau1_inv(y):
    return 0.5 * erf(np.asarray(y, dtype=np.float64) / math.sqrt(2.0))


def tau2(yt, shift):
    yt = np.asarray(yt, dtype=np.float64)
    u = yt - shift
    return np.where(yt < shift, -0.5 - 2.0 * u, np.where(yt < 0.5 + shift, -0.5 + 2.0 * u, 1.5 - 2.0 * u))


def tau2_inv(v, shift):
    return np.asarray(v, dtype=np.float64) / 2.0 + shift + 0.25


def phi_normal(yt, shift):
    return tau1(tau2(yt, shift))


def phi_normal_inv(y, shift):
    return tau2_inv(tau1_inv(y), shift)


def theta_of_node(prob, yt):
    """Theta_j at the torus point y~ (the sampling nodes of the usFFT)."""
    m = getattr(prob, "theta_map", MAP_PERIODIC)
    if m == MAP_PERIODIC:
        return np.sin(2.0 * np.pi * np.asarray(yt, dtype=np.float64))
    if m == MAP_TENT:
        return tent(yt, prob.map_alpha, prob.map_beta)
    if m == MAP_NORMAL:
        return phi_normal(yt, prob.map_shift)
    raise ValueError(f"unknown parameter map {m}")


def theta_of_parameter(prob, y):
    """Theta_j at a point y of the model's own parameter domain D_y (test points)."""
    m = getattr(prob, "theta_map", MAP_PERIODIC)
    y = np.asarray(y, dtype=np.float64)
    return np.sin(2.0 * np.pi * y) if m == MAP_PERIODIC else y


def to_torus(prob, y):
    """phi^-1(y): the torus point of a parameter y (identity for the periodic model)."""
    m = getattr(prob, "theta_map", MAP_PERIODIC)
    if m == MAP_PERIODIC:
        return np.asarray(y, dtype=np.float64)
    if m == MAP_TENT:
        return tent_inv(y, prob.map_alpha, prob.map_beta)
    return phi_normal_inv(y, prob.map_shift)


def d_factor(k: int, theta_map: int, shift: float = 0.0) -> complex:
    """D_{k_j} (periodic, tent) or D_{k_j,Delta} (lognormal) for one component."""
    if k == 0:
        return 1.0 + 0.0j
    if theta_map == MAP_PERIODIC or k % 2 == 0:
        return 0.0j
    f = 2j / (math.pi * k)
    if theta_map == MAP_NORMAL:
        f *= complex(math.cos(2 * math.pi * k * shift), math.sin(2 * math.pi * k * shift))
    return f


def expectation(I: np.ndarray, C: np.ndarray, theta_map: int, shift: float = 0.0) -> np.ndarray:
    """E(u^usFFT) per node: sum_k C[g, k] D_k, complex [G]."""
    D = np.array([np.prod([d_factor(int(v), theta_map, shift) for v in k]) for k in np.asarray(I)],
                 dtype=np.complex128)
    return C @ D if len(D) else np.zeros(C.shape[0], dtype=np.complex128)


def variance(I: np.ndarray, C: np.ndarray) -> np.ndarray:
    """sigma^2 per node: sum over k != 0 of |C[g, k]|^2."""
    nz = np.any(np.asarray(I) != 0, axis=1)
    return np.sum(np.abs(C[:, nz]) ** 2, axis=1)


def gsi(I: np.ndarray, C: np.ndarray, d: int) -> np.ndarray:
    """rho(J_l) for l = 1..d per node: [G, d] (0 where the variance is 0)."""
    I = np.asarray(I)
    order = np.count_nonzero(I, axis=1)
    var = variance(I, C)
    out = np.zeros((C.shape[0], d))
    for l in range(1, d + 1):
        sel = order == l
        part = np.sum(np.abs(C[:, sel]) ** 2, axis=1)
        out[:, l - 1] = np.divide(part, var, out=np.zeros_like(part), where=var > 0)
    return out
