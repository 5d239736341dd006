"""Random-coefficient models (oracle side).

The coefficient follows Eq. (1.2) with the periodic choice Theta_j(y) = sin(2 pi y_j)
(Sec. 1 and Sec. 4.2; periodic in y, so u is periodic in y, Sec. 3.2):

  affine-periodic:     a(x,y) = 1 + sum_j c j^-mu psi_j(x) sin(2 pi y_j)
  lognormal-periodic:  a(x,y) = exp( sum_j c j^-mu psi_j(x) sin(2 pi y_j) )

with spatial modes psi_j(x) = sin(j pi x) in 1-D and, in 2-D,
psi_j(x) = sin(j1 pi x1) sin(j2 pi x2), (j1, j2) = (m1(j-1)+1, m2(j-1)+1), using the
diagonal enumeration m1, m2, k of Sec. 4.3 (Table 4.2), so the modes run through
(1,1), (1,2), (2,1), (1,3), (2,2), (3,1), ... ordered by j1+j2.

Pins (tests/test_oracle_model.py): Table 4.2 itself (tests/golden/table_4_2.txt),
the affine example's a_min = 1 - c zeta(2) = 0.1 for c = 0.9/zeta(2) (Sec. 4.3), and
the periodic example's a_min/a_max = 1 -/+ (c/sqrt 6) zeta(mu) (Sec. 4.2) reproduced
from the closed-form bound.
"""
import math

import numpy as np

COEF_AFFINE_SIN = 1
COEF_LOGNORMAL_SIN = 2


def diag_k(j: int) -> int:
    """k(j) = floor(-1/2 + sqrt(1/4 + 2j)) of Sec. 4.3, computed in integers:
    the largest k >= 0 with k(k+1)/2 <= j."""
    k = 0
    while (k + 1) * (k + 2) // 2 <= j:
        k += 1
    return k


def diag_m(j: int):
    """(m1(j), m2(j)) of Sec. 4.3: m1 = j - k(k+1)/2, m2 = k - m1."""
    k = diag_k(j)
    m1 = j - k * (k + 1) // 2
    return m1, k - m1


def mode_2d(j: int):
    """Spatial mode indices (j1, j2) of the 2-D mode number j >= 1."""
    m1, m2 = diag_m(j - 1)
    return m1 + 1, m2 + 1


def psi(j: int, x: np.ndarray, dim: int) -> np.ndarray:
    """psi_j at points x (shape [..., dim]) without the c j^-mu factor."""
    if dim == 1:
        return np.sin(j * math.pi * x[..., 0])
    j1, j2 = mode_2d(j)
    return np.sin(j1 * math.pi * x[..., 0]) * np.sin(j2 * math.pi * x[..., 1])


def coefficient(model: int, scale: float, decay: float, x: np.ndarray, dim: int,
                theta: np.ndarray) -> np.ndarray:
    """a(x, y) at points x (shape [P, dim]) for one parameter y, given Theta_j(y), j=1..d
    (sin(2 pi y_j) in the periodic model; the parameter itself, y_j = phi_j(y~_j), in the
    affine and lognormal models after the periodization of Sec. 3.2)."""
    d = len(theta)
    s = np.zeros(x.shape[0])
    for j in range(1, d + 1):
        s = s + (scale * j ** (-decay) * theta[j - 1]) * psi(j, x, dim)
    if model == COEF_AFFINE_SIN:
        return 1.0 + s
    if model == COEF_LOGNORMAL_SIN:
        return np.exp(s)
    raise ValueError(f"unknown coefficient model {model}")


def ellipticity_bounds(model: int, scale: float, decay: float, d=None):
    """(a_min, a_max) of Eq. (2.1) from |psi_j| <= 1 and |sin| <= 1.

    Affine: 1 -/+ scale * sum_{j<=d} j^-decay (zeta(decay) when d is None, as in the
    bounds printed in Sec. 4.2 and Sec. 4.3).  Lognormal: exp(-/+ the same sum).
    """
    if d is None:
        from scipy.special import zeta
        tot = float(zeta(decay))
    else:
        tot = sum(j ** (-decay) for j in range(1, d + 1))
    if model == COEF_AFFINE_SIN:
        return 1.0 - scale * tot, 1.0 + scale * tot
    if model == COEF_LOGNORMAL_SIN:
        return math.exp(-scale * tot), math.exp(scale * tot)
    raise ValueError(f"unknown coefficient model {model}")
