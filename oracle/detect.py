"""Thresholding and union of detected frequency sets (oracle side).

Algorithm 1, steps 1/2a and 2d: for each mesh node g keep the indices of the at most
s~ largest coefficients (in absolute value) whose absolute value is at least the
absolute threshold theta; step 2e joins these sets over g (and over the detection
iterations i) into I^(1..t).

Readings fixed on both sides:
- |c|^2 = re*re + im*im in fp64, each product and the sum rounded separately (no
  fused multiply-add), compared with theta*theta;
- "among the s~ largest" and ">= theta" apply jointly; equal magnitudes are ordered
  by the smaller index (position in J_t, or in P_t(Gamma) for the 1-D detections);
- a relative threshold delta means theta = delta * A with
  A = max_g |c~_{g,0}| of the first 1-D detection (t = 1, i = 1).

Pins (tests/test_oracle_detect.py): brute force over all subsets on tiny inputs,
and the invariants union >= each node's set, |union| <= sum_g min(s~, count_g).
"""
import numpy as np


def magnitude2(c: np.ndarray) -> np.ndarray:
    re = np.ascontiguousarray(c.real)
    im = np.ascontiguousarray(c.imag)
    return re * re + im * im            # numpy never contracts this into an FMA


def select(c_g: np.ndarray, theta: float, s_tilde: int) -> np.ndarray:
    """Sorted indices of the <= s~ largest |c_g[k]| with |c_g[k]| >= theta."""
    mag2 = magnitude2(c_g)
    idx = np.arange(len(c_g))
    keep = mag2 >= theta * theta
    cand = idx[keep]
    order = np.lexsort((cand, -mag2[keep]))       # magnitude descending, then index ascending
    chosen = cand[order[:s_tilde]]
    return np.sort(chosen)


def union_over_nodes(C: np.ndarray, theta: float, s_tilde: int, into: set) -> set:
    """Add every node's selection (C is [G, n]) to the set `into` and return it."""
    for g in range(C.shape[0]):
        into.update(int(k) for k in select(C[g], theta, s_tilde))
    return into
