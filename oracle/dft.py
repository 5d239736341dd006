"""Projected Fourier coefficients by a naive DFT (oracle side).

Algorithm 1 (steps 1/2a) computes, for every mesh node g,
  c~_{g,k} = (1/M) sum_{i=0}^{M-1} u(x_g, y_i) exp(-2 pi i (i m_k)/M),
with M = K_t and m_k = k mod K_t for the 1-D detections, and with the rank-1 lattice
index m_k = k.z mod M in step 2d (single rank-1 lattice, Appendix A).  The oracle
evaluates this sum directly at the needed indices only: the phase index
(i m_k) mod M is reduced exactly in int64 before conversion to an angle, and each
sum is an fp64 matrix-vector product.  Cost O(M |J| G).

Pins (tests/test_oracle_dft.py): single tones give a unit delta; with m_k covering
all residues the result equals numpy.fft.fft / M; Parseval's identity.
"""
import numpy as np


def coefficients(U: np.ndarray, m: np.ndarray, M: int, chunk: int = 256) -> np.ndarray:
    """c~ [G, |m|] complex128 from samples U [M, G] (row i = lattice node i)."""
    U = np.asarray(U, dtype=np.float64)
    assert U.shape[0] == M
    G = U.shape[1]
    out = np.zeros((G, len(m)), dtype=np.complex128)
    i = np.arange(M, dtype=np.int64)
    for c0 in range(0, len(m), chunk):
        mk = np.asarray(m[c0:c0 + chunk], dtype=np.int64)
        phase_idx = np.mod(np.outer(i, mk), M)                  # exact integers
        ang = (2.0 * np.pi / M) * phase_idx.astype(np.float64)
        re = U.T @ np.cos(ang)
        im = -(U.T @ np.sin(ang))
        out[:, c0:c0 + chunk] = (re + 1j * im) / M
    return out


def partial_coefficients(U_rows: np.ndarray, rows: np.ndarray, m: np.ndarray, M: int,
                         chunk: int = 256) -> np.ndarray:
    """The contribution of the lattice nodes `rows` (samples U_rows [len(rows), G]) to
    coefficients(): (1/M) sum_{i in rows} U[i][g] exp(-2 pi i (i m_k)/M).  Summed over a
    partition of 0..M-1 it gives coefficients(); the cost per row is the same."""
    U_rows = np.asarray(U_rows, dtype=np.float64)
    G = U_rows.shape[1]
    out = np.zeros((G, len(m)), dtype=np.complex128)
    i = np.asarray(rows, dtype=np.int64)
    for c0 in range(0, len(m), chunk):
        mk = np.asarray(m[c0:c0 + chunk], dtype=np.int64)
        ang = (2.0 * np.pi / M) * np.mod(np.outer(i, mk), M).astype(np.float64)
        out[:, c0:c0 + chunk] = (U_rows.T @ np.cos(ang) - 1j * (U_rows.T @ np.sin(ang))) / M
    return out
