"""Evaluation of the sparse approximation and its errors (oracle side; test infrastructure).

- sample_points: the black box at explicit parameter points of the model's domain,
  u-check(x_g, y^(j)) -- the FE solution of Eq. (1.1) for the fixed parameter y^(j)
  (Section 4), or the test polynomial.
- evaluate: u~^usFFT(x_g, y~) = sum_{k in I} c_{g,k} e^{2 pi i k.y~} at torus points;
  evaluate_parameters: u^usFFT(x_g, y) = the same at y~ = phi^-1(y) (Eq. (3.1); phi is the
  identity for the periodic model).
- errors: err_2 and err_inf of Section 4 per mesh node, over the test points, with |.| the
  complex modulus.

Only tests, smoke checks and the CPU timing leg of the benchmark use this package.
Pins (tests/test_oracle_evaluate.py): a trigonometric polynomial with its own coefficients
is reproduced at random points; Parseval on the nodes of a reconstructing lattice; single
terms against cos/sin; err_2 <= err_inf with equality for a constant difference; the FE
samples at a lattice node equal the lattice sampler's.
"""
import numpy as np

from . import fe, periodization

PDE_1D, PDE_2D, TRIGPOLY = 1, 2, 3


def sample_points(prob, Y: np.ndarray, mesh=None) -> np.ndarray:
    """U [n, G]: the black box at the rows of Y."""
    Y = np.asarray(Y, dtype=np.float64).reshape(-1, prob.d)
    if prob.kind == TRIGPOLY:
        F = prob.tp_freqs.astype(np.int64)            # [G, T, d]
        U = np.zeros((len(Y), F.shape[0]))
        for g in range(F.shape[0]):
            for tt in range(F.shape[1]):
                c = prob.tp_coefs[g, tt]
                if c != 0:
                    U[:, g] += (c * np.exp(2j * np.pi * np.mod(Y @ F[g, tt], 1.0))).real
        return U
    if mesh is None:
        mesh = fe.make_mesh(prob.kind, prob.n)
    U = np.zeros((len(Y), mesh.G))
    for j, y in enumerate(Y):
        U[j] = fe.solve(prob, mesh, periodization.theta_of_parameter(prob, y))
    return U


def evaluate(I: np.ndarray, C: np.ndarray, Y: np.ndarray) -> np.ndarray:
    """V [n, G] = sum_k C[g, k] exp(2 pi i k.y_j) (I [|I|, d] integers, C [G, |I|])."""
    I = np.asarray(I, dtype=np.int64)
    Y = np.asarray(Y, dtype=np.float64).reshape(-1, I.shape[1] if I.size else 1)
    if I.shape[0] == 0:
        return np.zeros((len(Y), C.shape[0]), dtype=np.complex128)
    E = np.exp(2j * np.pi * np.mod(Y @ I.T.astype(np.float64), 1.0))     # [n, |I|]
    return E @ C.T


def evaluate_parameters(prob, I: np.ndarray, C: np.ndarray, Y: np.ndarray) -> np.ndarray:
    """u^usFFT at parameters Y of the model's own domain: evaluate() at phi^-1(Y) (Eq. (3.1))."""
    return evaluate(I, C, periodization.to_torus(prob, Y))


def errors(U: np.ndarray, V: np.ndarray):
    """(err_2 [G], err_inf [G]) over the rows (test points) of U (real) and V (complex)."""
    a = np.abs(U - V)
    return np.sqrt(np.mean(a * a, axis=0)), np.max(a, axis=0)
