"""Black-box sampler: P1 finite elements for Eq. (1.1) (oracle side).

The paper treats the PDE solver as a black box that returns u(x_g, y) at every mesh
node x_g for one parameter y (Sec. 2.1, "black box sampling"; Remark 1.2).  The
oracle uses the textbook P1 Galerkin discretisation of the weak form of Sec. 2.1:

  find u_h in V_h:  sum_T a_T int_T grad u_h . grad v = int f v   for all v in V_h,

with a_T = a(centroid of T, y) (one-point quadrature of the coefficient) and a
constant right-hand side f (the load int_T f phi_i = f |T| / (dim+1) is exact).

- 1-D: (0,1) with n interior nodes x_i = i h, h = 1/(n+1); elements [x_e, x_{e+1}].
- 2-D: the unit square with n*n interior nodes x_(p,q) = (p h, q h); every square
  [p,p+1]x[q,q+1] (in units of h) is split along its "/" diagonal into the triangles
  {(p,q),(p+1,q),(p+1,q+1)} and {(p,q),(p+1,q+1),(p,q+1)}.  Interior node (p,q) has
  mesh index g = (q-1) n + (p-1).

The element matrices come from the barycentric gradients of each element (no
stencil shortcut), are summed into a symmetric band matrix, and the system is
solved by banded Cholesky (LAPACK ?pbsv through scipy.linalg.solveh_banded).

Pins (tests/test_oracle_fe.py): 1-D nodal exactness against the closed-form
solution of the piecewise-constant-coefficient problem; O(h^2) convergence to the
continuous 1-D solution (adaptive quadrature of 1/a); the 2-D constant-coefficient
case against the DST-I eigen-expansion of the discrete problem; symmetry
u(x1,x2) = u(x2,x1) for a symmetric coefficient.
"""
import numpy as np
from scipy.linalg import solveh_banded

from . import model


class Mesh1D:
    def __init__(self, n: int):
        self.n = n
        self.G = n
        self.h = 1.0 / (n + 1)
        self.nodes = np.arange(1, n + 1) * self.h            # interior nodes
        self.centroids = ((np.arange(n + 1) + 0.5) * self.h)[:, None]   # element midpoints
        # element e couples global nodes e and e+1 (0 and n+1 are boundary)
        self.elem_nodes = np.stack([np.arange(n + 1), np.arange(1, n + 2)], axis=1)
        self.area = np.full(n + 1, self.h)
        # gradients of the two hat functions on each element: -1/h, +1/h
        self.grads = np.zeros((n + 1, 2, 1))
        self.grads[:, 0, 0] = -1.0 / self.h
        self.grads[:, 1, 0] = 1.0 / self.h
        self.interior_index = np.full(n + 2, -1)
        self.interior_index[1:n + 1] = np.arange(n)
        self.bandwidth = 1
        self.dim = 1


class Mesh2D:
    def __init__(self, n: int):
        self.n = n
        self.G = n * n
        h = 1.0 / (n + 1)
        self.h = h
        P, Q = np.meshgrid(np.arange(n + 1), np.arange(n + 1), indexing="xy")  # squares
        P = P.ravel()
        Q = Q.ravel()

        def nid(p, q):
            return q * (n + 2) + p      # global node id over the (n+2)^2 grid

        lower = np.stack([nid(P, Q), nid(P + 1, Q), nid(P + 1, Q + 1)], axis=1)
        upper = np.stack([nid(P, Q), nid(P + 1, Q + 1), nid(P, Q + 1)], axis=1)
        self.elem_nodes = np.concatenate([lower, upper], axis=0)
        gx = np.arange(n + 2) * h
        X, Y = np.meshgrid(gx, gx, indexing="xy")
        coords = np.stack([X.ravel(), Y.ravel()], axis=1)
        v = coords[self.elem_nodes]                       # [E, 3, 2]
        self.centroids = v.mean(axis=1)
        e1 = v[:, 1] - v[:, 0]
        e2 = v[:, 2] - v[:, 0]
        det = e1[:, 0] * e2[:, 1] - e1[:, 1] * e2[:, 0]
        self.area = 0.5 * np.abs(det)
        # barycentric gradients: grad phi_1 and grad phi_2 are the rows of B^{-1}
        # with B = [e1 e2] (columns), grad phi_0 = -(grad phi_1 + grad phi_2)
        B = np.stack([e1, e2], axis=2)                    # [E, 2, 2]
        Binv = np.linalg.inv(B)
        g1 = Binv[:, 0, :]
        g2 = Binv[:, 1, :]
        self.grads = np.stack([-(g1 + g2), g1, g2], axis=1)   # [E, 3, 2]
        interior = np.full((n + 2) * (n + 2), -1)
        for q in range(1, n + 1):
            for p in range(1, n + 1):
                interior[nid(p, q)] = (q - 1) * n + (p - 1)
        self.interior_index = interior
        self.bandwidth = n + 1
        self.dim = 2


def make_mesh(kind: int, n: int):
    return Mesh1D(n) if kind == 1 else Mesh2D(n)


def assemble_band(mesh, a_elem: np.ndarray, f_const: float):
    """Band storage (upper form of solveh_banded) of the stiffness matrix and the load vector."""
    u = mesh.bandwidth
    G = mesh.G
    ab = np.zeros((u + 1, G))
    b = np.zeros(G)
    nloc = mesh.elem_nodes.shape[1]
    loc = np.einsum("eid,ejd->eij", mesh.grads, mesh.grads) * (a_elem * mesh.area)[:, None, None]
    gi = mesh.interior_index[mesh.elem_nodes]             # [E, nloc]
    for i in range(nloc):
        rows = gi[:, i]
        np.add.at(b, rows[rows >= 0], (f_const * mesh.area / nloc)[rows >= 0])
        for j in range(nloc):
            cols = gi[:, j]
            keep = (rows >= 0) & (cols >= 0) & (rows <= cols)
            r = rows[keep]
            c = cols[keep]
            np.add.at(ab, (u + r - c, c), loc[keep, i, j])
    return ab, b


def element_coefficients(prob, mesh, theta: np.ndarray) -> np.ndarray:
    return model.coefficient(prob.coef_model, prob.coef_scale, prob.coef_decay,
                             mesh.centroids, mesh.dim, theta)


def solve(prob, mesh, theta: np.ndarray) -> np.ndarray:
    """u(x_g, y) at all interior nodes for one y, given Theta_j(y), j=1..d."""
    a = element_coefficients(prob, mesh, theta)
    ab, b = assemble_band(mesh, a, prob.f_const)
    return solveh_banded(ab, b, lower=False, check_finite=False)
