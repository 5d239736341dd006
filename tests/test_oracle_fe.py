"""Pins of the oracle's P1 finite-element sampler (CPU only)."""
import math

import numpy as np
import pytest
import scipy.fft
import scipy.integrate
import scipy.sparse
import scipy.sparse.linalg

import workloads as W
from oracle import fe, model


def _prob1d(n, d=4, scale=0.5471, f=1.0):
    return W.Problem(kind=W.PDE_1D, n=n, d=d, coef_scale=scale, f_const=f)


def test_1d_constant_coefficient_is_nodally_exact():
    # a == 1: u(x) = x(1-x)/2, and P1 is exact at the nodes
    p = _prob1d(31, scale=0.0)
    mesh = fe.make_mesh(1, 31)
    u = fe.solve(p, mesh, np.zeros(4))
    x = mesh.nodes
    assert np.max(np.abs(u - x * (1 - x) / 2)) < 1e-15


def _piecewise_closed_form(a_e, h, f):
    # -(a u')' = f with a = a_e on element e: a u' = f (C - x), u(0) = u(1) = 0
    n1 = len(a_e)
    xe = np.arange(n1 + 1) * h
    inv = h / a_e
    xs = (xe[1:] ** 2 - xe[:-1] ** 2) / 2 / a_e
    C = xs.sum() / inv.sum()
    incr = f * (C * inv - xs)
    return np.cumsum(incr)[:-1]          # values at the interior nodes 1..n


@pytest.mark.parametrize("n", [7, 31, 255])
def test_1d_matches_piecewise_constant_closed_form(n):
    p = _prob1d(n)
    mesh = fe.make_mesh(1, n)
    r = np.random.default_rng(n)
    for _ in range(5):
        sin_y = np.sin(2 * np.pi * r.random(4))
        a_e = fe.element_coefficients(p, mesh, sin_y)
        u = fe.solve(p, mesh, sin_y)
        want = _piecewise_closed_form(a_e, mesh.h, 1.0)
        assert np.max(np.abs(u - want)) < 1e-14 * max(1.0, np.max(np.abs(want))) * n


def test_1d_second_order_convergence_to_continuous_solution():
    sin_y = np.sin(2 * np.pi * np.array([0.1, 0.7, 0.35, 0.9]))

    def a(x):
        return model.coefficient(model.COEF_AFFINE_SIN, 0.5471, 2.0, np.array([[x]]), 1, sin_y)[0]

    q = lambda fn, lo, hi: scipy.integrate.quad(fn, lo, hi, epsabs=1e-14, epsrel=1e-14, limit=200)[0]
    C = q(lambda x: x / a(x), 0, 1) / q(lambda x: 1 / a(x), 0, 1)
    errs = []
    for n in (15, 31, 63, 127):
        mesh = fe.make_mesh(1, n)
        u = fe.solve(_prob1d(n), mesh, sin_y)
        exact = np.array([q(lambda x: (C - x) / a(x), 0, xi) for xi in mesh.nodes])
        errs.append(np.max(np.abs(u - exact)))
    ratios = [errs[i] / errs[i + 1] for i in range(3)]
    assert all(3.5 < r < 4.6 for r in ratios), ratios


def _dst_poisson(n, a0, f):
    # 5-point problem a0 (4u - sum of neighbours) = h^2 f solved by its DST-I eigenbasis
    h = 1.0 / (n + 1)
    b = np.full((n, n), h * h * f)
    k = np.arange(1, n + 1)
    lam1 = 2 - 2 * np.cos(k * np.pi * h)
    lam = a0 * (lam1[:, None] + lam1[None, :])
    bh = scipy.fft.dstn(b, type=1)
    return scipy.fft.idstn(bh / lam, type=1)


@pytest.mark.parametrize("n", [5, 15, 31])
def test_2d_constant_coefficient_matches_dst_eigen_expansion(n):
    p = W.Problem(kind=W.PDE_2D, n=n, d=3, coef_model=W.COEF_LOGNORMAL_SIN, coef_scale=0.0, f_const=2.0)
    mesh = fe.make_mesh(2, n)
    u = fe.solve(p, mesh, np.zeros(3)).reshape(n, n)      # [q][p]: x2 major
    want = _dst_poisson(n, 1.0, 2.0)
    assert np.max(np.abs(u - want)) < 1e-14 * 10 * n


def test_2d_symmetric_coefficient_gives_symmetric_solution():
    # mode 1 is sin(pi x1) sin(pi x2), symmetric under x1 <-> x2; the "/" mesh maps to itself
    n = 15
    p = W.Problem(kind=W.PDE_2D, n=n, d=1)
    mesh = fe.make_mesh(2, n)
    u = fe.solve(p, mesh, np.array([math.sin(2 * math.pi * 0.8)])).reshape(n, n)
    assert np.max(np.abs(u - u.T)) < 1e-15 * 100


def test_2d_matches_edge_weight_five_point_operator():
    # right isosceles triangles: the hypotenuse coupling of P1 vanishes, so the operator is
    # the 5-point stencil whose edge weight is the mean of the two triangles' coefficients
    n = 9
    h = 1.0 / (n + 1)
    p = W.Problem(kind=W.PDE_2D, n=n, d=6)
    mesh = fe.make_mesh(2, n)
    sin_y = np.sin(2 * np.pi * np.random.default_rng(5).random(6))
    aT = fe.element_coefficients(p, mesh, sin_y)
    nsq = (n + 1) * (n + 1)
    lower = aT[:nsq].reshape(n + 1, n + 1)     # [q][p] of square (p, q)
    upper = aT[nsq:].reshape(n + 1, n + 1)
    G = n * n
    A = scipy.sparse.lil_matrix((G, G))
    idx = lambda pp, qq: (qq - 1) * n + (pp - 1)
    for q in range(0, n + 2):
        for pp in range(0, n + 2):
            # horizontal edge (pp,q)-(pp+1,q): lower tri of square (pp,q), upper tri of (pp,q-1)
            if pp <= n and 1 <= q <= n:
                w = 0.5 * (lower[q, pp] + upper[q - 1, pp])
                for a_, b_ in (((pp, q), (pp + 1, q)),):
                    for (x1, y1), (x2, y2) in ((a_, b_), (b_, a_)):
                        if 1 <= x1 <= n:
                            A[idx(x1, y1), idx(x1, y1)] += w
                            if 1 <= x2 <= n:
                                A[idx(x1, y1), idx(x2, y2)] -= w
            # vertical edge (pp,q)-(pp,q+1): upper tri of square (pp,q), lower tri of (pp-1,q)
            if q <= n and 1 <= pp <= n:
                w = 0.5 * (upper[q, pp] + lower[q, pp - 1])
                for a_, b_ in (((pp, q), (pp, q + 1)),):
                    for (x1, y1), (x2, y2) in ((a_, b_), (b_, a_)):
                        if 1 <= y1 <= n:
                            A[idx(x1, y1), idx(x1, y1)] += w
                            if 1 <= y2 <= n:
                                A[idx(x1, y1), idx(x2, y2)] -= w
    u5 = scipy.sparse.linalg.spsolve(A.tocsc(), np.full(G, h * h))
    u = fe.solve(p, mesh, sin_y)
    assert np.max(np.abs(u - u5)) < 1e-14
