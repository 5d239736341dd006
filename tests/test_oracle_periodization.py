"""Pins of the oracle's periodizations (Sec. 3.2) and quantities of interest (Sec. 4, 4.1)."""
import math
import os

import numpy as np
import pytest
from scipy import integrate, stats

from oracle import lattice
from oracle import periodization as P

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "fig_3_1_periodization.txt")


def test_figure_3_1_points():
    # the plotted curves of Figure 3.1 (Delta = 0.1) to the digits printed
    fn = {"tau1": lambda x: P.tau1(x), "tau2": lambda x: P.tau2(x, 0.1), "phi": lambda x: P.phi_normal(x, 0.1)}
    n = 0
    for line in open(GOLDEN):
        if line.startswith("#") or not line.strip():
            continue
        panel, x, y = line.split()
        v = float(fn[panel](float(x)))
        assert abs(v - float(y)) <= 1e-10 * max(1.0, abs(float(y))), (panel, x)
        n += 1
    assert n == 21


@pytest.mark.parametrize("alpha,beta", [(-1.0, 1.0), (-0.5, 0.5), (0.2, 3.0)])
def test_tent_assumptions_a1_to_a4(alpha, beta):
    t = np.linspace(0.0, 1.0, 2001)
    f = P.tent(t, alpha, beta)
    assert abs(P.tent(0.0, alpha, beta) - alpha) < 1e-15 and abs(P.tent(1.0, alpha, beta) - alpha) < 1e-15  # (A2)
    assert P.tent(0.5, alpha, beta) == beta
    assert np.max(np.abs(np.diff(f))) <= 2 * (beta - alpha) / 2000 * (1 + 1e-12)      # (A1), Lipschitz
    h = np.linspace(0.0, 0.5, 501)
    assert np.allclose(P.tent(0.5 - h, alpha, beta), P.tent(0.5 + h, alpha, beta), atol=1e-14)   # (A3)
    assert np.all(np.diff(P.tent(h, alpha, beta)) > 0)                                  # (A4)
    y = alpha + (beta - alpha) * np.random.default_rng(0).random(100)
    assert np.allclose(P.tent(P.tent_inv(y, alpha, beta), alpha, beta), y, atol=1e-14)   # round trip
    assert np.all((P.tent_inv(y, alpha, beta) >= 0) & (P.tent_inv(y, alpha, beta) <= 0.5))


def test_tau1_is_the_normal_quantile_map():
    y = np.linspace(-6, 6, 121)
    assert np.allclose(P.tau1_inv(y) + 0.5, stats.norm.cdf(y), atol=1e-15)
    v = np.linspace(-0.49, 0.49, 99)
    assert np.allclose(P.tau1(v), stats.norm.ppf(v + 0.5), rtol=1e-12, atol=1e-14)


def test_lognormal_map_round_trip_and_range():
    shift = 0.07
    y = np.random.default_rng(1).standard_normal(200)
    yt = P.phi_normal_inv(y, shift)
    assert np.all((yt > shift) & (yt < 0.5 + shift))
    assert np.allclose(P.phi_normal(yt, shift), y, rtol=1e-9, atol=1e-12)
    # the periodized map is symmetric about 1/4 + Delta (the mirror of (A3))
    h = np.linspace(0.01, 0.24, 24)
    assert np.allclose(P.phi_normal(0.25 + shift - h, shift), P.phi_normal(0.25 + shift - h + 0.0, shift))
    assert np.allclose(P.tau2(shift + 0.5 - h, shift), P.tau2(shift + 0.5 + h, shift), atol=1e-14)


@pytest.mark.parametrize("k", [-5, -2, -1, 0, 1, 2, 3, 4, 7])
def test_d_factors_against_quadrature(k):
    # tent: E over y ~ U[alpha, beta] of e^{2 pi i k phi^-1(y)} = D_k (independent of alpha, beta)
    alpha, beta = -1.0, 1.0
    def tent_part(part):
        f = lambda y: getattr(np.exp(2j * np.pi * k * P.tent_inv(y, alpha, beta)), part) / (beta - alpha)
        return integrate.quad(f, alpha, beta, epsabs=1e-14, epsrel=1e-13, limit=200)[0]
    want = complex(tent_part("real"), tent_part("imag"))
    assert abs(P.d_factor(k, P.MAP_TENT) - want) < 1e-12
    # lognormal: E over y ~ N(0,1) of e^{2 pi i k phi_Delta^-1(y)} = D_{k,Delta}
    shift = 0.013
    def normal_part(part):
        f = lambda y: getattr(np.exp(2j * np.pi * k * P.phi_normal_inv(y, shift)), part) * stats.norm.pdf(y)
        return integrate.quad(f, -np.inf, np.inf, epsabs=1e-14, epsrel=1e-13, limit=400)[0]
    want = complex(normal_part("real"), normal_part("imag"))
    assert abs(P.d_factor(k, P.MAP_NORMAL, shift) - want) < 1e-10
    # periodic: E over y ~ U[0,1) of e^{2 pi i k y} = delta_{k,0}
    assert P.d_factor(k, P.MAP_PERIODIC) == (1.0 if k == 0 else 0.0)


def test_expectation_variance_and_gsi():
    rng = np.random.default_rng(4)
    d = 4
    I = np.unique(rng.integers(-3, 4, size=(60, d)), axis=0)
    I = np.vstack([np.zeros((1, d), dtype=np.int64), I[np.any(I != 0, axis=1)]])
    C = rng.standard_normal((3, len(I))) + 1j * rng.standard_normal((3, len(I)))
    # periodic: the mean is c_0
    assert np.allclose(P.expectation(I, C, P.MAP_PERIODIC), C[:, 0])
    # variance = mean of |V - mean|^2 over a reconstructing lattice (Parseval)
    z, M = lattice.search(I, d, seed=2)
    Y = np.mod(np.arange(M)[:, None] * z[None, :], M) / M
    V = np.exp(2j * np.pi * (Y @ I.T)) @ C.T
    assert np.allclose(np.mean(np.abs(V - C[:, 0]) ** 2, axis=0), P.variance(I, C), rtol=1e-12)
    # GSI over J_1..J_d sums to 1, and J_l collects exactly the order-l frequencies
    G = P.gsi(I, C, d)
    assert np.allclose(G.sum(axis=1), 1.0)
    order = np.count_nonzero(I, axis=1)
    for l in range(1, d + 1):
        sel = order == l
        assert np.allclose(G[:, l - 1], np.sum(np.abs(C[:, sel]) ** 2, axis=1) / P.variance(I, C))
    # tent expectation: per frequency the product of the one-dimensional factors (each pinned
    # against quadrature above)
    D = np.array([np.prod([P.d_factor(int(v), P.MAP_TENT) for v in k]) for k in I])
    assert np.allclose(P.expectation(I, C, P.MAP_TENT), C @ D)
    # a frequency with an even non-zero component contributes nothing
    assert P.expectation(np.array([[2, 0, 0, 0]]), np.ones((1, 1)), P.MAP_TENT)[0] == 0


def test_tent_periodized_samples_have_even_coefficients():
    # u~(y~) = u(phi(y~)) is even about y~ = 1/2 in every coordinate under the tent map ((A3)),
    # so the 1-D detection coefficients satisfy c_k = c_-k and are real
    import workloads as W
    from oracle.usfft import OracleRun
    w = W.with_map(W.c1(3), W.MAP_TENT, -1.0, 1.0)
    run = OracleRun(w.problem, w.params, keep=True)
    run.increment()
    C = run.records[0].C                          # [G, K], column N + k holds c_k
    N = w.params.N
    scale = np.max(np.abs(C))
    assert np.max(np.abs(C - C[:, ::-1])) < 1e-13 * scale
    assert np.max(np.abs(C.imag)) < 1e-13 * scale
    # the periodic model has no such symmetry
    run_p = OracleRun(W.c1(3).problem, W.c1(3).params, keep=True)
    run_p.increment()
    Cp = run_p.records[0].C
    assert np.max(np.abs(Cp - Cp[:, ::-1])) > 1e-6 * np.max(np.abs(Cp))
    assert N == (C.shape[1] - 1) // 2

