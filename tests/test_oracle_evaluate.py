"""Pins of the oracle's evaluation and error functions (Section 4) on the CPU."""
import math

import numpy as np

import workloads as W
from oracle import evaluate as ev
from oracle import lattice
from oracle.usfft import NodeSet, sample


def test_polynomial_with_its_own_coefficients_is_reproduced():
    prob = W.trigpoly(G=4, d=3, N=4, seed=6, base_terms=5, node_terms=2, kmax=3, mag_lo=1e-3)
    keys = sorted({tuple(int(v) for v in f) for g in range(prob.G)
                   for f, c in zip(prob.tp_freqs[g], prob.tp_coefs[g]) if c != 0})
    I = np.array(keys, dtype=np.int64)
    C = np.zeros((prob.G, len(I)), dtype=np.complex128)
    for g in range(prob.G):
        for f, c in zip(prob.tp_freqs[g], prob.tp_coefs[g]):
            if c != 0:
                C[g, keys.index(tuple(int(v) for v in f))] += c
    Y = np.random.default_rng(1).random((50, 3))
    U = ev.sample_points(prob, Y)
    V = ev.evaluate(I, C, Y)
    # the test polynomials are real-valued (Hermitian supports), so V is real as well
    assert np.max(np.abs(V - U)) < 1e-13
    e2, ei = ev.errors(U, V)
    assert np.all(e2 <= ei + 1e-300) and np.max(ei) < 1e-13


def test_single_terms_against_cos_and_sin():
    Y = np.array([[0.1, 0.7], [0.25, 0.0], [0.9, 0.33]])
    I = np.array([[2, -1]])
    C = np.array([[1.0 + 0j], [0.5j]])
    V = ev.evaluate(I, C, Y)
    for j, (y1, y2) in enumerate(Y):
        a = 2 * math.pi * (2 * y1 - y2)
        assert abs(V[j, 0] - complex(math.cos(a), math.sin(a))) < 1e-15
        assert abs(V[j, 1] - 0.5j * complex(math.cos(a), math.sin(a))) < 1e-15


def test_parseval_on_a_reconstructing_lattice():
    # mean over the M nodes of |sum_k c_k e^{2 pi i k.y}|^2 = sum_k |c_k|^2 when k -> k.z mod M
    # is injective on I (the lattice rule integrates the cross terms to zero exactly)
    rng = np.random.default_rng(3)
    I = np.unique(rng.integers(-5, 6, size=(40, 3)), axis=0)
    z, M = lattice.search(I, 3, seed=9)
    assert lattice.is_reconstructing(I, z, M)
    C = (rng.standard_normal((2, len(I))) + 1j * rng.standard_normal((2, len(I))))
    Y = np.mod(np.arange(M)[:, None] * z[None, :], M) / M
    V = ev.evaluate(I, C, Y)
    assert np.allclose(np.mean(np.abs(V) ** 2, axis=0), np.sum(np.abs(C) ** 2, axis=1), rtol=1e-12)
    # a lattice with fewer nodes than |I| aliases, and the identity fails
    M2 = len(I) // 2
    Y2 = np.mod(np.arange(M2)[:, None] * z[None, :], M2) / M2
    V2 = ev.evaluate(I, C, Y2)
    assert not np.allclose(np.mean(np.abs(V2) ** 2, axis=0), np.sum(np.abs(C) ** 2, axis=1), rtol=1e-6)


def test_error_norms():
    U = np.zeros((8, 3))
    V = np.full((8, 3), 0.25 + 0j)
    e2, ei = ev.errors(U, V)
    assert np.allclose(e2, 0.25) and np.allclose(ei, 0.25)         # constant difference: equal
    V[3, 1] = 1.0 + 1.0j                                             # one outlier at node 1
    e2, ei = ev.errors(U, V)
    assert ei[1] == abs(1.0 + 1.0j) and e2[1] < ei[1]
    assert math.isclose(e2[1], math.sqrt((7 * 0.0625 + 2.0) / 8), rel_tol=1e-15)


def test_fe_samples_at_a_lattice_node_match_the_lattice_sampler():
    w = W.small_2d(n=7, d=3, seed=2, N=4, s=10)
    nodes = NodeSet(3, [0, 1, 2], np.array([1, 5, 11]), 17, {})
    U_lat = sample(w.problem, nodes)
    Y = np.mod(np.arange(17)[:, None] * nodes.z[None, :], 17) / 17
    U_pts = ev.sample_points(w.problem, Y)
    assert np.max(np.abs(U_pts - U_lat)) < 1e-15 * np.max(np.abs(U_lat)) + 1e-17
