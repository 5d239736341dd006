"""Pins of the oracle's random draws and coefficient model (CPU only)."""
import math
import os

import numpy as np
import pytest

from oracle import model, rng

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _rows(name):
    with open(os.path.join(GOLD, name)) as fh:
        return [line.split() for line in fh if line.strip() and not line.startswith("#")]


def test_splitmix64_reference_stream():
    # the stream of SplitMix64 from state 0 is mix64(k * gamma), k = 1, 2, ...
    want = [int(r[0]) for r in _rows("splitmix64_seed0.txt")]
    got = [rng.mix64((k * rng.GOLDEN_GAMMA) & rng.MASK64) for k in range(1, len(want) + 1)]
    assert got == want


def _unmix64(z):
    # inverse of the finaliser, step by step (xorshift inverses and modular inverses)
    z &= rng.MASK64
    z ^= (z >> 31) ^ (z >> 62)
    z = (z * pow(0x94D049BB133111EB, -1, 1 << 64)) & rng.MASK64
    z ^= (z >> 27) ^ (z >> 54)
    z = (z * pow(0xBF58476D1CE4E5B9, -1, 1 << 64)) & rng.MASK64
    z ^= (z >> 30) ^ (z >> 60)
    return z


def test_mix64_is_bijective():
    r = np.random.default_rng(0)
    for _ in range(200):
        x = int(r.integers(0, 1 << 63)) * 2 + int(r.integers(0, 2))
        assert _unmix64(rng.mix64(x)) == x


def test_uniform_moments_and_chi_square():
    n = 20000
    u = np.array([rng.uniform(7, rng.PHASE_TAIL, 3, i, 5) for i in range(n)])
    assert u.min() >= 0.0 and u.max() < 1.0
    assert abs(u.mean() - 0.5) < 4 * math.sqrt(1 / 12 / n)
    assert abs(u.var() - 1 / 12) < 0.005
    hist, _ = np.histogram(u, bins=50, range=(0, 1))
    chi2 = ((hist - n / 50) ** 2 / (n / 50)).sum()
    assert chi2 < 100          # 49 dof: p ~ 3e-5
    ints = np.array([rng.uniform_int(1, 6, 11, rng.PHASE_LATTICE, 2, 97, i, 2) for i in range(6000)])
    assert ints.min() == 1 and ints.max() == 6
    counts = np.bincount(ints)[1:]
    assert np.all(np.abs(counts - 1000) < 150)


def test_keys_depend_on_every_field():
    base = rng.key(1, 2, 3, 4, 5)
    assert len({base, rng.key(1, 2, 3, 4, 6), rng.key(1, 2, 3, 5, 5), rng.key(1, 2, 4, 4, 5),
                rng.key(1, 3, 3, 4, 5), rng.key(2, 2, 3, 4, 5)}) == 6


def test_table_4_2_mode_ordering():
    for j, m1, m2, k in (map(int, r) for r in _rows("table_4_2.txt")):
        assert model.diag_k(j) == k
        assert model.diag_m(j) == (m1, m2)
        # Sec. 4.3 formula k(j) = floor(-1/2 + sqrt(1/4 + 2j)) in floating point agrees
        assert math.floor(-0.5 + math.sqrt(0.25 + 2 * j)) == k
    modes = [model.mode_2d(j) for j in range(1, 11)]
    assert modes[:6] == [(1, 1), (1, 2), (2, 1), (1, 3), (2, 2), (3, 1)]
    sums = [a + b for a, b in modes]
    assert sums == sorted(sums)


def test_printed_ellipticity_bounds():
    for mu, c, amin, amax in (map(float, r) for r in _rows("periodic_example_bounds.txt")):
        lo, hi = model.ellipticity_bounds(model.COEF_AFFINE_SIN, c / math.sqrt(6), mu)
        assert abs(lo - amin) < 6e-6 and abs(hi - amax) < 6e-6
    # affine example of Sec. 4.3: c = 0.9/zeta(2) gives a_min = 0.1, a_max = 1.9
    from scipy.special import zeta
    lo, hi = model.ellipticity_bounds(model.COEF_AFFINE_SIN, 0.9 / zeta(2), 2.0)
    assert abs(lo - 0.1) < 1e-14 and abs(hi - 1.9) < 1e-14
    import workloads
    assert abs(workloads.c1().problem.coef_scale - 0.9 / zeta(2)) < 1e-15


def test_coefficient_closed_form_points():
    c = 0.5471
    # 1-D at x = 1/2: psi_j(1/2) = sin(j pi/2) = 1, 0, -1, 0
    sin_y = np.array([1.0, 1.0, -1.0, 1.0])
    a = model.coefficient(model.COEF_AFFINE_SIN, c, 2.0, np.array([[0.5]]), 1, sin_y)
    assert abs(a[0] - (1 + c * (1 + 1 / 9))) < 1e-15
    # d = 1 attains the lower bound 1 - c at x = 1/2, sin = -1
    a = model.coefficient(model.COEF_AFFINE_SIN, c, 2.0, np.array([[0.5]]), 1, np.array([-1.0]))
    assert abs(a[0] - model.ellipticity_bounds(model.COEF_AFFINE_SIN, c, 2.0, d=1)[0]) < 1e-15
    # 2-D mode 3 is (2,1): at x = (1/4, 1/2), psi_3 = sin(pi/2) sin(pi/2) = 1
    sin_y = np.array([0.0, 0.0, 1.0])
    a = model.coefficient(model.COEF_LOGNORMAL_SIN, 0.5, 2.0, np.array([[0.25, 0.5]]), 2, sin_y)
    assert abs(a[0] - math.exp(0.5 / 9)) < 1e-15
    # random points stay within the finite-d bounds (Eq. (2.1))
    r = np.random.default_rng(3)
    x = r.random((500, 2))
    lo, hi = model.ellipticity_bounds(model.COEF_AFFINE_SIN, c, 2.0, d=10)
    for _ in range(20):
        a = model.coefficient(model.COEF_AFFINE_SIN, c, 2.0, x, 2, np.sin(2 * np.pi * r.random(10)))
        assert a.min() >= lo - 1e-15 and a.max() <= hi + 1e-15
