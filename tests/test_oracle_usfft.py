"""Pins of the oracle's increment driver: exact recovery of trigonometric polynomials
(Theorem 1.1) and the structural invariants of Algorithm 1 (CPU only)."""
import numpy as np
import pytest

import workloads as W
from oracle import rng
from oracle.usfft import OracleRun


def _support(prob):
    out = []
    for g in range(prob.G):
        terms = {}
        for f, c in zip(prob.tp_freqs[g], prob.tp_coefs[g]):
            if c != 0:
                terms[tuple(int(v) for v in f)] = c
        out.append(terms)
    return out


def _projected(terms, coords, tail_coords, tails):
    """sum over h with the same projection onto `coords` of c_h exp(2 pi i h_tail . y')."""
    acc = {}
    for h, c in terms.items():
        k = tuple(h[j] for j in coords)
        ph = sum(h[j] * tails[j] for j in tail_coords)
        acc[k] = acc.get(k, 0) + c * np.exp(2j * np.pi * ph)
    return acc


def _margins_ok(prob, params, theta):
    sup = _support(prob)
    d = prob.d
    for t in range(1, d + 1):
        for i in range(1, params.r + 1):
            tails = {j - 1: rng.uniform(params.seed, rng.PHASE_1D_TAIL, t, i, j) for j in range(1, d + 1) if j != t}
            for terms in sup:
                for v in _projected(terms, [t - 1], sorted(tails), tails).values():
                    if 0 < abs(v) < 10 * theta:
                        return False
        if t >= 2:
            for i in range(1, (params.r if t < d else 1) + 1):
                tails = {j - 1: rng.uniform(params.seed, rng.PHASE_TAIL, t, i, j) for j in range(t + 1, d + 1)}
                for terms in sup:
                    for v in _projected(terms, list(range(t)), sorted(tails), tails).values():
                        if 0 < abs(v) < 10 * theta:
                            return False
    return True


@pytest.mark.parametrize("G,seed", [(1, 3), (5, 11), (12, 4)])
def test_exact_recovery_of_trigonometric_polynomials(G, seed):
    d, N = 4, 5
    prob = W.trigpoly(G=G, d=d, N=N, seed=seed, base_terms=5, node_terms=2, kmax=3, mag_lo=1e-4)
    params = W.Params(N=N, s=40, s_local=40, delta=1e-9, delta_is_relative=False, r=1, seed=seed)
    assert _margins_ok(prob, params, params.delta)
    run = OracleRun(prob, params, keep=True)
    sup = _support(prob)
    union = set().union(*[set(s) for s in sup])
    prev = None
    for t in range(1, d + 1):
        I = run.increment()
        want = {k[:t] for k in union}
        got = {tuple(int(v) for v in row) for row in I}
        assert got == want, t
        # the detected set lies in J_t and projects into the previous detected set
        if t >= 2:
            Jset = {tuple(int(v) for v in row) for row in run.J}
            assert got <= Jset
            assert {k[:t - 1] for k in got} <= {tuple(int(v) for v in row) for row in prev}
        prev = I
    # at t = d there are no tails: the coefficients are the polynomial's own (Theorem 1.1)
    last = run.records[-1]
    assert last.coupled and last.t == d
    for g in range(G):
        for col, k in enumerate(run.J):
            want_c = sup[g].get(tuple(int(v) for v in k), 0.0)
            assert abs(last.C[g, col] - want_c) < 1e-13


def test_relative_threshold_uses_first_mean_coefficient():
    w = W.c1(2)
    run = OracleRun(w.problem, w.params, keep=True)
    run.increment()
    rec = run.records[0]
    A = np.max(np.abs(rec.C[:, w.params.N]))
    assert run.theta == w.params.delta * A
    # k = 0 is the mean over y_1 of u, so it is detected everywhere and A > 0
    assert 0 in run.I1d[1] and A > 0


def test_last_increment_uses_one_iteration_and_s():
    # Algorithm 1, step 2: r~ = 1 and s~ = s at t = d
    prob = W.trigpoly(G=3, d=3, N=4, seed=2, base_terms=4, node_terms=1, kmax=2, mag_lo=1e-3)
    params = W.Params(N=4, s=2, s_local=30, delta=1e-9, delta_is_relative=False, r=3, seed=5)
    run = OracleRun(prob, params, keep=True)
    for _ in range(3):
        run.increment()
    last = [r for r in run.records if r.coupled and r.t == 3]
    assert len(last) == 1
    assert all(len(s) <= 2 for s in last[0].selected)
    mid = [r for r in run.records if r.coupled and r.t == 2]
    assert len(mid) == 3


def test_step3_reconstruction_returns_the_polynomial_coefficients():
    # Algorithm 1, step 3: on the detected set I (= the union of the supports here) a
    # reconstructing rank-1 lattice samples the full d-variate function, so the lattice
    # DFT returns each node's own coefficients (Appendix A; no tails, no threshold)
    from oracle import lattice
    d, N, G = 4, 5, 7
    prob = W.trigpoly(G=G, d=d, N=N, seed=8, base_terms=5, node_terms=2, kmax=3, mag_lo=1e-4)
    params = W.Params(N=N, s=40, s_local=40, delta=1e-9, delta_is_relative=False, r=1, seed=8)
    assert _margins_ok(prob, params, params.delta)
    run = OracleRun(prob, params, keep=True)
    with pytest.raises(AssertionError):
        run.reconstruct()                        # only after all d increments
    for _ in range(d):
        run.increment()
    I, z, M, C = run.reconstruct()
    sup = _support(prob)
    assert {tuple(int(v) for v in k) for k in I} == set().union(*[set(s) for s in sup])
    assert lattice.is_reconstructing(I, z, M) and z[0] == 1
    # the phase-4 draws give a lattice of their own (not the last coupled step's)
    zs, Ms = lattice.search(I, d, params.seed, params.max_lattice_trials, phase=rng.PHASE_RECON)
    assert Ms == M and np.array_equal(zs, z)
    assert C.shape == (G, len(I))
    for g in range(G):
        want = np.array([sup[g].get(tuple(int(v) for v in k), 0.0) for k in I])
        assert np.max(np.abs(C[g] - want)) < 1e-13


@pytest.mark.parametrize("G,seed", [(3, 5), (9, 12)])
def test_random_lattices_recover_trigonometric_polynomials(G, seed):
    # random rank-1 lattices with the median estimate (Algorithm A, reading of the sizes and the
    # estimator): for sparse polynomials most lattices are free of collisions between non-zero
    # coefficients, so the median returns every projected coefficient exactly and the detected
    # sets are the projections of the union of the supports, as with reconstructing lattices
    from oracle import lattice
    d, N = 4, 5
    prob = W.trigpoly(G=G, d=d, N=N, seed=seed, base_terms=5, node_terms=2, kmax=3, mag_lo=1e-4)
    params = W.Params(N=N, s=40, s_local=40, delta=1e-9, delta_is_relative=False, r=1, seed=seed,
                      rr_lattices=5, rr_size_factor=4.0)
    assert _margins_ok(prob, params, params.delta)
    run = OracleRun(prob, params, keep=True)
    sup = _support(prob)
    union = set().union(*[set(s) for s in sup])
    single = 0
    for t in range(1, d + 1):
        I = run.increment()
        assert {tuple(int(v) for v in row) for row in I} == {k[:t] for k in union}, t
        if t >= 2:
            rec = run.records[-1]
            assert rec.coupled and len(rec.M) == 5 and len(set(rec.M)) == 5
            assert all(lattice.is_smooth7(M) for M in rec.M)
            assert rec.M[0] >= 4.0 * max(len(run.J) // max(len(run.I1d[t]), 1), len(run.I1d[t]))
            assert all(np.all((z >= 1) & (z < M)) for z, M in zip(rec.z, rec.M))
            single += lattice.search(run.J, t, seed)[1]
    last = run.records[-1]
    for g in range(G):
        for col, k in enumerate(run.J):
            assert abs(last.C[g, col] - sup[g].get(tuple(int(v) for v in k), 0.0)) < 1e-13
    # the step-3 reconstruction still uses one reconstructing lattice
    I, z, M, C = run.reconstruct()
    assert lattice.is_reconstructing(I, z, M)


@pytest.mark.parametrize("G,seed", [(3, 8), (9, 21)])
def test_step3_multiple_lattices_return_the_polynomial_coefficients(G, seed):
    # Algorithm 1, step 3 on multiple rank-1 lattices (Appendix A): in a lattice where k is alone
    # at its index, the lattice DFT at k.z mod M is c_k itself for a polynomial supported in I, so
    # reading every coefficient from its first such lattice recovers the polynomial exactly
    from oracle import lattice
    d, N = 4, 5
    prob = W.trigpoly(G=G, d=d, N=N, seed=seed, base_terms=5, node_terms=2, kmax=3, mag_lo=1e-4)
    params = W.Params(N=N, s=40, s_local=40, delta=1e-9, delta_is_relative=False, r=1, seed=seed)
    assert _margins_ok(prob, params, params.delta)
    run = OracleRun(prob, params, keep=True)
    for _ in range(d):
        run.increment()
    I, lats, C = run.reconstruct_multiple()
    sup = _support(prob)
    assert {tuple(int(v) for v in k) for k in I} == set().union(*[set(s) for s in sup])
    assert C.shape == (G, len(I))
    for g in range(G):
        want = np.array([sup[g].get(tuple(int(v) for v in k), 0.0) for k in I])
        assert np.max(np.abs(C[g] - want)) < 1e-13
    # sizes: the first one of the bound's range 2 (|I| - 1) and distinct 7-smooth sizes after it
    Ms = [M for _, M in lats]
    assert Ms[0] == lattice.next_admissible(max(2 * (len(I) - 1), 2))
    assert all(lattice.is_smooth7(M) for M in Ms) and all(a < b for a, b in zip(Ms, Ms[1:]))
    assert run.samples_used >= sum(Ms)


def _alone(I, z, M):
    m = [int(np.dot(k, z)) % M for k in I]
    return np.array([m.count(v) == 1 for v in m])


@pytest.mark.parametrize("seed,n,d", [(1, 40, 3), (2, 200, 5), (3, 700, 8)])
def test_multiple_lattices_cover_every_frequency(seed, n, d):
    # the construction's stopping rule, recomputed by brute force: every k of I is alone at its
    # index in the lattice first[k] and in no earlier one; the rule stops at the first lattice
    # that completes the cover; and the sample total stays within the paper's bound
    # ceil(2 ln(2|I|)) 4 (|I| - 1) (Appendix A, with c = 2 and delta = 1/2)
    import math
    from oracle import lattice
    rs = np.random.default_rng(seed)
    I = np.unique(rs.integers(-16, 17, size=(n, d)), axis=0).astype(np.int64)
    lats, first = lattice.multiple_lattices(I, d, seed)
    assert first is not None
    alone = np.array([_alone(I, z, M) for z, M in lats])            # [L, |I|]
    for k in range(len(I)):
        assert alone[first[k], k] and not alone[:first[k], k].any()
    assert first.max() == len(lats) - 1
    total = sum(M for _, M in lats)
    assert total <= math.ceil(2 * math.log(2 * len(I))) * 4 * (len(I) - 1)
    assert all(np.all((z >= 1) & (z < M)) and all(math.gcd(int(v), M) == 1 for v in z) for z, M in lats)


def test_lattice_dft_is_the_aliasing_sum():
    # brute force on a tiny set: the lattice DFT of a trigonometric polynomial at index m is the sum
    # of c_k over all k with k.z = m (mod M), so c_k alone at its index is read exactly, and a
    # shared index gives the sum of the colliding coefficients
    from oracle import dft, lattice
    rs = np.random.default_rng(4)
    d, M = 2, 7
    z = np.array([1, 3])
    K = np.array([[0, 0], [1, 0], [0, 1], [2, -1], [-1, 2], [3, 3]])
    c = rs.normal(size=len(K)) + 1j * rs.normal(size=len(K))
    nodes = (np.outer(np.arange(M), z) % M) / M                       # y_i = frac(i z / M)
    f = np.array([np.sum(c * np.exp(2j * np.pi * (K @ y))) for y in nodes])
    m = lattice.lattice_indices(K, z, M)
    got = dft.coefficients(f.real[:, None], m, M)[0] + 1j * dft.coefficients(f.imag[:, None], m, M)[0]
    for a in range(len(K)):
        assert abs(got[a] - c[m == m[a]].sum()) < 1e-13
