"""Parity at the 128x128-mesh shape (n = 127 interior nodes per side, G = 16129, lognormal-type
coefficient, d = 20): the large-mesh mixed-precision sampler against the oracle's banded FE
solves on sampled outputs (every oracle solve costs a fraction of a second at this size).

Covered: FE samples at explicit points; the first increment in full (65 lattice nodes, the
1-D detection of dimension 1 with r = 1: samples, coefficients and the detected set); the
coupled step t = 2 from the oracle's state: the lattice bit-exact and four sampled lattice
nodes of its samples.  Also the boundary sizes n = 64 and n = 100 on the small 2-D problem."""
import dataclasses

import numpy as np
import pytest

import workloads as W
from oracle import evaluate as ev
from oracle import lattice, rng
from oracle.usfft import NodeSet, OracleRun, sample_rows

pytestmark = pytest.mark.gpu

TOL = 1e-10


@pytest.fixture(scope="module")
def B():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    from paper_2109_04131_gb300 import binding
    binding.load_library()
    return binding


def node_rel(Cg, Co):
    den = np.max(np.abs(Co), axis=1)
    den[den == 0] = 1.0
    return float(np.max(np.max(np.abs(Cg - Co), axis=1) / den))


def test_c3_shape_sampled_parity(B):
    w = W.c3(1)
    params = dataclasses.replace(w.params, r=1)
    prob = w.problem
    plan = B.Plan(prob, params)
    run = OracleRun(prob, params, keep=True)
    # FE solutions at explicit parameters
    Y = W.test_points(2, prob.d, seed=3)
    U = plan.sample_points(Y)
    Uo = ev.sample_points(prob, Y, run.mesh)
    assert np.max(np.abs(U - Uo)) <= TOL * np.max(np.abs(Uo))
    # increment 1 in full: 65 solves on each side
    want = run.increment()
    info = plan.increment()
    rec = run.records[-1]
    Ug = plan.get_samples()
    assert np.max(np.abs(Ug - rec.U)) <= TOL * np.max(np.abs(rec.U))
    assert node_rel(plan.get_coefficients(), rec.C) < TOL
    got = plan.get_set()
    assert got.shape == want.shape and np.array_equal(got, want)
    assert info["cg_iters_max"] > 0
    # coupled step t = 2 from the oracle's state: lattice bit-exact, four sampled nodes
    plan.resume(1, run.I_prefix, run.theta)
    run.detect_1d(2)
    J = lattice.candidate_set(run.I_prefix, np.array(run.I1d[2], dtype=np.int64), params.N)
    z, M = lattice.search(J, 2, params.seed)
    plan.increment()
    zg, Mg = plan.get_lattice()
    assert Mg == M and np.array_equal(zg, z)
    tails = {j - 1: rng.uniform(params.seed, rng.PHASE_TAIL, 2, 1, j) for j in range(3, prob.d + 1)}
    rows = np.array([0, 1, M // 2, M - 1])
    Uo = sample_rows(prob, NodeSet(prob.d, [0, 1], z, M, tails), rows, run.mesh)
    Ug = plan.get_samples()[rows]
    assert np.max(np.abs(Ug - Uo)) <= TOL * np.max(np.abs(Uo))
    plan.close()


@pytest.mark.parametrize("n", [64, 100])
def test_large_mesh_boundary_sizes(B, n):
    w = W.with_precision(W.small_2d(n=n, d=3, seed=4, N=3, s=10), W.PRECISION_MIXED)
    plan = B.Plan(w.problem, w.params)
    run = OracleRun(w.problem, w.params, keep=True)
    Y = W.test_points(3, 3, seed=n)
    U = plan.sample_points(Y)
    Uo = ev.sample_points(w.problem, Y, run.mesh)
    assert np.max(np.abs(U - Uo)) <= TOL * np.max(np.abs(Uo))
    # the fp64 mode with the same preconditioner serves these sizes too
    p64 = B.Plan(w.problem, dataclasses.replace(w.params, precision=W.PRECISION_FP64_DST))
    U64 = p64.sample_points(Y)
    assert np.max(np.abs(U64 - Uo)) <= TOL * np.max(np.abs(Uo))
    p64.close()
    # the Jacobi modes stay limited to n <= 63
    with pytest.raises(B.UsfftError):
        B.Plan(w.problem, dataclasses.replace(w.params, precision=W.PRECISION_FP64))
    plan.close()


@pytest.mark.parametrize("precision", [W.PRECISION_MIXED, W.PRECISION_FP64_DST])
def test_largest_mesh_and_dimension(B, precision):
    # n = 127 with d = 64 (the largest mesh with the largest stochastic dimension; the mixed kernel's
    # shared-memory tables are then at their largest): FE samples at explicit points against the
    # oracle's banded solves
    prob = W.Problem(kind=W.PDE_2D, n=127, d=64)
    params = W.Params(N=3, s=10, s_local=10, delta=1e-8, delta_is_relative=True, r=1, seed=2, precision=precision)
    plan = B.Plan(prob, params)
    run = OracleRun(prob, params)
    Y = W.test_points(2, 64, seed=9)
    U = plan.sample_points(Y)
    Uo = ev.sample_points(prob, Y, run.mesh)
    assert np.max(np.abs(U - Uo)) <= TOL * np.max(np.abs(Uo))
    plan.close()
