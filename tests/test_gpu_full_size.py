"""Parity at the launch configurations the benchmark times (Algorithm 1, steps 2b-2e; Appendix A).

The 2-D workload's coupled step t = 3 (63x63 mesh, G = 3969, M = 6912 lattice nodes,
|J| = 4667 candidates: the in-place lattice FFT and the selection at full size), its step
t = 4 (a lattice too large for the in-place pass: the two-pass FFT), and the 128x128-mesh
lognormal workload's coupled step t = 3 (the large-mesh sampler).  The oracle cannot solve
every lattice node at these sizes in a test (tens of thousands of banded FE solves), so each
stage is checked against the oracle on the GPU's own input to that stage, for EVERY detection
iteration (usfft_set_keep_iterations keeps each iteration's samples, coefficients and union):
  - the candidate set J_t, the lattice (z, M) and the DFT indices: bit-exact with the oracle's
    (whose 1-D detection of dimension t runs in full);
  - FE samples: sampled lattice nodes against the oracle's banded Cholesky solves, 1e-10 relative;
  - lattice FFT + gather: the oracle's naive DFT of the GPU's samples U against the GPU's C,
    per node, 1e-10 relative (all mesh nodes, or a spread subset where the naive DFT would take
    too long);
  - selection + union: the oracle's selection over the GPU's C at every node, joined over the
    nodes and the iterations so far, against the GPU's union bitmap after that iteration: bit-exact
    (both sides decide on the same numbers with the same |c|^2 and tie rule);
  - the detected set: the rows of J_t the final bitmap marks.
The starting state (t - 1, I^(1..t-1), theta) is the oracle's own for the 63x63 workload at
t = 3 (the oracle runs increments 1 and 2 in full) and the GPU's for the later or larger steps
(their earlier increments are covered by the tests of the smaller steps)."""
import copy

import numpy as np
import pytest

import workloads as W
from oracle import detect, dft, lattice, rng
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


@pytest.fixture(scope="module")
def c2_state_t2():
    """The oracle's state after increments 1 and 2 of the 2-D workload (seed 1)."""
    w = W.c2(1)
    run = OracleRun(w.problem, w.params)
    run.increment()
    run.increment()
    return w, run


def check_coupled_step(B, plan, run, w, t, rows_per_iter=5, dft_nodes=None, ctx=""):
    """Run increment t on the plan (keeping every iteration) and on the oracle's planner from the
    same state, and check every stage of every detection iteration as the module docstring says."""
    prob, p = w.problem, w.params
    d = prob.d
    plan.set_keep_iterations(True)
    info = plan.increment()
    assert info["t"] == t
    # 1-D detection of dimension t (in full on the oracle), candidate set and lattice
    run.detect_1d(t)
    J = lattice.candidate_set(run.I_prefix, np.array(run.I1d[t], dtype=np.int64), p.N)
    z, M = lattice.search(J, t, p.seed, p.max_lattice_trials)
    m = lattice.lattice_indices(J, z, M)
    Jg, mg = plan.get_candidates()
    zg, Mg = plan.get_lattice()
    assert np.array_equal(Jg, J), f"{ctx}: candidate set"
    assert Mg == M and np.array_equal(zg, z), f"{ctx}: lattice"
    assert np.array_equal(mg, m), f"{ctx}: DFT indices"
    r_t = p.r if t < d else 1
    s_t = p.s_local if t < d else p.s
    assert plan.kept_iterations() == r_t
    mesh = run.mesh
    union = set()
    bits = None
    gen = np.random.default_rng(t)
    for i in range(1, r_t + 1):
        U, C, bits = plan.get_iteration(i)
        assert U.shape == (M, prob.G) and C.shape == (prob.G, len(J))
        # FE samples at sampled lattice nodes (first, last, spread, random)
        tails = {j - 1: rng.uniform(p.seed, rng.PHASE_TAIL, t, i, j) for j in range(t + 1, d + 1)}
        rows = np.unique(np.concatenate([[0, M - 1, M // 2], gen.integers(0, M, size=max(0, rows_per_iter - 3))]))
        Uo = sample_rows(prob, NodeSet(d, list(range(t)), z, M, tails), rows, mesh)
        err = np.max(np.abs(U[rows] - Uo)) / np.max(np.abs(Uo))
        assert err < TOL, f"{ctx}: iteration {i}: samples rel err {err:.2e}"
        # lattice FFT + gather against the naive DFT of the same samples
        nodes = np.arange(prob.G) if dft_nodes is None else np.unique(np.linspace(0, prob.G - 1, dft_nodes).astype(int))
        Co = dft.coefficients(U[:, nodes], m, M)
        e = node_rel(C[nodes], Co)
        assert e < TOL, f"{ctx}: iteration {i}: coefficient rel err {e:.2e}"
        # selection at every node over the GPU's coefficients, joined: the union bitmap
        detect.union_over_nodes(C, run.theta, s_t, union)
        want = np.zeros(len(J), dtype=bool)
        want[sorted(union)] = True
        assert np.array_equal(bits, want), f"{ctx}: iteration {i}: union differs at {np.nonzero(bits != want)[0][:8]}"
    got = plan.get_set()
    assert np.array_equal(got, J[bits]), f"{ctx}: detected set"
    plan.set_keep_iterations(False)
    return info, J, got


@pytest.mark.parametrize("precision", [W.PRECISION_MIXED, W.PRECISION_FP64, W.PRECISION_FP64_DST])
def test_c2_timed_step_t3_full_size(B, c2_state_t2, precision):
    w, run0 = c2_state_t2
    w = W.with_precision(w, precision)
    run = copy.deepcopy(run0)
    plan = B.Plan(w.problem, w.params)
    plan.resume(2, run.I_prefix, run.theta)
    run.t = 3
    info, J, got = check_coupled_step(B, plan, run, w, 3, ctx=f"c2 t=3 precision {precision}")
    # the benchmark's launch configuration: in-place FFT at M = 6912 over 4667 candidates
    assert info["M"] == 6912 and info["n_candidates"] == 4667
    plan.close()


def test_c2_two_pass_step_t4(B, c2_state_t2):
    # increment 4 from the GPU's state after increment 3: its lattice is too large for the
    # in-place FFT (two passes through the intermediate array)
    w, run0 = c2_state_t2
    w = W.with_precision(w, W.PRECISION_MIXED)
    plan = B.Plan(w.problem, w.params)
    plan.resume(2, run0.I_prefix, run0.theta)
    plan.increment()
    run = OracleRun(w.problem, w.params)
    run.resume(3, plan.get_set(), run0.theta)
    run.t = 4
    info, _, _ = check_coupled_step(B, plan, run, w, 4, rows_per_iter=4, dft_nodes=48, ctx="c2 t=4")
    assert 16 * info["M"] > 232448  # the in-place pass holds at most 232448 bytes of complex values
    plan.close()


@pytest.mark.parametrize("precision", [W.PRECISION_MIXED, W.PRECISION_FP64_DST])
def test_c3_coupled_step_t3(B, precision):
    # the 128x128 mesh (G = 16129), lognormal-type coefficient, d = 20, r = 2: increments 1 and 2 on
    # the GPU, then step 3 from that state against the oracle (the large-mesh mixed sampler and the
    # fp64 sampler with the same preconditioner)
    w = W.with_precision(W.c3(1), precision)
    plan = B.Plan(w.problem, w.params)
    plan.increment()
    info2 = plan.increment()
    run = OracleRun(w.problem, w.params)
    run.resume(2, plan.get_set(), info2["theta"])      # theta: fixed by the plan's first 1-D detection
    run.t = 3
    check_coupled_step(B, plan, run, w, 3, rows_per_iter=3, ctx=f"c3 t=3 precision {precision}")
    plan.close()
