"""Parity of the CUDA path (through the C ABI) with the CPU oracle.

Every increment starts both sides from the oracle's state (usfft_resume: t, I^(1..t),
theta).  Bars: lattice (z, M), candidate lists and DFT indices bit-exact; detected sets
bit-exact for the test polynomials (magnitudes far from the threshold and from each
other) and, for PDE samples, bit-exact except at near-ties of the oracle's magnitudes
(conjugate pairs have equal magnitude exactly, so rounding decides a cut between them);
samples U and coefficients C within 1e-10 relative on the fp64 path and the mixed path,
in the per-node norm max_k |C_gpu - C_orc| / max_k |C_orc| (the reading of "1e-10
relative" that ignores noise-level coefficients)."""
import dataclasses

import numpy as np
import pytest

import workloads as W
from oracle.usfft import OracleRun

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
    """max over nodes of max_k |Cg - Co| / max_k |Co|."""
    den = np.max(np.abs(Co), axis=1)
    den[den == 0] = 1.0
    return float(np.max(np.max(np.abs(Cg - Co), axis=1) / den))


def near_ties(records, theta, s_tilde_of, rel=2e-10):
    """Candidate positions whose oracle magnitude lies within rel * max_k |C_g| of the
    threshold or of the node's s~-th largest magnitude, in any iteration: the only
    places where rounding may decide the selection (|c_k| = |c_-k| for real samples)."""
    amb = set()
    for rec in records:
        s_t = s_tilde_of(rec)
        mags = np.abs(rec.C)
        for g in range(mags.shape[0]):
            mg = mags[g]
            tol = rel * mg.max()
            amb.update(np.nonzero(np.abs(mg - theta) <= tol)[0].tolist())
            elig = np.sort(mg[mg >= theta])[::-1]
            if len(elig) > s_t:
                tau = elig[s_t - 1]
                amb.update(np.nonzero(np.abs(mg - tau) <= tol)[0].tolist())
    return amb


def compare_increment(plan, run, ctx, exact=True):
    """Run increment t = run.t + 1 on both sides from the oracle's state and compare: lattice,
    candidates, every detection iteration's samples, coefficients and cumulative union, and the
    detected set."""
    if run.t > 0:
        plan.resume(run.t, run.I_prefix, run.theta)
    first = len(run.records)
    want = run.increment()
    plan.set_keep_iterations(True)
    info = plan.increment()
    got = plan.get_set()
    # every detection iteration of the last detection step (the coupled step, or the 1-D detection
    # at t = 1): samples and coefficients within TOL, the union of iterations 1..i against the
    # oracle's (exact, or up to near-ties)
    coupled = [r for r in run.records[first:] if r.coupled]
    recs = run.records[first:] if run.t == 1 else coupled      # none: an empty candidate set
    kept = plan.kept_iterations()
    if recs and recs[-1].U is not None and not isinstance(recs[-1].M, list):
        assert kept == len(recs), f"{ctx}: kept {kept} iterations, oracle ran {len(recs)}"
        union = set()
        for i, rec in enumerate(recs, start=1):
            U, C, bits = plan.get_iteration(i)
            assert np.max(np.abs(U - rec.U)) <= TOL * np.max(np.abs(rec.U)), f"{ctx}: iteration {i} samples"
            assert node_rel(C, rec.C) < TOL, f"{ctx}: iteration {i} coefficients"
            for sg in rec.selected:
                union.update(int(k) for k in sg)
            want_bits = np.zeros(len(bits), dtype=bool)
            want_bits[sorted(union)] = True
            if not np.array_equal(bits, want_bits):
                assert not exact, f"{ctx}: iteration {i} union differs"
                d = run.prob.d
                amb = near_ties(recs[:i], run.theta, lambda r: run.p.s_local if (r.t < d or not r.coupled) else run.p.s)
                assert set(np.nonzero(bits != want_bits)[0].tolist()) <= amb, f"{ctx}: iteration {i} union"
    plan.set_keep_iterations(False)
    assert info["t"] == run.t
    if not (got.shape == want.shape and np.array_equal(got, want)):
        assert not exact, f"{ctx}: detected sets differ at t={run.t}"
        recs = [r for r in run.records[first:] if r.coupled]
        d = run.prob.d
        amb = near_ties(recs, run.theta, lambda r: run.p.s_local if r.t < d else run.p.s)
        diff = {tuple(r) for r in got.tolist()} ^ {tuple(r) for r in want.tolist()}
        allowed = {tuple(int(v) for v in run.J[k]) for k in amb}
        assert diff <= allowed, f"{ctx}: t={run.t}: {len(diff - allowed)} differences are not near-ties"
    z, M = plan.get_lattice()
    last = run.records[-1]
    assert M == last.M and np.array_equal(z, last.z), ctx
    J, m = plan.get_candidates()
    if last.coupled:
        assert np.array_equal(J, run.J), ctx
    assert np.array_equal(m, last.m), ctx
    if last.U is not None:
        U = plan.get_samples()
        assert U.shape == last.U.shape
        err = np.max(np.abs(U - last.U)) / np.max(np.abs(last.U))
        assert err < TOL, f"{ctx}: samples rel err {err:.2e}"
        C = plan.get_coefficients()
        assert C.shape == last.C.shape
        e = node_rel(C, last.C)
        assert e < TOL, f"{ctx}: coefficient rel err {e:.2e}"
    return info


@pytest.mark.parametrize("seed", [1, 2])
def test_1d_workload_full_run(B, seed):
    w = W.c1(seed)
    plan = B.Plan(w.problem, w.params)
    run = OracleRun(w.problem, w.params, keep=True)
    for t in range(1, w.problem.d + 1):
        info = compare_increment(plan, run, f"c1 seed {seed}", exact=False)
        assert info["kernel_launches"] > 0
    plan.close()


@pytest.mark.parametrize("G,seed", [(1, 3), (12, 4), (37, 9)])
def test_trigpoly_exact_recovery(B, G, seed):
    d, N = 4, 5
    prob = W.trigpoly(G=G, d=d, N=N, seed=seed, base_terms=5, node_terms=2, kmax=3, mag_lo=1e-4)
    params = W.Params(N=N, s=40, s_local=40, delta=1e-9, delta_is_relative=False, r=1, seed=seed)
    plan = B.Plan(prob, params)
    run = OracleRun(prob, params, keep=True)
    union = set()
    for g in range(G):
        for f, c in zip(prob.tp_freqs[g], prob.tp_coefs[g]):
            if c != 0:
                union.add(tuple(int(v) for v in f))
    for t in range(1, d + 1):
        compare_increment(plan, run, f"trigpoly G={G}")
        got = {tuple(int(v) for v in row) for row in plan.get_set()}
        assert got == {k[:t] for k in union}
    # t = d: the coefficients are the polynomial's own
    C = plan.get_coefficients()
    J, _ = plan.get_candidates()
    for g in range(G):
        truth = {tuple(int(v) for v in f): c for f, c in zip(prob.tp_freqs[g], prob.tp_coefs[g]) if c != 0}
        want = np.array([truth.get(tuple(int(v) for v in k), 0.0) for k in J])
        assert np.max(np.abs(C[g] - want)) < 1e-13
    plan.close()


def test_trigpoly_full_grid_radix3_lattice(B):
    # full-grid support [-40,40]^2: |J| = 81^2 = 6561 candidates on the lattice of size 3^8 (the
    # in-place FFT with radix-3 stages only); the two-pass FFT is exercised by
    # test_largest_search_domain_two_pass_exact_recovery and the full-size step t = 4
    prob = W.trigpoly_grid(G=3, d=2, K=40, seed=5)
    params = W.Params(N=45, s=20000, s_local=20000, delta=1e-9, delta_is_relative=False, r=1, seed=3)
    plan = B.Plan(prob, params)
    run = OracleRun(prob, params, keep=True)
    compare_increment(plan, run, "grid t=1")
    info = compare_increment(plan, run, "grid t=2")
    assert info["M"] > 4096 and info["n_candidates"] == 81 * 81
    assert len(plan.get_set()) == 81 * 81
    plan.close()


@pytest.mark.parametrize("precision", [W.PRECISION_FP64, W.PRECISION_MIXED, W.PRECISION_MIXED_JACOBI,
                                       W.PRECISION_FP64_DST])
def test_small_2d_matches_oracle(B, precision):
    w = W.with_precision(W.small_2d(n=15, d=4, seed=2, N=6, s=30), precision)
    plan = B.Plan(w.problem, w.params)
    run = OracleRun(w.problem, w.params, keep=True)
    for t in range(1, 4):
        info = compare_increment(plan, run, f"2-D n=15 precision={precision}", exact=False)
        assert info["cg_iters_max"] > 0
    plan.close()


def test_largest_search_domain_two_pass_exact_recovery(B):
    # the largest search domain (N = 127, int8 frequencies): a polynomial supported on the full grid
    # [-127, 127]^2 has |J| = 255^2 = 65025 candidates at t = 2, far beyond the in-place FFT (two
    # passes with L1, L2 in the hundreds); its coefficients are recovered exactly (Theorem 1.1)
    prob = W.trigpoly_grid(G=2, d=2, K=127, seed=11)
    params = W.Params(N=127, s=70000, s_local=70000, delta=1e-9, delta_is_relative=False, r=1, seed=4)
    plan = B.Plan(prob, params)
    plan.increment()
    info = plan.increment()
    assert info["n_candidates"] == 255 * 255 and info["M"] >= 255 * 255
    z, M = plan.get_lattice()
    J, m = plan.get_candidates()
    from oracle import lattice
    zo, Mo = lattice.search(J, 2, params.seed)
    assert M == Mo and np.array_equal(z, zo)
    C = plan.get_coefficients()
    for g in range(prob.G):
        truth = {tuple(int(v) for v in f): c for f, c in zip(prob.tp_freqs[g], prob.tp_coefs[g]) if c != 0}
        want = np.array([truth[tuple(int(v) for v in k)] for k in J])
        assert np.max(np.abs(C[g] - want)) < 1e-13
    assert len(plan.get_set()) == 255 * 255
    plan.close()


def test_2d_ragged_mesh_sizes(B):
    # n = 9 (81 nodes: one partial warp) and n = 33 (1089 nodes: two nodes per thread, ragged;
    # DST tiles padded from 33 to 48), both precisions; the fp64 sine-transform mode also at
    # n = 1 and 2 (a single transform tile, odd and even sizes)
    for n, prec in ((9, W.PRECISION_FP64), (33, W.PRECISION_FP64), (9, W.PRECISION_MIXED), (33, W.PRECISION_MIXED),
                    (1, W.PRECISION_FP64_DST), (2, W.PRECISION_FP64_DST), (9, W.PRECISION_FP64_DST),
                    (33, W.PRECISION_FP64_DST)):
        w = W.with_precision(W.small_2d(n=n, d=3, seed=5, N=4, s=20), prec)
        plan = B.Plan(w.problem, w.params)
        run = OracleRun(w.problem, w.params, keep=True)
        for t in range(1, 3):
            compare_increment(plan, run, f"2-D n={n}", exact=False)
        plan.close()


@pytest.mark.parametrize("precision", [W.PRECISION_FP64, W.PRECISION_MIXED])
def test_c2_shape_first_increments(B, precision):
    # the 2-D workload at full mesh size (63x63 interior, d = 10): increment 1 in full,
    # increment 2 in full (about 1000 oracle solves)
    w = W.with_precision(W.c2(1), precision)
    plan = B.Plan(w.problem, w.params)
    run = OracleRun(w.problem, w.params, keep=True)
    compare_increment(plan, run, "c2 t=1", exact=False)
    compare_increment(plan, run, "c2 t=2", exact=False)
    plan.close()


def test_replay_and_rewind_reproduce_the_increment(B):
    w = W.small_2d(n=15, d=4, seed=3, N=6, s=30)
    plan = B.Plan(w.problem, w.params)
    for _ in range(3):
        plan.increment()
    S = plan.get_set()
    C = plan.get_coefficients()
    sel = plan.get_selection()
    n = plan.replay(sync=True)
    assert n > 0
    assert np.array_equal(plan.get_selection(), sel)
    assert np.array_equal(plan.get_coefficients(), C)
    plan.rewind(2)
    plan.increment()
    assert np.array_equal(plan.get_set(), S)
    plan.close()


def test_host_injected_failures(B):
    # invalid coefficient (a_min <= 0), an HBM budget that is too small, and a CG iteration
    # cap that cannot be met; all are reported as status codes, nothing faults
    w = W.c1(1)
    bad = W.Problem(kind=W.PDE_1D, n=31, d=4, coef_scale=2.0)
    with pytest.raises(B.UsfftError) as e:
        B.Plan(bad, w.params)
    assert e.value.status == 1
    import dataclasses
    tiny = dataclasses.replace(w.params, hbm_budget_bytes=4096)
    with pytest.raises(B.UsfftError) as e:
        p = B.Plan(w.problem, tiny)
        p.increment()
    assert e.value.status == 2
    w2 = W.small_2d(n=15, d=3, seed=1, N=4, s=10)
    capped = dataclasses.replace(w2.params, max_cg_iters=3)
    p = B.Plan(w2.problem, capped)
    with pytest.raises(B.UsfftError) as e:
        p.increment()
    assert e.value.status == 4
    p.close()
    # the context is still usable afterwards
    p = B.Plan(w.problem, w.params)
    p.increment()
    p.close()


def test_lattice_search_exhaustion_is_elattice(B):
    # full grid [-4,4]^2 (81 candidates at t = 2): with one size (M = 81) and one trial, the draw
    # of seed 3 is not reconstructing on either side (the oracle's search raises as well); the
    # plan reports USFFT_ELATTICE and stays usable
    from oracle import lattice
    prob = W.trigpoly_grid(G=2, d=2, K=4, seed=3)
    J = lattice.candidate_set(np.arange(-4, 5)[:, None], np.arange(-4, 5), N=4)
    with pytest.raises(RuntimeError):
        lattice.search(J, 2, 3, trials=1, max_sizes=1)
    params = W.Params(N=4, s=200, s_local=200, delta=1e-9, delta_is_relative=False, r=1, seed=3,
                      max_lattice_trials=1, max_lattice_sizes=1)
    plan = B.Plan(prob, params)
    plan.increment()
    assert len(plan.get_set()) == 9
    with pytest.raises(B.UsfftError) as e:
        plan.increment()
    assert e.value.status == 3
    plan.close()
    # the same increment with the default search succeeds
    plan = B.Plan(prob, dataclasses.replace(params, max_lattice_trials=64, max_lattice_sizes=400))
    plan.increment()
    plan.increment()
    assert len(plan.get_set()) == 81
    plan.close()


def test_host_deadline_is_etimeout_and_the_increment_can_be_retried(B, monkeypatch):
    # a host deadline of 1 ns around the first wait of a normal increment (2-D 63x63 mesh, fp64:
    # the first wait follows about a millisecond of FE solves, so the device is still busy): the
    # call returns USFFT_ETIMEOUT while the work finishes on the GPU; after a synchronize the same
    # plan runs the increment again and gives the result of a fresh plan
    import torch
    w = W.with_precision(W.c2(1), W.PRECISION_FP64)
    plan = B.Plan(w.problem, w.params)
    monkeypatch.setenv("USFFT_TIMEOUT_S", "1e-9")
    with pytest.raises(B.UsfftError) as e:
        plan.increment()
    assert e.value.status == 5
    monkeypatch.delenv("USFFT_TIMEOUT_S")
    torch.cuda.synchronize()
    info = plan.increment()
    assert info["t"] == 1
    fresh = B.Plan(w.problem, w.params)
    fresh.increment()
    assert np.array_equal(plan.get_set(), fresh.get_set())
    assert np.array_equal(plan.get_coefficients(), fresh.get_coefficients())
    fresh.close()
    plan.close()


def test_autotune_keeps_results_bit_identical(B):
    # the tuned parameters (sampler grid, two-pass FFT tiles) change no result: the replayed step
    # after tuning gives the same coefficients and selection bit for bit, and a later plan of the
    # same shape starts from the tuned grid
    B.usfft_tune_import(None)
    w = W.with_precision(W.small_2d(n=15, d=4, seed=3, N=6, s=30), W.PRECISION_MIXED)
    plan = B.Plan(w.problem, w.params)
    with pytest.raises(B.UsfftError) as e:
        plan.autotune()
    assert e.value.status == 7                    # needs a completed increment
    for _ in range(3):
        plan.increment()
    C, sel, S = plan.get_coefficients(), plan.get_selection(), plan.get_set()
    rep = plan.autotune(reps=2)
    assert rep["sampler_blocks"] > 0 and rep["ms_before"] > 0 and rep["ms_after"] > 0
    assert "1 " in B.usfft_tune_export()
    plan.replay(sync=True)
    assert np.array_equal(plan.get_coefficients(), C) and np.array_equal(plan.get_selection(), sel)
    assert np.array_equal(plan.get_set(), S)
    plan.close()
    # the two-pass FFT (the full grid [-127, 127]^2: M = 69120, beyond the in-place pass): tiles
    # tuned, result unchanged
    prob = W.trigpoly_grid(G=1, d=2, K=127, seed=5)
    params = W.Params(N=127, s=70000, s_local=70000, delta=1e-9, delta_is_relative=False, r=1, seed=4)
    plan = B.Plan(prob, params)
    plan.increment()
    plan.increment()
    C = plan.get_coefficients()
    rep = plan.autotune(reps=2)
    assert rep["fft_final_tile"] > 0
    plan.replay(sync=True)
    assert np.array_equal(plan.get_coefficients(), C)
    plan.close()
    B.usfft_tune_import(None)


def test_increment_after_last_is_a_state_error(B):
    prob = W.trigpoly(G=2, d=2, N=3, seed=1, base_terms=2, node_terms=1, kmax=2, mag_lo=1e-2)
    params = W.Params(N=3, s=10, s_local=10, delta=1e-9, delta_is_relative=False, r=1, seed=1)
    p = B.Plan(prob, params)
    p.increment()
    p.increment()
    with pytest.raises(B.UsfftError) as e:
        p.increment()
    assert e.value.status == 7
    p.close()


def _reconstruct_both(B, prob, params):
    plan = B.Plan(prob, params)
    run = OracleRun(prob, params, keep=True)
    for _ in range(prob.d):
        if run.t > 0:
            plan.resume(run.t, run.I_prefix, run.theta)
        run.increment()
        plan.increment()
    plan.resume(run.t, run.I_prefix, run.theta)
    I_o, z_o, M_o, C_o = run.reconstruct()
    I_g, C_g = plan.reconstruct()
    assert np.array_equal(I_g, I_o)
    z, M = plan.get_lattice()
    assert M == M_o and np.array_equal(z, z_o)
    return plan, I_g, C_g, C_o


def test_reconstruct_trigpoly_coefficients(B):
    prob = W.trigpoly(G=9, d=4, N=5, seed=8, base_terms=5, node_terms=2, kmax=3, mag_lo=1e-4)
    params = W.Params(N=5, s=40, s_local=40, delta=1e-9, delta_is_relative=False, r=1, seed=8)
    plan, I, C, C_o = _reconstruct_both(B, prob, params)
    for g in range(prob.G):
        truth = {tuple(int(v) for v in f): c for f, c in zip(prob.tp_freqs[g], prob.tp_coefs[g]) if c != 0}
        want = np.array([truth.get(tuple(int(v) for v in k), 0.0) for k in I])
        assert np.max(np.abs(C[g] - want)) < 1e-13
    plan.close()


@pytest.mark.parametrize("precision", [W.PRECISION_FP64, W.PRECISION_MIXED])
def test_reconstruct_2d_matches_oracle(B, precision):
    w = W.with_precision(W.small_2d(n=15, d=3, seed=2, N=4, s=20), precision)
    plan, I, C, C_o = _reconstruct_both(B, w.problem, w.params)
    assert C.shape == C_o.shape and len(I) > 0
    assert node_rel(C, C_o) < TOL
    # the device-pointer variant of the copy gives the same numbers
    import torch
    out = torch.empty((w.problem.G, len(I), 2), dtype=torch.float64, device="cuda")
    n = B.ctypes.c_int64(0)
    st = plan._lib.usfft_reconstruct(plan.handle, B.ctypes.byref(n), None, B.ctypes.c_void_p(out.data_ptr()), 1)
    assert st == 0 and n.value == len(I)
    Cd = out.cpu().numpy()
    assert np.max(np.abs((Cd[..., 0] + 1j * Cd[..., 1]) - C)) <= 1e-12 * np.max(np.abs(C))
    plan.close()



def _reconstruct_multiple_both(B, prob, params):
    plan = B.Plan(prob, params)
    run = OracleRun(prob, params, keep=True)
    for _ in range(prob.d):
        if run.t > 0:
            plan.resume(run.t, run.I_prefix, run.theta)
        run.increment()
        plan.increment()
    plan.resume(run.t, run.I_prefix, run.theta)
    I_o, lats, C_o = run.reconstruct_multiple()
    I_g, C_g = plan.reconstruct_multiple()
    assert np.array_equal(I_g, I_o)
    z, M = plan.get_random_lattices()          # step 3's lattices, bit-exact
    assert list(M) == [m for _, m in lats] and all(np.array_equal(z[l], lats[l][0]) for l in range(len(lats)))
    return plan, I_g, C_g, C_o


@pytest.mark.parametrize("precision", [W.PRECISION_FP64, W.PRECISION_MIXED])
def test_reconstruct_multiple_2d_matches_oracle(B, precision):
    # step 3 on multiple rank-1 lattices: every lattice's FE solves, FFTs and gathers, and the pick of
    # each coefficient from its first alias-free lattice, against the oracle element by element
    w = W.with_precision(W.small_2d(n=15, d=3, seed=2, N=4, s=20), precision)
    plan, I, C, C_o = _reconstruct_multiple_both(B, w.problem, w.params)
    assert C.shape == C_o.shape and len(I) > 0
    assert node_rel(C, C_o) < TOL
    _, M = plan.get_random_lattices()
    assert len(M) >= 1 and M[0] >= 2 * (len(I) - 1)
    # the stored reconstruction is this one: evaluate and the errors use it
    Y = np.random.default_rng(5).random((16, w.problem.d))
    assert np.all(np.isfinite(plan.evaluate(Y)))
    # and the single-lattice step 3 afterwards still gives its own result
    I1, C1 = plan.reconstruct()
    assert np.array_equal(I1, I) and C1.shape == C.shape
    plan.close()


@pytest.mark.parametrize("G,seed", [(9, 8), (600, 31)])
def test_reconstruct_multiple_trigpoly_coefficients(B, G, seed):
    # exact recovery (Appendix A): each coefficient of a polynomial supported in I comes out of the
    # first lattice where it is alone; at G = 600 the whole run is the library's alone
    prob = W.trigpoly(G=G, d=4, N=5, seed=seed, base_terms=5, node_terms=2, kmax=3, mag_lo=1e-4)
    params = W.Params(N=5, s=40, s_local=40, delta=1e-9, delta_is_relative=False, r=1, seed=seed)
    if G <= 9:
        plan, I, C, C_o = _reconstruct_multiple_both(B, prob, params)
        assert node_rel(C, C_o) < TOL
    else:
        plan = B.Plan(prob, params)
        for _ in range(prob.d):
            plan.increment()
        I, C = plan.reconstruct_multiple()
        _, M = plan.get_random_lattices()
        assert len(M) >= 2                      # |I| of several hundred needs more than one lattice
    assert len(I) > 0
    for g in range(prob.G):
        truth = {tuple(int(v) for v in f): c for f, c in zip(prob.tp_freqs[g], prob.tp_coefs[g]) if c != 0}
        want = np.array([truth.get(tuple(int(v) for v in k), 0.0) for k in I])
        assert np.max(np.abs(C[g] - want)) < 1e-13
    plan.close()


@pytest.mark.parametrize("precision", [W.PRECISION_FP64, W.PRECISION_MIXED])
def test_tent_and_lognormal_maps_match_oracle(B, precision):
    tent = W.with_map(W.small_2d(n=15, d=4, seed=3, N=5, s=30), W.MAP_TENT, -1.0, 1.0)
    logn = W.small_2d(n=15, d=4, seed=3, N=5, s=30)
    logn = W.with_map(W.Workload(logn.name, W.Problem(kind=W.PDE_2D, n=15, d=4, coef_model=W.COEF_LOGNORMAL_SIN,
                                                      coef_scale=0.5), logn.params), W.MAP_NORMAL, shift=0.0123456789)
    for w in (tent, logn):
        w = W.with_precision(w, precision)
        plan = B.Plan(w.problem, w.params)
        run = OracleRun(w.problem, w.params, keep=True)
        for t in range(1, 4):
            compare_increment(plan, run, f"map {w.problem.theta_map} precision {precision}", exact=False)
        plan.close()


def test_1d_tent_map_full_run_and_even_coefficients(B):
    w = W.with_map(W.c1(3), W.MAP_TENT, -1.0, 1.0)
    plan = B.Plan(w.problem, w.params)
    run = OracleRun(w.problem, w.params, keep=True)
    compare_increment(plan, run, "c1 tent t=1", exact=False)
    # u~ is even about y~ = 1/2 in every coordinate ((A3)): the 1-D coefficients are real and
    # c_k = c_-k -- a property of the library's own output, independent of the oracle
    C = plan.get_coefficients()
    scale = np.max(np.abs(C))
    assert np.max(np.abs(C - C[:, ::-1])) < 1e-13 * scale and np.max(np.abs(C.imag)) < 1e-13 * scale
    for t in range(2, w.problem.d + 1):
        compare_increment(plan, run, f"c1 tent t={t}", exact=False)
    plan.close()


def test_lognormal_map_rejects_a_lattice_node_on_a_pole(B):
    # K = 2N + 1 = 9: the 1-D detection nodes are i/9; Delta = 1/9 puts node 1 on a pole
    prob = W.Problem(kind=W.PDE_1D, n=15, d=2, coef_model=W.COEF_LOGNORMAL_SIN, coef_scale=0.5,
                     theta_map=W.MAP_NORMAL, map_shift=1.0 / 9.0)
    params = W.Params(N=4, s=10, s_local=10, delta=1e-8, delta_is_relative=True, r=1, seed=1)
    plan = B.Plan(prob, params)
    with pytest.raises(B.UsfftError) as e:
        plan.increment()
    assert e.value.status == 1 and "pole" in str(e.value)
    plan.close()
    # an affine coefficient with the unbounded lognormal parameters is refused at plan time
    bad = W.Problem(kind=W.PDE_1D, n=15, d=2, theta_map=W.MAP_NORMAL, map_shift=0.01)
    with pytest.raises(B.UsfftError):
        B.Plan(bad, params)


def compare_random_increment(plan, run, ctx):
    """Increment t = run.t + 1 with random rank-1 lattices on both sides from the oracle's
    state: lattices bit-exact, estimates within TOL per node, sets equal up to near-ties."""
    if run.t > 0:
        plan.resume(run.t, run.I_prefix, run.theta)
    first = len(run.records)
    want = run.increment()
    info = plan.increment()
    got = plan.get_set()
    recs = [r for r in run.records[first:] if r.coupled]
    if recs:
        z, M = plan.get_random_lattices()
        assert np.array_equal(M, np.concatenate([r.M for r in recs])), ctx
        assert np.array_equal(z, np.concatenate([np.array(r.z) for r in recs])), ctx
        assert info["samples"] == int(np.sum(M)) + (2 * run.p.N + 1) * run.p.r
        e = node_rel(plan.get_coefficients(), recs[-1].C)
        assert e < TOL, f"{ctx}: estimate rel err {e:.2e}"
    if not (got.shape == want.shape and np.array_equal(got, want)):
        d = run.prob.d
        amb = near_ties(recs, run.theta, lambda r: run.p.s_local if r.t < d else run.p.s)
        diff = {tuple(r) for r in got.tolist()} ^ {tuple(r) for r in want.tolist()}
        allowed = {tuple(int(v) for v in run.J[k]) for k in amb}
        assert diff <= allowed, f"{ctx}: t={run.t}: {len(diff - allowed)} differences are not near-ties"
    return info


def test_random_lattices_trigpoly_exact_recovery(B):
    d, N, G, seed = 4, 5, 9, 12
    prob = W.trigpoly(G=G, d=d, N=N, seed=seed, base_terms=5, node_terms=2, kmax=3, mag_lo=1e-4)
    params = W.Params(N=N, s=40, s_local=40, delta=1e-9, delta_is_relative=False, r=1, seed=seed,
                      rr_lattices=5, rr_size_factor=4.0)
    plan = B.Plan(prob, params)
    run = OracleRun(prob, params, keep=True)
    union = {tuple(int(v) for v in f) for g in range(G) for f, c in zip(prob.tp_freqs[g], prob.tp_coefs[g]) if c != 0}
    for t in range(1, d + 1):
        compare_random_increment(plan, run, "trigpoly random lattices")
        assert {tuple(int(v) for v in row) for row in plan.get_set()} == {k[:t] for k in union}
    # step 3 keeps the reconstructing lattice: the polynomial's own coefficients
    I, C = plan.reconstruct()
    for g in range(G):
        truth = {tuple(int(v) for v in f): c for f, c in zip(prob.tp_freqs[g], prob.tp_coefs[g]) if c != 0}
        assert np.max(np.abs(C[g] - np.array([truth.get(tuple(int(v) for v in k), 0.0) for k in I]))) < 1e-13
    plan.close()


@pytest.mark.parametrize("precision", [W.PRECISION_FP64, W.PRECISION_MIXED])
def test_random_lattices_pde_match_oracle(B, precision):
    for w in (W.c1(2), W.small_2d(n=15, d=4, seed=2, N=6, s=30, r=2)):
        w = W.with_precision(w, precision)
        w = W.Workload(w.name, w.problem, dataclasses.replace(w.params, rr_lattices=5, rr_size_factor=2.0))
        plan = B.Plan(w.problem, w.params)
        run = OracleRun(w.problem, w.params, keep=True)
        for t in range(1, min(w.problem.d, 4) + 1):
            compare_random_increment(plan, run, f"{w.name} random lattices precision {precision}")
        # replay of a random-lattice step reproduces its estimate
        C = plan.get_coefficients()
        plan.replay()
        assert np.array_equal(plan.get_coefficients(), C)
        plan.close()
