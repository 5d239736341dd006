"""usfft_sample_2d_static: the sampler variant for callers that cannot allocate device memory.

Such callers (a plug-in inside a framework that owns all of HBM, a loop that must never enter
the allocator) hand the library their own output buffer; the library's scratch lives in a
fixed static device array.  The tests call the entry point through the C ABI: twice in a row
against the samples usfft_increment produced for the same lattice nodes, with the device's
free memory unchanged across the second call; an empty call (the set-up call a caller makes
before reserving its pool); the largest problem the static scratch serves (n = 63, d = 64)
against the oracle's FE solves; and the size checks.  This file is collected last so that a
stop at its failure has run everything else."""
import numpy as np
import pytest

import workloads as W

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


def test_static_scratch_sampler_matches_increment_samples(B):
    import torch
    w = W.with_precision(W.small_2d(n=31, d=5, seed=4, N=5, s=30), W.PRECISION_MIXED)
    stream = torch.cuda.current_stream().cuda_stream
    # an empty call sets the static scratch up on this device and launches nothing
    U0 = torch.empty(1, dtype=torch.float64, device="cuda")
    assert B.usfft_sample_2d_static(w.problem, np.full(w.problem.d, -1), np.zeros(w.problem.d), 8, 0, 0,
                                    U0.data_ptr(), stream) == 0
    plan = B.Plan(w.problem, w.params)
    plan.increment()
    info = plan.increment()                      # coupled step t = 2, one detection iteration
    t = info["t"]
    z, M = plan.get_lattice()
    U_plan = plan.get_samples()                  # samples of the last detection iteration (i = 1)
    assert U_plan.shape == (M, w.problem.G)
    d = w.problem.d
    zfull = np.full(d, -1, dtype=np.int64)
    zfull[:t] = z
    tails = np.zeros(d)
    for j in range(t + 1, d + 1):
        tails[j - 1] = B.usfft_draw_uniform(w.params.seed, 2, t, 1, j)   # phase 2: tails of the coupled step
    scale = np.max(np.abs(U_plan))
    # first call: every lattice node
    U1 = torch.empty((M, w.problem.G), dtype=torch.float64, device="cuda")
    unc = B.usfft_sample_2d_static(w.problem, zfull, tails, M, 0, M, U1.data_ptr(), stream)
    assert unc == 0
    assert np.max(np.abs(U1.cpu().numpy() - U_plan)) <= TOL * scale
    # second call right after it: a sub-range of the nodes into another buffer; the device's
    # free memory is the same before and after the call (the library allocated nothing)
    i0, cnt = M // 3, M // 2
    U2 = torch.full((cnt, w.problem.G), float("nan"), dtype=torch.float64, device="cuda")
    torch.cuda.synchronize()
    free_before = torch.cuda.mem_get_info()[0]
    unc = B.usfft_sample_2d_static(w.problem, zfull, tails, M, i0, cnt, U2.data_ptr(), stream)
    torch.cuda.synchronize()
    free_after = torch.cuda.mem_get_info()[0]
    assert unc == 0
    assert free_after == free_before
    assert np.max(np.abs(U2.cpu().numpy() - U_plan[i0:i0 + cnt])) <= TOL * scale
    plan.close()


def test_static_scratch_serves_the_largest_problem(B):
    # n = 63, d = 64 (the largest the static scratch serves): three lattice nodes against the
    # oracle's banded FE solves
    import torch
    from oracle import fe
    from oracle.usfft import NodeSet, sample_rows
    prob = W.Problem(kind=W.PDE_2D, n=63, d=64)
    M = 97
    zfull = np.full(64, -1, dtype=np.int64)
    zfull[:3] = [1, 22, 41]
    tails = np.random.default_rng(5).random(64)
    rows = np.array([0, 13, 96])
    U = torch.empty((3, prob.G), dtype=torch.float64, device="cuda")
    for k, i in enumerate(rows):       # one node per call, into its own row of the caller's buffer
        assert B.usfft_sample_2d_static(prob, zfull, tails, M, int(i), 1, U[k].data_ptr()) == 0
    nodes = NodeSet(64, [0, 1, 2], zfull[:3], M, {j: float(tails[j]) for j in range(3, 64)})
    Uo = sample_rows(prob, nodes, rows, fe.make_mesh(prob.kind, prob.n))
    assert np.max(np.abs(U.cpu().numpy() - Uo)) <= TOL * np.max(np.abs(Uo))


def test_static_scratch_sampler_rejects_sizes_beyond_its_limits(B):
    import torch
    U = torch.empty(16, dtype=torch.float64, device="cuda")
    big = W.Problem(kind=W.PDE_2D, n=127, d=20)
    with pytest.raises(B.UsfftError) as e:
        B.usfft_sample_2d_static(big, np.full(20, -1), np.zeros(20), 8, 0, 1, U.data_ptr())
    assert e.value.status == 1 and "n must lie" in str(e.value)
    ok = W.Problem(kind=W.PDE_2D, n=7, d=2)
    with pytest.raises(B.UsfftError):
        B.usfft_sample_2d_static(ok, np.array([1, 9]), np.zeros(2), 8, 0, 1, U.data_ptr())   # z_j >= M
    with pytest.raises(B.UsfftError):
        B.usfft_sample_2d_static(ok, np.array([1, 3]), np.zeros(2), 8, 6, 3, U.data_ptr())   # i0 + count > M
