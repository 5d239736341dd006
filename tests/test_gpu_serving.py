"""The batched and served forms on the GPU: usfft_increment_many over several plans (each on
its own stream) gives every plan exactly the result it gives alone, and a continuous-batching
run of a small request stream returns, per request, the same detected sets and coefficients
as the requests run one at a time."""
import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def B():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    from paper_2109_04131_gb300 import binding
    binding.load_library()
    return binding


def _instances():
    # shapes that launch the same kernels with different shared-memory sizes at the same time
    # (selection over different |J|, FFTs of different lengths, samplers of different meshes)
    return [W.with_precision(W.small_2d(n=15, d=4, seed=2, N=5, s=30), W.PRECISION_MIXED),
            W.with_precision(W.small_2d(n=31, d=3, seed=3, N=4, s=20), W.PRECISION_FP64),
            W.c1(2),
            W.with_precision(W.small_2d(n=70, d=3, seed=4, N=3, s=10), W.PRECISION_MIXED),
            W.with_precision(W.small_2d(n=40, d=4, seed=5, N=8, s=40), W.PRECISION_MIXED),
            W.with_precision(W.small_2d(n=24, d=3, seed=6, N=12, s=60), W.PRECISION_MIXED),
            W.c1(5),
            W.with_precision(W.small_2d(n=9, d=5, seed=7, N=6, s=25), W.PRECISION_FP64)]


def _plan(B, w):
    import torch
    return B.Plan(w.problem, w.params, stream=torch.cuda.Stream().cuda_stream)


def test_increment_many_equals_alone(B):
    ws = _instances()
    together = [_plan(B, w) for w in ws]
    for _ in range(3):
        infos, sts = B.usfft_increment_many(together)
        assert sts == [0] * len(ws) and all(i["samples"] > 0 for i in infos)
    for w, pt in zip(ws, together):
        alone = B.Plan(w.problem, w.params)
        for _ in range(3):
            alone.increment()
        assert np.array_equal(pt.get_set(), alone.get_set())
        assert np.array_equal(pt.get_coefficients(), alone.get_coefficients())
        assert pt.bytes() > 0
        alone.close()
    with pytest.raises(B.UsfftError):
        B.usfft_increment_many([together[0], together[0]])
    for p in together:
        p.close()


def test_served_results_equal_one_at_a_time(B):
    from paper_2109_04131_gb300 import serving
    ws = _instances()
    # even requests run all d increments and step 3, odd ones two increments
    reqs = [serving.Request(k, 0.0, w, w.problem.d if k % 2 == 0 else 2, 256 << 20, reconstruct=(k % 2 == 0))
            for k, w in enumerate(ws)]

    def make_plan(r):
        return _plan(B, r.workload)

    def collect(inst):
        return inst.plan.get_set(), inst.plan.get_coefficients()

    srv = serving.Server(budget_bytes=8 << 30, make_plan=make_plan, increment_many=B.usfft_increment_many,
                         collect=collect)
    rep = srv.run(reqs)
    assert rep["requests"] == len(ws) and rep["failed"] == 0 and rep["peak_active"] >= 2
    alone = serving.run_one_at_a_time(reqs, make_plan, collect=collect)
    for inst in rep["instances"]:
        s1, c1 = inst.result
        s2, c2 = alone["results"][inst.req.rid]
        assert np.array_equal(s1, s2) and np.array_equal(c1, c2)
    assert rep["lattice_samples"] == alone["lattice_samples"]


def test_async_served_results_equal_one_at_a_time(B):
    from paper_2109_04131_gb300 import serving
    ws = _instances()
    reqs = [serving.Request(k, 0.0005 * k, w, w.problem.d if k % 2 == 0 else 2, 256 << 20,
                            reconstruct=(k % 2 == 0)) for k, w in enumerate(ws)]

    def make_plan(r):
        return _plan(B, r.workload)

    def collect(inst):
        return inst.plan.get_set(), inst.plan.get_coefficients()

    rep = serving.AsyncServer(budget_bytes=8 << 30, make_plan=make_plan, max_active=5, collect=collect).run(reqs)
    assert rep["requests"] == len(ws) and rep["failed"] == 0 and 2 <= rep["peak_active"] <= 5
    alone = serving.run_one_at_a_time(reqs, make_plan, collect=collect)
    for inst in rep["instances"]:
        s1, c1 = inst.result
        s2, c2 = alone["results"][inst.req.rid]
        assert np.array_equal(s1, s2) and np.array_equal(c1, c2)
