"""The continuous-batching scheduler (paper_2109_04131_gb300.serving) on the CPU with fake plans:
admission within the HBM budget and in arrival order, arrivals joining a running batch, the
latency bookkeeping and the failure path.  No GPU, no library."""
import pytest

from paper_2109_04131_gb300 import serving


class FakeClock:
    def __init__(self):
        self.t = 0.0

    def __call__(self):
        return self.t

    def sleep(self, dt):
        self.t += max(dt, 1e-6)


class FakePlan:
    def __init__(self, req, log, grow):
        self.req, self.log, self.grow = req, log, grow
        self.n = 0
        self.closed = False

    def bytes(self):
        return self.grow * self.n

    def increment(self):
        self.n += 1
        return {"samples": 10}

    def reconstruct(self):
        self.log.append(("recon", self.req.rid))

    def close(self):
        self.closed = True
        self.log.append(("close", self.req.rid))


def make(clock, log, grow=0, fail_rid=None, round_time=1.0):
    def make_plan(r):
        log.append(("admit", r.rid, clock()))
        return FakePlan(r, log, grow)

    def inc_many(plans):
        held = sum(max(p.bytes(), p.req.reserve_bytes) for p in plans)
        log.append(("round", tuple(p.req.rid for p in plans), held))
        clock.t += round_time
        infos, sts = [], []
        for p in plans:
            infos.append(p.increment())
            sts.append(4 if p.req.rid == fail_rid else 0)
        return infos, sts
    return make_plan, inc_many


def req(rid, arrival, inc, reserve, recon=False):
    return serving.Request(rid, arrival, None, inc, reserve, recon)


def test_budget_order_and_continuous_batching():
    clock, log = FakeClock(), []
    mk, inc = make(clock, log)
    srv = serving.Server(budget_bytes=100, make_plan=mk, increment_many=inc, clock=clock, sleep=clock.sleep)
    reqs = [req(0, 0.0, 3, 50), req(1, 0.0, 1, 30), req(2, 0.5, 2, 50), req(3, 0.6, 1, 10)]
    rep = srv.run(reqs)
    assert rep["requests"] == 4 and rep["failed"] == 0
    rounds = [e for e in log if e[0] == "round"]
    assert all(e[2] <= 100 for e in rounds)                        # never above the budget
    # the first scheduling round runs 0 and 1; request 2 (50) waits for 1 to leave, then joins 0's batch
    assert rounds[0][1] == (0, 1)
    assert rounds[1][1] == (0, 2)
    admits = [e for e in log if e[0] == "admit"]
    assert [a[1] for a in admits] == [0, 1, 2, 3]                   # arrival order, no overtaking
    assert rep["lattice_samples"] == 10 * (3 + 1 + 2 + 1)
    inst = {i.req.rid: i for i in rep["instances"]}
    assert inst[0].increment_latency == [1.0, 1.0, 1.0]
    assert inst[1].finished - inst[1].req.arrival == pytest.approx(1.0)
    assert all(("close", r) in log for r in range(4))


def test_plans_growing_into_their_reservation_and_beyond():
    clock, log = FakeClock(), []
    mk, inc = make(clock, log, grow=40)                             # 40 bytes more per increment
    srv = serving.Server(budget_bytes=100, make_plan=mk, increment_many=inc, clock=clock, sleep=clock.sleep)
    rep = srv.run([req(0, 0.0, 3, 10), req(1, 0.0, 3, 10)])
    rounds = [e for e in log if e[0] == "round"]
    # after the first round each plan holds 40 > its reservation: the held bytes are what they hold
    assert rounds[0][2] == 20 and rep["peak_bytes"] >= 80


def test_failure_and_reconstruct_and_oversize():
    clock, log = FakeClock(), []
    mk, inc = make(clock, log, fail_rid=1)
    srv = serving.Server(budget_bytes=100, make_plan=mk, increment_many=inc, clock=clock, sleep=clock.sleep)
    rep = srv.run([req(0, 0.0, 2, 10, recon=True), req(1, 0.0, 5, 10, recon=True)])
    inst = {i.req.rid: i for i in rep["instances"]}
    assert inst[1].status == 4 and inst[1].done_increments == 1     # leaves at its failure
    assert ("recon", 0) in log and ("recon", 1) not in log
    assert rep["failed"] == 1
    with pytest.raises(ValueError):
        serving.Server(budget_bytes=5, make_plan=mk, increment_many=inc, clock=clock,
                       sleep=clock.sleep).run([req(9, 0.0, 1, 6)])


def test_idle_server_waits_for_arrivals():
    clock, log = FakeClock(), []
    mk, inc = make(clock, log)
    srv = serving.Server(budget_bytes=100, make_plan=mk, increment_many=inc, clock=clock, sleep=clock.sleep)
    rep = srv.run([req(0, 5.0, 1, 10)])
    admit = [e for e in log if e[0] == "admit"][0]
    assert admit[2] >= 5.0 and rep["wall_s"] >= 6.0


def test_workload_generators_are_seeded_and_shaped():
    import workloads as W
    a = W.serving_requests(50, rate=200.0, seed=7)
    b = W.serving_requests(50, rate=200.0, seed=7)
    assert [x[0] for x in a] == [x[0] for x in b]
    assert all(x2[0] > x1[0] for x1, x2 in zip(a, a[1:]))
    kinds = {x[1].problem.kind for x in a}
    assert kinds == {W.PDE_1D, W.PDE_2D}
    for t, w, inc, res in a:
        if w.problem.kind == W.PDE_2D:
            assert w.problem.n == 127 and w.problem.d == 20 and inc == 2
        else:
            assert w.problem.n == 255 and 4 <= w.problem.d <= 20 and inc == w.problem.d
    bi = W.batch_instances(64, seed=42)
    assert len(bi) == 64 and all(5 <= w.problem.d <= 30 and 31 <= w.problem.n <= 127 for w, _ in bi)


def test_async_server_admission_and_completion():
    import threading
    import time as _t
    log = []
    lock = threading.Lock()

    class P(FakePlan):
        def increment(self):
            _t.sleep(0.002 * (1 + self.req.rid % 3))
            return super().increment()

    def make_plan(r):
        with lock:
            log.append(("admit", r.rid))
        return P(r, log, 0)

    srv = serving.AsyncServer(budget_bytes=100, make_plan=make_plan, max_active=3)
    reqs = [req(k, 0.001 * k, 2 + k % 3, 30) for k in range(10)]
    rep = srv.run(reqs)
    assert rep["requests"] == 10 and rep["failed"] == 0 and rep["peak_active"] <= 3
    assert [e[1] for e in log if e[0] == "admit"] == list(range(10))
    assert rep["lattice_samples"] == 10 * sum(2 + k % 3 for k in range(10))
    assert all(len(i.increment_latency) == i.req.increments for i in rep["instances"])
