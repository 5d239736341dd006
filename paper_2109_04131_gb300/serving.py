"""Continuous batching of usFFT instances (the served form).

Requests arrive over time; each asks for a number of dimension increments of one problem
instance (and optionally step 3).  The server keeps the admitted instances' plans resident on
the device and, round after round, runs one increment of every admitted instance at once
(`usfft_increment_many`: host planning in parallel threads, device work overlapping on the
plans' own streams).  Arrivals are admitted between rounds while the device bytes of the
resident plans plus the arrival's reservation stay within the HBM budget; an instance leaves
as soon as its last increment (and step 3) is done, so new requests join a running batch
instead of waiting for it to drain.

Everything numeric runs in the library; this module only schedules.  Its clock, plan factory
and batch executor are injectable, so the scheduling logic is tested on the CPU with fakes.
"""
from __future__ import annotations

import time
from dataclasses import dataclass, field
from typing import Callable, List, Optional


@dataclass
class Request:
    rid: int
    arrival: float                 # seconds after the start of the run
    workload: object               # workloads.Workload
    increments: int                # dimension increments to run (<= d)
    reserve_bytes: int             # device bytes reserved at admission (the plan grows into them)
    reconstruct: bool = False      # run step 3 after the last increment


@dataclass
class Instance:
    req: Request
    plan: object
    admitted: float
    done_increments: int = 0
    samples: int = 0
    increment_latency: List[float] = field(default_factory=list)
    finished: Optional[float] = None
    status: int = 0
    result: object = None          # (detected set, coefficients of the last step or of step 3)


def percentile(xs, q):
    if not xs:
        return None
    s = sorted(xs)
    k = (len(s) - 1) * q / 100.0
    lo, hi = int(k), min(int(k) + 1, len(s) - 1)
    return s[lo] + (s[hi] - s[lo]) * (k - lo)


class Server:
    def __init__(self, budget_bytes: int, make_plan: Callable, increment_many: Callable,
                 max_active: int = 64, clock: Callable = time.perf_counter, sleep: Callable = time.sleep,
                 collect: Optional[Callable] = None):
        self.budget = int(budget_bytes)
        self.make_plan = make_plan
        self.increment_many = increment_many
        self.max_active = max_active
        self.clock = clock
        self.sleep = sleep
        self.collect = collect        # collect(instance) -> result kept on the instance (may be None)

    def _held(self, active):
        return sum(max(int(i.plan.bytes()), i.req.reserve_bytes) for i in active)

    def run(self, requests: List[Request]) -> dict:
        pending = sorted(requests, key=lambda r: (r.arrival, r.rid))
        active: List[Instance] = []
        done: List[Instance] = []
        rounds = 0
        t0 = self.clock()
        peak_active = 0
        peak_bytes = 0
        while pending or active:
            now = self.clock() - t0
            # admission, in arrival order (no overtaking: a large request blocks smaller ones)
            while (pending and pending[0].arrival <= now and len(active) < self.max_active
                   and self._held(active) + pending[0].reserve_bytes <= self.budget):
                r = pending.pop(0)
                active.append(Instance(r, self.make_plan(r), admitted=self.clock() - t0))
            if pending and not active and pending[0].reserve_bytes > self.budget:
                raise ValueError(f"request {pending[0].rid} reserves more than the whole budget")
            if not active:
                self.sleep(max(0.0, pending[0].arrival - (self.clock() - t0)))
                continue
            peak_active = max(peak_active, len(active))
            t_round = self.clock() - t0
            infos, statuses = self.increment_many([i.plan for i in active])
            t_end = self.clock() - t0
            rounds += 1
            still = []
            for inst, info, st in zip(active, infos, statuses):
                inst.increment_latency.append(t_end - t_round)
                inst.samples += int(info["samples"]) if st == 0 else 0
                inst.done_increments += 1
                if st != 0:
                    inst.status = st
                if st != 0 or inst.done_increments >= inst.req.increments:
                    if st == 0 and inst.req.reconstruct:
                        inst.plan.reconstruct()
                    inst.finished = self.clock() - t0
                    if self.collect is not None:
                        inst.result = self.collect(inst)
                    peak_bytes = max(peak_bytes, self._held(active))
                    inst.plan.close()
                    done.append(inst)
                else:
                    still.append(inst)
            peak_bytes = max(peak_bytes, self._held(still)) if still else peak_bytes
            active = still
        wall = self.clock() - t0
        inc_lat = [x for i in done for x in i.increment_latency]
        inst_lat = [i.finished - i.req.arrival for i in done]
        samples = sum(i.samples for i in done)
        return {
            "requests": len(done), "failed": sum(1 for i in done if i.status != 0), "rounds": rounds,
            "wall_s": wall, "lattice_samples": samples, "samples_per_s": samples / wall if wall > 0 else None,
            "increment_latency_ms": {"p50": 1e3 * percentile(inc_lat, 50), "p99": 1e3 * percentile(inc_lat, 99)},
            "instance_latency_ms": {"p50": 1e3 * percentile(inst_lat, 50), "p99": 1e3 * percentile(inst_lat, 99)},
            "peak_active": peak_active, "peak_bytes": peak_bytes, "instances": done,
        }


class AsyncServer:
    """Continuous batching without a round barrier: every admitted instance runs its increments
    back to back in a worker thread of its own (the library call releases the interpreter, so
    the host planning of the instances runs in parallel and their device work overlaps on the
    plans' streams); a finished instance frees its place and bytes for the next arrival at once.
    Admission as in Server: arrival order, within the budget and at most max_active at a time."""

    def __init__(self, budget_bytes: int, make_plan: Callable, max_active: int = 64,
                 clock: Callable = time.perf_counter, collect: Optional[Callable] = None):
        self.budget = int(budget_bytes)
        self.make_plan = make_plan
        self.max_active = max_active
        self.clock = clock
        self.collect = collect

    def run(self, requests: List[Request]) -> dict:
        import threading
        pending = sorted(requests, key=lambda r: (r.arrival, r.rid))
        lock = threading.Condition()
        active: List[Instance] = []
        done: List[Instance] = []
        t0 = self.clock()
        peak = {"active": 0, "bytes": 0}

        def held():
            return sum(max(int(i.plan.bytes()), i.req.reserve_bytes) for i in active)

        def work(inst: Instance):
            for _ in range(inst.req.increments):
                t1 = self.clock()
                try:
                    info = inst.plan.increment()
                    inst.samples += int(info["samples"])
                except Exception as exc:          # the library's status, as an exception
                    inst.status = getattr(exc, "status", -1)
                    break
                finally:
                    inst.increment_latency.append(self.clock() - t1)
                    inst.done_increments += 1
            if inst.status == 0 and inst.req.reconstruct:
                inst.plan.reconstruct()
            inst.finished = self.clock() - t0
            if self.collect is not None:
                inst.result = self.collect(inst)
            with lock:
                peak["bytes"] = max(peak["bytes"], held())
                inst.plan.close()
                active.remove(inst)
                done.append(inst)
                lock.notify_all()

        threads = []
        with lock:
            while pending or active:
                now = self.clock() - t0
                while (pending and pending[0].arrival <= now and len(active) < self.max_active
                       and held() + pending[0].reserve_bytes <= self.budget):
                    r = pending.pop(0)
                    inst = Instance(r, self.make_plan(r), admitted=self.clock() - t0)
                    active.append(inst)
                    peak["active"] = max(peak["active"], len(active))
                    th = threading.Thread(target=work, args=(inst,), daemon=True)
                    threads.append(th)
                    th.start()
                if pending and not active and pending[0].reserve_bytes > self.budget:
                    raise ValueError(f"request {pending[0].rid} reserves more than the whole budget")
                wait = None
                if pending and pending[0].arrival > now:
                    wait = pending[0].arrival - now
                if active or wait is not None:
                    lock.wait(timeout=wait if wait is not None else 1.0)
        for th in threads:
            th.join()
        wall = self.clock() - t0
        inc_lat = [x for i in done for x in i.increment_latency]
        inst_lat = [i.finished - i.req.arrival for i in done]
        samples = sum(i.samples for i in done)
        return {
            "requests": len(done), "failed": sum(1 for i in done if i.status != 0), "rounds": None,
            "wall_s": wall, "lattice_samples": samples, "samples_per_s": samples / wall if wall > 0 else None,
            "increment_latency_ms": {"p50": 1e3 * percentile(inc_lat, 50), "p99": 1e3 * percentile(inc_lat, 99)},
            "instance_latency_ms": {"p50": 1e3 * percentile(inst_lat, 50), "p99": 1e3 * percentile(inst_lat, 99)},
            "peak_active": peak["active"], "peak_bytes": peak["bytes"], "instances": done,
        }


def run_one_at_a_time(requests: List[Request], make_plan: Callable, collect: Optional[Callable] = None,
                      clock: Callable = time.perf_counter) -> dict:
    """The requests in arrival order, each run alone to completion (no batching, no overlap)."""
    t0 = clock()
    samples = 0
    inst_ms = []
    results = {}
    for r in sorted(requests, key=lambda r: (r.arrival, r.rid)):
        t1 = clock()
        plan = make_plan(r)
        for _ in range(r.increments):
            samples += int(plan.increment()["samples"])
        if r.reconstruct:
            plan.reconstruct()
        inst = Instance(r, plan, admitted=0.0)
        if collect is not None:
            results[r.rid] = collect(inst)
        plan.close()
        inst_ms.append(1e3 * (clock() - t1))
    wall = clock() - t0
    return {"requests": len(requests), "wall_s": wall, "lattice_samples": samples,
            "samples_per_s": samples / wall if wall > 0 else None,
            "instance_compute_ms": {"p50": percentile(inst_ms, 50), "p99": percentile(inst_ms, 99)},
            "results": results}
