"""The sharded form of a coupled step (one instance over P ranks; usfft_increment_sharded).

CPU (no GPU): the lattice rule with sizes that are multiples of P is bit-exact with the oracle's;
two gloo ranks run the partition and exchange protocol of the sharded step with the product's
collective hook (paper_2109_04131_gb300.sharded.TorchAllreduce, called through its C function
pointer as the library calls it): each rank contributes the partial DFT of its residue class of
lattice nodes (the oracle's samples and partial sums standing in for the rank's kernels), the sum
over ranks is the oracle's full DFT, and the maximum over ranks of the per-block selection flags
is the oracle's union over all mesh nodes.

GPU: the library's sharded increments with P = 2 and 3 ranks emulated as host threads, each with
its own plan and stream on the one GPU, joined by a host-side all-reduce (the kernels never wait
for each other; the threads meet only between launches): lattice, candidates and DFT indices
bit-exact with the oracle under the same rule, coefficients within 1e-10 per node, detected sets
equal up to near-ties (bit-exact for trigonometric polynomials) and the same on every rank; a
failing hook is reported as USFFT_ECOMM."""
import ctypes
import os
import socket
import sys
import threading

import numpy as np
import pytest
import torch.multiprocessing as mp

import workloads as W
from oracle import detect, dft, lattice, rng
from oracle.usfft import NodeSet, OracleRun, sample_rows

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
TOL = 1e-10


@pytest.fixture(scope="module")
def binding():
    from paper_2109_04131_gb300 import binding as b
    b.load_library()
    return b


def test_lattice_rule_with_rank_divisor_is_bit_exact_with_the_oracle(binding):
    r = np.random.default_rng(3)
    for P in (1, 2, 3, 4, 5, 6, 7, 8):
        for t in (2, 3):
            prev = np.unique(r.integers(-4, 5, size=(int(r.integers(5, 60)), t - 1)), axis=0)
            J = lattice.candidate_set(prev, np.arange(-3, 4), N=6)
            z0, M0 = lattice.search(J, t, 11, divisor=P)
            z1, M1 = binding.usfft_search_lattice_multiple(J, t, 11, P)
            assert M0 == M1 and M1 % P == 0 and np.array_equal(z0, z1), (P, t)
            assert lattice.is_reconstructing(J, z1, M1)
    J = lattice.candidate_set(np.arange(-2, 3)[:, None], np.arange(-2, 3), N=3)
    for bad in (0, 11, 65):
        with pytest.raises(binding.UsfftError) as e:
            binding.usfft_search_lattice_multiple(J, 2, 1, bad)
        assert e.value.status == 1


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    from paper_2109_04131_gb300 import binding as B
    from paper_2109_04131_gb300 import sharded
    B.load_library()
    import datetime
    dist.init_process_group("gloo", rank=rank, world_size=world, timeout=datetime.timedelta(seconds=120))
    try:
        hook = sharded.TorchAllreduce(on_device=False)
        w = W.small_2d(n=7, d=3, seed=2, N=3, s=8)
        prob, p = w.problem, w.params
        run = OracleRun(prob, p, lattice_divisor=world)
        run.increment()
        t = 2
        run.detect_1d(t)
        J = lattice.candidate_set(run.I_prefix, np.array(run.I1d[t], dtype=np.int64), p.N)
        z, M = B.usfft_search_lattice_multiple(J, t, p.seed, world)          # the library's rule
        zo, Mo = lattice.search(J, t, p.seed, divisor=world)
        assert M == Mo and np.array_equal(z, zo) and M % world == 0
        m = lattice.lattice_indices(J, z, M)
        tails = {j - 1: rng.uniform(p.seed, rng.PHASE_TAIL, t, 1, j) for j in range(t + 1, prob.d + 1)}
        nodes = NodeSet(prob.d, list(range(t)), z, M, tails)
        # this rank's residue class of lattice nodes and its partial coefficients
        rows = np.arange(rank, M, world)
        Cp = dft.partial_coefficients(sample_rows(prob, nodes, rows, run.mesh), rows, m, M)
        buf = np.ascontiguousarray(np.stack([Cp.real, Cp.imag], axis=-1))
        fn = ctypes.cast(hook.fn, ctypes.c_void_p).value
        call = B.ALLREDUCE_FN(fn)
        assert call(buf.ctypes.data, buf.size, B.RED_F64, B.RED_SUM, None, None) == 0
        C = buf[..., 0] + 1j * buf[..., 1]
        # selection at this rank's block of mesh nodes, union by a maximum over the ranks
        G = prob.G
        g0, g1 = G * rank // world, G * (rank + 1) // world
        flags = np.zeros(len(J), dtype=np.uint8)
        for g in range(g0, g1):
            flags[detect.select(C[g], run.theta, p.s_local)] = 1
        assert call(flags.ctypes.data, flags.size, B.RED_U8, B.RED_MAX, None, None) == 0
        # the unsharded oracle step
        U = sample_rows(prob, nodes, np.arange(M), run.mesh)
        Co = dft.coefficients(U, m, M)
        union = detect.union_over_nodes(Co, run.theta, p.s_local, set())
        den = np.max(np.abs(Co), axis=1)
        err = float(np.max(np.max(np.abs(C - Co), axis=1) / np.where(den == 0, 1.0, den)))
        out.put((rank, err, sorted(np.nonzero(flags)[0].tolist()), sorted(union), hook.failures,
                 C.tobytes()))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_run_the_sharded_exchange():
    world = 2
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, out)) for r in range(world)]
    for p in procs:
        p.start()
    # drain the queue before joining: a rank cannot exit while its result is still in the pipe
    res = []
    try:
        for _ in range(world):
            res.append(out.get(timeout=300))
    finally:
        for p in procs:
            p.join(timeout=60)
            if p.exitcode is None:
                p.kill()
    assert all(p.exitcode == 0 for p in procs), [p.exitcode for p in procs]
    res = sorted(res)
    for rank, err, flags, union, failures, _ in res:
        assert failures == 0
        assert err < 1e-12, (rank, err)
        assert flags == union and len(union) > 0
    assert res[0][5] == res[1][5]        # every rank holds the same summed coefficients


# ---------------------------------------------------------------------------------------------
# GPU: the library's sharded increments, P ranks as host threads on one GPU
# ---------------------------------------------------------------------------------------------
class ThreadAllreduce:
    """All-reduce over P host threads (one per emulated rank): each thread copies its device buffer
    to the host on its plan's stream, the threads meet at a barrier, every thread forms the same
    sum (rank order) or maximum and copies it back on its stream."""

    def __init__(self, P, binding):
        self.P = P
        self.B = binding
        self.barrier = threading.Barrier(P, timeout=300)
        self.slots = [None] * P
        self.fns = [binding.ALLREDUCE_FN(self._make(r)) for r in range(P)]
        self.calls = 0

    def _make(self, rank):
        def call(buf, count, dtype, op, stream, ctx):
            try:
                return exchange(buf, count, dtype, op, stream)
            except Exception:            # noqa: BLE001 - a broken barrier is a failed collective
                self.barrier.abort()
                return 1

        def exchange(buf, count, dtype, op, stream):
            import torch
            from paper_2109_04131_gb300.sharded import _DeviceBuffer, _TYPESTR
            t = torch.as_tensor(_DeviceBuffer(buf, count, _TYPESTR[dtype]), device="cuda")
            s = torch.cuda.ExternalStream(stream) if stream else torch.cuda.default_stream()
            with torch.cuda.stream(s):
                host = t.cpu().numpy().copy()
            self.slots[rank] = host
            self.barrier.wait()
            if op == self.B.RED_SUM:
                tot = self.slots[0].copy()
                for x in self.slots[1:]:
                    tot = tot + x
            else:
                tot = np.maximum.reduce(self.slots)
            self.barrier.wait()
            with torch.cuda.stream(s):
                t.copy_(torch.from_numpy(tot))
            s.synchronize()
            if rank == 0:
                self.calls += 1
            return 0
        return call


def _run_ranks(B, w, P, increments, states=None):
    """Run `increments` sharded increments on P plans in P threads.  states (optional): for each
    increment the state (t, I^(1..t), theta) every rank resumes from before it (t = 0: none)."""
    import torch
    plans = [B.Plan(w.problem, w.params, stream=torch.cuda.Stream().cuda_stream) for _ in range(P)]
    red = ThreadAllreduce(P, B)
    results = [[None] * increments for _ in range(P)]
    errors = []

    def worker(rank):
        try:
            for k in range(increments):
                if states is not None and states[k][0] > 0:
                    plans[rank].resume(*states[k])
                info = B.usfft_increment_sharded(plans[rank], rank, P, red.fns[rank])
                results[rank][k] = (info, plans[rank].get_set(), plans[rank].get_lattice(),
                                    plans[rank].get_candidates(), plans[rank].get_coefficients())
        except Exception as e:       # noqa: BLE001 - reported below
            errors.append((rank, repr(e)))
            red.barrier.abort()

    threads = [threading.Thread(target=worker, args=(r,)) for r in range(P)]
    for th in threads:
        th.start()
    for th in threads:
        th.join(timeout=600)
    assert not errors, errors
    return plans, results, red


def near_ties(records, theta, s_tilde_of, rel=2e-10):
    """Candidate positions whose oracle magnitude lies within rel * max_k |C_g| of the threshold
    or of the node's s~-th largest magnitude: the only places where rounding may decide the
    selection (the summed coefficients differ from the oracle's at the rounding level)."""
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
                amb.update(np.nonzero(np.abs(mg - elig[s_t - 1]) <= tol)[0].tolist())
    return amb


def _node_rel(Cg, Co):
    den = np.max(np.abs(Co), axis=1)
    den[den == 0] = 1.0
    return float(np.max(np.max(np.abs(Cg - Co), axis=1) / den))


@pytest.mark.gpu
@pytest.mark.parametrize("P", [2, 3])
def test_sharded_increments_match_the_oracle(binding, P):
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    for w in (W.with_precision(W.small_2d(n=15, d=4, seed=2, N=6, s=30), W.PRECISION_MIXED),
              W.with_precision(W.small_2d(n=15, d=4, seed=5, N=6, s=30, r=2), W.PRECISION_FP64)):
        incs = 3
        # the oracle first; every sharded increment then starts from the oracle's state before it
        run = OracleRun(w.problem, w.params, keep=True, lattice_divisor=P)
        states, wants, firsts, lasts, Js = [], [], [], [], []
        for k in range(incs):
            states.append((run.t, np.array(run.I_prefix), run.theta))
            firsts.append(len(run.records))
            wants.append(run.increment().copy())
            lasts.append(run.records[-1])
            Js.append(None if run.J is None else np.array(run.J))
        plans, res, red = _run_ranks(binding, w, P, incs, states)
        for k in range(incs):
            first, want = firsts[k], wants[k]
            # every rank holds the same set, lattice and coefficients
            for rank in range(1, P):
                assert np.array_equal(res[rank][k][1], res[0][k][1])
                assert np.array_equal(res[rank][k][4], res[0][k][4])
            info, got, (z, M), (J, m), C = res[0][k]
            last = lasts[k]
            recs_k = run.records[first:firsts[k + 1]] if k + 1 < incs else run.records[first:]
            assert M == last.M and np.array_equal(z, last.z)
            if last.coupled:
                assert M % P == 0 and info["M"] == M
                assert np.array_equal(J, Js[k]) and np.array_equal(m, last.m)
                assert _node_rel(C, last.C) < TOL
                assert sum(res[r][k][0]["samples"] for r in range(P)) == \
                    sum(rec.M for rec in recs_k if rec.coupled) + P * run.p.r * (2 * run.p.N + 1)
            if not np.array_equal(got, want):
                recs = [rr for rr in recs_k if rr.coupled]
                amb = near_ties(recs, run.theta, lambda rr: run.p.s_local if rr.t < w.problem.d else run.p.s)
                diff = {tuple(x) for x in got.tolist()} ^ {tuple(x) for x in want.tolist()}
                assert diff <= {tuple(int(v) for v in Js[k][a]) for a in amb}
        # a replay of the last sharded step repeats its exchange and its result
        C_last = plans[0].get_coefficients()
        calls = red.calls
        errs = []

        def rep(rank):
            try:
                plans[rank].replay(sync=True)
            except Exception as e:   # noqa: BLE001
                errs.append(repr(e))
                red.barrier.abort()
        ths = [threading.Thread(target=rep, args=(r,)) for r in range(P)]
        for th in ths:
            th.start()
        for th in ths:
            th.join(timeout=600)
        assert not errs and red.calls > calls
        assert np.max(np.abs(plans[0].get_coefficients() - C_last)) <= 1e-15 * np.max(np.abs(C_last))
        for p in plans:
            p.close()


@pytest.mark.gpu
def test_sharded_trigpoly_recovery_is_exact(binding):
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    d, N, G, seed = 4, 5, 9, 6
    prob = W.trigpoly(G=G, d=d, N=N, seed=seed, base_terms=5, node_terms=2, kmax=3, mag_lo=1e-4)
    params = W.Params(N=N, s=40, s_local=40, delta=1e-9, delta_is_relative=False, r=1, seed=seed)
    w = W.Workload("trigpoly", prob, params)
    _, res, _ = _run_ranks(binding, w, 2, d)
    union = {tuple(int(v) for v in f) for g in range(G) for f, c in zip(prob.tp_freqs[g], prob.tp_coefs[g]) if c != 0}
    for t in range(1, d + 1):
        got = {tuple(int(v) for v in row) for row in res[0][t - 1][1]}
        assert got == {k[:t] for k in union}
        assert np.array_equal(res[1][t - 1][1], res[0][t - 1][1])


@pytest.mark.gpu
def test_failing_collective_is_ecomm(binding):
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    w = W.small_2d(n=7, d=3, seed=1, N=3, s=8)
    plan = binding.Plan(w.problem, w.params)
    bad = binding.ALLREDUCE_FN(lambda *a: 3)
    plan.increment()
    with pytest.raises(binding.UsfftError) as e:
        binding.usfft_increment_sharded(plan, 0, 2, bad)
    assert e.value.status == 8
    with pytest.raises(binding.UsfftError) as e:
        binding.usfft_increment_sharded(plan, 2, 2, bad)          # rank out of range
    assert e.value.status == 1
    torch.cuda.synchronize()
    plan.close()
    # the context is still usable
    p2 = binding.Plan(w.problem, w.params)
    p2.increment()
    p2.close()
