"""ctypes binding of the C ABI in include/usfft.h (argument marshalling only).

Every numeric step runs in libusfft.so.  If the library is missing this module raises;
there is no CPU fallback.  Device memory of a plan comes from PyTorch's caching
allocator (through the allocator hook of usfft_params) and its work runs on the
current PyTorch stream unless another stream is given.

Module-level functions carry the C names (usfft_plan, usfft_increment, usfft_replay,
usfft_rewind, usfft_resume, usfft_get_set, usfft_reconstruct, usfft_reconstruct_multiple, usfft_sample_points, usfft_evaluate,
usfft_errors, usfft_statistics, usfft_plan_bytes, usfft_increment_many, usfft_get_lattice, usfft_get_candidates,
usfft_get_samples, usfft_get_coefficients, usfft_get_selection, usfft_set_keep_iterations,
usfft_get_iteration, usfft_last_error,
usfft_destroy); ``Plan`` wraps them.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libusfft.so")

STATUS = {0: "OK", 1: "EINVAL", 2: "ENOMEM", 3: "ELATTICE", 4: "ENOCONV", 5: "ETIMEOUT", 6: "ECUDA", 7: "ESTATE",
          8: "ECOMM"}

ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p)
FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p)
# usfft_allreduce_fn(buf, count, dtype, op, stream, ctx) -> int
ALLREDUCE_FN = ctypes.CFUNCTYPE(ctypes.c_int, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_int, ctypes.c_int,
                                ctypes.c_void_p, ctypes.c_void_p)
RED_SUM, RED_MAX = 0, 1
RED_F64, RED_U8 = 0, 1


class UsfftProblem(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("n", ctypes.c_int), ("d", ctypes.c_int), ("coef_model", ctypes.c_int),
                ("coef_scale", ctypes.c_double), ("coef_decay", ctypes.c_double), ("f_const", ctypes.c_double),
                ("tp_nodes", ctypes.c_int), ("tp_nterms", ctypes.c_int),
                ("tp_freqs", ctypes.c_void_p), ("tp_coefs", ctypes.c_void_p),
                ("theta_map", ctypes.c_int), ("map_alpha", ctypes.c_double), ("map_beta", ctypes.c_double),
                ("map_shift", ctypes.c_double)]


class UsfftParams(ctypes.Structure):
    _fields_ = [("N", ctypes.c_int), ("s", ctypes.c_int), ("s_local", ctypes.c_int), ("delta", ctypes.c_double),
                ("delta_is_relative", ctypes.c_int), ("r", ctypes.c_int), ("seed", ctypes.c_uint64),
                ("precision", ctypes.c_int), ("hbm_budget_bytes", ctypes.c_size_t),
                ("max_cg_iters", ctypes.c_int), ("max_lattice_trials", ctypes.c_int), ("cg_tol", ctypes.c_double),
                ("alloc", ALLOC_FN), ("free", FREE_FN), ("alloc_ctx", ctypes.c_void_p),
                ("rr_lattices", ctypes.c_int), ("rr_size_factor", ctypes.c_double),
                ("max_lattice_sizes", ctypes.c_int)]


class UsfftIncrementInfo(ctypes.Structure):
    _fields_ = [("t", ctypes.c_int), ("M", ctypes.c_int64), ("n_candidates", ctypes.c_int64),
                ("n_detected", ctypes.c_int64), ("n_1d", ctypes.c_int64), ("samples", ctypes.c_int64),
                ("cg_iters_total", ctypes.c_int64), ("cg_iters_max", ctypes.c_int32),
                ("kernel_launches", ctypes.c_int32), ("theta", ctypes.c_double), ("ms_device", ctypes.c_double),
                ("ms_host_plan", ctypes.c_double), ("h2d_bytes", ctypes.c_int64), ("d2h_bytes", ctypes.c_int64)]


class UsfftStageTimes(ctypes.Structure):
    _fields_ = [("ms", ctypes.c_double * 3), ("launches", ctypes.c_int32 * 3), ("cg_iters_total", ctypes.c_int64),
                ("refine_steps_total", ctypes.c_int64)]


class UsfftTuneReport(ctypes.Structure):
    _fields_ = [("ms_before", ctypes.c_double), ("ms_after", ctypes.c_double), ("sampler_blocks", ctypes.c_int32),
                ("fft_pass1_tile", ctypes.c_int32), ("fft_final_tile", ctypes.c_int32)]


# exported symbols and their signatures (restype, argtypes)
_P = ctypes.c_void_p
SIGNATURES = {
    "usfft_plan": (ctypes.c_int, [ctypes.POINTER(UsfftProblem), ctypes.POINTER(UsfftParams), _P, ctypes.POINTER(_P)]),
    "usfft_increment": (ctypes.c_int, [_P, ctypes.POINTER(UsfftIncrementInfo)]),
    "usfft_replay": (ctypes.c_int, [_P, ctypes.c_int, ctypes.POINTER(ctypes.c_int32)]),
    "usfft_rewind": (ctypes.c_int, [_P, ctypes.c_int]),
    "usfft_resume": (ctypes.c_int, [_P, ctypes.c_int, _P, ctypes.c_int64, ctypes.c_double]),
    "usfft_set_timing": (ctypes.c_int, [_P, ctypes.c_int]),
    "usfft_get_stage_times": (ctypes.c_int, [_P, ctypes.POINTER(UsfftStageTimes)]),
    "usfft_get_set": (ctypes.c_int, [_P, _P, ctypes.c_int64, ctypes.POINTER(ctypes.c_int64),
                                     ctypes.POINTER(ctypes.c_int32)]),
    "usfft_reconstruct": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_int64), _P, _P, ctypes.c_int]),
    "usfft_reconstruct_multiple": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_int64), _P, _P, ctypes.c_int]),
    "usfft_sample_points": (ctypes.c_int, [_P, _P, ctypes.c_int64, _P, ctypes.c_int]),
    "usfft_evaluate": (ctypes.c_int, [_P, _P, ctypes.c_int64, _P, ctypes.c_int]),
    "usfft_errors": (ctypes.c_int, [_P, _P, ctypes.c_int64, ctypes.c_int, _P, _P]),
    "usfft_statistics": (ctypes.c_int, [_P, _P, _P, _P]),
    "usfft_get_random_lattices": (ctypes.c_int, [_P, _P, _P, ctypes.POINTER(ctypes.c_int32),
                                                 ctypes.POINTER(ctypes.c_int32)]),
    "usfft_get_lattice": (ctypes.c_int, [_P, _P, ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int32)]),
    "usfft_get_candidates": (ctypes.c_int, [_P, _P, ctypes.POINTER(ctypes.c_int64), _P]),
    "usfft_get_samples": (ctypes.c_int, [_P, _P, ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int64)]),
    "usfft_get_coefficients": (ctypes.c_int, [_P, _P, ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int64)]),
    "usfft_get_selection": (ctypes.c_int, [_P, _P, ctypes.POINTER(ctypes.c_int64)]),
    "usfft_set_keep_iterations": (ctypes.c_int, [_P, ctypes.c_int]),
    "usfft_get_iteration": (ctypes.c_int, [_P, ctypes.c_int, _P, _P, _P, ctypes.POINTER(ctypes.c_int32)]),
    "usfft_last_error": (ctypes.c_char_p, [_P]),
    "usfft_plan_bytes": (ctypes.c_size_t, [_P]),
    "usfft_increment_many": (ctypes.c_int, [ctypes.POINTER(_P), ctypes.c_int, ctypes.c_int,
                                            ctypes.POINTER(UsfftIncrementInfo), ctypes.POINTER(ctypes.c_int)]),
    "usfft_increment_sharded": (ctypes.c_int, [_P, ctypes.c_int, ctypes.c_int, ALLREDUCE_FN, _P,
                                               ctypes.POINTER(UsfftIncrementInfo)]),
    "usfft_search_lattice_multiple": (ctypes.c_int, [_P, ctypes.c_int64, ctypes.c_int, ctypes.c_uint64, ctypes.c_int,
                                                     ctypes.c_int, ctypes.c_int64, _P, ctypes.POINTER(ctypes.c_int64)]),
    "usfft_autotune": (ctypes.c_int, [_P, ctypes.c_int, ctypes.POINTER(UsfftTuneReport)]),
    "usfft_tune_export": (ctypes.c_int, [ctypes.c_char_p, ctypes.c_size_t, ctypes.POINTER(ctypes.c_size_t)]),
    "usfft_tune_import": (ctypes.c_int, [ctypes.c_char_p]),
    "usfft_destroy": (None, [_P]),
    "usfft_version": (ctypes.c_char_p, []),
    "usfft_search_lattice": (ctypes.c_int, [_P, ctypes.c_int64, ctypes.c_int, ctypes.c_uint64, ctypes.c_int,
                                            ctypes.c_int, _P, ctypes.POINTER(ctypes.c_int64)]),
    "usfft_random_lattices": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_int64, ctypes.c_int64, ctypes.c_int64,
                                             ctypes.c_int, ctypes.c_double, ctypes.c_uint64, _P, _P]),
    "usfft_multiple_lattices": (ctypes.c_int, [_P, ctypes.c_int64, ctypes.c_int, ctypes.c_uint64, ctypes.c_int, _P, _P,
                                               ctypes.POINTER(ctypes.c_int32)]),
    "usfft_draw_key": (ctypes.c_uint64, [ctypes.c_uint64, _P, ctypes.c_int]),
    "usfft_draw_uniform": (ctypes.c_double, [ctypes.c_uint64, _P, ctypes.c_int]),
    "usfft_sample_2d_static": (ctypes.c_int, [ctypes.POINTER(UsfftProblem), _P, _P, ctypes.c_int64, ctypes.c_int64,
                                              ctypes.c_int64, ctypes.c_double, ctypes.c_int, _P, _P,
                                              ctypes.POINTER(ctypes.c_uint32)]),
}

_lib = None


def load_library(force_reload: bool = False):
    """Load libusfft.so (raises if it has not been built)."""
    global _lib
    if _lib is not None and not force_reload:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is missing: run __graft_entry__.build() first (no CPU fallback)")
    lib = ctypes.CDLL(LIB_PATH)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


class UsfftError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


def _check(st, handle=None):
    if st != 0:
        lib = load_library()
        msg = lib.usfft_last_error(handle)
        raise UsfftError(st, msg.decode() if msg else "")


def _torch_allocator(device_index):
    import torch

    def alloc(nbytes, stream, ctx):
        try:
            return torch.cuda.caching_allocator_alloc(int(nbytes), device=device_index, stream=int(stream or 0))
        except Exception:
            return None

    def free(ptr, stream, ctx):
        torch.cuda.caching_allocator_delete(ptr)

    return ALLOC_FN(alloc), FREE_FN(free)


def make_problem(prob) -> tuple:
    """(UsfftProblem, keep-alive arrays) from a workloads.Problem."""
    p = UsfftProblem()
    p.kind = prob.kind
    p.n = prob.n
    p.d = prob.d
    p.coef_model = prob.coef_model
    p.coef_scale = prob.coef_scale
    p.coef_decay = prob.coef_decay
    p.f_const = prob.f_const
    p.theta_map = getattr(prob, "theta_map", 0)
    p.map_alpha = getattr(prob, "map_alpha", -1.0)
    p.map_beta = getattr(prob, "map_beta", 1.0)
    p.map_shift = getattr(prob, "map_shift", 0.0)
    keep = []
    if prob.tp_freqs is not None:
        f = np.ascontiguousarray(prob.tp_freqs, dtype=np.int8)
        c = np.ascontiguousarray(np.stack([prob.tp_coefs.real, prob.tp_coefs.imag], axis=-1), dtype=np.float64)
        p.tp_nodes = f.shape[0]
        p.tp_nterms = f.shape[1]
        p.tp_freqs = f.ctypes.data
        p.tp_coefs = c.ctypes.data
        keep += [f, c]
    return p, keep


def make_params(par, alloc=None, free=None) -> UsfftParams:
    q = UsfftParams()
    q.N = par.N
    q.s = par.s
    q.s_local = par.s_local
    q.delta = par.delta
    q.delta_is_relative = int(par.delta_is_relative)
    q.r = par.r
    q.seed = par.seed
    q.precision = par.precision
    q.hbm_budget_bytes = par.hbm_budget_bytes
    q.max_cg_iters = par.max_cg_iters
    q.max_lattice_trials = par.max_lattice_trials
    q.cg_tol = par.cg_tol
    q.rr_lattices = getattr(par, "rr_lattices", 0)
    q.rr_size_factor = getattr(par, "rr_size_factor", 0.0)
    q.max_lattice_sizes = getattr(par, "max_lattice_sizes", 0)
    q.alloc = alloc if alloc is not None else ALLOC_FN()
    q.free = free if free is not None else FREE_FN()
    q.alloc_ctx = None
    return q


# ---- C-named functions -------------------------------------------------------------------
def usfft_plan(problem, params, stream=None, torch_alloc=True):
    return Plan(problem, params, stream=stream, torch_alloc=torch_alloc)


def usfft_increment(plan):
    return plan.increment()


def usfft_replay(plan, sync=True):
    return plan.replay(sync)


def usfft_rewind(plan, t):
    return plan.rewind(t)


def usfft_resume(plan, t, I, theta):
    return plan.resume(t, I, theta)


def usfft_get_set(plan):
    return plan.get_set()


def usfft_reconstruct(plan):
    return plan.reconstruct()


def usfft_reconstruct_multiple(plan):
    return plan.reconstruct_multiple()


def usfft_sample_points(plan, Y):
    return plan.sample_points(Y)


def usfft_evaluate(plan, Y):
    return plan.evaluate(Y)


def usfft_errors(plan, Y):
    return plan.errors(Y)


def usfft_statistics(plan):
    return plan.statistics()


def usfft_plan_bytes(plan):
    return plan.bytes()


def usfft_increment_many(plans, max_threads=0):
    """One increment of every plan at once (the batched form): (infos, statuses), one entry per
    plan; no exception for a failed plan, its status says so."""
    lib = load_library()
    n = len(plans)
    handles = (_P * max(n, 1))(*[p.handle for p in plans])
    infos = (UsfftIncrementInfo * max(n, 1))()
    sts = (ctypes.c_int * max(n, 1))()
    st = lib.usfft_increment_many(handles, n, int(max_threads), infos, sts)
    if st == 1 and n and all(v == 0 for v in sts[:n]):
        _check(st, None)                                   # rejected before running (NULL / repeated plan)
    out = [{name: getattr(infos[k], name) for name, _ in UsfftIncrementInfo._fields_} for k in range(n)]
    return out, [int(v) for v in sts[:n]]


def usfft_get_lattice(plan):
    return plan.get_lattice()


def usfft_get_candidates(plan):
    return plan.get_candidates()


def usfft_get_samples(plan):
    return plan.get_samples()


def usfft_get_coefficients(plan):
    return plan.get_coefficients()


def usfft_get_selection(plan):
    return plan.get_selection()


def usfft_set_keep_iterations(plan, on=True):
    return plan.set_keep_iterations(on)


def usfft_get_iteration(plan, i):
    return plan.get_iteration(i)


def usfft_last_error(plan=None):
    lib = load_library()
    msg = lib.usfft_last_error(plan.handle if plan is not None else None)
    return msg.decode() if msg else ""


def usfft_destroy(plan):
    plan.close()


def usfft_search_lattice(J, t, seed, trials=64, max_sizes=400):
    """Host-only lattice search of the library: (z, M) for the candidate rows J [n][t]."""
    lib = load_library()
    Jc = np.ascontiguousarray(J, dtype=np.int8).reshape(-1, t) if len(J) else np.zeros((0, t), np.int8)
    z = np.zeros(t, dtype=np.int64)
    M = ctypes.c_int64(0)
    st = lib.usfft_search_lattice(Jc.ctypes.data if len(Jc) else None, len(Jc), t, seed, trials, max_sizes,
                                  z.ctypes.data, ctypes.byref(M))
    _check(st, None)
    return z, M.value


def usfft_search_lattice_multiple(J, t, seed, divisor, trials=64, max_sizes=400):
    """Host-only lattice rule of the sharded form: (z, M) with M a multiple of divisor."""
    lib = load_library()
    Jc = np.ascontiguousarray(J, dtype=np.int8).reshape(-1, t) if len(J) else np.zeros((0, t), np.int8)
    z = np.zeros(t, dtype=np.int64)
    M = ctypes.c_int64(0)
    st = lib.usfft_search_lattice_multiple(Jc.ctypes.data if len(Jc) else None, len(Jc), t, seed, trials, max_sizes,
                                           int(divisor), z.ctypes.data, ctypes.byref(M))
    _check(st, None)
    return z, M.value


def usfft_increment_sharded(plan, rank, nranks, allreduce_fn):
    """One increment of `plan` as rank `rank` of `nranks` through the collective hook allreduce_fn
    (an ALLREDUCE_FN); the info dict of the increment."""
    info = UsfftIncrementInfo()
    plan._ck(plan._lib.usfft_increment_sharded(plan.handle, int(rank), int(nranks), allreduce_fn, None,
                                               ctypes.byref(info)))
    return {name: getattr(info, name) for name, _ in UsfftIncrementInfo._fields_}


def usfft_autotune(plan, reps=3):
    return plan.autotune(reps)


def usfft_tune_export() -> str:
    """The process-wide table of tuned launch parameters as text."""
    lib = load_library()
    n = ctypes.c_size_t(0)
    _check(lib.usfft_tune_export(None, 0, ctypes.byref(n)), None)
    buf = ctypes.create_string_buffer(n.value + 1)
    _check(lib.usfft_tune_export(buf, n.value + 1, ctypes.byref(n)), None)
    return buf.value.decode()


def usfft_tune_import(text):
    """Add the entries of `text` to the table (None clears it)."""
    lib = load_library()
    _check(lib.usfft_tune_import(None if text is None else text.encode()), None)


def usfft_multiple_lattices(freqs, seed, max_lattices=64):
    """Host-only multiple rank-1 lattice rule of step 3 for the set freqs [n][d]: (z [L][d], M [L])."""
    lib = load_library()
    F = np.ascontiguousarray(np.asarray(freqs, dtype=np.int8))
    n, d = F.shape
    z = np.zeros((max_lattices, d), dtype=np.int64)
    M = np.zeros(max_lattices, dtype=np.int64)
    cnt = ctypes.c_int32(0)
    _check(lib.usfft_multiple_lattices(F.ctypes.data if n else None, n, d, seed, max_lattices, z.ctypes.data,
                                       M.ctypes.data, ctypes.byref(cnt)), None)
    return z[:cnt.value], M[:cnt.value]


def usfft_random_lattices(t, i, n_prev, n_t, s_t, L, factor, seed):
    """Host-only random rank-1 lattice rule of the library: (z [L][t], M [L])."""
    lib = load_library()
    z = np.zeros((L, t), dtype=np.int64)
    M = np.zeros(L, dtype=np.int64)
    _check(lib.usfft_random_lattices(t, i, n_prev, n_t, s_t, L, factor, seed, z.ctypes.data, M.ctypes.data), None)
    return z, M


def usfft_sample_2d_static(problem, z, tails, M, i0, count, U_ptr, stream=0, tol=0.0, max_iters=0,
                           sync=True):
    """Mixed-precision 2-D samples of nodes i0..i0+count-1 into the caller's device buffer
    U_ptr ([count][n*n] fp64) without any device allocation by the library.  Returns the
    number of unconverged solves (sync=True) or None."""
    lib = load_library()
    prob, keep = make_problem(problem)
    zc = np.ascontiguousarray(z, dtype=np.int64)
    tc = np.ascontiguousarray(tails, dtype=np.float64)
    unc = ctypes.c_uint32(0)
    st = lib.usfft_sample_2d_static(ctypes.byref(prob), zc.ctypes.data, tc.ctypes.data, int(M), int(i0), int(count),
                                    float(tol), int(max_iters), ctypes.c_void_p(int(U_ptr)),
                                    ctypes.c_void_p(int(stream or 0)), ctypes.byref(unc) if sync else None)
    _check(st, None)
    return unc.value if sync else None


def usfft_draw_key(seed, *fields):
    lib = load_library()
    f = (ctypes.c_uint64 * max(1, len(fields)))(*fields)
    return int(lib.usfft_draw_key(seed, f, len(fields)))


def usfft_draw_uniform(seed, *fields):
    lib = load_library()
    f = (ctypes.c_uint64 * max(1, len(fields)))(*fields)
    return float(lib.usfft_draw_uniform(seed, f, len(fields)))


class Plan:
    """One usFFT detection run (problem + parameters) on the current CUDA device."""

    def __init__(self, problem, params, stream=None, torch_alloc=True):
        lib = load_library()
        self._lib = lib
        self.problem = problem
        self.params = params
        self.handle = None
        self._keep = []
        alloc = free = None
        if stream is None or torch_alloc:
            import torch
            dev = torch.cuda.current_device()
            if stream is None:
                stream = torch.cuda.current_stream(dev).cuda_stream
            if torch_alloc:
                alloc, free = _torch_allocator(dev)
        self._alloc, self._free = alloc, free
        self.stream = int(stream or 0)
        prob, keep = make_problem(problem)
        self._keep += keep
        par = make_params(params, alloc, free)
        h = ctypes.c_void_p()
        st = lib.usfft_plan(ctypes.byref(prob), ctypes.byref(par), ctypes.c_void_p(self.stream), ctypes.byref(h))
        _check(st, None)
        self.handle = h

    def _ck(self, st):
        _check(st, self.handle)

    def bytes(self) -> int:
        """Device bytes the plan holds now."""
        return int(self._lib.usfft_plan_bytes(self.handle))

    def increment(self) -> dict:
        info = UsfftIncrementInfo()
        self._ck(self._lib.usfft_increment(self.handle, ctypes.byref(info)))
        return {name: getattr(info, name) for name, _ in UsfftIncrementInfo._fields_}

    def replay(self, sync=True) -> int:
        n = ctypes.c_int32(0)
        self._ck(self._lib.usfft_replay(self.handle, int(bool(sync)), ctypes.byref(n)))
        return n.value

    def rewind(self, t: int) -> None:
        self._ck(self._lib.usfft_rewind(self.handle, int(t)))

    def resume(self, t: int, I, theta: float) -> None:
        """Continue from the checkpoint (t, I^(1..t), theta)."""
        rows = np.ascontiguousarray(np.asarray(I, dtype=np.int8).reshape(-1, max(t, 1)))
        n = len(rows) if t > 0 else 0
        self._ck(self._lib.usfft_resume(self.handle, int(t), rows.ctypes.data if n else None, n, float(theta)))

    def set_timing(self, on: bool) -> None:
        self._ck(self._lib.usfft_set_timing(self.handle, int(bool(on))))

    def stage_times(self) -> dict:
        st = UsfftStageTimes()
        self._ck(self._lib.usfft_get_stage_times(self.handle, ctypes.byref(st)))
        names = ("sample", "fft", "select")
        return {"ms": {n: st.ms[i] for i, n in enumerate(names)},
                "launches": {n: st.launches[i] for i, n in enumerate(names)},
                "cg_iters_total": st.cg_iters_total, "refine_steps_total": st.refine_steps_total}

    def get_set(self) -> np.ndarray:
        n = ctypes.c_int64(0)
        t = ctypes.c_int32(0)
        self._ck(self._lib.usfft_get_set(self.handle, None, 0, ctypes.byref(n), ctypes.byref(t)))
        out = np.zeros((n.value, t.value), dtype=np.int8)
        if n.value:
            self._ck(self._lib.usfft_get_set(self.handle, out.ctypes.data, n.value, ctypes.byref(n), ctypes.byref(t)))
        return out.astype(np.int64)

    def reconstruct(self):
        """(I [n][d] int64, C [G][n] complex128): step 3 on the detected set."""
        n = ctypes.c_int64(0)
        self._ck(self._lib.usfft_reconstruct(self.handle, ctypes.byref(n), None, None, 0))
        d = self.problem.d
        I = np.zeros((n.value, d), dtype=np.int8)
        C = np.zeros((self.problem.G, n.value, 2))
        out = C if C.size else np.zeros(2)          # an empty set still records the (zero) approximation
        self._ck(self._lib.usfft_reconstruct(self.handle, ctypes.byref(n), I.ctypes.data if n.value else None,
                                             out.ctypes.data, 0))
        return I.astype(np.int64), C[..., 0] + 1j * C[..., 1]

    def reconstruct_multiple(self):
        """(I [n][d] int64, C [G][n] complex128): step 3 on multiple rank-1 lattices."""
        n = ctypes.c_int64(0)
        self._ck(self._lib.usfft_reconstruct_multiple(self.handle, ctypes.byref(n), None, None, 0))
        d = self.problem.d
        I = np.zeros((n.value, d), dtype=np.int8)
        C = np.zeros((self.problem.G, n.value, 2))
        out = C if C.size else np.zeros(2)          # an empty set still records the (zero) approximation
        self._ck(self._lib.usfft_reconstruct_multiple(self.handle, ctypes.byref(n), I.ctypes.data if n.value else None,
                                             out.ctypes.data, 0))
        return I.astype(np.int64), C[..., 0] + 1j * C[..., 1]

    def statistics(self):
        """(mean complex [G], variance [G], gsi [G][d]) of the last reconstruction."""
        G, d = self.problem.G, self.problem.d
        mean = np.zeros((G, 2))
        var = np.zeros(G)
        gsi = np.zeros((G, d))
        self._ck(self._lib.usfft_statistics(self.handle, mean.ctypes.data, var.ctypes.data, gsi.ctypes.data))
        return mean[:, 0] + 1j * mean[:, 1], var, gsi

    def _points(self, Y) -> np.ndarray:
        Y = np.ascontiguousarray(np.asarray(Y, dtype=np.float64).reshape(-1, self.problem.d))
        return Y

    def sample_points(self, Y) -> np.ndarray:
        """FE solutions (the black box) at the rows of Y: [n][G]."""
        Y = self._points(Y)
        U = np.zeros((len(Y), self.problem.G))
        self._ck(self._lib.usfft_sample_points(self.handle, Y.ctypes.data, len(Y), U.ctypes.data, 0))
        return U

    def evaluate(self, Y) -> np.ndarray:
        """u^usFFT at the rows of Y with the last reconstruction: complex [n][G]."""
        Y = self._points(Y)
        V = np.zeros((len(Y), self.problem.G, 2))
        self._ck(self._lib.usfft_evaluate(self.handle, Y.ctypes.data, len(Y), V.ctypes.data, 0))
        return V[..., 0] + 1j * V[..., 1]

    def errors(self, Y):
        """(err_2 [G], err_inf [G]) of the last reconstruction over the test points Y."""
        Y = self._points(Y)
        e2 = np.zeros(self.problem.G)
        ei = np.zeros(self.problem.G)
        self._ck(self._lib.usfft_errors(self.handle, Y.ctypes.data, len(Y), 0, e2.ctypes.data, ei.ctypes.data))
        return e2, ei

    def get_random_lattices(self):
        """([z_q] int64 [count][t], [M_q] int64 [count]) of the last random-lattice step,
        q = (i-1)*L + l in detection-iteration order (count 0 after a single-lattice step)."""
        cnt = ctypes.c_int32(0)
        t = ctypes.c_int32(0)
        self._ck(self._lib.usfft_get_random_lattices(self.handle, None, None, ctypes.byref(cnt), ctypes.byref(t)))
        z = np.zeros((cnt.value, t.value), dtype=np.int64)
        M = np.zeros(cnt.value, dtype=np.int64)
        if cnt.value:
            self._ck(self._lib.usfft_get_random_lattices(self.handle, z.ctypes.data, M.ctypes.data, ctypes.byref(cnt),
                                                         ctypes.byref(t)))
        return z, M

    def get_lattice(self):
        M = ctypes.c_int64(0)
        t = ctypes.c_int32(0)
        self._ck(self._lib.usfft_get_lattice(self.handle, None, ctypes.byref(M), ctypes.byref(t)))
        z = np.zeros(t.value, dtype=np.int64)
        self._ck(self._lib.usfft_get_lattice(self.handle, z.ctypes.data, ctypes.byref(M), ctypes.byref(t)))
        return z, M.value

    def get_candidates(self):
        n = ctypes.c_int64(0)
        self._ck(self._lib.usfft_get_candidates(self.handle, None, ctypes.byref(n), None))
        z, M = self.get_lattice()
        t = len(z)
        J = np.zeros((n.value, t), dtype=np.int8)
        m = np.zeros(n.value, dtype=np.int64)
        self._ck(self._lib.usfft_get_candidates(self.handle, J.ctypes.data, ctypes.byref(n), m.ctypes.data))
        return J.astype(np.int64), m

    def get_samples(self) -> np.ndarray:
        M = ctypes.c_int64(0)
        G = ctypes.c_int64(0)
        self._ck(self._lib.usfft_get_samples(self.handle, None, ctypes.byref(M), ctypes.byref(G)))
        U = np.zeros((M.value, G.value), dtype=np.float64)
        self._ck(self._lib.usfft_get_samples(self.handle, U.ctypes.data, ctypes.byref(M), ctypes.byref(G)))
        return U

    def get_coefficients(self) -> np.ndarray:
        G = ctypes.c_int64(0)
        n = ctypes.c_int64(0)
        self._ck(self._lib.usfft_get_coefficients(self.handle, None, ctypes.byref(G), ctypes.byref(n)))
        C = np.zeros((G.value, n.value, 2), dtype=np.float64)
        self._ck(self._lib.usfft_get_coefficients(self.handle, C.ctypes.data, ctypes.byref(G), ctypes.byref(n)))
        return C[..., 0] + 1j * C[..., 1]

    def get_selection(self) -> np.ndarray:
        n = ctypes.c_int64(0)
        self._ck(self._lib.usfft_get_selection(self.handle, None, ctypes.byref(n)))
        words = np.zeros((n.value + 31) // 32, dtype=np.uint32)
        self._ck(self._lib.usfft_get_selection(self.handle, words.ctypes.data, ctypes.byref(n)))
        bits = np.unpackbits(words.view(np.uint8), bitorder="little")[: n.value]
        return bits.astype(bool)

    def autotune(self, reps: int = 3) -> dict:
        """Tune the launch parameters on replays of the last step (usfft_autotune)."""
        rep = UsfftTuneReport()
        self._ck(self._lib.usfft_autotune(self.handle, int(reps), ctypes.byref(rep)))
        return {name: getattr(rep, name) for name, _ in UsfftTuneReport._fields_}

    def set_keep_iterations(self, on: bool) -> None:
        self._ck(self._lib.usfft_set_keep_iterations(self.handle, int(bool(on))))

    def kept_iterations(self) -> int:
        cnt = ctypes.c_int32(0)
        self._ck(self._lib.usfft_get_iteration(self.handle, 0, None, None, None, ctypes.byref(cnt)))
        return cnt.value

    def get_iteration(self, i: int):
        """(U [M][G], C [G][|J|] complex, union bitmap of iterations 1..i as bool [|J|]) of
        detection iteration i (1-based) of the last step (keeping must be on)."""
        M = ctypes.c_int64(0)
        G = ctypes.c_int64(0)
        n = ctypes.c_int64(0)
        self._ck(self._lib.usfft_get_samples(self.handle, None, ctypes.byref(M), ctypes.byref(G)))
        self._ck(self._lib.usfft_get_coefficients(self.handle, None, ctypes.byref(G), ctypes.byref(n)))
        U = np.zeros((M.value, G.value), dtype=np.float64)
        C = np.zeros((G.value, n.value, 2), dtype=np.float64)
        words = np.zeros(max(1, (n.value + 31) // 32), dtype=np.uint32)
        cnt = ctypes.c_int32(0)
        self._ck(self._lib.usfft_get_iteration(self.handle, int(i), U.ctypes.data, C.ctypes.data, words.ctypes.data,
                                               ctypes.byref(cnt)))
        bits = np.unpackbits(words.view(np.uint8), bitorder="little")[: n.value].astype(bool)
        return U, C[..., 0] + 1j * C[..., 1], bits

    def close(self):
        if self.handle:
            self._lib.usfft_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
