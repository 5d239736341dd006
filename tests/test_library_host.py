"""The C-ABI library without a GPU: it loads, exports every symbol include/usfft.h declares,
its struct layouts match the binding, and its host planner (draws, lattice search) agrees
bit for bit with the oracle.  No device work is started here."""
import ctypes
import math
import os
import re
import subprocess

import numpy as np
import pytest

import workloads as W
from oracle import lattice, rng

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "usfft.h")


@pytest.fixture(scope="module")
def binding():
    from paper_2109_04131_gb300 import binding as b
    if not os.path.exists(b.LIB_PATH):
        import __graft_entry__
        __graft_entry__.build()
    b.load_library()
    return b


def _declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(usfft_[a-z_]+)\s*\(", text)))


def test_every_declared_symbol_is_exported(binding):
    lib = binding.load_library()
    names = _declared_functions()
    assert "usfft_plan" in names and "usfft_increment" in names and "usfft_reconstruct" in names
    for name in names:
        assert hasattr(lib, name), name
    assert set(names) <= set(binding.SIGNATURES)
    assert lib.usfft_version().decode().startswith("usfft sm_103a")


def test_struct_layouts_match_the_header(binding, tmp_path):
    src = tmp_path / "layout.c"
    src.write_text("""
#include <stdio.h>
#include <stddef.h>
#include "usfft.h"
#define P(T, f) printf(#T " " #f " %zu\\n", offsetof(T, f));
int main(void) {
  printf("usfft_problem size %zu\\n", sizeof(usfft_problem));
  printf("usfft_params size %zu\\n", sizeof(usfft_params));
  printf("usfft_increment_info size %zu\\n", sizeof(usfft_increment_info));
  P(usfft_problem, tp_freqs) P(usfft_problem, tp_coefs) P(usfft_problem, coef_scale)
  P(usfft_problem, theta_map) P(usfft_problem, map_shift)
  P(usfft_params, seed) P(usfft_params, hbm_budget_bytes) P(usfft_params, cg_tol) P(usfft_params, alloc_ctx)
  P(usfft_params, rr_lattices) P(usfft_params, rr_size_factor) P(usfft_params, max_lattice_sizes)
  P(usfft_increment_info, M) P(usfft_increment_info, kernel_launches) P(usfft_increment_info, ms_host_plan)
  P(usfft_increment_info, d2h_bytes)
  return 0;
}
""")
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split("\n")
    got = {}
    for line in out:
        if line.strip():
            a, b, c = line.split()
            got[(a, b)] = int(c)
    S = {"usfft_problem": binding.UsfftProblem, "usfft_params": binding.UsfftParams,
         "usfft_increment_info": binding.UsfftIncrementInfo}
    for (tname, field), val in got.items():
        if field == "size":
            assert ctypes.sizeof(S[tname]) == val, tname
        else:
            assert getattr(S[tname], field).offset == val, (tname, field)


def test_draws_match_the_oracle(binding):
    for seed in (0, 1, 42, 2**63 + 5):
        for fields in ((1, 2, 3, 4), (3, 5, 97, 0, 2), (2,), ()):
            assert binding.usfft_draw_key(seed, *fields) == rng.key(seed, *fields)
            assert binding.usfft_draw_uniform(seed, *fields) == rng.uniform(seed, *fields)


@pytest.mark.parametrize("seed", [1, 7, 123])
def test_lattice_search_is_bit_exact_with_the_oracle(binding, seed):
    r = np.random.default_rng(seed)
    for t in (2, 3, 4):
        prev = np.unique(r.integers(-5, 6, size=(int(r.integers(5, 80)), t - 1)), axis=0)
        J = lattice.candidate_set(prev, np.arange(-4, 5), N=8)
        z0, M0 = lattice.search(J, t, seed)
        z1, M1 = binding.usfft_search_lattice(J, t, seed)
        assert M1 == M0 and np.array_equal(z1, z0)


@pytest.mark.parametrize("seed,t,n_prev,span", [(5, 3, 400, 10), (11, 3, 700, 12), (3, 4, 300, 5)])
def test_lattice_search_parallel_path_is_bit_exact_with_the_oracle(binding, seed, t, n_prev, span):
    # candidate sets of a few thousand rows (the size of the coupled steps of the 2-D workload):
    # the library shares the (size, trial) pairs out over host threads and must still return the
    # first success of the sequential scan, as the oracle's loop does
    r = np.random.default_rng(seed)
    prev = np.unique(r.integers(-span, span + 1, size=(n_prev, t - 1)), axis=0)
    J = lattice.candidate_set(prev, np.arange(-6, 7), N=32)
    assert len(J) >= 1024
    z0, M0 = lattice.search(J, t, seed)
    z1, M1 = binding.usfft_search_lattice(J, t, seed)
    assert M1 == M0 and np.array_equal(z1, z0)


def test_lattice_search_concurrent_callers_get_the_sequential_result(binding):
    # served instances plan in parallel host threads: searches that find the thread pool busy run
    # alone, and every caller must still get the (z, M) of the sequential scan
    from concurrent.futures import ThreadPoolExecutor
    r = np.random.default_rng(21)
    sets = []
    for k in range(6):
        prev = np.unique(r.integers(-8 - k, 9 + k, size=(300 + 60 * k, 2)), axis=0)
        sets.append(lattice.candidate_set(prev, np.arange(-6, 7), N=32))
    want = [binding.usfft_search_lattice(J, 3, 5) for J in sets]
    with ThreadPoolExecutor(max_workers=6) as ex:
        for _ in range(3):
            got = list(ex.map(lambda J: binding.usfft_search_lattice(J, 3, 5), sets))
            for (z0, M0), (z1, M1) in zip(want, got):
                assert M1 == M0 and np.array_equal(z1, z0)


@pytest.mark.parametrize("t", [10, 12])
def test_lattice_search_long_rows_and_repeated_rows(binding, t):
    # rows of more than 8 coordinates take the hashed repeated-row check: a planted duplicate is
    # still found (EINVAL), and distinct rows give the oracle's (z, M)
    r = np.random.default_rng(t)
    prev = np.unique(r.integers(-2, 3, size=(60, t - 1)), axis=0)
    J = lattice.candidate_set(prev, np.arange(-2, 3), N=8)
    z0, M0 = lattice.search(J, t, 3)
    z1, M1 = binding.usfft_search_lattice(J, t, 3)
    assert M1 == M0 and np.array_equal(z1, z0)
    Jd = np.concatenate([J, J[len(J) // 2:len(J) // 2 + 1]])
    with pytest.raises(binding.UsfftError):
        binding.usfft_search_lattice(Jd, t, 3)


def test_lattice_search_large_set_with_a_repeated_row(binding):
    # a candidate set of the parallel path's size with one row planted twice: no lattice can
    # separate it, and the search reports that (after its first batch of sizes) instead of a lattice
    r = np.random.default_rng(17)
    prev = np.unique(r.integers(-12, 13, size=(500, 2)), axis=0)
    J = lattice.candidate_set(prev, np.arange(-6, 7), N=32)
    assert len(J) >= 1024
    z0, M0 = lattice.search(J, 3, 9)
    z1, M1 = binding.usfft_search_lattice(J, 3, 9)
    assert M1 == M0 and np.array_equal(z1, z0)
    Jd = np.concatenate([J[:700], J[350:351], J[700:]])
    with pytest.raises(binding.UsfftError):
        binding.usfft_search_lattice(Jd, 3, 9)


def test_lattice_search_on_the_c1_increments(binding):
    # the candidate sets the oracle builds for the 1-D workload (increments 2..4)
    from oracle.usfft import OracleRun
    w = W.c1(3)
    run = OracleRun(w.problem, w.params)
    run.increment()
    for t in range(2, w.problem.d + 1):
        run.increment()
        z, M = binding.usfft_search_lattice(run.J, t, w.params.seed)
        assert M == run.M and np.array_equal(z, run.z)


def test_lattice_search_edge_cases(binding):
    z, M = binding.usfft_search_lattice(np.zeros((0, 2), np.int8), 2, 1)
    assert M == 0
    z, M = binding.usfft_search_lattice(np.array([[3, -2]], np.int8), 2, 1)
    assert M == 1
    with pytest.raises(binding.UsfftError):
        binding.usfft_search_lattice(np.zeros((4, 2), np.int8), 2, 1)   # duplicates never separate


@pytest.mark.parametrize("t,i,n_prev,n_t,s_t,L,factor,seed", [
    (2, 1, 33, 17, 50, 5, 2.0, 1), (5, 2, 1200, 13, 500, 7, 2.0, 3), (3, 1, 1, 1, 0, 1, 0.5, 9),
    (10, 2, 4000, 30, 1000, 31, 1.5, 12345)])
def test_random_lattice_rule_is_bit_exact_with_the_oracle(binding, t, i, n_prev, n_t, s_t, L, factor, seed):
    from oracle import lattice
    z, M = binding.usfft_random_lattices(t, i, n_prev, n_t, s_t, L, factor, seed)
    want = lattice.random_lattices(t, i, n_prev, n_t, s_t, L, factor, seed)
    assert [int(m) for m in M] == [m for _, m in want]
    assert np.array_equal(z, np.array([zz for zz, _ in want]))
    assert len(set(M.tolist())) == L and all(lattice.is_smooth7(int(m)) for m in M)
    assert all(math.gcd(int(v), int(m)) == 1 for row, m in zip(z, M) for v in row)
    with pytest.raises(binding.UsfftError):
        binding.usfft_random_lattices(t, i, n_prev, n_t, s_t, 32, factor, seed)


def test_lattice_search_exhaustion(binding):
    # one size and one trial: the oracle's search and the library's both give up (ELATTICE)
    J = lattice.candidate_set(np.arange(-4, 5)[:, None], np.arange(-4, 5), N=4)
    with pytest.raises(RuntimeError):
        lattice.search(J, 2, 3, trials=1, max_sizes=1)
    with pytest.raises(binding.UsfftError) as e:
        binding.usfft_search_lattice(J, 2, 3, trials=1, max_sizes=1)
    assert e.value.status == 3
    z0, M0 = lattice.search(J, 2, 2, trials=1, max_sizes=1)
    z1, M1 = binding.usfft_search_lattice(J, 2, 2, trials=1, max_sizes=1)
    assert M0 == M1 == 81 and np.array_equal(z0, z1)


def test_tune_table_import_export(binding):
    # the process-wide table of tuned launch parameters (host only): text round trip, a malformed
    # line leaves the table unchanged, None clears it
    binding.usfft_tune_import(None)
    assert binding.usfft_tune_export() == ""
    binding.usfft_tune_import("1 68 304 1.5\n2 8193 4 0.25\n")
    rows = sorted(tuple(line.split()[:3]) for line in binding.usfft_tune_export().strip().split("\n"))
    assert rows == [("1", "68", "304"), ("2", "8193", "4")]
    for bad in ("1 68\n", "3 1 1 1\n", "1 68 0 1\n", "1 68 304 1.5 extra\n"):
        with pytest.raises(binding.UsfftError) as e:
            binding.usfft_tune_import(bad)
        assert e.value.status == 1
    assert len(binding.usfft_tune_export().strip().split("\n")) == 2
    binding.usfft_tune_import("1 68 152 1.0\n")          # replaces the entry
    assert "1 68 152" in binding.usfft_tune_export()
    binding.usfft_tune_import(None)
    assert binding.usfft_tune_export() == ""
