"""The library's multiple rank-1 lattice rule of step 3 (usfft_multiple_lattices, host only, no GPU)
against the oracle's: the same lattices, bit for bit, for the same set and seed."""
import numpy as np
import pytest

from oracle import lattice


@pytest.fixture(scope="module")
def B():
    from paper_2109_04131_gb300 import binding
    binding.load_library()
    return binding


@pytest.mark.parametrize("seed,n,d", [(1, 1, 2), (2, 2, 3), (5, 60, 4), (7, 400, 10), (11, 1500, 10)])
def test_multiple_lattices_match_oracle(B, seed, n, d):
    rs = np.random.default_rng(seed)
    I = np.unique(rs.integers(-32, 33, size=(n, d)), axis=0).astype(np.int64)
    z, M = B.usfft_multiple_lattices(I, seed)
    lats, first = lattice.multiple_lattices(I, d, seed)
    assert first is not None
    assert list(M) == [m for _, m in lats]
    assert all(np.array_equal(z[l], lats[l][0]) for l in range(len(lats)))


def test_multiple_lattices_too_few(B):
    rs = np.random.default_rng(3)
    I = np.unique(rs.integers(-32, 33, size=(300, 6)), axis=0).astype(np.int64)
    with pytest.raises(B.UsfftError):
        B.usfft_multiple_lattices(I, 3, max_lattices=1)
    with pytest.raises(B.UsfftError):
        B.usfft_multiple_lattices(I, 3, max_lattices=0)
