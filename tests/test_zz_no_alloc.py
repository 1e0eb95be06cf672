"""The allocation-free entry point skolem_item_residues_noalloc, for callers
that cannot let the library allocate device memory (a framework's caching
allocator owns the budget, or the caller cannot absorb cudaFree's device-wide
synchronisation).  It must give exactly what skolem_item_residues gives --
the path is integer, so "within tolerance" means identical -- on two calls in
a row (the static scratch keeps the previous call's contents), and refuse
counts beyond its fixed scratch.  Collected last so that a stop at the first
failure has run every other test already."""
import ctypes

import pytest

import oracle
import paper_1507_00315_gb300 as sk

pytestmark = pytest.mark.gpu


def _noalloc(variant, n, m, q_lo, count, primes):
    k = len(primes)
    P = (ctypes.c_uint64 * k)(*primes)
    out = (ctypes.c_uint64 * (count * k))()
    st = sk.lib().skolem_item_residues_noalloc(variant, n, m, q_lo, count, k, P, None, out)
    return st, [list(out[i * k:(i + 1) * k]) for i in range(count)]


@pytest.mark.parametrize("variant,n,m,q_lo,count,nprimes", [
    (0, 12, 9, 7, 1000, 3),        # Skolem, ragged count
    (1, 16, 9, 12345, 4096, 4),    # Langford, mid-size order, 4 moduli
])
def test_noalloc_matches_allocating_entry_point_twice(variant, n, m, q_lo, count, nprimes):
    primes = sk.default_primes()[:nprimes]
    want = sk.item_residues(variant, n, m, q_lo, count, primes)
    for _ in range(2):
        st, got = _noalloc(variant, n, m, q_lo, count, primes)
        assert st == sk.SK_OK
        assert got == want
    # and, independently of the allocating path, the CPU oracle's block sums
    # (Lemma 2.1's summand over each item) for the first, last and some
    # inner items
    for i in sorted({0, 1, count // 3, count // 2, count - 2, count - 1}):
        for j, p in enumerate(primes):
            assert got[i][j] == oracle.partial_sum_mod(variant, n, m, q_lo + i, p), (i, p)


def test_noalloc_different_calls_in_a_row():
    # a smaller call after a larger one must not see stale residues
    primes = sk.default_primes()[:3]
    st1, a = _noalloc(2, 14, 8, 0, 2048, primes)
    st2, b = _noalloc(0, 13, 8, 3, 17, primes)
    assert st1 == st2 == sk.SK_OK
    assert a == sk.item_residues(2, 14, 8, 0, 2048, primes)
    assert b == sk.item_residues(0, 13, 8, 3, 17, primes)


def test_noalloc_rejects_counts_beyond_its_scratch():
    primes = sk.default_primes()[:3]
    st, _ = _noalloc(0, 16, 6, 0, sk.NOALLOC_MAX_ITEMS + 1, primes)
    assert st == sk.SK_EINVAL
