"""Extended Skolem sequences on the GPU (sk_count_extended, Sec. 1.2: one
hole anywhere in 1..2n+1, pairs of k at distance k; hole n+1 is Rosa's
problem, 2n the hooked one) against the oracle's backtracking on the same
position set, the special holes against the Skolem and hooked counts, and
single work items against the oracle's block sums -- bit-exact."""
import pytest

import oracle
import paper_1507_00315_gb300 as sk

pytestmark = pytest.mark.gpu


def test_every_hole_small_orders():
    for n in range(1, 11):
        for hole in range(1, 2 * n + 2):
            want = oracle.backtrack_count_hole(n, hole)
            try:
                got, rep = sk.count_extended(n, hole, convention=sk.COUNT_ALL, nprimes=4)
            except sk.SkolemError as e:
                # a hole (mirrored into the upper half) inside the unrolled
                # inner block of the walk: only tiny orders
                assert e.status == sk.SK_EINVAL and n <= 4 and 3 <= hole <= 2 * n - 1, (n, hole)
                continue
            assert got == want, (n, hole, got, want)
            assert rep["terms"] == 2 ** (2 * n - 1)


def test_special_holes_and_conventions(skolem_table):
    for n in (12, 13, 16, 17):
        assert sk.count_extended(n, 2 * n + 1)[0] == skolem_table.get(n, 0)     # Skolem
        assert sk.count_extended(n, 1)[0] == skolem_table.get(n, 0)
        h = sk.count(sk.HOOKED, n)
        assert sk.count_extended(n, 2 * n)[0] == h and sk.count_extended(n, 2)[0] == h
        rosa_all = sk.count_extended(n, n + 1, convention=sk.COUNT_ALL)[0]
        assert sk.count_extended(n, n + 1)[0] * 2 == rosa_all      # reflections identified
        if n <= 12:
            assert rosa_all == oracle.backtrack_count_hole(n, n + 1)


@pytest.mark.parametrize("n,hole,m", [(14, 15, 9), (16, 20, 10), (18, 33, 9), (20, 27, 12),
                                      (20, 40, 9), (24, 30, 8)])
def test_items_equal_the_oracle_blocks(n, hole, m):
    primes = sk.default_primes()[:4]
    nitems = 1 << (2 * n - 1 - m)
    for q_lo, cnt in ((0, 33), (nitems - 3, 3), ((0x9E3779B97F4A7C15 * hole) % (nitems - 40), 40)):
        got = sk.extended_item_residues(n, hole, m, q_lo, cnt, primes)
        for i in sorted({0, cnt // 2, cnt - 1}):
            want = [oracle.partial_sum_mod_hole(n, hole, m, q_lo + i, p) for p in primes]
            assert got[i] == want, (n, hole, q_lo + i)


def test_refusals():
    for args, kw in (((12, 0), {}), ((12, 26), {}), ((12, 13), {"symmetry": sk.SYMMETRY_NEGATION_EVEN}),
                     ((12, 13), {"walk_bits": 13})):       # the hole (bit 12) inside the walk
        with pytest.raises(sk.SkolemError) as e:
            sk.count_extended(*args, **kw)
        assert e.value.status == sk.SK_EINVAL, (args, kw)
    with pytest.raises(sk.SkolemError) as e:
        sk.extended_item_residues(12, 8, 9, 0, 1, sk.default_primes()[:3])   # a lower hole
    assert e.value.status == sk.SK_EINVAL
