"""The inclusion-exclusion count on the GPU (Sec. 2, the third counting
approach, after Larsen; sk_count_inclusion_exclusion, sk_ie_item_residues)
against the CPU oracle's inclusion-exclusion sum (itself pinned to
backtracking), against the paper's tables, and against the algebraic count
of Lemma 2.1 -- bit-exact, since the arithmetic is integer."""
import pytest

import oracle
import paper_1507_00315_gb300 as sk

pytestmark = pytest.mark.gpu
SK, LA, HO = sk.SKOLEM, sk.LANGFORD, sk.HOOKED


@pytest.mark.parametrize("variant", [SK, LA, HO])
def test_small_orders_equal_the_oracle(variant):
    for n in range(1, 11):
        got, rep = sk.count_inclusion_exclusion(variant, n, convention=sk.COUNT_ALL)
        assert got == oracle.ie_count(variant, n) == oracle.backtrack_count(variant, n), n
        assert rep["terms"] == 1 << (2 * n) and rep["complete"]


def test_tables_and_the_algebraic_count(skolem_table, langford_table):
    # Tables 7 / 8 (reflections identified, zeros included) at n = 11..18,
    # and the same residue-built integer as Lemma 2.1's count
    for n in range(11, 19):
        for variant, table in ((SK, skolem_table), (LA, langford_table)):
            got, rep = sk.count_inclusion_exclusion(variant, n, nprimes=4)
            assert got == table.get(n, 0), (variant, n)
            assert got == sk.count_ex(variant, n)[0]
        h_ie = sk.count_inclusion_exclusion(HO, n, convention=sk.COUNT_ALL)[0]
        assert h_ie == sk.count_ex(HO, n, convention=sk.COUNT_ALL)[0], n


@pytest.mark.parametrize("variant,n", [(SK, 20), (LA, 20)])
def test_full_size_against_the_table(variant, n, skolem_table, langford_table):
    # 2^40 terms, the same order as the largest job of the mid-size workload
    got, rep = sk.count_inclusion_exclusion(variant, n)
    assert got == (skolem_table if variant == SK else langford_table)[n]
    assert rep["terms"] == 1 << 40


@pytest.mark.parametrize("variant,n,m", [(SK, 12, 9), (LA, 16, 8), (HO, 17, 8), (SK, 20, 7),
                                         (LA, 24, 6), (HO, 24, 6)])
def test_items_equal_the_oracle_blocks(variant, n, m):
    # first, last and scattered items, ragged count; items of every order
    # run the same compile-time walk as the full counts
    primes = sk.default_primes()[:4]
    nitems = 1 << (2 * n - m)
    for q_lo, cnt in ((0, 37), (nitems - 5, 5), ((0x9E3779B97F4A7C15 * n) % (nitems - 64), 64)):
        got = sk.ie_item_residues(variant, n, m, q_lo, cnt, primes)
        for i in sorted({0, cnt // 2, cnt - 1}):
            want = [oracle.ie_partial_sum_mod(variant, n, m, q_lo + i, p) for p in primes]
            assert got[i] == want, (q_lo + i, got[i], want)


def test_schedule_independence():
    base = sk.count_inclusion_exclusion(LA, 12, nprimes=4)[1]["residues"]
    for kw in ({"walk_bits": 5}, {"walk_bits": 13}, {"block_threads": 64}, {"grid": 3},
               {"walk_bits": 9, "block_threads": 96, "grid": 7}):
        assert sk.count_inclusion_exclusion(LA, 12, nprimes=4, **kw)[1]["residues"] == base, kw


def test_checkpoint_resume(tmp_path):
    path = str(tmp_path / "ie.ckpt")
    c0, r0 = sk.count_inclusion_exclusion(SK, 13, checkpoint=path, chunk_items=1000,
                                           walk_bits=10, max_chunks=3)
    assert c0 is None and r0["chunks_done"] == 3
    c1, r1 = sk.count_inclusion_exclusion(SK, 13, checkpoint=path, chunk_items=1000, walk_bits=10)
    assert c1 == sk.count(SK, 13) and r1["chunks_resumed"] == 3
    # the algebraic count must not take the inclusion-exclusion file as its own
    with pytest.raises(sk.SkolemError) as e:
        sk.count_ex(SK, 13, checkpoint=path, chunk_items=1000, walk_bits=10)
    assert e.value.status == sk.SK_ECKPT
