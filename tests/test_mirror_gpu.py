"""The exact count with Lemma 2.3 (reversal) on top of Lemma 2.2
(SK_SYMMETRY_REVERSAL, csrc/sk_mirror.cuh): one of each pair of mirror-image
work items evaluated with weight 2, palindromic ones once.  The residues of
the whole sum must be the very residues of the plain half-sum (the two sums
are equal integers), the counts those of the tables, for every walk width
and schedule; about half the terms are evaluated."""
import pytest

import oracle
import paper_1507_00315_gb300 as sk

pytestmark = pytest.mark.gpu
SK, LA = sk.SKOLEM, sk.LANGFORD
REV = sk.SYMMETRY_REVERSAL


@pytest.mark.parametrize("variant", [SK, LA])
def test_same_residues_as_the_half_sum(variant):
    for n in range(1, 18):
        c0, r0 = sk.count_ex(variant, n, nprimes=4, convention=sk.COUNT_ALL)
        c1, r1 = sk.count_ex(variant, n, nprimes=4, convention=sk.COUNT_ALL, symmetry=REV)
        assert c1 == c0 and r1["residues"] == r0["residues"], n
        if n <= 9:
            assert c1 == oracle.backtrack_count(variant, n)
        if n >= 6:
            # the walk covers bits 1..h and their mirror images (h at least
            # the unrolled width), and of the middle's mirror pairs the
            # outermost min(8, pairs) decide: (1/2 + 2^-(depth+1)) of the
            # terms, all of them when no middle pair is left (n = 6)
            assert r1["symmetry"] == REV
            pairs = n - 1 - r1["walk_bits"] // 2
            depth = min(8, pairs)
            assert r1["terms"] <= (0.5 + 2.0 ** -(depth + 1)) * r0["terms"], (n, r1, r0)
            if n >= 12:
                assert r1["terms"] < 0.6 * r0["terms"], (n, r1["terms"], r0["terms"])
        else:
            assert r1["symmetry"] == sk.SYMMETRY_NEGATION


@pytest.mark.parametrize("variant,n", [(SK, 20), (LA, 20), (LA, 19)])
def test_full_size_against_the_tables(variant, n, skolem_table, langford_table):
    c, rep = sk.count_ex(variant, n, symmetry=REV)
    assert c == (skolem_table if variant == SK else langford_table)[n]
    assert rep["symmetry"] == REV


@pytest.mark.parametrize("variant", [SK, LA])
def test_reversal_and_lemma_2_4_together(variant, skolem_table, langford_table):
    # Lemmas 2.2, 2.3 and 2.4: zero outside the existence classes, else the
    # x_1 = +1 mirrored items doubled -- the same residues as the plain
    # half-sum, about a quarter of its terms
    both = sk.SYMMETRY_REVERSAL_EVEN
    for n in range(1, 18):
        c0, r0 = sk.count_ex(variant, n, nprimes=4, convention=sk.COUNT_ALL)
        c1, r1 = sk.count_ex(variant, n, nprimes=4, convention=sk.COUNT_ALL, symmetry=both)
        assert c1 == c0 and r1["residues"] == r0["residues"], n
        if n >= 6:
            assert r1["symmetry"] == both
            if c0:
                pairs = n - 1 - r1["walk_bits"] // 2
                frac = (0.5 + 2.0 ** -(min(8, pairs) + 1)) / 2
                assert r1["terms"] <= frac * r0["terms"] + 1, (n, r1["terms"], r0["terms"])
            else:
                assert r1["terms"] == 0
    n = 20
    c, rep = sk.count_ex(variant, n, symmetry=both)
    assert c == (skolem_table if variant == SK else langford_table).get(n, 0)


def test_walk_widths_and_schedules():
    base = sk.count_ex(LA, 14, nprimes=3)[1]["residues"]
    U = sk.count_plan(LA, 14)["inner_bits"]
    for kw in ({"walk_bits": 2 * U}, {"walk_bits": 2 * U + 2}, {"walk_bits": 20},
               {"block_threads": 64}, {"grid": 5}, {"walk_bits": 14, "block_threads": 96, "grid": 7}):
        r = sk.count_ex(LA, 14, nprimes=3, symmetry=REV, **kw)[1]
        assert r["residues"] == base, kw


def test_checkpoint_resume(tmp_path):
    path = str(tmp_path / "rev.ckpt")
    c0, r0 = sk.count_ex(SK, 13, symmetry=REV, checkpoint=path, chunk_items=300, max_chunks=2)
    assert c0 is None and r0["chunks_done"] == 2
    c1, r1 = sk.count_ex(SK, 13, symmetry=REV, checkpoint=path, chunk_items=300)
    assert c1 == sk.count(SK, 13) and r1["chunks_resumed"] == 2
    with pytest.raises(sk.SkolemError) as e:            # another symmetry: another job
        sk.count_ex(SK, 13, checkpoint=path, chunk_items=300)
    assert e.value.status == sk.SK_ECKPT
