"""Parity of the CUDA exact count with the CPU oracle (bit-exact), through
the C ABI.  Sizes: every order the oracle finishes in seconds, the paper's
printed values at the full sizes of the mid-size workload, and sampled work
items of those full-size launches recomputed one by one by the oracle."""
import os
import random

import pytest

import oracle
import paper_1507_00315_gb300 as sk

pytestmark = pytest.mark.gpu
SK, LA, HO = 0, 1, 2


ARITHS = [sk.ARITH_LIMBS, sk.ARITH_MONTGOMERY]


@pytest.mark.parametrize("arith", ARITHS)
@pytest.mark.parametrize("variant", [SK, LA, HO])
def test_small_orders_bit_exact_vs_backtracking(variant, arith):
    # Plain exact counts n = 1..12 (Skolem 4..12 and Langford 3..12 included).
    for n in range(1, 13):
        got, rep = sk.count_ex(variant, n, convention=sk.COUNT_ALL, arith=arith)
        want = oracle.backtrack_count(variant, n) if n <= 10 else oracle.coefficient(variant, n, threads=8)
        assert got == want, (variant, n, got, want)
        assert rep["complete"] and rep["terms"] == 1 << (2 * n - 1)


@pytest.mark.parametrize("arith", ARITHS)
@pytest.mark.parametrize("variant", [SK, LA, HO])
def test_residues_equal_oracle_sum(variant, arith):
    # H mod p of the whole half sum equals Algorithm 1's exact sum mod p.
    for n in (5, 9, 11):
        _, rep = sk.count_ex(variant, n, nprimes=4 if arith == sk.ARITH_LIMBS else 3, arith=arith)
        H = oracle.signed_sum(variant, n, half=True, threads=8)
        for p, r in zip(rep["primes"], rep["residues"]):
            assert r == H % p


def test_reflections_identified_convention(skolem_table, langford_table):
    for n, v in skolem_table.items():
        if n <= 13:
            assert sk.count(SK, n) == v
    for n, v in langford_table.items():
        if n <= 12:
            assert sk.count(LA, n) == v
    assert sk.count(SK, 1) == 1          # the palindrome 1,1


def test_zero_classes_up_to_16():
    for n in range(1, 17):
        if n % 4 in (2, 3):
            assert sk.count(SK, n) == 0
        if n % 4 in (1, 2):
            assert sk.count(LA, n) == 0
        if n % 4 in (0, 1):
            assert sk.count(HO, n) == 0


@pytest.mark.parametrize("variant,n", [(SK, 16), (SK, 17), (SK, 20), (LA, 16), (LA, 19), (LA, 20),
                                       (SK, 18), (SK, 19), (LA, 17), (LA, 18)])
def test_mid_size_against_paper(variant, n, skolem_table, langford_table):
    # Tables 7 / 8 at the mid-size workload (zeros from the existence classes).
    table = skolem_table if variant == SK else langford_table
    want = table.get(n, 0)
    got, rep = sk.count_ex(variant, n)
    assert got == want
    assert rep["complete"]


def test_mid_size_montgomery_form(skolem_table):
    assert sk.count_ex(SK, 20, arith=sk.ARITH_MONTGOMERY)[0] == skolem_table[20]


@pytest.mark.parametrize("arith", ARITHS)
@pytest.mark.parametrize("variant,n", [(SK, 16), (LA, 19), (HO, 18), (SK, 20)])
def test_sampled_items_at_full_size(variant, n, arith):
    # The full-size launch's own walk width; a few items recomputed by the
    # oracle one by one (first, last, random).
    _, rep = sk.count_ex(variant, n, arith=arith)
    m, items = rep["walk_bits"], rep["items"]
    if m > 18:
        pytest.skip("items too large for the oracle")
    primes = sk.default_primes()[:3]
    rng = random.Random(n)
    qs = sorted({0, items - 1, rng.randrange(items), rng.randrange(items)})
    for q in qs:
        got = sk.item_residues(variant, n, m, q, 1, primes, arith=arith)[0]
        want = [oracle.partial_sum_mod(variant, n, m, q, p) for p in primes]
        assert got == want, (q, got, want)


@pytest.mark.parametrize("variant", [SK, LA, HO])
def test_item_residues_ragged_tiles(variant):
    # many items per launch, a count that is not a multiple of 32 (ragged
    # last warp), several inner tiles per item
    n, m = 7, 7
    primes = [4611686017353646079, 4611686018427387847, 4611686018427387817]
    got = sk.item_residues(variant, n, m, 3, 61, primes)
    for i, q in enumerate(range(3, 64)):
        for j, p in enumerate(primes):
            assert got[i][j] == oracle.partial_sum_mod(variant, n, m, q, p)


@pytest.mark.parametrize("variant,n,m", [(SK, 24, 9), (LA, 24, 9), (HO, 26, 8), (SK, 28, 7),
                                         (LA, 28, 7), (HO, 21, 10), (SK, 29, 7), (LA, 30, 7),
                                         (HO, 31, 7), (SK, 31, 6), (LA, 31, 7)])
def test_large_orders_items_both_forms(variant, n, m):
    # the widest limb accumulators and the longest Montgomery chains, on
    # items small enough for the oracle (prefixes spread over the range)
    primes = sk.default_primes()[:4]
    F = 2 * n - 1
    for q in (0, (1 << (F - m)) - 1, 0x5A5A5A5A5A5 % (1 << (F - m))):
        a = sk.item_residues(variant, n, m, q, 1, primes, arith=sk.ARITH_LIMBS)[0]
        b = sk.item_residues(variant, n, m, q, 1, primes[:3], arith=sk.ARITH_MONTGOMERY)[0]
        want = [oracle.partial_sum_mod(variant, n, m, q, p) for p in primes]
        assert a == want and b == want[:3], (q, a, b, want)


def test_schedule_independence():
    # walk width, block size and grid change the schedule, not the residues
    base = sk.count_ex(SK, 13, nprimes=3)[1]["residues"]
    for kw in ({"walk_bits": 6}, {"walk_bits": 25}, {"block_threads": 64}, {"grid": 3},
               {"walk_bits": 9, "block_threads": 96, "grid": 7}, {"arith": sk.ARITH_MONTGOMERY},
               {"arith": sk.ARITH_MONTGOMERY, "walk_bits": 20, "block_threads": 128}):
        assert sk.count_ex(SK, 13, nprimes=3, **kw)[1]["residues"] == base, kw


def test_custom_primes_and_check_prime():
    # other primes of the accepted window (2^62 - 2^31, 2^62)
    primes = [4611686018427387751, 4611686018427387737, 4611686017353646079, 4611686016279916631]
    c, rep = sk.count_ex(LA, 12, nprimes=4, primes=primes)
    assert c == 108144
    assert rep["primes"] == primes


def test_invalid_arguments():
    for bad in ((3, 4), (SK, 0), (SK, 32), (-1, 5)):
        with pytest.raises(sk.SkolemError) as e:
            sk.count(*bad)
        assert e.value.status == sk.SK_EINVAL
    with pytest.raises(sk.SkolemError):
        sk.count_ex(SK, 8, primes=[4, 0, 0])
    with pytest.raises(sk.SkolemError):          # below the moduli window
        sk.count_ex(SK, 8, primes=[(1 << 61) - 1, 0, 0])
    with pytest.raises(sk.SkolemError):
        sk.count_ex(SK, 8, block_threads=100)
    with pytest.raises(sk.SkolemError):          # Montgomery form: three moduli
        sk.count_ex(SK, 8, nprimes=4, arith=sk.ARITH_MONTGOMERY)


def test_checkpoint_resume(tmp_path):
    path = str(tmp_path / "ck.txt")
    full, _ = sk.count_ex(SK, 13, convention=sk.COUNT_ALL)
    # stop after 3 chunks, then resume
    c1, r1 = sk.count_ex(SK, 13, convention=sk.COUNT_ALL, checkpoint=path, chunk_items=1 << 10,
                         walk_bits=9, max_chunks=3)
    assert c1 is None and r1["chunks_done"] == 3 and not r1["complete"]
    c2, r2 = sk.count_ex(SK, 13, convention=sk.COUNT_ALL, checkpoint=path, chunk_items=1 << 10,
                         walk_bits=9)
    assert c2 == full and r2["chunks_resumed"] == 3 and r2["complete"]
    # a torn last line (crash during a write) is ignored and redone
    with open(path, "a") as f:
        f.write("chunk 5 12")
    c3, r3 = sk.count_ex(SK, 13, convention=sk.COUNT_ALL, checkpoint=path, chunk_items=1 << 10,
                         walk_bits=9)
    assert c3 == full
    # a corrupted complete line is an error, not a wrong count
    lines = open(path).read().splitlines()
    lines[2] = lines[2].replace(lines[2].split()[2], str(int(lines[2].split()[2]) ^ 1), 1)
    open(path, "w").write("\n".join(lines) + "\n")
    with pytest.raises(sk.SkolemError) as e:
        sk.count_ex(SK, 13, convention=sk.COUNT_ALL, checkpoint=path, chunk_items=1 << 10, walk_bits=9)
    assert e.value.status == sk.SK_ECKPT
    # a checkpoint of another job is refused
    with pytest.raises(sk.SkolemError) as e:
        sk.count_ex(SK, 12, checkpoint=path, chunk_items=1 << 10, walk_bits=9)
    assert e.value.status == sk.SK_ECKPT


@pytest.mark.parametrize("variant", [SK, LA, HO])
def test_lemma_2_4_option_same_result_half_the_terms(variant):
    # Lemmas 2.2 + 2.4: the same residues H mod p and count as Lemma 2.2
    # alone; half the terms in the existence classes, none in the zero
    # classes; orders below 4 keep Lemma 2.2 alone.
    for n in range(1, 18):
        c0, r0 = sk.count_ex(variant, n, nprimes=4, convention=sk.COUNT_ALL)
        c1, r1 = sk.count_ex(variant, n, nprimes=4, convention=sk.COUNT_ALL,
                             symmetry=sk.SYMMETRY_NEGATION_EVEN)
        assert c1 == c0 and r1["residues"] == r0["residues"], (variant, n)
        if n < 4:
            assert r1["symmetry"] == sk.SYMMETRY_NEGATION and r1["terms"] == r0["terms"]
            continue
        assert r1["symmetry"] == sk.SYMMETRY_NEGATION_EVEN
        assert r1["terms"] == (r0["terms"] // 2 if c0 else 0), (variant, n)


def test_lemma_2_4_mid_size_against_the_paper(skolem_table, langford_table):
    for variant, n, table in ((SK, 20, skolem_table), (LA, 19, langford_table)):
        c, rep = sk.count_ex(variant, n, nprimes=4, symmetry=sk.SYMMETRY_NEGATION_EVEN)
        assert c == table[n] and rep["terms"] == 1 << (2 * n - 2)
    # a zero class of the same size costs nothing
    c, rep = sk.count_ex(SK, 19, symmetry=sk.SYMMETRY_NEGATION_EVEN)
    assert c == 0 and rep["terms"] == 0


def test_lemma_2_4_checkpoint(tmp_path):
    path = str(tmp_path / "ck24.txt")
    kw = dict(convention=sk.COUNT_ALL, chunk_items=1 << 8, walk_bits=9,
              symmetry=sk.SYMMETRY_NEGATION_EVEN)
    full, _ = sk.count_ex(HO, 14, convention=sk.COUNT_ALL)
    c1, r1 = sk.count_ex(HO, 14, checkpoint=path, max_chunks=3, **kw)
    assert c1 is None and r1["chunks_done"] == 3
    c2, r2 = sk.count_ex(HO, 14, checkpoint=path, **kw)
    assert c2 == full and r2["chunks_resumed"] == 3
    # the same order without Lemma 2.4 is another job
    with pytest.raises(sk.SkolemError) as e:
        sk.count_ex(HO, 14, convention=sk.COUNT_ALL, checkpoint=path, chunk_items=1 << 8,
                    walk_bits=9)
    assert e.value.status == sk.SK_ECKPT


@pytest.mark.parametrize("variant", [SK, LA, HO])
def test_every_order_one_item_vs_oracle(variant):
    # Each (delta, n) kernel has its own compile-time plan (grouping, tail or
    # digit form, product shape): one work item of every order 4..31, both
    # arithmetic forms, against the oracle's block sum.
    primes = sk.default_primes()[:4]
    for n in range(4, 32):
        F = 2 * n - 1
        m = min(9, F)
        q = (0x2D5A3C6B9E1F4 * (n + 7)) % (1 << (F - m))
        a = sk.item_residues(variant, n, m, q, 1, primes, arith=sk.ARITH_LIMBS)[0]
        b = sk.item_residues(variant, n, m, q, 1, primes[:3], arith=sk.ARITH_MONTGOMERY)[0]
        want = [oracle.partial_sum_mod(variant, n, m, q, p) for p in primes]
        assert a == want and b == want[:3], (variant, n, q, a, b, want)
