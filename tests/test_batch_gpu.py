"""The persistent batched sweep (one graph-captured launch over many uneven
jobs) against the per-job launches and the oracle, bit-exact; the
autotuner's choice is a valid configuration and does not change results."""
import pytest

import oracle
import paper_1507_00315_gb300 as sk

pytestmark = pytest.mark.gpu

SMALL = [(v, n) for v in (0, 1, 2) for n in range(1, 13)]


def test_batch_small_all_variants_vs_oracle():
    counts, stat, rep = sk.count_batch(SMALL, convention=sk.COUNT_ALL)
    assert all(s == 0 for s in stat)
    for (v, n), c in zip(SMALL, counts):
        want = oracle.backtrack_count(v, n) if n <= 10 else oracle.coefficient(v, n, threads=8)
        assert c == want, (v, n, c, want)
    assert rep["launches"] == 1 and rep["terms"] == sum(1 << (2 * n - 1) for _, n in SMALL)


@pytest.mark.parametrize("kw", [{}, {"no_graph": True}, {"mode": sk.BATCH_PER_JOB},
                                {"block_threads": 128, "repeats": 2},
                                {"walk_bits": {16: 8, 17: 18}, "nprimes": 4}])
def test_batch_modes_agree(kw, skolem_table, langford_table):
    jobs = [(0, 16), (1, 16), (2, 15), (0, 17), (1, 15), (0, 13), (2, 5), (1, 4), (0, 1)]
    counts, stat, rep = sk.count_batch(jobs, **kw)
    assert all(s == 0 for s in stat)
    singles = [sk.count(v, n) for v, n in jobs]
    assert counts == singles
    assert counts[0] == skolem_table[16] and counts[1] == langford_table[16]
    if kw.get("mode") == sk.BATCH_PER_JOB:
        assert rep["launches"] == len(jobs)


def test_batch_duplicate_and_unsorted_jobs():
    jobs = [(0, 8), (0, 12), (0, 8), (1, 11), (0, 12)]
    counts, _, _ = sk.count_batch(jobs)
    assert counts == [252, 227968, 252, 17792, 227968]


def test_autotune_then_batch():
    r = sk.autotune(0, 18)
    assert r["candidates"] >= 2 and r["terms_per_s"] > 0
    assert r["block_threads"] in (128, 256)
    counts, stat, _ = sk.count_batch([(0, 18), (1, 19), (0, 17)], autotune=True)
    assert counts == [0, 256814891280, 6124491248]


def test_batch_invalid():
    with pytest.raises(sk.SkolemError):
        sk.count_batch([(0, sk.MAX_N + 1)])      # beyond the compiled orders
    with pytest.raises(sk.SkolemError):
        sk.count_batch([])
