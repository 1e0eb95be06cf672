"""The exact count of a sum computed in parts (work-item ranges on different
GPUs): sk_count_from_residues adds the parts' residues modulo each prime and
rebuilds the count by the CRT with skolem_count_ex's checks (Lemma 2.1,
Lemma 2.2, Sec. 2.2's sums modulo co-primes).  Host code only: the item sums
here come from the oracle, and two gloo ranks stand in for two GPUs."""
import os
import sys

import numpy as np
import pytest

import oracle
import paper_1507_00315_gb300 as sk

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PRIMES = sk.default_primes()


def _items(variant, n):
    F = 2 * n - 1                          # free variables after Lemma 2.2
    m = max(0, F - 3)
    return m, 1 << (F - m)


def _item_residues(variant, n, m, qs):
    return [[oracle.partial_sum_mod(variant, n, m, q, p) for p in PRIMES] for q in qs]


def _add(rows):
    return [sum(r[i] for r in rows) % PRIMES[i] for i in range(len(PRIMES))]


@pytest.mark.parametrize("variant,n", [(0, 1), (0, 4), (0, 5), (0, 6), (0, 8), (1, 3), (1, 4),
                                       (1, 7), (1, 8), (2, 2), (2, 3), (2, 6), (2, 7)])
def test_parts_add_up_to_the_count(variant, n):
    m, nitems = _items(variant, n)
    rows = _item_residues(variant, n, m, range(nitems))
    rng = np.random.default_rng(variant * 100 + n)
    owner = rng.integers(0, 3, nitems)                     # three "GPUs", uneven shares
    parts = [_add([rows[q] for q in range(nitems) if owner[q] == g] or [[0] * len(PRIMES)])
             for g in range(3)]
    want_all = oracle.backtrack_count(variant, n)
    assert sk.count_from_residues(variant, n, parts, PRIMES, sk.COUNT_ALL) == want_all
    ident = want_all if variant == 2 else (1 if (variant, n) == (0, 1) else want_all // 2)
    assert sk.count_from_residues(variant, n, parts, PRIMES) == ident
    assert sk.count_from_residues(variant, n, rows, PRIMES, sk.COUNT_ALL) == want_all


def test_bad_parts_are_caught():
    variant, n = 0, 8
    m, nitems = _items(variant, n)
    rows = _item_residues(variant, n, m, range(nitems))
    assert sk.count_from_residues(variant, n, rows, PRIMES) == 252          # Table 7
    bad = [list(r) for r in rows]
    bad[3][1] = (bad[3][1] + 1) % PRIMES[1]                                # one corrupted residue
    with pytest.raises(sk.SkolemError) as e:
        sk.count_from_residues(variant, n, bad, PRIMES)
    assert e.value.status == sk.SK_EMISMATCH
    # a part added twice passes every check (each item sum is a multiple of
    # 2^{2n-1} here): covering the items exactly once is the caller's part
    assert all(oracle.partial_sum_mod(variant, n, m, 0, p) == rows[0][i] for i, p in enumerate(PRIMES))
    assert sk.count_from_residues(variant, n, rows + rows[:1], PRIMES) != 252


def test_argument_checks():
    row = [[0] * 4]
    for args, kw in (((3, 4, row, PRIMES), {}), ((0, 0, row, PRIMES), {}),
                     ((0, 4, [[PRIMES[0], 0, 0, 0]], PRIMES), {}),
                     ((0, 4, row, PRIMES), {"convention": 7}),
                     ((0, 4, [[0, 0]], [3, 5]), {})):
        with pytest.raises(sk.SkolemError) as e:
            sk.count_from_residues(*args, **kw)
        assert e.value.status == sk.SK_EINVAL


def _rank(rank, world, port, variant, n, out):
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        m, nitems = _items(variant, n)
        mine = _add(_item_residues(variant, n, m, range(rank, nitems, world)))
        parts = [None] * world
        dist.all_gather_object(parts, mine)                   # the one exchange step
        out.put((rank, sk.count_from_residues(variant, n, parts, PRIMES, sk.COUNT_ALL)))
    finally:
        dist.destroy_process_group()


def test_two_ranks_combine_their_shares():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = 29600 + os.getpid() % 1000
    procs = [ctx.Process(target=_rank, args=(r, 2, port, 1, 8, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = dict(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert res[0] == res[1] == oracle.backtrack_count(1, 8)                 # 300 (Table 8: 150)


@pytest.mark.parametrize("variant,n", [(0, 24), (0, 25), (0, 28), (0, 29), (1, 27), (1, 28)])
def test_crt_range_at_the_largest_printed_orders(variant, n, skolem_table, langford_table):
    # The host step at the largest orders the paper counts exactly (Tables 7
    # and 8, up to S(29) and L(28)): the signed sum of Lemma 2.1 after
    # Lemma 2.2 is H = 2 C 2^{2n-1} (C the printed count, reflections
    # identified), |H| < 2^{135} at S(29), far inside the three moduli's
    # range M ~ 2^{186}.  Its residues, as one part, must rebuild C exactly
    # (the 2n-1 low bits vanish, the quotient is the count), a fourth
    # modulus must agree, and a residue off by one modulo any prime must be
    # caught.
    C = (skolem_table if variant == 0 else langford_table)[n]
    H = 2 * C << (2 * n - 1)
    assert H < 1 << 135
    res = [H % p for p in PRIMES]
    assert sk.count_from_residues(variant, n, [res], PRIMES) == C
    assert sk.count_from_residues(variant, n, [res[:3]], PRIMES[:3]) == C
    assert sk.count_from_residues(variant, n, [res], PRIMES, sk.COUNT_ALL) == 2 * C
    for i in range(4):
        bad = list(res)
        bad[i] = (bad[i] + 1) % PRIMES[i]
        with pytest.raises(sk.SkolemError) as e:
            sk.count_from_residues(variant, n, [bad], PRIMES)
        assert e.value.status == sk.SK_EMISMATCH
