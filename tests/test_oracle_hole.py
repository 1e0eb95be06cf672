"""Pins of the oracle for extended Skolem sequences (Sec. 1.2: the hook may
sit anywhere): positions 1..2n+1 except one hole, pairs of k at distance k.
Backtracking against brute force over every placement at tiny n, the
special holes against the other problems (hole 2n+1 or 1: Skolem; hole 2n
or 2: hooked), the mirror symmetry hole -> 2n+2-hole, Algorithm 1 on the same
position set against backtracking, and the blocks adding up to the
half-sum."""
import itertools

import pytest

import oracle

P = 4611686018427387847


def _brute(n, hole):
    # every choice of a start for each pair, kept when the 2n occupied
    # positions are exactly {1..2n+1} minus the hole
    want = set(range(1, 2 * n + 2)) - {hole}
    count = 0
    for starts in itertools.product(*[range(1, 2 * n + 2 - k) for k in range(1, n + 1)]):
        used = []
        for k, a in zip(range(1, n + 1), starts):
            used += [a, a + k]
        if len(set(used)) == 2 * n and set(used) == want:
            count += 1
    return count


def test_backtracking_equals_brute_force():
    for n in range(1, 6):
        for hole in range(1, 2 * n + 2):
            assert oracle.backtrack_count_hole(n, hole) == _brute(n, hole), (n, hole)


def test_special_holes_and_mirror_symmetry():
    for n in range(1, 10):
        assert oracle.backtrack_count_hole(n, 2 * n + 1) == oracle.backtrack_count(0, n)
        assert oracle.backtrack_count_hole(n, 1) == oracle.backtrack_count(0, n)
        assert oracle.backtrack_count_hole(n, 2 * n) == oracle.backtrack_count(2, n)
        for hole in range(1, 2 * n + 2):
            assert oracle.backtrack_count_hole(n, hole) == \
                oracle.backtrack_count_hole(n, 2 * n + 2 - hole), (n, hole)


def test_algorithm_1_on_the_same_position_set():
    for n in range(1, 9):
        for hole in range(1, 2 * n + 2):
            assert oracle.coefficient_hole(n, hole) == oracle.backtrack_count_hole(n, hole), (n, hole)


@pytest.mark.parametrize("n,hole,m", [(5, 6, 4), (6, 9, 5), (7, 3, 6), (6, 13, 3)])
def test_blocks_add_up(n, hole, m):
    nfree = 2 * n - 1
    total = sum(oracle.partial_sum_mod_hole(n, hole, m, q, P) for q in range(1 << (nfree - m)))
    half = oracle.coefficient_hole(n, hole) << (2 * n - 1)
    assert total % P == half % P
