"""Pins of the oracle's inclusion-exclusion count (Sec. 2, the third
counting approach, after Larsen): it must equal Miller's backtracking (O1)
for every variant at small n, the paper's tables at n = 9..11, and the sum of
its blocks must be the whole sum modulo a prime.  A wrong sign convention
(-1)^{|T|} instead of (-1)^{|S|}, a pair counted with one end outside T, or
a dropped position would fail these."""
import pytest

import oracle

P = 4611686018427387847


@pytest.mark.parametrize("variant", [0, 1, 2])
def test_ie_equals_backtracking(variant):
    for n in range(1, 10):
        assert oracle.ie_count(variant, n) == oracle.backtrack_count(variant, n), n


def test_ie_worked_example_and_tables(skolem_table, langford_table):
    # F(4, X) of Sec. 2.1 has coefficient 6: the six Skolem sequences of order 4
    assert oracle.ie_count(0, 4) == 6
    # Tables 7 / 8 identify a sequence with its reflection
    for n in (9, 10, 11):
        assert oracle.ie_count(0, n) == 2 * skolem_table.get(n, 0), n
        assert oracle.ie_count(1, n) == 2 * langford_table.get(n, 0), n


@pytest.mark.parametrize("variant,n,m", [(0, 5, 4), (1, 5, 6), (2, 6, 7), (0, 4, 0), (1, 3, 6)])
def test_ie_blocks_add_up(variant, n, m):
    total = sum(oracle.ie_partial_sum_mod(variant, n, m, q, P) for q in range(1 << (2 * n - m)))
    assert total % P == oracle.ie_count(variant, n) % P


def test_ie_block_arguments():
    with pytest.raises(ValueError):
        oracle.ie_partial_sum_mod(0, 5, 4, 1 << 6, P)      # q beyond the 2n - m fixed variables
    with pytest.raises(ValueError):
        oracle.ie_partial_sum_mod(0, 5, 11, 0, P)           # more walk variables than positions
