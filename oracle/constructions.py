"""Explicit constructions of Sec. 1.1 -- TEST INFRASTRUCTURE ONLY.

Skolem's construction (Table 1) for n = 4k and n = 4k+1, and Davies'
construction (Table 2) of a Langford sequence for n = 4k-1 and n = 4k, plus a
validator.  Readings:
  * Table 1, n = 4k, the last family "(k+2+r, 3k-1-r) 0,...,k-3" runs over
    r = 0..k-3.
  * Table 2, "a, ..., b" is the run a, a-2, ..., b (or a, a+2, ..., b when
    a < b in the general pattern); when the run's end points cross for a
    small k the run is empty.
"""
from __future__ import annotations


def _run(a: int, b: int, descending: bool):
    """a, ..., b in steps of 2 in the stated direction; empty if crossed."""
    if descending:
        return list(range(a, b - 1, -2)) if a >= b else []
    return list(range(a, b + 1, 2)) if a <= b else []


def skolem_table1(n: int):
    """Pairs (a_r, b_r) of Table 1 (Skolem, n = 4k or 4k+1)."""
    pairs = []
    if n % 4 == 0:
        k = n // 4
        pairs += [(4 * k + r, 8 * k - r) for r in range(0, 2 * k)]
        pairs += [(2 * k + 1, 6 * k), (2 * k, 4 * k - 1)]
        pairs += [(r, 4 * k - 1 - r) for r in range(1, k)]
        pairs += [(k, k + 1)]
        pairs += [(k + 2 + r, 3 * k - 1 - r) for r in range(0, k - 2)]
    elif n % 4 == 1:
        k = n // 4
        pairs += [(4 * k + 2 + r, 8 * k + 2 - r) for r in range(0, 2 * k)]
        pairs += [(2 * k + 1, 6 * k + 2), (2 * k + 2, 4 * k + 1)]
        pairs += [(r, 4 * k + 1 - r) for r in range(1, k + 1)]
        pairs += [(k + 1, k + 2)]
        pairs += [(k + 2 + r, 3 * k + 1 - r) for r in range(1, k - 1)]
    else:
        raise ValueError("Table 1 covers n = 0, 1 (mod 4) only")
    return pairs


def pairs_to_sequence(pairs, span: int):
    """Label each position with the difference of the pair covering it."""
    seq = [0] * span
    for a, b in pairs:
        for p in (a, b):
            if not 1 <= p <= span or seq[p - 1]:
                return None                       # out of range or overlap
            seq[p - 1] = b - a
    return seq


def davies_table2(n: int):
    """Langford sequence of Table 2 (n = 4k-1 or 4k), as a list of labels."""
    if n % 4 == 3:
        k = (n + 1) // 4
        s = (_run(4 * k - 4, 2 * k, True) + [4 * k - 2] + _run(2 * k - 3, 1, True) + [4 * k - 1]
             + _run(1, 2 * k - 3, False) + _run(2 * k, 4 * k - 4, False) + [2 * k - 1]
             + _run(4 * k - 3, 2 * k + 1, True) + [4 * k - 2] + _run(2 * k - 2, 2, True)
             + [2 * k - 1, 4 * k - 1] + _run(2, 2 * k - 2, False) + _run(2 * k + 1, 4 * k - 3, False))
    elif n % 4 == 0:
        k = n // 4
        s = (_run(4 * k - 4, 2 * k, True) + [4 * k - 2] + _run(2 * k - 3, 1, True) + [4 * k - 1]
             + _run(1, 2 * k - 3, False) + _run(2 * k, 4 * k - 4, False) + [4 * k]
             + _run(4 * k - 3, 2 * k + 1, True) + [4 * k - 2] + _run(2 * k - 2, 2, True)
             + [2 * k - 1, 4 * k - 1] + _run(2, 2 * k - 2, False) + _run(2 * k + 1, 4 * k - 3, False)
             + [2 * k - 1, 4 * k])
    else:
        raise ValueError("Table 2 covers n = 0, 3 (mod 4) only")
    return s


def is_valid_sequence(seq, n: int, variant: int) -> bool:
    """True iff seq (labels per position, 0 = the hooked gap) places each
    k = 1..n exactly twice at distance d_k (k, k+1 for Langford) and fills
    every position of P (Sec. 1.1, 1.2)."""
    span = 2 * n + 1 if variant == 2 else 2 * n
    if len(seq) != span:
        return False
    where = {}
    for i, v in enumerate(seq, start=1):
        if variant == 2 and i == 2 * n:
            if v != 0:
                return False
            continue
        if not 1 <= v <= n:
            return False
        where.setdefault(v, []).append(i)
    for k in range(1, n + 1):
        p = where.get(k, [])
        if len(p) != 2:
            return False
        dk = k + 1 if variant == 1 else k
        if p[1] - p[0] != dk:
            return False
    return True
