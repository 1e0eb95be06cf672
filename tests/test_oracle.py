"""Pins of the CPU oracle against what the paper and the mathematics fix.

None of these compares the oracle with itself: each pin is a printed value
(tests/golden, cited there), a closed form, a brute-force count by a second
method, or an invariant proved in the paper (Lemmas 2.1-2.4)."""
import math
import random

import numpy as np
import pytest

import oracle
from oracle import constructions as cons
from tests.conftest import read_golden

SK, LA, HO = 0, 1, 2


@pytest.mark.parametrize("variant", [SK, LA, HO])
def test_backtracking_equals_signed_sum(variant):
    # Two independent methods (Sec. 2 enumeration vs Lemma 2.1 / Algorithm 1).
    for n in range(1, 9):
        assert oracle.backtrack_count(variant, n) == oracle.coefficient(variant, n)


@pytest.mark.parametrize("variant", [SK, LA, HO])
def test_full_sum_is_twice_half_sum(variant):
    # Lemma 2.2: fixing the variable at max P to +1 halves the sum; and
    # Lemma 2.1: the full sum is 2^{2n} times the coefficient.
    for n in range(1, 7):
        full = oracle.signed_sum(variant, n, half=False)
        half = oracle.signed_sum(variant, n, half=True)
        assert full == 2 * half
        assert full == (1 << (2 * n)) * oracle.backtrack_count(variant, n)


def test_worked_example_n4():
    # Sec. 2.1: coefficient 6 of x_1..x_8 in F(4, X), and its six sequences.
    want = {tuple(int(v) for v in r) for r in read_golden("n4_skolem_sequences.txt")}
    got = set(oracle.backtrack_list(SK, 4))
    assert oracle.coefficient(SK, 4) == 6
    assert got == want


def test_printed_single_sequences():
    for r in read_golden("examples.txt"):
        variant, n, seq = int(r[0]), int(r[1]), [int(v) for v in r[2:]]
        assert cons.is_valid_sequence(seq, n, variant)
        assert tuple(seq) in set(oracle.backtrack_list(variant, n, 100000))


def test_skolem_pairs_example_n4():
    # Sec. 1.1: (7,8) (3,5) (1,4) (2,6) partition 1..8 with differences 1..4.
    seq = cons.pairs_to_sequence([(7, 8), (3, 5), (1, 4), (2, 6)], 8)
    assert seq == [3, 4, 2, 3, 2, 4, 1, 1]


@pytest.mark.parametrize("variant,table", [(SK, "skolem_A059106.txt"), (LA, "langford_A014552.txt")])
def test_tables_7_8_small_n(variant, table):
    # Tables 7/8 count reflections as one (A059106, A014552): coefficient / 2.
    vals = {int(r[0]): int(r[1]) for r in read_golden(table)}
    for n, v in vals.items():
        if n <= 9:
            assert oracle.backtrack_count(variant, n) == 2 * v
            assert oracle.coefficient(variant, n) == 2 * v


@pytest.mark.parametrize("variant,n", [(SK, 12), (LA, 11), (LA, 12)])
def test_tables_7_8_n11_12(variant, n, skolem_table, langford_table):
    want = (skolem_table if variant == SK else langford_table)[n]
    assert oracle.coefficient(variant, n, threads=8) == 2 * want


def test_tables_4_5_doubles(skolem_table, langford_table):
    # Sec. 1.3: no sequence is a palindrome for n > 1, so all = 2 x identified.
    for r in read_golden("all_sequences.txt"):
        variant, n, c = int(r[0]), int(r[1]), int(r[2])
        tab = skolem_table if variant == SK else langford_table
        assert c == 2 * tab[n]


def test_existence_classes_zero():
    # Skolem iff n = 0,1 (mod 4) (Sec. 1.1); Langford iff n = 0,3 (mod 4).
    # Hooked: zero for n = 0,1 (mod 4) (the Lemma 2.4 sign argument).
    for n in range(1, 12):
        if n % 4 in (2, 3):
            assert oracle.backtrack_count(SK, n) == 0
        else:
            assert oracle.backtrack_count(SK, n) > 0
        if n % 4 in (1, 2):
            assert oracle.backtrack_count(LA, n) == 0
        elif n >= 3:
            assert oracle.backtrack_count(LA, n) > 0
        if n % 4 in (0, 1):
            assert oracle.backtrack_count(HO, n) == 0
        else:
            assert oracle.backtrack_count(HO, n) > 0


def test_table1_skolem_construction():
    # Table 1: valid for k >= 2 (at n = 4, 5 the printed pairs collide).
    for n in [8, 9, 12, 13, 16, 17, 20, 21, 24, 25, 28, 29]:
        seq = cons.pairs_to_sequence(cons.skolem_table1(n), 2 * n)
        assert seq is not None and cons.is_valid_sequence(seq, n, SK)
        if n <= 9:
            assert tuple(seq) in set(oracle.backtrack_list(SK, n, 10000))


def test_table2_davies_construction():
    for n in [3, 4, 7, 8, 11, 12, 15, 16, 19, 20, 23, 24, 27, 28]:
        seq = cons.davies_table2(n)
        assert cons.is_valid_sequence(seq, n, LA), n
        if n <= 8:
            assert tuple(seq) in set(oracle.backtrack_list(LA, n, 10000))


def _rand_x(rng, span):
    return [0] + [rng.choice((-1, 1)) for _ in range(span)]


@pytest.mark.parametrize("variant", [SK, LA, HO])
def test_lemma_2_2_negation(variant):
    rng = random.Random(1)
    for n in (4, 5, 7, 8):
        span, _, _ = oracle.layout(variant, n)
        for _ in range(20):
            x = _rand_x(rng, span)
            assert oracle.summand(variant, n, x) == oracle.summand(variant, n, [0] + [-v for v in x[1:]])


@pytest.mark.parametrize("variant", [SK, LA])
def test_lemma_2_3_reversal(variant):
    rng = random.Random(2)
    for n in (4, 5, 7, 8, 9):
        span, _, _ = oracle.layout(variant, n)
        for _ in range(20):
            x = _rand_x(rng, span)
            assert oracle.summand(variant, n, x) == oracle.summand(variant, n, [0] + x[1:][::-1])


def test_lemma_2_4_even_negation():
    # Skolem, n = 0,1 (mod 4): summand unchanged when even positions negate;
    # otherwise it changes sign (so the sum vanishes: the zero classes).
    rng = random.Random(3)
    for n in (4, 5, 6, 7, 8, 9):
        span, _, _ = oracle.layout(SK, n)
        for _ in range(20):
            x = _rand_x(rng, span)
            y = [0] + [(-v if i % 2 == 0 else v) for i, v in enumerate(x[1:], start=1)]
            a, b = oracle.summand(SK, n, x), oracle.summand(SK, n, y)
            assert a == (b if n % 4 in (0, 1) else -b)


def _lemma_2_4_sign(variant, n):
    # (-1)^{#even positions in P + #odd distances d_k}
    _, pos, d = oracle.layout(variant, n)
    e = sum(1 for q in pos if q % 2 == 0)
    o = sum(1 for x in d if x % 2 == 1)
    return -1 if (e + o) % 2 else 1


@pytest.mark.parametrize("variant", [SK, LA, HO])
def test_lemma_2_4_sign_all_variants(variant):
    # Negating the even positions multiplies the summand by s: the
    # correlations at an odd distance change sign, those at an even distance
    # do not, and prod x changes by (-1)^{#even positions}.  s = +1 exactly in
    # the classes where pairings exist (Skolem 0,1, Langford 0,3, hooked 2,3
    # mod 4).
    rng = random.Random(5 + variant)
    exist = {SK: (0, 1), LA: (0, 3), HO: (2, 3)}[variant]
    for n in range(3, 13):
        s = _lemma_2_4_sign(variant, n)
        assert (s == 1) == (n % 4 in exist), (variant, n)
        span, _, _ = oracle.layout(variant, n)
        for _ in range(10):
            x = _rand_x(rng, span)
            y = [0] + [(-v if i % 2 == 0 else v) for i, v in enumerate(x[1:], start=1)]
            assert oracle.summand(variant, n, y) == s * oracle.summand(variant, n, x)


@pytest.mark.parametrize("variant,n", [(SK, 8), (SK, 9), (SK, 6), (LA, 7), (LA, 8), (LA, 5),
                                       (HO, 6), (HO, 7), (HO, 8)])
def test_lemma_2_4_fixed_variable(variant, n):
    # With x_{max P} = +1 (Lemma 2.2), also holding one more variable at +1 --
    # position 2n-1 (Skolem, Langford) or 2n-2 (hooked) -- and multiplying by
    # 1 + s gives the half sum: the blocks with that variable at -1 add up to
    # s times the others.
    p = (1 << 61) - 1
    s = _lemma_2_4_sign(variant, n)
    fixed_pos = 2 * n - 2 if variant == HO else 2 * n - 1
    m = 4
    hole = fixed_pos - 1 - m                 # bit of the block index q
    nfree = 2 * n - 1
    kept = dropped = 0
    for q in range(1 << (nfree - m)):
        v = oracle.partial_sum_mod(variant, n, m, q, p)
        if (q >> hole) & 1:
            dropped = (dropped + v) % p
        else:
            kept = (kept + v) % p
    half = oracle.signed_sum(variant, n, half=True) % p
    assert dropped == (s * kept) % p
    assert ((1 + s) * kept) % p == half


def test_summand_brute_expansion():
    # The summand is sign(X) * prod_i sum_k x_k x_{k+i}; check it against the
    # expansion of F(4, X) printed in Sec. 2.1 at random points.
    rng = random.Random(4)
    for _ in range(50):
        x = _rand_x(rng, 8)
        f1 = sum(x[k] * x[k + 1] for k in range(1, 8))
        f2 = sum(x[k] * x[k + 2] for k in range(1, 7))
        f3 = sum(x[k] * x[k + 3] for k in range(1, 6))
        f4 = sum(x[k] * x[k + 4] for k in range(1, 5))
        assert oracle.summand(SK, 4, x) == math.prod(x[1:]) * f1 * f2 * f3 * f4


@pytest.mark.parametrize("variant,n,m", [(SK, 5, 4), (LA, 7, 6), (HO, 6, 5), (SK, 8, 9)])
def test_blocks_sum_to_total_mod_p(variant, n, m):
    # The blocks partition the 2^{2n-1} assignments of the half sum.
    p = (1 << 61) - 1
    nfree = 2 * n - 1
    tot = 0
    for q in range(1 << (nfree - m)):
        tot = (tot + oracle.partial_sum_mod(variant, n, m, q, p)) % p
    assert tot == oracle.signed_sum(variant, n, half=True) % p


def test_philox_known_answers():
    for r in read_golden("philox_kat.txt"):
        v = [int(t, 16) for t in r]
        assert oracle.philox4x32_10(v[0:4], v[4:6]) == v[6:10]


@pytest.mark.parametrize("variant", [SK, LA])
def test_simplified_problem_counts(variant):
    # Sec. 3: Z(0) = (2n-1)!/(n-1)! configurations (Skolem); E = 0 exactly
    # for the pairings (counted by O1 with reflections distinct).
    for n in range(2, 7):
        N = oracle.simplified_energy_hist(variant, n)
        z0 = oracle.simplified_size(variant, n)
        assert int(N.sum()) == z0
        if variant == SK:
            assert z0 == math.factorial(2 * n - 1) // math.factorial(n - 1)
        else:
            assert z0 == math.factorial(2 * n - 2) // math.factorial(n - 2)
        assert int(N[0]) == oracle.backtrack_count(variant, n)


def test_table6_arithmetic():
    # Table 6 caption: (1/2)(23!/11!) prod E[z_{i+1}/z_i] = 227009.
    ratios = [float(r[5]) for r in read_golden("table6_pt_s12.txt")]
    est = 0.5 * math.factorial(23) / math.factorial(11) * math.prod(ratios)
    assert abs(est - 227009) < 1.0


@pytest.mark.parametrize("variant,n", [(SK, 4), (SK, 5), (LA, 4)])
def test_pt_estimator_against_exact_partition_function(variant, n):
    # Algorithm 2 at tiny n: per-rung statistics must follow the exact
    # Boltzmann weights N(E) e^{-beta E} / Z(beta), and the estimate must hit
    # the exact count.  Samples of one chain are correlated, so the spread is
    # taken from 16 independent runs (batch means): each run's per-rung
    # distribution and estimate is one sample.
    beta = np.array([0.0, 0.5, 1.0, 1.6, 2.4, 3.5, 5.0, 8.0])
    N = oracle.simplified_energy_hist(variant, n).astype(np.float64)
    E = np.arange(2 * n + 1)
    exact = oracle.backtrack_count(variant, n) / 2
    dists, ests = [], []
    for seed in range(100, 116):
        res = oracle.pt_run(variant, n, beta, ladders=2, iters=20000, burnin=2000, seed=seed)
        h = res["hist"].astype(np.float64)
        dists.append(h / h.sum(axis=1, keepdims=True))
        ests.append(oracle.pt_estimate_from_hist(res["hist"], beta, variant, n) / exact)
    dists, ests = np.array(dists), np.array(ests)
    se = dists.std(axis=0, ddof=1) / np.sqrt(len(dists))
    for j, b in enumerate(beta):
        p = N * np.exp(-b * E)
        p /= p.sum()
        assert np.all(np.abs(dists[:, j].mean(axis=0) - p) <= 5 * se[j] + 1e-3), (j, p)
    assert abs(ests.mean() - 1) <= max(5 * ests.std(ddof=1) / np.sqrt(len(ests)), 0.01)
    assert abs(ests.mean() - 1) < 0.03


def test_pt_deterministic_and_seed_dependent():
    beta = np.linspace(0, 4, 6)
    a = oracle.pt_run(SK, 5, beta, 2, 500, 0, 11, want_final=True)
    b = oracle.pt_run(SK, 5, beta, 2, 500, 0, 11, want_final=True)
    c = oracle.pt_run(SK, 5, beta, 2, 500, 0, 12, want_final=True)
    assert np.array_equal(a["hist"], b["hist"]) and np.array_equal(a["final_slots"], b["final_slots"])
    assert not np.array_equal(a["final_slots"], c["final_slots"])
    # each state's slots are legal start bins
    d = [k for k in range(1, 6)]
    assert np.all(a["final_slots"] < np.array([10 - dk for dk in d]))


def _zigzag_bounds(M, T):
    # With every exchange accepted (equal temperatures) the positions follow
    # the brick-wall permutation: each configuration walks to one end, waits
    # one iteration there, walks back, a zigzag of period 2M; so a ladder of
    # M configurations completes T / 2 round trips over T iterations, up to
    # one partial trip per configuration at each end of the run.
    return T // 2 - M - 2, T // 2 + 1


@pytest.mark.parametrize("M,T,burnin", [(2, 3, 0), (2, 4, 0), (2, 7, 0), (2, 200, 0), (2, 200, 51)])
def test_pt_round_trips_two_rungs_closed_form(M, T, burnin):
    # Two rungs at the same temperature: the pair (0, 1) is exchanged at every
    # even iteration, so the configurations trade places every two
    # iterations; the first return to rung 0 after visiting rung 1 is seen at
    # iteration 3, then one at every odd iteration.
    beta = [1.0, 1.0]
    r = oracle.pt_run(SK, 5, beta, 1, T, burnin, 3, want_trips=True)
    want = len([t for t in range(max(3, burnin), T) if t % 2 == 1])
    assert r["round_trips"] == want


@pytest.mark.parametrize("M", [1, 3, 5, 8])
def test_pt_round_trips_equal_temperatures(M):
    T, L = 1000, 3
    r = oracle.pt_run(LA, 6, [0.7] * M, L, T, 0, 9, want_trips=True)
    if M == 1:
        assert r["round_trips"] == 0
        return
    lo, hi = _zigzag_bounds(M, T)
    assert L * lo <= r["round_trips"] <= L * hi, (M, r["round_trips"])
    # counting the trips changes nothing else
    q = oracle.pt_run(LA, 6, [0.7] * M, L, T, 0, 9)
    assert np.array_equal(q["hist"], r["hist"]) and np.array_equal(q["acc_swap"], r["acc_swap"])
    assert q["round_trips"] is None


def test_pt_round_trips_frozen_ladder():
    # Temperatures so far apart that no exchange is ever accepted once the
    # cold rungs sit at low energy: nearly no configuration travels, far
    # below the zigzag's T / 2 per ladder.
    T = 2000
    r = oracle.pt_run(SK, 8, [0.0, 60.0, 120.0], 2, T, T // 2, 5, want_trips=True)
    assert r["round_trips"] < 0.05 * T
