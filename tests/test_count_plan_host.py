"""The exact count's plan without a device (sk_count_plan): work items, walk
width, terms after Lemma 2.2 / Lemma 2.4, the zero classes Lemma 2.4's sign
finds, and the chunks of a checkpointed run (two of them pinned by recorded
GPU runs: L(23) in 2 chunks of 2^22 items at 21 walk bits and S(25) in 512 at
17, both with Lemma 2.4)."""
import pytest

import paper_1507_00315_gb300 as sk

NEG_EVEN = sk.SYMMETRY_NEGATION_EVEN


@pytest.mark.parametrize("variant", [0, 1, 2])
@pytest.mark.parametrize("n", [1, 2, 3, 4, 5, 8, 12, 16, 20, 21, 24, 28, 29, 30, 31])
def test_plan_covers_the_half_sum(variant, n):
    r = sk.count_plan(variant, n)
    assert r["terms"] == 2 ** (2 * n - 1)                    # Lemma 2.2: x at max P fixed
    assert r["items"] << r["walk_bits"] == r["terms"]
    assert r["inner_bits"] <= r["walk_bits"] <= 2 * n - 1
    assert r["chunks_total"] == 1 and r["symmetry"] == sk.SYMMETRY_NEGATION
    assert r["nprimes"] == 3 and r["primes"][:3] == sk.default_primes()[:3]


@pytest.mark.parametrize("variant", [0, 1, 2])
@pytest.mark.parametrize("n", range(4, 17))
def test_lemma_2_4_plan(variant, n):
    r = sk.count_plan(variant, n, symmetry=NEG_EVEN)
    assert r["symmetry"] == NEG_EVEN
    # existence classes (Sec. 1.1): Skolem n = 0, 1, Langford n = 0, 3, hooked
    # n = 2, 3 (mod 4); outside them the lemma's sign is -1: nothing to sum
    exists = n % 4 in ((0, 1), (0, 3), (2, 3))[variant]
    if not exists:
        assert r["terms"] == 0 and r["items"] == 0 and r["complete"] == 1
    else:
        assert r["terms"] == 2 ** (2 * n - 2) and r["items"] << r["walk_bits"] == r["terms"]


def test_checkpoint_chunks():
    ck = {"checkpoint": "unused.ckpt", "nprimes": 4}
    r = sk.count_plan(1, 23, symmetry=NEG_EVEN, **ck)
    assert (r["walk_bits"], r["items"], r["chunks_total"]) == (21, 2 ** 23, 2)
    r = sk.count_plan(0, 25, symmetry=NEG_EVEN, **ck)
    assert (r["walk_bits"], r["items"], r["chunks_total"]) == (17, 2 ** 31, 512)
    # every chunk at least 2^22 items, about 2^37 terms a launch
    r = sk.count_plan(0, 24, **ck)
    assert r["chunks_total"] == -(-r["items"] // max(2 ** 22, 2 ** (37 - r["walk_bits"])))
    # explicit chunk size and walk width
    r = sk.count_plan(0, 20, chunk_items=1000, walk_bits=20, **ck)
    assert (r["walk_bits"], r["items"], r["chunks_total"]) == (20, 2 ** 19, -(-2 ** 19 // 1000))
    assert sk.count_plan(0, 20, chunk_items=1000)["chunks_total"] == -(-sk.count_plan(0, 20)["items"] // 1000)


def test_plan_argument_checks():
    for args, kw in (((3, 8), {}), ((0, 32), {}), ((0, 12), {"walk_bits": 2}),
                     ((0, 12), {"convention": 3}), ((0, 12), {"nprimes": 2})):
        with pytest.raises(sk.SkolemError) as e:
            sk.count_plan(*args, **kw)
        assert e.value.status == sk.SK_EINVAL


@pytest.mark.parametrize("variant", [0, 1])
@pytest.mark.parametrize("n", [6, 8, 12, 16, 20, 24, 28, 31])
def test_reversal_plan(variant, n):
    # Lemma 2.3: x_1 and the middle positions fixed per item, an even walk
    # width; one of each mirror-image pair of items (decided by up to 8
    # mirror pairs of the middle), so the items are (1/2 + 2^-(depth+1)) of
    # the 2^{2n-1-m} of the plain half-sum (depth = min(8, middle pairs))
    r = sk.count_plan(variant, n, symmetry=sk.SYMMETRY_REVERSAL)
    m = r["walk_bits"]
    assert r["symmetry"] == sk.SYMMETRY_REVERSAL and m % 2 == 0
    assert r["inner_bits"] <= m // 2 <= n - 1
    pairs = n - 1 - m // 2
    depth = min(8, pairs)
    per_side = sum(2 ** (d + 2 * (pairs - 1 - d)) for d in range(depth)) + \
        2 ** (depth + 2 * (pairs - depth))
    assert r["items"] == 2 * per_side
    assert r["terms"] == r["items"] << m
    assert r["items"] * 2 ** m <= 2 ** (2 * n - 1) * (0.5 + 2.0 ** -(depth + 1)) + 1


@pytest.mark.parametrize("variant", [0, 1])
@pytest.mark.parametrize("n", [6, 7, 8, 9, 12, 16, 20, 24, 27, 28, 29, 31])
def test_reversal_with_lemma_2_4_plan(variant, n):
    # the x_1 = +1 half of the mirrored items in the existence classes
    # (Skolem n = 0, 1, Langford n = 0, 3 mod 4), nothing outside them
    r = sk.count_plan(variant, n, symmetry=sk.SYMMETRY_REVERSAL_EVEN)
    r2 = sk.count_plan(variant, n, symmetry=sk.SYMMETRY_REVERSAL)
    exists = n % 4 in ((0, 1), (0, 3))[variant]
    assert r["symmetry"] == sk.SYMMETRY_REVERSAL_EVEN
    if exists:
        assert r["walk_bits"] == r2["walk_bits"] and 2 * r["items"] == r2["items"]
    else:
        assert r["terms"] == 0 and r["items"] == 0 and r["complete"] == 1
