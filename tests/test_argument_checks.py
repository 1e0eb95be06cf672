"""Options the library refuses before any device work (SK_EINVAL), checked on
a machine without a GPU: the exact count's plan (moduli, arithmetic form,
walk width against the inner block and Lemma 2.4's fixed variable, block
size, symmetry, convention) and the tempering runs (variant, order, ladder,
iteration counts)."""
import math

import pytest

import paper_1507_00315_gb300 as sk


@pytest.mark.parametrize("variant,n,kw", [
    (3, 8, {}),                                     # no such variant
    (0, 0, {}), (0, 29, {}),                        # orders without a compiled kernel
    (0, 12, {"nprimes": 2}), (0, 12, {"nprimes": 5}),
    (0, 12, {"nprimes": 4, "primes": [4, 0, 0, 0]}),            # an even modulus
    (0, 12, {"nprimes": 3, "primes": [(1 << 62) + 1, 0, 0]}),   # above 2^62
    (0, 12, {"arith": 9}),
    (0, 12, {"walk_bits": 2}),                      # below the unrolled inner block
    (0, 12, {"walk_bits": 24}),                     # above the 2n - 1 free variables
    (0, 12, {"block_threads": 48}), (0, 12, {"block_threads": 512}),
    (0, 12, {"symmetry": 5}),
    # Lemma 2.4 holds x_22 at +1: a walk over it is refused
    (0, 12, {"symmetry": sk.SYMMETRY_NEGATION_EVEN, "walk_bits": 23}),
    (0, 12, {"convention": 3}),
])
def test_count_options(variant, n, kw):
    with pytest.raises(sk.SkolemError) as e:
        sk.count_ex(variant, n, **kw)
    assert e.value.status == sk.SK_EINVAL


@pytest.mark.parametrize("args", [
    (2, 8, [0.0, 1.0], 4, 10, 0, 1),                # hooked: no tempering variant
    (0, 1, [0.0, 1.0], 4, 10, 0, 1),                # n < 2
    (0, 41, [0.0, 1.0], 4, 10, 0, 1),               # above the largest order
    (0, 8, [float(j) for j in range(33)], 4, 10, 0, 1),   # 33 rungs
    (0, 8, [0.0, 1.0], 0, 10, 0, 1),                # no ladder
    (0, 8, [1.0, 0.5], 4, 10, 0, 1),                # decreasing ladder
    (0, 8, [-1.0, 0.5], 4, 10, 0, 1),               # negative beta
    (0, 8, [0.0, math.nan], 4, 10, 0, 1),
    (0, 8, [0.0, math.inf], 4, 10, 0, 1),
    (0, 8, [0.0, 1.0], 4, 1 << 32, 0, 1),           # iterations counted in 32 bits
])
def test_pt_run_arguments(args):
    with pytest.raises(sk.SkolemError) as e:
        sk.pt_run(*args)
    assert e.value.status == sk.SK_EINVAL


@pytest.mark.parametrize("variant,n,budget,kw", [
    (0, 8, 0, {}),                                  # no iterations
    (0, 8, 1 << 32, {}),
    (0, 8, 1000, {"rungs": 33}),
    (0, 8, 1000, {"burnin_frac": 1.0}),             # burn-in would take every iteration
    (2, 8, 1000, {}),
    (0, 41, 1000, {}),
])
def test_pt_estimate_arguments(variant, n, budget, kw):
    with pytest.raises(sk.SkolemError) as e:
        sk.pt_estimate(variant, n, budget, **kw)
    assert e.value.status == sk.SK_EINVAL
