"""Options the library refuses before any device work (SK_EINVAL), checked on
a machine without a GPU: the exact count's plan (moduli, arithmetic form,
walk width against the inner block and Lemma 2.4's fixed variable, block
size, symmetry, convention) and the tempering runs (variant, order, ladder,
iteration counts)."""
import math

import numpy as np
import pytest

import paper_1507_00315_gb300 as sk


@pytest.mark.parametrize("variant,n,kw", [
    (3, 8, {}),                                     # no such variant
    (0, 0, {}), (0, 32, {}),                        # orders without a compiled kernel
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
    (0, 65, [0.0, 1.0], 4, 10, 0, 1),               # above the largest order
    (0, 8, [float(j) for j in range(65)], 4, 10, 0, 1),   # 65 rungs
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
    (0, 8, 1000, {"rungs": 65}),
    (0, 8, 1000, {"rungs": 33, "proposal": sk.PT_LEARNED}),   # learned: one warp a ladder
    (0, 8, 1000, {"burnin_frac": 1.0}),             # burn-in would take every iteration
    (2, 8, 1000, {}),
    (0, 65, 1000, {}),
])
def test_pt_estimate_arguments(variant, n, budget, kw):
    with pytest.raises(sk.SkolemError) as e:
        sk.pt_estimate(variant, n, budget, **kw)
    assert e.value.status == sk.SK_EINVAL


def test_inclusion_exclusion_refusals_before_device_work():
    # orders beyond the compiled inclusion-exclusion kernels, and options the
    # method does not have (no symmetry halves it; exact-digit form only)
    for args, kw in (((0, sk.MAX_IE_N + 1), {}), ((0, 0), {}), ((3, 8), {}),
                     ((0, 12), {"arith": sk.ARITH_MONTGOMERY}),
                     ((0, 12), {"symmetry": sk.SYMMETRY_NEGATION_EVEN}),
                     ((0, 12), {"walk_bits": 2}), ((0, 12), {"nprimes": 2})):
        with pytest.raises(sk.SkolemError) as e:
            sk.count_inclusion_exclusion(*args, **kw)
        assert e.value.status == sk.SK_EINVAL, (args, kw)
    with pytest.raises(sk.SkolemError) as e:
        sk.ie_item_residues(0, 12, 9, 1 << 15, 1, sk.default_primes()[:3])   # beyond 2^{2n-m} items
    assert e.value.status == sk.SK_EINVAL


def test_reversal_refusals_before_device_work():
    # Lemma 2.3 needs a reversal-symmetric P (not hooked Skolem), the exact
    # digit form, and an even walk width 2h with U <= h <= n-1
    U = sk.count_plan(0, 14)["inner_bits"]
    for args, kw in (((2, 12), {}), ((0, 12), {"arith": sk.ARITH_MONTGOMERY}),
                     ((0, 14), {"walk_bits": 2 * U + 1}), ((0, 14), {"walk_bits": 2 * U - 2}),
                     ((0, 14), {"walk_bits": 28})):
        with pytest.raises(sk.SkolemError) as e:
            sk.count_plan(*args, symmetry=sk.SYMMETRY_REVERSAL, **kw)
        assert e.value.status == sk.SK_EINVAL, (args, kw)


def test_learned_proposal_orders():
    # the network's move table and input width hold n <= 40; the plain
    # chains go to n = 64
    with pytest.raises(sk.SkolemError) as e:
        sk.Mlp(0, 41, 128)
    assert e.value.status == sk.SK_EINVAL


def test_extended_refusals_before_device_work():
    # a hole outside 1..2n+1 (0 must not read as "no hole"), a symmetry
    # option, a walk reaching the hole, a lower hole for the item residues
    for args, kw in (((12, 0), {}), ((12, -1), {}), ((12, 26), {}), ((0, 1), {}),
                     ((12, 13), {"symmetry": sk.SYMMETRY_NEGATION_EVEN}),
                     ((12, 13), {"symmetry": sk.SYMMETRY_REVERSAL}),
                     ((12, 13), {"walk_bits": 13}), ((3, 4), {})):
        with pytest.raises(sk.SkolemError) as e:
            sk.count_extended(*args, **kw)
        assert e.value.status == sk.SK_EINVAL, (args, kw)
    for hole in (0, 8, 26):
        with pytest.raises(sk.SkolemError) as e:
            sk.extended_item_residues(12, hole, 9, 0, 1, sk.default_primes()[:3])
        assert e.value.status == sk.SK_EINVAL


def test_network_forwards_refuse_a_null_model():
    # both forwards check their arguments before any device work
    L = sk.lib()
    slots = np.zeros(64, np.uint8)
    for fn, out in ((L.sk_mlp_forward, np.zeros(64, np.float32)),
                    (L.sk_mlp_forward_bf16, np.zeros(64, np.uint16))):
        assert fn(None, slots.ctypes.data, 1, out.ctypes.data) == sk.SK_EINVAL
