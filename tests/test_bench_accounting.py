"""bench.py's accounting, on CPU: the work of one headline step and the
algorithmic operation counts behind its roofline (the figures quoted with
the measurements)."""
import bench


def test_terms_per_step():
    # S(n) and L(n), n = 16..20: 2^{2n-1} terms each after Lemma 2.2
    assert bench.terms_per_step() == 2 * sum(2 ** (2 * n - 1) for n in range(16, 21))
    assert bench.terms_per_step() == 1464583847936


def test_operations_per_term():
    # S(20): 20 correlation adds, 16 multiplies inside 4 int32 groups, 6
    # two-word partial products (12), 4 accumulate words
    assert bench.groups(0, 20) == 4
    assert bench.alg_ops_per_term(0, 20) == 52
    assert bench.alg_ops_per_term(0, 24) == 67
    # one cumulative bound-product length per int32 group, growing group by group
    for delta in (0, 1):
        for n in range(4, 32):
            bits = bench.group_bits(delta, n)
            assert len(bits) == bench.groups(delta, n)
            assert bits == sorted(bits) and bits[-1] >= bits[0]


def test_tempering_operations():
    # Philox-4x32-10 (80) + move (18) + histogram (3) + half an exchange (2)
    assert bench.PT_OPS_PER_LANE_ITERATION == 103


def test_oracle_sample_shape():
    # the CPU baseline: (terms/s, cores, description, measured seconds)
    v, cores, sample, dt = bench.oracle_sample(seconds_target=0.3)
    assert v > 0 and cores >= 1 and dt > 0 and "work items of S(20)/L(20)" in sample
