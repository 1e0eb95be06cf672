"""The tempering estimator and its standard error (host code of the library,
no device) against the oracle's estimator, Sec. 3 / Algorithm 2: on random
energy histograms, pooled over groups of ladders, and on the argument checks."""
import numpy as np
import pytest

import oracle
import paper_1507_00315_gb300 as sk


def _hist(rng, groups, M, n, zero_last=False):
    h = rng.integers(0, 5000, size=(groups, M, 2 * n + 1)).astype(np.uint64)
    if zero_last:
        h[:, -1, 0] = 0
    return h


@pytest.mark.parametrize("variant,n,M", [(0, 4, 1), (0, 9, 8), (1, 12, 16), (0, 24, 32), (1, 33, 32)])
def test_estimate_equals_the_oracle(variant, n, M):
    rng = np.random.default_rng(n * 100 + M)
    beta = np.sort(rng.uniform(0.0, 20.0, M))
    beta[0] = 0.0
    h = _hist(rng, 1, M, n)[0]
    est, ratios, se = sk.pt_estimate_hist(variant, n, beta, h)
    want = oracle.pt_estimate_from_hist(h, beta, variant, n)
    assert abs(est / want - 1) < 1e-12
    assert se == 0.0
    # Ratio(j) of Algorithm 2: mean of e^{-(beta_{j+1}-beta_j) E}; last rung P(E = 0)
    E = np.arange(2 * n + 1)
    for j in range(M):
        hj = h[j].astype(np.float64)
        r = (hj[0] / hj.sum()) if j == M - 1 else (hj * np.exp(-(beta[j + 1] - beta[j]) * E)).sum() / hj.sum()
        assert abs(ratios[j] / r - 1) < 1e-12


def test_groups_pool_and_give_the_standard_error():
    rng = np.random.default_rng(7)
    variant, n, M, G = 0, 12, 16, 16
    beta = np.linspace(0.0, 16.0, M)
    h = _hist(rng, G, M, n)
    est, _, se = sk.pt_estimate_hist(variant, n, beta, h)
    pooled = oracle.pt_estimate_from_hist(h.sum(axis=0), beta, variant, n)
    assert abs(est / pooled - 1) < 1e-12
    eg = np.array([oracle.pt_estimate_from_hist(h[g], beta, variant, n) for g in range(G)])
    want = eg.std(ddof=1) / np.sqrt(G) / eg.mean()
    assert abs(se / want - 1) < 1e-9


def test_standard_error_edge_cases():
    rng = np.random.default_rng(3)
    n, M = 6, 4
    beta = np.linspace(0.0, 8.0, M)
    same = np.repeat(_hist(rng, 1, M, n), 4, axis=0)
    assert sk.pt_estimate_hist(0, n, beta, same)[2] == 0.0          # identical groups
    est, _, se = sk.pt_estimate_hist(0, n, beta, _hist(rng, 3, M, n, zero_last=True))
    assert est == 0.0 and np.isnan(se)                               # no E = 0 sample anywhere


def test_argument_checks():
    beta = np.linspace(0.0, 4.0, 4)
    h = np.ones((4, 9), dtype=np.uint64)
    for args in ((2, 4, beta, h), (0, 1, beta, np.ones((4, 3), np.uint64)),
                 (0, 4, beta[::-1].copy(), h), (0, 65, beta, np.ones((4, 131), np.uint64))):
        with pytest.raises(sk.SkolemError) as e:
            sk.pt_estimate_hist(*args)
        assert e.value.status == sk.SK_EINVAL
