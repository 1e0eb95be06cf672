"""Pins of the FP64 proposal-network reference: finite differences of the
loss, the closed-form gradient of softmax cross-entropy, and the move/energy
bookkeeping against a direct recount."""
import numpy as np

import oracle
from oracle import mlp_ref
from tests import seeded_inputs as si


def _setup(seed=0, B=6, n=5, hidden=16):
    d = si.differences(0, n)
    off, nslot = mlp_ref.move_table(n, d)
    slots = si.random_slots(seed, B, n, d)
    x = mlp_ref.occupancy(slots, n, d)
    params = si.mlp_params(seed + 1, 2 * n, hidden, int(nslot.sum()), scale=1.5)
    mask = mlp_ref.valid_mask(slots, n, d)
    target = mlp_ref.target_distribution(slots, n, d, beta_star=2.0)
    return x, params, mask, target, slots, n, d


def test_gradients_match_finite_differences():
    x, params, mask, target, *_ = _setup()
    names = ["W1", "b1", "W2", "b2", "W3", "b3"]
    loss, g = mlp_ref.loss_and_grads(x, *params, mask, target)
    rng = np.random.default_rng(5)
    h = 1e-6
    for i, name in enumerate(names):
        P = [p.copy() for p in params]
        for _ in range(6):
            idx = tuple(rng.integers(0, s) for s in P[i].shape)
            P[i][idx] += h
            lp, _ = mlp_ref.loss_and_grads(x, *P, mask, target)
            P[i][idx] -= 2 * h
            lm, _ = mlp_ref.loss_and_grads(x, *P, mask, target)
            P[i][idx] += h
            fd = (lp - lm) / (2 * h)
            assert abs(fd - g[name][idx]) < 1e-6 + 1e-5 * abs(fd), (name, idx, fd, g[name][idx])


def test_softmax_cross_entropy_gradient_closed_form():
    # d/dz of -sum t log softmax(z) is softmax(z) - t (sum t = 1), per row.
    x, params, mask, target, *_ = _setup(seed=3)
    _, g = mlp_ref.loss_and_grads(x, *params, mask, target)
    z = g["z"]
    zm = np.where(mask, z, -np.inf)
    q = np.exp(zm - zm.max(1, keepdims=True))
    q /= q.sum(1, keepdims=True)
    assert np.allclose(g["dz"] * x.shape[0], q - target, atol=1e-12)
    assert np.allclose(target.sum(1), 1.0)
    assert np.all(target[~mask] == 0)


def test_delta_energy_matches_recount():
    # dE of a move equals the change of the number of empty bins, recounted
    # from scratch with the oracle's own energy definition (Sec. 3).
    _, _, _, _, slots, n, d = _setup(seed=9, B=3)
    dE = mlp_ref.delta_energy(slots, n, d)
    off, nslot = mlp_ref.move_table(n, d)
    for b in range(slots.shape[0]):
        E0 = int((mlp_ref.occupancy(slots[b:b + 1], n, d)[0] == 0).sum())
        for k in range(n):
            for s in range(nslot[k]):
                s2 = slots[b].copy()
                s2[k] = s
                E1 = int((mlp_ref.occupancy(s2[None], n, d)[0] == 0).sum())
                assert dE[b, off[k] + s] == E1 - E0


def test_move_table_size():
    # number of moves = sum_k (2n - d_k) = Z(0)'s factor count sum
    for n in (4, 12, 33):
        d = si.differences(0, n)
        _, nslot = mlp_ref.move_table(n, d)
        assert int(nslot.sum()) == n * (3 * n - 1) // 2
