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


def test_adam_step_hand_worked_two_steps():
    # Kingma & Ba's update with bias correction, worked by hand.  Constant
    # gradient: the corrected moments are g and g^2 at every t, so each step
    # is lr g / (|g| + eps).  Reversed gradient at t = 2: m = 0.9 (0.1 g) -
    # 0.1 g = -0.01 g, corrected by 1 - 0.9^2 = 0.19 to -g / 19; v = (0.999 *
    # 0.001 + 0.001) g^2 corrected by 1 - 0.999^2 = 0.001999 to g^2: the step
    # is -lr sign(g) / 19 (g the first gradient).  Zero then 0.3: m = 0.03 -> 0.3 / 1.9, v = 9e-5 ->
    # 0.09 / 1.999: the step is lr sqrt(1.999) / 1.9.  A gradient equal to
    # eps at t = 1 moves by lr / 2 (eps outside the square root).
    lr, eps = 0.01, 1e-8
    w0 = np.array([1.0, -2.0, 0.5, 3.0])
    g1 = np.array([0.1, -0.2, 0.0, 1e-8])
    g2 = np.array([0.1, 0.2, 0.3, 1e-8])
    w1, m1, v1 = mlp_ref.adam_step(w0, g1, np.zeros(4), np.zeros(4), 1, lr)
    assert np.allclose(m1, [0.01, -0.02, 0.0, 1e-9], rtol=1e-12, atol=0)
    assert np.allclose(v1, [1e-5, 4e-5, 0.0, 1e-19], rtol=1e-12, atol=0)
    want1 = [1.0 - lr * 0.1 / (0.1 + eps), -2.0 + lr * 0.2 / (0.2 + eps), 0.5, 3.0 - lr / 2]
    assert np.allclose(w1, want1, rtol=0, atol=1e-15)
    w2, m2, v2 = mlp_ref.adam_step(w1, g2, m1, v1, 2, lr)
    assert np.allclose(m2, [0.019, 0.002, 0.03, 1.9e-9], rtol=1e-12, atol=0)
    assert np.allclose(v2, [1.999e-5, 7.996e-5, 9e-5, 1.999e-19], rtol=1e-12, atol=0)
    step = [lr * 0.1 / (0.1 + eps),
            lr / 19 * 0.2 / (0.2 + eps),       # g = -0.2 first
            lr * (0.3 / 1.9) / (0.3 / np.sqrt(1.999) + eps),
            lr / 2]
    assert np.allclose(w2, np.array(want1) - np.array(step), rtol=0, atol=1e-15)
    # with the betas swapped the reversed-gradient step would be ~lr / 1999
    assert abs((w1[1] - w2[1]) / lr - 1 / 19) < 1e-6


def test_forward_of_a_hand_set_network():
    # 2 -> 2 -> 2 -> 3 with integer weights, worked on paper.  Row (1, 2):
    # a1 = (1 + 4, -1 + 2) + (0, -3) = (5, -2), h1 = (5, 0) (ReLU clips);
    # a2 = (5 - 1, -10 + 1) = (4, -9), h2 = (4, 0); z = (4 + 0.5, 0, -4 - 2).
    # Row (0, 1): a1 = (2, 1) + (0, -3) = (2, -2), h1 = (2, 0); a2 = (1, -3),
    # h2 = (1, 0); z = (1.5, 0, -3).  Weights are [in][out] (x @ W).
    W1 = np.array([[1.0, -1.0], [2.0, 1.0]])
    b1 = np.array([0.0, -3.0])
    W2 = np.array([[1.0, -2.0], [3.0, -1.0]])
    b2 = np.array([-1.0, 1.0])
    W3 = np.array([[1.0, 0.0, -1.0], [0.0, 1.0, 2.0]])
    b3 = np.array([0.5, 0.0, -2.0])
    x = np.array([[1.0, 2.0], [0.0, 1.0]])
    a1, h1, a2, h2, z = mlp_ref.forward(x, W1, b1, W2, b2, W3, b3)
    assert np.array_equal(a1, [[5, -2], [2, -2]])
    assert np.array_equal(h1, [[5, 0], [2, 0]])
    assert np.array_equal(a2, [[4, -9], [1, -3]])
    assert np.array_equal(h2, [[4, 0], [1, 0]])
    assert np.array_equal(z, [[4.5, 0, -6], [1.5, 0, -3]])


def test_loss_of_a_hand_set_network():
    # One state, three moves with logits (0, 0, ln 2) and all valid: q =
    # (1/4, 1/4, 1/2).  Target (1, 0, 0): loss = ln 4, dz = q - t =
    # (-3/4, 1/4, 1/2).  A masked move drops out of the softmax: with move 2
    # masked, q = (1/2, 1/2) and loss = ln 2.
    x = np.array([[1.0]])
    W1, b1 = np.array([[1.0]]), np.array([0.0])
    W2, b2 = np.array([[1.0]]), np.array([0.0])
    W3, b3 = np.array([[0.0, 0.0, 0.0]]), np.array([0.0, 0.0, np.log(2.0)])
    t = np.array([[1.0, 0.0, 0.0]])
    loss, g = mlp_ref.loss_and_grads(x, W1, b1, W2, b2, W3, b3, np.ones((1, 3), bool), t)
    assert abs(loss - np.log(4.0)) < 1e-15
    assert np.allclose(g["dz"], [[-0.75, 0.25, 0.5]], atol=1e-15)
    assert np.allclose(g["b3"], [-0.75, 0.25, 0.5], atol=1e-15)
    loss2, g2 = mlp_ref.loss_and_grads(x, W1, b1, W2, b2, W3, b3,
                                       np.array([[True, True, False]]), t)
    assert abs(loss2 - np.log(2.0)) < 1e-15
    assert np.allclose(g2["dz"], [[-0.5, 0.5, 0.0]], atol=1e-15)
