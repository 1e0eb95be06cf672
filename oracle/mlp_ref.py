"""FP64 reference of the move-proposal network -- TEST INFRASTRUCTURE ONLY.

The learned proposal is not in the paper (it is an addition used inside the
Metropolis step of Algorithm 2, Sec. 3).  Network: the bin occupancies of a
configuration of the simplified problem (2n values) -> 256 ReLU -> 256 ReLU ->
one logit per move (k, s): pair k to start slot s, s = 0..2n-d_k-1, ordered by
k then s.  The proposal is the softmax of the logits over the valid moves of
the state (every (k, s) except s = current slot of k).

Training target (also an addition): for a state C, t(m) proportional to
exp(-beta* dE(m)) over the valid moves m, dE the change of the number of empty
bins.  Loss = mean over the batch of -sum_m t(m) log q(m).

Everything here is float64 on the values it is given (the caller passes the
bf16-rounded weights and inputs the GPU uses), written out layer by layer so a
reader can check it against the formulas above.
"""
from __future__ import annotations

import numpy as np


def move_table(n: int, d):
    """Return (offsets[k], nslot[k]) with move (k, s) at offsets[k] + s (k = 0-based pair)."""
    nslot = [2 * n - dk for dk in d]
    off = np.concatenate([[0], np.cumsum(nslot)[:-1]]).astype(np.int64)
    return off, np.asarray(nslot, dtype=np.int64)


def occupancy(slots, n: int, d):
    """Balls per bin of each configuration.  slots: [B, n] start bins."""
    slots = np.asarray(slots, dtype=np.int64)
    B = slots.shape[0]
    occ = np.zeros((B, 2 * n), dtype=np.float64)
    for k in range(n):
        np.add.at(occ, (np.arange(B), slots[:, k]), 1.0)
        np.add.at(occ, (np.arange(B), slots[:, k] + d[k]), 1.0)
    return occ


def valid_mask(slots, n: int, d):
    """True for every move except moving a pair to the slot it already has."""
    off, nslot = move_table(n, d)
    slots = np.asarray(slots, dtype=np.int64)
    B = slots.shape[0]
    mask = np.ones((B, int(nslot.sum())), dtype=bool)
    for k in range(n):
        mask[np.arange(B), off[k] + slots[:, k]] = False
    return mask


def delta_energy(slots, n: int, d):
    """dE of every move (k, s) from each configuration (number of empty bins
    after minus before); invalid moves get 0."""
    off, nslot = move_table(n, d)
    slots = np.asarray(slots, dtype=np.int64)
    B = slots.shape[0]
    occ = occupancy(slots, n, d)
    out = np.zeros((B, int(nslot.sum())), dtype=np.float64)
    for b in range(B):
        E0 = int((occ[b] == 0).sum())
        for k in range(n):
            for s in range(nslot[k]):
                o = occ[b].copy()
                o[slots[b, k]] -= 1
                o[slots[b, k] + d[k]] -= 1
                o[s] += 1
                o[s + d[k]] += 1
                out[b, off[k] + s] = int((o == 0).sum()) - E0
    return out


def target_distribution(slots, n: int, d, beta_star: float):
    """t(m) proportional to exp(-beta* dE(m)) over valid moves."""
    dE = delta_energy(slots, n, d)
    mask = valid_mask(slots, n, d)
    w = np.where(mask, np.exp(-beta_star * dE), 0.0)
    return w / w.sum(axis=1, keepdims=True)


def forward(x, W1, b1, W2, b2, W3, b3):
    """Return (a1, h1, a2, h2, z): pre-activations, activations, logits."""
    a1 = x @ W1 + b1
    h1 = np.maximum(a1, 0.0)
    a2 = h1 @ W2 + b2
    h2 = np.maximum(a2, 0.0)
    z = h2 @ W3 + b3
    return a1, h1, a2, h2, z


def masked_log_softmax(z, mask):
    zm = np.where(mask, z, -np.inf)
    mx = zm.max(axis=1, keepdims=True)
    lse = mx + np.log(np.exp(zm - mx).sum(axis=1, keepdims=True))
    return np.where(mask, z - lse, -np.inf)


def loss_and_grads(x, W1, b1, W2, b2, W3, b3, mask, target):
    """Cross-entropy loss (batch mean) and the gradients of every parameter,
    by the chain rule written out layer by layer."""
    B = x.shape[0]
    a1, h1, a2, h2, z = forward(x, W1, b1, W2, b2, W3, b3)
    logq = masked_log_softmax(z, mask)
    loss = -(target * np.where(mask, logq, 0.0)).sum() / B
    q = np.where(mask, np.exp(logq), 0.0)
    dz = (q - target) / B                         # d loss / d z
    dW3 = h2.T @ dz
    db3 = dz.sum(axis=0)
    dh2 = dz @ W3.T
    da2 = dh2 * (a2 > 0)
    dW2 = h1.T @ da2
    db2 = da2.sum(axis=0)
    dh1 = da2 @ W2.T
    da1 = dh1 * (a1 > 0)
    dW1 = x.T @ da1
    db1 = da1.sum(axis=0)
    return loss, {"W1": dW1, "b1": db1, "W2": dW2, "b2": db2, "W3": dW3, "b3": db3,
                  "dz": dz, "z": z}


def adam_step(w, g, m, v, t: int, lr: float, b1: float = 0.9, b2: float = 0.999,
              eps: float = 1e-8):
    """Kingma & Ba (2015) Adam update, returns (w, m, v)."""
    m = b1 * m + (1 - b1) * g
    v = b2 * v + (1 - b2) * g * g
    mhat = m / (1 - b1 ** t)
    vhat = v / (1 - b2 ** t)
    return w - lr * mhat / (np.sqrt(vhat) + eps), m, v
