"""Seeded synthetic inputs shared by the oracle side and the CUDA side of the
tests.  Holds no arithmetic of the method: only random draws and format
conversion (rounding to bfloat16)."""
import numpy as np


def bf16_round(a):
    """Round float32/float64 values to the nearest bfloat16 (ties to even),
    returned as float64."""
    f = np.asarray(a, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    u = (u + 0x7FFF + lsb) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def differences(variant, n):
    """d_k of the Skolem (0) and Langford (1) problems."""
    return [k + 1 if variant == 1 else k for k in range(1, n + 1)]


def random_slots(seed, batch, n, d):
    """Configurations of the simplified problem: pair k at a uniform start
    slot in [0, 2n - d_k)."""
    rng = np.random.default_rng(seed)
    return np.stack([rng.integers(0, 2 * n - dk, size=batch) for dk in d], axis=1).astype(np.int64)


def mlp_params(seed, in_dim, hidden, out_dim, scale=1.0):
    """He-style random weights, rounded to bfloat16; biases small."""
    rng = np.random.default_rng(seed)
    W1 = bf16_round(rng.standard_normal((in_dim, hidden)) * scale * np.sqrt(2.0 / in_dim))
    W2 = bf16_round(rng.standard_normal((hidden, hidden)) * scale * np.sqrt(2.0 / hidden))
    W3 = bf16_round(rng.standard_normal((hidden, out_dim)) * scale * np.sqrt(1.0 / hidden))
    b1 = rng.standard_normal(hidden).astype(np.float32).astype(np.float64) * 0.1
    b2 = rng.standard_normal(hidden).astype(np.float32).astype(np.float64) * 0.1
    b3 = rng.standard_normal(out_dim).astype(np.float32).astype(np.float64) * 0.1
    return W1, b1, W2, b2, W3, b3
