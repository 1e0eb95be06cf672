"""CPU oracle for the counting method of "Counting Skolem Sequences".

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  It shares no code,
header, table or generator with the CUDA path in ``paper_1507_00315_gb300``;
neither side imports the other.

The arithmetic lives in ``skolem_oracle.c`` (plain C, compiled with gcc into
``liboracle.so`` beside it) plus two pure-Python modules:
``constructions`` (Tables 1 and 2) and ``mlp_ref`` (FP64 reference of the
move-proposal network).  See the header of ``skolem_oracle.c`` for the list of
functions, the passage each follows, and the readings taken where the paper is
silent.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "skolem_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

SKOLEM, LANGFORD, HOOKED = 0, 1, 2


def build(force: bool = False) -> str:
    """Compile liboracle.so with gcc (portable flags: no -march)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-pthread",
                               _SRC, "-o", tmp, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB)
            u64p = ctypes.POINTER(ctypes.c_uint64)
            lib.orc_layout.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_int),
                                       ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int)]
            lib.orc_backtrack.argtypes = [ctypes.c_int, ctypes.c_int, u64p, ctypes.c_void_p,
                                          ctypes.c_uint64]
            lib.orc_signed_sum.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                           u64p]
            lib.orc_summand.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_void_p, u64p]
            lib.orc_partial_sum_mod.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                                ctypes.c_uint64, ctypes.c_uint64, u64p]
            lib.orc_backtrack_hole.argtypes = [ctypes.c_int, ctypes.c_int, u64p]
            lib.orc_signed_sum_hole.argtypes = [ctypes.c_int, ctypes.c_int, u64p]
            lib.orc_partial_sum_mod_hole.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                                     ctypes.c_uint64, ctypes.c_uint64, u64p]
            lib.orc_ie_count.argtypes = [ctypes.c_int, ctypes.c_int, u64p]
            lib.orc_ie_partial_sum_mod.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                                   ctypes.c_uint64, ctypes.c_uint64, u64p]
            lib.orc_philox4x32_10.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
            lib.orc_pt_run.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_void_p,
                                       ctypes.c_int, ctypes.c_uint64, ctypes.c_uint64,
                                       ctypes.c_uint64, ctypes.c_void_p, ctypes.c_void_p,
                                       ctypes.c_void_p, ctypes.c_void_p]
            lib.orc_pt_run_trips.argtypes = lib.orc_pt_run.argtypes + [ctypes.c_void_p]
            lib.orc_simplified_energy_hist.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_void_p]
            _lib = lib
    return _lib


def _check(rc, what):
    if rc != 0:
        raise ValueError(f"oracle {what}: invalid arguments")


def layout(variant: int, n: int):
    """(span, sorted positions of P, [d_1..d_n]) -- Sec. 1.1 / 1.2."""
    lib = _load()
    span = ctypes.c_int()
    present = (ctypes.c_int * 100)()
    d = (ctypes.c_int * 50)()
    _check(lib.orc_layout(variant, n, ctypes.byref(span), present, d), "layout")
    pos = [i for i in range(1, span.value + 1) if present[i]]
    return span.value, pos, [d[k] for k in range(1, n + 1)]


def backtrack_count(variant: int, n: int) -> int:
    """O1: all pairings, reflections distinct (Sec. 2, Miller's order)."""
    lib = _load()
    c = ctypes.c_uint64()
    _check(lib.orc_backtrack(variant, n, ctypes.byref(c), None, 0), "backtrack")
    return c.value


def backtrack_list(variant: int, n: int, max_list: int = 10000):
    """O1 with the pairings themselves: list of tuples of span labels."""
    lib = _load()
    span, _, _ = layout(variant, n)
    buf = np.zeros((max_list, span), dtype=np.int8)
    c = ctypes.c_uint64()
    _check(lib.orc_backtrack(variant, n, ctypes.byref(c), buf.ctypes.data, max_list), "backtrack")
    k = min(c.value, max_list)
    return [tuple(int(v) for v in row) for row in buf[:k]]


def _s128(lo: int, hi: int) -> int:
    v = lo | (hi << 64)
    return v - (1 << 128) if v >= (1 << 127) else v


def signed_sum(variant: int, n: int, half: bool = True, threads: int = 1) -> int:
    """O2: Algorithm 1's sum S (exact for |S| < 2^127, i.e. n <= 26)."""
    lib = _load()
    out = (ctypes.c_uint64 * 2)()
    _check(lib.orc_signed_sum(variant, n, int(half), threads, out), "signed_sum")
    return _s128(out[0], out[1])


def coefficient(variant: int, n: int, threads: int = 1) -> int:
    """Lemma 2.1 with Lemma 2.2: the coefficient of x_1...x_2n, i.e. the
    number of pairings with reflections distinct."""
    s = signed_sum(variant, n, half=True, threads=threads)
    div = 1 << (2 * n - 1)
    if s % div:
        raise ArithmeticError(f"signed sum {s} not divisible by 2^{2 * n - 1}")
    return s // div


def summand(variant: int, n: int, x) -> int:
    """sign(X) F(n, X) for one assignment; x maps positions 1..span to +-1
    (x[0] unused; positions outside P ignored)."""
    lib = _load()
    span, _, _ = layout(variant, n)
    arr = np.zeros(span + 2, dtype=np.int32)
    arr[1:span + 1] = np.asarray(x, dtype=np.int32)[1:span + 1]
    out = (ctypes.c_uint64 * 2)()
    _check(lib.orc_summand(variant, n, arr.ctypes.data, out), "summand")
    return _s128(out[0], out[1])


def partial_sum_mod(variant: int, n: int, m: int, q: int, p: int) -> int:
    """sum over the block (low m free variables run, the rest fixed by q) of
    sign(X) F(n, X), modulo p."""
    lib = _load()
    out = ctypes.c_uint64()
    _check(lib.orc_partial_sum_mod(variant, n, m, q, p, ctypes.byref(out)), "partial_sum_mod")
    return out.value


def backtrack_count_hole(n: int, hole: int) -> int:
    """O1 for extended Skolem sequences (Sec. 1.2): positions 1..2n+1 except
    `hole`, differences 1..n; reflections distinct."""
    lib = _load()
    c = ctypes.c_uint64()
    _check(lib.orc_backtrack_hole(n, hole, ctypes.byref(c)), "backtrack_hole")
    return c.value


def coefficient_hole(n: int, hole: int) -> int:
    """Lemma 2.1 with Lemma 2.2 on the same position set: Algorithm 1's
    half-sum divided by 2^{2n-1}."""
    lib = _load()
    out = (ctypes.c_uint64 * 2)()
    _check(lib.orc_signed_sum_hole(n, hole, out), "signed_sum_hole")
    s = _s128(out[0], out[1])
    div = 1 << (2 * n - 1)
    if s % div:
        raise ArithmeticError(f"signed sum {s} not divisible by 2^{2 * n - 1}")
    return s // div


def partial_sum_mod_hole(n: int, hole: int, m: int, q: int, p: int) -> int:
    """One block of that half-sum modulo p (free variables: the positions
    below max P in increasing order; the low m run, the rest fixed by q)."""
    lib = _load()
    out = ctypes.c_uint64()
    _check(lib.orc_partial_sum_mod_hole(n, hole, m, q, p, ctypes.byref(out)), "partial_sum_mod_hole")
    return out.value


def ie_count(variant: int, n: int) -> int:
    """Inclusion-exclusion count (Sec. 2, third approach): the number of
    sequences with reflections distinct, from the alternating sum over the
    sets of avoided positions."""
    lib = _load()
    out = (ctypes.c_uint64 * 2)()
    _check(lib.orc_ie_count(variant, n, out), "ie_count")
    return out[0] | (out[1] << 64)


def ie_partial_sum_mod(variant: int, n: int, m: int, q: int, p: int) -> int:
    """The inclusion-exclusion sum over one block of sets (the low m of the
    2n position variables run, the rest fixed by q), modulo p."""
    lib = _load()
    out = ctypes.c_uint64()
    _check(lib.orc_ie_partial_sum_mod(variant, n, m, q, p, ctypes.byref(out)), "ie_partial_sum_mod")
    return out.value


def philox4x32_10(counter, key):
    lib = _load()
    c = np.asarray(counter, dtype=np.uint32)
    k = np.asarray(key, dtype=np.uint32)
    out = np.zeros(4, dtype=np.uint32)
    lib.orc_philox4x32_10(c.ctypes.data, k.ctypes.data, out.ctypes.data)
    return [int(v) for v in out]


def pt_run(variant: int, n: int, beta, ladders: int, iters: int, burnin: int, seed: int,
           want_final: bool = False, want_trips: bool = False):
    """O3: Algorithm 2.  Returns dict(hist[M, 2n+1], acc_move[M], acc_swap[M],
    final_slots[L, M, n] or None, round_trips or None)."""
    lib = _load()
    beta = np.ascontiguousarray(beta, dtype=np.float64)
    M = beta.shape[0]
    hist = np.zeros((M, 2 * n + 1), dtype=np.uint64)
    am = np.zeros(M, dtype=np.uint64)
    asw = np.zeros(M, dtype=np.uint64)
    fin = np.zeros((ladders, M, n), dtype=np.uint8) if want_final else None
    trips = np.zeros(1, dtype=np.uint64)
    rc = lib.orc_pt_run_trips(variant, n, M, beta.ctypes.data, ladders, iters, burnin, seed,
                              hist.ctypes.data, am.ctypes.data, asw.ctypes.data,
                              fin.ctypes.data if fin is not None else None,
                              trips.ctypes.data if want_trips else None)
    _check(rc, "pt_run")
    return {"hist": hist, "acc_move": am, "acc_swap": asw, "final_slots": fin,
            "round_trips": int(trips[0]) if want_trips else None}


def simplified_energy_hist(variant: int, n: int) -> np.ndarray:
    """O4: N(E), E = 0..2n, over all configurations of the simplified problem."""
    lib = _load()
    N = np.zeros(2 * n + 1, dtype=np.uint64)
    _check(lib.orc_simplified_energy_hist(variant, n, N.ctypes.data), "energy_hist")
    return N


def simplified_size(variant: int, n: int) -> int:
    """Z(0) = prod_k (2n - d_k): Sec. 3 gives (2n-1)!/(n-1)! for Skolem."""
    _, _, d = layout(variant, n)
    z = 1
    for dk in d:
        z *= 2 * n - dk
    return z


def pt_estimate_from_hist(hist, beta, variant: int, n: int) -> float:
    """Sec. 3 / Algorithm 2 final loop: S ~ 1/2 Z(0) prod_j Ratio(j), with
    Ratio(j) = mean of e^{-(beta_{j+1}-beta_j) E} at rung j and, for the last
    rung (beta_{M+1} = infinity), the fraction of samples with E = 0."""
    hist = np.asarray(hist, dtype=np.float64)
    beta = np.asarray(beta, dtype=np.float64)
    M, nb = hist.shape
    E = np.arange(nb, dtype=np.float64)
    logr = 0.0
    for j in range(M):
        tot = hist[j].sum()
        if j + 1 < M:
            r = (hist[j] * np.exp(-(beta[j + 1] - beta[j]) * E)).sum() / tot
        else:
            r = hist[j][0] / tot
        logr += np.log(r)
    return 0.5 * simplified_size(variant, n) * float(np.exp(logr))
