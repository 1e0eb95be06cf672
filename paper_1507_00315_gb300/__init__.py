"""Python binding of libskolem.so (argument marshalling only).

Every step of the counting runs in the library's CUDA kernels; this module
only converts Python values to the C structs of ``include/skolem.h`` and
back.  If the library has not been built, or no GB300-class device is
present, the calls raise: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libskolem.so")

SKOLEM, LANGFORD, HOOKED = 0, 1, 2
VARIANTS = {"skolem": SKOLEM, "langford": LANGFORD, "hooked": HOOKED}
REFLECTIONS_IDENTIFIED, COUNT_ALL = 0, 1
ARITH_LIMBS, ARITH_MONTGOMERY = 0, 1
SYMMETRY_NEGATION, SYMMETRY_NEGATION_EVEN = 0, 1      # Lemma 2.2; Lemmas 2.2 + 2.4
SYMMETRY_REVERSAL = 2                                  # Lemmas 2.2 + 2.3
SYMMETRY_REVERSAL_EVEN = 3                             # Lemmas 2.2 + 2.3 + 2.4
MAX_N = 31
MAX_IE_N = 24
MAX_PRIMES = 4
NOALLOC_MAX_ITEMS = 16384

SK_OK, SK_EINVAL, SK_ERANGE, SK_ECUDA, SK_ENOMEM, SK_ETIMEOUT, SK_EMISMATCH, SK_ECKPT = \
    0, -1, -2, -3, -4, -5, -6, -7


class SkolemError(RuntimeError):
    def __init__(self, status: int, what: str):
        self.status = status
        super().__init__(f"{what}: {strerror(status)} (status {status})")


class U128(ctypes.Structure):
    _fields_ = [("lo", ctypes.c_uint64), ("hi", ctypes.c_uint64)]

    def value(self) -> int:
        return self.lo | (self.hi << 64)


class CountOpts(ctypes.Structure):
    _fields_ = [("nprimes", ctypes.c_int),
                ("primes", ctypes.c_uint64 * MAX_PRIMES),
                ("convention", ctypes.c_int),
                ("walk_bits", ctypes.c_int),
                ("block_threads", ctypes.c_int),
                ("grid", ctypes.c_int),
                ("stream", ctypes.c_void_p),
                ("checkpoint_path", ctypes.c_char_p),
                ("chunk_items", ctypes.c_uint64),
                ("max_chunks", ctypes.c_uint64),
                ("arith", ctypes.c_int),
                ("symmetry", ctypes.c_int)]


class CountReport(ctypes.Structure):
    _fields_ = [("nprimes", ctypes.c_int),
                ("primes", ctypes.c_uint64 * MAX_PRIMES),
                ("residues", ctypes.c_uint64 * MAX_PRIMES),
                ("coefficient", U128),
                ("terms", ctypes.c_uint64),
                ("items", ctypes.c_uint64),
                ("walk_bits", ctypes.c_int),
                ("inner_bits", ctypes.c_int),
                ("arith", ctypes.c_int),
                ("block_threads", ctypes.c_int),
                ("grid", ctypes.c_int),
                ("chunks_total", ctypes.c_uint64),
                ("chunks_done", ctypes.c_uint64),
                ("chunks_resumed", ctypes.c_uint64),
                ("complete", ctypes.c_int),
                ("kernel_ms", ctypes.c_double),
                ("wall_ms", ctypes.c_double),
                ("symmetry", ctypes.c_int)]

    def as_dict(self) -> dict:
        k = self.nprimes
        return {"nprimes": k, "primes": list(self.primes[:k]), "residues": list(self.residues[:k]),
                "coefficient": self.coefficient.value(), "terms": self.terms, "items": self.items,
                "walk_bits": self.walk_bits, "inner_bits": self.inner_bits, "arith": self.arith,
                "block_threads": self.block_threads, "grid": self.grid,
                "chunks_total": self.chunks_total, "chunks_done": self.chunks_done,
                "chunks_resumed": self.chunks_resumed, "complete": bool(self.complete),
                "kernel_ms": self.kernel_ms, "wall_ms": self.wall_ms, "symmetry": self.symmetry}


class Job(ctypes.Structure):
    _fields_ = [("variant", ctypes.c_int), ("n", ctypes.c_int)]


class BatchOpts(ctypes.Structure):
    _fields_ = [("nprimes", ctypes.c_int),
                ("primes", ctypes.c_uint64 * MAX_PRIMES),
                ("convention", ctypes.c_int),
                ("mode", ctypes.c_int),
                ("no_graph", ctypes.c_int),
                ("repeats", ctypes.c_int),
                ("autotune", ctypes.c_int),
                ("block_threads", ctypes.c_int),
                ("walk_bits", ctypes.c_int * (MAX_N + 1)),
                ("stream", ctypes.c_void_p)]


class BatchReport(ctypes.Structure):
    _fields_ = [("kernel_ms", ctypes.c_double),
                ("kernel_ms_min", ctypes.c_double),
                ("wall_ms", ctypes.c_double),
                ("prepare_ms", ctypes.c_double),
                ("terms", ctypes.c_uint64),
                ("chunks", ctypes.c_uint64),
                ("launches", ctypes.c_int),
                ("grid", ctypes.c_int),
                ("block_threads", ctypes.c_int)]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_}


class TuneResult(ctypes.Structure):
    _fields_ = [("walk_bits", ctypes.c_int), ("block_threads", ctypes.c_int),
                ("terms_per_s", ctypes.c_double), ("candidates", ctypes.c_int)]


BATCH_PERSISTENT, BATCH_PER_JOB = 0, 1
PT_PLAIN, PT_LEARNED = 0, 1
MLP_KEEP_ORDER = (1 << 64) - 1      # sk_mlp_train seed: minibatches in the given order
PT_MAX_RUNGS = 64
PT_MAX_RUNGS_LEARNED = 32


class PtOpts(ctypes.Structure):
    _fields_ = [("rungs", ctypes.c_int), ("ladders", ctypes.c_int), ("seed", ctypes.c_uint64),
                ("burnin_frac", ctypes.c_double), ("beta", ctypes.POINTER(ctypes.c_double)),
                ("beta_max", ctypes.c_double), ("proposal", ctypes.c_int),
                ("model", ctypes.c_void_p), ("stream", ctypes.c_void_p),
                ("round_trips", ctypes.c_int)]


class PtReport(ctypes.Structure):
    _fields_ = [("rungs", ctypes.c_int), ("ladders", ctypes.c_int),
                ("iterations", ctypes.c_uint64), ("burnin", ctypes.c_uint64),
                ("beta", ctypes.c_double * PT_MAX_RUNGS), ("ratio", ctypes.c_double * PT_MAX_RUNGS),
                ("acc_move", ctypes.c_double * PT_MAX_RUNGS),
                ("acc_swap", ctypes.c_double * PT_MAX_RUNGS),
                ("estimate", ctypes.c_double), ("kernel_ms", ctypes.c_double),
                ("tune_ms", ctypes.c_double), ("wall_ms", ctypes.c_double),
                ("rel_stderr", ctypes.c_double), ("round_trips", ctypes.c_uint64)]

    def as_dict(self) -> dict:
        M = self.rungs
        return {"rungs": M, "ladders": self.ladders, "iterations": self.iterations,
                "burnin": self.burnin, "beta": list(self.beta[:M]), "ratio": list(self.ratio[:M]),
                "acc_move": list(self.acc_move[:M]), "acc_swap": list(self.acc_swap[:M]),
                "estimate": self.estimate, "kernel_ms": self.kernel_ms,
                "tune_ms": self.tune_ms, "wall_ms": self.wall_ms, "rel_stderr": self.rel_stderr,
                "round_trips": self.round_trips}

_lib = None


def lib():
    """The loaded libskolem.so (raises if it was not built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with __graft_entry__.build()")
        L = ctypes.CDLL(LIB_PATH)
        L.skolem_count.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.POINTER(U128)]
        L.skolem_count_ex.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.POINTER(CountOpts),
                                      ctypes.POINTER(U128), ctypes.POINTER(CountReport)]
        L.sk_count_plan.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.POINTER(CountOpts),
                                    ctypes.POINTER(CountReport)]
        L.skolem_item_residues.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_uint64,
                                           ctypes.c_uint64, ctypes.c_int,
                                           ctypes.POINTER(ctypes.c_uint64),
                                           ctypes.POINTER(ctypes.c_uint64)]
        L.sk_count_from_residues.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                             ctypes.POINTER(ctypes.c_uint64), ctypes.c_uint64,
                                             ctypes.POINTER(ctypes.c_uint64), ctypes.POINTER(U128)]
        L.skolem_item_residues_ex.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                              ctypes.c_uint64, ctypes.c_uint64, ctypes.c_int,
                                              ctypes.POINTER(ctypes.c_uint64), ctypes.c_int,
                                              ctypes.POINTER(ctypes.c_uint64)]
        L.skolem_item_residues_noalloc.argtypes = [
            ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_uint64, ctypes.c_uint64, ctypes.c_int,
            ctypes.POINTER(ctypes.c_uint64), ctypes.c_void_p, ctypes.POINTER(ctypes.c_uint64)]
        L.sk_count_inclusion_exclusion.argtypes = [ctypes.c_int, ctypes.c_int,
                                                   ctypes.POINTER(CountOpts),
                                                   ctypes.POINTER(U128), ctypes.POINTER(CountReport)]
        L.sk_ie_item_residues.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_uint64,
                                          ctypes.c_uint64, ctypes.c_int,
                                          ctypes.POINTER(ctypes.c_uint64),
                                          ctypes.POINTER(ctypes.c_uint64)]
        L.sk_count_extended.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.POINTER(CountOpts),
                                        ctypes.POINTER(U128), ctypes.POINTER(CountReport)]
        L.sk_extended_item_residues.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                                ctypes.c_uint64, ctypes.c_uint64, ctypes.c_int,
                                                ctypes.POINTER(ctypes.c_uint64),
                                                ctypes.POINTER(ctypes.c_uint64)]
        L.skolem_count_batch.argtypes = [ctypes.POINTER(Job), ctypes.c_int, ctypes.POINTER(BatchOpts),
                                         ctypes.POINTER(U128), ctypes.POINTER(ctypes.c_int),
                                         ctypes.POINTER(BatchReport)]
        L.skolem_autotune.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.POINTER(BatchOpts),
                                      ctypes.POINTER(TuneResult)]
        vp, u64, dp = ctypes.c_void_p, ctypes.c_uint64, ctypes.POINTER(ctypes.c_double)
        L.pt_estimate.argtypes = [ctypes.c_int, ctypes.c_int, u64, dp]
        L.pt_estimate_ex.argtypes = [ctypes.c_int, ctypes.c_int, u64, ctypes.POINTER(PtOpts), dp,
                                     ctypes.POINTER(PtReport)]
        L.sk_pt_run.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, vp, ctypes.c_int, u64, u64,
                                u64, vp, vp, vp, vp]
        L.sk_pt_run_trips.argtypes = L.sk_pt_run.argtypes + [vp]
        L.sk_pt_run_learned.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, vp, ctypes.c_int,
                                        u64, u64, u64, vp, vp, vp, vp]
        L.sk_pt_tune_ladder.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_double,
                                        u64, vp]
        L.sk_pt_estimate_hist.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, vp, ctypes.c_int,
                                          vp, ctypes.POINTER(ctypes.c_double), vp,
                                          ctypes.POINTER(ctypes.c_double)]
        L.sk_mlp_create.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, u64,
                                    ctypes.POINTER(ctypes.c_void_p)]
        L.sk_mlp_destroy.argtypes = [vp]
        L.sk_mlp_destroy.restype = None
        L.sk_mlp_dims.argtypes = [vp, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int)]
        L.sk_mlp_set_params.argtypes = [vp, vp]
        L.sk_mlp_get_params.argtypes = [vp, vp]
        L.sk_mlp_forward.argtypes = [vp, vp, ctypes.c_int, vp]
        L.sk_mlp_forward_bf16.argtypes = [vp, vp, ctypes.c_int, vp]
        L.sk_mlp_loss_grad.argtypes = [vp, vp, ctypes.c_int, ctypes.c_float, vp, vp]
        L.sk_mlp_get_train_state.argtypes = [vp, vp, vp, vp, ctypes.POINTER(ctypes.c_int64)]
        L.sk_mlp_set_gemm.argtypes = [vp, ctypes.c_int]
        L.sk_mlp_check.argtypes = [vp]
        L.sk_mlp_train.argtypes = [vp, vp, u64, ctypes.c_int, ctypes.c_int, ctypes.c_float,
                                   ctypes.c_float, u64, vp, vp]
        L.sk_int32_peak.argtypes = [ctypes.c_int, ctypes.POINTER(ctypes.c_double),
                                    ctypes.POINTER(ctypes.c_double)]
        L.sk_default_primes.argtypes = [ctypes.POINTER(ctypes.c_uint64)]
        L.sk_default_primes.restype = None
        L.sk_strerror.argtypes = [ctypes.c_int]
        L.sk_strerror.restype = ctypes.c_char_p
        L.sk_version.restype = ctypes.c_int
        _lib = L
    return _lib


def strerror(status: int) -> str:
    try:
        return lib().sk_strerror(status).decode()
    except Exception:  # library missing: still give a message
        return f"status {status}"


def _variant(v) -> int:
    if isinstance(v, str):
        return VARIANTS[v.lower()]
    return int(v)


def default_primes():
    out = (ctypes.c_uint64 * 4)()
    lib().sk_default_primes(out)
    return list(out)


def _opts(nprimes=0, primes=None, convention=REFLECTIONS_IDENTIFIED, walk_bits=0, block_threads=0,
          grid=0, stream=None, checkpoint=None, chunk_items=0, max_chunks=0, arith=ARITH_LIMBS,
          symmetry=SYMMETRY_NEGATION):
    o = CountOpts()
    o.nprimes = nprimes
    for i, p in enumerate(primes or []):
        o.primes[i] = p
    o.convention = convention
    o.walk_bits = walk_bits
    o.block_threads = block_threads
    o.grid = grid
    o.stream = stream
    o.checkpoint_path = checkpoint.encode() if checkpoint else None
    o.chunk_items = chunk_items
    o.max_chunks = max_chunks
    o.arith = arith
    o.symmetry = symmetry
    return o


def count(variant, n: int) -> int:
    """skolem_count: exact count, reflections identified (hooked: as is)."""
    out = U128()
    st = lib().skolem_count(_variant(variant), n, ctypes.byref(out))
    if st != SK_OK:
        raise SkolemError(st, f"skolem_count({variant}, {n})")
    return out.value()


def count_ex(variant, n: int, **kw):
    """skolem_count_ex: returns (count or None if incomplete, report dict).
    Keywords: nprimes, primes, convention, walk_bits, block_threads, grid,
    stream (int handle), checkpoint (path), chunk_items, max_chunks, arith,
    symmetry (SYMMETRY_NEGATION or SYMMETRY_NEGATION_EVEN)."""
    o = _opts(**kw)
    out = U128()
    rep = CountReport()
    st = lib().skolem_count_ex(_variant(variant), n, ctypes.byref(o), ctypes.byref(out),
                               ctypes.byref(rep))
    if st != SK_OK:
        raise SkolemError(st, f"skolem_count_ex({variant}, {n})")
    r = rep.as_dict()
    return (out.value() if r["complete"] else None), r


def count_inclusion_exclusion(variant, n: int, **kw):
    """sk_count_inclusion_exclusion: (count or None if incomplete, report
    dict), the same keywords as count_ex (arith and symmetry left at their
    defaults)."""
    o = _opts(**kw)
    out = U128()
    rep = CountReport()
    st = lib().sk_count_inclusion_exclusion(_variant(variant), n, ctypes.byref(o),
                                            ctypes.byref(out), ctypes.byref(rep))
    if st != SK_OK:
        raise SkolemError(st, f"sk_count_inclusion_exclusion({variant}, {n})")
    r = rep.as_dict()
    return (out.value() if r["complete"] else None), r


def count_extended(n: int, hole: int, **kw):
    """sk_count_extended: (count or None if incomplete, report dict) of the
    extended Skolem sequences with the given hole; keywords as count_ex."""
    o = _opts(**kw)
    out = U128()
    rep = CountReport()
    st = lib().sk_count_extended(n, hole, ctypes.byref(o), ctypes.byref(out), ctypes.byref(rep))
    if st != SK_OK:
        raise SkolemError(st, f"sk_count_extended({n}, {hole})")
    r = rep.as_dict()
    return (out.value() if r["complete"] else None), r


def extended_item_residues(n: int, hole: int, m: int, q_lo: int, count_: int, primes):
    """sk_extended_item_residues: list of per-item lists of residues."""
    k = len(primes)
    P = (ctypes.c_uint64 * k)(*primes)
    out = (ctypes.c_uint64 * (count_ * k))()
    st = lib().sk_extended_item_residues(n, hole, m, q_lo, count_, k, P, out)
    if st != SK_OK:
        raise SkolemError(st, "sk_extended_item_residues")
    return [list(out[i * k:(i + 1) * k]) for i in range(count_)]


def ie_item_residues(variant, n: int, m: int, q_lo: int, count_: int, primes):
    """sk_ie_item_residues: list of per-item lists of residues."""
    k = len(primes)
    P = (ctypes.c_uint64 * k)(*primes)
    out = (ctypes.c_uint64 * (count_ * k))()
    st = lib().sk_ie_item_residues(_variant(variant), n, m, q_lo, count_, k, P, out)
    if st != SK_OK:
        raise SkolemError(st, "sk_ie_item_residues")
    return [list(out[i * k:(i + 1) * k]) for i in range(count_)]


def count_plan(variant, n: int, **kw):
    """sk_count_plan: the report fields of the plan count_ex would run with
    these keywords (walk and inner bits, items, terms, chunks_total, ...),
    without running it; host code, no device."""
    o = _opts(**kw)
    rep = CountReport()
    st = lib().sk_count_plan(_variant(variant), n, ctypes.byref(o), ctypes.byref(rep))
    if st != SK_OK:
        raise SkolemError(st, f"sk_count_plan({variant}, {n})")
    return rep.as_dict()


def int32_peak(mode: int = 0):
    """sk_int32_peak: (ops per second, ms of the timed launch)."""
    v, ms = ctypes.c_double(), ctypes.c_double()
    st = lib().sk_int32_peak(mode, ctypes.byref(v), ctypes.byref(ms))
    if st != SK_OK:
        raise SkolemError(st, "sk_int32_peak")
    return v.value, ms.value


def item_residues(variant, n: int, m: int, q_lo: int, count_: int, primes, arith=ARITH_LIMBS):
    """skolem_item_residues(_ex): list of per-item lists of residues."""
    k = len(primes)
    P = (ctypes.c_uint64 * k)(*primes)
    out = (ctypes.c_uint64 * (count_ * k))()
    st = lib().skolem_item_residues_ex(_variant(variant), n, m, q_lo, count_, k, P, arith, out)
    if st != SK_OK:
        raise SkolemError(st, "skolem_item_residues")
    return [list(out[i * k:(i + 1) * k]) for i in range(count_)]


def count_from_residues(variant, n: int, residues, primes=None,
                        convention=REFLECTIONS_IDENTIFIED) -> int:
    """sk_count_from_residues: the exact count from the residues of a sum
    computed in parts (rows: parts, columns: one residue per prime, e.g. the
    item residues of each GPU's item range added modulo each prime); host
    code, no device."""
    rows = [list(r) for r in residues]
    if not rows:
        raise ValueError("no residues")
    k = len(primes) if primes is not None else len(rows[0])
    if any(len(r) != k for r in rows):
        raise ValueError("residues must be rows of one residue per prime")
    flat = (ctypes.c_uint64 * (len(rows) * k))(*[int(v) for r in rows for v in r])
    P = (ctypes.c_uint64 * k)(*primes) if primes is not None else None
    out = U128()
    st = lib().sk_count_from_residues(_variant(variant), n, convention, k, P, len(rows), flat,
                                      ctypes.byref(out))
    if st != SK_OK:
        raise SkolemError(st, "sk_count_from_residues")
    return out.value()


def item_residues_noalloc(variant, n: int, m: int, q_lo: int, count_: int, primes, stream=None):
    """skolem_item_residues_noalloc: as item_residues, with no device
    allocation inside the library (static scratch, at most NOALLOC_MAX_ITEMS
    items per call)."""
    k = len(primes)
    P = (ctypes.c_uint64 * k)(*primes)
    out = (ctypes.c_uint64 * (count_ * k))()
    st = lib().skolem_item_residues_noalloc(_variant(variant), n, m, q_lo, count_, k, P, stream, out)
    if st != SK_OK:
        raise SkolemError(st, "skolem_item_residues_noalloc")
    return [list(out[i * k:(i + 1) * k]) for i in range(count_)]


def _batch_opts(nprimes=0, primes=None, convention=REFLECTIONS_IDENTIFIED, mode=BATCH_PERSISTENT,
                no_graph=False, repeats=1, autotune=False, block_threads=0, walk_bits=None,
                stream=None):
    o = BatchOpts()
    o.nprimes = nprimes
    for i, p in enumerate(primes or []):
        o.primes[i] = p
    o.convention = convention
    o.mode = mode
    o.no_graph = int(bool(no_graph))
    o.repeats = repeats
    o.autotune = int(bool(autotune))
    o.block_threads = block_threads
    for n, m in (walk_bits or {}).items():
        o.walk_bits[n] = m
    o.stream = stream
    return o


def count_batch(jobs, **kw):
    """skolem_count_batch: jobs = [(variant, n), ...].  Returns (counts,
    statuses, report dict).  Keywords: nprimes, primes, convention, mode
    (BATCH_PERSISTENT / BATCH_PER_JOB), no_graph, repeats, autotune,
    block_threads, walk_bits ({n: m}), stream."""
    J = (Job * len(jobs))(*[Job(_variant(v), n) for v, n in jobs])
    o = _batch_opts(**kw)
    outs = (U128 * len(jobs))()
    stat = (ctypes.c_int * len(jobs))()
    rep = BatchReport()
    st = lib().skolem_count_batch(J, len(jobs), ctypes.byref(o), outs, stat, ctypes.byref(rep))
    if st != SK_OK:
        raise SkolemError(st, "skolem_count_batch")
    return [o_.value() for o_ in outs], list(stat), rep.as_dict()


def autotune(variant, n: int, **kw):
    """skolem_autotune: dict(walk_bits, block_threads, terms_per_s, candidates)."""
    o = _batch_opts(**kw)
    r = TuneResult()
    st = lib().skolem_autotune(_variant(variant), n, ctypes.byref(o), ctypes.byref(r))
    if st != SK_OK:
        raise SkolemError(st, "skolem_autotune")
    return {k: getattr(r, k) for k, _ in r._fields_}


# ------------------------------------------------------------- tempering

def _np():
    import numpy as np
    return np


def pt_run(variant, n: int, beta, ladders: int, iters: int, burnin: int, seed: int,
           want_final: bool = False, model=None, want_trips: bool = False):
    """sk_pt_run (sk_pt_run_trips with want_trips, sk_pt_run_learned with a
    model): dict(hist[M, 2n+1], acc_move[M], acc_swap[M], final_slots[L, M, n]
    or None, round_trips or None)."""
    np = _np()
    beta = np.ascontiguousarray(beta, dtype=np.float64)
    M = beta.shape[0]
    hist = np.zeros((M, 2 * n + 1), dtype=np.uint64)
    am = np.zeros(M, dtype=np.uint64)
    asw = np.zeros(M, dtype=np.uint64)
    if model is not None:
        st = lib().sk_pt_run_learned(_variant(variant), n, M, beta.ctypes.data, ladders, iters,
                                     burnin, seed, model.handle, hist.ctypes.data, am.ctypes.data,
                                     asw.ctypes.data)
        fin = None
    else:
        fin = np.zeros((ladders, M, n), dtype=np.uint8) if want_final else None
        args = (_variant(variant), n, M, beta.ctypes.data, ladders, iters, burnin, seed,
                hist.ctypes.data, am.ctypes.data, asw.ctypes.data,
                fin.ctypes.data if fin is not None else None)
        if want_trips:
            trips = np.zeros(1, dtype=np.uint64)
            st = lib().sk_pt_run_trips(*args, trips.ctypes.data)
        else:
            st = lib().sk_pt_run(*args)
    if st != SK_OK:
        raise SkolemError(st, "sk_pt_run")
    return {"hist": hist, "acc_move": am, "acc_swap": asw, "final_slots": fin,
            "round_trips": int(trips[0]) if want_trips and model is None else None}


def pt_estimate_hist(variant, n: int, beta, hist):
    """sk_pt_estimate_hist: (estimate, ratios, rel_stderr) of energy histograms
    shaped (M, 2n+1) or (groups, M, 2n+1); host code, no device."""
    np = _np()
    b = np.ascontiguousarray(beta, dtype=np.float64)
    h = np.ascontiguousarray(hist, dtype=np.uint64)
    M = b.shape[0]
    if h.ndim == 2:
        h = h[None]
    if h.ndim != 3 or h.shape[1:] != (M, 2 * n + 1):
        raise ValueError("hist must be (M, 2n+1) or (groups, M, 2n+1)")
    out, se = ctypes.c_double(), ctypes.c_double()
    ratios = np.zeros(M, dtype=np.float64)
    st = lib().sk_pt_estimate_hist(_variant(variant), n, M, b.ctypes.data, h.shape[0],
                                   h.ctypes.data, ctypes.byref(out), ratios.ctypes.data,
                                   ctypes.byref(se))
    if st != SK_OK:
        raise SkolemError(st, "sk_pt_estimate_hist")
    return out.value, ratios, se.value


def tune_ladder(variant, n: int, rungs: int = 32, beta_max: float = 32.0, seed: int = 0):
    np = _np()
    b = np.zeros(rungs, dtype=np.float64)
    st = lib().sk_pt_tune_ladder(_variant(variant), n, rungs, beta_max, seed, b.ctypes.data)
    if st != SK_OK:
        raise SkolemError(st, "sk_pt_tune_ladder")
    return b


def pt_estimate(variant, n: int, budget: int, rungs=0, ladders=0, seed=0, burnin_frac=0.0,
                beta=None, beta_max=0.0, model=None, stream=None, proposal=None,
                round_trips=False):
    """pt_estimate_ex: (estimate, report dict).  proposal defaults to PT_LEARNED
    with a model, else PT_PLAIN."""
    np = _np()
    o = PtOpts()
    o.rungs, o.ladders, o.seed, o.burnin_frac, o.beta_max = rungs, ladders, seed, burnin_frac, beta_max
    keep = None
    if beta is not None:
        keep = np.ascontiguousarray(beta, dtype=np.float64)
        o.rungs = keep.shape[0]
        o.beta = keep.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    if model is not None:
        o.proposal = PT_LEARNED
        o.model = model.handle
    if proposal is not None:
        o.proposal = proposal
    o.round_trips = 1 if round_trips else 0
    o.stream = stream
    out = ctypes.c_double()
    rep = PtReport()
    st = lib().pt_estimate_ex(_variant(variant), n, budget, ctypes.byref(o), ctypes.byref(out),
                              ctypes.byref(rep))
    if st != SK_OK:
        raise SkolemError(st, "pt_estimate_ex")
    return out.value, rep.as_dict()


class Mlp:
    """Handle of the move-proposal network (sk_mlp_*)."""

    def __init__(self, variant, n: int, max_batch: int = 4096, seed: int = 0):
        h = ctypes.c_void_p()
        st = lib().sk_mlp_create(_variant(variant), n, max_batch, seed, ctypes.byref(h))
        if st != SK_OK:
            raise SkolemError(st, "sk_mlp_create")
        self.handle, self.n, self.variant = h.value, n, _variant(variant)
        nm, npar = ctypes.c_int(), ctypes.c_int()
        lib().sk_mlp_dims(self.handle, ctypes.byref(nm), ctypes.byref(npar))
        self.n_moves, self.n_params = nm.value, npar.value

    def close(self):
        if self.handle:
            lib().sk_mlp_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_gemm(self, tensor_memory: bool):
        """True: tcgen05 forward (default); False: mma.sync forward."""
        st = lib().sk_mlp_set_gemm(self.handle, int(bool(tensor_memory)))
        if st != SK_OK:
            raise SkolemError(st, "sk_mlp_set_gemm")

    def check(self):
        st = lib().sk_mlp_check(self.handle)
        if st != SK_OK:
            raise SkolemError(st, "sk_mlp_check")

    def set_params(self, flat):
        np = _np()
        a = np.ascontiguousarray(flat, dtype=np.float32)
        assert a.size == self.n_params
        st = lib().sk_mlp_set_params(self.handle, a.ctypes.data)
        if st != SK_OK:
            raise SkolemError(st, "sk_mlp_set_params")

    def get_params(self):
        np = _np()
        a = np.zeros(self.n_params, dtype=np.float32)
        st = lib().sk_mlp_get_params(self.handle, a.ctypes.data)
        if st != SK_OK:
            raise SkolemError(st, "sk_mlp_get_params")
        return a

    def forward(self, slots):
        np = _np()
        s = np.ascontiguousarray(slots, dtype=np.uint8)
        out = np.zeros((s.shape[0], self.n_moves), dtype=np.float32)
        st = lib().sk_mlp_forward(self.handle, s.ctypes.data, s.shape[0], out.ctypes.data)
        if st != SK_OK:
            raise SkolemError(st, "sk_mlp_forward")
        return out

    def forward_bf16(self, slots):
        """sk_mlp_forward_bf16: the logits as the tempering chains read them,
        bf16 bit patterns (uint16, B x n_moves)."""
        np = _np()
        s = np.ascontiguousarray(slots, dtype=np.uint8)
        out = np.zeros((s.shape[0], self.n_moves), dtype=np.uint16)
        st = lib().sk_mlp_forward_bf16(self.handle, s.ctypes.data, s.shape[0], out.ctypes.data)
        if st != SK_OK:
            raise SkolemError(st, "sk_mlp_forward_bf16")
        return out

    def loss_grad(self, slots, beta_star: float):
        np = _np()
        s = np.ascontiguousarray(slots, dtype=np.uint8)
        loss = np.zeros(1, dtype=np.float32)
        g = np.zeros(self.n_params, dtype=np.float32)
        st = lib().sk_mlp_loss_grad(self.handle, s.ctypes.data, s.shape[0], beta_star,
                                    loss.ctypes.data, g.ctypes.data)
        if st != SK_OK:
            raise SkolemError(st, "sk_mlp_loss_grad")
        return float(loss[0]), g

    def train_state(self):
        """sk_mlp_get_train_state: dict(m, v, used, t) -- Adam's moments, the
        parameters the forward uses (BF16 weight copies widened, FP32 biases),
        and the step count; host parameter layout."""
        np = _np()
        m = np.zeros(self.n_params, dtype=np.float32)
        v = np.zeros(self.n_params, dtype=np.float32)
        u = np.zeros(self.n_params, dtype=np.float32)
        t = ctypes.c_int64()
        st = lib().sk_mlp_get_train_state(self.handle, m.ctypes.data, v.ctypes.data, u.ctypes.data,
                                          ctypes.byref(t))
        if st != SK_OK:
            raise SkolemError(st, "sk_mlp_get_train_state")
        return {"m": m, "v": v, "used": u, "t": t.value}

    def train(self, states, epochs: int = 1, batch: int = 4096, lr: float = 1e-3,
              beta_star: float = 2.0, seed: int = 0):
        np = _np()
        s = np.ascontiguousarray(states, dtype=np.uint8)
        loss = np.zeros(1, dtype=np.float32)
        ms = np.zeros(1, dtype=np.float64)
        st = lib().sk_mlp_train(self.handle, s.ctypes.data, s.shape[0], epochs, batch, lr,
                                beta_star, seed, loss.ctypes.data, ms.ctypes.data)
        if st != SK_OK:
            raise SkolemError(st, "sk_mlp_train")
        return float(loss[0]), float(ms[0])
