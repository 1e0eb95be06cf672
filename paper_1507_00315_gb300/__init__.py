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
MAX_N = 28
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
                ("arith", ctypes.c_int)]


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
                ("wall_ms", ctypes.c_double)]

    def as_dict(self) -> dict:
        k = self.nprimes
        return {"nprimes": k, "primes": list(self.primes[:k]), "residues": list(self.residues[:k]),
                "coefficient": self.coefficient.value(), "terms": self.terms, "items": self.items,
                "walk_bits": self.walk_bits, "inner_bits": self.inner_bits, "arith": self.arith,
                "block_threads": self.block_threads, "grid": self.grid,
                "chunks_total": self.chunks_total, "chunks_done": self.chunks_done,
                "chunks_resumed": self.chunks_resumed, "complete": bool(self.complete),
                "kernel_ms": self.kernel_ms, "wall_ms": self.wall_ms}


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
        L.skolem_item_residues.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_uint64,
                                           ctypes.c_uint64, ctypes.c_int,
                                           ctypes.POINTER(ctypes.c_uint64),
                                           ctypes.POINTER(ctypes.c_uint64)]
        L.skolem_item_residues_ex.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                              ctypes.c_uint64, ctypes.c_uint64, ctypes.c_int,
                                              ctypes.POINTER(ctypes.c_uint64), ctypes.c_int,
                                              ctypes.POINTER(ctypes.c_uint64)]
        L.skolem_item_residues_noalloc.argtypes = [
            ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_uint64, ctypes.c_uint64, ctypes.c_int,
            ctypes.POINTER(ctypes.c_uint64), ctypes.c_void_p, ctypes.POINTER(ctypes.c_uint64)]
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
          grid=0, stream=None, checkpoint=None, chunk_items=0, max_chunks=0, arith=ARITH_LIMBS):
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
    stream (int handle), checkpoint (path), chunk_items, max_chunks, arith."""
    o = _opts(**kw)
    out = U128()
    rep = CountReport()
    st = lib().skolem_count_ex(_variant(variant), n, ctypes.byref(o), ctypes.byref(out),
                               ctypes.byref(rep))
    if st != SK_OK:
        raise SkolemError(st, f"skolem_count_ex({variant}, {n})")
    r = rep.as_dict()
    return (out.value() if r["complete"] else None), r


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
