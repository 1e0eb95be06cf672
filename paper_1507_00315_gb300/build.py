"""In-tree build of libskolem.so for sm_103a (nvcc, no cmake).

The exact-count kernels are templates over (delta, n, number of moduli); one
small generated translation unit per n instantiates them so nvcc can compile
them in parallel.  Objects are cached in ``_build/`` and rebuilt when a source
or header is newer.
"""
from __future__ import annotations

import concurrent.futures as cf
import glob
import os
import shutil
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(os.path.dirname(PKG), "include")
BUILD = os.path.join(PKG, "_build")
LIB = os.path.join(PKG, "libskolem.so")
MAX_N = 31
MAX_IE_N = 24          # kMaxIeN of csrc/sk_ie.cuh: orders with an inclusion-exclusion kernel
MIN_MIRROR_N = 6       # kMirrorMinN of csrc/sk_mirror.cuh: orders with a mirrored (Lemma 2.3) kernel

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
# Relocatable device code: the batch kernel calls the per-n walk functions
# across translation units (resolved by the device-link step below); every
# function is held to 128 registers, the budget of the kernels that call them.
NVCC_FLAGS = ["-std=c++17", "-O3", "-lineinfo", "-rdc=true", "-maxrregcount=128",
              "-Xcompiler", "-fPIC", "-I", CSRC, "-I", INCLUDE]
# Extra nvcc flags (e.g. "-DSK_INNER_BITS=4" to change the unrolled Gray
# width); objects for each flag set live in their own build directory.
EXTRA = os.environ.get("SK_NVCC_FLAGS", "").split()
if EXTRA:
    import hashlib
    BUILD = os.path.join(PKG, "_build", "x" + hashlib.sha1(" ".join(EXTRA).encode()).hexdigest()[:8])


def _nvcc():
    cand = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(cand):
        raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libskolem.so")
    return cand


def _headers():
    return glob.glob(os.path.join(CSRC, "*.cuh")) + glob.glob(os.path.join(CSRC, "*.h")) + \
        glob.glob(os.path.join(INCLUDE, "*.h"))


def _sources():
    gen = os.path.join(PKG, "_build", "gen")
    os.makedirs(gen, exist_ok=True)
    srcs = sorted(glob.glob(os.path.join(CSRC, "*.cu")))
    for n in range(1, MAX_N + 1):
        p = os.path.join(gen, f"sk_exact_n{n:02d}.cu")
        text = (f'#include "sk_exact_launch.cuh"\n#include "sk_batch.cuh"\n'
                f'SK_INSTANTIATE_EXACT({n})\nSK_DEFINE_BATCH({n})\n')
        if n <= MAX_IE_N:
            text += f'#include "sk_ie.cuh"\nSK_INSTANTIATE_IE({n})\n'
        if n >= MIN_MIRROR_N:
            text += f'#include "sk_mirror.cuh"\nSK_INSTANTIATE_MIRROR({n})\n'
        if not os.path.exists(p) or open(p).read() != text:
            with open(p, "w") as f:
                f.write(text)
        srcs.append(p)
    return srcs


def _stale(obj, deps):
    if not os.path.exists(obj):
        return True
    t = os.path.getmtime(obj)
    return any(os.path.getmtime(d) > t for d in deps)


def build(jobs: int | None = None, verbose: bool = False) -> str:
    nvcc = _nvcc()
    os.makedirs(BUILD, exist_ok=True)
    srcs = _sources()
    hdrs = _headers()
    objs, todo = [], []
    for s in srcs:
        o = os.path.join(BUILD, os.path.splitext(os.path.basename(s))[0] + ".o")
        objs.append(o)
        if _stale(o, [s] + hdrs + [os.path.abspath(__file__)]):
            todo.append((s, o))
    jobs = jobs or max(2, os.cpu_count() or 2)

    def compile_one(so):
        s, o = so
        cmd = [nvcc] + NVCC_FLAGS + EXTRA + ARCH + ["-c", s, "-o", o + ".tmp"]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed on {s}:\n{r.stderr}")
        os.replace(o + ".tmp", o)
        return s

    if todo:
        # largest orders first: they take longest
        todo.sort(key=lambda so: -os.path.getsize(so[0]) if "gen" not in so[0] else -int(so[0][-5:-3]))
        with cf.ThreadPoolExecutor(max_workers=jobs) as ex:
            for s in ex.map(compile_one, todo):
                if verbose:
                    print("compiled", os.path.basename(s), file=sys.stderr)
    stamp = os.path.join(BUILD, "linked_flags")
    same = os.path.exists(stamp) and open(stamp).read() == " ".join(EXTRA) and \
        os.path.exists(LIB) and os.path.getmtime(LIB) >= max(os.path.getmtime(o) for o in objs)
    if todo or not same:
        dlink = os.path.join(BUILD, "sk_dlink.o")
        cmd = [nvcc] + ARCH + ["-dlink", "-Xcompiler", "-fPIC", "-o", dlink] + objs
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"device link failed:\n{r.stderr}")
        cmd = [nvcc] + ARCH + ["-shared", "-cudart", "shared", "-o", LIB + ".tmp"] + objs + \
              [dlink, "-Xlinker", "-rpath,/usr/local/cuda/lib64"]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"link failed:\n{r.stderr}")
        os.replace(LIB + ".tmp", LIB)
        with open(stamp, "w") as f:
            f.write(" ".join(EXTRA))
    return LIB


if __name__ == "__main__":
    print(build(verbose=True))
