"""The C ABI library loads and exports every function include/skolem.h
declares; argument checks answer before any device work; without a GPU the
computing calls fail loudly (no CPU fallback)."""
import ctypes
import os
import re

import pytest

import paper_1507_00315_gb300 as sk

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_functions():
    names = set()
    for h in os.listdir(os.path.join(ROOT, "include")):
        if not h.endswith(".h"):
            continue
        text = open(os.path.join(ROOT, "include", h)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?[A-Za-z_][\w\s\*]*?\b(\w+)\s*\([^;{]*\)\s*;", text, re.M):
            names.add(m.group(1))
    return names


def test_header_symbols_exported():
    L = sk.lib()
    names = _declared_functions()
    assert "skolem_count" in names and "sk_strerror" in names
    for name in names:
        assert hasattr(L, name), name


def test_strerror_and_version():
    assert sk.strerror(0) == "ok"
    assert "checkpoint" in sk.strerror(sk.SK_ECKPT)
    assert sk.lib().sk_version() >= 100
    p = sk.default_primes()
    assert len(set(p)) == 4 and all(x % 2 == 1 and x < 1 << 62 for x in p)


def test_argument_checks_without_device():
    for bad in ((3, 4), (0, 0), (0, 32)):
        with pytest.raises(sk.SkolemError) as e:
            sk.count(*bad)
        assert e.value.status == sk.SK_EINVAL


def test_fails_loudly_without_gpu():
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(sk.SkolemError) as e:
        sk.count(0, 8)
    assert e.value.status == sk.SK_ECUDA
