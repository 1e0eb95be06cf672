"""The binding's ctypes structures have the field offsets and sizes of the C
structures declared in include/skolem.h: a small C program compiled against
the header prints offsetof / sizeof, which must equal ctypes' view (no GPU)."""
import ctypes
import os
import shutil
import subprocess
import tempfile

import pytest

import paper_1507_00315_gb300 as sk

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

# C struct name -> binding class, fields compared by name
PAIRS = {
    "sk_u128": sk.U128,
    "sk_count_opts": sk.CountOpts,
    "sk_count_report": sk.CountReport,
    "sk_job": sk.Job,
    "sk_batch_opts": sk.BatchOpts,
    "sk_batch_report": sk.BatchReport,
    "sk_tune_result": sk.TuneResult,
    "sk_pt_opts": sk.PtOpts,
    "sk_pt_report": sk.PtReport,
}


def _c_layout():
    cc = shutil.which("gcc") or shutil.which("cc")
    if not cc:
        pytest.skip("no C compiler")
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "skolem.h"', 'int main(void) {']
    for cname, cls in PAIRS.items():
        lines.append(f'  printf("{cname} sizeof %zu\\n", sizeof({cname}));')
        for fname, _ in cls._fields_:
            lines.append(f'  printf("{cname} {fname} %zu\\n", offsetof({cname}, {fname}));')
    lines += ['  return 0;', '}']
    with tempfile.TemporaryDirectory() as d:
        src, exe = os.path.join(d, "layout.c"), os.path.join(d, "layout")
        with open(src, "w") as f:
            f.write("\n".join(lines) + "\n")
        subprocess.run([cc, "-std=c11", "-I", os.path.join(ROOT, "include"), src, "-o", exe],
                       check=True, capture_output=True)
        out = subprocess.run([exe], check=True, capture_output=True, text=True).stdout
    layout = {}
    for line in out.splitlines():
        cname, key, val = line.split()
        layout[(cname, key)] = int(val)
    return layout


def test_struct_layouts_match_header():
    layout = _c_layout()
    for cname, cls in PAIRS.items():
        assert layout[(cname, "sizeof")] == ctypes.sizeof(cls), cname
        for fname, _ in cls._fields_:
            assert layout[(cname, fname)] == getattr(cls, fname).offset, (cname, fname)


def test_every_c_field_is_bound():
    # every field the header declares for these structures has a ctypes field
    # of the same name (the C compiler rejects unknown names above; this
    # catches fields the binding forgot)
    import re
    text = open(os.path.join(ROOT, "include", "skolem.h")).read()
    for cname, cls in PAIRS.items():
        if cname == "sk_u128":
            continue
        m = re.search(r"typedef struct %s \{(.*?)\} %s;" % (cname, cname), text, re.S)
        assert m, cname
        body = re.sub(r"/\*.*?\*/", "", m.group(1), flags=re.S)
        declared = set()
        for decl in body.split(";"):
            decl = decl.strip()
            if not decl:
                continue
            for part in decl.split(","):
                name = re.findall(r"([A-Za-z_]\w*)\s*(?:\[[^\]]*\])?\s*$", part.strip())
                if name:
                    declared.add(name[-1])
        bound = {f for f, _ in cls._fields_}
        assert declared == bound, (cname, declared ^ bound)
