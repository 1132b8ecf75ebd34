"""C-ABI checks that need no GPU: the library builds and loads, exports every
function include/tess.h declares, the ctypes mirrors of the structs match the
C compiler's layout, and calls fail cleanly (error code + message) when no
device can be used."""
import ctypes
import os
import re
import subprocess
import tempfile

import pytest

import paper_1002_3446_gb300 as tess

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "tess.h")


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(tess_[a-z0-9_]+)\s*\(", src)))


def test_header_declares_binding_names():
    assert declared_functions() == sorted(tess.EXPORTED)


def test_header_constants_match_binding():
    src = re.sub(r"/\*.*?\*/", "", open(HEADER).read(), flags=re.S)
    defs = {}
    for m in re.finditer(r"#define\s+(TESS_[A-Z0-9_]+)\s+\(?(-?[0-9]+)u?(?:\s*<<\s*([0-9]+))?", src):
        defs[m.group(1)] = int(m.group(2)) << int(m.group(3) or 0)
    assert len(defs) >= 29
    for name, value in defs.items():
        assert getattr(tess, name) == value, name


def test_library_exports_every_declared_symbol():
    lib = tess._load()
    out = subprocess.run(["nm", "-D", "--defined-only", tess.library_path()], capture_output=True, text=True,
                         check=True).stdout
    exported = set(re.findall(r"\bT (tess_[a-z0-9_]+)\b", out))
    for name in declared_functions():
        assert name in exported, name
        assert hasattr(lib, name)


def test_struct_layout_matches_c():
    prog = r"""
#include <stdio.h>
#include <stddef.h>
#include "tess.h"
int main(void) {
  printf("%zu %zu %zu %zu %zu %zu\n", sizeof(tess_process), offsetof(tess_process, sqrt_s),
         offsetof(tess_process, hist_hi), sizeof(tess_outputs), offsetof(tess_outputs, hist),
         offsetof(tess_process, flags));
  return 0;
}
"""
    with tempfile.TemporaryDirectory() as d:
        c = os.path.join(d, "l.c")
        exe = os.path.join(d, "l")
        open(c, "w").write(prog)
        subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), c, "-o", exe], check=True)
        vals = [int(x) for x in subprocess.run([exe], capture_output=True, text=True, check=True).stdout.split()]
    P, O = tess.tess_process, tess.tess_outputs
    assert vals == [ctypes.sizeof(P), P.sqrt_s.offset, P.hist_hi.offset, ctypes.sizeof(O), O.hist.offset,
                    P.flags.offset]


def test_version_and_error_strings():
    assert tess.tess_version().startswith("tess-gb300")
    assert isinstance(tess.tess_last_error(), str)


def test_cost_model_counts():
    # splits C(L+1,3) and four-vertex triples C(L+1,4) for L = n-1 legs
    assert tess.splits_and_triples(10) == (120, 210)
    assert tess.splits_and_triples(4) == (4, 1)
    # per-event Berends-Giele work grows between n^3 and n^4
    r = tess.bg_flops(12) / tess.bg_flops(11)
    assert (12 / 11) ** 3 < r < (12 / 11) ** 5


def test_init_without_usable_gpu_fails_cleanly():
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present; covered by the gpu tests")
    with pytest.raises(tess.TessError) as e:
        tess.tess_init(0)
    assert e.value.code in (tess.TESS_E_CUDA, tess.TESS_E_INVALID, tess.TESS_E_UNSUPPORTED)
    assert tess.tess_last_error() != ""


def test_null_arguments_rejected_without_device():
    lib = tess._load()
    assert lib.tess_init(0, None) == tess.TESS_E_INVALID
    assert lib.tess_generate(None, None, 0, 0, 0, None, None, 0, None) == tess.TESS_E_INVALID
    assert lib.tess_result(None, None, None, None) == tess.TESS_E_INVALID
    assert lib.tess_workspace_size(None, None, 0, None) == tess.TESS_E_INVALID
