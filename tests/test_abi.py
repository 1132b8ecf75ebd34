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


def _counted_flops(n, leaf_zeros, right_leaves=True):
    """FLOPs of the recursion by replaying the operation sequence of the
    complex-vector helpers (mdot, axpy, radd, ...) with a mask of structural
    zeros per operand: a product with a structurally zero factor is dropped
    when leaf_zeros is set (the first kept product of a sum is a multiply, 1
    FLOP; every further one an FMA, 2).  right_leaves: the right part of a
    split, the last part of a triple and the final contraction vector are
    treated as leaves where they are single legs (the register forms), or as
    general vectors (the wavefront forms, whose step code knows only the left
    and middle parts' lengths at compile time)."""
    L = n - 1
    full = [(True, True)] * 4
    leaf = [(False, False), (True, True), (True, True), (True, False)] if leaf_zeros else full
    rleaf = leaf if right_leaves else full
    realk = [True] * 4

    def sum_cost(products):  # products: list of bools (kept)
        k = sum(products)
        return 0 if k == 0 else 1 + 2 * (k - 1)

    def mdot_cc(a, b):  # re: a_r b_r, a_i b_i per m; im: a_r b_i, a_i b_r per m
        re = [a[m][0] and b[m][0] for m in range(4)] + [a[m][1] and b[m][1] for m in range(4)]
        im = [a[m][0] and b[m][1] for m in range(4)] + [a[m][1] and b[m][0] for m in range(4)]
        return sum_cost(re) + sum_cost(im)

    def mdot_ck(a):
        return sum_cost([a[m][0] for m in range(4)]) + sum_cost([a[m][1] for m in range(4)])

    def axpy_c(v):  # acc += s v: per component two FMAs on v's real part, two on its imaginary part
        return sum(2 * 2 * (int(v[m][0]) + int(v[m][1])) for m in range(4))

    total = 0
    for ln in range(2, L + 1):
        for a in range(0, L - ln + 1):
            b = a + ln - 1
            for i in range(a, b):
                jl = leaf if i == a else full
                jr = rleaf if i + 1 == b else full
                total += mdot_cc(jl, jr) + mdot_ck(jl) + mdot_ck(jr)
                total += 2 + 2 + axpy_c(jr) + axpy_c(jl) + 4 + 16 + 2
                total += (2 if i > a else 0) + (2 if b > i + 1 else 0)
                for j in range(i + 1, b):
                    ja = leaf if i == a else full
                    jc = rleaf if j + 1 == b else full
                    jb = leaf if j == i + 1 else full
                    total += mdot_cc(ja, jc) + axpy_c(jb)
            total += 20 + (16 if ln < L else 0)
    return total + mdot_cc(rleaf, full)


def test_cost_model_matches_a_replay_of_the_operations():
    for n in range(4, 13):
        assert _counted_flops(n, False) == tess.bg_flops(n), n
        assert _counted_flops(n, True) == tess.bg_flops_leaf(n), n
        assert _counted_flops(n, True, right_leaves=False) == tess.bg_flops_wave(n), n
        # unrolled wavefront form: right leaves too, final contraction general
        assert _counted_flops(n, True) - 18 + 30 == tess.bg_flops_wave_unrolled(n), n
    assert tess.flops_per_event(6, tess.TESS_K2_REG_HI) == tess.bg_flops_leaf(6) == 3432
    assert tess.flops_per_event(10, tess.TESS_K2_WAVE2) == tess.bg_flops_wave(10) == 29330
    assert tess.flops_per_event(10, tess.TESS_K2_WAVE2P) == tess.bg_flops(10) == 32426
    assert tess.flops_per_event(10, tess.TESS_K2_WAVE2U) == tess.bg_flops_wave_unrolled(10) == 27602
    # the one-kernel form runs the register form's amplitude code
    assert tess.flops_per_event(6, tess.TESS_K2_FUSED) == tess.bg_flops_leaf(6)
    assert tess.flops_per_event(6, tess.TESS_K2_REAL, random_pol=True) == tess.bg_flops_real_leaf(6)
    # exact-sum mode: register form for FP64 up to n = 5, FP32 up to n = 7
    assert tess.flops_per_event(4, -1, precision=tess.TESS_FP64) == tess.bg_flops_leaf(4)
    assert tess.flops_per_event(6, -1, precision=tess.TESS_FP64) == tess.bg_flops(6)
    assert tess.flops_per_event(7, -1, precision=tess.TESS_FP32_DS) == tess.bg_flops_leaf(7)


def _counted_flops_real(n, leaf_zeros):
    """The same replay for the real-current recursion (bg_amplitude_real):
    real four-vectors, a single leg's polarisation vector with an exact zero
    time component."""
    L = n - 1
    full = [True] * 4
    leaf = [False, True, True, True] if leaf_zeros else full

    def dot(a, b):
        k = sum(x and y for x, y in zip(a, b))
        return 0 if k == 0 else 1 + 2 * (k - 1)

    def axpy(v):
        return 2 * sum(v)

    total = 0
    for ln in range(2, L + 1):
        for a in range(0, L - ln + 1):
            b = a + ln - 1
            for i in range(a, b):
                jl = leaf if i == a else full
                jr = leaf if i + 1 == b else full
                total += dot(jl, jr) + dot(jl, full) + 1 + dot(jr, full) + 1
                total += axpy(jr) + axpy(jl) + axpy(full) + 4 + 1
                total += (1 if i > a else 0) + (1 if b > i + 1 else 0)
                for j in range(i + 1, b):
                    total += dot(leaf if i == a else full, leaf if j + 1 == b else full)
                    total += axpy(leaf if j == i + 1 else full)
            total += 12 + (12 if ln < L else 0)
    return total + dot(leaf, full)


def test_real_cost_model_matches_a_replay_of_the_operations():
    for n in range(4, 13):
        assert _counted_flops_real(n, False) == tess.bg_flops_real(n), n
        assert _counted_flops_real(n, True) == tess.bg_flops_real_leaf(n), n
    assert tess.flops_per_event(6, tess.TESS_K2_REAL_HI, random_pol=True) == tess.bg_flops_real_leaf(6)
    assert tess.flops_per_event(10, tess.TESS_K2_ROWS_REAL, random_pol=True) == tess.bg_flops_real(10)
    # complex-current forms on real vectors: their own count
    assert tess.flops_per_event(6, tess.TESS_K2_REG_HI, random_pol=True) == tess.bg_flops_leaf(6)
