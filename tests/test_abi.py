"""The C-ABI library loads and exports every entry point of include/sme.h.

CPU only: no call here touches a GPU (host-only helpers and argument checks
that return before any CUDA call)."""
import ctypes as C
import math
import os
import re

import pytest

from conftest import ROOT
from paper_1002_1168_gb300 import build as cuda_build
from paper_1002_1168_gb300 import sme


@pytest.fixture(scope="module")
def lib():
    cuda_build.build()
    return sme._lib()


def header_entry_points():
    text = open(os.path.join(ROOT, "include", "sme.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(sme_[a-z_0-9]+)\s*\(", text)))


def test_every_declared_symbol_is_exported(lib):
    names = header_entry_points()
    assert len(names) >= 20
    assert sorted(sme.EXPORTS) == names
    for n in names:
        assert hasattr(lib, n), n


def test_exports_are_plain_c_symbols():
    out = os.popen(f"nm -D --defined-only {sme.LIB_PATH}").read()
    for n in header_entry_points():
        assert re.search(rf"\bT {n}$", out, re.M), n


def test_host_only_helpers(lib):
    assert lib.sme_psnr(0, 64, 64) == math.inf
    assert lib.sme_psnr(64 * 64, 64, 64) == pytest.approx(20 * math.log10(255.0), abs=1e-12)
    assert lib.sme_strerror(4).decode().startswith("a bounded device wait")
    assert lib.sme_packed_words(176) == 8 and lib.sme_packed_words(352) == 12 and lib.sme_packed_words(368) == 16
    p = sme.Params()
    lib.sme_default_params(C.byref(p), 352, 288)
    assert (p.search_range, p.subpel, p.theta, p.epsilon, p.max_iters, p.ref_distance) == (16, 1, 2.0, 1.0, 8, 1)


@pytest.mark.parametrize("field,value,code", [
    ("width", 100, 2), ("height", 0, 2), ("width", 8208, 2), ("search_range", 0, 1),
    ("search_range", 65, 1), ("subpel", 4, 1), ("theta", 0.0, 1), ("epsilon", 5.0, 1),
    ("max_iters", 17, 1), ("ref_distance", 0, 1),
])
def test_create_rejects_bad_params_before_touching_cuda(lib, field, value, code):
    p = sme.Params()
    lib.sme_default_params(C.byref(p), 176, 144)
    setattr(p, field, value)
    h = C.c_void_p()
    assert lib.sme_create(C.byref(h), C.byref(p), None) == code
    assert not h.value


def test_null_context_is_an_argument_error(lib):
    assert lib.sme_destroy(None) == 1
    assert lib.sme_synchronize(None) == 1
    assert lib.sme_estimate(None, None) == 1
    assert lib.sme_debug_set_fault(None, 0, 0) == 1


def header_enums():
    """name -> value of every `SME_* = n` enumerator in include/sme.h."""
    text = open(os.path.join(ROOT, "include", "sme.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return {m.group(1): int(m.group(2)) for m in re.finditer(r"\b(SME_[A-Z_0-9]+)\s*=\s*(\d+)", text)}


def test_binding_constants_match_the_header():
    """The binding's option, schedule and class constants are the header's."""
    enums = header_enums()
    names = [n for n in dir(sme) if n.startswith("SME_OPT_")]
    assert len(names) >= 8
    for n in names:
        assert getattr(sme, n) == enums[n], n
    for name, value in sme.SCHEDULES.items():
        assert enums[f"SME_SCHED_{name.upper()}"] == value, name
    assert set(n for n in enums if n.startswith("SME_OPT_")) == set(names)


def _fake_device_ptr(n=0):
    """A 16-byte aligned non-null address: the argument checks below return
    before any CUDA call, so nothing ever dereferences it."""
    return C.c_void_p(0x10000 + 256 * n)


def test_seeded_runs_above_eight_steps_are_rejected_before_touching_cuda(lib):
    """Seeds make an MB run up to two pixel-recursive searches, whose position
    record holds 5 + 2*9*8 entries: max_iters > 8 with seeds is an argument
    error in the batch and the allocation-free entry points."""
    p = sme.Params()
    lib.sme_default_params(C.byref(p), 176, 144)
    p.max_iters = 9
    out = sme.Outputs(_fake_device_ptr(3), *([None] * 8))
    seq = sme.Sequence(176, 144, 3, _fake_device_ptr(1), _fake_device_ptr(2), None, _fake_device_ptr(4), out)
    h = C.c_void_p()
    assert lib.sme_batch_create(C.byref(h), C.byref(p), C.byref(seq), 1, None) == 1
    assert not h.value
    assert lib.sme_estimate_sequence_noalloc(C.byref(p), _fake_device_ptr(1), _fake_device_ptr(2), 3, None,
                                             _fake_device_ptr(4), C.byref(out), None) == 1


@pytest.mark.parametrize("case", ["null_luma", "null_mv", "misaligned", "frames", "size", "scratch"])
def test_noalloc_argument_errors_before_touching_cuda(lib, case):
    """The allocation-free entry point validates everything before its first
    CUDA call: null or misaligned pointers, too few frames, bad sizes, and
    problems larger than its fixed scratch."""
    p = sme.Params()
    lib.sme_default_params(C.byref(p), 176, 144)
    luma, alpha, frames = _fake_device_ptr(1), _fake_device_ptr(2), 3
    out = sme.Outputs(_fake_device_ptr(3), *([None] * 8))
    want = 1
    if case == "null_luma":
        luma = None
    elif case == "null_mv":
        out.mv = None
    elif case == "misaligned":
        alpha = C.c_void_p(alpha.value + 4)
    elif case == "frames":
        frames = 1
    elif case == "size":
        p.width, want = 170, 2
    elif case == "scratch":
        lib.sme_default_params(C.byref(p), 1920, 1088)
        frames, want = 12, 8
    assert lib.sme_estimate_sequence_noalloc(C.byref(p), luma, alpha, frames, None, None, C.byref(out), None) == want


def test_packed_sad_rate_rejects_bad_arguments_before_touching_cuda(lib):
    """The measurement helper checks its arguments before any CUDA call."""
    out = (C.c_uint32 * 4)()
    grid = C.c_int(-1)
    f = lib.sme_packed_sad_rate_launch
    for cps, iters, o, g in ((0, 10, out, grid), (9, 10, out, grid), (1, 0, out, grid), (1, 10, None, grid),
                             (1, 10, out, None)):
        assert f(cps, iters, o, None, g if g is None else C.byref(g)) == 1  # SME_ERR_ARG
    assert grid.value == -1
