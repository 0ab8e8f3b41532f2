"""The allocation-free entry point against the regular one, through the C ABI.

sme_estimate_sequence_noalloc is for callers that cannot allocate device
memory (code running inside another framework's memory pool, or real-time
code that forbids allocation after start-up): it keeps its scratch in one
fixed-size array in device memory.  This file is collected last, so a run that
stops at the first failure has run every other test before it.  Each call's
outputs must equal those of sme_estimate_sequence on the same inputs, on two
calls in a row (the shared array keeps the previous call's contents).
"""
import ctypes as C

import numpy as np
import pytest

from paper_1002_1168_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

DISP_TOL = 1e-4  # px, the tolerance the parity tests use for FP32 updates
FIELDS = ("mv", "cost", "disp", "iters", "npos", "mb_class", "sse_mb", "sse", "pred")


@pytest.fixture(scope="module")
def sme():
    from paper_1002_1168_gb300 import build as cuda_build
    from paper_1002_1168_gb300 import sme as m

    cuda_build.build()
    return m


def _noalloc(sme, params, luma, alpha, out):
    st = sme.Outputs(*[C.c_void_p(out[k].data_ptr()) if k in out else None for k in sme.OUTPUT_FIELDS])
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    return sme._lib().sme_estimate_sequence_noalloc(C.byref(params), C.c_void_p(luma.data_ptr()),
                                                    C.c_void_p(alpha.data_ptr()), luma.shape[0], None,
                                                    None, C.byref(st), stream)


def _compare(a, b):
    for k in FIELDS:
        if k == "disp":
            assert torch.max(torch.abs(a[k] - b[k])).item() <= DISP_TOL
        else:
            assert torch.equal(a[k], b[k]), k


def test_noalloc_matches_regular_entry_point_on_two_calls(sme):
    W, H, S, h = 352, 288, 16, 2
    est = sme.Estimator(W, H, search_range=S, subpel=h)
    params = sme.Params(W, H, S, h, 2.0, 1.0, 8, 1)
    for call, seed in enumerate((1002, 1010)):
        seq = synth.cif_sequence(seed=seed, frames=10 if call == 0 else 7)
        luma = torch.from_numpy(seq.luma).cuda()
        alpha = torch.from_numpy(seq.alpha[0]).cuda()
        want = est.estimate_sequence(luma, alpha, want=FIELDS[1:])
        got = est._alloc_outputs(luma.shape[0] - 1, FIELDS[1:], luma.device)
        for v in got.values():
            v.fill_(0x5A) if v.dtype != torch.float32 else v.fill_(float("nan"))
        assert _noalloc(sme, params, luma, alpha, got) == 0
        _compare(got, want)
    est.close()


def test_noalloc_rejects_problems_beyond_its_scratch(sme):
    W, H = 1920, 1088
    params = sme.Params(W, H, 16, 2, 2.0, 1.0, 8, 1)
    luma = torch.zeros((12, H, W), dtype=torch.uint8, device="cuda")
    out = {"mv": torch.empty((11, (W // 16) * (H // 16), 2), dtype=torch.int16, device="cuda")}
    assert _noalloc(sme, params, luma, luma, out) == 8  # SME_ERR_SCRATCH
    assert sme._lib().sme_strerror(8).decode().startswith("problem exceeds the fixed 4 MiB")
    # 11 frames fit
    assert _noalloc(sme, params, luma[:11], luma[:11], {"mv": out["mv"][:10]}) == 0
    assert (out["mv"][:10] == 0).all()
