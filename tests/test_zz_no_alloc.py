"""The allocation-free entry point against the regular one, through the C ABI.

sme_estimate_sequence_noalloc is for callers that cannot allocate device
memory (code running inside another framework's memory pool, or real-time
code that forbids allocation after start-up): it keeps its scratch in one
fixed-size array in device memory.  This file is collected last, so a run that
stops at the first failure has run every other test before it.  Each call's
outputs must equal those of sme_estimate_sequence on the same inputs, on two
calls in a row (the shared array keeps the previous call's contents), with
and without a temporal field and seeds, on the default and on a separate
stream; and after a warm-up the calls must not change the device's free
memory.  The argument errors that return before any CUDA call are covered on
the CPU (tests/test_abi.py).
"""
import ctypes as C

import numpy as np
import pytest

from paper_1002_1168_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

DISP_TOL = 1e-4  # px, the tolerance the parity tests use for FP32 updates
FIELDS = ("mv", "cost", "disp", "iters", "npos", "mb_class", "sse_mb", "sse", "pred")
W, H, S, SUBPEL = 352, 288, 16, 2


@pytest.fixture(scope="module")
def sme():
    from paper_1002_1168_gb300 import build as cuda_build
    from paper_1002_1168_gb300 import sme as m

    cuda_build.build()
    return m


def _noalloc(sme, params, luma, alpha, out, temporal=None, seed=None, stream=None):
    st = sme.Outputs(*[C.c_void_p(out[k].data_ptr()) if k in out else None for k in sme.OUTPUT_FIELDS])
    s = stream if stream is not None else torch.cuda.current_stream()
    ptr = lambda t: None if t is None else C.c_void_p(t.data_ptr())  # noqa: E731
    return sme._lib().sme_estimate_sequence_noalloc(C.byref(params), ptr(luma), ptr(alpha), luma.shape[0],
                                                    ptr(temporal), ptr(seed), C.byref(st),
                                                    C.c_void_p(s.cuda_stream))


def _compare(a, b):
    for k in FIELDS:
        if k == "disp":
            assert torch.max(torch.abs(a[k] - b[k])).item() <= DISP_TOL
        else:
            assert torch.equal(a[k], b[k]), k


def _poisoned(est, P, device):
    got = est._alloc_outputs(P, FIELDS[1:], device)
    for v in got.values():
        v.fill_(0x5A) if v.dtype != torch.float32 else v.fill_(float("nan"))
    return got


def _case(seed, frames, with_temporal, with_seed):
    seq = synth.cif_sequence(seed=seed, frames=frames)
    luma = torch.from_numpy(seq.luma).cuda()
    alpha = torch.from_numpy(seq.alpha[0]).cuda()
    M, P = (W // 16) * (H // 16), frames - 1
    rng = np.random.default_rng(seed)
    tmp = sd = None
    if with_temporal:
        tmp = torch.from_numpy(rng.integers(-2 * S, 2 * S + 1, (M, 2)).astype(np.int16)).cuda()
    if with_seed:
        sd = torch.from_numpy(rng.normal(0, 6, (P, M, 2)).astype(np.float32)).cuda()
    return luma, alpha, tmp, sd


@pytest.mark.parametrize("with_temporal,with_seed", [(False, False), (True, False), (True, True)])
def test_noalloc_matches_regular_entry_point_on_two_calls(sme, with_temporal, with_seed):
    est = sme.Estimator(W, H, search_range=S, subpel=SUBPEL)
    params = sme.Params(W, H, S, SUBPEL, 2.0, 1.0, 8, 1)
    for call, (seed, frames) in enumerate(((1002, 10), (1010, 7))):
        luma, alpha, tmp, sd = _case(seed, frames, with_temporal, with_seed)
        want = est.estimate_sequence(luma, alpha, temporal_in=tmp, seed=sd, want=FIELDS[1:])
        got = _poisoned(est, frames - 1, luma.device)
        assert _noalloc(sme, params, luma, alpha, got, tmp, sd) == 0
        _compare(got, want)
    est.close()


def test_noalloc_on_a_separate_stream(sme):
    est = sme.Estimator(W, H, search_range=S, subpel=SUBPEL)
    params = sme.Params(W, H, S, SUBPEL, 2.0, 1.0, 8, 1)
    luma, alpha, tmp, sd = _case(1011, 8, True, True)
    want = est.estimate_sequence(luma, alpha, temporal_in=tmp, seed=sd, want=FIELDS[1:])
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        for _ in range(2):
            got = _poisoned(est, 7, luma.device)
            assert _noalloc(sme, params, luma, alpha, got, tmp, sd, stream=side) == 0
            _compare(got, want)  # the call synchronised its stream
    est.close()


def test_noalloc_allocates_nothing(sme):
    """After a warm-up call (which loads the kernels), further calls leave the
    device's free memory and PyTorch's pool exactly as they were."""
    est = sme.Estimator(W, H, search_range=S, subpel=SUBPEL)
    params = sme.Params(W, H, S, SUBPEL, 2.0, 1.0, 8, 1)
    luma, alpha, tmp, sd = _case(1012, 9, True, True)
    out = est._alloc_outputs(8, FIELDS[1:], luma.device)
    est.close()
    assert _noalloc(sme, params, luma, alpha, out, tmp, sd) == 0
    assert _noalloc(sme, params, luma, alpha, out) == 0
    torch.cuda.synchronize()
    free0, reserved0 = torch.cuda.mem_get_info()[0], torch.cuda.memory_reserved()
    for i in range(4):
        assert _noalloc(sme, params, luma, alpha, out, tmp if i % 2 else None, sd if i % 2 else None) == 0
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0
    assert torch.cuda.memory_reserved() == reserved0


def test_noalloc_rejects_problems_beyond_its_scratch(sme):
    W1, H1 = 1920, 1088
    params = sme.Params(W1, H1, 16, 2, 2.0, 1.0, 8, 1)
    luma = torch.zeros((12, H1, W1), dtype=torch.uint8, device="cuda")
    out = {"mv": torch.empty((11, (W1 // 16) * (H1 // 16), 2), dtype=torch.int16, device="cuda")}
    assert _noalloc(sme, params, luma, luma, out) == 8  # SME_ERR_SCRATCH
    assert sme._lib().sme_strerror(8).decode().startswith("problem exceeds the fixed 4 MiB")
    # 11 frames fit
    assert _noalloc(sme, params, luma[:11], luma[:11], {"mv": out["mv"][:10]}) == 0
    assert (out["mv"][:10] == 0).all()


def test_noalloc_rejects_seeds_above_eight_steps(sme):
    params = sme.Params(W, H, S, SUBPEL, 2.0, 1.0, 9, 1)
    luma, alpha, _, sd = _case(1013, 3, False, True)
    out = {"mv": torch.empty((2, (W // 16) * (H // 16), 2), dtype=torch.int16, device="cuda")}
    assert _noalloc(sme, params, luma, alpha, out, None, sd) == 1  # SME_ERR_ARG
