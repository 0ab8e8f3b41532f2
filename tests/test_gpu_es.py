"""GPU exhaustive search (the ES row of Table 1, the comparison method of
Table 2) against the oracle's: the same best vector (first minimum in raster
order over V) and the same SAD for every MB, full- and half-pel, interior and
edge MBs, and the invariant that the method never beats it."""
import numpy as np
import pytest

import oracle as O
from paper_1002_1168_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sme():
    from paper_1002_1168_gb300 import build as cuda_build
    from paper_1002_1168_gb300 import sme as m

    cuda_build.build()
    return m


def _check(sme, luma, S, h, rd=1):
    F, H, W = luma.shape
    est = sme.Estimator(W, H, search_range=S, subpel=h, ref_distance=rd)
    mv, sad = est.full_search(torch.from_numpy(luma).cuda())
    mv, sad = mv.cpu().numpy(), sad.cpu().numpy().view(np.uint32)
    for k in range(F - rd):
        bm, bs, _ = O.full_search(luma[k], luma[k + rd], W, H, h, S)
        assert np.array_equal(mv[k], bm), f"pair {k}: vectors"
        assert np.array_equal(sad[k], bs), f"pair {k}: SAD"
    est.close()
    return mv, sad


@pytest.mark.parametrize("S,h", [(16, 1), (7, 1), (16, 2), (3, 2)])
def test_qcif_pair(sme, S, h):
    seq = synth.qcif_pair()
    _check(sme, seq.luma, S, h)


def test_cif_pairs_halfpel_and_method_never_beats_it(sme):
    seq = synth.cif_sequence(frames=4)
    mv, sad = _check(sme, seq.luma, 16, 2)
    o = O.estimate_sequence(O.OracleParams(352, 288, 16, 2), seq.luma, seq.alpha[0])
    op = o["mbclass"] == 1
    assert (o["cost"][op] >= sad[op]).all()


@pytest.mark.parametrize("W,H,S,h", [(16, 16, 8, 2), (48, 48, 1, 2), (96, 64, 32, 2), (64, 32, 5, 1)])
def test_edges_and_ranges_random_content(sme, W, H, S, h):
    luma, _ = synth.random_frames(W, H, 3, seed=W + H + S)
    _check(sme, luma, S, h)


def test_flat_frames_tie_to_first_in_raster_order(sme):
    luma = np.full((2, 64, 64), 77, np.uint8)
    mv, sad = _check(sme, luma, 4, 2)
    assert (sad == 0).all()
    # every MB's first position in raster order is (lox, loy)
    for m in range(16):
        lox, hix, loy, hiy = O.valid_range(64, 64, 16, 4, 2, 16 * (m % 4), 16 * (m // 4))
        assert tuple(mv[0, m]) == (lox, loy)


def test_ref_distance_two(sme):
    seq = synth.cif_sequence(frames=4)
    _check(sme, seq.luma, 16, 2, rd=2)


def _vsad(a, b):
    return sum(abs(((a >> (8 * i)) & 0xFF) - ((b >> (8 * i)) & 0xFF)) for i in range(4))


def _fshr(lo, hi, sh):
    return (((hi << 32) | lo) >> (sh & 31)) & 0xFFFFFFFF


def test_packed_sad_rate_kernel_does_the_counted_work(sme):
    """The measurement kernel behind the integer rooflines' measured op-mix
    rate computes its chains exactly (checked for a few threads against a
    host restatement of funnel shift, packed absolute difference and add),
    so the timed work is the counted work."""
    import ctypes as C
    iters, cps = 7, 1
    n = torch.cuda.get_device_properties(0).multi_processor_count * cps * 256
    out = torch.zeros(n, dtype=torch.int32, device="cuda")
    grid = C.c_int()
    st = torch.cuda.current_stream()
    assert sme._lib().sme_packed_sad_rate_launch(cps, iters, C.c_void_p(out.data_ptr()), C.c_void_p(st.cuda_stream),
                                                 C.byref(grid)) == 0
    torch.cuda.synchronize()
    assert grid.value * 256 == n
    got = out.cpu().numpy().view(np.uint32)
    M = 0xFFFFFFFF
    for t in (0, 1, 77, 255, 256, n - 1):
        acc = [(t * 0x9E3779B9 + k * 0x85EBCA6B) & M for k in range(8)]
        z = [(t ^ ((k * 0x27D4EB2D) & M)) & M for k in range(8)]
        sh = (t & 3) * 8
        for _ in range(iters):
            for k in range(8):
                acc[k] = (_vsad(_fshr(acc[k], acc[(k + 1) & 7], sh), z[k]) + acc[k]) & M
        r = 0
        for k in range(8):
            r ^= acc[k]
        assert int(got[t]) == r, t
    assert sme.packed_sad_rate(ctas_per_sm=2, iters=2000, reps=1) > 0
