"""Parity at the limits of the interface: the largest search range (S = 64),
the most pixel-recursive steps (K = 16), the widest and the tallest frames
(8192 pixels), no pixel-recursive step at all (K = 0) and the largest
convergence factor, through every schedule, the four-vector mode and the
exhaustive search; and the errors one step beyond each limit."""
import ctypes as C

import numpy as np
import pytest

import oracle as O
from paper_1002_1168_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

SCHEDULES = ["pair", "pair_staged", "mb", "cluster"]


@pytest.fixture(scope="module")
def sme():
    from paper_1002_1168_gb300 import build as cuda_build
    from paper_1002_1168_gb300 import sme as m

    cuda_build.build()
    return m


def cuda(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _estimate(sme, luma, alpha, S, h, K, eps, schedule):
    F, H, W = luma.shape
    est = sme.Estimator(W, H, search_range=S, subpel=h, epsilon=eps, max_iters=K)
    if schedule == "pair_staged":
        est.set_schedule("pair")
        est.set_option(sme.SME_OPT_PAIR_DIRECT, 0)
    else:
        est.set_schedule(schedule)
    try:
        g = est.estimate_sequence(cuda(luma), cuda(alpha), want=("cost", "disp", "iters", "npos", "mb_class", "sse"))
    except sme.SmeError as e:
        est.close()
        if schedule == "cluster" and e.status == 2:  # SME_ERR_SIZE: the sequence does not fit one cluster
            pytest.skip("the sequence needs more shared memory than one cluster has")
        raise
    g = {k: v.cpu().numpy() for k, v in g.items()}
    est.close()
    return g


def _check(g, o):
    assert np.array_equal(g["mb_class"], o["mbclass"])
    assert np.array_equal(g["mv"], o["mv"])
    assert np.array_equal(g["cost"].view(np.uint32), o["cost"])
    assert np.array_equal(g["iters"], o["iters"])
    assert np.array_equal(g["npos"], o["npos"])
    assert np.array_equal(g["disp"].view(np.uint32), o["disp"].view(np.uint32))
    assert np.array_equal(g["sse"].view(np.uint64), o["sse"])


CASES = {
    # name: (W, H, F, S, h, K, eps)
    "largest_search_range_and_steps": (256, 192, 3, 64, 2, 16, 1.0),
    "widest_frame": (8192, 32, 3, 16, 2, 8, 1.0),
    "tallest_frame": (32, 8192, 3, 16, 2, 8, 1.0),
    "no_recursive_step_largest_eps": (128, 96, 3, 32, 1, 0, 4.0),
}


@pytest.mark.parametrize("schedule", SCHEDULES)
@pytest.mark.parametrize("case", list(CASES))
def test_limits_every_schedule(sme, case, schedule):
    W, H, F, S, h, K, eps = CASES[case]
    luma, alpha = synth.random_frames(W, H, F, seed=W + 3 * H + S)
    g = _estimate(sme, luma, alpha, S, h, K, eps, schedule)
    o = O.estimate_sequence(O.OracleParams(W, H, S, h, 2.0, eps, K), luma, alpha)
    _check(g, o)
    if K == 16:
        assert o["iters"].max() > 1


@pytest.mark.parametrize("schedule", ["mb", "pair"])
@pytest.mark.parametrize("case", list(CASES))
def test_limits_four_vectors(sme, case, schedule):
    W, H, F, S, h, K, eps = CASES[case]
    luma, alpha = synth.random_frames(W, H, F, seed=W + 5 * H + S)
    est = sme.Estimator(W, H, search_range=S, subpel=h, epsilon=eps, max_iters=K, four_mv=True)
    est.set_schedule(schedule)
    g = est.estimate_sequence(cuda(luma), cuda(alpha), want=("cost", "disp", "iters", "npos", "mb_class", "sse"))
    g = {k: v.cpu().numpy() for k, v in g.items()}
    est.close()
    o = O.estimate_sequence4(O.OracleParams(W, H, S, h, 2.0, eps, K), luma, alpha)
    _check(g, o)


@pytest.mark.parametrize("case", ["largest_search_range_and_steps", "widest_frame", "tallest_frame"])
def test_limits_exhaustive_search(sme, case):
    W, H, F, S, h, _, _ = CASES[case]
    luma, _ = synth.random_frames(W, H, 2, seed=W + 7 * H)
    est = sme.Estimator(W, H, search_range=S, subpel=h)
    mv, sad = est.full_search(cuda(luma))
    est.close()
    bm, bs, _ = O.full_search(luma[0], luma[1], W, H, h, S)
    assert np.array_equal(mv[0].cpu().numpy(), bm)
    assert np.array_equal(sad[0].cpu().numpy().view(np.uint32), bs)


@pytest.mark.parametrize("field,value,status", [
    ("width", 8192 + 16, 2), ("height", 8192 + 16, 2), ("width", 24, 2), ("search_range", 65, 1),
    ("search_range", 0, 1), ("max_iters", 17, 1), ("max_iters", -1, 1), ("epsilon", 4.5, 1), ("theta", 0.0, 1),
    ("subpel", 4, 1), ("ref_distance", 0, 1)])
def test_one_step_beyond_each_limit(sme, field, value, status):
    from paper_1002_1168_gb300.sme import Params, _lib

    p = Params(64, 64, 16, 2, 2.0, 1.0, 8, 1)
    setattr(p, field, value)
    h = C.c_void_p()
    assert _lib().sme_create(C.byref(h), C.byref(p), None) == status
    assert not h.value


@pytest.mark.parametrize("schedule", ["mb", "pair", "sparse"])
def test_seeded_search_at_the_position_log_bound(sme, schedule):
    """Seeds with max_iters = 8 on unstructured frames with far seeds: the
    seed often wins and both searches run (reading c21), filling the position
    record towards its 149-entry bound; every output equals the oracle's.
    One step more is refused before any GPU work."""
    W = H = 96
    rng = np.random.default_rng(17)
    luma = rng.integers(0, 256, (3, H, W), dtype=np.uint8)
    alpha = np.full((3, H, W), 255, np.uint8)
    M = (W // 16) * (H // 16)
    seed = rng.normal(0, 10, (2, M, 2)).astype(np.float32)
    est = sme.Estimator(W, H, search_range=16, subpel=2, max_iters=8)
    est.set_schedule(schedule)
    g = est.estimate_sequence(torch.from_numpy(luma).cuda(), torch.from_numpy(alpha).cuda(),
                              seed=torch.from_numpy(seed).cuda(), want=("cost", "iters", "npos", "mb_class", "sse"))
    o = O.estimate_sequence(O.OracleParams(W, H, 16, 2, max_iters=8), luma, alpha, seed=seed)
    assert np.array_equal(g["mv"].cpu().numpy(), o["mv"])
    assert np.array_equal(g["iters"].cpu().numpy(), o["iters"])
    assert np.array_equal(g["npos"].cpu().numpy(), o["npos"])
    assert int(o["npos"].max()) <= 149
    est.close()
    est = sme.Estimator(W, H, search_range=16, subpel=2, max_iters=9)
    with pytest.raises(sme.SmeError):
        est.estimate_sequence(torch.from_numpy(luma).cuda(), torch.from_numpy(alpha).cuda(),
                              seed=torch.from_numpy(seed).cuda())
    est.close()
