"""GPU four-vector mode (Sec. 3.2: the recursive search on 8x8 blocks, four
vectors per MB) against the oracle's: block vectors, costs, PRS steps,
positions, classes and per-pair SSE bit-exact, the FP32 block updates
bitwise; prediction images equal; through the device and host-buffer entry
points, full- and half-pel, edge MBs, a temporal field, the degenerate
alpha planes."""
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


def cuda(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


WANT = ("cost", "disp", "iters", "npos", "mb_class", "sse_mb", "sse", "pred")


SCHEDULES = ["mb", "pair"]  # the per-MB schedule (default) and the per-pair one


def run_both(sme, luma, alpha, S=16, h=2, K=8, rd=1, temporal4=None, warps=0, host=False, schedule="mb"):
    F, H, W = luma.shape
    est = sme.Estimator(W, H, search_range=S, subpel=h, max_iters=K, ref_distance=rd, four_mv=True)
    est.set_schedule(schedule, pair_warps=warps if schedule == "pair" else 0)
    tmp = None if temporal4 is None else temporal4.astype(np.int16)
    if host:
        g = est.estimate_sequence_host(torch.from_numpy(luma), torch.from_numpy(alpha),
                                       temporal_in=None if tmp is None else torch.from_numpy(tmp), want=WANT)
    else:
        g = est.estimate_sequence(cuda(luma), cuda(alpha), temporal_in=None if tmp is None else cuda(tmp), want=WANT)
    g = {k: v.cpu().numpy() for k, v in g.items()}
    est.close()
    o = O.estimate_sequence4(O.OracleParams(W, H, S, h, max_iters=K), luma, alpha, ref_distance=rd,
                             temporal_in4=temporal4, want_pred=True)
    return g, o


def assert_parity(g, o, luma, rd=1):
    assert np.array_equal(g["mb_class"], o["mbclass"]), "MB classes"
    assert np.array_equal(g["mv"], o["mv"]), "block vectors"
    assert np.array_equal(g["cost"].view(np.uint32), o["cost"]), "block costs"
    assert np.array_equal(g["iters"], o["iters"]), "block PRS steps"
    assert np.array_equal(g["npos"], o["npos"]), "block positions"
    assert np.array_equal(g["disp"].view(np.uint32), o["disp"].view(np.uint32)), "FP32 block updates (bitwise)"
    assert np.array_equal(g["sse"].view(np.uint64), o["sse"]), "SSE"
    assert np.array_equal(g["pred"], o["pred"]), "prediction"
    H, W = luma.shape[1:]
    for k in range(o["mv"].shape[0]):
        e = (luma[k + rd].astype(np.int64) - o["pred"][k]) ** 2
        per = e.reshape(H // 16, 16, W // 16, 16).sum(axis=(1, 3)).ravel()
        assert np.array_equal(g["sse_mb"][k].view(np.uint32).astype(np.int64), per), "per-MB SSE"


@pytest.mark.parametrize("schedule", SCHEDULES)
@pytest.mark.parametrize("h", [1, 2])
def test_qcif_pair(sme, h, schedule):
    seq = synth.qcif_pair()
    g, o = run_both(sme, seq.luma, seq.alpha, S=16, h=h, schedule=schedule)
    assert_parity(g, o, seq.luma)
    assert (o["mv"][..., 0, :] != o["mv"][..., 3, :]).any()  # blocks do differ


@pytest.mark.parametrize("schedule,warps", [("mb", 0), ("pair", 0), ("pair", 2), ("pair", 5)])
def test_cif_sequence_halfpel(sme, schedule, warps):
    seq = synth.cif_sequence(frames=6)
    g, o = run_both(sme, seq.luma, seq.alpha[0], S=16, h=2, warps=warps, schedule=schedule)
    assert_parity(g, o, seq.luma)


@pytest.mark.parametrize("schedule", SCHEDULES)
def test_host_buffers(sme, schedule):
    seq = synth.cif_sequence(frames=3)
    g, o = run_both(sme, seq.luma, seq.alpha[0], S=16, h=2, host=True, schedule=schedule)
    assert_parity(g, o, seq.luma)


@pytest.mark.parametrize("schedule", SCHEDULES)
def test_temporal_field_and_ref_distance_two(sme, schedule):
    seq = synth.cif_sequence(frames=5)
    rng = np.random.default_rng(3)
    tmp = rng.integers(-12, 13, (396, 4, 2))
    g, o = run_both(sme, seq.luma, seq.alpha[0], S=8, h=2, rd=2, temporal4=tmp, schedule=schedule)
    assert_parity(g, o, seq.luma, rd=2)


@pytest.mark.parametrize("schedule", SCHEDULES)
@pytest.mark.parametrize("W,H,F,S,h,K", [(48, 48, 3, 4, 2, 8), (64, 32, 4, 7, 1, 16), (96, 64, 3, 32, 2, 3)])
def test_edges_and_parameters_random_content(sme, W, H, F, S, h, K, schedule):
    luma, alpha = synth.random_frames(W, H, F, seed=W * H + S)
    g, o = run_both(sme, luma, alpha, S=S, h=h, K=K, schedule=schedule)
    assert_parity(g, o, luma)


@pytest.mark.parametrize("schedule", SCHEDULES)
@pytest.mark.parametrize("fill", [0, 255])
def test_all_transparent_or_all_opaque(sme, fill, schedule):
    seq = synth.cif_sequence(frames=3)
    alpha = np.full_like(seq.alpha[0], fill)
    g, o = run_both(sme, seq.luma, alpha, S=16, h=2, schedule=schedule)
    assert_parity(g, o, seq.luma)
    if fill == 0:
        assert not g["mv"].any() and not g["npos"].any()


def test_boundary_texture_variant_is_rejected(sme):
    from paper_1002_1168_gb300.sme import SmeError

    seq = synth.cif_sequence(frames=2)
    est = sme.Estimator(352, 288, search_range=16, subpel=2, four_mv=True, boundary_t_texture=True)
    with pytest.raises(SmeError):
        est.estimate_sequence(cuda(seq.luma), cuda(seq.alpha[0]))
    est.close()


def test_seeds_are_rejected(sme):
    from paper_1002_1168_gb300.sme import SmeError

    seq = synth.cif_sequence(frames=2)
    est = sme.Estimator(352, 288, search_range=16, subpel=2, four_mv=True)
    with pytest.raises(SmeError):
        est.estimate_sequence(cuda(seq.luma), cuda(seq.alpha[0]),
                              seed=cuda(np.zeros((1, 396, 2), np.float32)))
    est.close()


@pytest.mark.parametrize("schedule", SCHEDULES)
def test_bounded_wait_reports_timeout_and_context_recovers(sme, schedule):
    """One MB's ready words are never published: its consumers give up after
    a short limit, the host reads SME_ERR_TIMEOUT, and the next estimate on
    the same context is correct."""
    from paper_1002_1168_gb300.sme import SmeError

    luma, alpha = synth.translated_pair(64, 64, (1, 0), seed=3)
    luma = np.concatenate([luma, luma[:1]])
    alpha = np.concatenate([alpha, alpha[:1]])
    est = sme.Estimator(64, 64, search_range=8, subpel=1, four_mv=True)
    est.set_schedule(schedule)
    est.debug_set_fault(skip_ticket=0, timeout_ns=20_000_000)
    with pytest.raises(SmeError) as e:
        est.estimate_sequence(cuda(luma), cuda(alpha))
    assert e.value.status == 4
    est.debug_set_fault(-1, 0)
    g = est.estimate_sequence(cuda(luma), cuda(alpha))
    o = O.estimate_sequence4(O.OracleParams(64, 64, 8, 1), luma, alpha)
    assert np.array_equal(g["mv"].cpu().numpy(), o["mv"])
    est.close()


@pytest.mark.parametrize("schedule,param,flag", [("mb", 0, 1), ("pair", 8, 0), ("pair", 4, 0)])
def test_four_mv_batch_matches_oracle(sme, schedule, param, flag):
    """Four vectors per MB in a batch of uneven sequences (sme_batch_set_option):
    every VOP's block fields equal the oracle's, in both schedules of the
    mode, twice in a row; tuning keeps them; the sparse schedule, seeds and
    pair rounds are refused in this mode."""
    sizes = [(176, 144, 4), (352, 288, 3), (96, 64, 3)]
    seqs = []
    for i, (W, H, F) in enumerate(sizes):
        s = synth.make_sequence(W, H, F, seed=600 + i, n_objects=1 + i % 2, vmax=6.0, obj_frac=0.35)
        seqs += [(s.luma, s.alpha[j]) for j in range(s.alpha.shape[0])]
    b = sme.Batch([cuda(l) for l, _ in seqs], [cuda(a) for _, a in seqs], search_range=16, subpel=2,
                  want=WANT, four_mv=True)
    b.set_config(schedule, param, flag)
    for _ in range(2):
        outs = b.run()
        for (luma, alpha), g in zip(seqs, outs):
            F, H, W = luma.shape
            o = O.estimate_sequence4(O.OracleParams(W, H, 16, 2), luma, alpha, want_pred=True)
            g = {k: v.cpu().numpy() for k, v in g.items()}
            assert_parity(g, o, luma)
    with pytest.raises(sme.SmeError):
        b.set_config("sparse", 2, 0)
    with pytest.raises(sme.SmeError):
        b.set_pair_rounds(True)
    b.tune(trials=1)
    assert b.config()["schedule"] in ("mb", "pair")
    outs = b.run()
    for (luma, alpha), g in zip(seqs, outs):
        F, H, W = luma.shape
        o = O.estimate_sequence4(O.OracleParams(W, H, 16, 2), luma, alpha)
        assert np.array_equal(g["mv"].cpu().numpy(), o["mv"])
    b.close()
    seeds = [torch.zeros((l.shape[0] - 1, (l.shape[2] // 16) * (l.shape[1] // 16), 2), device="cuda") for l, _ in seqs]
    with pytest.raises(sme.SmeError):
        sme.Batch([cuda(l) for l, _ in seqs], [cuda(a) for _, a in seqs], search_range=16, subpel=2,
                  seed_list=seeds, four_mv=True)
