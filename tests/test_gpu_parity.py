"""GPU parity: the CUDA path (through the C ABI) against the CPU oracle.

Integer results (classes, packed alpha, SADs, mismatch counts, vectors,
iteration and position counts, SSE, predictions) must be bit-exact.  The FP32
gradient updates are computed with the same operation order on both sides, so
they are compared exactly and also against the 1e-4 px gate.
"""
import numpy as np
import pytest

import oracle as O
from paper_1002_1168_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

DISP_TOL = 1e-4  # px, gate for the FP32 gradient updates


@pytest.fixture(scope="module")
def sme():
    from paper_1002_1168_gb300 import build as cuda_build
    from paper_1002_1168_gb300 import sme as m

    cuda_build.build()
    return m


def cuda(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


# "pair_staged": the pair schedule with every MB staged by TMA (transparent
# MBs included) instead of finishing transparent runs from global memory.
# "sparse3": the sparse schedule with its search kernel built for three CTAs
# per SM (the most registers cut); "sparse5": built for five 4-warp CTAs.
SCHEDULES = ["pair", "pair_staged", "mb", "cluster", "sparse", "sparse3", "sparse5"]


def set_schedule(sme, est, schedule, pair_warps=0):
    if schedule == "pair_staged":
        est.set_schedule("pair", pair_warps=pair_warps)
        est.set_option(sme.SME_OPT_PAIR_DIRECT, 0)
    elif schedule in ("sparse3", "sparse5"):
        est.set_schedule("sparse")
        est.set_option(sme.SME_OPT_MB_CTAS_PER_SM, int(schedule[-1]))
    else:
        est.set_schedule(schedule, pair_warps=pair_warps if schedule == "pair" else 0)


def run_both(sme, luma, alpha, S=16, h=1, K=8, theta=2.0, eps=1.0, rd=1, temporal=None, seed=None,
             want_pred=True, schedule="pair", pair_warps=0, tt=False):
    F, H, W = luma.shape
    est = sme.Estimator(W, H, search_range=S, subpel=h, theta=theta, epsilon=eps, max_iters=K,
                        ref_distance=rd, boundary_t_texture=tt)
    set_schedule(sme, est, schedule, pair_warps)
    want = ("cost", "disp", "iters", "npos", "mb_class", "sse_mb", "sse") + (("pred",) if want_pred else ())
    g = est.estimate_sequence(cuda(luma), cuda(alpha),
                              temporal_in=None if temporal is None else cuda(temporal.astype(np.int16)),
                              seed=None if seed is None else cuda(seed.astype(np.float32)), want=want)
    g = {k: v.cpu().numpy() for k, v in g.items()}
    est.close()
    p = O.OracleParams(W, H, S, h, theta, eps, K, boundary_t_texture=int(tt))
    o = O.estimate_sequence(p, luma, alpha, ref_distance=rd, temporal_in=temporal, seed=seed,
                            want_pred=want_pred)
    return g, o, p


def assert_parity(g, o, p, luma=None, rd=1):
    assert np.array_equal(g["mb_class"], o["mbclass"]), "MB classes"
    assert np.array_equal(g["mv"], o["mv"]), "motion vectors"
    assert np.array_equal(g["cost"].view(np.uint32), o["cost"]), "costs"
    assert np.array_equal(g["iters"], o["iters"]), "PRS iterations"
    assert np.array_equal(g["npos"], o["npos"]), "evaluated positions"
    assert np.abs(g["disp"] - o["disp"]).max(initial=0) <= DISP_TOL
    assert np.array_equal(g["disp"].view(np.uint32), o["disp"].view(np.uint32)), "FP32 updates (bitwise)"
    assert np.array_equal(g["sse"].view(np.uint64), o["sse"]), "SSE"
    if "pred" in g and o.get("pred") is not None:
        assert np.array_equal(g["pred"], o["pred"]), "prediction"
    if "sse_mb" in g and luma is not None and o.get("pred") is not None:
        P = o["mv"].shape[0]
        H, W = luma.shape[1:]
        for k in range(P):
            e = (luma[k + rd].astype(np.int64) - o["pred"][k]) ** 2
            per = e.reshape(H // 16, 16, W // 16, 16).sum(axis=(1, 3)).ravel()
            assert np.array_equal(g["sse_mb"][k].astype(np.int64), per)
    psnr_g = [O.psnr(int(s), p.width, p.height) for s in g["sse"].view(np.uint64)]
    assert np.allclose(psnr_g, o["psnr"], atol=1e-3, rtol=0)


# ------------------------------------------------------------ unit level --
@pytest.mark.parametrize("W,H,blobs", [(176, 144, True), (48, 32, False), (16, 16, False), (368, 48, True)])
def test_classify_and_pack(sme, W, H, blobs):
    _, alpha = synth.random_frames(W, H, 3, seed=W + H, alpha_blobs=blobs)
    alpha[0, :16, :16] = 0
    alpha[1] = 255
    est = sme.Estimator(W, H)
    cls, packed = est.classify(cuda(alpha))
    cls, packed = cls.cpu().numpy(), packed.cpu().numpy().view(np.uint32)
    for f in range(3):
        assert np.array_equal(cls[f], O.classify_frame(alpha[f]))
        bits = np.packbits(alpha[f] != 0, axis=1, bitorder="little")
        wp = packed.shape[2]
        padded = np.zeros((H, wp * 4), np.uint8)
        padded[:, :bits.shape[1]] = bits
        assert np.array_equal(packed[f], padded.view("<u4"))
    est.close()


def _all_queries(W, H, S, h, mbs, stride=1):
    q = []
    for m in mbs:
        u, v = m % (W // 16), m // (W // 16)
        lox, hix, loy, hiy = O.valid_range(W, H, 16, S, h, 16 * u, 16 * v)
        for dy in range(loy, hiy + 1, stride):
            for dx in range(lox, hix + 1, stride):
                q.append((m, dx, dy))
    return np.array(q, np.int32)


@pytest.mark.parametrize("h", [1, 2])
@pytest.mark.parametrize("S", [7, 16])
def test_costs_every_offset_of_edge_and_inner_mbs(sme, h, S):
    W, H = 64, 48
    luma, alpha = synth.random_frames(W, H, 2, seed=5 + S + h, alpha_blobs=True)
    M = (W // 16) * (H // 16)
    q = _all_queries(W, H, S, h, range(M))
    est = sme.Estimator(W, H, search_range=S, subpel=h)
    ts, ss = est.eval_costs(cuda(luma[0]), cuda(luma[1]), cuda(alpha[0]), cuda(alpha[1]), q)
    ts, ss = ts.cpu().numpy().view(np.uint32), ss.cpu().numpy().view(np.uint32)
    for i, (m, dx, dy) in enumerate(q):
        X0, Y0 = 16 * (m % 4), 16 * (m // 4)
        assert ts[i] == O.texture_sad(luma[0], luma[1], h, X0, Y0, dx, dy), (m, dx, dy)
        assert ss[i] == O.shape_sad(alpha[0], alpha[1], h, X0, Y0, dx, dy), (m, dx, dy)
    est.close()


@pytest.mark.parametrize("h", [1, 2])
def test_gradient_step_bitwise(sme, h):
    W, H = 96, 64
    seq = synth.make_sequence(W, H, 2, seed=77, noise_sigma=2.0, obj_frac=0.45)
    luma = seq.luma
    q = _all_queries(W, H, 4, h, range(24), stride=2)
    est = sme.Estimator(W, H, search_range=4, subpel=h, theta=2.0, epsilon=0.75)
    d = est.gradient_step(cuda(luma[0]), cuda(luma[1]), q).cpu().numpy()
    p = O.OracleParams(W, H, 4, h, 2.0, 0.75)
    want = np.array([O.gradient_step(p, luma[0], luma[1], 16 * (m % 6), 16 * (m // 6), dx, dy)
                     for m, dx, dy in q])
    assert np.abs(d - want).max() <= DISP_TOL
    assert np.array_equal(d.view(np.uint32), want.view(np.uint32))
    est.close()


# ------------------------------------------------------- whole sequences --
@pytest.mark.parametrize("schedule", SCHEDULES)
def test_qcif_pair_fullpel(sme, schedule):
    seq = synth.qcif_pair(seed=1001)
    g, o, p = run_both(sme, seq.luma, seq.alpha[0], S=16, h=1, schedule=schedule)
    assert_parity(g, o, p, seq.luma)


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_qcif_pairs_various_shifts(sme, seed):
    seq = synth.qcif_pair(seed=2000 + seed)
    g, o, p = run_both(sme, seq.luma, seq.alpha[0], S=16, h=1)
    assert_parity(g, o, p, seq.luma)


@pytest.mark.parametrize("schedule", SCHEDULES)
def test_cif_30_frames_halfpel_full_size(sme, schedule):
    """The CIF 352x288, 30-frame, half-pel workload the benchmark times,
    compared on every MB of every pair."""
    seq = synth.cif_sequence(seed=1002, frames=30)
    g, o, p = run_both(sme, seq.luma, seq.alpha[0], S=16, h=2, schedule=schedule)
    assert_parity(g, o, p, seq.luma)
    assert (o["mbclass"] == 1).sum() > 1000 and (o["mbclass"] == 2).sum() > 500


@pytest.mark.parametrize("schedule", SCHEDULES)
@pytest.mark.parametrize("S,h,K", [(7, 1, 8), (32, 2, 16), (64, 1, 3), (1, 2, 8), (16, 2, 0), (16, 1, 1)])
def test_parameters(sme, S, h, K, schedule):
    seq = synth.make_sequence(160, 96, 4, seed=31 + S + K, vmax=6.0, noise_sigma=2.0, obj_frac=0.4)
    g, o, p = run_both(sme, seq.luma, seq.alpha[0], S=S, h=h, K=K, schedule=schedule)
    assert_parity(g, o, p, seq.luma)


@pytest.mark.parametrize("theta,eps", [(3.0, 1.0), (0.5, 0.5), (2.0, 4.0)])
def test_theta_epsilon(sme, theta, eps):
    seq = synth.make_sequence(128, 128, 3, seed=8, vmax=5.0, noise_sigma=3.0, obj_frac=0.45)
    g, o, p = run_both(sme, seq.luma, seq.alpha[0], S=16, h=2, theta=theta, eps=eps)
    assert_parity(g, o, p, seq.luma)


@pytest.mark.parametrize("schedule", SCHEDULES)
def test_ref_distance_two_temporal_and_seed(sme, schedule):
    seq = synth.make_sequence(176, 144, 6, seed=12, vmax=4.0, obj_frac=0.4)
    rng = np.random.default_rng(0)
    M = 99
    temporal = rng.integers(-12, 13, (M, 2)).astype(np.int16)
    seed = rng.normal(0, 4, (4, M, 2)).astype(np.float32)
    seed[0, :5] = [1e6, -1e6]  # saturates
    g, o, p = run_both(sme, seq.luma, seq.alpha[0], S=16, h=2, rd=2, temporal=temporal, seed=seed,
                       schedule=schedule)
    assert_parity(g, o, p, seq.luma, rd=2)


@pytest.mark.parametrize("schedule", SCHEDULES)
@pytest.mark.parametrize("W,H,F", [(16, 16, 2), (16, 512, 3), (512, 16, 3), (48, 48, 5)])
def test_degenerate_sizes_random_content(sme, W, H, F, schedule):
    luma, alpha = synth.random_frames(W, H, F, seed=W * 7 + H, alpha_blobs=False, alpha_density=0.97)
    alpha[:, :, : W // 2] = 255
    g, o, p = run_both(sme, luma, alpha, S=8, h=2, schedule=schedule)
    assert_parity(g, o, p, luma)


@pytest.mark.parametrize("schedule", SCHEDULES)
@pytest.mark.parametrize("fill", [0, 255])
def test_all_transparent_or_all_opaque(sme, fill, schedule):
    seq = synth.make_sequence(96, 64, 3, seed=4)
    alpha = np.full_like(seq.alpha[0], fill)
    g, o, p = run_both(sme, seq.luma, alpha, S=16, h=2, schedule=schedule)
    assert_parity(g, o, p, seq.luma)
    if fill == 0:
        assert (g["mv"] == 0).all() and (g["npos"] == 0).all()


@pytest.mark.parametrize("schedule", ["pair", "pair_staged"])
@pytest.mark.parametrize("warps", [2, 3])
def test_pair_row_slots_with_transparent_rows_below(sme, schedule, warps):
    """Opaque MB rows over transparent ones, few warps per pair: a warp whose
    rows are transparent finishes them quickly and must not reuse a row slot
    (one per warp + 1) while a slower warp still reads the row it holds."""
    luma, _ = synth.translated_pair(256, 256, (3, 1), seed=11, noise_sigma=1.0)
    luma = np.concatenate([luma, np.roll(luma[1:], (1, 3), axis=(0, 1))])
    alpha = np.zeros_like(luma)
    alpha[:, :128] = 255
    g, o, p = run_both(sme, luma, alpha, S=8, h=2, schedule=schedule, pair_warps=warps)
    assert_parity(g, o, p, luma)
    assert (g["mv"][:, :64] != 0).any(axis=-1).mean() > 0.5  # the rows read below carry vectors


@pytest.mark.parametrize("schedule", SCHEDULES)
@pytest.mark.parametrize("h", [1, 2])
def test_boundary_temporal_by_texture_variant(sme, schedule, h):
    """Sec. 3.1 variant (boundary T judged by texture): bit-exact with the
    oracle's variant on a VOP sequence where it changes the field."""
    seq = synth.cif_sequence(frames=6)
    g, o, p = run_both(sme, seq.luma, seq.alpha[0], S=16, h=h, schedule=schedule, tt=True)
    assert_parity(g, o, p, seq.luma)
    o0 = O.estimate_sequence(O.OracleParams(352, 288, 16, h), seq.luma, seq.alpha[0])
    assert (o0["mv"] != o["mv"]).any()


@pytest.mark.parametrize("schedule", SCHEDULES)
def test_batch_shapes_each_sequence(sme, schedule):
    """Sequences of the uneven-size batch (one of each frame size, 4 frames)."""
    sizes = [(176, 144), (352, 288), (704, 576), (1920, 1088)]
    for seq in synth.batch_sequences(seed=1003, frames=4, sizes=sizes):
        for i in range(seq.alpha.shape[0]):
            g, o, p = run_both(sme, seq.luma, seq.alpha[i], S=16, h=2, want_pred=False, schedule=schedule)
            assert_parity(g, o, p)


@pytest.mark.parametrize("schedule", SCHEDULES)
def test_golden_propagation_on_gpu(sme, schedule):
    """The hand-derived candidate-propagation fixture, through the GPU."""
    from conftest import read_golden

    W, H = 96, 64
    luma, alpha = synth.translated_pair(W, H, (0, -2), seed=11)
    temporal = np.zeros((24, 2), np.int16)
    temporal[2] = (0, 2)
    g, o, p = run_both(sme, luma, alpha, S=16, h=1, K=0, temporal=temporal, schedule=schedule)
    want = read_golden("candidate_propagation.txt")["scenario C"]
    want = np.array([[tok.split(",") for tok in r] for r in want], int).reshape(-1, 2)
    assert np.array_equal(g["mv"][0].astype(int), want)
    assert_parity(g, o, p, luma)


# --------------------------------------------------------- other calls --
def test_pair_interface_matches_sequence(sme):
    seq = synth.make_sequence(176, 144, 4, seed=21, vmax=5.0, obj_frac=0.4)
    luma, alpha = cuda(seq.luma), cuda(seq.alpha[0])
    est = sme.Estimator(176, 144, search_range=16, subpel=2)
    full = est.estimate_sequence(luma, alpha)
    est.set_reference(luma[0], alpha[0])
    for k in range(3):
        est.set_current(luma[k + 1], alpha[k + 1])
        r = est.estimate(want=("cost", "sse"))
        ps = est.score()
        assert torch.equal(r["mv"][0], full["mv"][k])
        assert torch.equal(r["cost"][0], full["cost"][k])
        assert ps == pytest.approx(O.psnr(int(full["sse"][k]), 176, 144), abs=1e-9)
        est.advance()
        assert torch.equal(est.get_temporal_field(), full["mv"][k])
    est.close()


@pytest.mark.parametrize("schedule", ["mb", "sparse"])
def test_pair_interface_with_seed_field(sme, schedule):
    """Seeds through the pair interface (sme_set_seed_field): each pair
    equals the oracle's pair estimate with the previous field as T and the
    same seeds; clearing the seeds gives the unseeded result back."""
    seq = synth.make_sequence(176, 144, 4, seed=22, vmax=5.0, obj_frac=0.4)
    luma, alpha = cuda(seq.luma), cuda(seq.alpha[0])
    p = O.OracleParams(176, 144, 16, 2)
    est = sme.Estimator(176, 144, search_range=16, subpel=2)
    set_schedule(sme, est, schedule)
    rng = np.random.default_rng(5)
    est.set_reference(luma[0], alpha[0])
    prev = None
    for k in range(3):
        seed = rng.normal(0, 4, (p.mbs, 2)).astype(np.float32)
        est.set_seed_field(cuda(seed))
        est.set_current(luma[k + 1], alpha[k + 1])
        r = est.estimate(want=("cost", "iters", "npos", "sse"))
        o = O.estimate_pair(p, seq.luma[k], seq.luma[k + 1], seq.alpha[0][k], seq.alpha[0][k + 1],
                            temporal=prev, seed=seed)
        assert np.array_equal(r["mv"][0].cpu().numpy(), o["mv"])
        assert np.array_equal(r["cost"][0].cpu().numpy().view(np.uint32), o["cost"])
        assert np.array_equal(r["iters"][0].cpu().numpy(), o["iters"])
        assert np.array_equal(r["npos"][0].cpu().numpy(), o["npos"])
        prev = o["mv"]
        est.advance()
    est.set_seed_field(None)
    est.set_current(luma[1], alpha[1])
    est.set_temporal_field(None)
    est.set_reference(luma[0], alpha[0])
    r = est.estimate(want=("cost",))
    o = O.estimate_pair(p, seq.luma[0], seq.luma[1], seq.alpha[0][0], seq.alpha[0][1])
    assert np.array_equal(r["mv"][0].cpu().numpy(), o["mv"])
    est.close()
    est = sme.Estimator(176, 144, search_range=16, subpel=2, max_iters=9)
    with pytest.raises(sme.SmeError):
        est.set_seed_field(cuda(np.zeros((p.mbs, 2), np.float32)))
    est.close()


@pytest.mark.parametrize("h", [1, 2])
def test_compensate_given_field(sme, h):
    W, H = 128, 96
    luma, _ = synth.random_frames(W, H, 2, seed=h)
    p = O.OracleParams(W, H, 16, h)
    rng = np.random.default_rng(h)
    mv = np.zeros((p.mbs, 2), np.int16)
    for m in range(p.mbs):
        lox, hix, loy, hiy = O.valid_range(W, H, 16, 16, h, 16 * (m % 8), 16 * (m // 8))
        mv[m] = (rng.integers(lox, hix + 1), rng.integers(loy, hiy + 1))
    est = sme.Estimator(W, H, search_range=16, subpel=h)
    sse, pred = est.compensate(cuda(luma[0]), cuda(luma[1]), cuda(mv))
    osse, opred = O.compensate(p, luma[0], luma[1], mv, want_pred=True)
    assert sse == osse and np.array_equal(pred.cpu().numpy(), opred)
    bad = mv.copy()
    bad[0] = (-1, 0)
    from paper_1002_1168_gb300.sme import SmeError

    with pytest.raises(SmeError) as e:
        est.compensate(cuda(luma[0]), cuda(luma[1]), cuda(bad))
    assert e.value.status == 7
    est.compensate(cuda(luma[0]), cuda(luma[1]), cuda(mv))  # context still usable
    est.close()


@pytest.mark.parametrize("pin_in,pin_out", [(True, False), (False, False), (True, True), (False, True)])
def test_host_buffers_match_device(sme, pin_in, pin_out):
    """Pinned inputs are read in place (alpha) or copied on a second stream
    (luma), pinned outputs written in place; pageable ones are staged.  Every
    combination gives the device results, twice in a row on one context."""
    seq = synth.cif_sequence(seed=1002, frames=6)
    est = sme.Estimator(352, 288, search_range=16, subpel=2)
    want = ("cost", "disp", "iters", "npos", "mb_class", "sse_mb", "sse", "pred")
    dev = est.estimate_sequence(cuda(seq.luma), cuda(seq.alpha[0]), want=want)
    hl, ha = torch.from_numpy(seq.luma), torch.from_numpy(seq.alpha[0])
    if pin_in:
        hl, ha = hl.pin_memory(), ha.pin_memory()
    out = est._alloc_outputs(5, want, "cpu")
    if pin_out:
        out = {k: v.pin_memory() for k, v in out.items()}
    for _ in range(2):
        for v in out.values():
            v.fill_(7)
        host = est.estimate_sequence_host(hl, ha, want=want, out=out)
        for k in ("mv",) + want:
            assert torch.equal(host[k], dev[k].cpu()), k
    est.close()


def test_repeated_runs_identical(sme):
    seq = synth.cif_sequence(seed=1002, frames=8)
    est = sme.Estimator(352, 288, search_range=16, subpel=2)
    luma, alpha = cuda(seq.luma), cuda(seq.alpha[0])
    first = est.estimate_sequence(luma, alpha)
    for _ in range(20):
        again = est.estimate_sequence(luma, alpha, sync=False)
    est.synchronize()
    for k in first:
        assert torch.equal(first[k], again[k]), k
    est.close()


@pytest.mark.parametrize("schedule", SCHEDULES)
def test_bounded_wait_reports_timeout_and_context_recovers(sme, schedule):
    """A result that is never published: dependants give up after a short
    limit, the launch ends, the host reads SME_ERR_TIMEOUT, and the next
    estimate on the same context is correct."""
    from paper_1002_1168_gb300.sme import SmeError

    W, H = 64, 64
    luma, alpha = synth.translated_pair(W, H, (1, 0), seed=3)
    luma = np.concatenate([luma, luma[:1]])
    alpha = np.concatenate([alpha, alpha[:1]])
    est = sme.Estimator(W, H, search_range=8, subpel=1)
    set_schedule(sme, est, schedule)
    # MB 0 of pair 0 is A of MB 1 and B of MB 4 (per-MB schedule) and T of
    # MB 0 of pair 1 (both schedules)
    est.debug_set_fault(skip_ticket=0, timeout_ns=20_000_000)
    with pytest.raises(SmeError) as e:
        est.estimate_sequence(cuda(luma), cuda(alpha))
    assert e.value.status == 4
    est.debug_set_fault(-1, 0)
    g = est.estimate_sequence(cuda(luma), cuda(alpha))
    o = O.estimate_sequence(O.OracleParams(W, H, 8, 1), luma, alpha)
    assert np.array_equal(g["mv"].cpu().numpy(), o["mv"])
    est.close()


def test_argument_errors(sme):
    import ctypes as C

    from paper_1002_1168_gb300.sme import _lib

    est = sme.Estimator(64, 64)
    lib = _lib()
    luma = torch.zeros((2, 64, 64), dtype=torch.uint8, device="cuda")
    out = sme.Outputs()
    assert lib.sme_estimate_sequence(est._h, C.c_void_p(luma.data_ptr()), C.c_void_p(luma.data_ptr()), 2,
                                     None, None, C.byref(out)) == 1  # no mv output
    out.mv = C.c_void_p(torch.empty((1, 16, 2), dtype=torch.int16, device="cuda").data_ptr())
    assert lib.sme_estimate_sequence(est._h, C.c_void_p(luma.data_ptr() + 1), C.c_void_p(luma.data_ptr()), 2,
                                     None, None, C.byref(out)) == 1  # misaligned
    assert lib.sme_estimate_sequence(est._h, C.c_void_p(luma.data_ptr()), C.c_void_p(luma.data_ptr()), 1,
                                     None, None, C.byref(out)) == 1  # no pair
    assert lib.sme_estimate(est._h, None) == 5  # no frames set
    est.close()


@pytest.mark.parametrize("schedule", SCHEDULES)
def test_learned_seed_fallback_paths(sme, schedule):
    """Seeds near the plain result (noisy): they win the candidate comparison
    on some MBs, so both pixel-recursive searches and the fallback run."""
    seq = synth.cif_sequence(seed=1002, frames=8)
    p = O.OracleParams(352, 288, 16, 2)
    plain = O.estimate_sequence(p, seq.luma, seq.alpha[0])
    rng = np.random.default_rng(1)
    seed = (plain["mv"].astype(np.float32) / 2 + rng.normal(0, 1.0, plain["mv"].shape)).astype(np.float32)
    g, o, p = run_both(sme, seq.luma, seq.alpha[0], S=16, h=2, seed=seed, schedule=schedule)
    assert_parity(g, o, p, seq.luma)
    assert (o["mv"] != plain["mv"]).any(axis=-1).sum() > 0  # the seeds changed some results
