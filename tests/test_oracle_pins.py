"""Pins of the CPU oracle against facts fixed by the paper and by mathematics.

Nothing here compares the oracle with itself: each test checks a closed form,
a value printed in the paper (Table 1), a hand-derived golden fixture, a
textbook definition (MPEG-4 half-sample interpolation), an exhaustive search,
or an invariant of the method (Fig. 1: transparent MBs carry no vector).
"""
import math

import numpy as np
import pytest

import oracle as O
from paper_1002_1168_gb300 import synth
from conftest import read_golden


# ---------------------------------------------------------------- Table 1 --
def test_table1_es_count_pins_valid_set():
    """Table 1, ES row: 204.2828 search points per block (QCIF, window 7)."""
    for row in read_golden("table1_es.txt")[None]:
        W, H, B, S, h, total, blocks = map(int, row[:7])
        mean = float(row[7])
        _, _, got = O.full_search(None, None, W, H, h, S, B)
        assert got == total
        assert (W // B) * (H // B) == blocks
        assert round(got / blocks, 4) == mean
    # the paper's value itself
    _, _, got = O.full_search(None, None, 176, 144, 1, 7, 8)
    assert abs(got / 396 - 204.2828) < 5e-5


def test_valid_set_edges():
    # interior block: the full +-S*h window
    assert O.valid_range(176, 144, 16, 16, 2, 64, 64) == (-32, 32, -32, 32)
    # top-left block: no negative offsets; bottom-right: no positive ones
    assert O.valid_range(176, 144, 16, 16, 1, 0, 0) == (0, 16, 0, 16)
    assert O.valid_range(176, 144, 16, 16, 2, 160, 128) == (-32, 0, -32, 0)


# ------------------------------------------------- half-sample interpolation --
def test_halfpel_mpeg4_rounding_control_zero():
    """MPEG-4 bilinear interpolation, rounding control 0: (a+b+1)>>1 on one
    axis and (a+b+c+d+2)>>2 on the diagonal (not an average of averages)."""
    ref = np.zeros((16, 16), np.uint8)
    ref[0, 0], ref[0, 1], ref[1, 0], ref[1, 1] = 0, 1, 0, 0
    assert O.interp(ref, 2, 1, 1) == 0          # (0+1+0+0+2)>>2 = 0; avg-of-avg gives 1
    ref[0, 0], ref[0, 1] = 1, 2
    assert O.interp(ref, 2, 1, 0) == 2          # (1+2+1)>>1: halves round up
    ref[1, 0] = 4
    assert O.interp(ref, 2, 0, 1) == 3          # (1+4+1)>>1
    assert O.interp(ref, 2, 0, 0) == 1 and O.interp(ref, 1, 1, 1) == 0
    ref[:2, :2] = [[0, 0], [0, 2]]
    assert O.interp(ref, 2, 1, 1) == 1          # (0+0+0+2+2)>>2 = 1: the rounding constant is 2
    ref[:2, :2] = [[0, 3], [0, 0]]
    assert O.interp(ref, 2, 1, 0) == 2 and O.interp(ref, 2, 0, 1) == 0   # (0+3+1)>>1, (0+0+1)>>1


def test_halfpel_on_ramp_closed_form():
    # f(x, y) = 4x + 8y: half-sample values are exact midpoints
    Y, X = np.mgrid[0:16, 0:16]
    ref = (4 * X + 8 * Y).astype(np.uint8) // 1
    ref = np.clip(4 * X + 8 * Y, 0, 255).astype(np.uint8)
    for x in range(0, 10):
        for y in range(0, 10):
            f = 4 * x + 8 * y
            assert O.interp(ref, 2, 2 * x + 1, 2 * y) == f + 2
            assert O.interp(ref, 2, 2 * x, 2 * y + 1) == f + 4
            assert O.interp(ref, 2, 2 * x + 1, 2 * y + 1) == f + 6
    flat = np.full((16, 16), 77, np.uint8)
    assert {O.interp(flat, 2, a, b) for a in range(20) for b in range(20)} == {77}


# ------------------------------------------------------------- texture SAD --
def test_texture_sad_identities_and_brute_force():
    rng = np.random.default_rng(3)
    ref = rng.integers(0, 256, (48, 64), dtype=np.uint8)
    assert O.texture_sad(ref, ref, 1, 16, 16, 0, 0) == 0
    cur = ref.astype(np.int32) + 5
    ok = cur <= 255
    cur = np.clip(cur, 0, 255).astype(np.uint8)
    blk_ok = ok[16:32, 16:32].all()
    if blk_ok:
        assert O.texture_sad(ref, cur, 1, 16, 16, 0, 0) == 256 * 5
    cur = rng.integers(0, 256, (48, 64), dtype=np.uint8)
    # brute force over every full-pel offset of one block
    for dy in range(-16, 17):
        for dx in range(-16, 33):
            if not (0 <= 16 + dx <= 48 and 0 <= 16 + dy <= 32):
                continue
            want = np.abs(ref[16 + dy:32 + dy, 16 + dx:32 + dx].astype(int)
                          - cur[16:32, 16:32].astype(int)).sum()
            assert O.texture_sad(ref, cur, 1, 16, 16, dx, dy) == want


# --------------------------------------------------------------- shape SAD --
def test_shape_sad_half_planes_and_truncation():
    W, H = 64, 48
    X = np.arange(W)[None, :].repeat(H, 0)
    acur = np.where(X < 40, 255, 0).astype(np.uint8)
    aref = np.where(X < 39, 255, 0).astype(np.uint8)
    # the edge of the MB at X0=32 moved one column: 16 rows x 1 column
    assert O.shape_sad(aref, acur, 1, 32, 16, 0, 0) == 16
    assert O.shape_sad(aref, acur, 1, 32, 16, -1, 0) == 0
    assert O.shape_sad(aref, acur, 1, 32, 16, -3, 0) == 32
    # half-pel vectors use the full-pel part trunc(d/h) (toward zero)
    assert O.shape_sad(aref, acur, 2, 32, 16, -2, 0) == 0
    assert O.shape_sad(aref, acur, 2, 32, 16, -3, 0) == 0     # trunc(-1.5) = -1
    assert O.shape_sad(aref, acur, 2, 32, 16, -4, 0) == 16    # -2
    assert O.shape_sad(aref, acur, 2, 32, 16, 1, 0) == 16     # trunc(0.5) = 0
    # identical masks, any vector keeping the edge outside the block
    assert O.shape_sad(acur, acur, 1, 0, 0, 5, 7) == 0


def test_classification_closed_forms():
    a = np.zeros((32, 48), np.uint8)
    a[0:16, 16:32] = 255          # MB(1,0) fully inside
    a[20, 40] = 1                 # MB(2,1): one pixel inside (any nonzero counts)
    a[16:32, 0:16] = 255
    a[31, 15] = 0                 # MB(0,1): 255 of 256 inside
    assert list(O.classify_frame(a)) == [0, 1, 0, 2, 0, 2]


# ----------------------------------------------------------- gradient step --
def _ramp_pair(a, s, axis):
    """cur = a*x + 32 (or y); ref = a*(x - s) + 32: cur(p) = ref(p + s)."""
    Y, X = np.mgrid[0:48, 0:48]
    c = X if axis == 0 else Y
    cur = np.clip(a * c + 32, 0, 255).astype(np.uint8)
    ref = np.clip(a * (c - s) + 32, 0, 255).astype(np.uint8)
    return ref, cur


@pytest.mark.parametrize("axis", [0, 1])
@pytest.mark.parametrize("h", [1, 2])
def test_gradient_step_recovers_ramp_shift(axis, h):
    """Eqs. 3-5 on a linear ramp: the inverse-gradient update equals the
    residual displacement exactly (u = 2/g with g = 2a; DPD = a (d - s))."""
    for a in (2, 4):
        for s in (-3, -1, 2, 3):
            ref, cur = _ramp_pair(a, s, axis)
            p = O.OracleParams(48, 48, 16, h)
            for d in range(-3 * h, 3 * h + 1):
                dv = (d, 0) if axis == 0 else (0, d)
                out = O.gradient_step(p, ref, cur, 16, 16, *dv)
                assert out[axis] == pytest.approx(s - d / h, abs=0)
                assert out[1 - axis] == 0.0


@pytest.mark.parametrize("axis", [0, 1])
def test_gradient_step_mean_is_over_pixels_with_a_gradient(axis):
    """Eq. 3's block update is the mean over the pixels whose u is defined
    (u != 0): in the corner MB the first row/column has no central
    difference (Eq. 5), so only 240 pixels count, and the update still equals
    the residual displacement exactly."""
    for h in (1, 2):
        ref, cur = _ramp_pair(2, 2, axis)
        p = O.OracleParams(48, 48, 16, h)
        for d in (0, h, 3 * h):
            dv = (d, 0) if axis == 0 else (0, d)
            out = O.gradient_step(p, ref, cur, 0, 0, *dv)
            assert out[axis] == pytest.approx(2 - d / h, abs=0)


def test_gradient_step_sum_is_the_pairwise_tree():
    """The FP32 sum of Eq. 3's terms is the contiguous pairwise tree (reading
    c9).  With u = 2/6 (not a binary fraction) and irregular DPD the tree
    and a running sum round differently; the oracle must give the tree."""
    X = np.mgrid[0:48, 0:48][1]
    cur = (3 * X + 40).astype(np.uint8)                    # g = 6 everywhere inside: u = 2/6
    rng = np.random.default_rng(1234)
    e = rng.integers(-40, 41, (48, 48))
    ref = (cur.astype(int) + e).astype(np.uint8)
    p = O.OracleParams(48, 48, 16, 1)
    u = np.float32(2.0) / np.float32(6.0)
    t = e[16:32, 16:32].astype(np.float32).ravel() * u       # DPD(0, p) * u, FP32
    tree = t.copy()
    while tree.size > 1:
        tree = tree[0::2] + tree[1::2]
    seq = np.float32(0.0)
    for v in t:
        seq = np.float32(seq + v)
    assert tree[0] != seq                                  # the construction discriminates
    want = -(np.float32(1.0) * (tree[0] / np.float32(256.0)))
    out = O.gradient_step(p, ref, cur, 16, 16, 0, 0)
    assert np.float32(out[0]) == want and out[1] == 0.0


def test_gradient_step_theta_and_epsilon():
    # a = 1: |df/dx| = 1 < Theta = 2 -> u = 0 everywhere -> no update
    ref, cur = _ramp_pair(1, 2, 0)
    p = O.OracleParams(48, 48, 16, 1)
    assert list(O.gradient_step(p, ref, cur, 16, 16, 0, 0)) == [0.0, 0.0]
    # Theta = 1 admits it: update = s - d
    p1 = O.OracleParams(48, 48, 16, 1, theta=1.0)
    assert O.gradient_step(p1, ref, cur, 16, 16, 0, 0)[0] == 2.0
    # the convergence factor scales the update (Eq. 2)
    ref, cur = _ramp_pair(4, 3, 0)
    p2 = O.OracleParams(48, 48, 16, 1, epsilon=0.5)
    assert O.gradient_step(p2, ref, cur, 16, 16, -1, 0)[0] == 2.0


# ----------------------------------------------------------------- PSNR / MC --
def test_psnr_closed_form():
    W, H = 64, 32
    for c in (1, 3, 17):
        assert O.psnr(c * c * W * H, W, H) == pytest.approx(20 * math.log10(255 / c), abs=1e-12)
    assert O.psnr(0, W, H) == math.inf


def test_compensate_zero_and_integer_field():
    rng = np.random.default_rng(5)
    W, H = 64, 48
    ref = rng.integers(0, 256, (H, W), dtype=np.uint8)
    cur = rng.integers(0, 256, (H, W), dtype=np.uint8)
    p = O.OracleParams(W, H, 16, 1)
    sse, pred = O.compensate(p, ref, cur, np.zeros((p.mbs, 2)), want_pred=True)
    assert np.array_equal(pred, ref)
    assert sse == int(((cur.astype(np.int64) - ref) ** 2).sum())
    # a constant field (2, 1) on the middle MB only
    mv = np.zeros((p.mbs, 2), np.int16)
    mv[4 + 1] = (2, 1)                 # MB (1, 1)
    _, pred = O.compensate(p, ref, cur, mv, want_pred=True)
    assert np.array_equal(pred[16:32, 16:32], ref[17:33, 18:34])
    # half-pel on a ramp: exact midpoint
    Y, X = np.mgrid[0:H, 0:W]
    ramp = (2 * X + 2 * Y).astype(np.uint8)
    p2 = O.OracleParams(W, H, 16, 2)
    mv2 = np.zeros((p2.mbs, 2), np.int16)
    mv2[5] = (1, 0)
    _, pred2 = O.compensate(p2, ramp, ramp, mv2, want_pred=True)
    assert np.array_equal(pred2[16:32, 16:32].astype(int), ramp[16:32, 16:32].astype(int) + 1)
    bad = np.zeros((p.mbs, 2), np.int16)
    bad[0] = (-1, 0)                    # outside V at the left edge
    with pytest.raises(ValueError):
        O.compensate(p, ref, cur, bad)


# --------------------------------------------------- whole method on one pair --
def _prop_case(scenario):
    W, H = 96, 64
    luma, alpha = synth.translated_pair(W, H, (0, -2), seed=11)
    temporal = np.zeros((24, 2), np.int16)
    if scenario == "C":
        temporal[2] = (0, 2)
    else:
        temporal[0] = (0, 2)
        alpha = alpha.copy()
        alpha[1, 0:16, 16:32] = 0
    p = O.OracleParams(W, H, 16, 1, max_iters=0)
    return p, luma, alpha, temporal


@pytest.mark.parametrize("scenario", ["C", "B"])
def test_candidate_propagation_golden(scenario):
    """Fig. 1 / Fig. 3 neighbour candidates and raster order (hand-derived)."""
    p, luma, alpha, temporal = _prop_case(scenario)
    o = O.estimate_pair(p, luma[0], luma[1], alpha[0], alpha[1], temporal=temporal)
    rows = read_golden("candidate_propagation.txt")[f"scenario {scenario}"]
    want = np.array([[tok.split(",") for tok in r] for r in rows], int).reshape(-1, 2)
    assert np.array_equal(o["mv"].astype(int), want)
    assert (o["iters"] == 0).all()


def test_flat_frame_tiebreak_and_position_count_golden():
    W = H = 64
    luma = np.full((2, H, W), 128, np.uint8)
    alpha = np.full((2, H, W), 255, np.uint8)
    temporal = np.tile(np.array([3, 1], np.int16), (16, 1))
    p = O.OracleParams(W, H, 4, 1, max_iters=8)
    o = O.estimate_pair(p, luma[0], luma[1], alpha[0], alpha[1], temporal=temporal)
    g = read_golden("flat_tiebreak.txt")
    want_mv = np.array([[t.split(",") for t in r] for r in g["mv"]], int).reshape(-1, 2)
    assert np.array_equal(o["mv"].astype(int), want_mv)
    assert np.array_equal(o["iters"].astype(int), np.array(g["iters"], int).ravel())
    assert np.array_equal(o["npos"].astype(int), np.array(g["npos"], int).ravel())
    assert (o["disp"] == 0).all() and (o["cost"] == 0).all()


@pytest.mark.parametrize("h", [1, 2])
def test_known_translation_recovery(h):
    """Noise-free low-frequency texture moved by an integer vector v: the
    exhaustive search finds SAD 0 at d = -v, and the method (started from
    zero candidates) reaches it on nearly every MB whose window contains it."""
    hit = tot = 0
    for seed in range(8):
        rng = np.random.default_rng(100 + seed)
        sh = rng.integers(-3, 4, 2)
        luma, alpha = synth.translated_pair(128, 96, sh, seed=seed)
        p = O.OracleParams(128, 96, 16, h)
        o = O.estimate_pair(p, luma[0], luma[1], alpha[0], alpha[1])
        _, bs, _ = O.full_search(luma[0], luma[1], 128, 96, h, 16)
        tgt = -sh * h
        for m in range(p.mbs):
            lox, hix, loy, hiy = O.valid_range(128, 96, 16, 16, h, 16 * (m % 8), 16 * (m // 8))
            if not (lox <= tgt[0] <= hix and loy <= tgt[1] <= hiy):
                continue
            tot += 1
            assert bs[m] == 0
            hit += bool((o["mv"][m] == tgt).all() and o["cost"][m] == 0)
            if h == 1 and o["cost"][m] == 0:
                assert (o["mv"][m] == tgt).all()
    assert hit >= 0.97 * tot


def test_invariants_on_cif_sequence():
    """Fig. 1 invariants on the CIF workload (first 6 frames): transparent MBs
    carry no vector; the method never beats the exhaustive search; a result
    below the iteration cap is a minimum over its eight clamped neighbours;
    positions per MB stay within the algorithm's bound."""
    seq = synth.cif_sequence(frames=6)
    p = O.OracleParams(352, 288, 16, 2)
    o = O.estimate_sequence(p, seq.luma, seq.alpha[0])
    cls = o["mbclass"]
    t = cls == 0
    assert (o["mv"][t] == 0).all() and (o["cost"][t] == 0).all()
    assert (o["iters"][t] == 0).all() and (o["npos"][t] == 0).all()
    assert (o["iters"][cls == 2] == 0).all()
    assert o["npos"][cls > 0].min() >= 1 and o["npos"].max() <= 4 + 9 * p.max_iters
    for k in (0, 3):
        ref, cur = seq.luma[k], seq.luma[k + 1]
        _, bs, _ = O.full_search(ref, cur, 352, 288, 2, 16)
        op = np.nonzero(cls[k] == 1)[0]
        assert (o["cost"][k][op] >= bs[op]).all()
        for m in op:
            if o["iters"][k][m] >= p.max_iters:
                continue
            X0, Y0 = 16 * (m % 22), 16 * (m // 22)
            lox, hix, loy, hiy = O.valid_range(352, 288, 16, 16, 2, X0, Y0)
            dx, dy = map(int, o["mv"][k][m])
            for j in (-1, 0, 1):
                for i in (-1, 0, 1):
                    nx, ny = min(max(dx + i, lox), hix), min(max(dy + j, loy), hiy)
                    assert O.texture_sad(ref, cur, 2, X0, Y0, nx, ny) >= o["cost"][k][m]
    # SSE matches the compensation of the returned field
    for k in range(o["mv"].shape[0]):
        sse, _ = O.compensate(p, seq.luma[k], seq.luma[k + 1], o["mv"][k])
        assert sse == o["sse"][k]


def test_sequence_equals_chained_pairs_and_is_deterministic():
    seq = synth.cif_sequence(frames=4)
    p = O.OracleParams(352, 288, 16, 2)
    o1 = O.estimate_sequence(p, seq.luma, seq.alpha[0])
    o2 = O.estimate_sequence(p, seq.luma, seq.alpha[0])
    for k in ("mv", "cost", "disp", "iters", "npos", "sse"):
        assert np.array_equal(o1[k], o2[k])
    tmp = None
    for k in range(3):
        r = O.estimate_pair(p, seq.luma[k], seq.luma[k + 1], seq.alpha[0][k], seq.alpha[0][k + 1],
                            temporal=tmp)
        assert np.array_equal(r["mv"], o1["mv"][k])
        tmp = r["mv"]


# ------------------------------------------------- learned-proposal seeds --
def test_seed_at_a_plain_candidate_changes_nothing():
    """A seed equal to the temporal candidate can never win strictly, so the
    seeded run equals the plain one (same vectors, costs, steps, positions)."""
    seq = synth.cif_sequence(frames=4)
    p = O.OracleParams(352, 288, 16, 2)
    plain = O.estimate_sequence(p, seq.luma, seq.alpha[0])
    P, M = plain["mv"].shape[:2]
    seed = np.zeros((P, M, 2), np.float32)
    seed[1:] = plain["mv"][:-1].astype(np.float32) / 2  # T of pairs 1.. in pixels
    seeded = O.estimate_sequence(p, seq.luma, seq.alpha[0], seed=seed)
    for k in ("mv", "cost", "iters", "npos", "disp", "sse"):
        assert np.array_equal(plain[k][1:], seeded[k][1:]), k


def test_seeded_result_never_worse_on_an_isolated_mb():
    """One MB per frame (no neighbours): whatever the seed, the kept search
    ends with a SAD no larger than the plain search's."""
    rng = np.random.default_rng(9)
    worse = better = 0
    for trial in range(60):
        luma, alpha = synth.translated_pair(48, 48, rng.integers(-5, 6, 2), seed=trial, noise_sigma=2.0)
        ref, cur = luma[0, 16:32, 16:32].copy(), luma[1, 16:32, 16:32].copy()
        # a 16x16 frame has V = {0}; use 48x48 frames with the middle MB only opaque
        a = np.zeros((2, 48, 48), np.uint8)
        a[:, 16:32, 16:32] = 255
        p = O.OracleParams(48, 48, 16, 2)
        plain = O.estimate_pair(p, luma[0], luma[1], a[0], a[1])
        seed = rng.normal(0, 6, (9, 2)).astype(np.float32)
        s = O.estimate_pair(p, luma[0], luma[1], a[0], a[1], seed=seed)
        assert s["cost"][4] <= plain["cost"][4]
        better += s["cost"][4] < plain["cost"][4]
    assert better > 0  # the seed path is taken sometimes


def test_perfect_seed_recovers_translation():
    """With a seed at the true vector every MB whose window contains it ends
    at SAD 0 there, with no plain candidate in reach."""
    W, H, sh = 128, 96, np.array([5, -6])
    luma, alpha = synth.translated_pair(W, H, sh, seed=4)
    p = O.OracleParams(W, H, 16, 2, max_iters=1)
    seed = np.tile(-sh.astype(np.float32), (p.mbs, 1))
    o = O.estimate_pair(p, luma[0], luma[1], alpha[0], alpha[1], seed=seed)
    tgt = -sh * 2
    for m in range(p.mbs):
        lox, hix, loy, hiy = O.valid_range(W, H, 16, 16, 2, 16 * (m % 8), 16 * (m // 8))
        if lox <= tgt[0] <= hix and loy <= tgt[1] <= hiy:
            assert (o["mv"][m] == tgt).all() and o["cost"][m] == 0


def test_seeded_runs_are_capped_at_eight_steps():
    """An opaque MB whose seed wins runs two pixel-recursive searches (reading
    c21), up to 5 + 2 * 9 * K evaluated positions; the count is a byte, which
    holds it only up to K = 8 (149).  Seeded runs above that cap are refused;
    unseeded ones keep the full cap of 16 steps (4 + 9 * 16 = 148)."""
    rng = np.random.default_rng(21)
    W = H = 96
    luma = rng.integers(0, 256, (2, H, W), dtype=np.uint8)
    a = np.full((2, H, W), 255, np.uint8)
    seed = rng.normal(0, 8, ((W // 16) * (H // 16), 2)).astype(np.float32)
    with pytest.raises(ValueError):
        O.estimate_pair(O.OracleParams(W, H, 16, 2, max_iters=9), luma[0], luma[1], a[0], a[1], seed=seed)
    with pytest.raises(ValueError):
        O.estimate_sequence(O.OracleParams(W, H, 16, 2, max_iters=16), luma, a, seed=seed[None])
    o = O.estimate_pair(O.OracleParams(W, H, 16, 2, max_iters=8), luma[0], luma[1], a[0], a[1], seed=seed)
    assert int(o["npos"].max()) <= 5 + 2 * 9 * 8
    assert int(o["iters"].max()) <= 8
    o = O.estimate_pair(O.OracleParams(W, H, 16, 2, max_iters=16), luma[0], luma[1], a[0], a[1])
    assert int(o["npos"].max()) <= 4 + 9 * 16


# ------------------------------------- one MB, hand-derived search paths --
def _middle_mb(ref, cur, h, seed_px=None):
    """48 x 48 frames with only the middle MB opaque (its neighbours are
    transparent, so A, B, C, T are all (0, 0)); outputs of that MB."""
    a = np.zeros((48, 48), np.uint8)
    a[16:32, 16:32] = 255
    p = O.OracleParams(48, 48, 16, h)
    seed = None
    if seed_px is not None:
        seed = np.zeros((9, 2), np.float32)
        seed[4] = seed_px
    o = O.estimate_pair(p, ref, cur, a, a, seed=seed)
    return {k: o[k][4] for k in ("mv", "cost", "iters", "npos")}


def _x_ramp(slope, offset):
    X = np.mgrid[0:48, 0:48][1]
    return (slope * X + 50 + offset).astype(np.uint8)


def test_prs_proposal_with_equal_sad_is_not_taken():
    """Fig. 4 reading: the proposal is taken only if its SAD is strictly
    lower.  cur = 2x + 50, ref = cur + 1: at d = 0 every DPD is 1, u = 1/2,
    the update is -1/2 px and rounds (half away from zero) to q = (-1, 0),
    whose SAD (256) equals SAD(0); no neighbour is strictly lower either."""
    o = _middle_mb(_x_ramp(2, 1), _x_ramp(2, 0), 1)
    assert tuple(o["mv"]) == (0, 0) and o["cost"] == 256 and o["iters"] == 1
    assert o["npos"] == 9  # (0,0), then q = (-1,0) and the eight neighbours


def test_prs_proposal_rounds_half_away_from_zero():
    """cur = 4x + 50, ref = 4x + 47 (content shifted by 3/4 px), half-pel.
    Step 1 at d = 0: DPD = -3, u = 1/4, update +3/4 px = 1.5 MV units ->
    q = 2 (SAD 256 < 768).  Step 2 at d = 2: update -1/4 px = -0.5 units ->
    q = 1, SAD 256 not lower; neighbours at best tie: stop at (2, 0)."""
    o = _middle_mb(_x_ramp(4, -3), _x_ramp(4, 0), 2)
    assert tuple(o["mv"]) == (2, 0) and o["cost"] == 256 and o["iters"] == 2
    assert o["npos"] == 10  # (0,0), (2,0), then (1,0) and the other seven neighbours of (2,0)


def test_eight_directions_take_the_first_strict_minimum_in_raster_order():
    """Flat current block (no gradient, so no proposal), reference 100 +
    |x + y - 46|: the SAD of a shift depends on s = dx + dy only and is
    lowest at s = -1, where (0, -1) and (-1, 0) tie.  Raster order (row -1
    first) reaches (0, -1) first; from there nothing is strictly lower."""
    Y, X = np.mgrid[0:48, 0:48]
    cur = np.full((48, 48), 100, np.uint8)
    ref = (100 + np.abs(X + Y - 46)).astype(np.uint8)
    o = _middle_mb(ref, cur, 1)
    assert tuple(o["mv"]) == (0, -1) and o["iters"] == 2


def test_seeded_search_is_kept_only_when_strictly_better():
    """Reading c21 on the 3/4-px ramp: a seed of 1/2 px (MV unit 1, SAD 256)
    beats A..T (SAD 768); its search stays at 1 (SAD 256), the plain search
    from 0 ends at 2 with the same SAD, so the plain result is kept."""
    o = _middle_mb(_x_ramp(4, -3), _x_ramp(4, 0), 2, seed_px=(0.5, 0.0))
    assert tuple(o["mv"]) == (2, 0) and o["cost"] == 256 and o["iters"] == 2


def test_seed_rounds_half_away_from_zero():
    """Reading c19: a seed of -0.2 px is -0.4 MV units and rounds to 0, a
    position already evaluated, so the result and the distinct-position
    count equal the unseeded ones."""
    ref, cur = _x_ramp(4, -3), _x_ramp(4, 0)
    plain = _middle_mb(ref, cur, 2)
    seeded = _middle_mb(ref, cur, 2, seed_px=(-0.2, 0.0))
    for k in plain:
        assert np.array_equal(plain[k], seeded[k]), k


# ------------------------------- Sec. 3.1 variant: boundary T judged by texture --
def _boundary_case(move_texture, move_alpha, flat=False):
    """48 x 48 frames, the middle MB a boundary MB (left half inside), every
    other MB transparent, so A = B = C = (0, 0); T = (-2, 0) is given.  The
    texture and/or the alpha move by +2 px (the displacement that matches
    them is -2)."""
    luma, _ = synth.translated_pair(48, 48, (2, 0) if move_texture else (0, 0), seed=4)
    if flat:
        luma = np.full_like(luma, 90)
    a = np.zeros((2, 48, 48), np.uint8)
    a[0, 16:32, 16:24] = 255
    a[1, 16:32, 16 + (2 if move_alpha else 0):24 + (2 if move_alpha else 0)] = 255
    tmp = np.zeros((9, 2), np.int16)
    tmp[4] = (-2, 0)
    return luma, a, tmp


def _run_boundary(variant, **kw):
    luma, a, tmp = _boundary_case(**kw)
    p = O.OracleParams(48, 48, 16, 1, boundary_t_texture=variant)
    o = O.estimate_pair(p, luma[0], luma[1], a[0], a[1], temporal=tmp)
    assert o["mbclass"][4] == 2
    return o, luma, a


def test_boundary_temporal_by_texture_takes_t_when_texture_says_so():
    """Texture moves, alpha does not: by shape (Fig. 1) A = (0,0) wins with 0
    mismatches; with the variant, the spatial winner (0,0) and T = (-2,0) are
    compared by texture SAD, T matches exactly and is kept, its cost being its
    shape cost (16 rows x 4 columns of mismatches, 2 on each side = 64)."""
    o, luma, a = _run_boundary(0, move_texture=True, move_alpha=False)
    assert tuple(o["mv"][4]) == (0, 0) and o["cost"][4] == 0
    o, luma, a = _run_boundary(1, move_texture=True, move_alpha=False)
    assert tuple(o["mv"][4]) == (-2, 0)
    assert o["cost"][4] == O.shape_sad(a[0], a[1], 1, 16, 16, -2, 0) == 64
    assert O.texture_sad(luma[0], luma[1], 1, 16, 16, -2, 0) == 0
    assert o["iters"][4] == 0 and o["npos"][4] == 2


def test_boundary_temporal_by_texture_not_by_shape():
    """Alpha moves, texture does not: by shape T = (-2,0) wins (0 mismatches
    against 64); with the variant T must beat the spatial winner (0,0) on
    texture, where (0,0) is exact, so (0,0) stays."""
    o, _, a = _run_boundary(0, move_texture=False, move_alpha=True)
    assert tuple(o["mv"][4]) == (-2, 0) and o["cost"][4] == 0
    o, _, a = _run_boundary(1, move_texture=False, move_alpha=True)
    assert tuple(o["mv"][4]) == (0, 0)
    assert o["cost"][4] == O.shape_sad(a[0], a[1], 1, 16, 16, 0, 0) == 64


def test_boundary_temporal_by_texture_tie_keeps_the_spatial_winner():
    """Flat luma: both texture SADs are 0, T is not strictly lower."""
    o, _, _ = _run_boundary(1, move_texture=True, move_alpha=False, flat=True)
    assert tuple(o["mv"][4]) == (0, 0) and o["cost"][4] == 0
