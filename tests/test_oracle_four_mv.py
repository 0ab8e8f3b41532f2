"""Pins of the oracle's four-vector mode (Sec. 3.2: MPEG-4 allows four
vectors per MB, so the recursive search works on 8x8 blocks) against facts
that do not come from the oracle itself: closed forms of the gradient step on
ramps, the reduction to the pinned 16x16 procedure when no pixel-recursive
step is taken, constructions whose block vectors and step counts follow from
how the frames were built, the exhaustive search with 8x8 blocks, and the
16x16 compensation routine assembled block by block.

Readings (four-vector mode): the block recursive search stays at MB level
(Fig. 1); its winner starts the pixel recursive search of each 8x8 block;
A = block 1 of the left MB, B = block 2 of the MB above, C = block 2 of the
MB above-right, T = block 0 of the same MB in the previous field; boundary
MBs give the winner to all four blocks, each costed by its own quadrant."""
import numpy as np
import pytest

import oracle as O
from paper_1002_1168_gb300 import synth


def _ramp(W, H, ax, ay, c=10):
    Y, X = np.mgrid[0:H, 0:W]
    return (c + ax * X + ay * Y).astype(np.uint8)


# ------------------------------------------------- Eqs. 3-5 on 8x8 blocks --
@pytest.mark.parametrize("X0,Y0", [(8, 8), (0, 0), (24, 16)])
def test_block_gradient_closed_form_on_ramps(X0, Y0):
    """cur = 2x + 4y + 10, ref = cur: Eq. 5 gives g_x = 4 (u_x = 1/2) and
    g_y = 8 (u_y = 1/4) wherever the central difference exists.  At d = (1, 0)
    the DPD is 2 at every pixel, so the updates are -1 and -1/2 exactly, the
    means taken over the pixels that have a gradient (56 on the corner block,
    whose first column and row have none)."""
    cur = _ramp(48, 32, 2, 4)  # at most 228: no wrap-around
    p = O.OracleParams(48, 32, 4, 1, theta=2.0, epsilon=1.0)
    assert np.array_equal(O.gradient_step_block(p, cur, cur, X0, Y0, 8, 1, 0), np.float32([-1.0, -0.5]))
    assert np.array_equal(O.gradient_step_block(p, cur, cur, X0, Y0, 8, 0, 1), np.float32([-2.0, -1.0]))
    # epsilon scales the update
    p2 = O.OracleParams(48, 32, 4, 1, theta=2.0, epsilon=0.5)
    assert np.array_equal(O.gradient_step_block(p2, cur, cur, X0, Y0, 8, 0, 1), np.float32([-1.0, -0.5]))
    if X0 > 0 and Y0 > 0:  # the sign follows the DPD (the displaced block stays inside the frame)
        assert np.array_equal(O.gradient_step_block(p, cur, cur, X0, Y0, 8, -1, 0), np.float32([1.0, 0.5]))
    # on the corner block (0, 0) only 56 pixels have each gradient: a mean over
    # all 64 would give -56/64 instead of -1


def test_block_gradient_reads_its_own_block():
    """Two ramps side by side: the block's update depends only on the ramp
    under it (cur = 2x in the left half, 4x in the right, y constant)."""
    cur = np.zeros((32, 64), np.uint8)
    X = np.arange(64)
    cur[:] = np.where(X < 32, 2 * X + 10, 4 * X - 50).astype(np.uint8)
    p = O.OracleParams(64, 32, 4, 1)
    # d = (1, 0): DPD = 2 (left) or 4 (right); u_x = 1/2 or 1/4: update -1 both;
    # d = (2, 0): -2 both; but with ref = cur + 8 the DPD is 8 + slope*dx.
    ref = (cur.astype(np.int32) + 8).astype(np.uint8)
    assert np.array_equal(O.gradient_step_block(p, ref, cur, 8, 8, 8, 0, 0), np.float32([-4.0, 0.0]))
    assert np.array_equal(O.gradient_step_block(p, ref, cur, 40, 8, 8, 0, 0), np.float32([-2.0, 0.0]))


def test_block_gradient_pairwise_tree_in_block_raster_order():
    """Terms of different magnitudes: the FP32 sum is the contiguous pairwise
    tree over the block's 64 terms in raster order (level by level, element i
    absorbs element i + s), not a sequential sum."""
    rng = np.random.default_rng(5)
    W = H = 32
    cur = np.zeros((H, W), np.uint8)
    cur[:] = (10 + 3 * np.arange(W))[None, :]  # g_x = 6 -> u_x = 1/3 everywhere inside
    ref = rng.integers(0, 256, (H, W)).astype(np.uint8)
    p = O.OracleParams(W, H, 4, 1)
    X0, Y0 = 8, 16
    u = np.float32(2.0) / np.float32(6.0)
    terms = [np.float32(int(ref[Y0 + j, X0 + i]) - int(cur[Y0 + j, X0 + i])) * u for j in range(8) for i in range(8)]
    t = list(terms)
    s = 1
    while s < 64:
        for i in range(0, 64 - s, 2 * s):
            t[i] = np.float32(t[i] + t[i + s])
        s *= 2
    expect = np.float32(-(np.float32(1.0) * np.float32(t[0] / np.float32(64))))
    got = O.gradient_step_block(p, ref, cur, X0, Y0, 8, 0, 0)
    assert got[0] == expect and got[1] == 0.0


# -------------------------------------------- reduction to the 16x16 pass --
@pytest.mark.parametrize("h", [1, 2])
def test_without_recursive_steps_equals_the_16x16_pass(h):
    """max_iters = 0: no block moves from the MB winner, so every block vector
    is the 16x16 vector, the block costs add up to the MB cost (SAD and alpha
    mismatches both split over the quadrants), the positions are the MB
    candidates, and the compensation is the 16x16 one."""
    seq = synth.cif_sequence(frames=4)
    p = O.OracleParams(352, 288, 16, h, max_iters=0)
    o16 = O.estimate_sequence(p, seq.luma, seq.alpha[0])
    o4 = O.estimate_sequence4(p, seq.luma, seq.alpha[0])
    assert np.array_equal(o4["mbclass"], o16["mbclass"])
    for b in range(4):
        assert np.array_equal(o4["mv"][:, :, b], o16["mv"])
        assert np.array_equal(o4["npos"][:, :, b], o16["npos"])
    assert np.array_equal(o4["cost"].sum(axis=2, dtype=np.uint64), o16["cost"].astype(np.uint64))
    assert not o4["iters"].any() and not o4["disp"].any()
    assert np.array_equal(o4["sse"], o16["sse"])
    assert (o16["mbclass"] == 2).any() and (o16["mbclass"] == 1).any()


# ------------------------------------------------ candidates by construction --
def _blockwise(ref, D):
    """cur(p) = ref(p + D[block of p]) for a per-8x8-block field D [H/8, W/8, 2] (pixels)."""
    H, W = ref.shape
    cur = ref.copy()
    for by in range(H // 8):
        for bx in range(W // 8):
            dx, dy = D[by, bx]
            cur[8 * by:8 * by + 8, 8 * bx:8 * bx + 8] = ref[8 * by + dy:8 * by + dy + 8, 8 * bx + dx:8 * bx + dx + 8]
    return cur


def _set_mb(D, u, v, vecs):
    """Block vectors of MB (u, v): vecs[b] for b = 2*by + bx."""
    for b, vec in enumerate(vecs):
        D[2 * v + (b >> 1), 2 * u + (b & 1)] = vec


def _descent_frame():
    """A ramp with slopes below Theta (every u of Eq. 4 is zero, so the pixel
    recursive search is the eight-direction descent of Fig. 4 alone), SAD 0
    only at the exact block displacement among nearby vectors."""
    Y, X = np.mgrid[0:48, 0:64]
    return np.rint(30 + 1.2 * X + 0.7 * Y).astype(np.uint8)


def _run(D, temporal4=None):
    ref = _descent_frame()
    cur = _blockwise(ref, D)
    p = O.OracleParams(64, 48, 4, 1, theta=2.0, max_iters=8)
    a = np.full((64, 48), 255, np.uint8).T.copy()
    return O.estimate_pair4(p, ref, cur, a, a, temporal4=temporal4), p


L_VECS = [(1, 1), (-1, 1), (1, -1), (-1, -1)]


def _n8_union(cands, d, V):
    lox, hix, loy, hiy = V
    pos = set(cands)
    for j in (-1, 0, 1):
        for i in (-1, 0, 1):
            q = (min(max(d[0] + i, lox), hix), min(max(d[1] + j, loy), hiy))
            pos.add(q)
    return len(pos)


@pytest.mark.parametrize("role", ["A", "B", "C", "T"])
def test_candidate_blocks_by_construction(role):
    """An MB L with four different block motions, and an MB X moved as a whole
    by the motion of the block of L that the role names (A: block 1 of the left
    MB, B / C: block 2 of the MB above / above-right; T: block 0 of the given
    previous field).  Every other block stays still.  L's blocks descend from
    the zero winner to their motions in one step each (two PRS steps, SAD 0);
    X's candidate from L has SAD 0, so X keeps it with one PRS step and no
    move.  Taking any other block of L would cost X further steps."""
    D = np.zeros((6, 8, 2), np.int64)
    temporal4 = None
    MBW = 4
    if role == "T":
        X = (1, 1)
        temporal4 = np.zeros((12, 4, 2), np.int16)
        temporal4[1 * MBW + 1] = L_VECS
        src = L_VECS[0]
    else:
        L, X, b = {"A": ((1, 1), (2, 1), 1), "B": ((1, 1), (1, 2), 2), "C": ((2, 1), (1, 2), 2)}[role]
        _set_mb(D, *L, L_VECS)
        src = L_VECS[b]
    _set_mb(D, *X, [src] * 4)
    o, p = _run(D, temporal4)
    if role != "T":
        mL = L[1] * MBW + L[0]
        assert np.array_equal(o["mv"][mL], np.int16(L_VECS)), "L's blocks reach their motions"
        assert not o["cost"][mL].any() and (o["iters"][mL] == 2).all()
    mX = X[1] * MBW + X[0]
    assert (o["mv"][mX] == np.int16(src)).all() and not o["cost"][mX].any()
    assert (o["iters"][mX] == 1).all(), "X's winning candidate came from the named block"
    V = O.valid_range(64, 48, 16, 4, 1, 16 * X[0], 16 * X[1])
    assert (o["npos"][mX] == _n8_union({tuple(src), (0, 0)}, src, V)).all()
    # every still block outside L and X stays at zero with one PRS step
    still = [m for m in range(12) if m != mX and (role == "T" or m != L[1] * MBW + L[0])]
    for m in still:
        assert not o["mv"][m].any() and not o["cost"][m].any()


def test_temporal_field_chains_block_zero():
    """Three frames, pair 1's T is block 0 of pair 0's field: X's blocks in
    pair 1 keep T with one step when X moves in pair 1 as block 0 of X moved in
    pair 0."""
    ref = _descent_frame()
    D0 = np.zeros((6, 8, 2), np.int64)
    _set_mb(D0, 1, 1, L_VECS)
    f1 = _blockwise(ref, D0)
    D1 = np.zeros((6, 8, 2), np.int64)
    _set_mb(D1, 1, 1, [L_VECS[0]] * 4)
    # frame 2 is frame 1 moved, MB (1, 1) as a whole by block 0's motion
    f2 = _blockwise(f1, D1)
    luma = np.stack([ref, f1, f2])
    alpha = np.full((3, 48, 64), 255, np.uint8)
    p = O.OracleParams(64, 48, 4, 1, max_iters=8)
    o = O.estimate_sequence4(p, luma, alpha)
    assert np.array_equal(o["mv"][0, 5], np.int16(L_VECS))
    assert (o["mv"][1, 5] == np.int16(L_VECS[0])).all() and (o["iters"][1, 5] == 1).all()


# ------------------------------------------------------------ invariants --
def test_known_translation_every_block():
    """Noise-free low-frequency texture moved by an integer vector: the
    exhaustive search with 8x8 blocks has SAD 0 at -v, and the four-vector
    search reaches it on nearly every block whose MB window contains it."""
    hit = tot = 0
    for seed in range(4):
        rng = np.random.default_rng(200 + seed)
        sh = rng.integers(-3, 4, 2)
        luma, alpha = synth.translated_pair(128, 96, sh, seed=seed)
        p = O.OracleParams(128, 96, 16, 2)
        o = O.estimate_pair4(p, luma[0], luma[1], alpha[0], alpha[1])
        tgt = -sh * 2
        for m in range(p.mbs):
            lox, hix, loy, hiy = O.valid_range(128, 96, 16, 16, 2, 16 * (m % 8), 16 * (m // 8))
            if not (lox <= tgt[0] <= hix and loy <= tgt[1] <= hiy):
                continue
            for b in range(4):
                tot += 1
                hit += bool((o["mv"][m, b] == tgt).all() and o["cost"][m, b] == 0)
    assert hit >= 0.97 * tot


def test_block_costs_never_beat_the_8x8_exhaustive_search_and_boundary_quadrants():
    """On a VOP sequence: every opaque block's SAD is at least the 8x8 ES
    optimum (the block's V contains the MB's); transparent MBs carry nothing;
    boundary MBs keep one vector, no PRS step, and quadrant costs adding up to
    the 16x16 alpha mismatch count."""
    seq = synth.cif_sequence(frames=3)
    W, H = 352, 288
    p = O.OracleParams(W, H, 16, 2)
    o = O.estimate_sequence4(p, seq.luma, seq.alpha[0])
    for k in range(2):
        _, es, _ = O.full_search(seq.luma[k], seq.luma[k + 1], W, H, 2, 16, block=8)
        es = es.reshape(H // 8, W // 8)
        cls = o["mbclass"][k]
        for m in range(p.mbs):
            u, v = m % (W // 16), m // (W // 16)
            if cls[m] == 0:
                assert not o["mv"][k, m].any() and not o["cost"][k, m].any() and not o["npos"][k, m].any()
            elif cls[m] == 1:
                for b in range(4):
                    assert o["cost"][k, m, b] >= es[2 * v + (b >> 1), 2 * u + (b & 1)]
            else:
                assert (o["mv"][k, m] == o["mv"][k, m, 0]).all() and not o["iters"][k, m].any()
                dx, dy = o["mv"][k, m, 0]
                assert o["cost"][k, m].sum() == O.shape_sad(seq.alpha[0, k], seq.alpha[0, k + 1], 2, 16 * u, 16 * v,
                                                             int(dx), int(dy))
        assert (o["iters"][k][cls == 1] >= 1).all()


def test_compensation_is_the_16x16_one_block_by_block():
    """The SSE with four vectors per MB equals the error of the image whose
    8x8 block b is taken from the 16x16 compensation with every MB at its
    block-b vector."""
    seq = synth.cif_sequence(frames=2)
    W, H = 352, 288
    p = O.OracleParams(W, H, 16, 2)
    o = O.estimate_sequence4(p, seq.luma, seq.alpha[0], want_pred=True)
    pred = np.zeros((H, W), np.uint8)
    for b in range(4):
        _, pb = O.compensate(p, seq.luma[0], seq.luma[1], o["mv"][0, :, b], want_pred=True)
        for v in range(H // 16):
            for u in range(W // 16):
                y, x = 16 * v + 8 * (b >> 1), 16 * u + 8 * (b & 1)
                pred[y:y + 8, x:x + 8] = pb[y:y + 8, x:x + 8]
    assert np.array_equal(pred, o["pred"][0])
    err = seq.luma[1].astype(np.int64) - pred
    assert int((err * err).sum()) == int(o["sse"][0])
    assert (o["mv"][0, :, 0] != o["mv"][0, :, 3]).any()  # the blocks do differ somewhere


def test_block_proposal_with_equal_sad_is_not_taken():
    """The 8x8 analogue of the 16x16 fixture: cur = 2x + 50, ref = cur + 1,
    only the middle MB opaque (all candidates (0, 0)).  Each block: DPD = 1,
    u = 1/2, the update -1/2 px rounds to q = (-1, 0), whose SAD (64) equals
    SAD(0); no neighbour is strictly lower, so every block stays at (0, 0)
    after one step with 9 positions."""
    X = np.mgrid[0:48, 0:48][1]
    cur, ref = (2 * X + 50).astype(np.uint8), (2 * X + 51).astype(np.uint8)
    a = np.zeros((48, 48), np.uint8)
    a[16:32, 16:32] = 255
    o = O.estimate_pair4(O.OracleParams(48, 48, 16, 1), ref, cur, a, a)
    assert not o["mv"][4].any() and (o["cost"][4] == 64).all()
    assert (o["iters"][4] == 1).all() and (o["npos"][4] == 9).all()
