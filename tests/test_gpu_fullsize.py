"""Parity at the full sizes of the large workloads, in the launch
configuration the benchmark times (LearnedBatch: the seed network's launches
in a CUDA graph, then every VOP in one persistent launch, autotuned and
replayed from a graph).

The oracle computes single pairs: for a sampled (sequence, VOP, pair) it
estimates that pair from the same frames, with the GPU's field of the
previous pair as the temporal candidates and the same seeds, and must agree
bit for bit.  Every pair of every VOP is checked on the device by properties
that hold at any size (Fig. 1: transparent MBs carry no vector and no cost;
every vector lies in the valid set V; the per-pair SSE is the sum of the
per-MB SSEs; iterations within the cap).

Workloads: 1920x1088, 300 frames, 4 VOPs, S = 16 (the learned proposal's
evaluation sequence) and 16 sequences of 3840x2160, 60 frames, 8 VOPs each,
S = 32 (learned proposal + batching at scale), rendered on the device
(synth_gpu).  The network has its initial weights (any weights give seeds;
parity is about what the search does with them)."""
import gc

import numpy as np
import pytest

import oracle as O
from oracle import seednet as SN

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    from paper_1002_1168_gb300 import build as cuda_build
    from paper_1002_1168_gb300 import seedtrain, sme, synth_gpu

    cuda_build.build()
    return sme, seedtrain, synth_gpu


def _net(sme, max_cells, seed=4):
    params = SN.init_params(seed)
    params = [(w * (30.0 if li == 4 else 1.0), b) for li, (w, b) in enumerate(params)]  # seeds of a few px
    net = sme.SeedNet(max_cells=max_cells)
    net.set_params(sme.pack_params(params))
    return net


def _properties(out, W, H, S, h, K):
    """Checks on the device over every pair of one VOP."""
    cls, mv = out["mb_class"].long(), out["mv"].long()
    P, M = cls.shape
    MBW = W // 16
    t = cls == 0
    assert not mv[t].any() and not out["cost"][t].any() and not out["iters"][t].any() and not out["npos"][t].any()
    u = torch.arange(M, device=mv.device) % MBW
    v = torch.arange(M, device=mv.device) // MBW
    X0, Y0 = (16 * u)[None], (16 * v)[None]
    dx, dy = mv[..., 0], mv[..., 1]
    assert (dx.abs() <= S * h).all() and (dy.abs() <= S * h).all()
    assert (dx >= -X0 * h).all() and (dx <= (W - 16 - X0) * h).all()
    assert (dy >= -Y0 * h).all() and (dy <= (H - 16 - Y0) * h).all()
    assert (out["iters"].long() <= K).all()
    assert torch.equal(out["sse_mb"].view(torch.int32).long().sum(dim=1),
                       out["sse"].view(torch.int64)), "per-pair SSE = sum of per-MB SSE"


def _oracle_pair(luma, alpha, k, S, h, out, seeds, W, H):
    """The oracle on pair k alone, given the GPU's previous field and the seeds."""
    ln = luma[k:k + 2].cpu().numpy()
    an = alpha[k:k + 2].cpu().numpy()
    tmp = None if k == 0 else out["mv"][k - 1].cpu().numpy()
    sd = seeds[k:k + 1].cpu().numpy()
    o = O.estimate_sequence(O.OracleParams(W, H, S, h), ln, an, temporal_in=tmp, seed=sd)
    g = {key: out[key][k].cpu().numpy() for key in ("mv", "cost", "iters", "npos", "mb_class", "disp")}
    assert np.array_equal(g["mb_class"], o["mbclass"][0])
    assert np.array_equal(g["mv"], o["mv"][0])
    assert np.array_equal(g["cost"].view(np.uint32), o["cost"][0])
    assert np.array_equal(g["iters"], o["iters"][0])
    assert np.array_equal(g["npos"], o["npos"][0])
    assert np.abs(g["disp"] - o["disp"][0]).max(initial=0) <= 1e-4
    assert int(out["sse"][k].view(torch.int64).item()) == int(o["sse"][0])


WANT = ("cost", "disp", "iters", "npos", "mb_class", "sse_mb", "sse")


def test_hd_300_frames_4_vops_learned(lib):
    sme, seedtrain, synth_gpu = lib
    W, H, S, h, K = 1920, 1088, 16, 2, 8
    luma, alpha, _ = synth_gpu.hd_learned_eval()
    F = luma.shape[0]
    net = _net(sme, (F - 1) * (H // 4) * (W // 4))
    lb = seedtrain.LearnedBatch(net, [(luma, [alpha[j] for j in range(alpha.shape[0])])], search_range=S, subpel=h,
                                want=WANT)
    lb.tune(trials=1)
    outs = lb.run()
    seeds = lb.seeds[0]
    for j, out in enumerate(outs):
        _properties(out, W, H, S, h, K)
    nt = sum(int((o["mb_class"] > 0).sum()) for o in outs)
    assert nt > 0
    for j, k in ((0, 0), (1, 150), (3, F - 2)):
        _oracle_pair(luma, alpha[j], k, S, h, outs[j], seeds, W, H)
    lb.close()
    net.close()
    del lb, luma, alpha, outs
    gc.collect()
    torch.cuda.empty_cache()


def test_uhd_16_sequences_8_vops_learned_batch(lib):
    sme, seedtrain, synth_gpu = lib
    W, H, S, h, K = 3840, 2160, 32, 2, 8
    seqs = synth_gpu.uhd_batch()
    F = seqs[0][0].shape[0]
    net = _net(sme, (F - 1) * (H // 4) * (W // 4))
    groups = [(l, [a[j] for j in range(a.shape[0])]) for l, a, _ in seqs]
    lb = seedtrain.LearnedBatch(net, groups, search_range=S, subpel=h, want=WANT)
    lb.tune(trials=1)
    outs = lb.run()
    total = sum(int(o["mb_class"].numel()) for o in outs)
    assert total == 16 * 8 * (F - 1) * (W // 16) * (H // 16)
    vis = 0
    for out in outs:
        _properties(out, W, H, S, h, K)
        vis += int((out["mb_class"] > 0).sum())
    assert 0.01 < vis / total < 0.1  # each VOP is one object covering a few per cent of the frame
    # (sequence, VOP, pair) samples; VOP i of sequence s is outs[8 s + i]
    for s, j, k in ((0, 0, 0), (7, 3, 30), (15, 7, F - 2)):
        luma, alpha, _ = seqs[s]
        _oracle_pair(luma, alpha[j], k, S, h, outs[8 * s + j], lb.seeds[8 * s + j], W, H)
    lb.close()
    net.close()
    del lb, seqs, outs, groups
    gc.collect()
    torch.cuda.empty_cache()
