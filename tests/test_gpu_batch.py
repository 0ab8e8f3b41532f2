"""GPU parity of the batched path: many sequences of uneven size and length in
one launch give, per sequence, exactly the oracle's results -- before and
after autotuning, and on replays of the captured graph."""
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


def _batch_inputs():
    sizes = [(176, 144, 4), (352, 288, 6), (96, 64, 3), (704, 576, 3), (176, 144, 2), (48, 32, 5)]
    seqs = []
    for i, (W, H, F) in enumerate(sizes):
        s = synth.make_sequence(W, H, F, seed=500 + i, n_objects=1 + i % 3, vmax=8.0, obj_frac=0.35)
        for j in range(s.alpha.shape[0]):
            seqs.append((s.luma, s.alpha[j]))
    return seqs


def _check_all(outs, seqs, S=16, h=2):
    for (luma, alpha), g in zip(seqs, outs):
        F, H, W = luma.shape
        o = O.estimate_sequence(O.OracleParams(W, H, S, h), luma, alpha)
        assert np.array_equal(g["mv"].cpu().numpy(), o["mv"])
        assert np.array_equal(g["cost"].cpu().numpy().view(np.uint32), o["cost"])
        assert np.array_equal(g["iters"].cpu().numpy(), o["iters"])
        assert np.array_equal(g["npos"].cpu().numpy(), o["npos"])
        assert np.array_equal(g["mb_class"].cpu().numpy(), o["mbclass"])
        assert np.array_equal(g["disp"].cpu().numpy().view(np.uint32), o["disp"].view(np.uint32))
        assert np.array_equal(g["sse"].cpu().numpy().view(np.uint64), o["sse"])


def test_batch_uneven_sequences_match_oracle(sme):
    seqs = _batch_inputs()
    lumas = [torch.from_numpy(l).cuda() for l, _ in seqs]
    alphas = [torch.from_numpy(a).cuda() for _, a in seqs]
    b = sme.Batch(lumas, alphas, search_range=16, subpel=2)
    outs = b.run()                      # default configuration, direct launches
    _check_all(outs, seqs)
    for o in outs:
        for v in o.values():
            v.zero_()
    b.tune(trials=2)                    # every configuration, then a captured graph
    cfg = b.config()
    assert cfg["tuned_ms"] > 0 and cfg["schedule"] in ("mb", "pair", "sparse")
    outs = b.run()
    _check_all(outs, seqs)
    outs = b.run()                      # graph replay keeps the same results
    _check_all(outs, seqs)
    b.close()


def test_autotune_context_keeps_results(sme):
    seq = synth.cif_sequence(seed=1002, frames=8)
    est = sme.Estimator(352, 288, search_range=16, subpel=2)
    luma, alpha = torch.from_numpy(seq.luma).cuda(), torch.from_numpy(seq.alpha[0]).cuda()
    est.autotune(luma, alpha, trials=2)
    g = est.estimate_sequence(luma, alpha)
    o = O.estimate_sequence(O.OracleParams(352, 288, 16, 2), seq.luma, seq.alpha[0])
    assert np.array_equal(g["mv"].cpu().numpy(), o["mv"])
    assert np.array_equal(g["sse"].cpu().numpy().view(np.uint64), o["sse"])
    est.close()


@pytest.mark.parametrize("schedule,param,flag", [("sparse", 1, 1), ("sparse", 2, 0), ("sparse", 3, 0), ("sparse", 5, 0),
                                                 ("mb", 0, 1),
                                                 ("pair", 8, 1), ("pair", 4, 0)])
def test_batch_each_configuration_matches_oracle(sme, schedule, param, flag):
    """Every execution configuration of a batch, set explicitly, gives the
    oracle's results on every sequence, on two runs in a row (the second
    run reuses every scratch buffer of the first)."""
    seqs = _batch_inputs()
    lumas = [torch.from_numpy(l).cuda() for l, _ in seqs]
    alphas = [torch.from_numpy(a).cuda() for _, a in seqs]
    b = sme.Batch(lumas, alphas, search_range=16, subpel=2,
                  want=("cost", "disp", "iters", "npos", "mb_class", "sse", "sse_mb", "pred"))
    b.set_config(schedule, param, flag)
    assert b.config()["schedule"] == schedule
    for _ in range(2):
        outs = b.run()
        _check_all(outs, seqs)
        for (luma, alpha), g in zip(seqs, outs):
            F, H, W = luma.shape
            o = O.estimate_sequence(O.OracleParams(W, H, 16, 2), luma, alpha, want_pred=True)
            assert np.array_equal(g["pred"].cpu().numpy(), o["pred"])
            per = ((luma[1:].astype(np.int64) - o["pred"]) ** 2).reshape(F - 1, H // 16, 16, W // 16, 16)
            assert np.array_equal(g["sse_mb"].cpu().numpy().astype(np.int64), per.sum(axis=(2, 4)).reshape(F - 1, -1))
        for o_ in outs:
            for v in o_.values():
                v.fill_(0x55) if v.dtype != torch.float32 else v.fill_(float("nan"))
    b.close()


def test_batch_set_config_rejects_bad_values(sme):
    seqs = _batch_inputs()[:2]
    b = sme.Batch([torch.from_numpy(l).cuda() for l, _ in seqs], [torch.from_numpy(a).cuda() for _, a in seqs])
    with pytest.raises(sme.SmeError):
        b.set_config("cluster")
    for bad in (4, 6):
        with pytest.raises(sme.SmeError):
            b.set_config("sparse", bad)
    with pytest.raises(sme.SmeError):
        b.set_config("pair", 17)
    b.close()


def _read_device(ptr, nbytes):
    """Bytes at a raw device address (the CUDA runtime's cudaMemcpy through
    ctypes; the library hands out addresses it owns, not tensors)."""
    import ctypes as C

    rt = None
    for name in ("/usr/local/cuda/lib64/libcudart.so", "libcudart.so"):
        try:
            rt = C.CDLL(name)
            break
        except OSError:
            pass
    if rt is None:
        pytest.skip("CUDA runtime library not found")
    out = np.empty(nbytes, np.uint8)
    torch.cuda.synchronize()
    assert rt.cudaMemcpy(C.c_void_p(out.ctypes.data), C.c_void_p(ptr), C.c_size_t(nbytes), 2) == 0
    return out


@pytest.mark.parametrize("schedule,param,flag", [("sparse", 2, 0), ("mb", 0, 1), ("pair", 8, 1)])
def test_batch_two_stage_run_and_class_maps(sme, schedule, param, flag):
    """Stage 1 then stage 2 equals a whole run; after stage 1 each sequence's
    class map [F, M] holds the oracle's class of every MB of every frame."""
    seqs = _batch_inputs()
    lumas = [torch.from_numpy(l).cuda() for l, _ in seqs]
    alphas = [torch.from_numpy(a).cuda() for _, a in seqs]
    b = sme.Batch(lumas, alphas, search_range=16, subpel=2)
    b.set_config(schedule, param, flag)
    b.run_stage(1)
    for i, (luma, alpha) in enumerate(seqs):
        F, H, W = luma.shape
        M = (W // 16) * (H // 16)
        got = _read_device(b.class_map_ptr(i), F * M).reshape(F, M)
        want = np.stack([O.classify_frame(alpha[f]) for f in range(F)])
        assert np.array_equal(got, want), i
    b.run_stage(2)
    b.synchronize()
    _check_all(b.outputs, seqs)
    b.close()


@pytest.mark.parametrize("pinned", [True, False])
def test_batch_host_upload_run_download(sme, pinned):
    """Host-to-host pass: the batch is created over empty device buffers,
    the inputs come from host memory (sme_batch_upload, a luma plane shared
    by the VOPs of one scene copied once), the results go back to host memory
    (sme_batch_download); they equal the oracle's."""
    seqs = _batch_inputs()
    dev_luma, lumas, alphas = {}, [], []
    for l, a in seqs:
        key = l.ctypes.data  # the VOPs of one scene share one luma array
        if key not in dev_luma:
            dev_luma[key] = torch.zeros(l.shape, dtype=torch.uint8, device="cuda")
        lumas.append(dev_luma[key])
        alphas.append(torch.zeros(a.shape, dtype=torch.uint8, device="cuda"))
    b = sme.Batch(lumas, alphas, search_range=16, subpel=2)
    b.set_config("sparse", 2, 0)
    pin = (lambda t: t.pin_memory()) if pinned else (lambda t: t)
    host_in = [(pin(torch.from_numpy(l)), pin(torch.from_numpy(a))) for l, a in seqs]
    host_out = [{"mv": pin(torch.zeros(tuple(o["mv"].shape), dtype=torch.int16)),
                 "sse": pin(torch.zeros(tuple(o["sse"].shape), dtype=torch.int64)),
                 "cost": pin(torch.zeros(tuple(o["cost"].shape), dtype=torch.int32))} for o in b.outputs]
    io = b.host_io(host_in, host_out)
    for _ in range(2):
        b.upload(io)
        b.run(sync=False)
        b.download(io)
        b.synchronize()
        for (luma, alpha), h in zip(seqs, host_out):
            F, H, W = luma.shape
            o = O.estimate_sequence(O.OracleParams(W, H, 16, 2), luma, alpha)
            assert np.array_equal(h["mv"].numpy(), o["mv"])
            assert np.array_equal(h["sse"].numpy().view(np.uint64), o["sse"])
            assert np.array_equal(h["cost"].numpy().view(np.uint32), o["cost"])
        for h in host_out:
            for v in h.values():
                v.zero_()
    # an output that was not requested at creation cannot be downloaded
    bad = b.host_io(host_in, [{"pred": torch.zeros(1, dtype=torch.uint8)} for _ in host_out])
    with pytest.raises(sme.SmeError):
        b.download(bad)
    b.close()


def test_batch_pair_rounds_match_oracle(sme):
    """Pair rounds: the whole run, and stage 1 followed by the rounds one by
    one, give the oracle's results; switching back gives them too; other
    schedules are refused while rounds are on."""
    seqs = _batch_inputs()
    lumas = [torch.from_numpy(l).cuda() for l, _ in seqs]
    alphas = [torch.from_numpy(a).cuda() for _, a in seqs]
    b = sme.Batch(lumas, alphas, search_range=16, subpel=2)
    b.set_pair_rounds(True)
    assert b.config()["schedule"] == "sparse"
    _check_all(b.run(), seqs)
    for o in b.outputs:
        for v in o.values():
            v.zero_()
    b.run_stage(1)
    rounds = max(l.shape[0] for l, _ in seqs) - 1
    for k in range(rounds):
        b.run_pair(k)
    b.synchronize()
    _check_all(b.outputs, seqs)
    with pytest.raises(sme.SmeError):
        b.run_pair(rounds)
    with pytest.raises(sme.SmeError):
        b.set_config("mb")
    b.tune(trials=1)
    assert b.config()["schedule"] == "sparse"
    _check_all(b.run(), seqs)
    b.set_pair_rounds(False)
    _check_all(b.run(), seqs)
    b.close()
