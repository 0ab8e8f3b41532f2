"""Benchmark of the shape-adaptive motion estimation pass on one GB300.

One step = the whole per-MB pass (classification, block recursive search,
pixel recursive search, motion compensation + SSE) over the largest
workload that fits one GPU: 16 synthetic sequences of 3840x2160, 60 frames,
8 video objects (VOPs) each -- 128 VOPs, 244.7 M macroblock estimates --
search range 32, half-pel, rendered on the device (inputs 72 GB, far above
L2).  `value` is the learned-seeded form (a seed network trained here on the
GPU, seeds as a fifth candidate with the plain search as fallback) in
macroblocks per second over all frame-grid MBs; the plain batched form is
timed beside it in the same line.  Both are one persistent batch replayed
from a CUDA graph.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

The same line carries: the device time of each stage and the roofline of the
dominant kernel; the end-to-end rate through the host-buffer calls
(sme_batch_upload / sme_batch_download); the CPU oracle on the first two
pairs of every VOP on all host cores, with the plain field checked against
it; sampled pairs of the learned field against the oracle given the same
seeds.  Secondary keys: the CIF 352x288 x 30-frame single sequence (cif30:
plain, end to end, exhaustive search, four vectors per MB, learned), the
64-sequence batch of uneven sizes (batched), the 1920x1088 x 300-frame,
4-VOP learned evaluation (hd_learned_eval) and the paper's QCIF setting
(paper_setup).

--impl reference times the CPU oracle on a bounded sample of the headline
workload (the first two pairs of every VOP), one VOP per host thread.
Under torchrun (N > 1) every rank runs an independent replica (its own
scenes); the data path has no collective, so scaling is weak.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "macroblocks/s (MV field matches oracle) learned-seeded vs plain; iters/MB; PSNR"
UNIT = "MB/s"
W, H, FRAMES, S, SUBPEL = 352, 288, 30, 16, 2
WORKLOAD = "CIF 352x288, 30 frames (29 pairs), 1 VOP, half-pel, S=16"
UHD_W, UHD_H, UHD_S = 3840, 2160, 32  # the headline workload's frame size and search range
OUT_FIELDS = ("cost", "disp", "iters", "npos", "mb_class", "sse")


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def max_over_ranks(x, dist, device="cuda"):
    """The largest value of x over all ranks (the job's time is its slowest
    replica's); x itself without a process group."""
    if dist is None:
        return x
    import torch

    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(units_per_rank, n_ranks, seconds):
    """Whole-job throughput of weakly scaled replicas: every rank processed
    units_per_rank in its own time; the job took the slowest one's."""
    return n_ranks * units_per_rank / seconds


def workload(rank=0):
    from paper_1002_1168_gb300 import synth

    return synth.cif_sequence(seed=1002 + rank, frames=FRAMES)


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""

    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []
        self._t = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.QUERY}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (FileNotFoundError, OSError):
            self.proc = None
            return
        self._t = threading.Thread(target=self._read, daemon=True)
        self._t.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        if self._t:
            self._t.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return d.get("hbm_gbs", 6800.0), "measured"
    return 6800.0, "fallback"


# DRAM bytes (read + write) of one me_kernel launch on this workload, from the
# ncu capture summarised in profiles/me_kernel_cif30_halfpel.md (set to None
# whenever the kernel changes until it is captured again).
ME_KERNEL_TRAFFIC_BYTES = 3510016 + 13568
# DRAM bytes of one sparse search launch of the headline's learned run: the
# ncu capture of the same build on one scene of the headline (20 frames,
# 115,920 searched MBs; 66.18 MB read + 3.59 MB written, the
# me_sparse_kernel profile summary) scaled by the searched MBs of the full
# run (5,544,264).
SEARCH_KERNEL_TRAFFIC_BYTES = int(round((66.178304e6 + 3.585536e6) * 5544264 / 115920))


def algorithmic_bytes(P, M, F):
    """Minimum DRAM bytes of one ME launch: every luma frame once (each frame
    is the current frame of one pair and the reference of the next), the packed
    alpha rows of every frame once, the class of every estimated MB, the
    requested per-MB outputs (mv 4, cost 4, disp 8, iters 1, npos 1, class 1
    bytes) and 8 bytes of SSE per pair."""
    wp = (W + 31) // 32 + 1
    return F * W * H + F * H * wp * 4 + P * M + P * M * 19 + P * 8


# Integer pipe of a GB300: 152 SMs x 128 32-bit integer lanes x 2.07 GHz
# (maximum SM clock), counting a packed 4-byte SIMD operation as one op.
ALU_PEAK_TOPS = 152 * 128 * 2.07e9 / 1e12


def algorithmic_int_ops(res):
    """Integer (and gradient FP32) operations the method needs for one pass,
    from its own counters: per evaluated texture position 64 packed words x 3
    ops (interpolate, absolute difference, accumulate); per pixel-recursive
    iteration 256 pixels x 5 ops (Eqs. 3-5); per evaluated shape position 16
    rows x 4 ops (XOR, popcount, shift, add); per MB the compensation and SSE,
    64 words x 3 ops."""
    cls, npos, iters = res["mb_class"], res["npos"].astype(np.int64), res["iters"].astype(np.int64)
    op, bd = cls == 1, cls == 2
    return int(192 * npos[op].sum() + 1280 * iters[op].sum() + 64 * npos[bd].sum() + 192 * cls.size)


def uhd_oracle_sample(seed=1005, n_seq=16, frames=60, keep=3):
    """The first `keep` frames of every sequence of the headline workload
    (the same scenes as synth_gpu.uhd_batch; only those frames are rendered,
    on the GPU when there is one): the bounded sample the CPU oracle runs."""
    import torch

    from paper_1002_1168_gb300 import synth_gpu

    dev = "cuda" if torch.cuda.is_available() else "cpu"
    out = []
    rng = np.random.default_rng(seed)
    for i in range(n_seq):
        luma, alpha, _ = synth_gpu.make_sequence_gpu(
            UHD_W, UHD_H, frames, seed * 1000 + i, n_objects=8, vmax=32.0, bg_step=tuple(rng.uniform(-4, 4, 2)),
            noise_sigma=2.0, change_every=20, max_rot_deg=3.0, scale_range=(1.0, 1.0), obj_frac=0.35, device=dev,
            render_frames=keep)
        out.append((luma.cpu().numpy(), alpha.cpu().numpy()))
    return out


def run_reference(args):
    """The reference arm: the CPU oracle (as it stands) on a bounded sample of
    the headline workload -- the first two frame pairs of every VOP of the
    16 x 3840x2160 x 60-frame batch, plain method -- one VOP per host thread."""
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    import oracle as O

    sample = uhd_oracle_sample(n_seq=args.scale_seqs, frames=args.scale_frames)
    p = O.OracleParams(UHD_W, UHD_H, UHD_S, 2)
    units = [(p, l, a[j], None) for l, a in sample for j in range(a.shape[0])]
    threads = os.cpu_count() or 1
    M = (UHD_W // 16) * (UHD_H // 16)
    mbs = len(units) * 2 * M
    for _ in range(args.warmup):
        oracle_units(units, threads)
    dt = 0.0
    for _ in range(args.steps):
        dt += oracle_units(units, threads)[1]
    v = mbs * args.steps / dt
    smp = (f"first 2 pairs of every VOP of the headline workload ({len(units)} VOPs, {mbs} MBs per step), "
           f"plain method, one VOP per thread on {threads} threads")
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u8+f32",
            "data": "synthetic",
            "config": {"workload": uhd_workload(args.scale_seqs, args.scale_frames), "mbs_per_step": mbs,
                       "sample": smp},
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": threads, "kind": "oracle", "sample": smp,
                             **host_cpu()},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def cpu_baseline(seq, budget_s=10.0):
    """The oracle as it stands, timed on this host's cores (single thread)."""
    import oracle as O

    p = O.OracleParams(W, H, S, SUBPEL)
    P = seq.luma.shape[0] - 1
    n, t0 = 0, time.perf_counter()
    res = None
    while True:
        res = O.estimate_sequence(p, seq.luma, seq.alpha[0])
        n += 1
        if time.perf_counter() - t0 >= budget_s:
            break
    dt = time.perf_counter() - t0
    return {"value": n * P * p.mbs / dt, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"{n} full passes over the workload ({n * P * p.mbs} MBs, {dt:.1f} s), single-threaded C"}, res


def train_seednet(sme, torch, args):
    """The learned proposal, trained here on the GPU by the library's own
    forward/backward kernels: args.learn_pairs CIF VOP frame pairs (1-2
    objects, rotation <= 5 deg, scale 0.95-1.05) labelled by the plain method,
    args.learn_steps Adam steps of 32 pairs."""
    from paper_1002_1168_gb300 import seedtrain, synth

    t0 = time.perf_counter()
    # three-frame sequences: each VOP gives a first pair (no previous field)
    # and a second one with the plain method's first field as network input
    pairs = seedtrain.training_pairs(args.learn_pairs, seed=11, workers=min(os.cpu_count() or 1, 16), frames=3)
    gen_s = time.perf_counter() - t0
    net = sme.SeedNet(max_cells=len(pairs) * (H // 4) * (W // 4))
    net.set_params(sme.pack_params(synth.seednet_init(3)))
    feats, labels, mask = seedtrain.build_dataset(pairs, net, search_range=S, subpel=SUBPEL)
    torch.cuda.synchronize()
    t1 = time.perf_counter()
    hist = seedtrain.train(net, feats, labels, mask, steps=args.learn_steps, batch=32, lr=1e-3, seed=0,
                           log_every=max(args.learn_steps // 4, 1))
    torch.cuda.synchronize()
    info = {"pairs": len(pairs), "labelled_mbs": int(mask.sum().item()), "steps": args.learn_steps, "batch": 32,
            "lr": 1e-3, "generation_s": gen_s, "train_s": time.perf_counter() - t1,
            "loss": [[st, round(float(l), 4)] for st, l in hist]}
    del feats, labels, mask
    return net, info


def measure_learned(sme, torch, args, net, est, luma, alpha, flush):
    """The learned-seeded pass on the headline workload, timed like the plain
    one (L2 flushed between steps): classification, features of all pairs,
    the sparse network forward near the object, estimation with the seeds as
    fifth candidate (plain search as fallback)."""
    P, M = FRAMES - 1, (W // 16) * (H // 16)
    dev = luma.device
    cls = torch.empty((FRAMES, M), dtype=torch.uint8, device=dev)
    feat = torch.empty((P, H // 4, W // 4, 16), dtype=torch.int16, device=dev)
    seeds = torch.empty((P, M, 2), dtype=torch.float32, device=dev)
    out = est._alloc_outputs(P, OUT_FIELDS, dev)

    def seed_pass():
        est.classify(alpha, want_packed=False, out=cls, sync=False)
        net.features(luma, 0, 1, subpel=SUBPEL, n_pairs=P, out=feat)
        net.forward_active(feat, cls[1:], out=seeds)

    def full_pass():
        seed_pass()
        est.estimate_sequence(luma, alpha, seed=seeds, out=out, sync=False)

    def timed(fn, steps):
        for _ in range(3):
            fn()
        est.synchronize()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        for i, (e0, e1) in enumerate(ev):
            flush.fill_(i & 0xff)
            e0.record()
            fn()
            e1.record()
        torch.cuda.synchronize()
        est.synchronize()
        return sum(e0.elapsed_time(e1) for e0, e1 in ev) / steps

    ms = timed(full_pass, args.steps)
    ms_seeds = timed(seed_pass, max(args.steps // 2, 5))
    ms_me = timed(lambda: est.estimate_sequence(luma, alpha, seed=seeds, out=out, sync=False),
                  max(args.steps // 2, 5))
    full_pass()
    est.synchronize()
    res = {k: v.cpu().numpy() for k, v in out.items()}
    return {"value": P * M / (ms / 1e3), "unit": UNIT, "ms_per_step": ms, "ms_seed_pass": ms_seeds,
            "ms_estimation_only": ms_me, "gpu_launches_per_step": 11}, res, seeds.cpu().numpy()


def learned_oracle_leg(seq, plain, learned, seeds, pairs_judged=(0, 9, 18, 27)):
    """Oracle leg of the learned measurement: the learned-seeded MV field
    against the oracle given the same seeds, and both fields measured
    against exhaustive search (the ES row of Table 1) on a sample of pairs:
    mean SAD above the ES optimum over the opaque MBs."""
    import oracle as O

    p = O.OracleParams(W, H, S, SUBPEL)
    orc = O.estimate_sequence(p, seq.luma, seq.alpha[0], seed=seeds)
    exact = all(np.array_equal(learned[a].view(np.uint8), orc[b].view(np.uint8)) for a, b in
                [("mv", "mv"), ("cost", "cost"), ("iters", "iters"), ("npos", "npos"), ("disp", "disp"),
                 ("mb_class", "mbclass"), ("sse", "sse")])
    gp, gl, n = 0, 0, 0
    for k in pairs_judged:
        _, es, _ = O.full_search(seq.luma[k], seq.luma[k + 1], W, H, SUBPEL, S)
        op = plain["mb_class"][k] == 1
        gp += int((plain["cost"][k].view(np.uint32)[op].astype(np.int64) - es[op]).sum())
        gl += int((learned["cost"][k].view(np.uint32)[op].astype(np.int64) - es[op]).sum())
        n += int(op.sum())
    return exact, {"pairs": list(pairs_judged), "opaque_mbs": n, "mean_sad_above_es_plain": gp / max(n, 1),
                   "mean_sad_above_es_learned": gl / max(n, 1)}


def stats(res, width, height):
    """iters/opaque MB, positions/non-transparent MB, mean PSNR (dB) of one output set."""
    from paper_1002_1168_gb300 import sme

    cls = res["mb_class"]
    return {"iters_per_opaque_mb": float(res["iters"][cls == 1].mean()),
            "positions_per_mb": float(res["npos"][cls > 0].mean()),
            "psnr_db_mean": float(np.mean([sme.psnr(int(x), width, height) for x in res["sse"].view(np.uint64)]))}


def batch_quality(outputs, host):
    """iters/opaque MB, positions/non-transparent MB and mean PSNR over every
    pair of every VOP of a batch."""
    from paper_1002_1168_gb300 import sme

    it, itn, pos, posn, ps = 0, 0, 0, 0, []
    for o_, (sq, _) in zip(outputs, host):
        cls = o_["mb_class"]
        it += int(o_["iters"][cls == 1].sum().item())
        itn += int((cls == 1).sum().item())
        pos += int(o_["npos"][cls > 0].sum().item())
        posn += int((cls > 0).sum().item())
        ps += [sme.psnr(int(x), sq.width, sq.height) for x in o_["sse"].cpu().numpy().view(np.uint64)]
    return {"iters_per_opaque_mb": it / max(itn, 1), "positions_per_mb": pos / max(posn, 1),
            "psnr_db_mean": float(np.mean(ps))}


def measure_batch(sme, torch, args, rank, dist, net=None):
    """Secondary measurement: 64 sequences of uneven size (16 QCIF, 24 CIF,
    16 4CIF, 8 1920x1088), 10 frames, 1-4 objects each (one VOP per object),
    |v| <= 16, S=16, half-pel, estimated in one persistent launch replayed
    from a CUDA graph.  Inputs (0.9 GB) exceed L2, so no flush is needed."""
    import oracle as O
    from paper_1002_1168_gb300 import synth

    t0 = time.perf_counter()
    sizes = {"full": None, "hd8": [(1920, 1088)] * 8}[args.batch_preset]
    seqs = synth.batch_sequences(seed=1003 + 100 * rank, frames=10, sizes=sizes)
    gen_s = time.perf_counter() - t0
    lumas, alphas, host, groups = [], [], [], []
    for sq in seqs:
        lt = torch.from_numpy(sq.luma).cuda()
        vops = []
        for j in range(sq.alpha.shape[0]):
            vops.append(torch.from_numpy(sq.alpha[j]).cuda())
            lumas.append(lt)
            alphas.append(vops[-1])
            host.append((sq, j))
        groups.append((lt, vops))  # VOP order = host order
    b = sme.Batch(lumas, alphas, search_range=16, subpel=2, want=("cost", "iters", "npos", "mb_class", "sse"))
    b.tune(trials=3)
    cfg = b.config()
    total = sum((l.shape[0] - 1) * (l.shape[1] // 16) * (l.shape[2] // 16) for l in lumas)
    steps = max(3, args.steps // 5)
    for _ in range(2):
        b.run(sync=False)
    b.synchronize()
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    for i in range(steps):
        starts[i].record()
        b.run(sync=False)
        ends[i].record()
    torch.cuda.synchronize()
    b.synchronize()
    ms = sum(s_.elapsed_time(e_) for s_, e_ in zip(starts, ends)) / steps
    ms = max_over_ranks(ms, dist)
    ws = dist.get_world_size() if dist else 1
    # parity on a sample of VOP sequences (every 7th, all frame sizes), about
    # args.cpu_seconds of oracle time; the CPU baseline is that same sample
    exact, cpu_mbs, cpu_s, sample = True, 0, 0.0, []
    for i in list(range(0, len(host), 7)) + list(range(1, len(host), 7)):
        if cpu_s >= args.cpu_seconds:
            break
        sq, j = host[i]
        tc = time.perf_counter()
        o = O.estimate_sequence(O.OracleParams(sq.width, sq.height, 16, 2), sq.luma, sq.alpha[j])
        cpu_s += time.perf_counter() - tc
        cpu_mbs += o["mv"].shape[0] * o["mv"].shape[1]
        sample.append(i)
        g = b.outputs[i]
        exact &= bool(np.array_equal(g["mv"].cpu().numpy(), o["mv"]) and
                      np.array_equal(g["sse"].cpu().numpy().view(np.uint64), o["sse"]) and
                      np.array_equal(g["cost"].cpu().numpy().view(np.uint32), o["cost"]))
    nt = sum(int((o_["mb_class"] > 0).sum().item()) for o_ in b.outputs)
    plain_q = batch_quality(b.outputs, host)
    b.close()
    learned = None
    if net is not None:
        from paper_1002_1168_gb300 import seedtrain

        lb = seedtrain.LearnedBatch(net, groups, search_range=16, subpel=2)
        lb.tune(trials=3)
        for _ in range(2):
            lb.run(sync=False)
        lb.synchronize()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        if dist:
            dist.barrier()
        torch.cuda.synchronize()
        for e0, e1 in ev:
            e0.record(lb.stream)
            lb.run(sync=False)
            e1.record(lb.stream)
        torch.cuda.synchronize()
        lb.synchronize()
        lms = sum(e0.elapsed_time(e1) for e0, e1 in ev) / steps
        lms = max_over_ranks(lms, dist)
        lq = batch_quality(lb.outputs, host)
        lexact, lsample, lcpu = True, [], 0.0
        for i in sample:  # the oracle, given the same seeds, on the plain parity sample
            if lcpu >= args.cpu_seconds / 2:
                break
            sq, j = host[i]
            tc = time.perf_counter()
            o = O.estimate_sequence(O.OracleParams(sq.width, sq.height, 16, 2), sq.luma, sq.alpha[j],
                                    seed=lb.seeds[i].cpu().numpy())
            lcpu += time.perf_counter() - tc
            lsample.append(i)
            g = lb.outputs[i]
            lexact &= bool(np.array_equal(g["mv"].cpu().numpy(), o["mv"]) and
                           np.array_equal(g["sse"].cpu().numpy().view(np.uint64), o["sse"]) and
                           np.array_equal(g["cost"].cpu().numpy().view(np.uint32), o["cost"]))
        learned = {"value": job_rate(total, ws, lms / 1e3), "unit": UNIT, "ms_per_run": lms, "config": lb.config(),
                   "vs_plain_batched": ms / lms, **lq, "psnr_delta_db": lq["psnr_db_mean"] - plain_q["psnr_db_mean"],
                   "bit_exact_vs_oracle_sample": lexact, "sample_sequences": len(lsample),
                   "network": "classes + features + sparse forward per sequence, one CUDA graph"}
        lb.close()
    name = {"full": "64 sequences (16 QCIF, 24 CIF, 16 4CIF, 8 1920x1088)",
            "hd8": "8 sequences of 1920x1088"}[args.batch_preset]
    return {"workload": f"{name}, 10 frames, {len(lumas)} VOPs, half-pel, S=16", "mb_per_run": total,
            "value": job_rate(total, ws, ms / 1e3), "unit": UNIT, "ms_per_run": ms, "runs": steps,
            "non_transparent_frac": nt / total, "config": cfg, "generation_s": gen_s, **plain_q,
            "learned_seeded": learned,
            "bit_exact_vs_oracle_sample": exact, "sample_sequences": len(sample),
            "cpu_baseline": {"value": cpu_mbs / cpu_s, "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": f"{len(sample)} of the batch's VOP sequences (every 7th), "
                                       f"{cpu_mbs} MBs, {cpu_s:.1f} s, single-threaded C"}}


def _device_quality(outputs, W, H):
    """iters/opaque MB, positions/non-transparent MB, mean PSNR over every pair
    of every VOP, reduced on the device (the fields are too large to copy)."""
    import torch

    from paper_1002_1168_gb300 import sme

    it = itn = pos = posn = 0
    ps = []
    for o in outputs:
        op, nt = o["mb_class"] == 1, o["mb_class"] > 0
        it += int(o["iters"][op].sum(dtype=torch.int64))
        itn += int(op.sum())
        pos += int(o["npos"][nt].sum(dtype=torch.int64))
        posn += int(nt.sum())
        ps += [sme.psnr(int(x), W, H) for x in o["sse"].cpu().numpy().view(np.uint64)]
    return {"iters_per_opaque_mb": it / max(itn, 1), "positions_per_mb": pos / max(posn, 1),
            "psnr_db_mean": float(np.mean(ps)), "non_transparent_frac": posn / sum(o["mb_class"].numel() for o in outputs)}


def es_psnr_like_method(sme, est, luma, mv_es, cls, rd, W_, H_):
    """Mean PSNR of the exhaustive-search field with the transparent MBs at
    (0,0), as Fig. 1 leaves them: the comparison with the method on the same
    MBs (the method does not estimate the background outside its VOP)."""
    import torch

    mv = mv_es.clone()
    mv[torch.from_numpy(cls == 0).to(mv.device)] = 0
    return float(np.mean([sme.psnr(est.compensate(luma[k], luma[k + rd], mv[k].contiguous(), want_pred=False)[0],
                                   W_, H_) for k in range(mv.shape[0])]))


def measure_es(sme, torch, est, luma, flush, steps):
    """The exhaustive search on the headline workload (the ES of Table 1,
    the comparison method of Table 2): its time, positions per MB, the PSNR
    of its field and the integer-pipe roofline of its kernel.  Returns the
    record and the fields (for the oracle leg)."""
    P = FRAMES - 1
    for _ in range(3):
        est.full_search(luma, sync=False)
    est.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    for i, (e0, e1) in enumerate(ev):
        flush.fill_(i & 0xff)
        e0.record()
        est.full_search(luma, sync=False)
        e1.record()
    torch.cuda.synchronize()
    est.synchronize()
    ms = sum(e0.elapsed_time(e1) for e0, e1 in ev) / steps
    mv, sad = est.full_search(luma)
    psnr = []
    for k in range(P):
        sse, _ = est.compensate(luma[k], luma[k + 1], mv[k].contiguous(), want_pred=False)
        psnr.append(sme.psnr(sse, W, H))
    # |V| per MB (Table 1's ES count at 16 x 16, half-pel)
    npos = 0
    for v in range(H // 16):
        for u in range(W // 16):
            lox, hix = max(-S * SUBPEL, -16 * u * SUBPEL), min(S * SUBPEL, (W - 16 - 16 * u) * SUBPEL)
            loy, hiy = max(-S * SUBPEL, -16 * v * SUBPEL), min(S * SUBPEL, (H - 16 - 16 * v) * SUBPEL)
            npos += (hix - lox + 1) * (hiy - loy + 1)
    M = (W // 16) * (H // 16)
    ops = P * npos * 16 * 4 * 3  # per position and row: 4 words x (align, absolute difference, add)
    rec = {"mb_per_s": P * M / (ms / 1e3), "ms_per_step": ms, "positions_per_mb": npos / M,
           "psnr_db_mean": float(np.mean(psnr)),
           "roofline": {"bound": "alu", "kernel": "es_kernel", "achieved_tops": ops / (ms / 1e3) / 1e12,
                        "peak_tops": ALU_PEAK_TOPS, "frac": ops / (ms / 1e3) / 1e12 / ALU_PEAK_TOPS,
                        "ops_per_launch": ops}}
    return rec, mv, sad.cpu().numpy().view(np.uint32)


def measure_four_mv(sme, torch, seq, luma, alpha, flush, steps):
    """Four vectors per MB (Sec. 3.2, the recursive search on 8x8 blocks) on
    the headline workload: time of the whole pass (autotuned warps per CTA,
    L2 flushed between runs), PSNR of the block-wise compensation, PRS steps
    and distinct positions per 8x8 block, and the whole field checked against
    the oracle."""
    import oracle as O

    P = FRAMES - 1
    est4 = sme.Estimator(W, H, search_range=S, subpel=SUBPEL, four_mv=True)
    want = ("cost", "disp", "iters", "npos", "mb_class", "sse")
    out = est4._alloc_outputs(P, want, luma.device)
    est4.autotune(luma, alpha, out=out, trials=2, want=want)
    for _ in range(3):
        est4.estimate_sequence(luma, alpha, out=out, sync=False)
    est4.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    for i, (e0, e1) in enumerate(ev):
        flush.fill_(i & 0xff)
        e0.record()
        est4.estimate_sequence(luma, alpha, out=out, sync=False)
        e1.record()
    torch.cuda.synchronize()
    est4.synchronize()
    ms = sum(e0.elapsed_time(e1) for e0, e1 in ev) / steps
    cfg = est4.config()
    g = {k: v.cpu().numpy() for k, v in out.items()}
    est4.close()
    o = O.estimate_sequence4(O.OracleParams(W, H, S, SUBPEL), seq.luma, seq.alpha[0])
    exact = all(np.array_equal(g[a_].view(np.uint8), o[b_].view(np.uint8)) for a_, b_ in
                [("mv", "mv"), ("cost", "cost"), ("iters", "iters"), ("npos", "npos"), ("mb_class", "mbclass"),
                 ("sse", "sse"), ("disp", "disp")])
    cls = g["mb_class"]
    M = (W // 16) * (H // 16)
    return {"mb_per_s": P * M / (ms / 1e3), "ms_per_step": ms,
            "config": {"schedule": cfg["schedule"], "pair_warps": cfg["pair_warps"]},
            "psnr_db_mean": float(np.mean([sme.psnr(int(x), W, H) for x in g["sse"].view(np.uint64)])),
            "iters_per_opaque_block": float(g["iters"][cls == 1].mean()),
            "positions_per_block": float(g["npos"][cls > 0].mean()),
            "bit_exact_vs_oracle": bool(exact)}


def measure_paper_setup(sme, torch):
    """The paper's own experimental setting, on a synthetic stand-in (the
    QCIF test sequences of Sec. 4 are not available): QCIF 176x144, 30
    frames, reference two frames back (ref_distance 2), 16x16 MBs, half-pel,
    search range 7 (the window of Table 1's exhaustive-search count).  Reports
    the method's distinct search points per block against the exhaustive
    search's (Table 1) and both PSNRs (Table 2), with the whole field checked
    against the oracle and the ES field against the oracle's ES."""
    import oracle as O
    from paper_1002_1168_gb300 import synth

    Wq, Hq, Sq, rd, Fq = 176, 144, 7, 2, 30
    seq = synth.make_sequence(Wq, Hq, Fq, seed=1006, n_objects=1, vmax=3.0, bg_step=(0.75, -0.25), noise_sigma=2.0,
                              obj_frac=0.45)
    est = sme.Estimator(Wq, Hq, search_range=Sq, subpel=2, ref_distance=rd)
    luma = torch.from_numpy(seq.luma).cuda()
    g = est.estimate_sequence(luma, torch.from_numpy(seq.alpha[0]).cuda())
    g = {k: v.cpu().numpy() for k, v in g.items()}
    mv_es, sad_es = est.full_search(luma)
    P = Fq - rd
    psnr_es = [sme.psnr(est.compensate(luma[k], luma[k + rd], mv_es[k].contiguous(), want_pred=False)[0], Wq, Hq)
               for k in range(P)]
    o = O.estimate_sequence(O.OracleParams(Wq, Hq, Sq, 2), seq.luma, seq.alpha[0], ref_distance=rd)
    exact = all(np.array_equal(g[a_].view(np.uint8), o[b_].view(np.uint8)) for a_, b_ in
                [("mv", "mv"), ("cost", "cost"), ("iters", "iters"), ("npos", "npos"), ("mb_class", "mbclass"),
                 ("sse", "sse")])
    es_ok = True
    for k in (0, P - 1):
        bm, bs, _ = O.full_search(seq.luma[k], seq.luma[k + rd], Wq, Hq, 2, Sq)
        es_ok &= bool(np.array_equal(mv_es[k].cpu().numpy(), bm) and
                      np.array_equal(sad_es[k].cpu().numpy().view(np.uint32), bs))
    _, _, es_total = O.full_search(None, None, Wq, Hq, 2, Sq)
    cls = g["mb_class"]
    psnr_es_vop = es_psnr_like_method(sme, est, luma, mv_es, cls, rd, Wq, Hq)
    est.close()
    # four vectors per MB: the 8x8-block form of Table 1's search-point count
    est4 = sme.Estimator(Wq, Hq, search_range=Sq, subpel=2, ref_distance=rd, four_mv=True)
    g4 = est4.estimate_sequence(luma, torch.from_numpy(seq.alpha[0]).cuda())
    g4 = {k: v.cpu().numpy() for k, v in g4.items()}
    est4.close()
    o4 = O.estimate_sequence4(O.OracleParams(Wq, Hq, Sq, 2), seq.luma, seq.alpha[0], ref_distance=rd)
    exact4 = all(np.array_equal(g4[a_].view(np.uint8), o4[b_].view(np.uint8)) for a_, b_ in
                 [("mv", "mv"), ("cost", "cost"), ("iters", "iters"), ("npos", "npos"), ("sse", "sse")])
    _, _, es8_total = O.full_search(None, None, Wq, Hq, 2, Sq, block=8)
    _, _, es8_full = O.full_search(None, None, Wq, Hq, 1, Sq, block=8)
    four_mv = {"search_points_per_8x8_block": {"method": float(g4["npos"][g4["mb_class"] > 0].mean()),
                                                "es_halfpel": es8_total / 396, "es_fullpel": es8_full / 396,
                                                "paper_table1_pa": "6.43-6.51", "paper_table1_es": 204.2828},
               "psnr_db": float(np.mean([sme.psnr(int(x), Wq, Hq) for x in g4["sse"].view(np.uint64)])),
               "iters_per_opaque_block": float(g4["iters"][g4["mb_class"] == 1].mean()),
               "bit_exact_vs_oracle": bool(exact4)}
    psnr_pa = [sme.psnr(int(x), Wq, Hq) for x in g["sse"].view(np.uint64)]
    return {"workload": "QCIF 176x144, 30 frames, ref_distance 2, 16x16, half-pel, S=7, 1 VOP",
            "search_points_per_mb": {"method": float(g["npos"][cls > 0].mean()), "es": es_total / 99,
                                     "paper_table1_pa_qcif_8x8": "6.43-6.51", "paper_table1_es_8x8_fullpel": 204.2828},
            "psnr_db": {"method": float(np.mean(psnr_pa)), "es": float(np.mean(psnr_es)),
                        "es_transparent_at_zero": psnr_es_vop,
                        "paper_table2_pa_minus_es": "-0.03 to -0.88 (real QCIF sequences, 8x8)"},
            "iters_per_opaque_mb": float(g["iters"][cls == 1].mean()),
            "bit_exact_vs_oracle": bool(exact), "es_bit_exact_vs_oracle_sample": es_ok, "four_mv": four_mv}


def uhd_workload(n_seq, frames):
    return (f"{n_seq} sequences of 3840x2160, {frames} frames, 8 VOPs each ({8 * n_seq} VOPs), |v| <= 32 px, "
            "rotation <= 3 deg, S=32, half-pel, rendered on the device")


def stage_times(torch, run_stage, seed_pass, stream, steps):
    """Device time of each stage of a run (events on the run's stream):
    stage 1 (classification: the sparse schedule's streaming pass, count,
    scan, scatter), the seed pass (learned form), stage 2 (the search: one
    me_sparse_kernel launch).  Returns the mean ms of each."""
    ev = [[torch.cuda.Event(enable_timing=True) for _ in range(4)] for _ in range(steps)]
    with torch.cuda.stream(stream):
        for e in ev:
            e[0].record(stream)
            run_stage(1)
            e[1].record(stream)
            if seed_pass:
                seed_pass()
            e[2].record(stream)
            run_stage(2)
            e[3].record(stream)
    torch.cuda.synchronize()
    return tuple(sum(e[i].elapsed_time(e[i + 1]) for e in ev) / steps for i in range(3))


def _int_ops_device(torch, outputs):
    """Algorithmic integer operations of a run from the method's own counters
    (see algorithmic_int_ops), summed on the device."""
    tot = 0
    for o in outputs:
        cls, npos, it = o["mb_class"], o["npos"].to(torch.int64), o["iters"].to(torch.int64)
        op, bd = cls == 1, cls == 2
        tot += int(192 * npos[op].sum() + 1280 * it[op].sum() + 64 * npos[bd].sum() + 192 * cls.numel())
    return tot


def uhd_alg_bytes(n_vops, n_luma, F, total_mbs, transparent_mbs=None):
    """Algorithmic DRAM bytes of one run: every VOP's u8 alpha plane once,
    every distinct luma plane once (the VOPs of a scene share it), 19 output
    bytes per MB (vector 4, cost 4, update 8, steps, positions, class) and 8
    per pair of each VOP.  With transparent_mbs: the streaming pass's share
    (alpha, luma, the transparent MBs' outputs)."""
    fs = UHD_W * UHD_H
    inputs = n_vops * F * fs + n_luma * F * fs
    mbs = total_mbs if transparent_mbs is None else transparent_mbs
    return inputs + 19 * mbs + 8 * n_vops * (F - 1)


def oracle_units(units, threads):
    """The oracle on independent (params, luma, alpha, seed) units on `threads`
    host threads (the C library releases the GIL), with the wall time."""
    import oracle as O
    from concurrent.futures import ThreadPoolExecutor

    def one(u):
        p, l, a, sd = u
        return O.estimate_sequence(p, l, a, seed=sd)

    t0 = time.perf_counter()
    with ThreadPoolExecutor(threads) as ex:
        res = list(ex.map(one, units))
    return res, time.perf_counter() - t0


def host_cpu():
    model = ""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for ln in out.splitlines():
            if ln.lower().startswith("model name"):
                model = ln.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    return {"nproc": os.cpu_count(), "cpu_model": model}


def sized_net(sme, net, max_cells):
    """A network with net's trained parameters and room for max_cells cells."""
    big = sme.SeedNet(max_cells=max_cells)
    big.set_params(net.get_params())
    return big


def measure_headline(sme, torch, args, net, dist, rank):
    """The headline: learned proposal + batching at scale, 16 sequences of
    3840x2160, 60 frames, 8 VOPs each (|v| <= 32 px, rotation <= 3 deg),
    S = 32, half-pel, rendered on the device (inputs 72 GB: far above L2).
    The plain batch and the learned batch (the network trained in this run)
    are both autotuned and replayed from CUDA graphs; `steps` timed runs of
    each.  Also: device time per stage, end to end through the host-buffer
    calls, the oracle on the first two pairs of every VOP on the host's
    cores (with the plain field checked against it) and on sampled pairs of
    the learned field given the same seeds."""
    import gc

    import oracle as O
    from paper_1002_1168_gb300 import seedtrain, synth_gpu

    ws = dist.get_world_size() if dist else 1
    t0 = time.perf_counter()
    seqs = synth_gpu.uhd_batch(seed=1005 + 100 * rank, n_seq=args.scale_seqs, frames=args.scale_frames)
    torch.cuda.synchronize()
    gen_s = time.perf_counter() - t0
    F = seqs[0][0].shape[0]
    P, M = F - 1, (UHD_W // 16) * (UHD_H // 16)
    groups = [(l, [a[j] for j in range(a.shape[0])]) for l, a, _ in seqs]
    lumas = [l for l, vops in groups for _ in vops]
    alphas = [a for _, vops in groups for a in vops]
    n_vops, n_seq = len(alphas), len(seqs)
    total = n_vops * P * M
    want = ("cost", "disp", "iters", "npos", "mb_class", "sse")
    steps = max(args.steps, 3)
    warm = max(args.warmup, 3)

    def timed(run, stream, clocks=None):
        for _ in range(warm):
            run()
        torch.cuda.synchronize()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        if dist:
            dist.barrier()
        torch.cuda.synchronize()
        if clocks:
            clocks.start()
            time.sleep(0.3)
        w0 = time.perf_counter()
        for e0, e1 in ev:
            e0.record(stream)
            run()
            e1.record(stream)
        torch.cuda.synchronize()
        wall = time.perf_counter() - w0
        clk = clocks.stop() if clocks else None
        ms = sum(e0.elapsed_time(e1) for e0, e1 in ev) / steps
        return max_over_ranks(ms, dist), wall, clk

    # ---- plain batch
    b = sme.Batch(lumas, alphas, search_range=UHD_S, subpel=2, want=want)
    b.tune(trials=2)
    pstream = torch.cuda.current_stream()
    clocks = ClockSampler(int(os.environ.get("LOCAL_RANK", "0")))
    ms_plain, wall, clk = timed(lambda: b.run(sync=False), pstream, clocks if net is None else None)
    b.synchronize()
    plain_cfg = b.config()
    b.set_config(plain_cfg["schedule"], plain_cfg["param"], plain_cfg["flag"])  # direct launches, same configuration
    st_plain = stage_times(torch, b.run_stage, None, pstream, max(3, steps // 4))
    b.synchronize()
    plain_q = _device_quality(b.outputs, UHD_W, UHD_H)
    plain_ops = _int_ops_device(torch, b.outputs)
    transparent = sum(int((o["mb_class"] == 0).sum()) for o in b.outputs)
    # the plain fields of pairs 0, 1 of every VOP, for the oracle leg below
    plain01 = [{k: o[k][:2].cpu().numpy() for k in ("mv", "cost", "sse")} for o in b.outputs]
    if net is not None:
        b.close()
        del b
        gc.collect()
        torch.cuda.empty_cache()

    # ---- the oracle on sampled pairs of a learned field, given the GPU's
    # previous field and the same seeds
    samples = [(min(7, n_seq - 1), 3, min(30, F - 2)), (0, 0, 1), (n_seq - 1, 7, F - 2)]

    def oracle_pairs(outputs, seeds):
        ok = True
        for s_, j_, k_ in samples:
            q = 8 * s_ + j_
            out = outputs[q]
            luma, alpha, _ = seqs[s_]
            tmp = None if k_ == 0 else out["mv"][k_ - 1].cpu().numpy()
            o = O.estimate_sequence(O.OracleParams(UHD_W, UHD_H, UHD_S, 2), luma[k_:k_ + 2].cpu().numpy(),
                                    alpha[j_, k_:k_ + 2].cpu().numpy(), temporal_in=tmp,
                                    seed=seeds[q][k_:k_ + 1].cpu().numpy())
            ok &= bool(np.array_equal(out["mv"][k_].cpu().numpy(), o["mv"][0]) and
                       np.array_equal(out["cost"][k_].cpu().numpy().view(np.uint32), o["cost"][0]) and
                       np.array_equal(out["iters"][k_].cpu().numpy(), o["iters"][0]) and
                       int(out["sse"][k_].item()) == int(o["sse"][0]))
        return ok

    # ---- learned, pair rounds: the previous pair's field as network input
    rounds = None
    if net is not None and not args.no_rounds:
        rnet = sized_net(sme, net, n_seq * (UHD_H // 4) * (UHD_W // 4))
        lr = seedtrain.LearnedRounds(rnet, groups, search_range=UHD_S, subpel=2, want=want)
        lr.tune(trials=1)
        ms_r, _, _ = timed(lambda: lr.run(sync=False), lr.stream)
        lr.synchronize()
        rq = _device_quality(lr.outputs, UHD_W, UHD_H)
        rounds = {"value": job_rate(total, ws, ms_r / 1e3), "unit": UNIT, "ms_per_run": ms_r,
                  "config": lr.config(), **rq, "psnr_delta_db": rq["psnr_db_mean"] - plain_q["psnr_db_mean"],
                  "iters_delta_pct": 100.0 * (rq["iters_per_opaque_mb"] / plain_q["iters_per_opaque_mb"] - 1.0),
                  "vs_plain_batched": ms_plain / ms_r,
                  "bit_exact_vs_oracle_sample": oracle_pairs(lr.outputs, lr.seeds),
                  "form": "pair rounds: the network of pair k sees the final field of pair k-1",
                  "launches_per_run": 5 + lr.rounds * (1 + 7 + 1) - 1}
        lr.close()
        rnet.close()
        del lr
        gc.collect()
        torch.cuda.empty_cache()

    # ---- learned batch (the headline; the plain batch when no network is trained)
    if net is not None:
        net = sized_net(sme, net, P * (UHD_H // 4) * (UHD_W // 4))
        lb = seedtrain.LearnedBatch(net, groups, search_range=UHD_S, subpel=2, want=want)
        lb.tune(trials=2)
        ms_learned, wall, clk = timed(lambda: lb.run(sync=False), lb.stream, clocks)
        lb.synchronize()
        learned_cfg = lb.config()
        n_chunks = len(lb.chunks)
        st_learned = stage_times(torch, lb.batch.run_stage, lb._seed_pass, lb.stream, max(3, steps // 4))
        lb.synchronize()
        lq = _device_quality(lb.outputs, UHD_W, UHD_H)
        learned_ops = _int_ops_device(torch, lb.outputs)
        head_batch, head_runner = lb.batch, lb
    else:
        lb = None
        ms_learned, learned_cfg, n_chunks, st_learned = ms_plain, plain_cfg, 0, st_plain
        lq, learned_ops = plain_q, plain_ops
        head_batch, head_runner = b, b

    lexact = oracle_pairs(lb.outputs, lb.seeds) if lb is not None else True

    # ---- end to end through the host-buffer calls (pinned host memory)
    e2e = None
    if not args.no_e2e:
        host_in, host_out = [], []
        luma_host = {}
        for l, a in zip(lumas, alphas):
            if l.data_ptr() not in luma_host:
                luma_host[l.data_ptr()] = l.cpu().pin_memory()
            host_in.append((luma_host[l.data_ptr()], a.cpu().pin_memory()))
        for o in head_batch.outputs:
            host_out.append({"mv": torch.empty(tuple(o["mv"].shape), dtype=torch.int16).pin_memory(),
                             "sse": torch.empty(tuple(o["sse"].shape), dtype=torch.int64).pin_memory()})
        io = head_batch.host_io(host_in, host_out)
        head_runner.run_host(io)
        e2e_steps = 3
        if dist:
            dist.barrier()
        t1 = time.perf_counter()
        for _ in range(e2e_steps):
            head_runner.run_host(io)
        e2e_s = max_over_ranks((time.perf_counter() - t1) / e2e_steps, dist)
        h2d = sum(t.numel() for t in luma_host.values()) + sum(a.numel() for _, a in host_in)
        d2h = sum(v.numel() * v.element_size() for h in host_out for v in h.values())
        e2e_exact = all(torch.equal(h["mv"], o["mv"].cpu()) for h, o in zip(host_out[:8], head_batch.outputs[:8]))
        e2e = {"value": job_rate(total, ws, e2e_s), "unit": UNIT, "h2d_bytes_per_step": int(h2d),
               "d2h_bytes_per_step": int(d2h), "s_per_step": e2e_s, "steps": e2e_steps,
               "api": "sme_batch_upload -> run (one CUDA graph) -> sme_batch_download, pinned host buffers",
               "mv_equals_device_run": bool(e2e_exact)}
        del host_in, host_out, luma_host, io
        gc.collect()

    # ---- CPU oracle on the first two pairs of every VOP (plain method), all host cores
    cpu = None
    if rank == 0:
        units, refs = [], []
        for s_, (l, a, _) in enumerate(seqs):
            l3 = l[:3].cpu().numpy()
            for j in range(a.shape[0]):
                units.append((O.OracleParams(UHD_W, UHD_H, UHD_S, 2), l3, a[j, :3].cpu().numpy(), None))
                refs.append(plain01[8 * s_ + j])
        threads = os.cpu_count() or 1
        res, dt = oracle_units(units, threads)
        mbs = len(units) * 2 * M
        exact = all(np.array_equal(r["mv"], g["mv"]) and np.array_equal(r["cost"], g["cost"].view(np.uint32)) and
                    np.array_equal(r["sse"], g["sse"].view(np.uint64)) for r, g in zip(res, refs))
        _, dt1 = oracle_units(units[:4], 1)
        cpu = {"value": mbs / dt, "unit": UNIT, "cores": threads, "kind": "oracle",
               "sample": f"first 2 pairs of every VOP sequence ({len(units)} VOPs, {mbs} MBs), {dt:.1f} s on "
                         f"{threads} threads (C oracle, one VOP per thread)",
               "single_thread_value": 4 * 2 * M / dt1, **host_cpu(),
               "plain_field_bit_exact_vs_oracle": bool(exact)}
    head_runner.close()
    if net is not None:
        net.close()
    del lb, head_batch, head_runner, seqs, groups, lumas, alphas
    gc.collect()
    torch.cuda.empty_cache()
    hbm, peak_kind = peaks()
    alg_run = uhd_alg_bytes(n_vops, n_seq, F, total)
    alg_stream = uhd_alg_bytes(n_vops, n_seq, F, total, transparent)
    return {
        "ms_learned": ms_learned, "ms_plain": ms_plain, "wall_s_timed": wall, "clocks": clk, "steps": steps,
        "warmup": warm, "total_mbs": total, "generation_s": gen_s, "n_seq": n_seq, "frames": F,
        "workload": uhd_workload(n_seq, F),
        "plain": {"value": job_rate(total, ws, ms_plain / 1e3), "unit": UNIT, "ms_per_run": ms_plain,
                  "config": plain_cfg, **plain_q,
                  "stage_ms": {"classify_stream": st_plain[0], "search": st_plain[2]},
                  "bit_exact_vs_oracle_sample": cpu["plain_field_bit_exact_vs_oracle"] if cpu else None},
        "learned_rounds": rounds,
        "learned": {"value": job_rate(total, ws, ms_learned / 1e3), "ms_per_run": ms_learned, "config": learned_cfg,
                    **lq, "psnr_delta_db": lq["psnr_db_mean"] - plain_q["psnr_db_mean"],
                    "vs_plain_batched": ms_plain / ms_learned,
                    "stage_ms": {"classify_stream": st_learned[0], "seed_network": st_learned[1],
                                 "search": st_learned[2]},
                    "bit_exact_vs_oracle_sample": lexact, "oracle_samples": samples},
        "launches_per_run": {"sparse": 6 + 7 * n_chunks, "mb": 2 + 7 * n_chunks, "pair": 2 + 7 * n_chunks}.get(
            learned_cfg["schedule"], 2 + 7 * n_chunks),
        "roofline_search": {"bound": "alu", "kernel": {"sparse": "me_sparse_kernel", "mb": "me_kernel",
                                                        "pair": "me_pair_kernel"}.get(learned_cfg["schedule"]),
                            "achieved": learned_ops / (st_learned[2] / 1e3) / 1e12,
                            "peak": ALU_PEAK_TOPS, "unit": "Tops/s", "frac": learned_ops / (st_learned[2] / 1e3) / 1e12 / ALU_PEAK_TOPS,
                            "ops_per_launch": learned_ops, "avg_launch_ms": st_learned[2],
                            "peak_kind": "derived upper bound: 152 SMs x 128 int32 lanes x 2.07 GHz, one packed op per lane per cycle"},
        "roofline_stream": {"bound": "hbm", "kernel": "sparse_stream_kernel (+ count, scan, scatter)",
                            "achieved": alg_stream / (st_learned[0] / 1e3) / 1e9, "peak": hbm, "unit": "GB/s",
                            "frac": alg_stream / (st_learned[0] / 1e3) / 1e9 / hbm, "alg_bytes_per_launch": alg_stream,
                            "avg_launch_ms": st_learned[0], "peak_kind": f"{peak_kind} hbm_gbs"},
        "run_hbm": {"alg_bytes_per_run": alg_run, "achieved_learned": alg_run / (ms_learned / 1e3) / 1e9,
                    "achieved_plain": alg_run / (ms_plain / 1e3) / 1e9, "peak": hbm, "unit": "GB/s",
                    "frac_plain": alg_run / (ms_plain / 1e3) / 1e9 / hbm,
                    "frac_learned": alg_run / (ms_learned / 1e3) / 1e9 / hbm},
        "e2e": e2e, "cpu_baseline": cpu,
    }


def measure_hd(sme, torch, args, net):
    """The learned proposal's evaluation workload: 1920x1088, 300 frames, 4
    objects (4 VOPs), |v| <= 8 px, rotation <= 5 deg, scale 0.95-1.05, S = 16,
    half-pel; plain batch against the learned batch (trained network), both
    autotuned and replayed from graphs; one sampled pair of each against the
    oracle."""
    import gc

    import oracle as O
    from paper_1002_1168_gb300 import seedtrain, synth_gpu

    W4, H4, S4 = 1920, 1088, 16
    t0 = time.perf_counter()
    luma, alpha, _ = synth_gpu.hd_learned_eval(seed=1004, frames=args.hd_frames)
    torch.cuda.synchronize()
    gen_s = time.perf_counter() - t0
    F = luma.shape[0]
    vops = [alpha[j] for j in range(alpha.shape[0])]
    total = len(vops) * (F - 1) * (W4 // 16) * (H4 // 16)
    want = ("cost", "disp", "iters", "npos", "mb_class", "sse")
    steps = max(3, args.steps // 4)

    def timed(run, stream):
        for _ in range(3):
            run()
        torch.cuda.synchronize()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        for e0, e1 in ev:
            e0.record(stream)
            run()
            e1.record(stream)
        torch.cuda.synchronize()
        return sum(e0.elapsed_time(e1) for e0, e1 in ev) / steps

    k_smp, j_smp = min(150, F - 2), 1

    def oracle_ok(out, seeds=None):
        tmp = None if k_smp == 0 else out["mv"][k_smp - 1].cpu().numpy()
        sd = None if seeds is None else seeds[k_smp:k_smp + 1].cpu().numpy()
        o = O.estimate_sequence(O.OracleParams(W4, H4, S4, 2), luma[k_smp:k_smp + 2].cpu().numpy(),
                                alpha[j_smp, k_smp:k_smp + 2].cpu().numpy(), temporal_in=tmp, seed=sd)
        return bool(np.array_equal(out["mv"][k_smp].cpu().numpy(), o["mv"][0]) and
                    np.array_equal(out["cost"][k_smp].cpu().numpy().view(np.uint32), o["cost"][0]) and
                    int(out["sse"][k_smp].item()) == int(o["sse"][0]))

    b = sme.Batch([luma] * len(vops), vops, search_range=S4, subpel=2, want=want)
    b.tune(trials=2)
    ms = timed(lambda: b.run(sync=False), torch.cuda.current_stream())
    b.synchronize()
    pq = _device_quality(b.outputs, W4, H4)
    plain = {"value": total / (ms / 1e3), "unit": UNIT, "ms_per_run": ms, "config": b.config(), **pq,
             "bit_exact_vs_oracle_sample": oracle_ok(b.outputs[j_smp])}
    b.close()
    net = sized_net(sme, net, (F - 1) * (H4 // 4) * (W4 // 4))
    lb = seedtrain.LearnedBatch(net, [(luma, vops)], search_range=S4, subpel=2, want=want)
    lb.tune(trials=2)
    lms = timed(lambda: lb.run(sync=False), lb.stream)
    lb.synchronize()
    lq = _device_quality(lb.outputs, W4, H4)
    learned = {"value": total / (lms / 1e3), "unit": UNIT, "ms_per_run": lms, "config": lb.config(), **lq,
               "vs_plain_batched": ms / lms, "psnr_delta_db": lq["psnr_db_mean"] - pq["psnr_db_mean"],
               "iters_delta_pct": 100.0 * (lq["iters_per_opaque_mb"] / pq["iters_per_opaque_mb"] - 1.0),
               "bit_exact_vs_oracle_sample": oracle_ok(lb.outputs[j_smp], lb.seeds[j_smp])}
    lb.close()
    net.close()
    del b, lb, luma, alpha, vops
    gc.collect()
    torch.cuda.empty_cache()
    return {"workload": f"1920x1088, {F} frames, 4 VOPs, |v| <= 8, rotation <= 5 deg, scale 0.95-1.05, S=16, half-pel",
            "mb_per_run": total, "generation_s": gen_s, "runs": steps, "plain": plain, "learned_seeded": learned}


def measure_cif(sme, torch, args, rank, dist, net, train_info):
    """The single-sequence workload: CIF 352x288, 30 frames (29 pairs), one
    VOP, S = 16, half-pel (latency-bound: one dependency chain).  The plain
    pass (autotuned, L2 flushed between steps), end to end through
    sme_estimate_sequence_host, the oracle on the same sequence (parity and
    its single-threaded time), the exhaustive search, four vectors per MB,
    and the learned-seeded pass."""
    import oracle as O

    ws = dist.get_world_size() if dist else 1
    seq = workload(rank)
    P, M = FRAMES - 1, (W // 16) * (H // 16)
    est = sme.Estimator(W, H, search_range=S, subpel=SUBPEL)
    luma = torch.from_numpy(seq.luma).cuda()
    alpha = torch.from_numpy(seq.alpha[0]).cuda()
    out = est._alloc_outputs(P, OUT_FIELDS, luma.device)
    flush = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device=luma.device)
    if args.schedule == "auto":
        est.autotune(luma, alpha, out=out, trials=5)  # outside the timed region
    else:
        est.set_schedule(args.schedule)
    est_cfg = est.config()
    steps = max(args.steps, 3)
    for _ in range(max(args.warmup, 3)):
        est.estimate_sequence(luma, alpha, out=out, sync=False)
    est.synchronize()
    res = {k: v.cpu().numpy() for k, v in out.items()}
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    est.profile_begin(steps)
    for i in range(steps):
        flush.fill_(i & 0xff)  # L2 flush, outside the timed events
        starts[i].record()
        est.estimate_sequence(luma, alpha, out=out, sync=False)
        ends[i].record()
    torch.cuda.synchronize()
    calls, cls_ms, me_ms = est.profile_end()
    est.synchronize()  # raises on a device-side failure
    dev_ms = max_over_ranks(sum(s_.elapsed_time(e_) for s_, e_ in zip(starts, ends)), dist)

    # end-to-end through the public API with host buffers (pinned)
    hl = torch.from_numpy(seq.luma).pin_memory()
    ha = torch.from_numpy(seq.alpha[0]).pin_memory()
    hout = {k: v.pin_memory() for k, v in est._alloc_outputs(P, OUT_FIELDS, "cpu").items()}
    for _ in range(3):
        est.estimate_sequence_host(hl, ha, out=hout)
    e2e_steps = max(steps, 5)
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        est.estimate_sequence_host(hl, ha, out=hout)
    e2e_s = max_over_ranks(time.perf_counter() - t0, dist)
    h2d = int(hl.numel() + ha.numel())
    d2h = int(sum(v.numel() * v.element_size() for v in hout.values()))

    es_rec, es_mv, es_sad = measure_es(sme, torch, est, luma, flush, max(steps // 4, 3))
    four_mv_rec = measure_four_mv(sme, torch, seq, luma, alpha, flush, max(steps // 4, 3))
    learned = None
    if net is not None:
        learned, lres, lseeds = measure_learned(sme, torch, args, net, est, luma, alpha, flush)

    mbs_step = P * M
    value = job_rate(mbs_step * steps, ws, dev_ms / 1e3)
    cls = res["mb_class"]
    hbm, peak_kind = peaks()
    me_avg_s = me_ms / max(calls, 1) / 1e3
    alg = algorithmic_bytes(P, M, FRAMES)
    cb, orc = cpu_baseline(seq, budget_s=args.cpu_seconds)
    exact = all(np.array_equal(res[a].view(np.uint8), orc[b].view(np.uint8)) for a, b in
                [("mv", "mv"), ("cost", "cost"), ("iters", "iters"), ("npos", "npos"), ("disp", "disp"),
                 ("mb_class", "mbclass"), ("sse", "sse")])
    psnr = [O.psnr(int(x), W, H) for x in res["sse"].view(np.uint64)]
    op = cls == 1
    es_exact = True
    es_mv_np = es_mv.cpu().numpy()
    for k in (0, P // 2):
        bm, bs, _ = O.full_search(seq.luma[k], seq.luma[k + 1], W, H, SUBPEL, S)
        es_exact &= bool(np.array_equal(es_mv_np[k], bm) and np.array_equal(es_sad[k], bs))
    es_vop = es_psnr_like_method(sme, est, luma, es_mv, cls, 1, W, H)
    es_rec.update({"bit_exact_vs_oracle_sample": es_exact, "pairs_checked": [0, P // 2],
                   "search_points_ratio_method_vs_es": float(res["npos"][cls > 0].mean()) / es_rec["positions_per_mb"],
                   "psnr_db_mean_transparent_at_zero": es_vop,
                   "psnr_method_minus_es_db": float(np.mean(psnr)) - es_vop})
    if learned is not None:
        lexact, judge = learned_oracle_leg(seq, res, lres, lseeds)
        lq = stats(lres, W, H)
        learned.update({"vs_plain": learned["value"] / value, **lq,
                        "psnr_delta_db": lq["psnr_db_mean"] - float(np.mean(psnr)),
                        "bit_exact_vs_oracle": lexact,
                        "seed_changed_mbs": int((lres["mv"] != res["mv"]).any(axis=-1).sum()),
                        "es_judge": judge, "training": train_info})
    est.close()
    return {"workload": WORKLOAD, "value": value, "unit": UNIT, "ms_per_step": dev_ms / steps, "steps": steps,
            "execution": est_cfg, "l2": "flushed between steps (256 MiB write outside the timed events)",
            "e2e": {"value": job_rate(mbs_step * e2e_steps, ws, e2e_s), "unit": UNIT, "h2d_bytes_per_step": h2d,
                    "d2h_bytes_per_step": d2h},
            "roofline": {"bound": "hbm", "achieved": alg / me_avg_s / 1e9, "peak": hbm, "unit": "GB/s",
                         "frac": alg / me_avg_s / 1e9 / hbm, "traffic": ME_KERNEL_TRAFFIC_BYTES, "kernel": "me_kernel",
                         "peak_kind": f"{peak_kind} hbm_gbs", "alg_bytes_per_launch": alg,
                         "avg_launch_ms": me_avg_s * 1e3, "classify_avg_ms": cls_ms / max(calls, 1),
                         "critical_path_steps": (W // 16 - 1) + 2 * (H // 16 - 1) + P,
                         "alu": {"achieved_tops": algorithmic_int_ops(res) / me_avg_s / 1e12,
                                 "peak_tops": ALU_PEAK_TOPS,
                                 "frac": algorithmic_int_ops(res) / me_avg_s / 1e12 / ALU_PEAK_TOPS,
                                 "ops_per_launch": algorithmic_int_ops(res),
                                 "peak_kind": "derived upper bound: 152 SMs x 128 int32 lanes x 2.07 GHz"}},
            "cpu_baseline": cb,
            "quality": {"bit_exact_vs_oracle": exact, "mb_per_s_non_transparent": value * float((cls > 0).mean()),
                        "iters_per_opaque_mb": float(res["iters"][op].mean()),
                        "positions_per_mb": float(res["npos"][cls > 0].mean()),
                        "psnr_db_mean": float(np.mean(psnr)), "learned_seeded": learned,
                        "exhaustive_search": es_rec, "four_mv": four_mv_rec}}


def run_ours(args):
    import torch

    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    dist = None
    if ws > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    from paper_1002_1168_gb300 import build as cuda_build
    from paper_1002_1168_gb300 import sme

    cuda_build.build()
    # the packed-SAD operation mix of the integer rooflines, measured on this GPU
    mix_tops = sme.packed_sad_rate() / 1e12
    net, train_info = None, None
    if not args.no_learned:
        net, train_info = train_seednet(sme, torch, args)
    if args.cif_only:  # profiling: the CIF x 30 leg alone (ES, four vectors, learned), as its own line
        cif = measure_cif(sme, torch, args, rank, dist, net, train_info)
        if net is not None:
            net.close()
        if rank == 0:
            print(json.dumps({"cif30": cif}))
        if dist:
            dist.destroy_process_group()
        return
    head = measure_headline(sme, torch, args, net, dist, rank)
    if args.headline_only:
        args.no_cif = args.no_batch = args.no_hd = args.no_paper = True
    cif = None if args.no_cif else measure_cif(sme, torch, args, rank, dist, net, train_info)
    batched = None if args.no_batch else measure_batch(sme, torch, args, rank, dist, net)
    hd = None if (args.no_hd or net is None) else measure_hd(sme, torch, args, net)
    paper_setup = measure_paper_setup(sme, torch) if (rank == 0 and not args.no_paper) else None
    if net is not None:
        net.close()
    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return

    learned = head["learned"] if net is not None else None
    value = learned["value"] if learned else head["plain"]["value"]
    ms = head["ms_learned"] if learned else head["ms_plain"]
    rs = head["roofline_search"]
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": head["steps"],
        "warmup": head["warmup"], "ms_per_step": ms, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "u8+f32", "data": "synthetic",
        "config": {"workload": head["workload"], "form": "learned-seeded" if learned else "plain",
                   "mbs_per_step": head["total_mbs"], "seed": 1005, "search_range": UHD_S, "subpel": 2,
                   "l2": "inputs (72 GB) far above L2; no flush needed",
                   "parallelism": f"replicas x{ws}" if ws > 1 else "single GPU",
                   "execution": learned["config"] if learned else head["plain"]["config"]},
        "plain": head["plain"], "learned_seeded": learned, "learned_seeded_pair_rounds": head["learned_rounds"],
        "clocks": head["clocks"],
        "e2e": head["e2e"] or {"value": None, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        "gpu_launches": head["launches_per_run"] * head["steps"],
        "roofline": {"bound": rs["bound"], "achieved": rs["achieved"], "peak": rs["peak"], "unit": rs["unit"],
                     "frac": rs["frac"], "traffic": SEARCH_KERNEL_TRAFFIC_BYTES, "kernel": rs["kernel"],
                     "peak_kind": rs["peak_kind"], "ops_per_launch": rs["ops_per_launch"],
                     "avg_launch_ms": rs["avg_launch_ms"],
                     "stream_pass": head["roofline_stream"], "run_hbm": head["run_hbm"]},
        "cpu_baseline": head["cpu_baseline"],
        "wall_s_timed": head["wall_s_timed"], "generation_s": head["generation_s"],
        "cif30": cif, "batched": batched, "hd_learned_eval": hd, "paper_setup": paper_setup,
    }
    mix = {"peak": mix_tops, "unit": "Tops/s",
           "kind": "measured: the same operation mix (funnel-shift align, __vsadu4, add) on independent "
                   "register-resident chains, sme_packed_sad_rate_launch, 8 CTAs x 256 threads per SM"}
    line["roofline"]["measured_op_mix"] = {**mix, "frac": rs["achieved"] / mix_tops}
    if cif is not None:
        es = cif["quality"]["exhaustive_search"]["roofline"]
        es["measured_op_mix"] = {**mix, "frac": es["achieved_tops"] / mix_tops}
    print(json.dumps(line))
    if dist:
        dist.destroy_process_group()


def profile_seednet(args):
    """The seed network alone, for profiling: the dense forward over the
    features of the CIF workload's 29 pairs (random initial weights),
    args.steps times after args.warmup; prints the mean time per forward."""
    import torch
    from paper_1002_1168_gb300 import build as cuda_build
    from paper_1002_1168_gb300 import sme, synth

    cuda_build.build()
    seq = workload(0)
    P = FRAMES - 1
    net = sme.SeedNet(max_cells=P * (H // 4) * (W // 4))
    net.set_params(sme.pack_params(synth.seednet_init(3)))
    luma = torch.from_numpy(seq.luma).cuda()
    feats = net.features(luma, 0, 1, subpel=SUBPEL, n_pairs=P)
    for _ in range(max(args.warmup, 1)):
        net.forward(feats)
    net.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(args.steps):
        net.forward(feats)
    e1.record()
    net.synchronize()
    print(json.dumps({"seednet_forward_us": 1e3 * e0.elapsed_time(e1) / args.steps, "cells": P * (H // 4) * (W // 4),
                      "steps": args.steps}))
    net.close()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--cpu-seconds", type=float, default=10.0)
    ap.add_argument("--schedule", default="auto", choices=["auto", "pair", "mb", "cluster"])
    ap.add_argument("--no-batch", action="store_true", help="skip the secondary batched measurement")
    ap.add_argument("--no-learned", action="store_true", help="skip training and the learned-seeded measurements")
    ap.add_argument("--no-cif", action="store_true", help="skip the CIF x 30 single-sequence measurements")
    ap.add_argument("--no-hd", action="store_true", help="skip the 1920x1088 x 300-frame learned evaluation")
    ap.add_argument("--no-paper", action="store_true", help="skip the paper-setting QCIF measurement")
    ap.add_argument("--no-e2e", action="store_true", help="skip the headline's host-buffer (end-to-end) runs")
    ap.add_argument("--no-rounds", action="store_true", help="skip the pair-round learned form at the headline")
    ap.add_argument("--headline-only", action="store_true", help="only the headline measurement (profiling)")
    ap.add_argument("--cif-only", action="store_true", help="only the CIF x 30 measurements (profiling)")
    ap.add_argument("--hd-frames", type=int, default=300, help="frames of the 1920x1088 learned evaluation")
    ap.add_argument("--learn-pairs", type=int, default=2000, help="CIF VOP pairs the seed network is trained on")
    ap.add_argument("--learn-steps", type=int, default=800, help="Adam steps (32 pairs each)")
    ap.add_argument("--batch-only", action="store_true", help="only the batched measurement (profiling)")
    ap.add_argument("--seednet-only", action="store_true", help="only the seed network's forward (profiling)")
    ap.add_argument("--scale-only", action="store_true",
                    help="only the plain 3840x2160 batch measurement (profiling)")
    ap.add_argument("--scale-seqs", type=int, default=16, help="3840x2160 sequences of the at-scale measurement")
    ap.add_argument("--scale-frames", type=int, default=60, help="frames per 3840x2160 sequence")
    ap.add_argument("--batch-preset", default="full", choices=["full", "hd8"],
                    help="batched workload: the 64-sequence batch, or 8 HD sequences (profiling)")
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
    elif args.seednet_only:
        profile_seednet(args)
    elif args.batch_only:
        import torch
        from paper_1002_1168_gb300 import build as cuda_build
        from paper_1002_1168_gb300 import sme

        cuda_build.build()
        print(json.dumps({"batched": measure_batch(sme, torch, args, 0, None)}))
    elif args.scale_only:
        import torch
        from paper_1002_1168_gb300 import build as cuda_build
        from paper_1002_1168_gb300 import sme

        cuda_build.build()
        args.no_e2e = True
        print(json.dumps({"headline_plain": measure_headline(sme, torch, args, None, None, 0)}))
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
