"""GPU parity of the learned seed network against its CPU oracle.

Hidden activations and gradients are bfloat16 on both sides at the same
points; the GPU accumulates in FP32 on tensor cores, the oracle in float64, so
an element can land one bfloat16 step apart.  The comparisons are therefore
relative-norm tolerances: 1e-2 for the forward outputs, 3e-2 for the
gradients, and one bfloat16 step (2^-7 relative) for the input features."""
import numpy as np
import pytest

from oracle import seednet as SN
from paper_1002_1168_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sme():
    from paper_1002_1168_gb300 import build as cuda_build
    from paper_1002_1168_gb300 import sme as m

    cuda_build.build()
    return m


def as_float(t16):
    return t16.view(torch.bfloat16).float().cpu().numpy().astype(np.float64)


def rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-30))


def test_features_match_oracle(sme):
    seq = synth.cif_sequence(seed=1002, frames=3)
    rng = np.random.default_rng(2)
    tmp = rng.integers(-20, 21, (396, 2)).astype(np.int16)
    net = sme.SeedNet(max_cells=88 * 72)
    luma = torch.from_numpy(seq.luma).cuda()
    f = as_float(net.features(luma, 1, 2, temporal=torch.from_numpy(tmp).cuda(), subpel=2))
    o = SN.features(seq.luma[1], seq.luma[2], tmp, 2)
    assert f.shape == o.shape == (72, 88, 16)
    assert np.all(np.abs(f - o) <= 2.0 ** -7 * np.abs(o) + 1e-12)
    assert np.mean(f == o) > 0.99
    net.close()


def test_features_batched_pairs_match_single(sme):
    # one launch over P pairs (ref frame q, current frame q + 2) equals P
    # single-pair launches, bit for bit, and the oracle within one bf16 step
    seq = synth.cif_sequence(seed=1002, frames=6)
    net = sme.SeedNet(max_cells=4 * 88 * 72)
    luma = torch.from_numpy(seq.luma).cuda()
    many = net.features(luma, 0, 2, subpel=2, n_pairs=4).cpu()
    assert many.shape == (4, 72, 88, 16)
    for q in range(4):
        one = net.features(luma, q, q + 2, subpel=2).cpu()
        assert torch.equal(many[q], one)
        o = SN.features(seq.luma[q], seq.luma[q + 2], None, 2)
        f = as_float(many[q])
        assert np.all(np.abs(f - o) <= 2.0 ** -7 * np.abs(o) + 1e-12)
    net.close()


def test_table_launches_equal_per_sequence_launches(sme):
    """Classes and features gathered through frame-address tables (frames of
    two sequences in any order, empty planes for missing VOPs) equal the
    per-sequence launches bit for bit."""
    s1 = synth.cif_sequence(seed=1002, frames=4)
    s2 = synth.cif_sequence(seed=1009, frames=3)
    l1, l2 = torch.from_numpy(s1.luma).cuda(), torch.from_numpy(s2.luma).cuda()
    a1, a2 = torch.from_numpy(s1.alpha[0]).cuda(), torch.from_numpy(s2.alpha[0]).cuda()
    FS = 352 * 288
    est = sme.Estimator(352, 288)
    tab = torch.tensor([a2.data_ptr() + 2 * FS, 0, a1.data_ptr() + 1 * FS, a1.data_ptr() + 3 * FS],
                       dtype=torch.int64, device="cuda")
    got = est.classify_table(tab).cpu()
    c1, _ = est.classify(a1, want_packed=False)
    c2, _ = est.classify(a2, want_packed=False)
    assert torch.equal(got[0], c2[2].cpu()) and torch.equal(got[2], c1[1].cpu()) and torch.equal(got[3], c1[3].cpu())
    assert not got[1].any()  # an empty plane: every MB transparent
    net = sme.SeedNet(max_cells=3 * 88 * 72)
    ftab = torch.tensor([[l1.data_ptr(), l1.data_ptr() + 2 * FS], [l2.data_ptr() + FS, l2.data_ptr() + 2 * FS],
                         [l1.data_ptr() + 3 * FS, l1.data_ptr()]], dtype=torch.int64, device="cuda")
    many = net.features_table(ftab, 352, 288, subpel=2).cpu()
    assert torch.equal(many[0], net.features(l1, 0, 2, subpel=2).cpu())
    assert torch.equal(many[1], net.features(l2, 1, 2, subpel=2).cpu())
    assert torch.equal(many[2], net.features(l1, 3, 0, subpel=2).cpu())
    net.close()
    est.close()


def test_forward_active_equals_dense(sme):
    # the layers run only near non-transparent MBs; their seeds are those of
    # the dense pass bit for bit, transparent MBs get (0, 0)
    _, params, x, net, xt = _setup(sme, N=3, W=160, H=128, seed=8)
    N, Hc, Wc, _ = x.shape
    M = (Hc // 4) * (Wc // 4)
    rng = np.random.default_rng(9)
    cls = np.zeros((N, M), np.uint8)
    cls[0, 0] = 1                                   # corner
    cls[1, rng.choice(M, 6, replace=False)] = 1     # scattered
    cls[1, rng.choice(M, 6, replace=False)] = 2     # boundary MBs use seeds too
    cls[2, :] = 1                                   # all opaque
    dense = net.forward(xt).cpu().numpy()
    sparse = net.forward_active(xt, torch.from_numpy(cls).cuda()).cpu().numpy()
    op = cls != 0
    assert np.array_equal(sparse[op], dense[op])
    assert np.all(sparse[~op] == 0)
    net.close()


def _setup(sme, N=2, W=96, H=64, seed=5):
    rng = np.random.default_rng(seed)
    params = SN.init_params(seed)
    params = [(w * (3.0 if li == 4 else 1.0), rng.normal(0, 0.05, b.shape)) for li, (w, b) in enumerate(params)]
    x = SN.bf16(rng.normal(0, 0.5, (N, H // 4, W // 4, 16)))
    net = sme.SeedNet(max_cells=N * (H // 4) * (W // 4))
    net.set_params(sme.pack_params(params))
    xt = torch.from_numpy(x.astype(np.float32)).to(torch.bfloat16).view(torch.int16).cuda()
    return rng, params, x, net, xt


def test_forward_matches_oracle(sme):
    _, params, x, net, xt = _setup(sme)
    seeds, cells = net.forward(xt, want_cells=True)
    net.synchronize()  # no device-side wait gave up
    acts = SN.forward(x, params)
    assert rel(cells.cpu().numpy(), acts[-1]) < 1e-2
    assert rel(seeds.cpu().numpy(), SN.pool_seeds(acts[-1])) < 1e-2
    net.close()


def test_gradients_match_oracle(sme):
    rng, params, x, net, xt = _setup(sme, seed=6)
    N, Hc, Wc, _ = x.shape
    M = (Hc // 4) * (Wc // 4)
    labels = rng.normal(0, 2, (N, M, 2))
    mask = (rng.random((N, M)) < 0.8).astype(np.uint8)
    loss_g, g = net.gradients(xt, torch.from_numpy(labels.astype(np.float32)).cuda(), torch.from_numpy(mask).cuda())
    acts = SN.forward(x, params)
    loss_o, d = SN.loss_and_grad(acts[-1], labels, mask)
    grads = SN.backward(acts, params, d)
    assert loss_g == pytest.approx(loss_o, rel=1e-2)
    gg = sme.unpack_params(g)
    for li in range(5):
        assert rel(gg[li][0], grads[li][0]) < 3e-2, li
        assert rel(gg[li][1], grads[li][1]) < 3e-2, li
    net.close()


def test_training_reduces_loss(sme):
    rng, params, x, net, xt = _setup(sme, N=4, seed=7)
    N, Hc, Wc, _ = x.shape
    M = (Hc // 4) * (Wc // 4)
    # a learnable target: the seed is a fixed linear function of the inputs
    tgt = 8 * x[..., :2].reshape(N, Hc // 4, 4, Wc // 4, 4, 2).mean(axis=(2, 4)).reshape(N, M, 2)
    labels = torch.from_numpy(tgt.astype(np.float32)).cuda()
    mask = torch.ones((N, M), dtype=torch.uint8, device="cuda")
    first = net.train_step(xt, labels, mask, 1e-3, want_loss=True)
    for _ in range(150):
        last = net.train_step(xt, labels, mask, 1e-3, want_loss=True)
    assert last < 0.5 * first
    net.close()


def test_adam_update_matches_oracle(sme):
    """Two sme_seednet_train_step updates from fresh moments against the
    oracle's FP32 Adam step, fed with the gradients the GPU computes at each
    point (sme_seednet_gradients).  The weight gradients are summed with
    float atomics, so a recomputed gradient can differ in its last bits: the
    comparison is tight (0.1 % of the update plus a few ulps) where the
    gradient is well above that noise, and bounded by the step size
    elsewhere."""
    rng, params, x, net, xt = _setup(sme, seed=8)
    N, Hc, Wc, _ = x.shape
    M = (Hc // 4) * (Wc // 4)
    labels = torch.from_numpy(rng.normal(0, 2, (N, M, 2)).astype(np.float32)).cuda()
    mask = torch.ones((N, M), dtype=torch.uint8, device="cuda")
    lr = 1e-3
    p = net.get_params()
    m = np.zeros_like(p)
    v = np.zeros_like(p)
    prev = p.copy()
    for t in (1, 2):
        _, g = net.gradients(xt, labels, mask)
        net.train_step(xt, labels, mask, lr)
        got = net.get_params()
        p, m, v = SN.adam_step(p, g, m, v, t, lr)
        firm = np.abs(g) >= 1e-3 * np.abs(g).max()
        assert firm.sum() > 1000  # thousands of parameters are tested tightly
        tol = 4 * np.spacing(np.abs(p)) + 1e-3 * lr
        bad = np.abs(got - p) > tol
        assert not np.any(bad & firm), (t, np.flatnonzero(bad & firm)[:8])
        assert np.all(np.abs(got - p) <= 3 * lr)
        assert np.any(got != prev)  # the parameters moved
        prev = got
    net.close()


def test_forward_active_table_equals_strided_maps(sme):
    """The class maps given as a table of class-row addresses (some rows
    absent: an empty plane) select the same MBs, hence the same seeds, as the
    same maps given as one strided tensor."""
    _, params, x, net, xt = _setup(sme, N=3)
    N, Hc, Wc, _ = x.shape
    M = (Hc // 4) * (Wc // 4)
    rng = np.random.default_rng(12)
    cls = np.zeros((2, N, M), np.uint8)
    cls[0, 0, rng.choice(M, 5, replace=False)] = 1
    cls[1, 1, rng.choice(M, 4, replace=False)] = 2
    cls[0, 2, :] = 1
    ct = torch.from_numpy(cls).cuda()
    want = net.forward_active(xt, ct).cpu().numpy()
    rows = torch.tensor([[ct[j, i].data_ptr() for i in range(N)] for j in range(2)], dtype=torch.int64).cuda()
    got = net.forward_active_table(xt, rows.reshape(-1), 2).cpu().numpy()
    assert np.array_equal(got, want)
    # an absent row (0) is an empty plane: map 1 of pair 1 dropped
    rows[1, 1] = 0
    cls2 = cls.copy()
    cls2[1, 1] = 0
    want2 = net.forward_active(xt, torch.from_numpy(cls2).cuda()).cpu().numpy()
    got2 = net.forward_active_table(xt, rows.reshape(-1), 2).cpu().numpy()
    assert np.array_equal(got2, want2)
    net.close()
