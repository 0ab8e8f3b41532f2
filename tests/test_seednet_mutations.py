"""Pin strength of the seed-network oracle: plant a plausible mistake in a
copy of oracle/seednet.py and check that a CPU pin
(tests/test_seednet_oracle.py) fails on it.  The mutant runs from a copy of
the oracle package in a temporary directory placed first on the import
path; the shipped oracle is never modified."""
import os
import shutil
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PKG = os.path.join(ROOT, "oracle")

MUTANTS = [
    ("bfloat16 ties away from zero", "rounded = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16",
     "rounded = ((u + 0x8000) >> 16) << 16"),
    ("kernel taps transposed", 'y += np.einsum("nhwc,oc->nhwo", xp[:, dy:dy + H, dx:dx + W], w[:, dy, dx])',
     'y += np.einsum("nhwc,oc->nhwo", xp[:, dy:dy + H, dx:dx + W], w[:, dx, dy])'),
    ("bias dropped", "y = np.zeros((N, H, W, w.shape[0])) + b", "y = np.zeros((N, H, W, w.shape[0]))"),
    ("input gradient without the tap shift",
     'dxp[:, dy:dy + H, dx:dx + W] += np.einsum("nhwo,oc->nhwc", dy_, w[:, dy, dx])',
     'dxp[:, 1:1 + H, 1:1 + W] += np.einsum("nhwo,oc->nhwc", dy_, w[:, dy, dx])'),
    ("weight gradient of the wrong tap",
     'dw[:, dy, dx] = np.einsum("nhwo,nhwc->oc", dy_, xp[:, dy:dy + H, dx:dx + W])',
     'dw[:, dy, dx] = np.einsum("nhwo,nhwc->oc", dy_, xp[:, dx:dx + H, dy:dy + W])'),
    ("ReLU mask from the layer output", "g = dx * (acts[li] > 0)", "g = dx * (acts[li + 1] > 0)"),
    ("ReLU on the last layer too", "if li < len(params) - 1:\n            y = np.maximum(y, 0.0)",
     "if True:\n            y = np.maximum(y, 0.0)"),
    ("seed scale missing in the gradient", "g = gs.reshape(N, Hc // 4, 1, Wc // 4, 1, 2) * (SEED_SCALE / 16.0)",
     "g = gs.reshape(N, Hc // 4, 1, Wc // 4, 1, 2) / 16.0"),
    ("Huber gradient not clipped", "gs = np.clip(r, -HUBER, HUBER) * m / n", "gs = r * m / n"),
    ("loss averaged over all MBs", "n = max(float(m.sum()), 1.0)", "n = float(m.size)"),
    ("pooling over one cell row", "s = out[..., :2].reshape(N, Hc // 4, 4, Wc // 4, 4, 2).mean(axis=(2, 4))",
     "s = out[..., :2].reshape(N, Hc // 4, 4, Wc // 4, 4, 2)[:, :, 0].mean(axis=3)"),
    ("current and reference swapped", "x[..., 0] = c / 255.0 - 0.5\n    x[..., 1] = r / 255.0 - 0.5",
     "x[..., 0] = r / 255.0 - 0.5\n    x[..., 1] = c / 255.0 - 0.5"),
    ("feature offset missing", "x[..., 0] = c / 255.0 - 0.5", "x[..., 0] = c / 255.0"),
    ("difference reversed", "x[..., 2] = (c - r) / 255.0", "x[..., 2] = (r - c) / 255.0"),
    ("temporal channel scaled by 16 only", "/ (16.0 * subpel)", "/ 16.0"),
    ("temporal channel scaled by 16 * h * h", "/ (16.0 * subpel)", "/ (16.0 * subpel * subpel)"),
    ("temporal axes swapped", "x[..., 3] = np.repeat(np.repeat(t[..., 0], 4, 0), 4, 1)",
     "x[..., 3] = np.repeat(np.repeat(t[..., 1], 4, 0), 4, 1)"),
    ("cell mean over 2x2 pixels", "c = cur.astype(np.float64).reshape(Hc, 4, Wc, 4).mean(axis=(1, 3))",
     "c = cur.astype(np.float64).reshape(Hc, 4, Wc, 4)[:, :2, :, :2].mean(axis=(1, 3))"),
    ("Adam without bias correction", "p = p - lr * (m / c1) / (np.sqrt(v / c2) + eps)",
     "p = p - lr * m / (np.sqrt(v) + eps)"),
    ("Adam moments' rates swapped", "m = b1 * m + (f32(1) - b1) * g\n    v = b2 * v + (f32(1) - b2) * g * g",
     "m = b2 * m + (f32(1) - b2) * g\n    v = b1 * v + (f32(1) - b1) * g * g"),
    ("Adam ascends", "p = p - lr * (m / c1)", "p = p + lr * (m / c1)"),
    ("Adam epsilon inside the root", "(np.sqrt(v / c2) + eps)", "np.sqrt(v / c2 + eps)"),
]


def _run(tmpdir, i, name, old, new):
    d = os.path.join(tmpdir, f"m{i}")
    shutil.copytree(PKG, os.path.join(d, "oracle"), ignore=shutil.ignore_patterns("_build", "__pycache__"))
    path = os.path.join(d, "oracle", "seednet.py")
    src = open(path).read()
    if old not in src:
        return name, "anchor not found"
    with open(path, "w") as f:
        f.write(src.replace(old, new, 1))
    env = dict(os.environ, PYTHONPATH=os.pathsep.join([d, ROOT, os.path.join(ROOT, "tests")]),
               OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1")
    r = subprocess.run([sys.executable, "-m", "pytest", os.path.join(ROOT, "tests", "test_seednet_oracle.py"), "-x",
                        "-q", "-p", "no:cacheprovider"], cwd=d, env=env, capture_output=True, text=True, timeout=600)
    return name, ("killed" if r.returncode not in (0, 5) else "survived")


def test_every_planted_mistake_fails_a_pin(tmp_path):
    with ThreadPoolExecutor(min(8, os.cpu_count() or 1)) as ex:
        results = list(ex.map(lambda a: _run(str(tmp_path), *a), [(i, *m) for i, m in enumerate(MUTANTS)]))
    bad = [(n, s) for n, s in results if s != "killed"]
    assert not bad, f"mutants not caught by the pins: {bad}"


def test_mutant_copy_is_the_module_under_test(tmp_path):
    """The subprocess imports the copy, not the shipped oracle (else every
    mutant would trivially 'survive' or 'die' for the wrong reason)."""
    d = str(tmp_path)
    shutil.copytree(PKG, os.path.join(d, "oracle"), ignore=shutil.ignore_patterns("_build", "__pycache__"))
    env = dict(os.environ, PYTHONPATH=os.pathsep.join([d, ROOT]))
    r = subprocess.run([sys.executable, "-c", "import oracle.seednet as s; print(s.__file__)"], cwd=d, env=env,
                       capture_output=True, text=True, check=True)
    assert r.stdout.strip().startswith(d)
