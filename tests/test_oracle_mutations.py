"""Pin strength: plant a plausible mistake in a copy of the C oracle and
check that at least one CPU pin (tests/test_oracle_pins.py) fails on it.

Each mutant is compiled with the oracle's own flags into a temporary
directory and the pins run against it in a subprocess (SME_ORACLE_LIB); the
shipped oracle is never modified.  The mistakes cover every part of the
method: interpolation (Fig. 5 half-sample accuracy), the valid set (Table 1),
costs and classes (Fig. 1), candidate gathering and selection (Fig. 1,
Fig. 3), the gradient step (Eqs. 3-5), the pixel recursive loop (Fig. 4), the
seeded fallback, compensation and PSNR (Sec. 4)."""
import os
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "sme_oracle.c")

# (name, original text, planted mistake)
MUTANTS = [
    ("diagonal half-sample rounds with +1",
     "return (a + r[1] + r[W] + r[W + 1] + 2) >> 2;", "return (a + r[1] + r[W] + r[W + 1] + 1) >> 2;"),
    ("horizontal half-sample truncates",
     "if (fx && !fy) return (a + r[1] + 1) >> 1;", "if (fx && !fy) return (a + r[1]) >> 1;"),
    ("vertical half-sample reads the right neighbour",
     "if (!fx && fy) return (a + r[W] + 1) >> 1;", "if (!fx && fy) return (a + r[1] + 1) >> 1;"),
    ("texture SAD without absolute value",
     "s += (uint32_t)abs(p - c);", "s += (uint32_t)(p - c);"),
    ("valid set one pixel too wide on the right",
     "*hix = imin(S * h, (W - block - X0) * h);", "*hix = imin(S * h, (W - block - X0 + 1) * h);"),
    ("search range not scaled to MV units",
     "*lox = imax(-S * h, -X0 * h);", "*lox = imax(-S, -X0 * h);"),
    ("shape cost floors instead of truncating",
     "int fx = dx / h, fy = dy / h;", "int fx = dx >> (h - 1), fy = dy >> (h - 1);"),
    ("opaque threshold 255",
     "if (n == 256) return ORC_OPAQUE;", "if (n >= 255) return ORC_OPAQUE;"),
    ("Theta test strict",
     "if ((float)abs(g) >= lim) ux = 2.0f / (float)g;", "if ((float)abs(g) > lim) ux = 2.0f / (float)g;"),
    ("DPD sign flipped",
     "int dpd = ref_sample(ref, W, h, x * h + dx, y * h + dy) - (int)cur[(size_t)y * W + x];",
     "int dpd = (int)cur[(size_t)y * W + x] - ref_sample(ref, W, h, x * h + dx, y * h + dy);"),
    ("update without the minus sign of Eq. 3",
     "out[0] = nx ? -(P->epsilon * (sx / (float)nx)) : 0.0f;", "out[0] = nx ? (P->epsilon * (sx / (float)nx)) : 0.0f;"),
    ("x gradient taken along y",
     "int g = (int)cur[(size_t)y * W + x + 1] - (int)cur[(size_t)y * W + x - 1];",
     "int g = (y > 0 && y < H - 1) ? (int)cur[(size_t)(y + 1) * W + x] - (int)cur[(size_t)(y - 1) * W + x] : 0;"),
    ("mean over all 256 pixels",
     "out[1] = ny ? -(P->epsilon * (sy / (float)ny)) : 0.0f;", "out[1] = ny ? -(P->epsilon * (sy / 256.0f)) : 0.0f;"),
    ("epsilon ignored",
     "out[0] = nx ? -(P->epsilon * (sx / (float)nx)) : 0.0f;", "out[0] = nx ? -(sx / (float)nx) : 0.0f;"),
    ("sequential instead of pairwise sum",
     "for (int i = 0; i + s < n; i += 2 * s) t[i] = t[i] + t[i + s];",
     "if (s == 1) for (int i = 1; i < n; ++i) t[0] = t[0] + t[i];"),
    ("last minimum wins ties",
     "if (best < 0 || c < bc) { best = k; bc = c; }", "if (best < 0 || c <= bc) { best = k; bc = c; }"),
    ("B taken from the upper-right MB",
     "if (v > 0) { cx[1] = mv[m - mbw].dx; cy[1] = mv[m - mbw].dy; }",
     "if (v > 0 && u < mbw - 1) { cx[1] = mv[m - mbw + 1].dx; cy[1] = mv[m - mbw + 1].dy; }"),
    ("C taken from the upper-left MB",
     "if (v > 0 && u < mbw - 1) { cx[2] = mv[m - mbw + 1].dx; cy[2] = mv[m - mbw + 1].dy; }",
     "if (v > 0 && u > 0) { cx[2] = mv[m - mbw - 1].dx; cy[2] = mv[m - mbw - 1].dy; }"),
    ("temporal candidate dropped",
     "if (temporal) { cx[3] = temporal[m].dx; cy[3] = temporal[m].dy; }", ""),
    ("temporal field not chained between pairs",
     "const orc_mv* tmp = k == 0 ? temporal_in : mv + (size_t)(k - 1) * M;", "const orc_mv* tmp = temporal_in;"),
    ("proposal taken on equal SAD",
     "if (cq < c) { dx = qx; dy = qy; c = cq; continue; }", "if (cq <= c) { dx = qx; dy = qy; c = cq; continue; }"),
    ("proposal rounded toward zero",
     "int qx = iclamp(dx + (int)roundf((float)h * last[0]), lox, hix);",
     "int qx = iclamp(dx + (int)((float)h * last[0]), lox, hix);"),
    ("eight directions in column order",
     "int nx = iclamp(dx + ii, lox, hix), ny = iclamp(dy + jj, loy, hiy);",
     "int nx = iclamp(dx + jj, lox, hix), ny = iclamp(dy + ii, loy, hiy);"),
    ("eight directions skipped",
     "if (bcost < c) { dx = bx; dy = by; c = bcost; continue; }", ""),
    ("iteration cap off by one",
     "while (k < P->max_iters) {", "while (k <= P->max_iters) {"),
    ("seeded search kept on a tie",
     "if (!(c < pc)) {", "if (!(c <= pc)) {"),
    ("seed rounded down",
     "cx[4] = (int)roundf(fminf(fmaxf((float)h * seed[2 * m], -1024.0f), 1024.0f));",
     "cx[4] = (int)floorf(fminf(fmaxf((float)h * seed[2 * m], -1024.0f), 1024.0f));"),
    ("seeded search only from the seed",
     "int pk = prs_search(P, ref, cur, X0, Y0, lox, hix, loy, hiy, &pdx, &pdy, &pc, plast, &ps);",
     "int pk = 0; pc = 0xffffffffu; plast[0] = plast[1] = 0.0f;"),
    ("compensation with the vector negated",
     "int p = ref_sample(ref, W, h, x * h + d.dx, y * h + d.dy);",
     "int p = ref_sample(ref, W, h, x * h - d.dx, y * h - d.dy);"),
    ("PSNR with 255 instead of 255 squared",
     "return 10.0 * log10(255.0 * 255.0 * (double)W * (double)H / (double)sse);",
     "return 10.0 * log10(255.0 * (double)W * (double)H / (double)sse);"),
    ("distinct positions count repeats",
     "if (s->pos[k] == key) return;", "if (s->pos[k] == key) break;"),
    ("boundary texture-T variant ignored",
     "if (cls == ORC_BOUNDARY && P->boundary_t_texture) {", "if (0) {"),
    ("boundary texture-T variant: T wins ties",
     "best = tex_t < tex_s ? 3 : sb;", "best = tex_t <= tex_s ? 3 : sb;"),
    ("boundary texture-T variant: T in the shape competition",
     "if (q != 3 && (sb < 0 || costs[q] < costs[sb])) sb = q;", "if (sb < 0 || costs[q] < costs[sb]) sb = q;"),
    ("boundary texture-T variant: cost is the texture SAD",
     "best = tex_t < tex_s ? 3 : sb;\n                bc = costs[best];",
     "best = tex_t < tex_s ? 3 : sb;\n                bc = best == 3 ? tex_t : tex_s;"),
]


# Mistakes in the four-vector mode (Sec. 3.2, 8x8 blocks), caught by the pins
# of tests/test_oracle_four_mv.py.
MUTANTS4 = [
    ("A from block 0 of the left MB",
     "if (u > 0) { cx[0] = mv4[4 * (m - 1) + 1].dx; cy[0] = mv4[4 * (m - 1) + 1].dy; }",
     "if (u > 0) { cx[0] = mv4[4 * (m - 1) + 0].dx; cy[0] = mv4[4 * (m - 1) + 0].dy; }"),
    ("B from block 3 of the MB above",
     "if (v > 0) { cx[1] = mv4[4 * (m - mbw) + 2].dx; cy[1] = mv4[4 * (m - mbw) + 2].dy; }",
     "if (v > 0) { cx[1] = mv4[4 * (m - mbw) + 3].dx; cy[1] = mv4[4 * (m - mbw) + 3].dy; }"),
    ("C from block 3 of the MB above-right",
     "cx[2] = mv4[4 * (m - mbw + 1) + 2].dx;\n                cy[2] = mv4[4 * (m - mbw + 1) + 2].dy;",
     "cx[2] = mv4[4 * (m - mbw + 1) + 3].dx;\n                cy[2] = mv4[4 * (m - mbw + 1) + 3].dy;"),
    ("T from block 1 of the previous field",
     "if (temporal4) { cx[3] = temporal4[4 * m].dx; cy[3] = temporal4[4 * m].dy; }",
     "if (temporal4) { cx[3] = temporal4[4 * m + 1].dx; cy[3] = temporal4[4 * m + 1].dy; }"),
    ("temporal field of four vectors not chained",
     "const orc_mv* tmp = k == 0 ? temporal_in4 : mv4 + (size_t)4 * (k - 1) * M;",
     "const orc_mv* tmp = temporal_in4;"),
    ("blocks in column order",
     "const int BX = X0 + 8 * (b & 1), BY = Y0 + 8 * (b >> 1);",
     "const int BX = X0 + 8 * (b >> 1), BY = Y0 + 8 * (b & 1);"),
    ("block search starts from the 16x16 cost",
     "c = block_sad(ref, cur, W, h, 8, BX, BY, dx, dy);", "c = bc;"),
    ("boundary quadrant costed at the MB origin",
     "c = shape_block(aref, acur, W, h, 8, BX, BY, dx, dy);", "c = shape_block(aref, acur, W, h, 8, X0, Y0, dx, dy);"),
    ("block positions without the MB candidates",
     "pos_set ps = brs;", "pos_set ps;\n                ps.n = 0;"),
    ("block gradient mean over all 64 pixels",
     "out[0] = (nx > 0) ? -(P->epsilon * (sx / (float)nx)) : 0.0f;",
     "out[0] = (nx > 0) ? -(P->epsilon * (sx / (float)(n * n))) : 0.0f;"),
    ("block gradient terms laid out 16 wide",
     "tx[j * n + i] = (float)dpd * ux;", "tx[j * 16 + i] = (float)dpd * ux;"),
    ("block gradient summed sequentially",
     "float sx = pairwise_sum(tx, n * n), sy = pairwise_sum(ty, n * n);",
     "float sx = 0.0f, sy = pairwise_sum(ty, n * n);\n    for (int q = 0; q < n * n; ++q) sx = sx + tx[q];"),
    ("compensation block index transposed",
     "const int b = 2 * ((y % 16) / 8) + (x % 16) / 8;", "const int b = 2 * ((x % 16) / 8) + (y % 16) / 8;"),
    ("block proposal taken on equal SAD",
     "uint32_t cq = block_sad(ref, cur, W, h, n, X0, Y0, qx, qy);\n            pos_note(ps, qx, qy);\n            if (cq < c)",
     "uint32_t cq = block_sad(ref, cur, W, h, n, X0, Y0, qx, qy);\n            pos_note(ps, qx, qy);\n            if (cq <= c)"),
    ("block neighbours use the 16x16 SAD",
     "uint32_t cn = block_sad(ref, cur, W, h, n, X0, Y0, nx, ny);",
     "uint32_t cn = block_sad(ref, cur, W, h, 16, X0 - 8 * ((X0 / 8) & 1), Y0 - 8 * ((Y0 / 8) & 1), nx, ny);"),
]


def _run_mutant(tmpdir, i, name, old, new, pins="test_oracle_pins.py"):
    src = open(SRC).read()
    if src.count(old) < 1:
        return name, "anchor not found"
    mutated = src.replace(old, new, 1)
    d = os.path.join(tmpdir, f"m{i}")
    os.makedirs(d, exist_ok=True)
    c_path, so_path = os.path.join(d, "mutant.c"), os.path.join(d, "libmutant.so")
    with open(c_path, "w") as f:
        f.write(mutated)
    subprocess.run(["gcc", "-std=c99", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
                    "-o", so_path, c_path, "-lm"], check=True, capture_output=True)
    env = dict(os.environ, SME_ORACLE_LIB=so_path, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1")
    r = subprocess.run([sys.executable, "-m", "pytest", os.path.join(ROOT, "tests", pins), "-x",
                        "-q", "-p", "no:cacheprovider", "-m", "not gpu"], cwd=ROOT, env=env, capture_output=True,
                       text=True, timeout=600)
    return name, ("killed" if r.returncode not in (0, 5) else "survived")


def test_every_planted_mistake_fails_a_pin(tmp_path):
    workers = min(8, os.cpu_count() or 1)
    with ThreadPoolExecutor(workers) as ex:
        results = list(ex.map(lambda a: _run_mutant(str(tmp_path), *a),
                              [(i, *m) for i, m in enumerate(MUTANTS)]))
    bad = [(n, s) for n, s in results if s != "killed"]
    assert not bad, f"mutants not caught by the pins: {bad}"


def test_every_planted_four_vector_mistake_fails_a_pin(tmp_path):
    workers = min(8, os.cpu_count() or 1)
    with ThreadPoolExecutor(workers) as ex:
        results = list(ex.map(lambda a: _run_mutant(str(tmp_path), *a, pins="test_oracle_four_mv.py"),
                              [(100 + i, *m) for i, m in enumerate(MUTANTS4)]))
    bad = [(n, s) for n, s in results if s != "killed"]
    assert not bad, f"mutants not caught by the four-vector pins: {bad}"
