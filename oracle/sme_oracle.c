/*
 * CPU oracle for shape-adaptive motion estimation -- TEST INFRASTRUCTURE ONLY.
 *
 * A plain, slow, single-threaded restatement of the method of Benboubker,
 * Abdi and Ahaitouf, "Shape-Adaptive Motion Estimation Algorithm for MPEG-4
 * Video Coding": the per-macroblock procedure of Fig. 1, the block recursive
 * search of Sec. 3.1 (Fig. 3) and the pixel recursive search of Sec. 3.2
 * (Eqs. 2-5, Fig. 4), followed by motion compensation and PSNR (Sec. 4), plus
 * an exhaustive search (ES, Sec. 1 and Table 1) used only to judge results.
 *
 * Only the test suite, the smoke check and the CPU-baseline leg of the
 * benchmark may load this library.  It shares no code, header, table or
 * helper with the CUDA path and must never be called by the product path.
 *
 * Build: gcc -std=c99 -O2 -ffp-contract=off -fno-fast-math -shared -fPIC.
 * -ffp-contract=off matters: the FP32 gradient step is defined operation by
 * operation with round-to-nearest and no fused multiply-add.
 *
 * Readings of the paper taken here (each is argued in the design notes):
 *  - MB classes from the CURRENT binary alpha block: no pixel inside ->
 *    transparent (0), all 256 inside -> opaque (1), else boundary (2).
 *  - Cost of a candidate d for the MB at X: backward matching of the current
 *    block against the reference displaced by d; the prediction of pixel p is
 *    ref(p + d).  Texture cost = SAD of luma (Sec. 2, Fig. 1 opaque branch);
 *    shape cost = number of alpha mismatches (Fig. 1 boundary branch).
 *  - Candidates in the order A=(h-1,v), B=(h,v-1), C=(h+1,v-1), T=previous
 *    field at X (Fig. 1, Fig. 3); a missing one is (0,0); each is clamped
 *    into the valid set V; the first strict minimum wins (the garbled
 *    Min[...] of Fig. 1 read as a minimum over A, B, C, T).
 *  - V: the displaced block lies inside the reference frame and each
 *    component is at most S pixels (Table 1's ES count fixes this).
 *  - Half-sample positions use MPEG-4 bilinear interpolation with rounding
 *    control 0.  Shape costs use the full-pel part trunc(d/h).
 *  - PRS on opaque MBs only, gradient of the current frame by central
 *    differences (Eq. 5), u = 1/gradient when |gradient| >= Theta else 0
 *    (Eq. 4), the block update = -eps * mean of DPD*u over pixels with u != 0
 *    (Eq. 3), DPD(d,p) = ref(p+d) - cur(p).  The mean uses a contiguous
 *    pairwise summation tree in FP32.  A proposal that lowers the SAD is
 *    taken; otherwise the eight neighbours at one MV unit are tried (Fig. 4);
 *    the loop stops when neither lowers the SAD or after max_iters steps.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef struct {
    int16_t dx, dy;
} orc_mv;

typedef struct {
    int width, height;  /* multiples of 16 */
    int search_range;   /* S, pixels */
    int subpel;         /* h = 1 (full-pel) or 2 (half-pel); MV unit = 1/h px */
    float theta;        /* Theta of Eq. 4 */
    float epsilon;      /* convergence factor of Eq. 2 */
    int max_iters;      /* cap on PRS iterations */
    int boundary_t_texture; /* variant of Sec. 3.1 (see orc_estimate_pair); 0 = Fig. 1 */
} orc_params;

enum { ORC_TRANSPARENT = 0, ORC_OPAQUE = 1, ORC_BOUNDARY = 2 };

static int imin(int a, int b) { return a < b ? a : b; }
static int imax(int a, int b) { return a > b ? a : b; }
static int iclamp(int v, int lo, int hi) { return v < lo ? lo : (v > hi ? hi : v); }

/* ------------------------------------------------------------------ */
/* Valid set V (Table 1's exhaustive-search count fixes it): the block  */
/* of size `block` at (X0, Y0) displaced by d (MV units 1/h px) lies     */
/* inside the frame, and |d| <= S*h per component.                       */
/* ------------------------------------------------------------------ */
void orc_valid_range(int W, int H, int block, int S, int h, int X0, int Y0,
                     int* lox, int* hix, int* loy, int* hiy)
{
    *lox = imax(-S * h, -X0 * h);
    *hix = imin(S * h, (W - block - X0) * h);
    *loy = imax(-S * h, -Y0 * h);
    *hiy = imin(S * h, (H - block - Y0) * h);
}

/* Reference sample at a position given in 1/h pixel units (x2, y2).
 * MPEG-4 bilinear half-sample interpolation, rounding control 0:
 * (a+b+1)>>1 on one axis, (a+b+c+d+2)>>2 on the diagonal. */
static int ref_sample(const uint8_t* ref, int W, int h, int x2, int y2)
{
    if (h == 1) return ref[(size_t)y2 * W + x2];
    int fx = x2 & 1, fy = y2 & 1;
    int ix = (x2 - fx) / 2, iy = (y2 - fy) / 2;
    const uint8_t* r = ref + (size_t)iy * W + ix;
    int a = r[0];
    if (!fx && !fy) return a;
    if (fx && !fy) return (a + r[1] + 1) >> 1;
    if (!fx && fy) return (a + r[W] + 1) >> 1;
    return (a + r[1] + r[W] + r[W + 1] + 2) >> 2;
}

int orc_interp(const uint8_t* ref, int W, int h, int x2, int y2)
{
    return ref_sample(ref, W, h, x2, y2);
}

/* Fig. 1, opaque branch: SAD between the current 16x16 block at (X0,Y0)
 * and the reference block displaced by d. */
uint32_t orc_texture_sad(const uint8_t* ref, const uint8_t* cur, int W, int h,
                         int X0, int Y0, int dx, int dy)
{
    uint32_t s = 0;
    for (int j = 0; j < 16; ++j)
        for (int i = 0; i < 16; ++i) {
            int x = X0 + i, y = Y0 + j;
            int p = ref_sample(ref, W, h, x * h + dx, y * h + dy);
            int c = cur[(size_t)y * W + x];
            s += (uint32_t)abs(p - c);
        }
    return s;
}

/* General block size variant (exhaustive search with 8x8 blocks). */
static uint32_t block_sad(const uint8_t* ref, const uint8_t* cur, int W, int h,
                          int block, int X0, int Y0, int dx, int dy)
{
    uint32_t s = 0;
    for (int j = 0; j < block; ++j)
        for (int i = 0; i < block; ++i) {
            int x = X0 + i, y = Y0 + j;
            int p = ref_sample(ref, W, h, x * h + dx, y * h + dy);
            s += (uint32_t)abs(p - (int)cur[(size_t)y * W + x]);
        }
    return s;
}

/* Fig. 1, boundary branch: number of pixels of the 16x16 binary alpha
 * block whose inside/outside state differs between the current BAB and the
 * reference BAB displaced by the full-pel part of d (trunc toward zero). */
uint32_t orc_shape_sad(const uint8_t* aref, const uint8_t* acur, int W, int h,
                       int X0, int Y0, int dx, int dy)
{
    int fx = dx / h, fy = dy / h; /* C division truncates toward zero */
    uint32_t s = 0;
    for (int j = 0; j < 16; ++j)
        for (int i = 0; i < 16; ++i) {
            int x = X0 + i, y = Y0 + j;
            int c = acur[(size_t)y * W + x] != 0;
            int r = aref[(size_t)(y + fy) * W + (x + fx)] != 0;
            s += (uint32_t)(c != r);
        }
    return s;
}

/* Fig. 1 "Type = Block_Type[h,v]": class of the MB from its BAB. */
int orc_classify_mb(const uint8_t* alpha, int W, int X0, int Y0)
{
    int n = 0;
    for (int j = 0; j < 16; ++j)
        for (int i = 0; i < 16; ++i)
            n += alpha[(size_t)(Y0 + j) * W + X0 + i] != 0;
    if (n == 0) return ORC_TRANSPARENT;
    if (n == 256) return ORC_OPAQUE;
    return ORC_BOUNDARY;
}

void orc_classify_frame(const uint8_t* alpha, int W, int H, uint8_t* out)
{
    int mbw = W / 16, mbh = H / 16;
    for (int v = 0; v < mbh; ++v)
        for (int u = 0; u < mbw; ++u)
            out[v * mbw + u] = (uint8_t)orc_classify_mb(alpha, W, 16 * u, 16 * v);
}

/* Contiguous pairwise sum of n = 2^k terms: level by level, element i
 * absorbs element i + s for s = 1, 2, 4, ...  FP32 round to nearest. */
static float pairwise_sum(float* t, int n)
{
    for (int s = 1; s < n; s *= 2)
        for (int i = 0; i + s < n; i += 2 * s) t[i] = t[i] + t[i + s];
    return t[0];
}

/* Sec. 3.2, Eqs. 3-5: one gradient update of the block displacement at d.
 * Returns the update in pixels in out[0] (x) and out[1] (y).
 *   gradient (Eq. 5): g = f(x+1,y) - f(x-1,y) on the current frame, i.e.
 *     twice the central difference; pixels on the first/last column (row)
 *     have no central difference and get u = 0.
 *   Eq. 4: u = 1 / (g/2) = 2/g when |g/2| >= Theta, else 0.
 *   Eq. 3: the per-pixel update is -eps * DPD(d,p) * u(p), with
 *     DPD(d,p) = ref(p+d) - cur(p); the block update is its mean over the
 *     pixels with u != 0. */
void orc_gradient_step(const orc_params* P, const uint8_t* ref, const uint8_t* cur,
                       int X0, int Y0, int dx, int dy, float out[2])
{
    const int W = P->width, H = P->height, h = P->subpel;
    float tx[256], ty[256];
    int nx = 0, ny = 0;
    const float lim = 2.0f * P->theta;
    for (int j = 0; j < 16; ++j)
        for (int i = 0; i < 16; ++i) {
            int x = X0 + i, y = Y0 + j;
            int dpd = ref_sample(ref, W, h, x * h + dx, y * h + dy) - (int)cur[(size_t)y * W + x];
            float ux = 0.0f, uy = 0.0f;
            if (x > 0 && x < W - 1) {
                int g = (int)cur[(size_t)y * W + x + 1] - (int)cur[(size_t)y * W + x - 1];
                if ((float)abs(g) >= lim) ux = 2.0f / (float)g;
            }
            if (y > 0 && y < H - 1) {
                int g = (int)cur[(size_t)(y + 1) * W + x] - (int)cur[(size_t)(y - 1) * W + x];
                if ((float)abs(g) >= lim) uy = 2.0f / (float)g;
            }
            nx += ux != 0.0f;
            ny += uy != 0.0f;
            tx[j * 16 + i] = (float)dpd * ux;
            ty[j * 16 + i] = (float)dpd * uy;
        }
    float sx = pairwise_sum(tx, 256), sy = pairwise_sum(ty, 256);
    out[0] = nx ? -(P->epsilon * (sx / (float)nx)) : 0.0f;
    out[1] = ny ? -(P->epsilon * (sy / (float)ny)) : 0.0f;
}

/* Distinct MV positions whose cost was evaluated for one MB (the quantity
 * averaged in Table 1). */
typedef struct {
    int n;
    int32_t pos[512];
} pos_set;

static void pos_note(pos_set* s, int dx, int dy)
{
    int32_t key = (int32_t)(((uint32_t)(uint16_t)dx) | ((uint32_t)(uint16_t)dy << 16));
    for (int k = 0; k < s->n; ++k)
        if (s->pos[k] == key) return;
    if (s->n < 512) s->pos[s->n++] = key;
}

static uint32_t mb_cost(const orc_params* P, int cls, const uint8_t* ref, const uint8_t* cur,
                        const uint8_t* aref, const uint8_t* acur, int X0, int Y0, int dx, int dy)
{
    if (cls == ORC_BOUNDARY) return orc_shape_sad(aref, acur, P->width, P->subpel, X0, Y0, dx, dy);
    return orc_texture_sad(ref, cur, P->width, P->subpel, X0, Y0, dx, dy);
}

/* Sec. 3.2 pixel recursive search from (dx, dy) with SAD c: gradient step,
 * proposal, eight directions (Fig. 4), repeated while the SAD drops, at most
 * max_iters steps.  Updates the vector and SAD, returns the steps taken and
 * the last update in last[2]; evaluated positions go to ps. */
static int prs_search(const orc_params* P, const uint8_t* ref, const uint8_t* cur, int X0, int Y0,
                      int lox, int hix, int loy, int hiy, int* pdx, int* pdy, uint32_t* pc,
                      float last[2], pos_set* ps)
{
    const int W = P->width, h = P->subpel;
    int dx = *pdx, dy = *pdy, k = 0;
    uint32_t c = *pc;
    last[0] = last[1] = 0.0f;
    while (k < P->max_iters) {
        ++k;
        orc_gradient_step(P, ref, cur, X0, Y0, dx, dy, last);
        int qx = iclamp(dx + (int)roundf((float)h * last[0]), lox, hix);
        int qy = iclamp(dy + (int)roundf((float)h * last[1]), loy, hiy);
        if (qx != dx || qy != dy) {
            uint32_t cq = orc_texture_sad(ref, cur, W, h, X0, Y0, qx, qy);
            pos_note(ps, qx, qy);
            if (cq < c) { dx = qx; dy = qy; c = cq; continue; }
        }
        /* Fig. 4: the eight directions at one MV unit */
        int bx = dx, by = dy;
        uint32_t bcost = c;
        for (int jj = -1; jj <= 1; ++jj)
            for (int ii = -1; ii <= 1; ++ii) {
                if (!ii && !jj) continue;
                int nx = iclamp(dx + ii, lox, hix), ny = iclamp(dy + jj, loy, hiy);
                if (nx == dx && ny == dy) continue;
                uint32_t cn = orc_texture_sad(ref, cur, W, h, X0, Y0, nx, ny);
                pos_note(ps, nx, ny);
                if (cn < bcost) { bcost = cn; bx = nx; by = ny; }
            }
        if (bcost < c) { dx = bx; dy = by; c = bcost; continue; }
        break;
    }
    *pdx = dx;
    *pdy = dy;
    *pc = c;
    return k;
}

/* One frame pair, Fig. 1: raster scan over the MB grid (Sec. 3.1).
 * With seeds (the learned proposal), the seed is a fifth candidate after T;
 * on an opaque MB whose seed strictly wins the candidate comparison, the
 * pixel recursive search runs from the seed and from the best of A, B, C, T,
 * and the seeded result is kept only if its final SAD is strictly lower (the
 * plain search stays the fallback).  Steps and update are those of the kept
 * search; the evaluated positions of both count. */
int orc_estimate_pair(const orc_params* P, const uint8_t* ref, const uint8_t* cur,
                      const uint8_t* aref, const uint8_t* acur,
                      const orc_mv* temporal, const float* seed,
                      orc_mv* mv, uint32_t* cost, float* disp, uint8_t* iters,
                      uint8_t* npos, uint8_t* mbclass)
{
    const int W = P->width, H = P->height, h = P->subpel, S = P->search_range;
    if (W <= 0 || H <= 0 || W % 16 || H % 16) return 1;
    if (h != 1 && h != 2) return 1;
    /* With seeds an MB may run two searches of up to 1 + 8 positions per
     * step; the distinct-position count (a byte) is guaranteed below 256 only
     * up to 8 steps (5 + 2 * 9 * 8 = 149), so seeded runs cap the steps there. */
    if (seed && P->max_iters > 8) return 1;
    const int mbw = W / 16, mbh = H / 16;
    for (int v = 0; v < mbh; ++v)
        for (int u = 0; u < mbw; ++u) {
            const int m = v * mbw + u, X0 = 16 * u, Y0 = 16 * v;
            const int cls = orc_classify_mb(acur, W, X0, Y0);
            mbclass[m] = (uint8_t)cls;
            if (cls == ORC_TRANSPARENT) { /* Fig. 1: no vector computed */
                mv[m].dx = mv[m].dy = 0;
                cost[m] = 0;
                disp[2 * m] = disp[2 * m + 1] = 0.0f;
                iters[m] = 0;
                npos[m] = 0;
                continue;
            }
            int lox, hix, loy, hiy;
            orc_valid_range(W, H, 16, S, h, X0, Y0, &lox, &hix, &loy, &hiy);
            int cx[5] = {0, 0, 0, 0, 0}, cy[5] = {0, 0, 0, 0, 0};
            if (u > 0) { cx[0] = mv[m - 1].dx; cy[0] = mv[m - 1].dy; }                      /* A */
            if (v > 0) { cx[1] = mv[m - mbw].dx; cy[1] = mv[m - mbw].dy; }                  /* B */
            if (v > 0 && u < mbw - 1) { cx[2] = mv[m - mbw + 1].dx; cy[2] = mv[m - mbw + 1].dy; } /* C */
            if (temporal) { cx[3] = temporal[m].dx; cy[3] = temporal[m].dy; }              /* T */
            int nc = 4;
            if (seed) { /* injected proposal: saturated to +-1024 MV units, rounded to the grid */
                cx[4] = (int)roundf(fminf(fmaxf((float)h * seed[2 * m], -1024.0f), 1024.0f));
                cy[4] = (int)roundf(fminf(fmaxf((float)h * seed[2 * m + 1], -1024.0f), 1024.0f));
                nc = 5;
            }
            pos_set ps;
            ps.n = 0;
            int best = -1;
            uint32_t bc = 0, costs[5] = {0, 0, 0, 0, 0};
            for (int k = 0; k < nc; ++k) {
                cx[k] = iclamp(cx[k], lox, hix);
                cy[k] = iclamp(cy[k], loy, hiy);
                uint32_t c = mb_cost(P, cls, ref, cur, aref, acur, X0, Y0, cx[k], cy[k]);
                costs[k] = c;
                pos_note(&ps, cx[k], cy[k]);
                if (best < 0 || c < bc) { best = k; bc = c; }
            }
            if (cls == ORC_BOUNDARY && P->boundary_t_texture) {
                /* Sec. 3.1's prose for boundary MBs: the spatial candidates are
                 * judged by shape, the temporal one by texture.  The winner of
                 * the others by shape (first strict minimum) and T are compared
                 * by texture SAD; T replaces it only if strictly lower.  The
                 * cost stays the shape cost of the vector kept. */
                int sb = -1;
                for (int q = 0; q < nc; ++q)
                    if (q != 3 && (sb < 0 || costs[q] < costs[sb])) sb = q;
                uint32_t tex_s = orc_texture_sad(ref, cur, W, h, X0, Y0, cx[sb], cy[sb]);
                uint32_t tex_t = orc_texture_sad(ref, cur, W, h, X0, Y0, cx[3], cy[3]);
                best = tex_t < tex_s ? 3 : sb;
                bc = costs[best];
            }
            int dx = cx[best], dy = cy[best];
            uint32_t c = bc;
            float last[2] = {0.0f, 0.0f};
            int k = 0;
            if (cls == ORC_OPAQUE && best == 4) {
                /* the seed won: search from it and from the plain winner */
                int pb = 0;
                for (int q = 1; q < 4; ++q)
                    if (costs[q] < costs[pb]) pb = q;
                int pdx = cx[pb], pdy = cy[pb];
                uint32_t pc = costs[pb];
                float plast[2];
                int pk = prs_search(P, ref, cur, X0, Y0, lox, hix, loy, hiy, &pdx, &pdy, &pc, plast, &ps);
                k = prs_search(P, ref, cur, X0, Y0, lox, hix, loy, hiy, &dx, &dy, &c, last, &ps);
                if (!(c < pc)) { /* the plain search is kept unless the seeded one is strictly better */
                    dx = pdx; dy = pdy; c = pc; k = pk;
                    last[0] = plast[0]; last[1] = plast[1];
                }
            } else if (cls == ORC_OPAQUE) {
                k = prs_search(P, ref, cur, X0, Y0, lox, hix, loy, hiy, &dx, &dy, &c, last, &ps);
            }
            mv[m].dx = (int16_t)dx;
            mv[m].dy = (int16_t)dy;
            cost[m] = c;
            disp[2 * m] = last[0];
            disp[2 * m + 1] = last[1];
            iters[m] = (uint8_t)k;
            npos[m] = (uint8_t)ps.n;
        }
    return 0;
}

/* Motion compensation (Sec. 4): pred(p) = ref(p + MV(mb(p))); returns the
 * sum of squared errors against cur.  Every MV must lie in V; returns
 * UINT64_MAX otherwise. */
uint64_t orc_compensate(const orc_params* P, const uint8_t* ref, const uint8_t* cur,
                        const orc_mv* mv, uint8_t* pred)
{
    const int W = P->width, H = P->height, h = P->subpel, mbw = W / 16;
    uint64_t sse = 0;
    for (int v = 0; v < H / 16; ++v)
        for (int u = 0; u < mbw; ++u) {
            int lox, hix, loy, hiy;
            orc_valid_range(W, H, 16, P->search_range, h, 16 * u, 16 * v, &lox, &hix, &loy, &hiy);
            const orc_mv d = mv[v * mbw + u];
            if (d.dx < lox || d.dx > hix || d.dy < loy || d.dy > hiy) return UINT64_MAX;
        }
    for (int y = 0; y < H; ++y)
        for (int x = 0; x < W; ++x) {
            const orc_mv d = mv[(y / 16) * mbw + x / 16];
            int p = ref_sample(ref, W, h, x * h + d.dx, y * h + d.dy);
            int e = (int)cur[(size_t)y * W + x] - p;
            sse += (uint64_t)(e * e);
            if (pred) pred[(size_t)y * W + x] = (uint8_t)p;
        }
    return sse;
}

/* PSNR of an 8-bit frame of W*H pixels from its SSE, in dB. */
double orc_psnr(uint64_t sse, int W, int H)
{
    if (sse == 0) return INFINITY;
    return 10.0 * log10(255.0 * 255.0 * (double)W * (double)H / (double)sse);
}

/* A whole sequence: pair k uses frame k as reference and frame
 * k + ref_distance as current; the temporal candidate of pair k is the
 * field of pair k-1 (temporal_in for k = 0; NULL means zero vectors).
 * Outputs are [P][M] with P = F - ref_distance pairs. */
int orc_estimate_sequence(const orc_params* P, const uint8_t* luma, const uint8_t* alpha,
                          int n_frames, int ref_distance, const orc_mv* temporal_in,
                          const float* seed, orc_mv* mv, uint32_t* cost, float* disp,
                          uint8_t* iters, uint8_t* npos, uint8_t* mbclass, uint64_t* sse,
                          uint8_t* pred)
{
    const size_t fs = (size_t)P->width * P->height;
    const int M = (P->width / 16) * (P->height / 16);
    const int np = n_frames - ref_distance;
    if (ref_distance < 1 || np < 1) return 1;
    for (int k = 0; k < np; ++k) {
        const uint8_t* ref = luma + fs * k;
        const uint8_t* cur = luma + fs * (k + ref_distance);
        const uint8_t* aref = alpha + fs * k;
        const uint8_t* acur = alpha + fs * (k + ref_distance);
        const orc_mv* tmp = k == 0 ? temporal_in : mv + (size_t)(k - 1) * M;
        int rc = orc_estimate_pair(P, ref, cur, aref, acur, tmp,
                                   seed ? seed + (size_t)2 * k * M : NULL,
                                   mv + (size_t)k * M, cost + (size_t)k * M,
                                   disp + (size_t)2 * k * M, iters + (size_t)k * M,
                                   npos + (size_t)k * M, mbclass + (size_t)k * M);
        if (rc) return rc;
        sse[k] = orc_compensate(P, ref, cur, mv + (size_t)k * M, pred ? pred + fs * k : NULL);
    }
    return 0;
}

/* Exhaustive search (ES) over V for blocks of size `block` on the whole
 * frame grid; raster order dy outer, dx inner, first strict minimum.
 * Writes the best vector and SAD per block and returns the total number of
 * positions compared (Table 1's ES row is that total over the block count). */
uint64_t orc_full_search(const uint8_t* ref, const uint8_t* cur, int W, int H, int h,
                         int S, int block, orc_mv* best_mv, uint32_t* best_sad)
{
    uint64_t total = 0;
    const int bw = W / block, bh = H / block;
    for (int v = 0; v < bh; ++v)
        for (int u = 0; u < bw; ++u) {
            int X0 = u * block, Y0 = v * block, lox, hix, loy, hiy;
            orc_valid_range(W, H, block, S, h, X0, Y0, &lox, &hix, &loy, &hiy);
            uint32_t bs = UINT32_MAX;
            int bx = 0, by = 0;
            for (int dy = loy; dy <= hiy; ++dy)
                for (int dx = lox; dx <= hix; ++dx) {
                    ++total;
                    if (!ref || !cur) continue;
                    uint32_t s = block_sad(ref, cur, W, h, block, X0, Y0, dx, dy);
                    if (s < bs) { bs = s; bx = dx; by = dy; }
                }
            if (best_mv) { best_mv[v * bw + u].dx = (int16_t)bx; best_mv[v * bw + u].dy = (int16_t)by; }
            if (best_sad) best_sad[v * bw + u] = bs;
        }
    return total;
}

/* ================================================================== */
/* Four motion vectors per macroblock (Sec. 3.2: MPEG-4 allows four    */
/* vectors per MB, so the recursive search works on 8x8 blocks).        */
/* Readings taken here:                                                 */
/*  - The block recursive search stays at MB level exactly as in Fig. 1 */
/*    (classes, 16x16 costs, first strict minimum of A, B, C, T); its   */
/*    winner starts the pixel recursive search of each 8x8 block        */
/*    b = 2*by + bx (raster order inside the MB), and every block keeps */
/*    its own vector.                                                   */
/*  - A neighbouring MB contributes the vector of its block nearest to  */
/*    the first block of the current MB (the MPEG-4 predictor layout):  */
/*    A = block 1 of the left MB, B = block 2 of the MB above, C = block */
/*    2 of the MB above-right, T = block 0 of the same MB in the        */
/*    previous field.                                                   */
/*  - Block searches use the MB's valid set V; the gradient step of     */
/*    Eqs. 3-5 runs over the block's 64 pixels, summed by the contiguous */
/*    pairwise tree in block raster order.                              */
/*  - Boundary MBs: the winner for all four blocks, each block costed by */
/*    the alpha mismatches of its own quadrant; transparent MBs: zero.  */
/*  - Positions of a block (Table 1 counts per 8x8 block): the distinct */
/*    MB candidates plus the block's own PRS positions.                 */
/* Arrays are [M][4] (block-major inside each MB).                      */
/* ================================================================== */

/* Eqs. 3-5 over the n x n block at (X0, Y0): as orc_gradient_step, for a
 * block of any size n (n*n a power of two, at most 256). */
void orc_gradient_step_block(const orc_params* P, const uint8_t* ref, const uint8_t* cur,
                             int X0, int Y0, int n, int dx, int dy, float out[2])
{
    const int W = P->width, H = P->height, h = P->subpel;
    float tx[256], ty[256];
    int nx = 0, ny = 0;
    const float lim = 2.0f * P->theta;
    for (int j = 0; j < n; ++j)
        for (int i = 0; i < n; ++i) {
            int x = X0 + i, y = Y0 + j;
            int dpd = ref_sample(ref, W, h, x * h + dx, y * h + dy) - (int)cur[(size_t)y * W + x];
            float ux = 0.0f, uy = 0.0f;
            if (x > 0 && x < W - 1) {
                int g = (int)cur[(size_t)y * W + x + 1] - (int)cur[(size_t)y * W + x - 1];
                if ((float)abs(g) >= lim) ux = 2.0f / (float)g;
            }
            if (y > 0 && y < H - 1) {
                int g = (int)cur[(size_t)(y + 1) * W + x] - (int)cur[(size_t)(y - 1) * W + x];
                if ((float)abs(g) >= lim) uy = 2.0f / (float)g;
            }
            nx += ux != 0.0f;
            ny += uy != 0.0f;
            tx[j * n + i] = (float)dpd * ux;
            ty[j * n + i] = (float)dpd * uy;
        }
    float sx = pairwise_sum(tx, n * n), sy = pairwise_sum(ty, n * n);
    out[0] = (nx > 0) ? -(P->epsilon * (sx / (float)nx)) : 0.0f;
    out[1] = (ny > 0) ? -(P->epsilon * (sy / (float)ny)) : 0.0f;
}

/* Alpha mismatches over the n x n block at (X0, Y0), reference displaced by
 * the full-pel part of d (trunc toward zero), as orc_shape_sad. */
static uint32_t shape_block(const uint8_t* aref, const uint8_t* acur, int W, int h, int n,
                            int X0, int Y0, int dx, int dy)
{
    int fx = dx / h, fy = dy / h;
    uint32_t s = 0;
    for (int j = 0; j < n; ++j)
        for (int i = 0; i < n; ++i) {
            int x = X0 + i, y = Y0 + j;
            s += (uint32_t)((acur[(size_t)y * W + x] != 0) != (aref[(size_t)(y + fy) * W + (x + fx)] != 0));
        }
    return s;
}

/* Sec. 3.2 pixel recursive search of the n x n block at (X0, Y0), the same
 * loop as prs_search with the block's SAD and gradient step. */
static int prs_block(const orc_params* P, const uint8_t* ref, const uint8_t* cur, int X0, int Y0, int n,
                     int lox, int hix, int loy, int hiy, int* pdx, int* pdy, uint32_t* pc,
                     float last[2], pos_set* ps)
{
    const int W = P->width, h = P->subpel;
    int dx = *pdx, dy = *pdy, k = 0;
    uint32_t c = *pc;
    last[0] = last[1] = 0.0f;
    while (k < P->max_iters) {
        ++k;
        orc_gradient_step_block(P, ref, cur, X0, Y0, n, dx, dy, last);
        int qx = iclamp(dx + (int)roundf((float)h * last[0]), lox, hix);
        int qy = iclamp(dy + (int)roundf((float)h * last[1]), loy, hiy);
        if (qx != dx || qy != dy) {
            uint32_t cq = block_sad(ref, cur, W, h, n, X0, Y0, qx, qy);
            pos_note(ps, qx, qy);
            if (cq < c) { dx = qx; dy = qy; c = cq; continue; }
        }
        int bx = dx, by = dy;
        uint32_t bcost = c;
        for (int jj = -1; jj <= 1; ++jj)
            for (int ii = -1; ii <= 1; ++ii) {
                if (!ii && !jj) continue;
                int nx = iclamp(dx + ii, lox, hix), ny = iclamp(dy + jj, loy, hiy);
                if (nx == dx && ny == dy) continue;
                uint32_t cn = block_sad(ref, cur, W, h, n, X0, Y0, nx, ny);
                pos_note(ps, nx, ny);
                if (cn < bcost) { bcost = cn; bx = nx; by = ny; }
            }
        if (bcost < c) { dx = bx; dy = by; c = bcost; continue; }
        break;
    }
    *pdx = dx;
    *pdy = dy;
    *pc = c;
    return k;
}

/* One frame pair with four vectors per MB; temporal4 is the previous
 * field [M][4] (NULL: zero vectors).  Outputs [M][4] except mbclass [M]. */
int orc_estimate_pair4(const orc_params* P, const uint8_t* ref, const uint8_t* cur,
                       const uint8_t* aref, const uint8_t* acur, const orc_mv* temporal4,
                       orc_mv* mv4, uint32_t* cost4, float* disp4, uint8_t* iters4,
                       uint8_t* npos4, uint8_t* mbclass)
{
    const int W = P->width, H = P->height, h = P->subpel, S = P->search_range;
    if (W <= 0 || H <= 0 || W % 16 || H % 16) return 1;
    if (h != 1 && h != 2) return 1;
    const int mbw = W / 16, mbh = H / 16;
    for (int v = 0; v < mbh; ++v)
        for (int u = 0; u < mbw; ++u) {
            const int m = v * mbw + u, X0 = 16 * u, Y0 = 16 * v;
            const int cls = orc_classify_mb(acur, W, X0, Y0);
            mbclass[m] = (uint8_t)cls;
            if (cls == ORC_TRANSPARENT) {
                for (int b = 0; b < 4; ++b) {
                    mv4[4 * m + b].dx = mv4[4 * m + b].dy = 0;
                    cost4[4 * m + b] = 0;
                    disp4[8 * m + 2 * b] = disp4[8 * m + 2 * b + 1] = 0.0f;
                    iters4[4 * m + b] = 0;
                    npos4[4 * m + b] = 0;
                }
                continue;
            }
            int lox, hix, loy, hiy;
            orc_valid_range(W, H, 16, S, h, X0, Y0, &lox, &hix, &loy, &hiy);
            int cx[4] = {0, 0, 0, 0}, cy[4] = {0, 0, 0, 0};
            if (u > 0) { cx[0] = mv4[4 * (m - 1) + 1].dx; cy[0] = mv4[4 * (m - 1) + 1].dy; }   /* A */
            if (v > 0) { cx[1] = mv4[4 * (m - mbw) + 2].dx; cy[1] = mv4[4 * (m - mbw) + 2].dy; } /* B */
            if (v > 0 && u < mbw - 1) {                                                       /* C */
                cx[2] = mv4[4 * (m - mbw + 1) + 2].dx;
                cy[2] = mv4[4 * (m - mbw + 1) + 2].dy;
            }
            if (temporal4) { cx[3] = temporal4[4 * m].dx; cy[3] = temporal4[4 * m].dy; }      /* T */
            pos_set brs;
            brs.n = 0;
            int best = -1;
            uint32_t bc = 0;
            for (int k = 0; k < 4; ++k) {
                cx[k] = iclamp(cx[k], lox, hix);
                cy[k] = iclamp(cy[k], loy, hiy);
                uint32_t c = mb_cost(P, cls, ref, cur, aref, acur, X0, Y0, cx[k], cy[k]);
                pos_note(&brs, cx[k], cy[k]);
                if (best < 0 || c < bc) { best = k; bc = c; }
            }
            for (int b = 0; b < 4; ++b) {
                const int BX = X0 + 8 * (b & 1), BY = Y0 + 8 * (b >> 1);
                int dx = cx[best], dy = cy[best], k = 0;
                float last[2] = {0.0f, 0.0f};
                uint32_t c;
                pos_set ps = brs;
                if (cls == ORC_BOUNDARY) {
                    c = shape_block(aref, acur, W, h, 8, BX, BY, dx, dy);
                } else {
                    c = block_sad(ref, cur, W, h, 8, BX, BY, dx, dy);
                    k = prs_block(P, ref, cur, BX, BY, 8, lox, hix, loy, hiy, &dx, &dy, &c, last, &ps);
                }
                mv4[4 * m + b].dx = (int16_t)dx;
                mv4[4 * m + b].dy = (int16_t)dy;
                cost4[4 * m + b] = c;
                disp4[8 * m + 2 * b] = last[0];
                disp4[8 * m + 2 * b + 1] = last[1];
                iters4[4 * m + b] = (uint8_t)k;
                npos4[4 * m + b] = (uint8_t)ps.n;
            }
        }
    return 0;
}

/* Motion compensation with four vectors per MB: pred(p) = ref(p + MV of the
 * 8x8 block holding p); the SSE against cur.  Every vector must lie in its
 * MB's V; returns UINT64_MAX otherwise. */
uint64_t orc_compensate4(const orc_params* P, const uint8_t* ref, const uint8_t* cur,
                         const orc_mv* mv4, uint8_t* pred)
{
    const int W = P->width, H = P->height, h = P->subpel, mbw = W / 16;
    uint64_t sse = 0;
    for (int v = 0; v < H / 16; ++v)
        for (int u = 0; u < mbw; ++u) {
            int lox, hix, loy, hiy;
            orc_valid_range(W, H, 16, P->search_range, h, 16 * u, 16 * v, &lox, &hix, &loy, &hiy);
            for (int b = 0; b < 4; ++b) {
                const orc_mv d = mv4[4 * (v * mbw + u) + b];
                if (d.dx < lox || d.dx > hix || d.dy < loy || d.dy > hiy) return UINT64_MAX;
            }
        }
    for (int y = 0; y < H; ++y)
        for (int x = 0; x < W; ++x) {
            const int b = 2 * ((y % 16) / 8) + (x % 16) / 8;
            const orc_mv d = mv4[4 * ((y / 16) * mbw + x / 16) + b];
            int p = ref_sample(ref, W, h, x * h + d.dx, y * h + d.dy);
            int e = (int)cur[(size_t)y * W + x] - p;
            sse += (uint64_t)(e * e);
            if (pred) pred[(size_t)y * W + x] = (uint8_t)p;
        }
    return sse;
}

/* A whole sequence with four vectors per MB (as orc_estimate_sequence; the
 * temporal candidate of pair k is block 0 of the field of pair k-1). */
int orc_estimate_sequence4(const orc_params* P, const uint8_t* luma, const uint8_t* alpha,
                           int n_frames, int ref_distance, const orc_mv* temporal_in4,
                           orc_mv* mv4, uint32_t* cost4, float* disp4, uint8_t* iters4,
                           uint8_t* npos4, uint8_t* mbclass, uint64_t* sse, uint8_t* pred)
{
    const size_t fs = (size_t)P->width * P->height;
    const int M = (P->width / 16) * (P->height / 16);
    const int np = n_frames - ref_distance;
    if (ref_distance < 1 || np < 1) return 1;
    for (int k = 0; k < np; ++k) {
        const uint8_t* ref = luma + fs * k;
        const uint8_t* cur = luma + fs * (k + ref_distance);
        const orc_mv* tmp = k == 0 ? temporal_in4 : mv4 + (size_t)4 * (k - 1) * M;
        int rc = orc_estimate_pair4(P, ref, cur, alpha + fs * k, alpha + fs * (k + ref_distance), tmp,
                                    mv4 + (size_t)4 * k * M, cost4 + (size_t)4 * k * M,
                                    disp4 + (size_t)8 * k * M, iters4 + (size_t)4 * k * M,
                                    npos4 + (size_t)4 * k * M, mbclass + (size_t)k * M);
        if (rc) return rc;
        sse[k] = orc_compensate4(P, ref, cur, mv4 + (size_t)4 * k * M, pred ? pred + fs * k : NULL);
    }
    return 0;
}
