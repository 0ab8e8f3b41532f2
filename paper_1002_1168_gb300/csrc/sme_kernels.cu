// Device kernels of the shape-adaptive motion estimation pass (sm_103a).
//
//   classify_pack_kernel  Fig. 1 "Block_Type": per-MB class from the binary
//                         alpha block + bit-packed alpha rows (one pass).
//   me_kernel             Fig. 1 / Sec. 3.1 / Sec. 3.2 for every MB of every
//                         frame pair of a sequence, one persistent launch:
//                         tickets in wavefront order, bounded waits on the
//                         A/B/C/T results, block recursive search (shape cost
//                         on boundary MBs, texture SAD on opaque MBs), pixel
//                         recursive gradient search (Eqs. 3-5, Fig. 4) and the
//                         fused motion compensation + SSE of Sec. 4.
//   compensate_kernel     Sec. 4 motion compensation of a given field.
//   query_kernel          Single cost / gradient evaluations through the same
//                         device functions as me_kernel (unit checks).
//
// One CTA of 256 threads handles one MB: thread t owns pixel (t & 15, t >> 4)
// of the 16x16 block, so block-wide sums over the 256 pixels follow the
// row-major pixel order.
#include <stdint.h>

#include "sme_internal.h"

namespace sme {
namespace {

constexpr int kThreads = 256;
constexpr unsigned kFull = 0xffffffffu;

// ------------------------------------------------------------------ sync --
__device__ __forceinline__ unsigned ld_acquire(const unsigned* p)
{
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ unsigned ld_relaxed(const unsigned* p)
{
    unsigned v;
    asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_release(unsigned* p, unsigned v)
{
    asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ unsigned long long globaltimer()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Spin until *flag == epoch.  Bounded by `timeout_ns` of %globaltimer and by
// an iteration cap; gives up early when another CTA raised the abort word.
__device__ bool wait_flag(const unsigned* flag, unsigned epoch, const DevStatus* st,
                          long long timeout_ns)
{
    if (ld_acquire(flag) == epoch) return true;
    const unsigned long long t0 = globaltimer();
    for (unsigned it = 1; it < (1u << 24); ++it) {
        if (ld_acquire(flag) == epoch) return true;
        if ((it & 15u) == 0) {
            if (ld_relaxed(&st->abort)) return false;
            if ((long long)(globaltimer() - t0) > timeout_ns) return false;
        }
    }
    return false;
}

__device__ __forceinline__ void raise_error(DevStatus* st, int code, bool abort_launch)
{
    atomicCAS(&st->err, 0, code);
    if (abort_launch) atomicExch(&st->abort, 1u);
}

// ------------------------------------------------------------ reductions --
// Integer block sums of N per-thread values (every thread gets the totals).
// `red` is one of two alternating [16][8] buffers: one barrier per call.
template <int N>
__device__ __forceinline__ void block_sum(unsigned (&v)[N], unsigned (*red)[8], int lane, int warp)
{
#pragma unroll
    for (int c = 0; c < N; ++c) {
        unsigned s = __reduce_add_sync(kFull, v[c]);
        if (lane == 0) red[c][warp] = s;
    }
    __syncthreads();
#pragma unroll
    for (int c = 0; c < N; ++c) {
        unsigned s = 0;
#pragma unroll
        for (int w = 0; w < 8; ++w) s += red[c][w];
        v[c] = s;
    }
}

// FP32 sum of one term per thread over the 256 pixels as a contiguous
// pairwise tree in row-major pixel order: within a warp, offsets 1..16 pair
// neighbouring partial sums; across the eight warps ((w0+w1)+(w2+w3)) +
// ((w4+w5)+(w6+w7)).  Round-to-nearest adds only (no contraction).
__device__ __forceinline__ void tree_sum2(float& a, float& b, float (*red)[8], int lane, int warp)
{
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        float pa = __shfl_down_sync(kFull, a, o);
        float pb = __shfl_down_sync(kFull, b, o);
        a = __fadd_rn(a, pa);
        b = __fadd_rn(b, pb);
    }
    if (lane == 0) {
        red[0][warp] = a;
        red[1][warp] = b;
    }
    __syncthreads();
    float r[2];
#pragma unroll
    for (int c = 0; c < 2; ++c) {
        const float* p = red[c];
        r[c] = __fadd_rn(__fadd_rn(__fadd_rn(p[0], p[1]), __fadd_rn(p[2], p[3])),
                         __fadd_rn(__fadd_rn(p[4], p[5]), __fadd_rn(p[6], p[7])));
    }
    a = r[0];
    b = r[1];
}

// --------------------------------------------------------------- geometry --
__device__ __forceinline__ int ceil16(int v) { return (v + 15) & ~15; }
__device__ __forceinline__ int win_pitch(const Geom& g) { return 16 + 2 * ceil16(g.S); }
__device__ __forceinline__ int clampi(int v, int lo, int hi) { return min(max(v, lo), hi); }
__device__ __forceinline__ int pack_mv(int dx, int dy)
{
    return (int)((unsigned)(dx & 0xffff) | ((unsigned)dy << 16));
}
__device__ __forceinline__ int mv_x(int key) { return (int)(short)(key & 0xffff); }
__device__ __forceinline__ int mv_y(int key) { return key >> 16; }

struct VRange {
    int lox, hix, loy, hiy;
};
// Valid set V of the MB at (X0, Y0): displaced block inside the frame and
// |d| <= S*h per component (MV units).
__device__ __forceinline__ VRange valid_range(const Geom& g, int X0, int Y0)
{
    VRange r;
    r.lox = max(-g.S * g.h, -X0 * g.h);
    r.hix = min(g.S * g.h, (g.W - 16 - X0) * g.h);
    r.loy = max(-g.S * g.h, -Y0 * g.h);
    r.hiy = min(g.S * g.h, (g.H - 16 - Y0) * g.h);
    return r;
}

// Stage the reference rows/columns every vector of V can touch into shared
// memory with coalesced 16-byte loads.  Window origin returned in wx0/wy0.
__device__ __forceinline__ void stage_window(uint8_t* win, const uint8_t* ref, const Geom& g,
                                             int X0, int Y0, int tid, int& wx0, int& wy0)
{
    const int cs = ceil16(g.S), pitch = win_pitch(g);
    wy0 = max(0, Y0 - g.S);
    const int wy1 = min(g.H - 1, Y0 + 15 + g.S);
    wx0 = max(0, X0 - cs);
    const int wx1 = min(g.W, X0 + 16 + cs);
    const int nch = (wx1 - wx0) >> 4, n = (wy1 - wy0 + 1) * nch;
    for (int c = tid; c < n; c += kThreads) {
        const int r = c / nch, ch = c - r * nch;
        const uint4 val = __ldg(reinterpret_cast<const uint4*>(ref + (size_t)(wy0 + r) * g.W + wx0 + 16 * ch));
        *reinterpret_cast<uint4*>(win + r * pitch + 16 * ch) = val;
    }
}

// Reference sample at this thread's pixel displaced by d, from the window.
// MPEG-4 bilinear half-sample interpolation, rounding control 0.
__device__ __forceinline__ int ref_at(const uint8_t* win, int pitch, int lx, int ly, int dx, int dy, int h)
{
    int ix = dx, iy = dy, fx = 0, fy = 0;
    if (h == 2) {
        ix = dx >> 1;
        iy = dy >> 1;
        fx = dx & 1;
        fy = dy & 1;
    }
    const uint8_t* r = win + (ly + iy) * pitch + lx + ix;
    const int a = r[0];
    if (fx) {
        const int b = r[1];
        if (fy) return (a + b + r[pitch] + r[pitch + 1] + 2) >> 2;
        return (a + b + 1) >> 1;
    }
    if (fy) return (a + r[pitch] + 1) >> 1;
    return a;
}

// Eq. 4 / Eq. 5 factors of this pixel: u = 2/g when |g| >= 2*Theta, g the
// central difference of the current frame (twice the derivative); 0 on the
// frame's outer rows/columns.
__device__ __forceinline__ void grad_factors(const uint8_t* cur, const Geom& g, int x, int y,
                                             float& ux, float& uy)
{
    ux = 0.0f;
    uy = 0.0f;
    const float lim = 2.0f * g.theta;
    const uint8_t* p = cur + (size_t)y * g.W + x;
    if (x > 0 && x < g.W - 1) {
        const int gx = (int)__ldg(p + 1) - (int)__ldg(p - 1);
        if (fabsf((float)gx) >= lim) ux = __fdiv_rn(2.0f, (float)gx);
    }
    if (y > 0 && y < g.H - 1) {
        const int gy = (int)__ldg(p + g.W) - (int)__ldg(p - g.W);
        if (fabsf((float)gy) >= lim) uy = __fdiv_rn(2.0f, (float)gy);
    }
}

// Eq. 3 block update from the pixel sums: -eps * mean over pixels with u != 0.
__device__ __forceinline__ float update_of(float sum, int n, float eps)
{
    return n ? -__fmul_rn(eps, __fdiv_rn(sum, (float)n)) : 0.0f;
}

// Alpha mismatches of one BAB row: current row bits vs the reference row
// displaced by the full-pel vector (fdx, fdy).
__device__ __forceinline__ unsigned shape_row(const uint32_t* pcur, const uint32_t* pref, const Geom& g,
                                              int X0, int Y0, int r, int fdx, int fdy)
{
    const uint32_t* rc = pcur + (size_t)(Y0 + r) * g.Wp;
    const unsigned cb = (__ldg(rc + (X0 >> 5)) >> (X0 & 31)) & 0xffffu;
    const int xr = X0 + fdx;
    const uint32_t* rr = pref + (size_t)(Y0 + r + fdy) * g.Wp;
    const unsigned rb = __funnelshift_r(__ldg(rr + (xr >> 5)), __ldg(rr + (xr >> 5) + 1), xr & 31) & 0xffffu;
    return __popc(cb ^ rb);
}

// ============================================================ classify ==
__global__ void __launch_bounds__(kThreads) classify_pack_kernel(const Geom g, const ClassifyArgs a)
{
    __shared__ unsigned cnt[kMaxDim / 16];
    const int v = blockIdx.x, f = blockIdx.y, tid = threadIdx.x;
    if (v == 0 && f == 0) {
        if (a.status && tid == 0) {
            a.status->ticket = 0;
            a.status->abort = 0;
        }
        if (a.sse)
            for (int i = tid; i < a.n_sse; i += kThreads) a.sse[i] = 0ull;
    }
    for (int i = tid; i < g.MBW; i += kThreads) cnt[i] = 0;
    __syncthreads();
    const size_t FS = (size_t)g.W * g.H;
    const uint8_t* al = a.alpha + (size_t)f * FS + (size_t)v * 16 * g.W;
    uint16_t* pk = a.packed ? reinterpret_cast<uint16_t*>(a.packed + ((size_t)f * g.H + v * 16) * g.Wp) : nullptr;
    const int segs = g.MBW, hw = 2 * g.Wp;  // 16-pixel segments per row; u16 slots per packed row
    for (int it = tid; it < 16 * hw; it += kThreads) {
        const int r = it / hw, s = it - r * hw;
        unsigned m = 0;
        if (s < segs) {
            const uint4 q = __ldg(reinterpret_cast<const uint4*>(al + (size_t)r * g.W + 16 * s));
            const unsigned w[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
            for (int b = 0; b < 4; ++b) {
                const unsigned nz = __vcmpne4(w[b], 0u) & 0x01010101u;  // 1 per nonzero byte
                const unsigned bits = (nz | (nz >> 7) | (nz >> 14) | (nz >> 21)) & 0xfu;
                m |= bits << (4 * b);
            }
            atomicAdd(&cnt[s], (unsigned)__popc(m));
        }
        if (pk) pk[(size_t)r * hw + s] = (uint16_t)m;
    }
    __syncthreads();
    for (int s = tid; s < segs; s += kThreads) {
        const unsigned n = cnt[s];
        a.cls[(size_t)f * g.M + v * g.MBW + s] =
            (uint8_t)(n == 0 ? SME_TRANSPARENT : (n == 256 ? SME_OPAQUE : SME_BOUNDARY));
    }
}

// ================================================================== ME ==
__global__ void __launch_bounds__(kThreads) me_kernel(const Geom g, const MeArgs a)
{
    extern __shared__ __align__(16) uint8_t win[];
    __shared__ int s_ticket, s_stop;
    __shared__ int s_cand[5];
    __shared__ unsigned s_cost[5];
    __shared__ unsigned s_red[2][16][8];
    __shared__ float s_fred[2][2][8];
    __shared__ int s_log[kMaxLog];

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int pi = tid & 15, pj = tid >> 4;
    const size_t FS = (size_t)g.W * g.H;
    const int pitch = win_pitch(g), h = g.h;
    int rb = 0;

    for (;;) {
        if (tid == 0) {
            int t = (int)atomicAdd(&a.status->ticket, 1u);
            if (ld_relaxed(&a.status->abort)) t = a.total;
            s_ticket = t;
            s_stop = 0;
        }
        __syncthreads();
        const int t = s_ticket;
        if (t >= a.total) break;
        const int idx = a.sched[t];
        const int k = idx / g.M, mb = idx - k * g.M;
        const int u = mb % g.MBW, v = mb / g.MBW;
        const int X0 = 16 * u, Y0 = 16 * v, x = X0 + pi, y = Y0 + pj;
        const uint8_t* ref = a.luma + (size_t)k * FS;
        const uint8_t* cur = a.luma + (size_t)(k + a.rd) * FS;
        const int cls = __ldg(a.cls + (size_t)(k + a.rd) * g.M + mb);
        const int cval = __ldg(cur + (size_t)y * g.W + x);

        if (cls == SME_TRANSPARENT) {
            // Fig. 1: no vector is computed; (0,0) is final at once.
            if (tid == 0) {
                a.mv[idx] = sme_mv{0, 0};
                if (t != a.fault_ticket) st_release(a.ready + idx, a.epoch);
                if (a.cost) a.cost[idx] = 0;
                if (a.disp) { a.disp[2 * idx] = 0.0f; a.disp[2 * idx + 1] = 0.0f; }
                if (a.iters) a.iters[idx] = 0;
                if (a.npos) a.npos[idx] = 0;
                if (a.out_cls) a.out_cls[idx] = (uint8_t)cls;
            }
            const int r = __ldg(ref + (size_t)y * g.W + x);
            unsigned sq[1] = {(unsigned)((cval - r) * (cval - r))};
            if (a.pred) a.pred[(size_t)k * FS + (size_t)y * g.W + x] = (uint8_t)r;
            if (a.sse || a.sse_mb) {
                block_sum<1>(sq, s_red[rb], lane, warp);
                rb ^= 1;
                if (tid == 0) {
                    if (a.sse) atomicAdd(a.sse + k, (unsigned long long)sq[0]);
                    if (a.sse_mb) a.sse_mb[idx] = sq[0];
                }
            }
            __syncthreads();
            continue;
        }

        // ---- work that does not depend on the neighbours: prefetch ----
        int wx0, wy0;
        stage_window(win, ref, g, X0, Y0, tid, wx0, wy0);
        const int lx = x - wx0, ly = y - wy0;
        float ux = 0.0f, uy = 0.0f;
        if (cls == SME_OPAQUE) grad_factors(cur, g, x, y, ux, uy);
        const int nx = __syncthreads_count(ux != 0.0f);
        const int ny = __syncthreads_count(uy != 0.0f);
        const VRange V = valid_range(g, X0, Y0);

        // ---- candidates A, B, C, T (Fig. 1, Fig. 3) + optional seed ----
        if (tid < 4) {
            int dep = -1;
            if (tid == 0 && u > 0) dep = idx - 1;                          // A
            if (tid == 1 && v > 0) dep = idx - g.MBW;                      // B
            if (tid == 2 && v > 0 && u < g.MBW - 1) dep = idx - g.MBW + 1; // C
            if (tid == 3 && k > 0) dep = idx - g.M;                        // T
            int key = 0;
            if (dep >= 0) {
                if (wait_flag(a.ready + dep, a.epoch, a.status, a.timeout_ns)) {
                    const unsigned raw = __ldcg(reinterpret_cast<const unsigned*>(a.mv + dep));
                    key = (int)raw;
                } else {
                    if (!ld_relaxed(&a.status->abort)) raise_error(a.status, SME_ERR_TIMEOUT, true);
                    atomicExch(&s_stop, 1);
                }
            } else if (tid == 3 && a.temporal_in) {
                key = (int)__ldg(reinterpret_cast<const unsigned*>(a.temporal_in + mb));
            }
            s_cand[tid] = pack_mv(clampi(mv_x(key), V.lox, V.hix), clampi(mv_y(key), V.loy, V.hiy));
        } else if (tid == 4 && a.seed) {
            const float sx = fminf(fmaxf(__fmul_rn((float)h, __ldg(a.seed + 2 * (size_t)idx)), -1024.0f), 1024.0f);
            const float sy = fminf(fmaxf(__fmul_rn((float)h, __ldg(a.seed + 2 * (size_t)idx + 1)), -1024.0f), 1024.0f);
            s_cand[4] = pack_mv(clampi((int)roundf(sx), V.lox, V.hix), clampi((int)roundf(sy), V.loy, V.hiy));
        }
        __syncthreads();
        if (s_stop) break;
        const int nc = a.seed ? 5 : 4;
        if (tid < nc) s_log[tid] = s_cand[tid];
        int nlog = nc;

        int dx, dy;
        unsigned cost;
        int iters = 0;
        float lastx = 0.0f, lasty = 0.0f;
        int diff;
        if (cls == SME_BOUNDARY) {
            // Fig. 1 boundary branch: alpha mismatch of the BABs.
            unsigned part = 0;
            if (tid < nc * 16) {
                const int key = s_cand[tid >> 4];
                const int fdx = mv_x(key) / h, fdy = mv_y(key) / h;  // trunc toward zero
                part = shape_row(a.packed + (size_t)(k + a.rd) * g.H * g.Wp, a.packed + (size_t)k * g.H * g.Wp,
                                 g, X0, Y0, tid & 15, fdx, fdy);
            }
            part += __shfl_xor_sync(kFull, part, 8);
            part += __shfl_xor_sync(kFull, part, 4);
            part += __shfl_xor_sync(kFull, part, 2);
            part += __shfl_xor_sync(kFull, part, 1);
            if (tid < nc * 16 && (tid & 15) == 0) s_cost[tid >> 4] = part;
            __syncthreads();
            int best = 0;
            for (int c = 1; c < nc; ++c)
                if (s_cost[c] < s_cost[best]) best = c;
            dx = mv_x(s_cand[best]);
            dy = mv_y(s_cand[best]);
            cost = s_cost[best];
            diff = ref_at(win, pitch, lx, ly, dx, dy, h) - cval;
        } else {
            // Fig. 1 opaque branch: texture SAD of the candidates.
            unsigned sad[5];
#pragma unroll
            for (int c = 0; c < 5; ++c) {
                const int key = s_cand[c < nc ? c : 0];
                sad[c] = c < nc ? (unsigned)abs(ref_at(win, pitch, lx, ly, mv_x(key), mv_y(key), h) - cval) : 0u;
            }
            block_sum<5>(sad, s_red[rb], lane, warp);
            rb ^= 1;
            int best = 0;
            unsigned bestc = sad[0];
#pragma unroll
            for (int c = 1; c < 5; ++c)
                if (c < nc && sad[c] < bestc) {
                    best = c;
                    bestc = sad[c];
                }
            dx = mv_x(s_cand[best]);
            dy = mv_y(s_cand[best]);
            cost = bestc;
            diff = ref_at(win, pitch, lx, ly, dx, dy, h) - cval;

            // Sec. 3.2: pixel recursive search.
            while (iters < g.K) {
                ++iters;
                float sx = __fmul_rn((float)diff, ux), sy = __fmul_rn((float)diff, uy);
                tree_sum2(sx, sy, s_fred[rb], lane, warp);
                rb ^= 1;
                lastx = update_of(sx, nx, g.eps);
                lasty = update_of(sy, ny, g.eps);
                const int qx = clampi(dx + (int)roundf(__fmul_rn((float)h, lastx)), V.lox, V.hix);
                const int qy = clampi(dy + (int)roundf(__fmul_rn((float)h, lasty)), V.loy, V.hiy);
                const bool qmove = (qx != dx) || (qy != dy);
                unsigned val[9];
                val[0] = qmove ? (unsigned)abs(ref_at(win, pitch, lx, ly, qx, qy, h) - cval) : 0u;
#pragma unroll
                for (int n = 1; n < 9; ++n) {
                    const int e = n < 5 ? n - 1 : n;  // skip the centre of the 3x3 raster
                    const int ii = e % 3 - 1, jj = e / 3 - 1;
                    const int ex = clampi(dx + ii, V.lox, V.hix), ey = clampi(dy + jj, V.loy, V.hiy);
                    val[n] = (ex != dx || ey != dy) ? (unsigned)abs(ref_at(win, pitch, lx, ly, ex, ey, h) - cval) : 0u;
                }
                block_sum<9>(val, s_red[rb], lane, warp);
                rb ^= 1;
                if (qmove) {
                    if (tid == 0) s_log[nlog] = pack_mv(qx, qy);
                    ++nlog;
                    if (val[0] < cost) {
                        dx = qx;
                        dy = qy;
                        cost = val[0];
                        diff = ref_at(win, pitch, lx, ly, dx, dy, h) - cval;
                        continue;
                    }
                }
                // Fig. 4: eight directions at one MV unit, first strict minimum.
                unsigned bc = cost;
                int bx = dx, by = dy;
#pragma unroll
                for (int n = 1; n < 9; ++n) {
                    const int e = n < 5 ? n - 1 : n;
                    const int ii = e % 3 - 1, jj = e / 3 - 1;
                    const int ex = clampi(dx + ii, V.lox, V.hix), ey = clampi(dy + jj, V.loy, V.hiy);
                    if (ex != dx || ey != dy) {
                        if (tid == 0) s_log[nlog] = pack_mv(ex, ey);
                        ++nlog;
                        if (val[n] < bc) {
                            bc = val[n];
                            bx = ex;
                            by = ey;
                        }
                    }
                }
                if (bc < cost) {
                    dx = bx;
                    dy = by;
                    cost = bc;
                    diff = ref_at(win, pitch, lx, ly, dx, dy, h) - cval;
                    continue;
                }
                break;
            }
        }

        // ---- publish the vector first: it is on the dependency chain ----
        if (tid == 0) {
            a.mv[idx] = sme_mv{(int16_t)dx, (int16_t)dy};
            if (t != a.fault_ticket) st_release(a.ready + idx, a.epoch);
            if (a.cost) a.cost[idx] = cost;
            if (a.disp) { a.disp[2 * idx] = lastx; a.disp[2 * idx + 1] = lasty; }
            if (a.iters) a.iters[idx] = (uint8_t)iters;
            if (a.out_cls) a.out_cls[idx] = (uint8_t)cls;
        }
        // ---- distinct evaluated positions (Table 1 unit) ----
        __syncthreads();
        int first = 0;
        if (tid < nlog) {
            const int key = s_log[tid];
            first = 1;
            for (int j = 0; j < tid; ++j)
                if (s_log[j] == key) { first = 0; break; }
        }
        const int np = __syncthreads_count(first);
        if (tid == 0 && a.npos) a.npos[idx] = (uint8_t)np;
        // ---- Sec. 4: motion-compensated prediction and its SSE ----
        if (a.pred) a.pred[(size_t)k * FS + (size_t)y * g.W + x] = (uint8_t)(cval + diff);
        if (a.sse || a.sse_mb) {
            unsigned sq[1] = {(unsigned)(diff * diff)};
            block_sum<1>(sq, s_red[rb], lane, warp);
            rb ^= 1;
            if (tid == 0) {
                if (a.sse) atomicAdd(a.sse + k, (unsigned long long)sq[0]);
                if (a.sse_mb) a.sse_mb[idx] = sq[0];
            }
        }
        __syncthreads();
    }
}

// ========================================================== compensate ==
__global__ void __launch_bounds__(kThreads) compensate_kernel(const Geom g, const CompArgs a)
{
    __shared__ unsigned s_red[1][8];
    const int mb = blockIdx.x, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int u = mb % g.MBW, v = mb / g.MBW, X0 = 16 * u, Y0 = 16 * v;
    const int x = X0 + (tid & 15), y = Y0 + (tid >> 4);
    const unsigned raw = __ldg(reinterpret_cast<const unsigned*>(a.mv + mb));
    const int dx = mv_x((int)raw), dy = mv_y((int)raw);
    const VRange V = valid_range(g, X0, Y0);
    if (dx < V.lox || dx > V.hix || dy < V.loy || dy > V.hiy) {
        if (tid == 0) raise_error(a.status, SME_ERR_RANGE, false);
        return;
    }
    // Same interpolation as ref_at, read straight from global memory.
    int ix = dx, iy = dy, fx = 0, fy = 0;
    if (g.h == 2) { ix = dx >> 1; iy = dy >> 1; fx = dx & 1; fy = dy & 1; }
    const uint8_t* r = a.ref + (size_t)(y + iy) * g.W + (x + ix);
    int p = __ldg(r);
    if (fx && fy) p = (p + __ldg(r + 1) + __ldg(r + g.W) + __ldg(r + g.W + 1) + 2) >> 2;
    else if (fx) p = (p + __ldg(r + 1) + 1) >> 1;
    else if (fy) p = (p + __ldg(r + g.W) + 1) >> 1;
    const int e = (int)__ldg(a.cur + (size_t)y * g.W + x) - p;
    if (a.pred) a.pred[(size_t)y * g.W + x] = (uint8_t)p;
    unsigned sq[1] = {(unsigned)(e * e)};
    block_sum<1>(sq, s_red, lane, warp);
    if (tid == 0) atomicAdd(a.sse, (unsigned long long)sq[0]);
}

// ============================================================= queries ==
__global__ void __launch_bounds__(kThreads) query_kernel(const Geom g, const QueryArgs a)
{
    extern __shared__ __align__(16) uint8_t win[];
    __shared__ unsigned s_red[1][16][8];
    __shared__ float s_fred[2][8];
    __shared__ unsigned s_shape;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int qi = blockIdx.x;
    const int mb = __ldg(a.q + 3 * qi), dx = __ldg(a.q + 3 * qi + 1), dy = __ldg(a.q + 3 * qi + 2);
    if (mb < 0 || mb >= g.M) {
        if (tid == 0) raise_error(a.status, SME_ERR_ARG, false);
        return;
    }
    const int u = mb % g.MBW, v = mb / g.MBW, X0 = 16 * u, Y0 = 16 * v;
    const VRange V = valid_range(g, X0, Y0);
    if (dx < V.lox || dx > V.hix || dy < V.loy || dy > V.hiy) {
        if (tid == 0) raise_error(a.status, SME_ERR_RANGE, false);
        return;
    }
    const int x = X0 + (tid & 15), y = Y0 + (tid >> 4);
    int wx0, wy0;
    stage_window(win, a.ref, g, X0, Y0, tid, wx0, wy0);
    float ux, uy;
    grad_factors(a.cur, g, x, y, ux, uy);
    const int nx = __syncthreads_count(ux != 0.0f);
    const int ny = __syncthreads_count(uy != 0.0f);
    const int cval = __ldg(a.cur + (size_t)y * g.W + x);
    const int diff = ref_at(win, win_pitch(g), x - wx0, y - wy0, dx, dy, g.h) - cval;
    unsigned sad[1] = {(unsigned)abs(diff)};
    block_sum<1>(sad, s_red[0], lane, warp);
    float sx = __fmul_rn((float)diff, ux), sy = __fmul_rn((float)diff, uy);
    tree_sum2(sx, sy, s_fred, lane, warp);
    if (a.pcur && a.pref) {
        unsigned part = 0;
        if (tid < 16) part = shape_row(a.pcur, a.pref, g, X0, Y0, tid, dx / g.h, dy / g.h);
        part += __shfl_xor_sync(kFull, part, 8);
        part += __shfl_xor_sync(kFull, part, 4);
        part += __shfl_xor_sync(kFull, part, 2);
        part += __shfl_xor_sync(kFull, part, 1);
        if (tid == 0) s_shape = part;
        __syncthreads();
    }
    if (tid == 0) {
        if (a.tsad) a.tsad[qi] = sad[0];
        if (a.ssad && a.pcur) a.ssad[qi] = s_shape;
        if (a.delta) {
            a.delta[2 * qi] = update_of(sx, nx, g.eps);
            a.delta[2 * qi + 1] = update_of(sy, ny, g.eps);
        }
    }
}

}  // namespace

size_t me_smem_bytes(const Geom& g)
{
    const int cs = (g.S + 15) & ~15;
    return (size_t)(16 + 2 * g.S) * (size_t)(16 + 2 * cs);
}

cudaError_t launch_classify(const Geom& g, const ClassifyArgs& a, cudaStream_t s)
{
    dim3 grid(g.MBH, a.n_frames);
    classify_pack_kernel<<<grid, kThreads, 0, s>>>(g, a);
    return cudaGetLastError();
}

cudaError_t me_occupancy(const Geom& g, int* blocks_per_sm)
{
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, me_kernel, kThreads, me_smem_bytes(g));
}

cudaError_t launch_me(const Geom& g, const MeArgs& a, int grid, cudaStream_t s)
{
    // Blocks wait on results of other blocks of the same launch, so the
    // launch is cooperative: every block is resident at once.
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(kThreads);
    cfg.dynamicSmemBytes = me_smem_bytes(g);
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, me_kernel, g, a);
}

cudaError_t launch_compensate(const Geom& g, const CompArgs& a, cudaStream_t s)
{
    compensate_kernel<<<g.M, kThreads, 0, s>>>(g, a);
    return cudaGetLastError();
}

cudaError_t launch_queries(const Geom& g, const QueryArgs& a, cudaStream_t s)
{
    if (a.n <= 0) return cudaSuccess;
    query_kernel<<<a.n, kThreads, me_smem_bytes(g), s>>>(g, a);
    return cudaGetLastError();
}

}  // namespace sme
