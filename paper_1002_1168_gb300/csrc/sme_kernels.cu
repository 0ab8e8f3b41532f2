// Device kernels of the shape-adaptive motion estimation pass (sm_103a).
//
//   classify_pack_kernel  Fig. 1 "Block_Type": per-MB class from the binary
//                         alpha block + bit-packed alpha rows (one pass).
//   me_kernel             Fig. 1 / Sec. 3.1 / Sec. 3.2 for every MB of every
//                         frame pair of one or more sequences, one persistent
//                         launch: one warp per MB, tickets in wavefront order,
//                         bounded waits on the A/B/C/T results, block
//                         recursive search (shape cost on boundary MBs, texture
//                         SAD on opaque MBs), pixel recursive gradient search
//                         (Eqs. 3-5, Fig. 4) and the fused motion compensation
//                         + SSE of Sec. 4.
//   compensate_kernel     Sec. 4 motion compensation of a given field.
//   query_kernel          Single cost / gradient evaluations through the same
//                         device functions as me_kernel (unit checks).
//
// Lane l of the warp that owns an MB holds the 8 pixels (8*(l&1) .. +7) of
// row l>>1 of the 16x16 block, i.e. pixels 8l .. 8l+7 in row-major order, as
// two packed 32-bit words.  Sums over the 256 pixels therefore follow the
// row-major pixel order: a lane's 8 terms, then the lanes.
#include <stdint.h>

#include <algorithm>

#include "sme_internal.h"

namespace sme {
namespace {

constexpr unsigned kFull = 0xffffffffu;

// ------------------------------------------------------------------ sync --
// The ready word carries the published vector itself, so a consumer needs no
// other data from the producer: relaxed (coherent, unfenced) 64-bit accesses
// at GPU scope are enough -- an aligned 64-bit access is single-copy atomic.
__device__ __forceinline__ unsigned long long ld_ready(const unsigned long long* p)
{
    unsigned long long v;
    asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ unsigned ld_relaxed(const unsigned* p)
{
    unsigned v;
    asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_ready(unsigned long long* p, unsigned long long v)
{
    asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
__device__ __forceinline__ unsigned long long globaltimer()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Wait until the ready word carries `epoch` in its high half; its low half
// (the published vector) is returned in `val`.  Bounded by `timeout_ns` of
// %globaltimer and by an iteration cap; gives up early when the launch's
// abort word is raised.
__device__ bool wait_ready(const unsigned long long* w, unsigned epoch, const DevStatus* st,
                           long long timeout_ns, unsigned& val)
{
    unsigned long long v = ld_ready(w);
    if ((unsigned)(v >> 32) == epoch) {
        val = (unsigned)v;
        return true;
    }
    const unsigned long long t0 = globaltimer();
    for (unsigned it = 1; it < (1u << 24); ++it) {
        v = ld_ready(w);
        if ((unsigned)(v >> 32) == epoch) {
            val = (unsigned)v;
            return true;
        }
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

// --------------------------------------------------------------- geometry --
__host__ __device__ __forceinline__ int ceil16(int v) { return (v + 15) & ~15; }
__host__ __device__ __forceinline__ int win_pitch(int S) { return 16 + 2 * ceil16(S); }
__host__ __device__ __forceinline__ int win_rows(int S) { return 16 + 2 * S; }
// Per-warp shared memory: the reference window (+32 bytes of slack for the
// 16- and 24-byte row reads at the right edge) and the evaluated-position log.
__host__ __device__ __forceinline__ int win_bytes(int S) { return ceil16(win_rows(S) * win_pitch(S) + 32); }
__host__ __device__ __forceinline__ int warp_smem(int S) { return win_bytes(S) + ceil16(kMaxLog * 4); }

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
__device__ __forceinline__ VRange valid_range(int W, int H, const Method& m, int X0, int Y0)
{
    VRange r;
    r.lox = max(-m.S * m.h, -X0 * m.h);
    r.hix = min(m.S * m.h, (W - 16 - X0) * m.h);
    r.loy = max(-m.S * m.h, -Y0 * m.h);
    r.hiy = min(m.S * m.h, (H - 16 - Y0) * m.h);
    return r;
}

// Issue the copies of the reference rows/columns every vector of V can touch
// into this warp's window (coalesced 16-byte asynchronous copies), without
// waiting for them.  Window origin in wx0/wy0.
__device__ __forceinline__ void stage_window_issue(uint8_t* win, const uint8_t* ref, int W, int H, int S,
                                                   int X0, int Y0, int lane, int& wx0, int& wy0)
{
    const int cs = ceil16(S), pitch = win_pitch(S);
    wy0 = max(0, Y0 - S);
    const int wy1 = min(H - 1, Y0 + 15 + S);
    wx0 = max(0, X0 - cs);
    const int wx1 = min(W, X0 + 16 + cs);
    const int nch = (wx1 - wx0) >> 4, n = (wy1 - wy0 + 1) * nch;
    // c / nch by a multiply and a shift: exact for nch <= 9 and c < 4000
    // (windows hold at most 144 rows of 9 chunks).
    const unsigned inv = (65536u + (unsigned)nch - 1u) / (unsigned)nch;
    // Asynchronous 16-byte copies straight into shared memory: every chunk of
    // the lane is in flight at once, and one wait covers them all.
    const uint8_t* src0 = ref + (size_t)wy0 * W + wx0;
    const unsigned dst0 = (unsigned)__cvta_generic_to_shared(win);
    for (int c = lane; c < n; c += 32) {
        const int r = (int)(((unsigned)c * inv) >> 16), ch = c - r * nch;
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(dst0 + (unsigned)(r * pitch + 16 * ch)),
                     "l"(src0 + (size_t)r * W + 16 * ch)
                     : "memory");
    }
}

// Wait for this lane's window copies, then make the whole window visible to
// the warp.
__device__ __forceinline__ void stage_window_wait()
{
    asm volatile("cp.async.wait_all;" ::: "memory");
    __syncwarp();
}

// Stage the window and wait for it.
__device__ __forceinline__ void stage_window(uint8_t* win, const uint8_t* ref, int W, int H, int S,
                                             int X0, int Y0, int lane, int& wx0, int& wy0)
{
    stage_window_issue(win, ref, W, H, S, X0, Y0, lane, wx0, wy0);
    stage_window_wait();
}

// ------------------------------------------------- packed 8-pixel samples --
struct P8 {
    unsigned lo, hi;  // pixel k in byte k (k = 0..3 in lo, 4..7 in hi)
};

// 16 bytes of a window row starting at the 8-byte boundary at or before
// byte `pos`; `off` = pos & 7.
__device__ __forceinline__ void row16(const uint8_t* win, int pos, unsigned (&w)[4], int& off)
{
    off = pos & 7;
    const uint2 a = *reinterpret_cast<const uint2*>(win + (pos - off));
    const uint2 b = *reinterpret_cast<const uint2*>(win + (pos - off) + 8);
    w[0] = a.x;
    w[1] = a.y;
    w[2] = b.x;
    w[3] = b.y;
}

// Bytes off .. off+7 (off in 0..8) of the 16 bytes in w.
__device__ __forceinline__ P8 extract8(const unsigned (&w)[4], int off)
{
    unsigned a = w[0], b = w[1], c = w[2];
    if (off >= 4) {
        a = w[1];
        b = w[2];
        c = w[3];
        off -= 4;
    }
    P8 r;
    r.lo = __funnelshift_rc(a, b, 8 * off);
    r.hi = __funnelshift_rc(b, c, 8 * off);
    return r;
}

// Per-byte (a + b + 1) >> 1 (MPEG-4 rounding control 0, one axis).
__device__ __forceinline__ unsigned avg2w(unsigned a, unsigned b)
{
    return (a | b) - ((a ^ b) >> 1 & 0x7f7f7f7fu);
}
// Per-byte (a + b + c + d + 2) >> 2 (diagonal half-sample), in 16-bit lanes.
__device__ __forceinline__ unsigned avg4w(unsigned a, unsigned b, unsigned c, unsigned d)
{
    const unsigned m = 0x00ff00ffu;
    const unsigned lo = (a & m) + (b & m) + (c & m) + (d & m) + 0x00020002u;
    const unsigned hi = (a >> 8 & m) + (b >> 8 & m) + (c >> 8 & m) + (d >> 8 & m) + 0x00020002u;
    return (lo >> 2 & m) | ((hi >> 2 & m) << 8);
}

// Reference samples of this lane's 8 pixels displaced by d, from the window
// (window coordinates of the lane's first pixel: lx, ly).  MPEG-4 bilinear
// half-sample interpolation, rounding control 0.
__device__ __forceinline__ P8 ref8(const uint8_t* win, int pitch, int lx, int ly, int dx, int dy, int h)
{
    int ix = dx, iy = dy, fx = 0, fy = 0;
    if (h == 2) {
        ix = dx >> 1;
        iy = dy >> 1;
        fx = dx & 1;
        fy = dy & 1;
    }
    unsigned w[4];
    int off;
    const int pos = (ly + iy) * pitch + lx + ix;
    row16(win, pos, w, off);
    const P8 a = extract8(w, off);
    if (!fx && !fy) return a;
    P8 r;
    if (fx) {
        const P8 b = extract8(w, off + 1);
        if (!fy) {
            r.lo = avg2w(a.lo, b.lo);
            r.hi = avg2w(a.hi, b.hi);
            return r;
        }
        unsigned v[4];
        int o2;
        row16(win, pos + pitch, v, o2);
        const P8 c = extract8(v, o2), d = extract8(v, o2 + 1);
        r.lo = avg4w(a.lo, b.lo, c.lo, d.lo);
        r.hi = avg4w(a.hi, b.hi, c.hi, d.hi);
        return r;
    }
    unsigned v[4];
    int o2;
    row16(win, pos + pitch, v, o2);
    const P8 c = extract8(v, o2);
    r.lo = avg2w(a.lo, c.lo);
    r.hi = avg2w(a.hi, c.hi);
    return r;
}

__device__ __forceinline__ unsigned sad8(const P8& r, const P8& c)
{
    return __vsadu4(r.lo, c.lo) + __vsadu4(r.hi, c.hi);
}
__device__ __forceinline__ int byte_of(const P8& p, int k)
{
    return (int)(((k < 4 ? p.lo : p.hi) >> (8 * (k & 3))) & 0xffu);
}
// Sum of squared differences of the 8 pixels: sum r^2 + sum c^2 - 2 sum rc
// with unsigned byte dot products (exact integer arithmetic).
__device__ __forceinline__ unsigned sq8(const P8& r, const P8& c)
{
    const unsigned rr = __dp4a(r.lo, r.lo, __dp4a(r.hi, r.hi, 0u));
    const unsigned cc = __dp4a(c.lo, c.lo, __dp4a(c.hi, c.hi, 0u));
    const unsigned rc = __dp4a(r.lo, c.lo, __dp4a(r.hi, c.hi, 0u));
    return rr + cc - 2u * rc;
}

// Warp sums of two per-lane values below 2^16 whose totals stay below 2^16
// (SADs of 8 pixels: at most 8*255 per lane, 65280 per MB), in one reduction.
__device__ __forceinline__ void warp_sum2(unsigned a, unsigned b, unsigned& sa, unsigned& sb)
{
    const unsigned t = __reduce_add_sync(kFull, a | (b << 16));
    sa = t & 0xffffu;
    sb = t >> 16;
}

// 24 bytes of a window row from the 8-byte boundary at or before `pos`.
__device__ __forceinline__ void row24(const uint8_t* win, int pos, unsigned (&w)[6], int& off)
{
    off = pos & 7;
    const uint8_t* q = win + (pos - off);
    const uint2 a = *reinterpret_cast<const uint2*>(q);
    const uint2 b = *reinterpret_cast<const uint2*>(q + 8);
    const uint2 c = *reinterpret_cast<const uint2*>(q + 16);
    w[0] = a.x;
    w[1] = a.y;
    w[2] = b.x;
    w[3] = b.y;
    w[4] = c.x;
    w[5] = c.y;
}
// Bytes off .. off+7 (off in 0..11) of the 24 bytes in w.
__device__ __forceinline__ P8 extract8w(const unsigned (&w)[6], int off)
{
    const int b = off >> 2, sh = 8 * (off & 3);
    unsigned a0 = w[0], a1 = w[1], a2 = w[2];
    if (b == 1) {
        a0 = w[1];
        a1 = w[2];
        a2 = w[3];
    }
    if (b == 2) {
        a0 = w[2];
        a1 = w[3];
        a2 = w[4];
    }
    if (b == 3) {
        a0 = w[3];
        a1 = w[4];
        a2 = w[5];
    }
    P8 r;
    r.lo = __funnelshift_r(a0, a1, sh);
    r.hi = __funnelshift_r(a1, a2, sh);
    return r;
}
__device__ __forceinline__ P8 avg2p(const P8& a, const P8& b)
{
    P8 r;
    r.lo = avg2w(a.lo, b.lo);
    r.hi = avg2w(a.hi, b.hi);
    return r;
}
__device__ __forceinline__ P8 avg4p(const P8& a, const P8& b, const P8& c, const P8& d)
{
    P8 r;
    r.lo = avg4w(a.lo, b.lo, c.lo, d.lo);
    r.hi = avg4w(a.hi, b.hi, c.hi, d.hi);
    return r;
}

// ref8 without branches on the half-sample parity: every combination is
// computed and the right one selected, so that several evaluations can
// interleave.  The second row is the next one only when it is used (dy odd),
// so every read stays inside the window as in ref8.
__device__ __forceinline__ P8 ref8_nb(const uint8_t* win, int pitch, int lx, int ly, int dx, int dy, int h)
{
    if (h == 1) return ref8(win, pitch, lx, ly, dx, dy, 1);
    const int fx = dx & 1, fy = dy & 1;
    const int pos = (ly + (dy >> 1)) * pitch + lx + (dx >> 1);
    unsigned w[4], v[4];
    int off, o2;
    row16(win, pos, w, off);
    row16(win, fy ? pos + pitch : pos, v, o2);
    const P8 a = extract8(w, off), b = extract8(w, off + 1), c = extract8(v, off), d = extract8(v, off + 1);
    const P8 hz = avg2p(a, b), vt = avg2p(a, c), dg = avg4p(a, b, c, d);
    P8 r;
    r.lo = fx ? (fy ? dg.lo : hz.lo) : (fy ? vt.lo : a.lo);
    r.hi = fx ? (fy ? dg.hi : hz.hi) : (fy ? vt.hi : a.hi);
    return r;
}

// Half-sample positions d-1, d, d+1 along one axis, for the parity P of d:
// position i reads integer sample (base) and, when frac, averages it with
// the next one.  Even d: (-1,frac) (0) (0,frac); odd d: (0) (0,frac) (1).
template <int P>
__device__ __forceinline__ constexpr int rc_base(int i)
{
    return P ? (i == 2 ? 1 : 0) : (i == 0 ? -1 : 0);
}
template <int P>
__device__ __forceinline__ constexpr bool rc_frac(int i)
{
    return P ? (i == 1) : (i != 1);
}

// Samples of the lane's 8 pixels at the nine positions d + (i, j), i, j in
// {-1, 0, 1} MV units, s[(j+1)*3 + (i+1)], from the 3x3 integer
// neighbourhood X (rows/columns -1..1 around floor(d/h)).  Same MPEG-4
// rounding as ref8.
template <int PX, int PY>
__device__ __forceinline__ void combine9(const P8 (&X)[3][3], P8 (&s)[9])
{
#pragma unroll
    for (int j = 0; j < 3; ++j)
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            const int bx = rc_base<PX>(i) + 1, by = rc_base<PY>(j) + 1;
            const bool fx = rc_frac<PX>(i), fy = rc_frac<PY>(j);
            const P8 a = X[by][bx];
            P8 r = a;
            if (fx && !fy) r = avg2p(a, X[by][bx + 1]);
            if (!fx && fy) r = avg2p(a, X[by + 1][bx]);
            if (fx && fy) r = avg4p(a, X[by][bx + 1], X[by + 1][bx], X[by + 1][bx + 1]);
            s[j * 3 + i] = r;
        }
}

// All nine samples around d; every position d + (i, j) must lie in V.  Only
// the integer rows/columns the nine positions use are read (for an odd
// half-sample coordinate the row/column before floor(d/2) is not used, and
// it may lie outside the window), so every read stays inside the window.
__device__ __forceinline__ void block3x3(const uint8_t* win, int pitch, int lx, int ly, int dx, int dy, int h,
                                         P8 (&s)[9])
{
    int cx = dx, cy = dy, px = 0, py = 0;
    if (h == 2) {
        cx = dx >> 1;
        cy = dy >> 1;
        px = dx & 1;
        py = dy & 1;
    }
    P8 X[3][3];
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
        for (int t = 0; t < 3; ++t) X[r][t] = P8{0u, 0u};
#pragma unroll
    for (int r = 0; r < 3; ++r) {
        if (r < py) continue;
        unsigned w[6];
        int off;
        row24(win, (ly + cy + r - 1) * pitch + lx + cx - 1 + px, w, off);
#pragma unroll
        for (int t = 0; t < 3; ++t)
            if (t >= px) X[r][t] = extract8w(w, off + t - px);
    }
    if (h == 1) {
#pragma unroll
        for (int j = 0; j < 3; ++j)
#pragma unroll
            for (int i = 0; i < 3; ++i) s[j * 3 + i] = X[j][i];
        return;
    }
    if (!px && !py) combine9<0, 0>(X, s);
    else if (px && !py) combine9<1, 0>(X, s);
    else if (!px && py) combine9<0, 1>(X, s);
    else combine9<1, 1>(X, s);
}

// Eq. 4 / Eq. 5 factors of the lane's 8 pixels (x0..x0+7, row y): u = 2/g
// when |g| >= 2*Theta, g the central difference of the current frame (twice
// the derivative); 0 on the frame's outer rows/columns.  `c` holds the 8
// current pixels.
// rcp[g + 255] = 2/g in IEEE FP32 (round to nearest), g = -255..255.
__device__ __forceinline__ void fill_rcp(float* rcp)
{
    for (int i = threadIdx.x; i < 511; i += blockDim.x) {
        const int g = i - 255;
        rcp[i] = g ? __fdiv_rn(2.0f, (float)g) : 0.0f;
    }
}

// The samples around the lane's 8 pixels that the gradients need: the left
// and right neighbours in the row, the rows above and below (0 outside).
struct GradNb {
    int left, right;
    P8 up, dn;
};
__device__ __forceinline__ GradNb grad_loads(const uint8_t* cur, int W, int H, int x0, int y)
{
    const uint8_t* row = cur + (size_t)y * W;
    GradNb n;
    n.left = x0 > 0 ? (int)__ldg(row + x0 - 1) : 0;
    n.right = x0 + 8 < W ? (int)__ldg(row + x0 + 8) : 0;
    n.up = P8{0u, 0u};
    n.dn = P8{0u, 0u};
    if (y > 0) {
        const uint2 t = __ldg(reinterpret_cast<const uint2*>(row - W + x0));
        n.up.lo = t.x;
        n.up.hi = t.y;
    }
    if (y < H - 1) {
        const uint2 t = __ldg(reinterpret_cast<const uint2*>(row + W + x0));
        n.dn.lo = t.x;
        n.dn.hi = t.y;
    }
    return n;
}

__device__ __forceinline__ void grad_factors8(const GradNb& n, int W, int H, int x0, int y, const P8& c, float theta,
                                              const float* rcp, float (&ux)[8], float (&uy)[8])
{
    const float lim = 2.0f * theta;
    const int left = n.left, right = n.right;
    const P8 up = n.up, dn = n.dn;
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        const int x = x0 + k;
        ux[k] = 0.0f;
        uy[k] = 0.0f;
        if (x > 0 && x < W - 1) {
            const int r = k < 7 ? byte_of(c, k + 1) : right;
            const int l = k > 0 ? byte_of(c, k - 1) : left;
            const int g = r - l;
            if (fabsf((float)g) >= lim) ux[k] = rcp[g + 255];
        }
        if (y > 0 && y < H - 1) {
            const int g = byte_of(dn, k) - byte_of(up, k);
            if (fabsf((float)g) >= lim) uy[k] = rcp[g + 255];
        }
    }
}

// FP32 sums of the terms DPD*ux and DPD*uy over the 256 pixels as one
// contiguous pairwise tree in row-major order: the lane's 8 terms
// ((t0+t1)+(t2+t3))+((t4+t5)+(t6+t7)), then lanes paired at offsets 1..16.
// Round-to-nearest products and adds only (no contraction).  Every lane
// receives both sums.
__device__ __forceinline__ void grad_sums(const P8& r, const P8& c, const float (&ux)[8], const float (&uy)[8],
                                          float& sx, float& sy)
{
    float tx[8], ty[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        const float dpd = (float)(byte_of(r, k) - byte_of(c, k));
        tx[k] = __fmul_rn(dpd, ux[k]);
        ty[k] = __fmul_rn(dpd, uy[k]);
    }
    float a = __fadd_rn(__fadd_rn(__fadd_rn(tx[0], tx[1]), __fadd_rn(tx[2], tx[3])),
                        __fadd_rn(__fadd_rn(tx[4], tx[5]), __fadd_rn(tx[6], tx[7])));
    float b = __fadd_rn(__fadd_rn(__fadd_rn(ty[0], ty[1]), __fadd_rn(ty[2], ty[3])),
                        __fadd_rn(__fadd_rn(ty[4], ty[5]), __fadd_rn(ty[6], ty[7])));
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const float pa = __shfl_down_sync(kFull, a, o);
        const float pb = __shfl_down_sync(kFull, b, o);
        a = __fadd_rn(a, pa);
        b = __fadd_rn(b, pb);
    }
    sx = __shfl_sync(kFull, a, 0);
    sy = __shfl_sync(kFull, b, 0);
}

// Eq. 3 block update from the pixel sums: -eps * mean over pixels with u != 0.
__device__ __forceinline__ float update_of(float sum, int n, float eps)
{
    return n ? -__fmul_rn(eps, __fdiv_rn(sum, (float)n)) : 0.0f;
}

// Alpha mismatches of one BAB row: current row bits vs the reference row
// displaced by the full-pel vector (fdx, fdy).
__device__ __forceinline__ unsigned shape_row(const uint32_t* pcur, const uint32_t* pref, int Wp, int X0, int Y0,
                                              int r, int fdx, int fdy)
{
    const uint32_t* rc = pcur + (size_t)(Y0 + r) * Wp;
    const unsigned cb = (__ldg(rc + (X0 >> 5)) >> (X0 & 31)) & 0xffffu;
    const int xr = X0 + fdx;
    const uint32_t* rr = pref + (size_t)(Y0 + r + fdy) * Wp;
    const unsigned rb = __funnelshift_r(__ldg(rr + (xr >> 5)), __ldg(rr + (xr >> 5) + 1), xr & 31) & 0xffffu;
    return __popc(cb ^ rb);
}

// Shape costs of up to 5 candidates (keys in cand[]) with one warp: lane l
// takes row l&15 of candidates (l>>4), (l>>4)+2, (l>>4)+4.  All lanes get
// the totals.
__device__ __forceinline__ void shape_costs(const uint32_t* pcur, const uint32_t* pref, int Wp, int X0, int Y0,
                                            const int (&cand)[5], int nc, int h, int lane, unsigned (&cost)[5])
{
    const int r = lane & 15, half = lane >> 4;
    unsigned s[3] = {0u, 0u, 0u};
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        const int c = half + 2 * j;
        if (c < nc) {
            int key = cand[0];
#pragma unroll
            for (int q = 1; q < 5; ++q)
                if (q == c) key = cand[q];
            s[j] = shape_row(pcur, pref, Wp, X0, Y0, r, mv_x(key) / h, mv_y(key) / h);  // trunc toward zero
        }
    }
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        s[j] += __shfl_xor_sync(kFull, s[j], 8);
        s[j] += __shfl_xor_sync(kFull, s[j], 4);
        s[j] += __shfl_xor_sync(kFull, s[j], 2);
        s[j] += __shfl_xor_sync(kFull, s[j], 1);
    }
    cost[0] = __shfl_sync(kFull, s[0], 0);
    cost[1] = __shfl_sync(kFull, s[0], 16);
    cost[2] = __shfl_sync(kFull, s[1], 0);
    cost[3] = __shfl_sync(kFull, s[1], 16);
    cost[4] = __shfl_sync(kFull, s[2], 0);
}

// ============================================================ classify ==
__global__ void __launch_bounds__(256) classify_pack_kernel(const Geom g, const ClassifyArgs a)
{
    __shared__ unsigned cnt[kMaxDim / 16];
    const int v = blockIdx.x, f = blockIdx.y, tid = threadIdx.x;
    if (v == 0 && f == 0) {
        if (a.status && tid == 0) {
            a.status->ticket = 0;
            a.status->abort = 0;
            const unsigned e = a.status->epoch + 1u;
            a.status->epoch = e ? e : 1u;
        }
        if (a.desc_out && tid == 0) *a.desc_out = a.desc;
        if (a.sse)
            for (int i = tid; i < a.n_sse; i += blockDim.x) a.sse[i] = 0ull;
    }
    for (int i = tid; i < g.MBW; i += blockDim.x) cnt[i] = 0;
    __syncthreads();
    const size_t FS = (size_t)g.W * g.H;
    const uint8_t* fr = a.frames ? a.frames[f] : a.alpha + (size_t)f * FS;
    if (!fr) {  // an empty alpha plane: every MB transparent
        for (int s = tid; s < g.MBW; s += blockDim.x) a.cls[(size_t)f * g.M + v * g.MBW + s] = SME_TRANSPARENT;
        return;
    }
    const uint8_t* al = fr + (size_t)v * 16 * g.W;
    uint16_t* pk = a.packed ? reinterpret_cast<uint16_t*>(a.packed + ((size_t)f * g.H + v * 16) * g.Wp) : nullptr;
    const int segs = g.MBW, hw = 2 * g.Wp;  // 16-pixel segments per row; u16 slots per packed row
    for (int it = tid; it < 16 * hw; it += blockDim.x) {
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
    for (int s = tid; s < segs; s += blockDim.x) {
        const unsigned n = cnt[s];
        a.cls[(size_t)f * g.M + v * g.MBW + s] =
            (uint8_t)(n == 0 ? SME_TRANSPARENT : (n == 256 ? SME_OPAQUE : SME_BOUNDARY));
    }
}

// One BAB row segment: 16 alpha bytes -> 16-bit mask.
__device__ __forceinline__ unsigned bab_bits16(const uint8_t* p)
{
    const uint4 q = __ldg(reinterpret_cast<const uint4*>(p));
    const unsigned w[4] = {q.x, q.y, q.z, q.w};
    unsigned m = 0;
#pragma unroll
    for (int b = 0; b < 4; ++b) {
        const unsigned nz = __vcmpne4(w[b], 0u) & 0x01010101u;
        m |= ((nz | (nz >> 7) | (nz >> 14) | (nz >> 21)) & 0xfu) << (4 * b);
    }
    return m;
}

// Fig. 1 "Block_Type" for every frame of every sequence of a batch (same
// arithmetic as classify_pack_kernel, geometry from the descriptors).  Block
// (0,0) also starts the launch (status words, epoch); the first row block of
// each sequence's first frame zeroes that sequence's SSE outputs.
__global__ void __launch_bounds__(256) classify_batch_kernel(const ClassifyBatchArgs a)
{
    __shared__ unsigned cnt[kMaxDim / 16];
    const int v = blockIdx.x, g = blockIdx.y, tid = threadIdx.x;
    if (v == 0 && g == 0 && tid == 0) {
        a.status->ticket = 0;
        a.status->abort = 0;
        const unsigned e = a.status->epoch + 1u;
        a.status->epoch = e ? e : 1u;
    }
    const SeqDesc* sd = a.seqs + a.fseq[g];
    const int f = a.ffrm[g];
    const int W = sd->W, H = sd->H, MBW = sd->MBW, Wp = sd->Wp;
    if (v >= sd->MBH) return;
    if (v == 0 && f == 0 && sd->sse)
        for (int i = tid; i < sd->P; i += blockDim.x) sd->sse[i] = 0ull;
    for (int i = tid; i < MBW; i += blockDim.x) cnt[i] = 0;
    __syncthreads();
    const uint8_t* al = sd->alpha + (size_t)f * W * H + (size_t)v * 16 * W;
    uint16_t* pk = reinterpret_cast<uint16_t*>(sd->packed_w + ((size_t)f * H + v * 16) * Wp);
    const int hw = 2 * Wp;
    for (int it = tid; it < 16 * hw; it += blockDim.x) {
        const int r = it / hw, sg = it - r * hw;
        unsigned m = 0;
        if (sg < MBW) {
            m = bab_bits16(al + (size_t)r * W + 16 * sg);
            atomicAdd(&cnt[sg], (unsigned)__popc(m));
        }
        pk[(size_t)r * hw + sg] = (uint16_t)m;
    }
    __syncthreads();
    for (int sg = tid; sg < MBW; sg += blockDim.x) {
        const unsigned n = cnt[sg];
        sd->cls_w[(size_t)f * sd->M + v * MBW + sg] =
            (uint8_t)(n == 0 ? SME_TRANSPARENT : (n == 256 ? SME_OPAQUE : SME_BOUNDARY));
    }
}

// ======================================================= per-MB search ==
struct MbResult {
    int dx, dy, iters, nlog;
    unsigned cost;
    float lastx, lasty;
    P8 r8;  // reference samples of the lane's pixels at the final vector
};

// One pixel-recursive step at d (Sec. 3.2): the FP32 update (Eqs. 3-5), the
// proposal q, and -- when d lies inside V, so that clamping is the identity --
// the SADs of the eight neighbours (Fig. 4) from one 3x3 neighbourhood.
struct PrsStep {
    float lastx, lasty;
    int qx, qy;
    bool qmove, inner;
    unsigned cq;      // SAD at q (when qmove)
    P8 q8;            // samples at q (when qmove)
    unsigned sad9[9]; // neighbour SADs, raster order (when inner)
};

__device__ __forceinline__ PrsStep prs_eval(const Method& m, const uint8_t* win, int pitch, int lx, int ly,
                                            const P8& c8, const float (&ux)[8], const float (&uy)[8], int nx, int ny,
                                            const VRange& V, int dx, int dy, const P8& r8, unsigned cost)
{
    const int h = m.h;
    PrsStep st;
    float sx, sy;
    grad_sums(r8, c8, ux, uy, sx, sy);
    st.lastx = update_of(sx, nx, m.eps);
    st.lasty = update_of(sy, ny, m.eps);
    st.qx = clampi(dx + (int)roundf(__fmul_rn((float)h, st.lastx)), V.lox, V.hix);
    st.qy = clampi(dy + (int)roundf(__fmul_rn((float)h, st.lasty)), V.loy, V.hiy);
    st.qmove = (st.qx != dx) || (st.qy != dy);
    st.inner = dx > V.lox && dx < V.hix && dy > V.loy && dy < V.hiy;
    st.cq = 0u;
    st.q8 = r8;
    const bool qnear = st.qmove && abs(st.qx - dx) <= 1 && abs(st.qy - dy) <= 1;
    if (st.inner) {
        P8 nb9[9];
        block3x3(win, pitch, lx, ly, dx, dy, h, nb9);
        warp_sum2(sad8(nb9[0], c8), sad8(nb9[1], c8), st.sad9[0], st.sad9[1]);
        warp_sum2(sad8(nb9[2], c8), sad8(nb9[3], c8), st.sad9[2], st.sad9[3]);
        warp_sum2(sad8(nb9[5], c8), sad8(nb9[6], c8), st.sad9[5], st.sad9[6]);
        warp_sum2(sad8(nb9[7], c8), sad8(nb9[8], c8), st.sad9[7], st.sad9[8]);
        st.sad9[4] = cost;
        if (qnear) {
            const int qi = (st.qy - dy + 1) * 3 + (st.qx - dx + 1);
#pragma unroll
            for (int n = 0; n < 9; ++n)
                if (n == qi) {
                    st.cq = st.sad9[n];
                    st.q8 = nb9[n];
                }
            return st;
        }
    }
    if (st.qmove) {
        st.q8 = ref8(win, pitch, lx, ly, st.qx, st.qy, h);
        st.cq = __reduce_add_sync(kFull, sad8(st.q8, c8));
    }
    return st;
}

// The decision of one step in the paper's order: the proposal if it lowers
// the SAD, else the first strict minimum of the eight clamped neighbours,
// else stop.  Logs the evaluated positions.  Returns true when d moved.
__device__ __forceinline__ bool prs_decide(const Method& m, const uint8_t* win, int pitch, int lx, int ly,
                                           const P8& c8, const VRange& V, const PrsStep& st, int& dx, int& dy,
                                           unsigned& cost, P8& r8, int* slog, int& nlog, int lane)
{
    const int h = m.h;
    if (st.qmove) {
        if (lane == 0) slog[nlog] = pack_mv(st.qx, st.qy);
        ++nlog;
        if (st.cq < cost) {
            dx = st.qx;
            dy = st.qy;
            cost = st.cq;
            r8 = st.q8;
            return true;
        }
    }
    if (st.inner) {
        unsigned bc = cost;
        int bn = 4;
#pragma unroll
        for (int n = 0; n < 9; ++n) {
            if (n == 4) continue;
            if (lane == 0) slog[nlog] = pack_mv(dx + n % 3 - 1, dy + n / 3 - 1);
            ++nlog;
            if (st.sad9[n] < bc) {
                bc = st.sad9[n];
                bn = n;
            }
        }
        if (bc < cost) {
            dx += bn % 3 - 1;
            dy += bn / 3 - 1;
            cost = bc;
            r8 = ref8(win, pitch, lx, ly, dx, dy, h);
            return true;
        }
        return false;
    }
    // d on the edge of V: the clamped neighbours one by one.
    unsigned bc = cost;
    int bx = dx, by = dy;
#pragma unroll
    for (int n = 1; n < 9; ++n) {
        const int e = n < 5 ? n - 1 : n;  // 3x3 raster without its centre
        const int ex = clampi(dx + e % 3 - 1, V.lox, V.hix), ey = clampi(dy + e / 3 - 1, V.loy, V.hiy);
        if (ex != dx || ey != dy) {
            const unsigned cn = __reduce_add_sync(kFull, sad8(ref8(win, pitch, lx, ly, ex, ey, h), c8));
            if (lane == 0) slog[nlog] = pack_mv(ex, ey);
            ++nlog;
            if (cn < bc) {
                bc = cn;
                bx = ex;
                by = ey;
            }
        }
    }
    if (bc < cost) {
        dx = bx;
        dy = by;
        cost = bc;
        r8 = ref8(win, pitch, lx, ly, dx, dy, h);
        return true;
    }
    return false;
}

// Sec. 3.2 pixel recursive search from (dx, dy): steps until neither the
// proposal nor a neighbour lowers the SAD, at most K.  When use_first is set,
// `first` is the already computed first step at the starting position.
// Returns the steps taken; the last update goes to lastx/lasty.
__device__ __forceinline__ int prs_run(const Method& m, const uint8_t* win, int pitch, int lx, int ly, const P8& c8,
                                       const float (&ux)[8], const float (&uy)[8], int nx, int ny, const VRange& V,
                                       int& dx, int& dy, unsigned& cost, P8& r8, float& lastx, float& lasty,
                                       int* slog, int& nlog, int lane, bool use_first, const PrsStep& first)
{
    int iters = 0;
    lastx = 0.0f;
    lasty = 0.0f;
    while (iters < m.K) {
        const PrsStep st = (iters == 0 && use_first) ? first
                                                     : prs_eval(m, win, pitch, lx, ly, c8, ux, uy, nx, ny, V, dx, dy, r8, cost);
        ++iters;
        lastx = st.lastx;
        lasty = st.lasty;
        if (!prs_decide(m, win, pitch, lx, ly, c8, V, st, dx, dy, cost, r8, slog, nlog, lane)) break;
    }
    return iters;
}

// The same search with the two searches of a seed-won MB inlined one after
// the other.
__device__ __forceinline__ void opaque_search_two_sites(const Method& m, const uint8_t* win, int pitch, int lx, int ly,
                                              const P8& c8, const float (&ux)[8], const float (&uy)[8], int nx,
                                              int ny, const VRange& V, const int (&cand)[5],
                                              const unsigned (&costs)[5], const P8 (&cs8)[5], int nc, int best,
                                              int* slog, int& nlog, int lane, bool spec, int spec_key,
                                              const PrsStep& sp, MbResult& res)
{
    int dx = mv_x(cand[0]), dy = mv_y(cand[0]);
    unsigned cost = costs[0];
    P8 r8 = cs8[0];
#pragma unroll
    for (int c = 1; c < 5; ++c)
        if (c == best) {
            dx = mv_x(cand[c]);
            dy = mv_y(cand[c]);
            cost = costs[c];
            r8 = cs8[c];
        }
    float lastx, lasty;
    int iters;
    if (nc == 5 && best == 4) {
        int pb = 0;
        unsigned pc = costs[0];
#pragma unroll
        for (int c = 1; c < 4; ++c)
            if (costs[c] < pc) {
                pb = c;
                pc = costs[c];
            }
        int px = mv_x(cand[0]), py = mv_y(cand[0]);
        P8 pr8 = cs8[0];
#pragma unroll
        for (int c = 1; c < 4; ++c)
            if (c == pb) {
                px = mv_x(cand[c]);
                py = mv_y(cand[c]);
                pr8 = cs8[c];
            }
        float plx, ply;
        const int pit = prs_run(m, win, pitch, lx, ly, c8, ux, uy, nx, ny, V, px, py, pc, pr8, plx, ply, slog, nlog,
                                lane, spec && pack_mv(px, py) == spec_key, sp);
        iters = prs_run(m, win, pitch, lx, ly, c8, ux, uy, nx, ny, V, dx, dy, cost, r8, lastx, lasty, slog, nlog,
                        lane, spec && pack_mv(dx, dy) == spec_key, sp);
        if (!(cost < pc)) {
            dx = px;
            dy = py;
            cost = pc;
            r8 = pr8;
            iters = pit;
            lastx = plx;
            lasty = ply;
        }
    } else {
        iters = prs_run(m, win, pitch, lx, ly, c8, ux, uy, nx, ny, V, dx, dy, cost, r8, lastx, lasty, slog, nlog,
                        lane, spec && pack_mv(dx, dy) == spec_key, sp);
    }
    res.dx = dx;
    res.dy = dy;
    res.cost = cost;
    res.r8 = r8;
    res.iters = iters;
    res.lastx = lastx;
    res.lasty = lasty;
}

// Opaque MB after the candidate comparison: the pixel recursive search from
// the winner; when a learned seed (candidate 4) won strictly, the search runs
// from the best plain candidate and then from the seed, and the plain result
// is kept unless the seeded one ends strictly lower.  kOneSite: both searches
// go through one call site (in the sparse search the rarely taken second
// search was a cold copy of the search code, slow to fetch and evicting the
// hot one: 54 -> 38 ms on the learned headline search); else two inlined
// searches (the per-MB and per-pair kernels keep their register allocation).
// cand/costs/cs8 are the candidates in order A, B, C, T(, seed); best is the
// winning index.
template <bool kOneSite>
__device__ __forceinline__ void opaque_search(const Method& m, const uint8_t* win, int pitch, int lx, int ly,
                                              const P8& c8, const float (&ux)[8], const float (&uy)[8], int nx,
                                              int ny, const VRange& V, const int (&cand)[5],
                                              const unsigned (&costs)[5], const P8 (&cs8)[5], int nc, int best,
                                              int* slog, int& nlog, int lane, bool spec, int spec_key,
                                              const PrsStep& sp, MbResult& res)
{
    if constexpr (!kOneSite) {
        opaque_search_two_sites(m, win, pitch, lx, ly, c8, ux, uy, nx, ny, V, cand, costs, cs8, nc, best, slog, nlog,
                                lane, spec, spec_key, sp, res);
        return;
    }
    const bool two = nc == 5 && best == 4;
    // The first pass starts from the winner, or (two passes) from the first
    // strict minimum of A, B, C, T.
    int first = best;
    if (two) {
        first = 0;
#pragma unroll
        for (int c = 1; c < 4; ++c)
            if (costs[c] < costs[first]) first = c;
    }
    int dx = mv_x(cand[0]), dy = mv_y(cand[0]);
    unsigned cost = costs[0];
    P8 r8 = cs8[0];
#pragma unroll
    for (int c = 1; c < 5; ++c)
        if (c == first) {
            dx = mv_x(cand[c]);
            dy = mv_y(cand[c]);
            cost = costs[c];
            r8 = cs8[c];
        }
    float lastx, lasty;
    int iters;
    int px = 0, py = 0, pit = 0;
    unsigned pc = 0;
    P8 pr8 = r8;
    float plx = 0.0f, ply = 0.0f;
#pragma unroll 1
    for (int pass = 0;; ++pass) {
        iters = prs_run(m, win, pitch, lx, ly, c8, ux, uy, nx, ny, V, dx, dy, cost, r8, lastx, lasty, slog, nlog,
                        lane, spec && pack_mv(dx, dy) == spec_key, sp);
        if (!two || pass == 1) break;
        px = dx;
        py = dy;
        pc = cost;
        pr8 = r8;
        pit = iters;
        plx = lastx;
        ply = lasty;
        dx = mv_x(cand[4]);
        dy = mv_y(cand[4]);
        cost = costs[4];
        r8 = cs8[4];
    }
    if (two && !(cost < pc)) {
        dx = px;
        dy = py;
        cost = pc;
        r8 = pr8;
        iters = pit;
        lastx = plx;
        lasty = ply;
    }
    res.dx = dx;
    res.dy = dy;
    res.cost = cost;
    res.r8 = r8;
    res.iters = iters;
    res.lastx = lastx;
    res.lasty = lasty;
}

// Fig. 1 from the candidate comparison on: shape cost (boundary) or texture
// SAD (opaque) of the candidates, first strict minimum, and on opaque MBs the
// pixel recursive search of Sec. 3.2.  The candidates are already logged in
// slog[0..nc); the evaluated PRS positions are appended by lane 0.
__device__ __forceinline__ MbResult search_mb(const Method& m, int cls, const uint8_t* win, int pitch, int lx,
                                              int ly, const P8& c8, const float (&ux)[8], const float (&uy)[8],
                                              int nx, int ny, const VRange& V, const int (&cand)[5], int nc,
                                              const uint32_t* pcur, const uint32_t* pref, int Wp, int X0, int Y0,
                                              int* slog, int lane)
{
    const int h = m.h;
    MbResult res;
    res.iters = 0;
    res.lastx = 0.0f;
    res.lasty = 0.0f;
    int nlog = nc;
    int dx, dy;
    unsigned cost;
    if (cls == SME_BOUNDARY) {
        // Fig. 1 boundary branch: alpha mismatch of the BABs.
        unsigned sc[5];
        shape_costs(pcur, pref, Wp, X0, Y0, cand, nc, h, lane, sc);
        int best = cand[0];
        cost = sc[0];
#pragma unroll
        for (int c = 1; c < 5; ++c)
            if (c < nc && sc[c] < cost) {
                cost = sc[c];
                best = cand[c];
            }
        dx = mv_x(best);
        dy = mv_y(best);
        res.r8 = ref8(win, pitch, lx, ly, dx, dy, h);
    } else {
        // Fig. 1 opaque branch: texture SAD of the candidates.
        P8 cs8[5];
        unsigned part[5];
#pragma unroll
        for (int c = 0; c < 5; ++c) {
            cs8[c] = c < nc ? ref8(win, pitch, lx, ly, mv_x(cand[c]), mv_y(cand[c]), h) : c8;
            part[c] = sad8(cs8[c], c8);
        }
        unsigned sad[5];
        warp_sum2(part[0], part[1], sad[0], sad[1]);
        warp_sum2(part[2], part[3], sad[2], sad[3]);
        sad[4] = nc > 4 ? __reduce_add_sync(kFull, part[4]) : 0u;
        int best = 0;
        cost = sad[0];
#pragma unroll
        for (int c = 1; c < 5; ++c)
            if (c < nc && sad[c] < cost) {
                cost = sad[c];
                best = c;
            }
        PrsStep none;
        opaque_search<false>(m, win, pitch, lx, ly, c8, ux, uy, nx, ny, V, cand, sad, cs8, nc, best, slog, nlog,
                             lane, false, 0, none, res);
        res.nlog = nlog;
        return res;
    }
    res.dx = dx;
    res.dy = dy;
    res.cost = cost;
    res.nlog = nlog;
    return res;
}

// Sec. 3.1 variant for a boundary MB whose candidates carry shape costs:
// the first strict minimum over the candidates other than T (index 3) is
// compared with T by 16x16 texture SAD; T is kept only if strictly lower.
// bi/cost become the index kept and its shape cost.
__device__ __forceinline__ void boundary_t_by_texture(const uint8_t* win, int pitch, int lx, int ly, const P8& c8,
                                                      const int (&cand)[5], const unsigned (&scost)[5], int nc, int h,
                                                      int& bi, unsigned& cost)
{
    int sb = 0;
#pragma unroll
    for (int c = 1; c < 5; ++c)
        if (c != 3 && c < nc && scost[c] < scost[sb]) sb = c;
    int ks = cand[0];
#pragma unroll
    for (int c = 1; c < 5; ++c)
        if (c == sb) ks = cand[c];
    unsigned tex_s, tex_t;
    warp_sum2(sad8(ref8(win, pitch, lx, ly, mv_x(ks), mv_y(ks), h), c8),
              sad8(ref8(win, pitch, lx, ly, mv_x(cand[3]), mv_y(cand[3]), h), c8), tex_s, tex_t);
    bi = tex_t < tex_s ? 3 : sb;
    cost = sb == bi ? scost[sb] : scost[3];
}

// Shape cost of one candidate: lanes 0..15 take the 16 rows (lanes 16..31
// repeat them); every lane gets the total.
__device__ __forceinline__ unsigned shape_cost1(const uint32_t* pcur, const uint32_t* pref, int Wp, int X0, int Y0,
                                                int key, int h, int lane)
{
    unsigned s = shape_row(pcur, pref, Wp, X0, Y0, lane & 15, mv_x(key) / h, mv_y(key) / h);
    s += __shfl_xor_sync(kFull, s, 8);
    s += __shfl_xor_sync(kFull, s, 4);
    s += __shfl_xor_sync(kFull, s, 2);
    s += __shfl_xor_sync(kFull, s, 1);
    return s;
}

// Off the dependency chain: per-MB outputs, the distinct evaluated positions
// (Table 1 unit), and the motion-compensated prediction with its SSE (Sec. 4).
__device__ __forceinline__ void finish_mb(const SeqDesc* sd, int idx, int k, int cls, const MbResult& r, const P8& c8,
                                          const int* slog, int lane, size_t FS, int W, int y, int x0)
{
    if (lane == 1) {
        if (sd->cost) sd->cost[idx] = r.cost;
        if (sd->iters) sd->iters[idx] = (uint8_t)r.iters;
        if (sd->out_cls) sd->out_cls[idx] = (uint8_t)cls;
    }
    if (lane == 2 && sd->disp) {
        sd->disp[2 * idx] = r.lastx;
        sd->disp[2 * idx + 1] = r.lasty;
    }
    __syncwarp();
    unsigned first = 0;
    if (r.nlog <= 32) {
        // Lanes holding equal keys match; the lowest such lane counts once.
        // Unused lanes hold keys no vector can have (|dy| <= 128).
        const int kk = lane < r.nlog ? slog[lane] : (0x7fff0000 | lane);
        const unsigned eq = __match_any_sync(kFull, kk);
        first = (lane < r.nlog && (__ffs(eq) - 1) == lane) ? 1u : 0u;
    } else {
        for (int e = lane; e < r.nlog; e += 32) {
            const int kk = slog[e];
            bool f = true;
            for (int j = 0; j < e; ++j)
                if (slog[j] == kk) {
                    f = false;
                    break;
                }
            first += f;
        }
    }
    // One reduction for both: the MB's SSE is below 2^24 (256 * 255^2) and the
    // position count below 2^8.
    const unsigned both = __reduce_add_sync(kFull, sq8(r.r8, c8) | (first << 24));
    const unsigned sse = both & 0xffffffu;
    if (lane == 0) {
        if (sd->npos) sd->npos[idx] = (uint8_t)(both >> 24);
        if (sd->sse) atomicAdd(sd->sse + k, (unsigned long long)sse);
        if (sd->sse_mb) sd->sse_mb[idx] = sse;
    }
    if (sd->pred)
        *reinterpret_cast<uint2*>(sd->pred + (size_t)k * FS + (size_t)y * W + x0) = make_uint2(r.r8.lo, r.r8.hi);
    __syncwarp();
}

// Fig. 1: a transparent MB gets no vector; its outputs and its co-located
// prediction error (Sec. 4).  The vector (0,0) is published by the caller.
__device__ __forceinline__ void transparent_mb(const SeqDesc* sd, int idx, int k, const uint8_t* ref, const P8& c8,
                                               int lane, size_t FS, int W, int y, int x0)
{
    if (lane == 0) {
        sd->mv[idx] = sme_mv{0, 0};
        if (sd->cost) sd->cost[idx] = 0;
        if (sd->disp) {
            sd->disp[2 * idx] = 0.0f;
            sd->disp[2 * idx + 1] = 0.0f;
        }
        if (sd->iters) sd->iters[idx] = 0;
        if (sd->npos) sd->npos[idx] = 0;
        if (sd->out_cls) sd->out_cls[idx] = (uint8_t)SME_TRANSPARENT;
    }
    const uint2 t2 = __ldg(reinterpret_cast<const uint2*>(ref + (size_t)y * W + x0));
    P8 r8;
    r8.lo = t2.x;
    r8.hi = t2.y;
    if (sd->pred) *reinterpret_cast<uint2*>(sd->pred + (size_t)k * FS + (size_t)y * W + x0) = t2;
    if (sd->sse || sd->sse_mb) {
        const unsigned s = __reduce_add_sync(kFull, sq8(r8, c8));
        if (lane == 0) {
            if (sd->sse) atomicAdd(sd->sse + k, (unsigned long long)s);
            if (sd->sse_mb) sd->sse_mb[idx] = s;
        }
    }
    __syncwarp();
}

// Eq. 4 factors of the lane's pixels and their counts over the MB.
__device__ __forceinline__ void mb_factors(const GradNb& gn, int W, int H, int x0, int y, const P8& c8, float theta,
                                           const float* rcp, float (&ux)[8], float (&uy)[8], int& nx, int& ny)
{
    grad_factors8(gn, W, H, x0, y, c8, theta, rcp, ux, uy);
    int cx = 0, cy = 0;
#pragma unroll
    for (int q = 0; q < 8; ++q) {
        cx += ux[q] != 0.0f;
        cy += uy[q] != 0.0f;
    }
    nx = (int)__reduce_add_sync(kFull, (unsigned)cx);
    ny = (int)__reduce_add_sync(kFull, (unsigned)cy);
}

// A seed (pixels) in MV units, rounded and clamped to V (reading c19).
__device__ __forceinline__ int seed_key_of(float x, float y, int h, const VRange& V)
{
    const float sx = fminf(fmaxf(__fmul_rn((float)h, x), -1024.0f), 1024.0f);
    const float sy = fminf(fmaxf(__fmul_rn((float)h, y), -1024.0f), 1024.0f);
    return pack_mv(clampi((int)roundf(sx), V.lox, V.hix), clampi((int)roundf(sy), V.loy, V.hiy));
}
__device__ __forceinline__ int seed_key(const SeqDesc* sd, int idx, int h, const VRange& V)
{
    return seed_key_of(__ldg(sd->seed + 2 * (size_t)idx), __ldg(sd->seed + 2 * (size_t)idx + 1), h, V);
}

__device__ __forceinline__ P8 load8(const uint8_t* p)
{
    const uint2 t2 = __ldg(reinterpret_cast<const uint2*>(p));
    P8 r;
    r.lo = t2.x;
    r.hi = t2.y;
    return r;
}

// ====================================================== ME, per-MB warps ==
// Where the candidate vectors of an MB come from and where its own vector
// goes.  GlobalLinks: a ready word per MB in global memory, (epoch << 32) |
// vector, polled by whichever warp of the grid holds a consumer.
struct GlobalLinks {
    unsigned long long* ready;
    unsigned epoch;
    int fault;  // an MB whose vector is never published (failure-detection tests)
    __device__ __forceinline__ unsigned long long poll(int dep, int) const { return ld_ready(ready + dep); }
    __device__ __forceinline__ bool arrived(unsigned long long w) const { return (unsigned)(w >> 32) == epoch; }
    __device__ __forceinline__ void publish(int gid, int key, int lane) const
    {
        if (lane == 0 && gid != fault) st_ready(ready + gid, ((unsigned long long)epoch << 32) | (unsigned)key);
    }
    // A poll through L2 already takes long enough to leave the SM's issue
    // slots to the other warps.
    __device__ __forceinline__ void idle() const {}
};

// ClusterLinks: the CTAs of one thread-block cluster share a sequence, and
// every MB's consumers -- the MBs that take it as A, B, C or T -- are known
// in advance.  The producer stores (1 << 32) | vector straight into each
// consumer's slot in the consumer CTA's shared memory (distributed shared
// memory); a consumer polls its own slots.  slots: this CTA's slots, four per
// item (roles A, B, C, T), zeroed at launch.
struct ClusterLinks {
    unsigned long long* slots;
    int slot;   // the item's position in this CTA's list
    int cons;   // lanes 0..3: the consumer slot in role `lane` (rank << 20 | slot * 4 + role), or -1
    int fault;
    __device__ __forceinline__ unsigned long long poll(int, int role) const
    {
        return *reinterpret_cast<volatile unsigned long long*>(slots + 4 * slot + role);
    }
    __device__ __forceinline__ bool arrived(unsigned long long w) const { return (w >> 32) != 0; }
    __device__ __forceinline__ void publish(int gid, int key, int lane) const
    {
        if (lane >= 4 || gid == fault) return;
        const int c = cons;
        if (c < 0) return;
        const uint32_t local = (uint32_t)__cvta_generic_to_shared(slots + (c & 0xFFFFF));
        uint32_t remote;
        asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(remote) : "r"(local), "r"(c >> 20));
        asm volatile("st.relaxed.cluster.shared::cluster.u64 [%0], %1;" ::"r"(remote),
                     "l"((1ull << 32) | (unsigned)key)
                     : "memory");
    }
    __device__ __forceinline__ void idle() const {}
};

// One MB (global id gid of sequence sd) by one warp: Fig. 1 from the class
// on, with the candidates of Fig. 3 taken from `L`.  Returns false when a
// bounded wait gave up (the launch's error status is raised).
// kVariants: the code of the Sec. 3.1 boundary variant is compiled in (taken
// when m.tt); the default instantiation leaves it out, since even an untaken
// branch after the wait loop measurably slowed the search.
// kSparse: transparent MBs publish nothing (the sparse schedule finishes them
// in its streaming pass); a candidate whose MB is transparent is (0,0) by
// Fig. 1 and is taken from the class map without a wait.  The speculative
// first step is compiled out: in that throughput form the candidates have
// mostly arrived already, and the extra code cost more than it saved.

template <class Links, bool kVariants, bool kSparse = false>
__device__ __forceinline__ bool me_one_mb(const MeArgs& a, const Method& m, int gid, const SeqDesc* sd, uint8_t* win,
                                          int* slog, const float* s_rcp, const Links& L, int lane, int pitch)
{
    const int h = m.h;
    const int W = sd->W, H = sd->H, M = sd->M, MBW = sd->MBW, rd = sd->rd;
    const int idx = gid - sd->gid_base;
    const int k = idx / M, mb = idx - k * M;
    const int u = mb % MBW, v = mb / MBW;
    const int X0 = 16 * u, Y0 = 16 * v;
    const int x0 = X0 + 8 * (lane & 1), y = Y0 + (lane >> 1);
    const size_t FS = (size_t)W * H;
    const uint8_t* ref = sd->luma + (size_t)k * FS;
    const uint8_t* cur = sd->luma + (size_t)(k + rd) * FS;
    const int cls = __ldg(sd->cls + (size_t)(k + rd) * M + mb);
    const P8 c8 = load8(cur + (size_t)y * W + x0);
    // The sparse schedule lists only non-transparent MBs: their window copies
    // and the samples of the gradient factors are requested at once, with the
    // loads above, so that one memory round trip serves them all.
    int wx0, wy0;
    GradNb gn;
    float seed_x = 0.0f, seed_y = 0.0f;
    if constexpr (kSparse) {
        stage_window_issue(win, ref, W, H, m.S, X0, Y0, lane, wx0, wy0);
        gn = grad_loads(cur, W, H, x0, y);
        if (lane == 4 && sd->seed) {  // the learned seed: its read flies with the others
            seed_x = __ldg(sd->seed + 2 * (size_t)idx);
            seed_y = __ldg(sd->seed + 2 * (size_t)idx + 1);
        }
    }

    if (cls == SME_TRANSPARENT) {
        if constexpr (kSparse) stage_window_wait();
        L.publish(gid, 0, lane);
        transparent_mb(sd, idx, k, ref, c8, lane, FS, W, y, x0);
        return true;
    }

    // ---- work that does not depend on the neighbours: prefetch ----
    if constexpr (!kSparse) stage_window(win, ref, W, H, m.S, X0, Y0, lane, wx0, wy0);
    float ux[8], uy[8];
    int nx = 0, ny = 0;
    if constexpr (kSparse) {
        if (cls == SME_OPAQUE) mb_factors(gn, W, H, x0, y, c8, m.theta, s_rcp, ux, uy, nx, ny);
        stage_window_wait();
    } else {
        if (cls == SME_OPAQUE)
            mb_factors(grad_loads(cur, W, H, x0, y), W, H, x0, y, c8, m.theta, s_rcp, ux, uy, nx, ny);
    }
    const VRange V = valid_range(W, H, m, X0, Y0);

    // ---- candidates A, B, C, T (Fig. 1, Fig. 3) + optional seed ----
    // Lanes 0..3 poll the ready words of A, B, C, T.  While the warp
    // waits, every candidate whose vector has arrived is costed at once,
    // and the first pixel-recursive step is taken speculatively at the
    // first costed position; the results are exactly those the search
    // computes after the wait, so nothing changes but the latency.
    int dep = -1;
    if (lane == 0 && u > 0) dep = gid - 1;                       // A
    if (lane == 1 && v > 0) dep = gid - MBW;                     // B
    if (lane == 2 && v > 0 && u < MBW - 1) dep = gid - MBW + 1;  // C
    if (lane == 3 && k > 0) dep = gid - M;                       // T
    if constexpr (kSparse) {
        if (dep >= 0) {
            const int dmb = lane == 3 ? mb : (lane == 0 ? mb - 1 : (lane == 1 ? mb - MBW : mb - MBW + 1));
            const int dfr = lane == 3 ? k - 1 + rd : k + rd;
            if (__ldg(sd->cls + (size_t)dfr * M + dmb) == SME_TRANSPARENT) dep = -1;
        }
    }
    int key = 0;
    if (lane == 3 && k == 0 && sd->temporal_in)
        key = (int)__ldg(reinterpret_cast<const unsigned*>(sd->temporal_in + mb));
    if (lane == 4 && sd->seed) key = kSparse ? seed_key_of(seed_x, seed_y, h, V) : seed_key(sd, idx, h, V);
    if (lane < 4) key = pack_mv(clampi(mv_x(key), V.lox, V.hix), clampi(mv_y(key), V.loy, V.hiy));
    const int nc = sd->seed ? 5 : 4;
    bool res_l = dep < 0;
    unsigned have = __ballot_sync(kFull, lane < nc && res_l) & ((1u << nc) - 1u);
    const unsigned all = (1u << nc) - 1u;
    unsigned costed = 0;
    unsigned ccost[5] = {0u, 0u, 0u, 0u, 0u};
    int ckey[5] = {0, 0, 0, 0, 0};
    P8 cs8[5];
#pragma unroll
    for (int c = 0; c < 5; ++c) cs8[c] = c8;
    bool spec = false;
    int spec_key = 0;
    PrsStep sp;
    const uint32_t* pcur = sd->packed + (size_t)(k + rd) * H * sd->Wp;
    const uint32_t* pref = sd->packed + (size_t)k * H * sd->Wp;
    const int lx = x0 - wx0, ly = y - wy0;
    bool failed = false;
    unsigned long long t_start = 0;
    if constexpr (kSparse) {
        // Throughput form: the producers are mostly done already, so wait for
        // all of them, then cost every candidate in one branch-free block
        // (equal positions give equal costs, so nothing needs deduplicating).
        for (unsigned it = 0; have != all; ++it) {
            const unsigned long long w = (lane < 4 && !res_l) ? L.poll(dep, lane) : 0ull;
            if (lane < 4 && !res_l && L.arrived(w)) {
                const int kk = (int)(unsigned)w;
                key = pack_mv(clampi(mv_x(kk), V.lox, V.hix), clampi(mv_y(kk), V.loy, V.hiy));
                res_l = true;
            }
            have = __ballot_sync(kFull, lane < nc && res_l) & all;
            if ((it & 15u) == 15u && have != all) {
                int give_up = 0;
                if (lane == 0) {
                    const unsigned long long now = globaltimer();
                    if (t_start == 0) t_start = now;
                    give_up = ld_relaxed(&a.status->abort) || (long long)(now - t_start) > a.timeout_ns ||
                              it > (1u << 24);
                }
                if (__shfl_sync(kFull, give_up, 0)) {
                    if (lane == 0 && !ld_relaxed(&a.status->abort)) raise_error(a.status, SME_ERR_TIMEOUT, true);
                    return false;
                }
            }
        }
#pragma unroll
        for (int c = 0; c < 5; ++c) ckey[c] = __shfl_sync(kFull, key, c);
        if (cls == SME_BOUNDARY) {
            shape_costs(pcur, pref, sd->Wp, X0, Y0, ckey, nc, h, lane, ccost);
        } else {
            unsigned part[5];
#pragma unroll
            for (int c = 0; c < 5; ++c) {
                cs8[c] = c < nc ? ref8_nb(win, pitch, lx, ly, mv_x(ckey[c]), mv_y(ckey[c]), h) : c8;
                part[c] = sad8(cs8[c], c8);
            }
            warp_sum2(part[0], part[1], ccost[0], ccost[1]);
            warp_sum2(part[2], part[3], ccost[2], ccost[3]);
            ccost[4] = __reduce_add_sync(kFull, part[4]);
        }
        costed = all;
    }
    for (unsigned it = 0; !kSparse; ++it) {
        // The next poll is issued first, so its latency overlaps the
        // costing below; its result is consumed at the end of the pass.
        unsigned long long w = 0;
        if (lane < 4 && !res_l) w = L.poll(dep, lane);
        const unsigned fresh = (kSparse || a.speculate || have == all) ? (have & ~costed) : 0u;
#pragma unroll
        for (int c = 0; c < 5; ++c)
            if (fresh & (1u << c)) {
                const int kc = __shfl_sync(kFull, key, c);
                ckey[c] = kc;
                // A position already costed is not evaluated again.
                bool dup = false;
#pragma unroll
                for (int e = 0; e < 5; ++e)
                    if (e != c && !dup && (costed & (1u << e)) && ckey[e] == kc) {
                        ccost[c] = ccost[e];
                        cs8[c] = cs8[e];
                        dup = true;
                    }
                if (!dup) {
                    if (cls == SME_BOUNDARY) {
                        ccost[c] = shape_cost1(pcur, pref, sd->Wp, X0, Y0, kc, h, lane);
                    } else {
                        cs8[c] = ref8(win, pitch, lx, ly, mv_x(kc), mv_y(kc), h);
                        ccost[c] = __reduce_add_sync(kFull, sad8(cs8[c], c8));
                    }
                }
                costed |= 1u << c;
            }
        if (costed == all) break;
        if (!kSparse && a.speculate && cls == SME_OPAQUE && costed && m.K > 0) {
            // The first pixel-recursive step at the provisional winner
            // (first strict minimum among the candidates costed so far).
            int pb = -1;
            unsigned pc = 0;
#pragma unroll
            for (int c = 0; c < 5; ++c)
                if ((costed & (1u << c)) && (pb < 0 || ccost[c] < pc)) {
                    pb = c;
                    pc = ccost[c];
                }
            int pk = ckey[0];
            P8 r0 = cs8[0];
#pragma unroll
            for (int c = 1; c < 5; ++c)
                if (c == pb) {
                    pk = ckey[c];
                    r0 = cs8[c];
                }
            if (!spec || pk != spec_key) {
                sp = prs_eval(m, win, pitch, lx, ly, c8, ux, uy, nx, ny, V, mv_x(pk), mv_y(pk), r0, pc);
                spec_key = pk;
                spec = true;
            }
        }
        if (lane < 4 && !res_l && L.arrived(w)) {
            const int kk = (int)(unsigned)w;
            key = pack_mv(clampi(mv_x(kk), V.lox, V.hix), clampi(mv_y(kk), V.loy, V.hiy));
            res_l = true;
        }
        const unsigned before = have;
        have = __ballot_sync(kFull, lane < nc && res_l) & all;
        if (have == before && !fresh) L.idle();  // nothing arrived, nothing to cost
        if ((it & 15u) == 15u) {
            // Bounded wait: the launch's abort word, a time limit, an iteration cap.
            int give_up = 0;
            if (lane == 0) {
                const unsigned long long now = globaltimer();
                if (t_start == 0) t_start = now;
                give_up = ld_relaxed(&a.status->abort) || (long long)(now - t_start) > a.timeout_ns ||
                          it > (1u << 24);
            }
            if (__shfl_sync(kFull, give_up, 0)) {
                if (lane == 0 && !ld_relaxed(&a.status->abort)) raise_error(a.status, SME_ERR_TIMEOUT, true);
                failed = true;
                break;
            }
        }
    }
    if (failed) return false;
    int cand[5];
#pragma unroll
    for (int c = 0; c < 5; ++c) cand[c] = __shfl_sync(kFull, key, c);
    if (lane < nc) slog[lane] = key;

    // First strict minimum in the order A, B, C, T (+ seed).
    MbResult r;
    int bi = 0;
    unsigned bcost = ccost[0];
#pragma unroll
    for (int c = 1; c < 5; ++c)
        if (c < nc && ccost[c] < bcost) {
            bcost = ccost[c];
            bi = c;
        }
    if constexpr (kVariants)
        if (cls == SME_BOUNDARY && m.tt) boundary_t_by_texture(win, pitch, lx, ly, c8, cand, ccost, nc, h, bi, bcost);
    int nlog = nc;
    if (cls == SME_OPAQUE) {
        // Sec. 3.2 (the first step may be the speculative one, taken at
        // the same position).
        opaque_search<kSparse>(m, win, pitch, lx, ly, c8, ux, uy, nx, ny, V, cand, ccost, cs8, nc, bi, slog, nlog,
                               lane, spec, spec_key, sp, r);
    } else {
        int bk = cand[0];
#pragma unroll
        for (int c = 1; c < 5; ++c)
            if (c == bi) bk = cand[c];
        r.dx = mv_x(bk);
        r.dy = mv_y(bk);
        r.cost = bcost;
        r.iters = 0;
        r.lastx = r.lasty = 0.0f;
        r.r8 = ref8(win, pitch, lx, ly, r.dx, r.dy, h);  // prediction at the shape winner
    }
    r.nlog = nlog;

    // ---- publish the vector first: it is on the dependency chain ----
    L.publish(gid, pack_mv(r.dx, r.dy), lane);
    if (lane == 0) sd->mv[idx] = sme_mv{(int16_t)r.dx, (int16_t)r.dy};
    finish_mb(sd, idx, k, cls, r, c8, slog, lane, FS, W, y, x0);
    return true;
}

template <bool kVariants>
__global__ void __launch_bounds__(32 * kMeWarps) me_kernel(const MeArgs a)
{
    extern __shared__ __align__(16) uint8_t smem[];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const Method m = a.m;
    const int pitch = win_pitch(m.S);
    uint8_t* win = smem + (size_t)wid * warp_smem(m.S);
    int* slog = reinterpret_cast<int*>(win + win_bytes(m.S));
    const GlobalLinks L{a.ready, ld_relaxed(&a.status->epoch), a.fault_ticket};
    __shared__ float s_rcp[512];
    fill_rcp(s_rcp);
    __syncthreads();

    for (;;) {
        int t = 0;
        if (lane == 0) {
            t = (int)atomicAdd(&a.status->ticket, 1u);
            if (ld_relaxed(&a.status->abort)) t = a.total;
        }
        t = __shfl_sync(kFull, t, 0);
        if (t >= a.total) break;
        const int gid = __ldg(a.sched + t);
        const SeqDesc* sd = a.seqs + (a.sched_seq ? __ldg(a.sched_seq + t) : 0);
        if (!me_one_mb<GlobalLinks, kVariants>(a, m, gid, sd, win, slog, s_rcp, L, lane, pitch)) break;
    }
}


// ==================================================== host-buffer copies ==
// dst <- src for n 16-byte words, src a pinned host buffer read through its
// device mapping: every SM takes part, four loads in flight per thread, so
// the CPU-GPU link rather than the copy engines sets the rate.
__global__ void __launch_bounds__(1024) host_copy_kernel(uint4* __restrict__ dst, const uint4* __restrict__ src,
                                                         size_t n)
{
    size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    const size_t stride = (size_t)gridDim.x * blockDim.x;
    for (; i + 3 * stride < n; i += 4 * stride) {
        const uint4 a = src[i], b = src[i + stride], c = src[i + 2 * stride], d = src[i + 3 * stride];
        dst[i] = a;
        dst[i + stride] = b;
        dst[i + 2 * stride] = c;
        dst[i + 3 * stride] = d;
    }
    for (; i < n; i += stride) dst[i] = src[i];
}


// ===================================================== sparse schedule ==
// Throughput form for batches where most MBs are transparent.  Fig. 1 gives
// a transparent MB the vector (0,0) without any evaluation, so its outputs
// need only its class and the co-located prediction error; the dependency
// ordered search is needed only for the other MBs.
//   sparse_reset_kernel    zeroes the per-pair SSE, the step counts and the
//                          counters, starts a new epoch of ready words;
//   sparse_stream_kernel   one pass over every (luma group, frame, MB row):
//                          the co-located SSE of every MB once per shared
//                          luma, then for each VOP of the group the class and
//                          packed alpha rows of every MB, the outputs of its
//                          transparent MBs, the count of the other MBs per
//                          row and the VOP's first wavefront step;
//   sparse_count_kernel    MBs per list key (step relative to the VOP's first);
//   sparse_scan_kernel     key counts -> list offsets;
//   sparse_scatter_kernel  lists every non-transparent MB by key;
//   me_sparse_kernel       the per-MB search over that list only.
__global__ void __launch_bounds__(256) sparse_reset_kernel(const SparseArgs a, const SeqDesc desc, int use_desc)
{
    const int tid = threadIdx.x;
    if (blockIdx.x == 0) {
        if (tid == 0) {
            if (use_desc) *a.desc_dst = desc;
            a.status->ticket = 0;
            a.status->abort = 0;
            const unsigned e = a.status->epoch + 1u;
            a.status->epoch = e ? e : 1u;
            a.ctr->total = 0;
            a.ctr->ticket = 0;
        }
        for (int i = tid; i <= a.steps; i += blockDim.x) a.hist[8 * (size_t)i] = 0;
        for (int i = tid; i < a.rounds; i += blockDim.x) a.round_ticket[i] = 0;
    }
    for (int q = blockIdx.x; q < a.nseq; q += gridDim.x) {
        if (tid == 0) a.first_step[q] = 0x7fffffff;
        const SeqDesc& d = use_desc ? desc : a.seqs[q];
        if (d.sse)
            for (int i = tid; i < d.P; i += blockDim.x) d.sse[i] = 0ull;
    }
}

// The sequence that holds flat row r (rows of sequence q start at row_base[q]).
__device__ __forceinline__ int seq_of_row(const long long* row_base, int n, long long r)
{
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (__ldg(row_base + mid) <= r) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// Sum of squared differences of 16 packed pixels (exact integer).
__device__ __forceinline__ unsigned sq16(const uint4& x, const uint4& y)
{
    unsigned d = __vabsdiffu4(x.x, y.x), acc = __dp4a(d, d, 0u);
    d = __vabsdiffu4(x.y, y.y);
    acc = __dp4a(d, d, acc);
    d = __vabsdiffu4(x.z, y.z);
    acc = __dp4a(d, d, acc);
    d = __vabsdiffu4(x.w, y.w);
    return __dp4a(d, d, acc);
}

__global__ void __launch_bounds__(256) sparse_stream_kernel(const SparseArgs a)
{
    __shared__ unsigned long long s_sse[kGroupMax];
    __shared__ unsigned s_cnt[kGroupMax];
    __shared__ int s_umin[kGroupMax];
    const int v = blockIdx.x, gf = blockIdx.y, tid = threadIdx.x;
    const int grp = __ldg(a.gf_group + gf), f = __ldg(a.gf_frame + gf);
    const int m0 = __ldg(a.grp_first + grp), nm = __ldg(a.grp_first + grp + 1) - m0;
    const SeqDesc* s0 = a.seqs + __ldg(a.grp_members + m0);
    const int W = s0->W, H = s0->H, MBW = s0->MBW, MBH = s0->MBH, M = s0->M, Wp = s0->Wp, rd = s0->rd;
    if (v >= MBH) return;
    const int k = f - rd;  // the pair whose current frame is f (none when negative)
    for (int j = tid; j < nm; j += blockDim.x) {
        s_sse[j] = 0ull;
        s_cnt[j] = 0u;
        s_umin[j] = 0x7fffffff;
    }
    __syncthreads();
    const size_t FS = (size_t)W * H;
    const int hw = 2 * Wp;  // u16 slots per packed row (the slots from MBW on stay zero)
    const int lane = tid & 31;
    // Warp-uniform passes over the MB columns u (lane = column), so the
    // per-VOP counts and sums are warp reductions, not shared atomics.
    for (int u0 = tid & ~31; u0 < hw; u0 += blockDim.x) {
        const int u = u0 + lane;
        const bool col = u < MBW;
        const size_t px = (size_t)(16 * v) * W + 16 * (col ? u : 0);
        // Sec. 4: the co-located prediction error of the MB, shared by every
        // VOP of the group (a transparent MB predicts from (0,0)).
        unsigned sse0 = 0;
        if (k >= 0 && col) {
            const uint8_t* cur = s0->luma + (size_t)f * FS + px;
            const uint8_t* ref = s0->luma + (size_t)k * FS + px;
#pragma unroll 4
            for (int r = 0; r < 16; ++r)
                sse0 += sq16(__ldg(reinterpret_cast<const uint4*>(cur + (size_t)r * W)),
                             __ldg(reinterpret_cast<const uint4*>(ref + (size_t)r * W)));
        }
        for (int j = 0; j < nm; ++j) {
            const SeqDesc* sd = a.seqs + __ldg(a.grp_members + m0 + j);
            uint16_t* pk = reinterpret_cast<uint16_t*>(sd->packed_w + ((size_t)f * H + 16 * v) * Wp);
            int cls = SME_TRANSPARENT;
            if (col) {
                const uint8_t* al = sd->alpha + (size_t)f * FS + px;
                unsigned n = 0;
#pragma unroll 8
                for (int r = 0; r < 16; ++r) {
                    const unsigned bits = bab_bits16(al + (size_t)r * W);
                    n += __popc(bits);
                    pk[(size_t)r * hw + u] = (uint16_t)bits;
                }
                cls = n == 0 ? SME_TRANSPARENT : (n == 256 ? SME_OPAQUE : SME_BOUNDARY);
                sd->cls_w[(size_t)f * M + v * MBW + u] = (uint8_t)cls;
            } else if (u < hw) {
#pragma unroll
                for (int r = 0; r < 16; ++r) pk[(size_t)r * hw + u] = 0;
            }
            if (k < 0) continue;  // uniform: frames before the first pair's current frame
            const unsigned listed = __ballot_sync(kFull, col && cls != SME_TRANSPARENT);
            if (lane == 0 && listed) {
                atomicAdd(&s_cnt[j], (unsigned)__popc(listed));
                atomicMin(&s_umin[j], u0 + __ffs(listed) - 1);
            }
            const bool tr = col && cls == SME_TRANSPARENT;
            if (sd->sse) {  // below 32 x 2^24: one 32-bit reduction
                const unsigned ws = __reduce_add_sync(kFull, tr ? sse0 : 0u);
                if (lane == 0 && ws) atomicAdd(&s_sse[j], (unsigned long long)ws);
            }
            if (!tr) continue;
            // Fig. 1: no vector is computed for a transparent MB.
            const size_t idx = (size_t)k * M + v * MBW + u;
            sd->mv[idx] = sme_mv{0, 0};
            if (sd->cost) sd->cost[idx] = 0;
            if (sd->disp) {
                sd->disp[2 * idx] = 0.0f;
                sd->disp[2 * idx + 1] = 0.0f;
            }
            if (sd->iters) sd->iters[idx] = 0;
            if (sd->npos) sd->npos[idx] = 0;
            if (sd->out_cls) sd->out_cls[idx] = (uint8_t)SME_TRANSPARENT;
            if (sd->sse_mb) sd->sse_mb[idx] = sse0;
            if (sd->pred) {
                const uint8_t* ref = sd->luma + (size_t)k * FS + px;
                uint8_t* pr = sd->pred + (size_t)k * FS + px;
#pragma unroll 4
                for (int r = 0; r < 16; ++r) {  // 8-byte stores, as every kernel writes the prediction
                    const uint4 q = __ldg(reinterpret_cast<const uint4*>(ref + (size_t)r * W));
                    *reinterpret_cast<uint2*>(pr + (size_t)r * W) = make_uint2(q.x, q.y);
                    *reinterpret_cast<uint2*>(pr + (size_t)r * W + 8) = make_uint2(q.z, q.w);
                }
            }
        }
    }
    __syncthreads();
    for (int j = tid; j < nm; j += blockDim.x) {
        const int q = __ldg(a.grp_members + m0 + j);
        const SeqDesc* sd = a.seqs + q;
        a.rowcnt[__ldg(a.row_base + q) + (long long)f * MBH + v] = s_cnt[j];
        if (k >= 0 && sd->sse && s_sse[j]) atomicAdd(sd->sse + k, s_sse[j]);
        // the VOP's first wavefront step t = u + 2v + k with a listed MB
        if (s_cnt[j]) atomicMin(a.first_step + q, s_umin[j] + 2 * v + k);
    }
}

// The list key of a non-transparent MB: its wavefront step t = u + 2v + k
// minus its VOP's first such step.  The shift is constant within a VOP, so
// every dependency (A, B, C of the same pair, T of the previous pair: steps
// t - 1 and t - 2) keeps a smaller key; VOPs have no dependencies on each
// other, so aligning their first steps lets all of them start at once
// instead of waiting for the work of other VOPs at smaller absolute steps.
__device__ __forceinline__ int list_key(const SparseArgs& a, int q, int u, int v, int k)
{
    if (a.pair_keys) return k * a.pair_keys + u + 2 * v;  // pair rounds: A, B, C before, T a round earlier
    return u + 2 * v + k - __ldg(a.first_step + q);
}

// Shared by the counting and the scattering pass: warps walk the row counts
// 32 at a time and visit every non-transparent MB of the rows that have any.
template <class Visit>
__device__ __forceinline__ void sparse_walk(const SparseArgs& a, Visit visit)
{
    const int lane = threadIdx.x & 31;
    const long long nw = (long long)gridDim.x * (blockDim.x >> 5);
    for (long long r0 = ((long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5)) * 32; r0 < a.total_rows;
         r0 += nw * 32) {
        const long long r = r0 + lane;
        const unsigned c = r < a.total_rows ? a.rowcnt[r] : 0u;
        unsigned todo = __ballot_sync(kFull, c != 0);
        while (todo) {
            const int l = __ffs(todo) - 1;
            todo &= todo - 1;
            const long long rr = r0 + l;
            const int q = seq_of_row(a.row_base, a.nseq, rr);
            const SeqDesc* sd = a.seqs + q;
            const long long loc = rr - __ldg(a.row_base + q);
            const int f = (int)(loc / sd->MBH), v = (int)(loc - (long long)f * sd->MBH);
            const int k = f - sd->rd, MBW = sd->MBW;
            for (int u = lane; u < MBW; u += 32) {
                const int mb = v * MBW + u;
                if (sd->cls[(size_t)f * sd->M + mb] != SME_TRANSPARENT)
                    visit(list_key(a, q, u, v, k), sd->gid_base + k * sd->M + mb);
            }
        }
    }
}

__global__ void __launch_bounds__(256) sparse_count_kernel(const SparseArgs a)
{
    sparse_walk(a, [&](int key, int) { atomicAdd(a.hist + 8 * (size_t)key, 1u); });
}

// One CTA: exclusive prefix sums of the step counts (list offsets), the
// cursors of the scatter, and the list length.
__global__ void __launch_bounds__(1024) sparse_scan_kernel(const SparseArgs a)
{
    __shared__ unsigned wsum[32];
    __shared__ unsigned carry;
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    if (tid == 0) carry = 0;
    __syncthreads();
    for (int base = 0; base < a.steps; base += 1024) {
        const int i = base + tid;
        const unsigned x = i < a.steps ? a.hist[8 * (size_t)i] : 0u;
        unsigned inc = x;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned y = __shfl_up_sync(kFull, inc, o);
            if (lane >= o) inc += y;
        }
        if (lane == 31) wsum[wid] = inc;
        __syncthreads();
        if (wid == 0) {
            unsigned w = wsum[lane], wi = w;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const unsigned y = __shfl_up_sync(kFull, wi, o);
                if (lane >= o) wi += y;
            }
            wsum[lane] = wi - w;  // exclusive prefix of the warps
        }
        __syncthreads();
        const unsigned excl = carry + wsum[wid] + inc - x;
        if (i < a.steps) {
            a.hist[8 * (size_t)i] = excl;  // kept: the pair rounds' list segments
            a.cursor[8 * (size_t)i] = excl;
        }
        __syncthreads();
        if (tid == 1023) carry = excl + x;
        __syncthreads();
    }
    if (tid == 0) {
        a.ctr->total = carry;
        a.hist[8 * (size_t)a.steps] = carry;
    }
}

// Every non-transparent MB goes to the next slot of its key.
__global__ void __launch_bounds__(256) sparse_scatter_kernel(const SparseArgs a)
{
    sparse_walk(a, [&](int key, int gid) { a.list[atomicAdd(a.cursor + 8 * (size_t)key, 1u)] = gid; });
}

// The sequence of global MB id gid (sequences' ids start at seq_base[q]).
__device__ __forceinline__ int seq_of_gid(const int* seq_base, int n, int gid)
{
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (__ldg(seq_base + mid) <= gid) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// The per-MB search over the list of non-transparent MBs.  Every dependency
// of an MB has a smaller key, hence an earlier ticket, so the warps (all
// resident) can always make progress, as in me_kernel.
// kMinBlocks: CTAs per SM the register budget is cut for (1: one 8-warp CTA
// per SM, 2: two without spills, 3: three with some spills; 5: five CTAs of
// 4 warps, 20 warps per SM at 96 registers), chosen by tuning.
template <bool kVariants, int kMinBlocks>
__global__ void __launch_bounds__(32 * sparse_cta_warps(kMinBlocks), kMinBlocks) me_sparse_kernel(const MeArgs a)
{
    extern __shared__ __align__(16) uint8_t smem[];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const Method m = a.m;
    const int pitch = win_pitch(m.S);
    uint8_t* win = smem + (size_t)wid * warp_smem(m.S);
    int* slog = reinterpret_cast<int*>(win + win_bytes(m.S));
    const GlobalLinks L{a.ready, ld_relaxed(&a.status->epoch), a.fault_ticket};
    __shared__ float s_rcp[512];
    fill_rcp(s_rcp);
    __syncthreads();
    // The whole list, or (pair rounds) the segment of pair `round`, whose
    // T candidates were published by the previous round's launch.
    unsigned begin = 0, total = ld_relaxed(&a.ctr->total);
    unsigned* ticket = &a.ctr->ticket;
    if (a.round >= 0) {
        begin = __ldg(a.offs + 8 * (size_t)a.round * a.pair_keys);
        total = __ldg(a.offs + 8 * (size_t)(a.round + 1) * a.pair_keys);
        ticket = a.round_ticket + a.round;
    }
    // The next ticket is taken while the current MB is searched (a warp holds
    // at most one ticket it has not started, later than its current one,
    // which keeps the progress argument above).
    unsigned t = 0;
    if (lane == 0) t = begin + atomicAdd(ticket, 1u);
    t = __shfl_sync(kFull, t, 0);
    while (t < total) {
        unsigned next = 0;
        if (lane == 0) next = ld_relaxed(&a.status->abort) ? total : begin + atomicAdd(ticket, 1u);
        const int gid = __ldg(a.list + t);
        const SeqDesc* sd = a.seqs + seq_of_gid(a.seq_base, a.nseq, gid);
        if (!me_one_mb<GlobalLinks, kVariants, true>(a, m, gid, sd, win, slog, s_rcp, L, lane, pitch)) return;
        t = __shfl_sync(kFull, next, 0);
    }
}


// ============================================ ME, one cluster per sequence ==
// The first cluster of the launch (the chain cluster) estimates every
// non-transparent MB of one sequence; the other clusters (helpers) finish the
// transparent MBs, whose vector (0,0) is known from the classes alone.  The
// host deals all MBs, in wavefront order, round robin to the chain cluster's
// CTAs (a.cl_items: CTA r's list, a.cl_cap entries apart; a.cl_count[r]
// items).  Each CTA keeps the non-transparent items of its list (order kept),
// fills the slots whose producer is transparent with (0,0) itself, and its
// warps take the kept items in order; every other dependency travels through
// ClusterLinks, so no link is polled through L2.  Deadlock-free for the same
// reason as the per-MB schedule: an item waits only on items of smaller
// wavefront step, which every CTA takes first.  Dynamic shared memory: the
// warps' windows, the item slots, the kept-item list.
__device__ __forceinline__ int item_class(const SeqDesc* sd, int gid)
{
    const int k = gid / sd->M, mb = gid - k * sd->M;
    return __ldg(sd->cls + (size_t)(k + sd->rd) * sd->M + mb);
}

__device__ __forceinline__ void cluster_sync_all()
{
    asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}

__global__ void __launch_bounds__(32 * kClusterWarps, 1) me_cluster_kernel(const MeArgs a)
{
    extern __shared__ __align__(16) uint8_t smem[];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, tid = threadIdx.x, nw = blockDim.x >> 5;
    const Method m = a.m;
    const SeqDesc* sd = a.seqs;
    unsigned rank, cid, csize;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(rank));
    asm volatile("mov.u32 %0, %%clusterid.x;" : "=r"(cid));
    asm volatile("mov.u32 %0, %%cluster_nctarank;" : "=r"(csize));

    if (cid > 0) {
        // ---- helpers: outputs and prediction error of every transparent MB
        const int nhw = ((int)gridDim.x - (int)csize) * nw;
        const int W = sd->W, M = sd->M, MBW = sd->MBW, rd = sd->rd;
        const size_t FS = (size_t)W * sd->H;
        for (int gid = ((int)blockIdx.x - (int)csize) * nw + wid; gid < a.total; gid += nhw) {
            if (item_class(sd, gid) != SME_TRANSPARENT) continue;
            const int k = gid / M, mb = gid - k * M, u = mb % MBW, v = mb / MBW;
            const int x0 = 16 * u + 8 * (lane & 1), y = 16 * v + (lane >> 1);
            const uint8_t* ref = sd->luma + (size_t)k * FS;
            const P8 c8 = load8(sd->luma + (size_t)(k + rd) * FS + (size_t)y * W + x0);
            transparent_mb(sd, gid, k, ref, c8, lane, FS, W, y, x0);
        }
        return;
    }

    // ---- the chain cluster
    const int pitch = win_pitch(m.S);
    uint8_t* win = smem + (size_t)wid * warp_smem(m.S);
    int* slog = reinterpret_cast<int*>(win + win_bytes(m.S));
    unsigned long long* slots =
        reinterpret_cast<unsigned long long*>(smem + (size_t)nw * warp_smem(m.S));
    int* work = reinterpret_cast<int*>(slots + 4 * (size_t)a.cl_cap);  // kept positions, then their MB ids
    __shared__ float s_rcp[512];
    __shared__ int s_ticket, s_nwork, s_warp[kClusterWarps];
    const int n_items = __ldg(a.cl_count + rank);
    const int* items = a.cl_items + (size_t)rank * a.cl_cap;
    for (int i = tid; i < 4 * n_items; i += blockDim.x) slots[i] = 0ull;
    if (tid == 0) s_ticket = 0;
    fill_rcp(s_rcp);
    // Keep the non-transparent items, in order: each thread counts a
    // contiguous chunk, a block scan gives its offset, then it writes them.
    const int per = (n_items + (int)blockDim.x - 1) / (int)blockDim.x;
    const int i0 = min(n_items, tid * per), i1 = min(n_items, i0 + per);
    int cnt = 0;
    for (int i = i0; i < i1; ++i) cnt += item_class(sd, __ldg(items + i)) != SME_TRANSPARENT;
    int incl = cnt;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int t = __shfl_up_sync(kFull, incl, o);
        if (lane >= o) incl += t;
    }
    if (lane == 31) s_warp[wid] = incl;
    __syncthreads();
    int base = 0;
    for (int w = 0; w < wid; ++w) base += s_warp[w];
    if (tid == blockDim.x - 1) s_nwork = base + incl;
    int o = base + incl - cnt;
    for (int i = i0; i < i1; ++i)
        if (item_class(sd, __ldg(items + i)) != SME_TRANSPARENT) work[o++] = i;
    __syncthreads();
    int* work_gid = work + s_nwork;
    for (int j = tid; j < s_nwork; j += blockDim.x) work_gid[j] = __ldg(items + work[j]);
    // A transparent producer's vector is (0,0): its consumers' slots here are
    // filled now rather than by the producer.
    const int n_work = s_nwork, M = sd->M, MBW = sd->MBW;
    for (int j = tid; j < n_work; j += blockDim.x) {
        const int i = work[j], gid = work_gid[j];
        const int k = gid / M, mb = gid - k * M, u = mb % MBW, v = mb / MBW;
        const int prod[4] = {u > 0 ? gid - 1 : -1, v > 0 ? gid - MBW : -1,
                             (v > 0 && u < MBW - 1) ? gid - MBW + 1 : -1, k > 0 ? gid - M : -1};
#pragma unroll
        for (int role = 0; role < 4; ++role)
            if (prod[role] >= 0 && item_class(sd, prod[role]) == SME_TRANSPARENT) slots[4 * i + role] = 1ull << 32;
    }
    // every slot of the cluster is settled before any producer stores into it
    cluster_sync_all();

    for (;;) {
        int t = 0;
        if (lane == 0) {
            t = atomicAdd(&s_ticket, 1);
            if (ld_relaxed(&a.status->abort)) t = n_work;
        }
        t = __shfl_sync(kFull, t, 0);
        if (t >= n_work) break;
        const int i = work[t], gid = work_gid[t];
        // the consumer slots are fetched now; they are needed only at the end
        const int cons = lane < 4 ? __ldg(a.cl_consumers + 4 * (size_t)gid + lane) : -1;
        const ClusterLinks L{slots, i, cons, a.fault_ticket};
        if (!me_one_mb<ClusterLinks, true>(a, m, gid, sd, win, slog, s_rcp, L, lane, pitch)) break;
    }
    // no CTA leaves while a peer may still store into its slots
    cluster_sync_all();
}

// ================================================ ME, per-pair CTAs ==
// One CTA processes one frame pair of one sequence at a time (tickets in
// pair order, so the previous pair -- the T candidate -- was always taken
// earlier).  Warp w handles MB rows w, w + nw, ... left to right: the A
// candidate is the warp's own previous vector, B and C come from the row
// above through a ring of nw + 1 row slots in shared memory (a row's slot is
// reused only after the row below it -- this warp's previous row -- is done),
// and T comes from the previous pair's ready words in global memory, loaded
// one MB ahead.  Everything else an MB reads -- the reference window, the
// current block with a one-pixel halo, and the packed alpha rows of both
// frames -- is fetched by TMA into the warp's other buffer while the current
// MB is searched, so the only wait on the row's path is the row above.

__host__ __device__ __forceinline__ int ceil128(int v) { return (v + 127) & ~127; }

// Packed-alpha words of the reference strip: enough for every full-pel
// shift of V plus the funnel-shift word and the 4-word alignment of the box.
__host__ __device__ __forceinline__ int aref_words(int S) { return (((2 * S + 15) >> 5) + 6 + 3) & ~3; }
constexpr int kCurBoxW = 48, kCurBoxH = 18;  // current block + halo: x from X0-16, y from Y0-1
constexpr int kAcurWords = 4;                // current BAB: 16 rows x 4 words from (X0>>5)&~3

struct PairLayout {
    int o_ref, o_cur, o_aref, o_acur, buf_bytes;  // one buffer (all sections 128-byte aligned)
    int cls_off;                                  // the warp's copy of its row's MB classes
    int log_off, bar_off, warp_bytes;
    int R;                                        // row slots
    int rows_off, prog_off, unit_off, total;
};

__host__ __device__ __forceinline__ PairLayout pair_layout(int S, int nw, int mbw_max, bool four_mv = false)
{
    PairLayout L;
    L.o_ref = 0;
    L.o_cur = L.o_ref + ceil128(win_rows(S) * win_pitch(S) + 32);
    L.o_aref = L.o_cur + ceil128(kCurBoxW * kCurBoxH + 16);
    L.o_acur = L.o_aref + ceil128(aref_words(S) * 4 * win_rows(S));
    L.buf_bytes = L.o_acur + ceil128(kAcurWords * 4 * 16);
    L.log_off = 2 * L.buf_bytes;
    L.bar_off = L.log_off + ceil16(kMaxLog * 4 * (four_mv ? 4 : 1));  // one log per 8x8 block in that mode
    L.cls_off = L.bar_off + 16;
    L.warp_bytes = ceil128(L.cls_off + ceil16(mbw_max));
    L.R = nw + 1;
    L.rows_off = nw * L.warp_bytes;
    L.prog_off = L.rows_off + ceil16(L.R * mbw_max * 4);
    L.unit_off = L.prog_off + ceil16(L.R * 4);
    L.total = L.unit_off + 16;
    return L;
}

__host__ __device__ __forceinline__ unsigned pair_tx_bytes(int S)
{
    return (unsigned)(win_rows(S) * win_pitch(S) + kCurBoxW * kCurBoxH + aref_words(S) * 4 * win_rows(S) +
                      kAcurWords * 4 * 16);
}

__device__ __forceinline__ unsigned smem_u32(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* bar)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, unsigned parity)
{
    unsigned ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
// Bounded wait for the TMA copies that fill a buffer.
__device__ bool mbar_wait(uint64_t* bar, unsigned parity, long long timeout_ns)
{
    if (mbar_try_wait(bar, parity)) return true;
    const unsigned long long t0 = globaltimer();
    for (unsigned it = 1; it < (1u << 24); ++it) {
        if (mbar_try_wait(bar, parity)) return true;
        if ((it & 15u) == 0 && (long long)(globaltimer() - t0) > timeout_ns) return false;
    }
    return false;
}
// 3-D tiled TMA load of one box at (x, y, z) into dst, completing on bar.
// x * element size is a multiple of 16 bytes; x and y may be negative or run
// past the tensor, where the box is filled with zeros.
__device__ __forceinline__ void tma_box(void* dst, const CUtensorMap* map, int x, int y, int z, uint64_t* bar)
{
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], "
        "[%5];" ::"r"(smem_u32(dst)),
        "l"(map), "r"(x), "r"(y), "r"(z), "r"(smem_u32(bar))
        : "memory");
}

// The four tensor maps of one sequence (luma window, current block, packed
// alpha strips of the reference and current frames).
struct alignas(128) PairMaps {
    CUtensorMap ref, cur, aref, acur;
};

// Issue the four boxes of MB (X0, Y0) of pair k into buffer `buf`.
__device__ __forceinline__ void issue_mb_boxes(uint8_t* buf, const PairLayout& L, const PairMaps* mp, int S, int X0,
                                               int Y0, int k, int kc, uint64_t* bar, unsigned tx)
{
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(tx) : "memory");
    tma_box(buf + L.o_ref, &mp->ref, X0 - ceil16(S), Y0 - S, k, bar);
    tma_box(buf + L.o_cur, &mp->cur, X0 - 16, Y0 - 1, kc, bar);
    tma_box(buf + L.o_aref, &mp->aref, ((X0 - S) >> 5) & ~3, Y0 - S, k, bar);
    tma_box(buf + L.o_acur, &mp->acur, (X0 >> 5) & ~3, Y0, kc, bar);
}

__device__ __forceinline__ int ld_acquire_cta(const int* p)
{
    int v;
    asm volatile("ld.acquire.cta.shared::cta.u32 %0, [%1];" : "=r"(v) : "r"(smem_u32(p)) : "memory");
    return v;
}
__device__ __forceinline__ void st_release_cta(int* p, int v)
{
    asm volatile("st.release.cta.shared::cta.u32 [%0], %1;" ::"r"(smem_u32(p)), "r"(v) : "memory");
}
// Bounded wait until the row slot's progress word reaches `target`.
__device__ bool wait_progress(const int* prog, int target, const DevStatus* st, long long timeout_ns)
{
    if (ld_acquire_cta(prog) >= target) return true;
    const unsigned long long t0 = globaltimer();
    for (unsigned it = 1; it < (1u << 26); ++it) {
        if (ld_acquire_cta(prog) >= target) return true;
        if ((it & 63u) == 0) {
            if (ld_relaxed(&st->abort)) return false;
            if ((long long)(globaltimer() - t0) > timeout_ns) return false;
        }
    }
    return false;
}

// Shape costs from the staged packed-alpha strips (same arithmetic as
// shape_costs): lane l takes row l&15 of candidates (l>>4) + 2j.
__device__ __forceinline__ void shape_costs_smem(const uint32_t* acur, const uint32_t* aref, int arw, int S, int X0,
                                                 const int (&cand)[5], int nc, int h, int lane, unsigned (&cost)[5])
{
    const int r = lane & 15, half = lane >> 4;
    const unsigned cb = (acur[r * kAcurWords + (X0 >> 5) - ((X0 >> 5) & ~3)] >> (X0 & 31)) & 0xffffu;
    const int xw0 = ((X0 - S) >> 5) & ~3;
    unsigned s[3] = {0u, 0u, 0u};
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        const int c = half + 2 * j;
        if (c < nc) {
            int key = cand[0];
#pragma unroll
            for (int q = 1; q < 5; ++q)
                if (q == c) key = cand[q];
            const int fdx = mv_x(key) / h, fdy = mv_y(key) / h;  // trunc toward zero
            const int xr = X0 + fdx, wr = (xr >> 5) - xw0;
            const uint32_t* row = aref + (r + fdy + S) * arw;
            const unsigned rb = __funnelshift_r(row[wr], row[wr + 1], xr & 31) & 0xffffu;
            s[j] = __popc(cb ^ rb);
        }
    }
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        s[j] += __shfl_xor_sync(kFull, s[j], 8);
        s[j] += __shfl_xor_sync(kFull, s[j], 4);
        s[j] += __shfl_xor_sync(kFull, s[j], 2);
        s[j] += __shfl_xor_sync(kFull, s[j], 1);
    }
    cost[0] = __shfl_sync(kFull, s[0], 0);
    cost[1] = __shfl_sync(kFull, s[0], 16);
    cost[2] = __shfl_sync(kFull, s[1], 0);
    cost[3] = __shfl_sync(kFull, s[1], 16);
    cost[4] = __shfl_sync(kFull, s[2], 0);
}

// Eq. 4 factors from the staged current block (box row 1 + (lane>>1), box
// column 16 + 8*(lane&1) is the lane's first pixel).
__device__ __forceinline__ void factors_smem(const uint8_t* cb, int W, int H, int x0, int y, const P8& c,
                                             float theta, const float* rcp, float (&ux)[8], float (&uy)[8],
                                             int& nx, int& ny, int lane)
{
    const float lim = 2.0f * theta;
    const uint8_t* row = cb + (1 + (lane >> 1)) * kCurBoxW + 16 + 8 * (lane & 1);
    const int left = row[-1], right = row[8];
    P8 up, dn;
    {
        const uint2 t = *reinterpret_cast<const uint2*>(row - kCurBoxW);
        up.lo = t.x;
        up.hi = t.y;
        const uint2 b = *reinterpret_cast<const uint2*>(row + kCurBoxW);
        dn.lo = b.x;
        dn.hi = b.y;
    }
    int cx = 0, cy = 0;
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        const int x = x0 + k;
        ux[k] = 0.0f;
        uy[k] = 0.0f;
        if (x > 0 && x < W - 1) {
            const int rr = k < 7 ? byte_of(c, k + 1) : right;
            const int ll = k > 0 ? byte_of(c, k - 1) : left;
            const int g = rr - ll;
            if (fabsf((float)g) >= lim) ux[k] = rcp[g + 255];
        }
        if (y > 0 && y < H - 1) {
            const int g = byte_of(dn, k) - byte_of(up, k);
            if (fabsf((float)g) >= lim) uy[k] = rcp[g + 255];
        }
        cx += ux[k] != 0.0f;
        cy += uy[k] != 0.0f;
    }
    nx = (int)__reduce_add_sync(kFull, (unsigned)cx);
    ny = (int)__reduce_add_sync(kFull, (unsigned)cy);
}

// First MB at or after `from` in the row whose class is not transparent (n if none).
__device__ __forceinline__ int next_visible(const uint8_t* rowcls, int from, int n, int lane)
{
    for (int b = from; b < n; b += 32) {
        const unsigned bal = __ballot_sync(kFull, b + lane < n && rowcls[b + lane] != SME_TRANSPARENT);
        if (bal) return b + __ffs(bal) - 1;
    }
    return n;
}

// Transparent MBs u0..u1-1 of row v of pair k (Fig. 1: no vector, (0,0) is
// final at once): published to the row below and the next pair, and their
// outputs and co-located prediction error computed from global memory, four
// MBs per pass so that their loads are in flight together.
__device__ __forceinline__ void transparent_run(const SeqDesc* sd, const MeArgs& a, int k, int v, int u0, int u1,
                                                int base, int slot, int* rowmv, int* prog, unsigned long long tag,
                                                int lane)
{
    const int W = sd->W, MBW = sd->MBW, M = sd->M, y = 16 * v + (lane >> 1);
    const size_t FS = (size_t)W * sd->H;
    const uint8_t* ref = sd->luma + (size_t)k * FS + (size_t)y * W;
    const uint8_t* cur = sd->luma + (size_t)(k + sd->rd) * FS + (size_t)y * W;
    for (int u = u0; u < u1; u += 4) {
        const int n = min(4, u1 - u);
        P8 c8[4], r8[4];
#pragma unroll
        for (int j = 0; j < 4; ++j)
            if (j < n) {
                const int x0 = 16 * (u + j) + 8 * (lane & 1);
                c8[j] = load8(cur + x0);
                const uint2 t2 = __ldg(reinterpret_cast<const uint2*>(ref + x0));
                r8[j].lo = t2.x;
                r8[j].hi = t2.y;
            }
#pragma unroll
        for (int j = 0; j < 4; ++j)
            if (j < n) {
                const int mb = v * MBW + u + j, idx = k * M + mb, gid = base + mb;
                if (lane == 0) {
                    rowmv[slot * a.mbw_max + u + j] = 0;
                    st_release_cta(&prog[slot], v * 1024 + u + j + 1);
                    if (gid != a.fault_ticket) st_ready(a.ready + gid, tag);
                    sd->mv[idx] = sme_mv{0, 0};
                    if (sd->cost) sd->cost[idx] = 0;
                    if (sd->disp) {
                        sd->disp[2 * idx] = 0.0f;
                        sd->disp[2 * idx + 1] = 0.0f;
                    }
                    if (sd->iters) sd->iters[idx] = 0;
                    if (sd->npos) sd->npos[idx] = 0;
                    if (sd->out_cls) sd->out_cls[idx] = (uint8_t)SME_TRANSPARENT;
                }
                if (sd->pred)
                    *reinterpret_cast<uint2*>(sd->pred + (size_t)k * FS + (size_t)y * W + 16 * (u + j) + 8 * (lane & 1)) =
                        make_uint2(r8[j].lo, r8[j].hi);
                if (sd->sse || sd->sse_mb) {
                    const unsigned e = __reduce_add_sync(kFull, sq8(r8[j], c8[j]));
                    if (lane == 0) {
                        if (sd->sse) atomicAdd(sd->sse + k, (unsigned long long)e);
                        if (sd->sse_mb) sd->sse_mb[idx] = e;
                    }
                }
            }
    }
    __syncwarp();
}


// ===================================================== four vectors per MB ==
// Sec. 3.2 with 8x8 blocks (MPEG-4's four vectors per MB).  Lane l holds the
// 8 pixels of MB row l>>1, columns 8*(l&1)..+7, which lie in block
// b = 2*((l>>1) >= 8) + (l&1); the 8 lanes of a block differ in bits 1-3 of l
// (bit 1-3 = the row inside the block), so block sums are xor shuffles over
// bits 1, 2, 3 and every lane of the block holds the same block state.
__device__ __forceinline__ int blk_of(int lane) { return ((lane >> 4) << 1) | (lane & 1); }

__device__ __forceinline__ unsigned blk_sum(unsigned v)
{
    v += __shfl_xor_sync(kFull, v, 2);
    v += __shfl_xor_sync(kFull, v, 4);
    v += __shfl_xor_sync(kFull, v, 8);
    return v;
}

// Two block sums of values whose block totals stay below 2^16 (SADs of an
// 8x8 block: at most 64 * 255), in one pass of shuffles.
__device__ __forceinline__ void blk_sum2(unsigned a, unsigned b, unsigned& sa, unsigned& sb)
{
    const unsigned t = blk_sum(a | (b << 16));
    sa = t & 0xffffu;
    sb = t >> 16;
}

// Eq. 3 sums over the block's 64 pixels: the lane's 8 terms pairwise, then
// rows pairwise (xor 2, 4, 8): the contiguous pairwise tree in block raster
// order (FP32 addition is commutative, so both lanes of a pair agree).
__device__ __forceinline__ void blk_grad_sums(const P8& r, const P8& c, const float (&ux)[8], const float (&uy)[8],
                                              float& sx, float& sy)
{
    float tx[8], ty[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        const float dpd = (float)(byte_of(r, k) - byte_of(c, k));
        tx[k] = __fmul_rn(dpd, ux[k]);
        ty[k] = __fmul_rn(dpd, uy[k]);
    }
    float a = __fadd_rn(__fadd_rn(__fadd_rn(tx[0], tx[1]), __fadd_rn(tx[2], tx[3])),
                        __fadd_rn(__fadd_rn(tx[4], tx[5]), __fadd_rn(tx[6], tx[7])));
    float b = __fadd_rn(__fadd_rn(__fadd_rn(ty[0], ty[1]), __fadd_rn(ty[2], ty[3])),
                        __fadd_rn(__fadd_rn(ty[4], ty[5]), __fadd_rn(ty[6], ty[7])));
#pragma unroll
    for (int o = 2; o <= 8; o <<= 1) {
        a = __fadd_rn(a, __shfl_xor_sync(kFull, a, o));
        b = __fadd_rn(b, __shfl_xor_sync(kFull, b, o));
    }
    sx = a;
    sy = b;
}

// The state of the lane's block.
struct Blk4 {
    int dx, dy, iters, nlog;
    unsigned cost;
    float lastx, lasty;
    P8 r8;
    bool done;
};

// Pixel recursive search of the four blocks at once, each from the MB winner
// (already in s), in the order of prs_run: proposal if strictly lower, else
// the first strict minimum of the eight clamped neighbours, else stop; at
// most K steps.  Positions go to the block's own log (blog) from its first
// lane.  Control flow is uniform over the warp; blocks that have stopped
// compute along and discard.
__device__ __forceinline__ void prs_blocks(const Method& m, const uint8_t* win, int pitch, int lx, int ly,
                                           const P8& c8, const float (&ux)[8], const float (&uy)[8], int nxb, int nyb,
                                           const VRange& V, Blk4& s, int* blog, int lane)
{
    const int h = m.h;
    const bool first = (lane & 14) == 0;
    for (int it = 0; it < m.K; ++it) {
        if (!__any_sync(kFull, !s.done)) break;
        float sx, sy;
        blk_grad_sums(s.r8, c8, ux, uy, sx, sy);
        const float ux_ = update_of(sx, nxb, m.eps), uy_ = update_of(sy, nyb, m.eps);
        const int qx = clampi(s.dx + (int)roundf(__fmul_rn((float)h, ux_)), V.lox, V.hix);
        const int qy = clampi(s.dy + (int)roundf(__fmul_rn((float)h, uy_)), V.loy, V.hiy);
        const bool qmove = qx != s.dx || qy != s.dy;
        // The lane's samples at the 3x3 neighbourhood of its block's d (one
        // staged read when d is inside V, so that clamping is the identity;
        // clamped one by one on the edge of V), and at the proposal q.
        P8 nb9[9];
        const bool inner = s.dx > V.lox && s.dx < V.hix && s.dy > V.loy && s.dy < V.hiy;
        if (inner) {
            block3x3(win, pitch, lx, ly, s.dx, s.dy, h, nb9);
        } else {
#pragma unroll
            for (int n = 0; n < 9; ++n)
                nb9[n] = n == 4 ? s.r8
                                : ref8(win, pitch, lx, ly, clampi(s.dx + n % 3 - 1, V.lox, V.hix),
                                       clampi(s.dy + n / 3 - 1, V.loy, V.hiy), h);
        }
        P8 q8;
        if (abs(qx - s.dx) <= 1 && abs(qy - s.dy) <= 1 && (inner || !qmove)) {
            const int qi = (qy - s.dy + 1) * 3 + (qx - s.dx + 1);
            q8 = nb9[4];
#pragma unroll
            for (int n = 0; n < 9; ++n)
                if (n == qi) q8 = nb9[n];
        } else {
            q8 = ref8(win, pitch, lx, ly, qx, qy, h);
        }
        const unsigned cq = blk_sum(sad8(q8, c8));
        bool moved = false, need_nb = false;
        if (!s.done) {
            ++s.iters;
            s.lastx = ux_;
            s.lasty = uy_;
            if (qmove) {
                if (first) blog[s.nlog] = pack_mv(qx, qy);
                ++s.nlog;
                moved = cq < s.cost;
            }
            need_nb = !moved;
        }
        if (moved) {
            s.dx = qx;
            s.dy = qy;
            s.cost = cq;
            s.r8 = q8;
        }
        if (__any_sync(kFull, need_nb)) {
            const int cx = s.dx, cy = s.dy;  // unchanged where need_nb
            unsigned bc = s.cost;
            int bx = cx, by = cy;
            P8 b8 = s.r8;
            unsigned sad9[9];
            blk_sum2(sad8(nb9[0], c8), sad8(nb9[1], c8), sad9[0], sad9[1]);
            blk_sum2(sad8(nb9[2], c8), sad8(nb9[3], c8), sad9[2], sad9[3]);
            blk_sum2(sad8(nb9[5], c8), sad8(nb9[6], c8), sad9[5], sad9[6]);
            blk_sum2(sad8(nb9[7], c8), sad8(nb9[8], c8), sad9[7], sad9[8]);
#pragma unroll
            for (int n = 0; n < 9; ++n) {
                if (n == 4) continue;  // 3x3 raster without its centre
                const int ex = clampi(cx + n % 3 - 1, V.lox, V.hix), ey = clampi(cy + n / 3 - 1, V.loy, V.hiy);
                const unsigned ce = sad9[n];
                if (need_nb && (ex != cx || ey != cy)) {
                    if (first) blog[s.nlog] = pack_mv(ex, ey);
                    ++s.nlog;
                    if (ce < bc) {
                        bc = ce;
                        bx = ex;
                        by = ey;
                        b8 = nb9[n];
                    }
                }
            }
            if (need_nb) {
                if (bc < s.cost) {
                    s.dx = bx;
                    s.dy = by;
                    s.cost = bc;
                    s.r8 = b8;
                } else {
                    s.done = true;
                }
            }
        }
    }
}

// Alpha mismatches of the lane's quadrant at the full-pel part of key (the
// boundary cost of one block), from the staged BABs as in shape_costs_smem.
__device__ __forceinline__ unsigned shape_quadrant_smem(const uint32_t* acur, const uint32_t* aref, int arw, int S,
                                                        int X0, int key, int h, int lane)
{
    const int r = lane & 15;
    const unsigned cb = (acur[r * kAcurWords + (X0 >> 5) - ((X0 >> 5) & ~3)] >> (X0 & 31)) & 0xffffu;
    const int xw0 = ((X0 - S) >> 5) & ~3;
    const int fdx = mv_x(key) / h, fdy = mv_y(key) / h;  // trunc toward zero
    const int xr = X0 + fdx, wr = (xr >> 5) - xw0;
    const uint32_t* row = aref + (r + fdy + S) * arw;
    const unsigned diff = (cb ^ __funnelshift_r(row[wr], row[wr + 1], xr & 31)) & 0xffffu;
    unsigned lo = __popc(diff & 0xffu), hi = __popc(diff >> 8);
    // sums over rows 0-7 (lanes 0-7) and 8-15 (lanes 8-15)
#pragma unroll
    for (int o = 1; o <= 4; o <<= 1) {
        lo += __shfl_xor_sync(kFull, lo, o);
        hi += __shfl_xor_sync(kFull, hi, o);
    }
    const int src = (lane >> 4) << 3;  // lane 0: rows 0-7, lane 8: rows 8-15
    const unsigned qlo = __shfl_sync(kFull, lo, src), qhi = __shfl_sync(kFull, hi, src);
    return (lane & 1) ? qhi : qlo;
}

// Distinct positions of the lane's block: its log (the MB candidates, then
// its own PRS positions), counted by the block's 8 lanes.
__device__ __forceinline__ unsigned blk_distinct(const int* blog, int n, int lane)
{
    unsigned first = 0;
    for (int e = (lane >> 1) & 7; e < n; e += 8) {
        const int kk = blog[e];
        bool f = true;
        for (int j = 0; j < e; ++j)
            if (blog[j] == kk) {
                f = false;
                break;
            }
        first += f;
    }
    return blk_sum(first);
}

// Outputs of one MB in the four-vector mode ([M][4] arrays): the lane's block
// state s, the MB's SSE from every lane's 8 pixels at its block's vector.
__device__ __forceinline__ void finish_mb4(const SeqDesc* sd, int idx, int k, int cls, const Blk4& s, const P8& c8,
                                           const int* blog, int lane, size_t FS, int W, int y, int x0)
{
    __syncwarp();
    const unsigned npos = blk_distinct(blog, s.nlog, lane);
    if ((lane & 14) == 0) {
        const int o = 4 * idx + blk_of(lane);
        sd->mv[o] = sme_mv{(int16_t)s.dx, (int16_t)s.dy};
        if (sd->cost) sd->cost[o] = s.cost;
        if (sd->iters) sd->iters[o] = (uint8_t)s.iters;
        if (sd->npos) sd->npos[o] = (uint8_t)npos;
        if (sd->disp) {
            sd->disp[2 * o] = s.lastx;
            sd->disp[2 * o + 1] = s.lasty;
        }
    }
    if (lane == 0 && sd->out_cls) sd->out_cls[idx] = (uint8_t)cls;
    const unsigned e = __reduce_add_sync(kFull, sq8(s.r8, c8));
    if (lane == 0) {
        if (sd->sse) atomicAdd(sd->sse + k, (unsigned long long)e);
        if (sd->sse_mb) sd->sse_mb[idx] = e;
    }
    if (sd->pred)
        *reinterpret_cast<uint2*>(sd->pred + (size_t)k * FS + (size_t)y * W + x0) = make_uint2(s.r8.lo, s.r8.hi);
    __syncwarp();
}

__device__ __forceinline__ Blk4 opaque_blocks4(const Method& m, const uint8_t* win, int pitch, int lx, int ly,
                                               const P8& c8, const float (&ux)[8], const float (&uy)[8],
                                               const VRange& V, const int (&cand)[5], int* blog, int lane);

// The four block searches of an opaque MB from the MB winner `key` (r8: the
// lane's reference samples there).
__device__ __forceinline__ Blk4 blocks_from_winner(const Method& m, const uint8_t* win, int pitch, int lx, int ly,
                                                   const P8& c8, const float (&ux)[8], const float (&uy)[8],
                                                   const VRange& V, int key, const P8& r8, int* blog, int lane)
{
    Blk4 s;
    s.iters = 0;
    s.nlog = 4;
    s.lastx = s.lasty = 0.0f;
    s.done = false;
    s.dx = mv_x(key);
    s.dy = mv_y(key);
    s.r8 = r8;
    s.cost = blk_sum(sad8(r8, c8));
    unsigned cx = 0, cy = 0;
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        cx += ux[k] != 0.0f;
        cy += uy[k] != 0.0f;
    }
    prs_blocks(m, win, pitch, lx, ly, c8, ux, uy, (int)blk_sum(cx), (int)blk_sum(cy), V, s, blog, lane);
    return s;
}

// Fig. 1 at MB level (16x16 costs of the candidates A, B, C, T) and, on
// opaque MBs, the block searches from the winner.  The candidates are in
// cand[0..4); each block log starts with them.
__device__ __forceinline__ Blk4 search_mb4(const Method& m, int cls, const uint8_t* win, int pitch, int lx, int ly,
                                           const P8& c8, const float (&ux)[8], const float (&uy)[8],
                                           const VRange& V, const int (&cand)[5], const uint32_t* acur,
                                           const uint32_t* aref, int arw, int S, int X0, int* blog, int lane)
{
    const int h = m.h;
    Blk4 s;
    s.iters = 0;
    s.nlog = 4;
    s.lastx = s.lasty = 0.0f;
    s.done = false;
    if (cls == SME_BOUNDARY) {
        unsigned sc[5];
        shape_costs_smem(acur, aref, arw, S, X0, cand, 4, h, lane, sc);
        int best = cand[0];
        unsigned cost = sc[0];
#pragma unroll
        for (int c = 1; c < 4; ++c)
            if (sc[c] < cost) {
                cost = sc[c];
                best = cand[c];
            }
        s.dx = mv_x(best);
        s.dy = mv_y(best);
        s.cost = shape_quadrant_smem(acur, aref, arw, S, X0, best, h, lane);
        s.r8 = ref8(win, pitch, lx, ly, s.dx, s.dy, h);
        return s;
    }
    return opaque_blocks4(m, win, pitch, lx, ly, c8, ux, uy, V, cand, blog, lane);
}

// Opaque MB in the four-vector mode: 16x16 texture SADs of the candidates A,
// B, C, T, first strict minimum, then the four block searches from it.
__device__ __forceinline__ Blk4 opaque_blocks4(const Method& m, const uint8_t* win, int pitch, int lx, int ly,
                                               const P8& c8, const float (&ux)[8], const float (&uy)[8],
                                               const VRange& V, const int (&cand)[5], int* blog, int lane)
{
    const int h = m.h;
    Blk4 s;
    s.iters = 0;
    s.nlog = 4;
    s.lastx = s.lasty = 0.0f;
    s.done = false;
    P8 cs8[4];
    unsigned part[4];
#pragma unroll
    for (int c = 0; c < 4; ++c) {
        cs8[c] = ref8(win, pitch, lx, ly, mv_x(cand[c]), mv_y(cand[c]), h);
        part[c] = sad8(cs8[c], c8);
    }
    unsigned sad[4];
    warp_sum2(part[0], part[1], sad[0], sad[1]);
    warp_sum2(part[2], part[3], sad[2], sad[3]);
    int best = 0;
    unsigned cost = sad[0];
#pragma unroll
    for (int c = 1; c < 4; ++c)
        if (sad[c] < cost) {
            cost = sad[c];
            best = c;
        }
    P8 r8 = cs8[0];
    int key = cand[0];
#pragma unroll
    for (int c = 1; c < 4; ++c)
        if (c == best) {
            r8 = cs8[c];
            key = cand[c];
        }
    return blocks_from_winner(m, win, pitch, lx, ly, c8, ux, uy, V, key, r8, blog, lane);
}

// ============================== ME, per-MB warps, four vectors per MB ==
// The per-MB schedule of me_kernel with the four-vector mode (Sec. 3.2, 8x8
// blocks; reading of the candidate layout as in the pair kernel).  A consumer
// needs a different block of its producer by role, so every MB publishes
// three ready words, each (epoch << 32) | vector: block 0 (for T), block 1
// (for A), block 2 (for B and C).
struct Links4 {
    unsigned long long* rt;
    unsigned long long* ra;
    unsigned long long* rbc;
    unsigned epoch;
    int fault;
    __device__ __forceinline__ void publish(int gid, int k0, int k1, int k2, int lane) const
    {
        if (lane == 0 && gid != fault) {
            const unsigned long long t = (unsigned long long)epoch << 32;
            st_ready(rt + gid, t | (unsigned)k0);
            st_ready(ra + gid, t | (unsigned)k1);
            st_ready(rbc + gid, t | (unsigned)k2);
        }
    }
};

__host__ __device__ __forceinline__ int warp_smem4(int S) { return win_bytes(S) + ceil16(4 * kMaxLog * 4); }

// Alpha mismatches of the lane's quadrant at the full-pel part of key, from
// the packed alpha in global memory (as shape_row).
__device__ __forceinline__ unsigned shape_quadrant_g(const uint32_t* pcur, const uint32_t* pref, int Wp, int X0,
                                                     int Y0, int key, int h, int lane)
{
    const int r = lane & 15, fdx = mv_x(key) / h, fdy = mv_y(key) / h;  // trunc toward zero
    const uint32_t* rc = pcur + (size_t)(Y0 + r) * Wp;
    const unsigned cb = (__ldg(rc + (X0 >> 5)) >> (X0 & 31)) & 0xffffu;
    const int xr = X0 + fdx;
    const uint32_t* rr = pref + (size_t)(Y0 + r + fdy) * Wp;
    const unsigned diff = (cb ^ __funnelshift_r(__ldg(rr + (xr >> 5)), __ldg(rr + (xr >> 5) + 1), xr & 31)) & 0xffffu;
    unsigned lo = __popc(diff & 0xffu), hi = __popc(diff >> 8);
#pragma unroll
    for (int o = 1; o <= 4; o <<= 1) {
        lo += __shfl_xor_sync(kFull, lo, o);
        hi += __shfl_xor_sync(kFull, hi, o);
    }
    const int src = (lane >> 4) << 3;
    const unsigned qlo = __shfl_sync(kFull, lo, src), qhi = __shfl_sync(kFull, hi, src);
    return (lane & 1) ? qhi : qlo;
}

__device__ __forceinline__ bool me_one_mb4(const MeArgs& a, const Method& m, int gid, const SeqDesc* sd,
                                           uint8_t* win, int* slog, const float* s_rcp, const Links4& L, int lane,
                                           int pitch)
{
    const int h = m.h;
    const int W = sd->W, H = sd->H, M = sd->M, MBW = sd->MBW, rd = sd->rd;
    const int idx = gid - sd->gid_base;
    const int k = idx / M, mb = idx - k * M;
    const int u = mb % MBW, v = mb / MBW;
    const int X0 = 16 * u, Y0 = 16 * v;
    const int x0 = X0 + 8 * (lane & 1), y = Y0 + (lane >> 1);
    const size_t FS = (size_t)W * H;
    const uint8_t* ref = sd->luma + (size_t)k * FS;
    const uint8_t* cur = sd->luma + (size_t)(k + rd) * FS;
    const int cls = __ldg(sd->cls + (size_t)(k + rd) * M + mb);
    const P8 c8 = load8(cur + (size_t)y * W + x0);

    if (cls == SME_TRANSPARENT) {
        L.publish(gid, 0, 0, 0, lane);
        Blk4 s4;
        s4.dx = s4.dy = s4.iters = s4.nlog = 0;
        s4.cost = 0;
        s4.lastx = s4.lasty = 0.0f;
        s4.done = true;
        s4.r8 = load8(ref + (size_t)y * W + x0);
        finish_mb4(sd, idx, k, cls, s4, c8, slog, lane, FS, W, y, x0);
        return true;
    }

    int wx0, wy0;
    stage_window(win, ref, W, H, m.S, X0, Y0, lane, wx0, wy0);
    float ux[8], uy[8];
    int nx = 0, ny = 0;
    if (cls == SME_OPAQUE) mb_factors(grad_loads(cur, W, H, x0, y), W, H, x0, y, c8, m.theta, s_rcp, ux, uy, nx, ny);
    const VRange V = valid_range(W, H, m, X0, Y0);
    const int lx = x0 - wx0, ly = y - wy0;

    // ---- candidates: A = block 1 of the left MB, B / C = block 2 of the MBs
    // above / above-right, T = block 0 of the previous pair (reading c22) ----
    int dep = -1;
    const unsigned long long* src = L.rt;
    if (lane == 0 && u > 0) { dep = gid - 1; src = L.ra; }
    if (lane == 1 && v > 0) { dep = gid - MBW; src = L.rbc; }
    if (lane == 2 && v > 0 && u < MBW - 1) { dep = gid - MBW + 1; src = L.rbc; }
    if (lane == 3 && k > 0) dep = gid - M;
    int key = 0;
    if (lane == 3 && k == 0 && sd->temporal_in)
        key = (int)__ldg(reinterpret_cast<const unsigned*>(sd->temporal_in + 4 * mb));
    if (lane < 4) key = pack_mv(clampi(mv_x(key), V.lox, V.hix), clampi(mv_y(key), V.loy, V.hiy));
    bool res = dep < 0;
    const uint32_t* pcur = sd->packed + (size_t)(k + rd) * H * sd->Wp;
    const uint32_t* pref = sd->packed + (size_t)k * H * sd->Wp;
    // Every candidate is costed (16x16 shape or texture) as soon as its
    // vector arrives, so after the last arrival only its own cost is left.
    unsigned costed = 0;
    unsigned ccost[4] = {0u, 0u, 0u, 0u};
    int ckey[4] = {0, 0, 0, 0};
    P8 cs8[4];
#pragma unroll
    for (int c = 0; c < 4; ++c) cs8[c] = c8;
    unsigned long long t_start = 0;
    for (unsigned it = 0;; ++it) {
        unsigned long long w = 0;
        if (lane < 4 && !res) w = ld_ready(src + dep);  // issued first: its latency overlaps the costing
        const unsigned fresh = __ballot_sync(kFull, lane < 4 && res) & 0xfu & ~costed;
#pragma unroll
        for (int c = 0; c < 4; ++c)
            if (fresh & (1u << c)) {
                const int kc = __shfl_sync(kFull, key, c);
                ckey[c] = kc;
                bool dup = false;
#pragma unroll
                for (int e = 0; e < 4; ++e)
                    if (e != c && !dup && (costed & (1u << e)) && ckey[e] == kc) {
                        ccost[c] = ccost[e];
                        cs8[c] = cs8[e];
                        dup = true;
                    }
                if (!dup) {
                    if (cls == SME_BOUNDARY) {
                        ccost[c] = shape_cost1(pcur, pref, sd->Wp, X0, Y0, kc, h, lane);
                    } else {
                        cs8[c] = ref8(win, pitch, lx, ly, mv_x(kc), mv_y(kc), h);
                        ccost[c] = __reduce_add_sync(kFull, sad8(cs8[c], c8));
                    }
                }
                costed |= 1u << c;
            }
        if (costed == 0xfu) break;
        if (lane < 4 && !res && (unsigned)(w >> 32) == L.epoch) {
            const int kk = (int)(unsigned)w;
            key = pack_mv(clampi(mv_x(kk), V.lox, V.hix), clampi(mv_y(kk), V.loy, V.hiy));
            res = true;
        }
        if ((it & 15u) == 15u) {
            // Bounded wait: the launch's abort word, a time limit, an iteration cap.
            int give_up = 0;
            if (lane == 0) {
                const unsigned long long now = globaltimer();
                if (t_start == 0) t_start = now;
                give_up = ld_relaxed(&a.status->abort) || (long long)(now - t_start) > a.timeout_ns ||
                          it > (1u << 24);
            }
            if (__shfl_sync(kFull, give_up, 0)) {
                if (lane == 0 && !ld_relaxed(&a.status->abort)) raise_error(a.status, SME_ERR_TIMEOUT, true);
                return false;
            }
        }
    }
    if (lane < 16) slog[(lane >> 2) * kMaxLog + (lane & 3)] = ckey[lane & 3];
    __syncwarp();
    int* blog = slog + blk_of(lane) * kMaxLog;
    // first strict minimum in the order A, B, C, T
    int bi = 0;
#pragma unroll
    for (int c = 1; c < 4; ++c)
        if (ccost[c] < ccost[bi]) bi = c;
    int bk = ckey[0];
    P8 br8 = cs8[0];
#pragma unroll
    for (int c = 1; c < 4; ++c)
        if (c == bi) {
            bk = ckey[c];
            br8 = cs8[c];
        }
    Blk4 s4;
    if (cls == SME_BOUNDARY) {
        s4.dx = mv_x(bk);
        s4.dy = mv_y(bk);
        s4.iters = 0;
        s4.nlog = 4;
        s4.lastx = s4.lasty = 0.0f;
        s4.done = true;
        s4.cost = shape_quadrant_g(pcur, pref, sd->Wp, X0, Y0, bk, h, lane);
        s4.r8 = ref8(win, pitch, lx, ly, s4.dx, s4.dy, h);
    } else {
        s4 = blocks_from_winner(m, win, pitch, lx, ly, c8, ux, uy, V, bk, br8, blog, lane);
    }
    const int kb = pack_mv(s4.dx, s4.dy);
    L.publish(gid, __shfl_sync(kFull, kb, 0), __shfl_sync(kFull, kb, 1), __shfl_sync(kFull, kb, 16), lane);
    finish_mb4(sd, idx, k, cls, s4, c8, blog, lane, FS, W, y, x0);
    return true;
}

__global__ void __launch_bounds__(32 * kMeWarps) me4_kernel(const MeArgs a)
{
    extern __shared__ __align__(16) uint8_t smem[];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const Method m = a.m;
    const int pitch = win_pitch(m.S);
    uint8_t* win = smem + (size_t)wid * warp_smem4(m.S);
    int* slog = reinterpret_cast<int*>(win + win_bytes(m.S));
    const Links4 L{a.ready, a.ready_a, a.ready_bc, ld_relaxed(&a.status->epoch), a.fault_ticket};
    __shared__ float s_rcp[512];
    fill_rcp(s_rcp);
    __syncthreads();
    for (;;) {
        int t = 0;
        if (lane == 0) {
            t = (int)atomicAdd(&a.status->ticket, 1u);
            if (ld_relaxed(&a.status->abort)) t = a.total;
        }
        t = __shfl_sync(kFull, t, 0);
        if (t >= a.total) break;
        const int gid = __ldg(a.sched + t);
        const SeqDesc* sd = a.seqs + (a.sched_seq ? __ldg(a.sched_seq + t) : 0);
        if (!me_one_mb4(a, m, gid, sd, win, slog, s_rcp, L, lane, pitch)) break;
    }
}


// kDirect: runs of transparent MBs (known from the classification launch)
// are finished by transparent_run and only the other MBs are staged by TMA;
// otherwise every MB is staged and classified from its staged BAB.  Two
// instantiations rather than a runtime switch, so that each keeps only its
// own code.  The direct one is bounded at 8 warps per CTA, which lets it keep
// its state in registers (at 16 warps it spilled and ran 18 % slower on
// 3840x2160 VOPs).  kFourMv: four vectors per
// MB (Sec. 3.2, 8x8 blocks; staged only): A is block 1 of the left MB (the
// warp's previous MB), B and C block 2 of the MBs above (the row slots hold
// block 2), T block 0 of the previous pair (the ready words hold block 0).
template <bool kDirect, bool kFourMv>
__global__ void __launch_bounds__(32 * (kDirect ? 8 : kPairWarpsMax)) me_pair_kernel(const MeArgs a, const __grid_constant__ PairMaps maps0)
{
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = reinterpret_cast<uint8_t*>(((uintptr_t)smem_raw + 127) & ~(uintptr_t)127);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const Method m = a.m;
    const int h = m.h, S = m.S, cs = ceil16(S), pitch = win_pitch(S), arw = aref_words(S);
    const unsigned tx = pair_tx_bytes(S);
    const PairLayout L = pair_layout(S, nw, a.mbw_max, kFourMv);
    uint8_t* wbase = smem + (size_t)wid * L.warp_bytes;
    int* slog = reinterpret_cast<int*>(wbase + L.log_off);
    uint64_t* bars = reinterpret_cast<uint64_t*>(wbase + L.bar_off);
    uint8_t* s_rowcls = wbase + L.cls_off;
    int* rowmv = reinterpret_cast<int*>(smem + L.rows_off);
    int* prog = reinterpret_cast<int*>(smem + L.prog_off);
    int* s_unit = reinterpret_cast<int*>(smem + L.unit_off);
    const unsigned epoch = ld_relaxed(&a.status->epoch);
    const unsigned long long tag = (unsigned long long)epoch << 32;
    const int lx = cs + 8 * (lane & 1), ly = S + (lane >> 1);  // lane's first pixel in the window

    __shared__ float s_rcp[512];
    fill_rcp(s_rcp);
    if (lane == 0) {
        mbar_init(&bars[0]);
        mbar_init(&bars[1]);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    unsigned parity = 0;   // bit b: parity of the next completion of buffer b
    unsigned pending = 0;  // bit b: copies into buffer b are in flight
    int cur = 0;           // buffer of the MB being processed
    bool failed = false;

    for (;;) {
        if (threadIdx.x == 0) {
            int t = (int)atomicAdd(&a.status->ticket, 1u);
            if (ld_relaxed(&a.status->abort)) t = a.total_units;
            *s_unit = t;
        }
        for (int i = threadIdx.x; i < L.R; i += blockDim.x) prog[i] = -1;
        __syncthreads();
        const int unit = *s_unit;
        if (unit >= a.total_units) break;  // uniform: a failure raised the abort word
        const int sid = a.unit_seq ? __ldg(a.unit_seq + unit) : 0;
        const int k = a.unit_pair ? __ldg(a.unit_pair + unit) : unit;
        const SeqDesc* sd = a.seqs + sid;
        const PairMaps* mp = a.tmaps ? reinterpret_cast<const PairMaps*>(a.tmaps) + sid : &maps0;
        const int W = sd->W, H = sd->H, M = sd->M, MBW = sd->MBW, MBH = sd->MBH, rd = sd->rd;
        const size_t FS = (size_t)W * H;
        const int base = sd->gid_base + k * M;

        for (int v = wid; v < MBH && !failed; v += nw) {
            const int slot = v % L.R, pslot = (v + L.R - 1) % L.R;
            const int Y0 = 16 * v, y = Y0 + (lane >> 1);
            if constexpr (kDirect) {
                // the row's MB classes (Fig. 1 Block_Type, from the classification launch)
                const uint8_t* rowcls = sd->cls + (size_t)(k + rd) * M + (size_t)v * MBW;
                for (int i = lane; i < MBW; i += 32) s_rowcls[i] = __ldg(rowcls + i);
            }
            // Row slots are reused every R = nw + 1 rows.  Row v - R + 1, the one
            // that reads slot v % R last, is this warp's previous row; waiting
            // here until row v - R has filled the slot makes sure that the slot
            // holds no older row, whose reader could still be running: a warp
            // with transparent rows publishes without waiting for the row above
            // and could otherwise run more than R rows ahead.
            if (v >= L.R) {
                bool ok = true;
                if (lane == 0) ok = wait_progress(&prog[slot], (v - L.R) * 1024 + MBW, a.status, a.timeout_ns);
                if (!__shfl_sync(kFull, ok, 0)) {
                    if (lane == 0 && !ld_relaxed(&a.status->abort)) raise_error(a.status, SME_ERR_TIMEOUT, true);
                    failed = true;
                    break;
                }
            }
            __syncwarp();
            int akey = 0;  // A: this row's previous vector
            // The boxes of the next staged MB are always in flight while the
            // current one (or a transparent run before it) is processed.
            int nt = 0;
            if constexpr (kDirect) nt = next_visible(s_rowcls, 0, MBW, lane);
            unsigned long long tnext = 0;
            if (nt < MBW) {
                if (lane == 0) issue_mb_boxes(wbase + cur * L.buf_bytes, L, mp, S, 16 * nt, Y0, k, k + rd, &bars[cur], tx);
                pending |= 1u << cur;
                if (lane == 3 && k > 0) tnext = ld_ready(a.ready + base + v * MBW + nt - M);
            }
            for (int u = 0; u < MBW && !failed;) {
                if constexpr (kDirect) {
                    if (u < nt) {
                        transparent_run(sd, a, k, v, u, nt, base, slot, rowmv, prog, tag, lane);
                        akey = 0;
                        u = nt;
                        continue;
                    }
                }
                const int mb = v * MBW + u, idx = k * M + mb, gid = base + mb;
                const int X0 = 16 * u, x0 = X0 + 8 * (lane & 1);
                int nn = u + 1;
                if constexpr (kDirect) nn = next_visible(s_rowcls, u + 1, MBW, lane);
                const int nb = cur ^ 1;
                if (nn < MBW) {
                    if (lane == 0)
                        issue_mb_boxes(wbase + nb * L.buf_bytes, L, mp, S, 16 * nn, Y0, k, k + rd, &bars[nb], tx);
                    pending |= 1u << nb;
                }
                const unsigned long long tcur = tnext;
                if (lane == 3 && k > 0 && nn < MBW) tnext = ld_ready(a.ready + base + v * MBW + nn - M);

                bool ok = true;
                if (lane == 0) ok = mbar_wait(&bars[cur], (parity >> cur) & 1u, a.timeout_ns);
                ok = __shfl_sync(kFull, ok, 0);
                if (!ok) {
                    // the copies of `cur` stay pending: the drain below waits for them too
                    if (lane == 0) raise_error(a.status, SME_ERR_TIMEOUT, true);
                    failed = true;
                    break;
                }
                parity ^= 1u << cur;
                pending &= ~(1u << cur);
                const uint8_t* buf = wbase + cur * L.buf_bytes;
                const uint8_t* win = buf + L.o_ref;
                const uint32_t* acur = reinterpret_cast<const uint32_t*>(buf + L.o_acur);
                int cls;
                if constexpr (kDirect) {
                    cls = s_rowcls[u];  // boundary or opaque
                } else {
                    // Fig. 1 Block_Type from the staged current BAB (16 rows of 16 bits).
                    unsigned ones = 0;
                    if (lane < 16)
                        ones = __popc((acur[lane * kAcurWords + (X0 >> 5) - ((X0 >> 5) & ~3)] >> (X0 & 31)) & 0xffffu);
                    ones = __reduce_add_sync(kFull, ones);
                    cls = ones == 0 ? SME_TRANSPARENT : (ones == 256 ? SME_OPAQUE : SME_BOUNDARY);
                }
                P8 c8;
                {
                    const uint2 t2 = *reinterpret_cast<const uint2*>(buf + L.o_cur + (1 + (lane >> 1)) * kCurBoxW + 16 +
                                                                     8 * (lane & 1));
                    c8.lo = t2.x;
                    c8.hi = t2.y;
                }

                if (!kDirect && cls == SME_TRANSPARENT) {
                    // Fig. 1: (0,0) is final at once.
                    if (lane == 0) {
                        rowmv[slot * a.mbw_max + u] = 0;
                        st_release_cta(&prog[slot], v * 1024 + u + 1);
                        if (gid != a.fault_ticket) st_ready(a.ready + gid, tag);
                        if (!kFourMv) sd->mv[idx] = sme_mv{0, 0};
                    }
                    akey = 0;
                    if constexpr (kFourMv) {
                        Blk4 s4;
                        s4.dx = s4.dy = s4.iters = s4.nlog = 0;
                        s4.cost = 0;
                        s4.lastx = s4.lasty = 0.0f;
                        s4.done = true;
                        s4.r8 = ref8(win, pitch, lx, ly, 0, 0, h);
                        finish_mb4(sd, idx, k, cls, s4, c8, slog, lane, FS, W, y, x0);
                        cur = nb;
                        nt = nn;
                        ++u;
                        continue;
                    }
                    MbResult r;
                    r.dx = r.dy = r.iters = r.nlog = 0;
                    r.cost = 0;
                    r.lastx = r.lasty = 0.0f;
                    r.r8 = ref8(win, pitch, lx, ly, 0, 0, h);
                    finish_mb(sd, idx, k, cls, r, c8, slog, lane, FS, W, y, x0);
                } else {
                    float ux[8], uy[8];
                    int nx = 0, ny = 0;
                    if (cls == SME_OPAQUE)
                        factors_smem(buf + L.o_cur, W, H, x0, y, c8, m.theta, s_rcp, ux, uy, nx, ny, lane);
                    const VRange V = valid_range(W, H, m, X0, Y0);
                    // ---- candidates A, B, C, T (Fig. 1, Fig. 3) + optional seed ----
                    if (v > 0 && lane == 0)
                        ok = wait_progress(&prog[pslot], (v - 1) * 1024 + min(u + 2, MBW), a.status, a.timeout_ns);
                    int key = 0;
                    if (lane == 3) {
                        if (k > 0) {
                            unsigned val = (unsigned)tcur;
                            if ((unsigned)(tcur >> 32) != epoch)
                                ok = wait_ready(a.ready + gid - M, epoch, a.status, a.timeout_ns, val);
                            key = (int)val;
                        } else if (sd->temporal_in) {
                            key = (int)__ldg(reinterpret_cast<const unsigned*>(sd->temporal_in + (kFourMv ? 4 * mb : mb)));
                        }
                    }
                    if (__any_sync(kFull, !ok)) {
                        if (lane == 0 && !ld_relaxed(&a.status->abort)) raise_error(a.status, SME_ERR_TIMEOUT, true);
                        failed = true;
                        break;
                    }
                    __syncwarp();  // lane 0's acquire of the row above orders the reads below
                    if (lane == 0) key = akey;
                    if (lane == 1 && v > 0) key = rowmv[pslot * a.mbw_max + u];
                    if (lane == 2 && v > 0 && u + 1 < MBW) key = rowmv[pslot * a.mbw_max + u + 1];
                    if (lane < 4) key = pack_mv(clampi(mv_x(key), V.lox, V.hix), clampi(mv_y(key), V.loy, V.hiy));
                    if (!kFourMv && lane == 4 && sd->seed) key = seed_key(sd, idx, h, V);
                    const int nc = (!kFourMv && sd->seed) ? 5 : 4;
                    int cand[5];
#pragma unroll
                    for (int c = 0; c < 5; ++c) cand[c] = __shfl_sync(kFull, key, c);
                    if constexpr (kFourMv) {
                        // every block's log starts with the MB candidates
                        if (lane < 16) slog[(lane >> 2) * kMaxLog + (lane & 3)] = cand[lane & 3];
                        __syncwarp();
                        int* blog = slog + blk_of(lane) * kMaxLog;
                        const Blk4 s4 = search_mb4(m, cls, win, pitch, lx, ly, c8, ux, uy, V, cand, acur,
                                                   reinterpret_cast<const uint32_t*>(buf + L.o_aref), arw, S, X0, blog,
                                                   lane);
                        const int kb = pack_mv(s4.dx, s4.dy);
                        const int k0 = __shfl_sync(kFull, kb, 0), k1 = __shfl_sync(kFull, kb, 1);
                        const int k2 = __shfl_sync(kFull, kb, 16);
                        if (lane == 0) {
                            rowmv[slot * a.mbw_max + u] = k2;
                            st_release_cta(&prog[slot], v * 1024 + u + 1);
                            if (gid != a.fault_ticket) st_ready(a.ready + gid, tag | (unsigned)k0);
                        }
                        akey = k1;
                        finish_mb4(sd, idx, k, cls, s4, c8, blog, lane, FS, W, y, x0);
                        cur = nb;
                        nt = nn;
                        ++u;
                        continue;
                    }
                    if (lane < nc) slog[lane] = key;
                    MbResult r;
                    if (cls == SME_BOUNDARY) {
                        unsigned sc[5];
                        shape_costs_smem(acur, reinterpret_cast<const uint32_t*>(buf + L.o_aref), arw, S, X0, cand, nc,
                                         h, lane, sc);
                        int bi = 0;
                        unsigned cost = sc[0];
#pragma unroll
                        for (int c = 1; c < 5; ++c)
                            if (c < nc && sc[c] < cost) {
                                cost = sc[c];
                                bi = c;
                            }
                        if (m.tt) boundary_t_by_texture(win, pitch, lx, ly, c8, cand, sc, nc, h, bi, cost);
                        int best = cand[0];
#pragma unroll
                        for (int c = 1; c < 5; ++c)
                            if (c == bi) best = cand[c];
                        r.dx = mv_x(best);
                        r.dy = mv_y(best);
                        r.cost = cost;
                        r.iters = 0;
                        r.nlog = nc;
                        r.lastx = r.lasty = 0.0f;
                        r.r8 = ref8(win, pitch, lx, ly, r.dx, r.dy, h);
                    } else {
                        r = search_mb(m, cls, win, pitch, lx, ly, c8, ux, uy, nx, ny, V, cand, nc, nullptr, nullptr, 0,
                                      X0, Y0, slog, lane);
                    }
                    // ---- publish: row slot for the row below, ready word for the next pair ----
                    const int key_out = pack_mv(r.dx, r.dy);
                    if (lane == 0) {
                        rowmv[slot * a.mbw_max + u] = key_out;
                        st_release_cta(&prog[slot], v * 1024 + u + 1);
                        if (gid != a.fault_ticket) st_ready(a.ready + gid, tag | (unsigned)key_out);
                        sd->mv[idx] = sme_mv{(int16_t)r.dx, (int16_t)r.dy};
                    }
                    akey = key_out;
                    finish_mb(sd, idx, k, cls, r, c8, slog, lane, FS, W, y, x0);
                }
                cur = nb;
                nt = nn;
                ++u;
            }
            // A failing warp drains its own copies in flight -- including the
            // one whose wait gave up -- before the CTA moves on.  Each drain is
            // bounded too: a copy still outstanding after a second full wait
            // limit (a TMA stall of seconds) is the one case this path cannot
            // cover; the launch has then already reported SME_ERR_TIMEOUT.
            if (failed) {
                for (int b = 0; b < 2; ++b)
                    if (pending & (1u << b)) {
                        if (lane == 0) mbar_wait(&bars[b], (parity >> b) & 1u, a.timeout_ns);
                        __syncwarp();
                        parity ^= 1u << b;
                    }
                pending = 0;
            }
        }
        __syncthreads();
    }
}

// ========================================================== compensate ==
__global__ void __launch_bounds__(256) compensate_kernel(const Geom g, const Method mth, const CompArgs a)
{
    __shared__ unsigned s_red[8];
    const int mb = blockIdx.x, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int u = mb % g.MBW, v = mb / g.MBW, X0 = 16 * u, Y0 = 16 * v;
    const int x = X0 + (tid & 15), y = Y0 + (tid >> 4);
    const unsigned raw = __ldg(reinterpret_cast<const unsigned*>(a.mv + mb));
    const int dx = mv_x((int)raw), dy = mv_y((int)raw);
    const VRange V = valid_range(g.W, g.H, mth, X0, Y0);
    if (dx < V.lox || dx > V.hix || dy < V.loy || dy > V.hiy) {
        if (tid == 0) raise_error(a.status, SME_ERR_RANGE, false);
        return;
    }
    // One pixel per thread, read straight from global memory.
    int ix = dx, iy = dy, fx = 0, fy = 0;
    if (mth.h == 2) {
        ix = dx >> 1;
        iy = dy >> 1;
        fx = dx & 1;
        fy = dy & 1;
    }
    const uint8_t* r = a.ref + (size_t)(y + iy) * g.W + (x + ix);
    int p = __ldg(r);
    if (fx && fy) p = (p + __ldg(r + 1) + __ldg(r + g.W) + __ldg(r + g.W + 1) + 2) >> 2;
    else if (fx) p = (p + __ldg(r + 1) + 1) >> 1;
    else if (fy) p = (p + __ldg(r + g.W) + 1) >> 1;
    const int e = (int)__ldg(a.cur + (size_t)y * g.W + x) - p;
    if (a.pred) a.pred[(size_t)y * g.W + x] = (uint8_t)p;
    const unsigned s = __reduce_add_sync(kFull, (unsigned)(e * e));
    if (lane == 0) s_red[warp] = s;
    __syncthreads();
    if (tid == 0) {
        unsigned long long tot = 0;
        for (int w = 0; w < 8; ++w) tot += s_red[w];
        atomicAdd(a.sse, tot);
    }
}

// ============================================================= queries ==
// One warp per (MB, d) query, through the ME kernel's device functions.
constexpr int kQueryWarps = 4;

__global__ void __launch_bounds__(32 * kQueryWarps) query_kernel(const Geom g, const Method m, const QueryArgs a)
{
    extern __shared__ __align__(16) uint8_t smem[];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int qi = blockIdx.x * kQueryWarps + wid;
    __shared__ float s_rcp[512];
    fill_rcp(s_rcp);
    __syncthreads();
    if (qi >= a.n) return;
    uint8_t* win = smem + (size_t)wid * warp_smem(m.S);
    const int mb = __ldg(a.q + 3 * qi), dx = __ldg(a.q + 3 * qi + 1), dy = __ldg(a.q + 3 * qi + 2);
    if (mb < 0 || mb >= g.M) {
        if (lane == 0) raise_error(a.status, SME_ERR_ARG, false);
        return;
    }
    const int u = mb % g.MBW, v = mb / g.MBW, X0 = 16 * u, Y0 = 16 * v;
    const VRange V = valid_range(g.W, g.H, m, X0, Y0);
    if (dx < V.lox || dx > V.hix || dy < V.loy || dy > V.hiy) {
        if (lane == 0) raise_error(a.status, SME_ERR_RANGE, false);
        return;
    }
    const int x0 = X0 + 8 * (lane & 1), y = Y0 + (lane >> 1);
    int wx0, wy0;
    stage_window(win, a.ref, g.W, g.H, m.S, X0, Y0, lane, wx0, wy0);
    P8 c8;
    const uint2 t2 = __ldg(reinterpret_cast<const uint2*>(a.cur + (size_t)y * g.W + x0));
    c8.lo = t2.x;
    c8.hi = t2.y;
    const P8 r8 = ref8(win, win_pitch(m.S), x0 - wx0, y - wy0, dx, dy, m.h);
    const unsigned sad = __reduce_add_sync(kFull, sad8(r8, c8));
    float ux[8], uy[8];
    grad_factors8(grad_loads(a.cur, g.W, g.H, x0, y), g.W, g.H, x0, y, c8, m.theta, s_rcp, ux, uy);
    int cx = 0, cy = 0;
#pragma unroll
    for (int q = 0; q < 8; ++q) {
        cx += ux[q] != 0.0f;
        cy += uy[q] != 0.0f;
    }
    const int nx = (int)__reduce_add_sync(kFull, (unsigned)cx);
    const int ny = (int)__reduce_add_sync(kFull, (unsigned)cy);
    float sx, sy;
    grad_sums(r8, c8, ux, uy, sx, sy);
    unsigned shp = 0;
    if (a.pcur && a.pref) {
        int cand[5] = {pack_mv(dx, dy), 0, 0, 0, 0};
        unsigned sc[5];
        shape_costs(a.pcur, a.pref, g.Wp, X0, Y0, cand, 1, m.h, lane, sc);
        shp = sc[0];
    }
    if (lane == 0) {
        if (a.tsad) a.tsad[qi] = sad;
        if (a.ssad && a.pcur) a.ssad[qi] = shp;
        if (a.delta) {
            a.delta[2 * qi] = update_of(sx, nx, m.eps);
            a.delta[2 * qi + 1] = update_of(sy, ny, m.eps);
        }
    }
}

}  // namespace

size_t me_smem_bytes(int S) { return (size_t)kMeWarps * warp_smem(S); }

cudaError_t launch_host_copy(void* dst, const void* src, size_t bytes, int num_sms, cudaStream_t s)
{
    host_copy_kernel<<<2 * num_sms, 1024, 0, s>>>(reinterpret_cast<uint4*>(dst), reinterpret_cast<const uint4*>(src),
                                                   bytes / 16);
    return cudaGetLastError();
}

cudaError_t launch_classify(const Geom& g, const ClassifyArgs& a, cudaStream_t s)
{
    dim3 grid(g.MBH, a.n_frames);
    classify_pack_kernel<<<grid, 256, 0, s>>>(g, a);
    return cudaGetLastError();
}

cudaError_t launch_classify_batch(const ClassifyBatchArgs& a, int max_mbh, int total_frames, cudaStream_t s)
{
    classify_batch_kernel<<<dim3(max_mbh, total_frames), 256, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t me_occupancy(int S, int* blocks_per_sm, bool variants)
{
    const size_t smem = me_smem_bytes(S);
    const void* fn = variants ? (const void*)me_kernel<true> : (const void*)me_kernel<false>;
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, fn, 32 * kMeWarps, smem);
}

cudaError_t me4_occupancy(int S, int* blocks_per_sm)
{
    const size_t smem = (size_t)kMeWarps * warp_smem4(S);
    cudaError_t e = cudaFuncSetAttribute(me4_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, me4_kernel, 32 * kMeWarps, smem);
}

cudaError_t launch_me4(const Method& m, const MeArgs& a, int grid, cudaStream_t s)
{
    // cooperative for the same reason as launch_me
    const size_t smem = (size_t)kMeWarps * warp_smem4(m.S);
    cudaError_t e = cudaFuncSetAttribute(me4_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(32 * kMeWarps);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, me4_kernel, a);
}

cudaError_t launch_me(const Method& m, const MeArgs& a, int grid, cudaStream_t s)
{
    // Warps wait on results of other warps of the same launch, so the launch
    // is cooperative: every block is resident at once.
    const size_t smem = me_smem_bytes(m.S);
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(m.tt ? me_kernel<true> : me_kernel<false>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(32 * kMeWarps);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, m.tt ? me_kernel<true> : me_kernel<false>, a);
}

cudaError_t launch_sparse_prep(const SparseArgs& a, const SeqDesc* desc, cudaStream_t s)
{
    SeqDesc d{};
    if (desc) d = *desc;
    sparse_reset_kernel<<<std::max(1, std::min(a.nseq, 1024)), 256, 0, s>>>(a, d, desc ? 1 : 0);
    sparse_stream_kernel<<<dim3(a.max_mbh, a.n_gf), 256, 0, s>>>(a);
    const long long warps = (a.total_rows + 31) / 32;
    const int grid = (int)std::max(1LL, std::min<long long>((warps + 7) / 8, 152 * 16));
    sparse_count_kernel<<<grid, 256, 0, s>>>(a);
    sparse_scan_kernel<<<1, 1024, 0, s>>>(a);
    sparse_scatter_kernel<<<grid, 256, 0, s>>>(a);
    return cudaGetLastError();
}

template <bool kVariants, int kMinBlocks>
cudaError_t sparse_attr(const void** fn, size_t smem)
{
    *fn = (const void*)me_sparse_kernel<kVariants, kMinBlocks>;
    if (smem > 48 * 1024) return cudaFuncSetAttribute(*fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    return cudaSuccess;
}

cudaError_t sparse_kernel(bool variants, int min_blocks, size_t smem, const void** fn)
{
    if (min_blocks == 5) return variants ? sparse_attr<true, 5>(fn, smem) : sparse_attr<false, 5>(fn, smem);
    if (variants)
        return min_blocks >= 3   ? sparse_attr<true, 3>(fn, smem)
               : min_blocks == 2 ? sparse_attr<true, 2>(fn, smem)
                                 : sparse_attr<true, 1>(fn, smem);
    return min_blocks >= 3   ? sparse_attr<false, 3>(fn, smem)
           : min_blocks == 2 ? sparse_attr<false, 2>(fn, smem)
                             : sparse_attr<false, 1>(fn, smem);
}

cudaError_t me_sparse_occupancy(int S, int min_blocks, int* blocks_per_sm, bool variants)
{
    const int warps = sparse_cta_warps(min_blocks);
    const size_t smem = (size_t)warps * warp_smem(S);
    const void* fn = nullptr;
    cudaError_t e = sparse_kernel(variants, min_blocks, smem, &fn);
    if (e != cudaSuccess) return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, fn, 32 * warps, smem);
}

cudaError_t launch_me_sparse(const Method& m, const MeArgs& a, int grid, int min_blocks, cudaStream_t s)
{
    // cooperative for the same reason as launch_me: warps wait on each other
    const int warps = sparse_cta_warps(min_blocks);
    const size_t smem = (size_t)warps * warp_smem(m.S);
    const void* fn = nullptr;
    cudaError_t e = sparse_kernel(m.tt != 0, min_blocks, smem, &fn);
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(32 * warps);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    void* args[] = {const_cast<MeArgs*>(&a)};
    return cudaLaunchKernelExC(&cfg, fn, args);
}

size_t me_cluster_smem_bytes(int S, int cap, int warps)
{
    return (size_t)warps * warp_smem(S) + (size_t)cap * (4 * sizeof(unsigned long long) + 2 * sizeof(int));
}

int me_cluster_fits(int S, int cap, int cluster, int warps)
{
    const size_t smem = me_cluster_smem_bytes(S, cap, warps);
    if (smem > 227 * 1024 ||
        cudaFuncSetAttribute(me_cluster_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
            cudaSuccess ||
        cudaFuncSetAttribute(me_cluster_kernel, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(cluster);
    cfg.blockDim = dim3(32 * warps);
    cfg.dynamicSmemBytes = smem;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = cluster;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int n = 0;
    if (cudaOccupancyMaxActiveClusters(&n, me_cluster_kernel, &cfg) == cudaSuccess && n >= 1) return n;
    cudaGetLastError();
    return 0;
}

cudaError_t launch_me_cluster(const Method& m, const MeArgs& a, int cluster, int warps, int helpers, cudaStream_t s)
{
    // The chain cluster's CTAs wait on one another only through distributed
    // shared memory, and a cluster is always resident as a whole; the helper
    // clusters wait on nothing.
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(cluster * (1 + helpers));
    cfg.blockDim = dim3(32 * warps);
    cfg.dynamicSmemBytes = me_cluster_smem_bytes(m.S, a.cl_cap, warps);
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = cluster;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, me_cluster_kernel, a);
}

void pair_boxes(int S, unsigned (&box)[4][2])
{
    box[0][0] = (unsigned)win_pitch(S);
    box[0][1] = (unsigned)win_rows(S);
    box[1][0] = kCurBoxW;
    box[1][1] = kCurBoxH;
    box[2][0] = (unsigned)aref_words(S);
    box[2][1] = (unsigned)win_rows(S);
    box[3][0] = kAcurWords;
    box[3][1] = 16;
}

size_t me_pair_smem_bytes(int S, int nwarps, int mbw_max, bool four_mv)
{
    return (size_t)pair_layout(S, nwarps, mbw_max, four_mv).total + 128;  // + alignment slack
}

cudaError_t me_pair_occupancy(int S, int nwarps, int mbw_max, bool direct, bool four_mv, int* blocks_per_sm)
{
    const size_t smem = me_pair_smem_bytes(S, nwarps, mbw_max, four_mv);
    const void* fn = four_mv  ? (const void*)me_pair_kernel<false, true>
                     : direct ? (const void*)me_pair_kernel<true, false>
                              : (const void*)me_pair_kernel<false, false>;
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, fn, 32 * nwarps, smem);
}

cudaError_t launch_me_pair(const Method& m, const MeArgs& a, const void* maps, int nwarps, int grid, cudaStream_t s)
{
    const size_t smem = me_pair_smem_bytes(m.S, nwarps, a.mbw_max, a.four_mv != 0);
    auto* fn = a.four_mv ? me_pair_kernel<false, true> : a.pair_direct ? me_pair_kernel<true, false> : me_pair_kernel<false, false>;
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(32 * nwarps);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, fn, a, *reinterpret_cast<const PairMaps*>(maps));
}

cudaError_t launch_compensate(const Geom& g, const Method& m, const CompArgs& a, cudaStream_t s)
{
    compensate_kernel<<<g.M, 256, 0, s>>>(g, m, a);
    return cudaGetLastError();
}

cudaError_t launch_queries(const Geom& g, const Method& m, const QueryArgs& a, cudaStream_t s)
{
    if (a.n <= 0) return cudaSuccess;
    const size_t smem = (size_t)kQueryWarps * warp_smem(m.S);
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(query_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    query_kernel<<<(a.n + kQueryWarps - 1) / kQueryWarps, 32 * kQueryWarps, smem, s>>>(g, m, a);
    return cudaGetLastError();
}

}  // namespace sme
