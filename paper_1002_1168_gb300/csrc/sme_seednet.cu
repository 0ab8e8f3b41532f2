// Learned seed proposal network (sm_103a): a 5-layer 3x3 convolutional
// network on a quarter-resolution grid (one cell = 4x4 pixels) that predicts
// one (dx, dy) seed per MB, used as the fifth candidate of the block recursive
// search.  The paper has no learned component (its seeds are the neighbour and
// temporal vectors of Sec. 3.1); the network only proposes, the search of
// Fig. 1 / Sec. 3.2 decides.
//
// Layers 16 -> 32 -> 32 -> 32 -> 32 -> 16 channels, ReLU after the first four,
// activations channels-last in bfloat16, FP32 accumulation on tensor cores
// (mma.sync m16n8k16).  Input gradients use the same convolution kernel with
// flipped, transposed weights and the ReLU mask fused; weight gradients are a
// tensor-core GEMM over pixels; Adam keeps FP32 master weights.
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <string.h>

#include <new>
#include <vector>

#include "sme_internal.h"

namespace sme {
namespace {

constexpr int kLayers = 5;
// Channels entering layer l (l = 0..5): 16, 32, 32, 32, 32, 16.
__host__ __device__ constexpr int chan(int l) { return (l == 0 || l == kLayers) ? 16 : 32; }
constexpr float kSeedScale = 8.0f;
constexpr float kHuber = 1.0f;
constexpr unsigned kFull = 0xffffffffu;

__host__ __device__ constexpr int wsize(int l) { return chan(l + 1) * 9 * chan(l); }
__host__ __device__ constexpr int lsize(int l) { return wsize(l) + chan(l + 1); }
__host__ __device__ constexpr int loff(int l) { return l == 0 ? 0 : loff(l - 1) + lsize(l - 1); }
constexpr int kParams = loff(kLayers);

__device__ __forceinline__ float bf2f(__nv_bfloat16 v) { return __bfloat162float(v); }

// ------------------------------------------------------------ features --
// Per 4x4 cell: current and reference mean luma (/255 - 0.5), their
// difference, the temporal candidate of the cell's MB (pixels / 16).
// Pair q of the launch (blockIdx.y) uses frames ref_f + q and cur_f + q.
__global__ void features_kernel(const uint8_t* luma, int W, int H, int ref_f0, int cur_f0, const sme_mv* temporal,
                                int subpel, __nv_bfloat16* out_all)
{
    const int Wc = W / 4, Hc = H / 4;
    const int cell = blockIdx.x * blockDim.x + threadIdx.x;
    if (cell >= Wc * Hc) return;
    const int q = blockIdx.y, ref_f = ref_f0 + q, cur_f = cur_f0 + q;
    __nv_bfloat16* out = out_all + (size_t)q * Wc * Hc * 16;
    const int ci = cell / Wc, cj = cell - ci * Wc;
    const uint8_t* r = luma + (size_t)ref_f * W * H + (size_t)(4 * ci) * W + 4 * cj;
    const uint8_t* c = luma + (size_t)cur_f * W * H + (size_t)(4 * ci) * W + 4 * cj;
    int sr = 0, sc = 0;
    for (int y = 0; y < 4; ++y)
        for (int x = 0; x < 4; ++x) {
            sr += r[y * W + x];
            sc += c[y * W + x];
        }
    const float mc = (float)sc / 16.0f, mr = (float)sr / 16.0f;
    float f[16];
    for (int k = 0; k < 16; ++k) f[k] = 0.0f;
    f[0] = mc / 255.0f - 0.5f;
    f[1] = mr / 255.0f - 0.5f;
    f[2] = (mc - mr) / 255.0f;
    if (temporal) {
        const sme_mv t = temporal[(ci / 4) * (W / 16) + cj / 4];
        f[3] = (float)t.dx / (16.0f * subpel);
        f[4] = (float)t.dy / (16.0f * subpel);
    }
    __nv_bfloat16* o = out + (size_t)cell * 16;
    for (int k = 0; k < 16; ++k) o[k] = __float2bfloat16_rn(f[k]);
}

// -------------------------------------------------------- tensor cores --
__device__ __forceinline__ void mma16816(float (&d)[4], const unsigned (&a)[4], unsigned b0, unsigned b1)
{
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}
__device__ __forceinline__ unsigned pack_bf2(__nv_bfloat16 lo, __nv_bfloat16 hi)
{
    return (unsigned)__bfloat16_as_ushort(lo) | ((unsigned)__bfloat16_as_ushort(hi) << 16);
}

// 3x3 convolution, implicit GEMM: M = output pixels (16 consecutive cells of
// one row per warp), N = COUT, K = 9 taps x CIN.  y = conv(x, w) (+ bias)
// (ReLU) (* [mask > 0]) stored as bfloat16 or FP32.  Zero padding.
template <int CIN, int COUT>
__global__ void __launch_bounds__(256) conv3x3_kernel(const __nv_bfloat16* __restrict__ x,
                                                      const __nv_bfloat16* __restrict__ w,
                                                      const float* __restrict__ bias,
                                                      const __nv_bfloat16* __restrict__ mask, int relu, int N,
                                                      int Hc, int Wc, const int* __restrict__ units,
                                                      __nv_bfloat16* y16, float* y32)
{
    constexpr int KT = 9 * CIN;        // K per output channel
    constexpr int WST = KT / 2 + 4;    // smem row stride in 32-bit words (padded against bank conflicts)
    __shared__ unsigned ws[COUT * WST];
    for (int i = threadIdx.x; i < COUT * (KT / 2); i += blockDim.x) {
        const int o = i / (KT / 2), k = i - o * (KT / 2);
        ws[o * WST + k] = reinterpret_cast<const unsigned*>(w)[i];
    }
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    const int g = lane >> 2, tq = lane & 3;
    const int mbw = Wc >> 2, per = mbw * (Hc >> 2);
    // A warp's tile is the 4x4 cells of one MB: tile row r is cell (r / 4, r % 4),
    // so this lane's rows g and g + 8 are cells (g/4, g%4) and (g/4 + 2, g%4).
    // units = NULL: every MB of the N grids; else units[0] MBs listed in units[1..].
    const int total = units ? units[0] : N * per;
    // Persistent CTAs: each warp walks MBs, the weights staged once.
    for (int k = blockIdx.x * nwarps + warp; k < total; k += gridDim.x * nwarps) {
    const int u = units ? units[1 + k] : k;
    const int n = u / per, mb = u - n * per;
    const int mv = mb / mbw, mu = mb - mv * mbw;
    const int i0 = 4 * mv + (g >> 2), j = 4 * mu + (g & 3);
    float acc[COUT / 8][4];
#pragma unroll
    for (int t = 0; t < COUT / 8; ++t)
#pragma unroll
        for (int q = 0; q < 4; ++q) acc[t][q] = 0.0f;
    const unsigned* xw = reinterpret_cast<const unsigned*>(x);
#pragma unroll
    for (int tap = 0; tap < 9; ++tap) {
        const int ii0 = i0 + tap / 3 - 1, ii1 = ii0 + 2, jj = j + tap % 3 - 1;
        const bool col_ok = jj >= 0 && jj < Wc;
        const bool ok0 = col_ok && ii0 >= 0 && ii0 < Hc, ok1 = col_ok && ii1 >= 0 && ii1 < Hc;
        const size_t p0 = ((size_t)n * Hc + ii0) * Wc + jj, p1 = p0 + 2 * (size_t)Wc;
#pragma unroll
        for (int cb = 0; cb < CIN / 16; ++cb) {
            const int c0 = cb * 16 + 2 * tq;
            unsigned a[4];
            a[0] = ok0 ? __ldg(xw + (p0 * CIN + c0) / 2) : 0u;
            a[1] = ok1 ? __ldg(xw + (p1 * CIN + c0) / 2) : 0u;
            a[2] = ok0 ? __ldg(xw + (p0 * CIN + c0 + 8) / 2) : 0u;
            a[3] = ok1 ? __ldg(xw + (p1 * CIN + c0 + 8) / 2) : 0u;
            const int k0 = (tap * CIN + c0) / 2;
#pragma unroll
            for (int t = 0; t < COUT / 8; ++t) {
                const unsigned* wr = ws + (t * 8 + g) * WST + k0;
                mma16816(acc[t], a, wr[0], wr[4]);
            }
        }
    }
    // epilogue: tile rows g and g+8 (cells (i0, j), (i0 + 2, j)), channels t*8 + 2*tq (+1)
#pragma unroll
    for (int half = 0; half < 2; ++half) {
        const size_t p = ((size_t)n * Hc + i0 + 2 * half) * Wc + j;
#pragma unroll
        for (int t = 0; t < COUT / 8; ++t) {
            const int ch = t * 8 + 2 * tq;
            float v0 = acc[t][2 * half], v1 = acc[t][2 * half + 1];
            if (bias) {
                v0 += bias[ch];
                v1 += bias[ch + 1];
            }
            if (relu) {
                v0 = fmaxf(v0, 0.0f);
                v1 = fmaxf(v1, 0.0f);
            }
            if (mask) {
                if (!(bf2f(mask[p * COUT + ch]) > 0.0f)) v0 = 0.0f;
                if (!(bf2f(mask[p * COUT + ch + 1]) > 0.0f)) v1 = 0.0f;
            }
            if (y32) {
                y32[p * COUT + ch] = v0;
                y32[p * COUT + ch + 1] = v1;
            } else {
                reinterpret_cast<unsigned*>(y16)[(p * COUT + ch) / 2] =
                    pack_bf2(__float2bfloat16_rn(v0), __float2bfloat16_rn(v1));
            }
        }
    }
    }
}

// The MBs the seeds of the non-transparent MBs (the only ones that use a
// seed) depend on.  A seed reads layer 5 on its MB's cells; layer l (1..5) is
// needed on those cells dilated by 5 - l cells, at most 4 cells = one MB.  So
// every layer is evaluated only on the MBs within one MB (Chebyshev) of a
// non-transparent MB; each needed value then reads only needed (hence
// evaluated) values of the layer before, and the seeds equal those of the
// dense pass bit for bit.
// units[0] = count (zeroed by the caller), units[1..] = MB indices n * M + mb
// in no particular order (each MB's arithmetic does not depend on it).
// With several class maps (VOPs over the same frames, maps `stride` bytes
// apart) an MB counts as non-transparent if it is so in any map.
__device__ __forceinline__ bool any_visible(const uint8_t* cls, int n_maps, long long stride, size_t i)
{
    for (int k = 0; k < n_maps; ++k)
        if (cls[k * stride + i] != 0) return true;
    return false;
}

__global__ void active_units_kernel(const uint8_t* __restrict__ cls, int n_maps, long long stride, int N, int mbw,
                                    int mbh, int* units)
{
    const int M = mbw * mbh;
    const int id = blockIdx.x * blockDim.x + threadIdx.x;
    if (id >= N * M) return;
    const int n = id / M, mb = id - n * M, v = mb / mbw, u = mb - v * mbw;
    bool act = false;
    for (int dv = -1; dv <= 1; ++dv)
        for (int du = -1; du <= 1; ++du) {
            const int vv = v + dv, uu = u + du;
            if (vv >= 0 && vv < mbh && uu >= 0 && uu < mbw &&
                any_visible(cls, n_maps, stride, (size_t)n * M + vv * mbw + uu))
                act = true;
        }
    if (act) units[1 + atomicAdd(units, 1)] = id;
}

// Weight and bias gradients: dW[o][tap][c] = sum_p dY[p][o] x[p + tap][c],
// db[o] = sum_p dY[p][o].  Nine warps per CTA (one per tap); the CTA stages a
// 16-cell row segment of dY and the three input rows it needs, each warp runs
// the GEMM M = COUT (o), N = CIN (c), K = the 16 cells; partial sums are
// added to the FP32 gradients at the end.
template <int CIN, int COUT>
__global__ void __launch_bounds__(288) conv3x3_wgrad_kernel(const __nv_bfloat16* __restrict__ x,
                                                            const __nv_bfloat16* __restrict__ dy, int N, int Hc,
                                                            int Wc, float* dw, float* db)
{
    __shared__ __nv_bfloat16 sdy[16][COUT + 2];
    __shared__ __nv_bfloat16 sx[3][18][CIN + 2];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;  // warp = tap
    const int g = lane >> 2, tq = lane & 3;
    const int segs = (Wc + 15) / 16, nseg = N * Hc * segs;
    float acc[COUT / 16][CIN / 8][4];
#pragma unroll
    for (int a_ = 0; a_ < COUT / 16; ++a_)
#pragma unroll
        for (int b_ = 0; b_ < CIN / 8; ++b_)
#pragma unroll
            for (int q = 0; q < 4; ++q) acc[a_][b_][q] = 0.0f;
    float bacc = 0.0f;  // threads < COUT of warp 0 hold db partials
    for (int seg = blockIdx.x; seg < nseg; seg += gridDim.x) {
        const int n = seg / (Hc * segs), rem = seg - n * Hc * segs;
        const int i = rem / segs, j0 = (rem - i * segs) * 16;
        __syncthreads();
        for (int e = threadIdx.x; e < 16 * COUT; e += blockDim.x) {
            const int m = e / COUT, o = e - m * COUT, j = j0 + m;
            sdy[m][o] = j < Wc ? dy[(((size_t)n * Hc + i) * Wc + j) * COUT + o] : __float2bfloat16_rn(0.0f);
        }
        for (int e = threadIdx.x; e < 3 * 18 * CIN; e += blockDim.x) {
            const int r = e / (18 * CIN), rr = e - r * 18 * CIN, m = rr / CIN, c = rr - m * CIN;
            const int ii = i + r - 1, j = j0 + m - 1;
            sx[r][m][c] = (ii >= 0 && ii < Hc && j >= 0 && j < Wc) ? x[(((size_t)n * Hc + ii) * Wc + j) * CIN + c]
                                                                   : __float2bfloat16_rn(0.0f);
        }
        __syncthreads();
        const int r = warp / 3, dx = warp % 3;
        // A = dY^T (rows o, cols cells), B = x shifted (rows cells, cols c)
#pragma unroll
        for (int mt = 0; mt < COUT / 16; ++mt) {
            unsigned a[4];
            const int o0 = mt * 16 + g, k0 = 2 * tq;
            a[0] = pack_bf2(sdy[k0][o0], sdy[k0 + 1][o0]);
            a[1] = pack_bf2(sdy[k0][o0 + 8], sdy[k0 + 1][o0 + 8]);
            a[2] = pack_bf2(sdy[k0 + 8][o0], sdy[k0 + 9][o0]);
            a[3] = pack_bf2(sdy[k0 + 8][o0 + 8], sdy[k0 + 9][o0 + 8]);
#pragma unroll
            for (int nt = 0; nt < CIN / 8; ++nt) {
                const int c = nt * 8 + g;
                const unsigned b0 = pack_bf2(sx[r][k0 + dx][c], sx[r][k0 + 1 + dx][c]);
                const unsigned b1 = pack_bf2(sx[r][k0 + 8 + dx][c], sx[r][k0 + 9 + dx][c]);
                mma16816(acc[mt][nt], a, b0, b1);
            }
        }
        if (warp == 0)
            for (int o = lane; o < COUT; o += 32)
                for (int m = 0; m < 16; ++m) bacc += bf2f(sdy[m][o]);
    }
    // accumulator element q of tile (mt, nt): o = mt*16 + g (+8 for q >= 2), c = nt*8 + 2*tq + (q & 1)
#pragma unroll
    for (int mt = 0; mt < COUT / 16; ++mt)
#pragma unroll
        for (int nt = 0; nt < CIN / 8; ++nt)
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int o = mt * 16 + g + (q >= 2 ? 8 : 0), c = nt * 8 + 2 * tq + (q & 1);
                atomicAdd(dw + ((size_t)o * 9 + warp) * CIN + c, acc[mt][nt][q]);
            }
    if (warp == 0)
        for (int o = lane; o < COUT; o += 32) atomicAdd(db + o, bacc);
}

// Per-MB seeds (SEED_SCALE x mean of output channels 0, 1 over the MB's 4x4
// cells) and, with labels, the Huber loss over the masked MBs (mean) and its
// gradient w.r.t. the cell outputs (bfloat16, channels 0, 1; others 0).
// With cls (seeds only): transparent MBs (class 0) get seed 0 and their cells
// are not read.
__global__ void pool_loss_kernel(const float* out, int N, int Hc, int Wc, float* seeds, const float* labels,
                                 const uint8_t* mask, const int* count, float* loss, __nv_bfloat16* dout,
                                 const uint8_t* cls = nullptr, int n_maps = 0, long long stride = 0)
{
    const int MBW = Wc / 4, MBH = Hc / 4, M = MBW * MBH;
    const int id = blockIdx.x * blockDim.x + threadIdx.x;
    if (id >= N * M) return;
    if (cls && !any_visible(cls, n_maps, stride, id)) {
        seeds[2 * (size_t)id] = 0.0f;
        seeds[2 * (size_t)id + 1] = 0.0f;
        return;
    }
    const int n = id / M, mb = id - n * M, u = mb % MBW, v = mb / MBW;
    float s[2] = {0.0f, 0.0f};
    for (int y = 0; y < 4; ++y)
        for (int x = 0; x < 4; ++x) {
            const float* c = out + (((size_t)n * Hc + 4 * v + y) * Wc + 4 * u + x) * 16;
            s[0] += c[0];
            s[1] += c[1];
        }
    s[0] = kSeedScale * s[0] / 16.0f;
    s[1] = kSeedScale * s[1] / 16.0f;
    if (seeds) {
        seeds[2 * (size_t)id] = s[0];
        seeds[2 * (size_t)id + 1] = s[1];
    }
    if (!labels) return;
    const float inv = 1.0f / (float)max(*count, 1);
    float g[2] = {0.0f, 0.0f}, l = 0.0f;
    if (mask[id]) {
        for (int k = 0; k < 2; ++k) {
            const float r = s[k] - labels[2 * (size_t)id + k], a = fabsf(r);
            l += a <= kHuber ? 0.5f * r * r : kHuber * (a - 0.5f * kHuber);
            g[k] = fminf(fmaxf(r, -kHuber), kHuber) * inv * (kSeedScale / 16.0f);
        }
        atomicAdd(loss, l * inv);
    }
    for (int y = 0; y < 4; ++y)
        for (int x = 0; x < 4; ++x) {
            __nv_bfloat16* d = dout + (((size_t)n * Hc + 4 * v + y) * Wc + 4 * u + x) * 16;
            d[0] = __float2bfloat16_rn(g[0]);
            d[1] = __float2bfloat16_rn(g[1]);
            for (int k = 2; k < 16; ++k) d[k] = __float2bfloat16_rn(0.0f);
        }
}

__global__ void count_kernel(const uint8_t* mask, int n, int* count)
{
    int c = 0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) c += mask[i] != 0;
    c = __reduce_add_sync(kFull, c);
    if ((threadIdx.x & 31) == 0 && c) atomicAdd(count, c);
}

// Adam on the FP32 master parameters (bias-corrected), then the bfloat16
// weights and their flipped, transposed copies for the input gradients:
// wt[c][8 - tap][o] = w[o][tap][c].
__global__ void adam_kernel(float* p, const float* grad, float* m, float* v, int n, float lr, float b1, float b2,
                            float eps, float c1, float c2)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float g = grad[i];
    const float mi = b1 * m[i] + (1.0f - b1) * g, vi = b2 * v[i] + (1.0f - b2) * g * g;
    m[i] = mi;
    v[i] = vi;
    p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

__global__ void convert_kernel(const float* p, __nv_bfloat16* w16, __nv_bfloat16* wt16)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    int l = 0;
    while (l < kLayers - 1 && i >= loff(l + 1)) ++l;
    if (i >= kParams) return;
    const int local = i - loff(l);
    if (local >= wsize(l)) return;  // bias
    const int cin = chan(l), cout = chan(l + 1);
    const int o = local / (9 * cin), rem = local - o * 9 * cin, tap = rem / cin, c = rem - tap * cin;
    const __nv_bfloat16 b = __float2bfloat16_rn(p[i]);
    int woff = 0;
    for (int q = 0; q < l; ++q) woff += wsize(q);
    w16[woff + local] = b;
    wt16[woff + ((size_t)c * 9 + (8 - tap)) * cout + o] = b;
}

int g_conv_sms = 148;  // CTAs per launch scale with the SM count (set at create)

// units: NULL for every MB of the N grids, else a device list (count first)
// of at most N * MBs entries.
template <int CIN, int COUT>
cudaError_t conv(const __nv_bfloat16* x, const __nv_bfloat16* w, const float* b, const __nv_bfloat16* mask, int relu,
                 int N, int Hc, int Wc, const int* units, __nv_bfloat16* y16, float* y32, cudaStream_t s)
{
    static int per_sm = 0;  // resident CTAs per SM of this instance
    if (per_sm == 0 &&
        (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, conv3x3_kernel<CIN, COUT>, 256, 0) != cudaSuccess ||
         per_sm < 1))
        per_sm = 1;
    const int mbs = N * (Hc / 4) * (Wc / 4);
    int grid = (mbs + 7) / 8;
    if (grid > per_sm * g_conv_sms) grid = per_sm * g_conv_sms;
    conv3x3_kernel<CIN, COUT><<<grid, 256, 0, s>>>(x, w, b, mask, relu, N, Hc, Wc, units, y16, y32);
    return cudaGetLastError();
}

template <int CIN, int COUT>
cudaError_t wgrad(const __nv_bfloat16* x, const __nv_bfloat16* dy, int N, int Hc, int Wc, float* dw, float* db,
                  int sms, cudaStream_t s)
{
    const int nseg = N * Hc * ((Wc + 15) / 16);
    const int grid = nseg < 2 * sms ? nseg : 2 * sms;
    conv3x3_wgrad_kernel<CIN, COUT><<<grid, 288, 0, s>>>(x, dy, N, Hc, Wc, dw, db);
    return cudaGetLastError();
}

}  // namespace
}  // namespace sme

using namespace sme;

struct sme_seednet {
    cudaStream_t stream = nullptr;
    int sms = 0, max_cells = 0, step = 0;
    float* master = nullptr;  // FP32 parameters: per layer W [cout][9][cin] then b [cout]
    float* grad = nullptr;
    float* adam_m = nullptr;
    float* adam_v = nullptr;
    __nv_bfloat16* w16 = nullptr;
    __nv_bfloat16* wt16 = nullptr;
    __nv_bfloat16* act[kLayers] = {};  // outputs of layers 0..3 (inputs of layers 1..4)
    float* out32 = nullptr;            // output of the last layer
    __nv_bfloat16* d0 = nullptr;       // gradient ping-pong buffers
    __nv_bfloat16* d1 = nullptr;
    float* scal = nullptr;             // loss (float) + count (int)
    int* units = nullptr;              // active MB list of the sparse forward (count first)
};

namespace {

int woff_of(int l)
{
    int o = 0;
    for (int q = 0; q < l; ++q) o += wsize(q);
    return o;
}

int forward(sme_seednet* s, const __nv_bfloat16* feat, int N, int Hc, int Wc, const int* units = nullptr)
{
    cudaStream_t st = s->stream;
    const float* b[kLayers];
    const __nv_bfloat16* w[kLayers];
    for (int l = 0; l < kLayers; ++l) {
        w[l] = s->w16 + woff_of(l);
        b[l] = s->master + loff(l) + wsize(l);
    }
    if (conv<16, 32>(feat, w[0], b[0], nullptr, 1, N, Hc, Wc, units, s->act[1], nullptr, st) ||
        conv<32, 32>(s->act[1], w[1], b[1], nullptr, 1, N, Hc, Wc, units, s->act[2], nullptr, st) ||
        conv<32, 32>(s->act[2], w[2], b[2], nullptr, 1, N, Hc, Wc, units, s->act[3], nullptr, st) ||
        conv<32, 32>(s->act[3], w[3], b[3], nullptr, 1, N, Hc, Wc, units, s->act[4], nullptr, st) ||
        conv<32, 16>(s->act[4], w[4], b[4], nullptr, 0, N, Hc, Wc, units, nullptr, s->out32, st))
        return SME_ERR_CUDA;
    return SME_OK;
}

int check_geom(sme_seednet* s, const void* feat, int N, int width, int height)
{
    if (!s || !feat || N < 1 || width <= 0 || height <= 0 || width % 16 || height % 16) return SME_ERR_ARG;
    if ((long long)N * (width / 4) * (height / 4) > s->max_cells) return SME_ERR_SIZE;
    return SME_OK;
}

// Loss, gradients into s->grad (zeroed first); no update.
int backward(sme_seednet* s, const __nv_bfloat16* feat, int N, int Hc, int Wc, const float* labels,
             const uint8_t* mask, float* loss_host)
{
    cudaStream_t st = s->stream;
    const int M = N * (Hc / 4) * (Wc / 4);
    if (cudaMemsetAsync(s->scal, 0, 16, st) || cudaMemsetAsync(s->grad, 0, sizeof(float) * kParams, st))
        return SME_ERR_CUDA;
    int* count = reinterpret_cast<int*>(s->scal + 1);
    count_kernel<<<64, 256, 0, st>>>(mask, M, count);
    pool_loss_kernel<<<(M + 127) / 128, 128, 0, st>>>(s->out32, N, Hc, Wc, nullptr, labels, mask, count, s->scal,
                                                      s->d0);
    const __nv_bfloat16* wt[kLayers];
    float* dw[kLayers];
    float* db[kLayers];
    for (int l = 0; l < kLayers; ++l) {
        wt[l] = s->wt16 + woff_of(l);
        dw[l] = s->grad + loff(l);
        db[l] = s->grad + loff(l) + wsize(l);
    }
    // layer 4 (32 -> 16): weights from act[4] and d0; input gradient into d1 (masked by act[4])
    if (wgrad<32, 16>(s->act[4], s->d0, N, Hc, Wc, dw[4], db[4], s->sms, st) ||
        conv<16, 32>(s->d0, wt[4], nullptr, s->act[4], 0, N, Hc, Wc, nullptr, s->d1, nullptr, st) ||
        wgrad<32, 32>(s->act[3], s->d1, N, Hc, Wc, dw[3], db[3], s->sms, st) ||
        conv<32, 32>(s->d1, wt[3], nullptr, s->act[3], 0, N, Hc, Wc, nullptr, s->d0, nullptr, st) ||
        wgrad<32, 32>(s->act[2], s->d0, N, Hc, Wc, dw[2], db[2], s->sms, st) ||
        conv<32, 32>(s->d0, wt[2], nullptr, s->act[2], 0, N, Hc, Wc, nullptr, s->d1, nullptr, st) ||
        wgrad<32, 32>(s->act[1], s->d1, N, Hc, Wc, dw[1], db[1], s->sms, st) ||
        conv<32, 32>(s->d1, wt[1], nullptr, s->act[1], 0, N, Hc, Wc, nullptr, s->d0, nullptr, st) ||
        wgrad<16, 32>(feat, s->d0, N, Hc, Wc, dw[0], db[0], s->sms, st))
        return SME_ERR_CUDA;
    if (loss_host) {
        if (cudaMemcpyAsync(loss_host, s->scal, sizeof(float), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
            cudaStreamSynchronize(st) != cudaSuccess)
            return SME_ERR_CUDA;
    }
    return SME_OK;
}

int refresh_weights(sme_seednet* s)
{
    convert_kernel<<<(kParams + 255) / 256, 256, 0, s->stream>>>(s->master, s->w16, s->wt16);
    return cudaGetLastError() == cudaSuccess ? SME_OK : SME_ERR_CUDA;
}

}  // namespace

extern "C" {

int sme_seednet_param_count(void) { return kParams; }

int sme_seednet_create(sme_seednet** out, int max_cells, void* stream)
{
    if (!out || max_cells < 16) return SME_ERR_ARG;
    *out = nullptr;
    sme_seednet* s = new (std::nothrow) sme_seednet();
    if (!s) return SME_ERR_NOMEM;
    s->stream = (cudaStream_t)stream;
    s->max_cells = max_cells;
    int dev = 0;
    bool ok = cudaGetDevice(&dev) == cudaSuccess &&
              cudaDeviceGetAttribute(&s->sms, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess;
    if (ok) g_conv_sms = s->sms;
    const size_t P = kParams, C = (size_t)max_cells;
    int wtot = woff_of(kLayers);
    ok = ok && cudaMalloc(&s->master, P * 4) == cudaSuccess && cudaMalloc(&s->grad, P * 4) == cudaSuccess &&
         cudaMalloc(&s->adam_m, P * 4) == cudaSuccess && cudaMalloc(&s->adam_v, P * 4) == cudaSuccess &&
         cudaMalloc(&s->w16, wtot * 2) == cudaSuccess && cudaMalloc(&s->wt16, wtot * 2) == cudaSuccess &&
         cudaMalloc(&s->out32, C * 16 * 4) == cudaSuccess && cudaMalloc(&s->d0, C * 32 * 2) == cudaSuccess &&
         cudaMalloc(&s->d1, C * 32 * 2) == cudaSuccess && cudaMalloc(&s->scal, 16) == cudaSuccess &&
         cudaMalloc(&s->units, (C / 16 + 1) * sizeof(int)) == cudaSuccess;
    for (int l = 1; l < kLayers && ok; ++l) ok = cudaMalloc(&s->act[l], C * 32 * 2) == cudaSuccess;
    ok = ok && cudaMemset(s->master, 0, P * 4) == cudaSuccess && cudaMemset(s->adam_m, 0, P * 4) == cudaSuccess &&
         cudaMemset(s->adam_v, 0, P * 4) == cudaSuccess;
    if (!ok) {
        cudaGetLastError();
        *out = s;
        sme_seednet_destroy(s);
        *out = nullptr;
        return SME_ERR_NOMEM;
    }
    *out = s;
    return refresh_weights(s);
}

int sme_seednet_destroy(sme_seednet* s)
{
    if (!s) return SME_ERR_ARG;
    cudaStreamSynchronize(s->stream);
    void* ptrs[] = {s->master, s->grad, s->adam_m, s->adam_v, s->w16,  s->wt16,
                    s->out32,  s->d0,   s->d1,     s->scal,   s->units};
    for (void* p : ptrs)
        if (p) cudaFree(p);
    for (int l = 1; l < kLayers; ++l)
        if (s->act[l]) cudaFree(s->act[l]);
    delete s;
    return SME_OK;
}

int sme_seednet_set_params(sme_seednet* s, const float* params)
{
    if (!s || !params) return SME_ERR_ARG;
    if (cudaMemcpyAsync(s->master, params, sizeof(float) * kParams, cudaMemcpyHostToDevice, s->stream) ||
        cudaMemsetAsync(s->adam_m, 0, sizeof(float) * kParams, s->stream) ||
        cudaMemsetAsync(s->adam_v, 0, sizeof(float) * kParams, s->stream))
        return SME_ERR_CUDA;
    s->step = 0;
    const int rc = refresh_weights(s);
    if (rc) return rc;
    return cudaStreamSynchronize(s->stream) == cudaSuccess ? SME_OK : SME_ERR_CUDA;
}

int sme_seednet_get_params(sme_seednet* s, float* params)
{
    if (!s || !params) return SME_ERR_ARG;
    if (cudaMemcpyAsync(params, s->master, sizeof(float) * kParams, cudaMemcpyDeviceToHost, s->stream) ||
        cudaStreamSynchronize(s->stream))
        return SME_ERR_CUDA;
    return SME_OK;
}

int sme_seednet_features(sme_seednet* s, const uint8_t* luma, int width, int height, int ref_frame,
                         int cur_frame, int n_pairs, const sme_mv* temporal, int subpel, uint16_t* feat)
{
    if (!s || !luma || !feat || width % 16 || height % 16 || width <= 0 || height <= 0 || ref_frame < 0 ||
        cur_frame < 0 || n_pairs < 1 || n_pairs > 65535 || (subpel != 1 && subpel != 2) || (temporal && n_pairs != 1))
        return SME_ERR_ARG;
    const int cells = (width / 4) * (height / 4);
    features_kernel<<<dim3((cells + 127) / 128, n_pairs), 128, 0, s->stream>>>(
        luma, width, height, ref_frame, cur_frame, temporal, subpel, reinterpret_cast<__nv_bfloat16*>(feat));
    return cudaGetLastError() == cudaSuccess ? SME_OK : SME_ERR_CUDA;
}

int sme_seednet_forward(sme_seednet* s, const uint16_t* feat, int n, int width, int height, float* seeds,
                        float* out_cells)
{
    int rc = check_geom(s, feat, n, width, height);
    if (rc) return rc;
    const int Hc = height / 4, Wc = width / 4;
    if ((rc = forward(s, reinterpret_cast<const __nv_bfloat16*>(feat), n, Hc, Wc))) return rc;
    const int M = n * (Hc / 4) * (Wc / 4);
    if (seeds) {
        pool_loss_kernel<<<(M + 127) / 128, 128, 0, s->stream>>>(s->out32, n, Hc, Wc, seeds, nullptr, nullptr,
                                                                 nullptr, nullptr, nullptr);
        if (cudaGetLastError() != cudaSuccess) return SME_ERR_CUDA;
    }
    if (out_cells &&
        cudaMemcpyAsync(out_cells, s->out32, sizeof(float) * 16 * (size_t)n * Hc * Wc, cudaMemcpyDeviceToDevice,
                        s->stream) != cudaSuccess)
        return SME_ERR_CUDA;
    return SME_OK;
}

int sme_seednet_forward_active(sme_seednet* s, const uint16_t* feat, int n, int width, int height,
                               const uint8_t* mb_class, int n_maps, long long map_stride, float* seeds)
{
    int rc = check_geom(s, feat, n, width, height);
    if (rc) return rc;
    const int Hc = height / 4, Wc = width / 4, M = n * (Hc / 4) * (Wc / 4);
    if (!mb_class || !seeds || n_maps < 1 || (n_maps > 1 && map_stride < M)) return SME_ERR_ARG;
    if (cudaMemsetAsync(s->units, 0, sizeof(int), s->stream) != cudaSuccess) return SME_ERR_CUDA;
    active_units_kernel<<<(M + 127) / 128, 128, 0, s->stream>>>(mb_class, n_maps, map_stride, n, Wc / 4, Hc / 4,
                                                                s->units);
    if (cudaGetLastError() != cudaSuccess) return SME_ERR_CUDA;
    if ((rc = forward(s, reinterpret_cast<const __nv_bfloat16*>(feat), n, Hc, Wc, s->units))) return rc;
    pool_loss_kernel<<<(M + 127) / 128, 128, 0, s->stream>>>(s->out32, n, Hc, Wc, seeds, nullptr, nullptr, nullptr,
                                                             nullptr, nullptr, mb_class, n_maps, map_stride);
    return cudaGetLastError() == cudaSuccess ? SME_OK : SME_ERR_CUDA;
}

int sme_seednet_set_stream(sme_seednet* s, void* stream)
{
    if (!s) return SME_ERR_ARG;
    s->stream = (cudaStream_t)stream;
    return SME_OK;
}

int sme_seednet_gradients(sme_seednet* s, const uint16_t* feat, int n, int width, int height, const float* labels,
                          const uint8_t* mask, float* grads, float* loss)
{
    int rc = check_geom(s, feat, n, width, height);
    if (rc) return rc;
    if (!labels || !mask) return SME_ERR_ARG;
    const int Hc = height / 4, Wc = width / 4;
    const __nv_bfloat16* f = reinterpret_cast<const __nv_bfloat16*>(feat);
    if ((rc = forward(s, f, n, Hc, Wc)) || (rc = backward(s, f, n, Hc, Wc, labels, mask, loss))) return rc;
    if (grads && (cudaMemcpyAsync(grads, s->grad, sizeof(float) * kParams, cudaMemcpyDeviceToHost, s->stream) ||
                  cudaStreamSynchronize(s->stream)))
        return SME_ERR_CUDA;
    return SME_OK;
}

int sme_seednet_train_step(sme_seednet* s, const uint16_t* feat, int n, int width, int height, const float* labels,
                           const uint8_t* mask, float lr, float* loss)
{
    int rc = check_geom(s, feat, n, width, height);
    if (rc) return rc;
    if (!labels || !mask || !(lr > 0.0f)) return SME_ERR_ARG;
    const int Hc = height / 4, Wc = width / 4;
    const __nv_bfloat16* f = reinterpret_cast<const __nv_bfloat16*>(feat);
    if ((rc = forward(s, f, n, Hc, Wc)) || (rc = backward(s, f, n, Hc, Wc, labels, mask, nullptr))) return rc;
    ++s->step;
    const float b1 = 0.9f, b2 = 0.999f;
    const float c1 = 1.0f - powf(b1, (float)s->step), c2 = 1.0f - powf(b2, (float)s->step);
    adam_kernel<<<(kParams + 255) / 256, 256, 0, s->stream>>>(s->master, s->grad, s->adam_m, s->adam_v, kParams, lr,
                                                               b1, b2, 1e-8f, c1, c2);
    if (cudaGetLastError() != cudaSuccess) return SME_ERR_CUDA;
    if ((rc = refresh_weights(s))) return rc;
    if (loss && (cudaMemcpyAsync(loss, s->scal, sizeof(float), cudaMemcpyDeviceToHost, s->stream) ||
                 cudaStreamSynchronize(s->stream)))
        return SME_ERR_CUDA;
    return SME_OK;
}

}  // extern "C"
