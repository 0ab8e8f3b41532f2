// Learned seed proposal network (sm_103a): a 5-layer 3x3 convolutional
// network on a quarter-resolution grid (one cell = 4x4 pixels) that predicts
// one (dx, dy) seed per MB, used as the fifth candidate of the block recursive
// search.  The paper has no learned component (its seeds are the neighbour and
// temporal vectors of Sec. 3.1); the network only proposes, the search of
// Fig. 1 / Sec. 3.2 decides.
//
// Layers 16 -> 32 -> 32 -> 32 -> 32 -> 16 channels, ReLU after the first four,
// activations channels-last in bfloat16, FP32 accumulation in tensor memory
// (tcgen05.mma, kind::f16).  Input gradients use the same convolution kernel
// with flipped, transposed weights and the ReLU mask fused; weight gradients
// are a tensor-core GEMM over pixels (mma.sync m16n8k16, training only); Adam
// keeps FP32 master weights.
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>
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

// ------------------------------------------------------------ features --
// Per 4x4 cell: current and reference mean luma (/255 - 0.5), their
// difference, the temporal candidate of the cell's MB (pixels / 16).
// Pair q of the launch (blockIdx.y) uses frames ref_f + q and cur_f + q.
// frames: when non-null, pair q reads frames[2q] (reference) and frames[2q + 1]
// (current) instead of frames ref_f0 + q and cur_f0 + q of luma.  tmp_tab:
// when non-null, pair q's temporal field is tmp_tab[q] (NULL: zeros).
__global__ void features_kernel(const uint8_t* luma, const uint8_t* const* frames, int W, int H, int ref_f0,
                                int cur_f0, const sme_mv* temporal, const sme_mv* const* tmp_tab, int subpel,
                                __nv_bfloat16* out_all)
{
    const int Wc = W / 4, Hc = H / 4;
    const int cell = blockIdx.x * blockDim.x + threadIdx.x;
    if (cell >= Wc * Hc) return;
    const int q = blockIdx.y, ref_f = ref_f0 + q, cur_f = cur_f0 + q;
    const int ci = cell / Wc, cj = cell - ci * Wc;
    const size_t off = (size_t)(4 * ci) * W + 4 * cj;
    const uint8_t* rf = frames ? frames[2 * q] : luma + (size_t)ref_f * W * H;
    const uint8_t* cf = frames ? frames[2 * q + 1] : luma + (size_t)cur_f * W * H;
    const uint32_t* r = reinterpret_cast<const uint32_t*>(rf + off);
    const uint32_t* c = reinterpret_cast<const uint32_t*>(cf + off);
    unsigned sr = 0, sc = 0;  // exact byte sums of the 4 x 4 cell
#pragma unroll
    for (int y = 0; y < 4; ++y) {
        sr = __dp4a(r[y * (W / 4)], 0x01010101u, sr);
        sc = __dp4a(c[y * (W / 4)], 0x01010101u, sc);
    }
    const float mc = (float)sc / 16.0f, mr = (float)sr / 16.0f;
    float f[16];
#pragma unroll
    for (int k = 0; k < 16; ++k) f[k] = 0.0f;
    f[0] = mc / 255.0f - 0.5f;
    f[1] = mr / 255.0f - 0.5f;
    f[2] = (mc - mr) / 255.0f;
    if (tmp_tab) temporal = tmp_tab[q];
    if (temporal) {
        const sme_mv t = temporal[(ci / 4) * (W / 16) + cj / 4];
        f[3] = (float)t.dx / (16.0f * subpel);
        f[4] = (float)t.dy / (16.0f * subpel);
    }
    uint4 o[2];
    unsigned* ow = reinterpret_cast<unsigned*>(o);
#pragma unroll
    for (int k = 0; k < 8; ++k) ow[k] = pack_bf2(__float2bfloat16_rn(f[2 * k]), __float2bfloat16_rn(f[2 * k + 1]));
    uint4* dst = reinterpret_cast<uint4*>(out_all + ((size_t)q * Wc * Hc + cell) * 16);
    dst[0] = o[0];
    dst[1] = o[1];
}

// Class maps deciding which MBs use a seed: an MB counts as non-transparent
// if it is so in any of n_maps maps.  Either `cls`: maps `stride` bytes apart,
// each [N][M] (pair-major); or `rows`: a device table [n_maps][N] of pointers
// to [M] class rows (a NULL entry is an empty plane), so the maps can stay
// wherever another launch wrote them (e.g. a batch's own classification).
// seed_rows: when non-null, the seeds of grid n go to seed_rows[n] ([M][2])
// instead of the contiguous seed output.
struct ClsMaps {
    const uint8_t* cls;
    const uint8_t* const* rows;
    int n_maps;
    long long stride;
    int N, M;
    float* const* seed_rows;
};
__device__ __forceinline__ bool any_visible(const ClsMaps& c, size_t i)
{
    if (c.rows) {
        const int p = (int)(i / c.M), mb = (int)(i - (size_t)p * c.M);
        for (int k = 0; k < c.n_maps; ++k) {
            const uint8_t* r = c.rows[(size_t)k * c.N + p];
            if (r && r[mb] != 0) return true;
        }
        return false;
    }
    for (int k = 0; k < c.n_maps; ++k)
        if (c.cls[k * c.stride + i] != 0) return true;
    return false;
}

// ------------------------------------------------ tcgen05 convolution --
// 3x3 convolution as an implicit GEMM on the 5th-generation tensor cores:
// y = conv(x, w) (+ bias) (ReLU) (* [mask > 0]), zero padding, stored as
// bfloat16 or FP32, or pooled into per-MB seeds.  One tile = 16 x 8 output
// cells, GEMM M = 128 (tile row r, column c is GEMM row 8r + c), N = COUT,
// K = 9 taps x CIN in MMAs of K = 16, accumulated in FP32 in tensor memory.
// Both operands sit in shared memory in the no-swizzle K-major layout, whose
// unit is the core matrix (8 rows x 16 bytes, rows 16 bytes apart):
//  A, the input halo (18 x 10 cells), one plane per 8-channel chunk, each
//    [18][10] x 16 bytes (plane stride kPlaneStride).  The A operand of tap
//    (dy, dx) is the plane set shifted by dy * 10 + dx cells: the 8 rows of a
//    core matrix are 8 consecutive cells of a halo row, 8-row groups are halo
//    rows (SBO = 160 bytes), K chunks are planes (LBO = kPlaneStride).
//  B, the weights, K-major per output channel, [K/8][COUT] x 16 bytes (8-row
//    groups of output channels 128 bytes apart, K chunks COUT x 16 apart);
//    the weights are kept in this layout in global memory, so one bulk copy
//    stages them.
// Persistent CTAs, warp-specialised: warp 0 loads each tile's halo with one
// TMA box per 8-channel chunk (zero fill outside the grid) into a ring of
// kStages buffers; warp 1 owns tensor memory, and its lane 0 issues the 18
// (or 9) MMAs of a tile into one of kAccs accumulators and commits them to
// the buffer's "empty" and the accumulator's "full" mbarriers; warps 2-5
// (one per 32-lane quarter of tensor memory) drain accumulators with
// tcgen05.ld, release them, and run the epilogue.  Every wait is bounded; a
// wait that gives up raises the CTA's abort flag and the launch's error word.
constexpr int kTileH = 16, kTileW = 8;
constexpr int kHaloH = kTileH + 2, kHaloW = kTileW + 2;
constexpr int kPlaneBytes = kHaloH * kHaloW * 16;  // one 8-channel halo plane (2880)
constexpr int kPlaneStride = 2944;                 // planes 128-byte aligned
constexpr int kStages = 4;                         // halo buffers in flight
constexpr int kAccs = 4;                           // accumulators in tensor memory
constexpr int kAccCols = 32;                       // FP32 columns per accumulator (>= COUT)
constexpr int kTmemCols = kAccs * kAccCols;        // a power of two >= 32
constexpr int kConvThreads = 192;
constexpr int kConvCtasPerSm = 3;
constexpr long long kConvTimeoutNs = 1000000000ll;

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// Shared-memory matrix descriptor of the tensor cores (no swizzle): start
// address, leading (K) and stride (M/N) byte offsets, all in 16-byte units;
// descriptor version 1 (bits 46-47); layout type 0 (bits 61-63).
__device__ __forceinline__ uint64_t umma_desc(uint32_t addr, uint32_t lbo, uint32_t sbo)
{
    return (uint64_t)((addr >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}

// kind::f16 instruction descriptor: D FP32 (bits 4-5 = 1), A and B bfloat16
// (bits 7-9, 10-12 = 1), both K-major (bits 15, 16 = 0), N >> 3 at bit 17,
// M >> 4 at bit 24.
__host__ __device__ constexpr uint32_t umma_idesc(int M, int N)
{
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ long long globaltimer()
{
    long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ void mbar_init(uint32_t bar, int count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint32_t bar)
{
    asm volatile("mbarrier.arrive.release.cta.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.release.cta.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
                 : "memory");
}

// Bounded wait for the phase of parity `parity`; false when it timed out
// (the abort flag is then raised) or another thread raised the flag.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, volatile int* abort_flag)
{
    const long long t0 = globaltimer();
    for (long long k = 0;; ++k) {
        uint32_t done;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(done)
            : "r"(bar), "r"(parity)
            : "memory");
        if (done) return true;
        if ((k & 63) == 63) {
            if (*abort_flag) return false;
            if (globaltimer() - t0 > kConvTimeoutNs || k > (1ll << 32)) {
                *abort_flag = 1;
                return false;
            }
        }
    }
}

// 4-D tiled TMA load (coordinates innermost first) completing on bar.
__device__ __forceinline__ void tma_load_4d(uint32_t dst, const CUtensorMap* map, int c0, int c1, int c2, int c3,
                                            uint32_t bar)
{
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, "
        "%5}], [%6];" ::"r"(dst),
        "l"(map), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(bar)
        : "memory");
}

__device__ __forceinline__ void bulk_load(uint32_t dst, const void* src, uint32_t bytes, uint32_t bar)
{
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
                 "l"(src), "r"(bytes), "r"(bar)
                 : "memory");
}

template <int NC>
__device__ __forceinline__ void tmem_load(uint32_t taddr, uint32_t (&r)[NC]);

template <>
__device__ __forceinline__ void tmem_load<16>(uint32_t taddr, uint32_t (&r)[16])
{
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];\n"
        "tcgen05.wait::ld.sync.aligned;\n"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr)
        : "memory");
}

template <>
__device__ __forceinline__ void tmem_load<32>(uint32_t taddr, uint32_t (&r)[32])
{
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];\n"
        "tcgen05.wait::ld.sync.aligned;\n"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr)
        : "memory");
}

__host__ __device__ constexpr int align_up(int v, int a) { return (v + a - 1) / a * a; }

// Dynamic shared memory of one CTA.
template <int CIN, int COUT>
struct ConvLayout {
    static constexpr int KC = CIN / 8;      // 8-channel chunks of an input cell
    static constexpr int KB = 9 * CIN / 8;  // K chunks of the weights
    static constexpr int w_bytes = KB * COUT * 16;
    static constexpr int stage_bytes = KC * kPlaneStride;
    static constexpr int a_off = align_up(w_bytes, 128);
    static constexpr int bias_off = a_off + kStages * stage_bytes;
    static constexpr int bar_off = align_up(bias_off + COUT * 4, 8);
    // mbarriers: full[kStages], empty[kStages], acc_full[kAccs], acc_empty[kAccs], weights
    static constexpr int n_bars = 2 * kStages + 2 * kAccs + 1;
    static constexpr int misc_off = bar_off + 8 * n_bars;  // tensor-memory address, abort flag
    static constexpr int bytes = misc_off + 16;
};

// Tiles: t -> (n, tr, tc) over N x ceil(Hc/16) x ceil(Wc/8); units = NULL for
// every tile, else units[0] tiles listed in units[1..].  Output: y16
// (bfloat16), y32 (FP32) or, with seeds, the per-MB seeds (SEED_SCALE x mean
// of channels 0, 1 over the MB's 4 x 4 cells); with cls, MBs transparent in
// every class map are left alone (the caller zeroed the seeds).
// err: set when a wait gave up (the launch's outputs are then not valid).
template <int CIN, int COUT>
__global__ void __launch_bounds__(kConvThreads) conv3x3_tc_kernel(
    const __grid_constant__ CUtensorMap xmap, const __nv_bfloat16* __restrict__ w, const float* __restrict__ bias,
    const __nv_bfloat16* __restrict__ mask, int relu, int N, int Hc, int Wc, const int* __restrict__ units,
    __nv_bfloat16* y16, float* y32, float* seeds, const ClsMaps cm, int* err)
{
    static_assert(CIN % 16 == 0 && COUT % 16 == 0 && COUT <= kAccCols, "tile shape");
    using L = ConvLayout<CIN, COUT>;
    constexpr int KC = L::KC;
    extern __shared__ __align__(1024) uint8_t dsm[];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int TR = (Hc + kTileH - 1) / kTileH, TC = (Wc + kTileW - 1) / kTileW, per = TR * TC;
    const int total = units ? units[0] : N * per;
    if ((int)blockIdx.x >= total) return;  // uniform over the CTA
    const int n_tiles = (total - (int)blockIdx.x + (int)gridDim.x - 1) / (int)gridDim.x;

    const uint32_t sbase = smem_u32(dsm);
    const uint32_t s_w = sbase, s_a = sbase + L::a_off, s_bar = sbase + L::bar_off;
    float* s_bias = reinterpret_cast<float*>(dsm + L::bias_off);
    uint32_t* s_tmem = reinterpret_cast<uint32_t*>(dsm + L::misc_off);
    volatile int* s_abort = reinterpret_cast<volatile int*>(dsm + L::misc_off + 4);
    auto full = [&](int s) { return s_bar + 8 * s; };
    auto empty = [&](int s) { return s_bar + 8 * (kStages + s); };
    auto acc_full = [&](int a) { return s_bar + 8 * (2 * kStages + a); };
    auto acc_empty = [&](int a) { return s_bar + 8 * (2 * kStages + kAccs + a); };
    const uint32_t wbar = s_bar + 8 * (2 * kStages + 2 * kAccs);

    if (tid < COUT) s_bias[tid] = bias ? bias[tid] : 0.0f;
    if (tid == 0) {
        *s_abort = 0;
        for (int s = 0; s < kStages; ++s) {
            mbar_init(full(s), 1);
            mbar_init(empty(s), 1);
        }
        for (int a = 0; a < kAccs; ++a) {
            mbar_init(acc_full(a), 1);
            mbar_init(acc_empty(a), 4);  // one arrival per epilogue warp
        }
        mbar_init(wbar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(s_tmem)),
                     "r"(kTmemCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *s_tmem;

    auto tile_of = [&](int t, int& n, int& tr, int& tc) {
        const int u = units ? units[1 + t] : t;
        n = u / per;
        const int rem = u - n * per;
        tr = rem / TC;
        tc = rem - tr * TC;
    };

    if (warp == 0) {
        // ---- producer: weights once, then one halo per tile
        if (lane == 0) {
            mbar_expect_tx(wbar, L::w_bytes);
            bulk_load(s_w, w, L::w_bytes, wbar);
            for (int i = 0; i < n_tiles; ++i) {
                const int s = i % kStages, t = blockIdx.x + i * gridDim.x;
                if (!mbar_wait(empty(s), ((i / kStages) & 1) ^ 1, s_abort)) break;
                int n, tr, tc;
                tile_of(t, n, tr, tc);
                mbar_expect_tx(full(s), KC * kPlaneBytes);
                for (int c = 0; c < KC; ++c)
                    tma_load_4d(s_a + s * L::stage_bytes + c * kPlaneStride, &xmap, 8 * c, tc * kTileW - 1,
                                tr * kTileH - 1, n, full(s));
            }
        }
    } else if (warp == 1) {
        // ---- MMA issuer
        if (lane == 0 && mbar_wait(wbar, 0, s_abort)) {
            const uint32_t idesc = umma_idesc(128, COUT);
            for (int i = 0; i < n_tiles; ++i) {
                const int s = i % kStages, a = i % kAccs;
                if (!mbar_wait(full(s), (i / kStages) & 1, s_abort)) break;
                if (!mbar_wait(acc_empty(a), ((i / kAccs) & 1) ^ 1, s_abort)) break;
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                const uint32_t abase = s_a + s * L::stage_bytes, d = tmem + a * kAccCols;
#pragma unroll
                for (int tap = 0; tap < 9; ++tap) {
#pragma unroll
                    for (int ks = 0; ks < CIN / 16; ++ks) {
                        const uint64_t ad = umma_desc(abase + 2 * ks * kPlaneStride + ((tap / 3) * kHaloW + tap % 3) * 16,
                                                      kPlaneStride, kHaloW * 16);
                        const uint64_t bd = umma_desc(s_w + ((tap * CIN + ks * 16) / 8) * COUT * 16, COUT * 16, 128);
                        const uint32_t accumulate = (tap | ks) != 0;
                        asm volatile(
                            "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                            " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d),
                            "l"(ad), "l"(bd), "r"(idesc), "r"(accumulate)
                            : "memory");
                    }
                }
                asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                                 empty(s))
                             : "memory");
                asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                                 acc_full(a))
                             : "memory");
            }
            // the buffers' last releases have landed before the CTA ends
            for (int j = n_tiles > kStages ? n_tiles - kStages : 0; j < n_tiles && !*s_abort; ++j)
                mbar_wait(empty(j % kStages), (j / kStages) & 1, s_abort);
        }
    } else {
        // ---- epilogue: warp w drains lanes 32 (w % 4) .. + 31 of each accumulator
        const int q = warp & 3, m = 32 * q + lane;
        for (int i = 0; i < n_tiles; ++i) {
            const int a = i % kAccs, t = blockIdx.x + i * gridDim.x;
            const bool ok = mbar_wait(acc_full(a), (i / kAccs) & 1, s_abort);
            if (__any_sync(kFull, !ok)) break;
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            uint32_t r[COUT];
            tmem_load<COUT>(tmem + ((uint32_t)(32 * q) << 16) + a * kAccCols, r);
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
            __syncwarp();
            if (lane == 0) mbar_arrive(acc_empty(a));
            int n, tr, tc;
            tile_of(t, n, tr, tc);
            const int i_cell = tr * kTileH + (m >> 3), j_cell = tc * kTileW + (m & 7);
            const bool inside = i_cell < Hc && j_cell < Wc;
            const size_t p = ((size_t)n * Hc + i_cell) * Wc + j_cell;
            float v[COUT];
#pragma unroll
            for (int c = 0; c < COUT; ++c) {
                v[c] = __uint_as_float(r[c]) + s_bias[c];
                if (relu) v[c] = fmaxf(v[c], 0.0f);
            }
            if (seeds || cm.seed_rows) {
                // MB = 4 x 4 cells: this warp's 4 tile rows are one MB row of
                // the tile; lanes (row = lane >> 3, col = lane & 7) -> MB
                // column col >> 2.  Sum over lane bits 0, 1 (columns) and
                // 3, 4 (rows).
                float s0 = v[0], s1 = v[1];
#pragma unroll
                for (int o = 1; o <= 16; o <<= 1) {
                    if (o == 4) continue;
                    s0 += __shfl_xor_sync(kFull, s0, o);
                    s1 += __shfl_xor_sync(kFull, s1, o);
                }
                if ((lane & 0x1B) == 0 && inside) {
                    const int mbw = Wc >> 2, mb = (i_cell >> 2) * mbw + (j_cell >> 2);
                    const size_t id = (size_t)n * mbw * (Hc >> 2) + mb;
                    if ((!cm.cls && !cm.rows) || any_visible(cm, id)) {
                        float* dst = cm.seed_rows ? cm.seed_rows[n] + 2 * mb : seeds + 2 * id;
                        dst[0] = kSeedScale * s0 / 16.0f;
                        dst[1] = kSeedScale * s1 / 16.0f;
                    }
                }
                continue;
            }
            if (!inside) continue;
            if (mask) {
#pragma unroll
                for (int qq = 0; qq < COUT / 8; ++qq) {
                    const uint4 mk = *reinterpret_cast<const uint4*>(mask + p * COUT + 8 * qq);
                    const unsigned mw[4] = {mk.x, mk.y, mk.z, mk.w};
#pragma unroll
                    for (int e = 0; e < 8; ++e) {
                        const unsigned short h = (unsigned short)(mw[e >> 1] >> (16 * (e & 1)));
                        if (!(bf2f(__ushort_as_bfloat16(h)) > 0.0f)) v[8 * qq + e] = 0.0f;
                    }
                }
            }
            if (y32) {
#pragma unroll
                for (int qq = 0; qq < COUT / 4; ++qq)
                    *reinterpret_cast<float4*>(y32 + p * COUT + 4 * qq) =
                        make_float4(v[4 * qq], v[4 * qq + 1], v[4 * qq + 2], v[4 * qq + 3]);
            } else {
#pragma unroll
                for (int qq = 0; qq < COUT / 8; ++qq) {
                    uint4 o;
                    o.x = pack_bf2(__float2bfloat16_rn(v[8 * qq]), __float2bfloat16_rn(v[8 * qq + 1]));
                    o.y = pack_bf2(__float2bfloat16_rn(v[8 * qq + 2]), __float2bfloat16_rn(v[8 * qq + 3]));
                    o.z = pack_bf2(__float2bfloat16_rn(v[8 * qq + 4]), __float2bfloat16_rn(v[8 * qq + 5]));
                    o.w = pack_bf2(__float2bfloat16_rn(v[8 * qq + 6]), __float2bfloat16_rn(v[8 * qq + 7]));
                    *reinterpret_cast<uint4*>(y16 + p * COUT + 8 * qq) = o;
                }
            }
        }
    }
    __syncwarp();
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (tid == 0 && *s_abort) atomicExch(err, 1);
    if (warp == 1) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols) : "memory");
    }
}

// The tiles the seeds of the non-transparent MBs (the only ones that use a
// seed) depend on.  A seed reads layer 5 on its MB's cells; layer l (1..5) is
// needed on those cells dilated by 5 - l cells, at most 4 cells = one MB.  So
// every layer is evaluated only on the tiles holding an MB within one MB
// (Chebyshev) of a non-transparent MB; each needed value then reads only
// needed (hence evaluated) values of the layer before, and the seeds equal
// those of the dense pass bit for bit.  A tile covers MB rows 4tr..4tr+3 and
// MB columns 2tc, 2tc+1.
// units[0] = count (zeroed by the caller), units[1..] = tile indices in no
// particular order (a tile's arithmetic does not depend on it).
__global__ void active_tiles_kernel(const ClsMaps cm, int N, int mbw, int mbh, int TR, int TC, int* units)
{
    const int id = blockIdx.x * blockDim.x + threadIdx.x;
    if (id >= N * TR * TC) return;
    const int n = id / (TR * TC), rem = id - n * TR * TC, tr = rem / TC, tc = rem - tr * TC;
    const size_t M = (size_t)mbw * mbh;
    bool act = false;
    for (int v = 4 * tr - 1; v <= 4 * tr + 4 && !act; ++v)
        for (int u = 2 * tc - 1; u <= 2 * tc + 2; ++u)
            if (v >= 0 && v < mbh && u >= 0 && u < mbw && any_visible(cm, n * M + v * mbw + u)) {
                act = true;
                break;
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
__global__ void pool_loss_kernel(const float* out, int N, int Hc, int Wc, float* seeds, const float* labels,
                                 const uint8_t* mask, const int* count, float* loss, __nv_bfloat16* dout)
{
    const int MBW = Wc / 4, MBH = Hc / 4, M = MBW * MBH;
    const int id = blockIdx.x * blockDim.x + threadIdx.x;
    if (id >= N * M) return;
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

// Adam on the FP32 master parameters (bias-corrected).
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

// The bfloat16 weights of every layer in the tensor cores' K-major operand
// layout, [K/8][Cout][8] with k = tap * Cin + c (so one bulk copy stages a
// layer), and the flipped, transposed copies for the input gradients: the
// convolution with Cin' = Cout, Cout' = Cin and w'[c][8 - tap][o] = w[o][tap][c].
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
    const int k = tap * cin + c, kt = (8 - tap) * cout + o;
    w16[woff + ((k >> 3) * cout + o) * 8 + (k & 7)] = b;
    wt16[woff + ((kt >> 3) * cin + c) * 8 + (kt & 7)] = b;
}

int g_conv_sms = 148;  // CTAs per launch scale with the SM count (set at create)

// CTAs of `threads` threads of kernel f (with dyn_smem bytes of dynamic
// shared memory) that fit on one SM at once: the minimum over shared memory,
// registers, threads and tensor-memory columns (every CTA allocates
// kTmemCols of the SM's 512).
int resident_ctas(const void* f, int threads, int dyn_smem)
{
    cudaFuncAttributes fa;
    int dev = 0, smem = 0, regs = 0, thr = 0, maxb = 0;
    if (cudaFuncGetAttributes(&fa, f) != cudaSuccess || cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&smem, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&regs, cudaDevAttrMaxRegistersPerMultiprocessor, dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&thr, cudaDevAttrMaxThreadsPerMultiProcessor, dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&maxb, cudaDevAttrMaxBlocksPerMultiprocessor, dev) != cudaSuccess) {
        cudaGetLastError();
        return 1;
    }
    int n = 512 / kTmemCols;
    const int per_cta_smem = (int)fa.sharedSizeBytes + dyn_smem + 1024;  // + the per-CTA reservation
    const int warp_regs = ((fa.numRegs * 32 + 255) / 256) * 256;  // registers are allocated per warp
    n = std::min(n, smem / per_cta_smem);
    if (warp_regs > 0) n = std::min(n, regs / (warp_regs * ((threads + 31) / 32)));
    n = std::min(n, thr / threads);
    n = std::min(n, maxb);
    return n < 1 ? 1 : n;
}

// One convolution launch.  x: [N][Hc][Wc][CIN] bfloat16 (16-byte aligned),
// read through a 4-D tensor map (channels, columns, rows, grids) with an
// 8 x 10 x 18 x 1 box.  units: NULL for every tile of the N grids, else a
// device list (count first) of at most N * tiles entries.  Exactly one of
// y16, y32, seeds receives the result.
template <int CIN, int COUT>
cudaError_t conv(const __nv_bfloat16* x, const __nv_bfloat16* w, const float* b, const __nv_bfloat16* mask, int relu,
                 int N, int Hc, int Wc, const int* units, __nv_bfloat16* y16, float* y32, float* seeds,
                 const ClsMaps& cm, int* err, cudaStream_t s)
{
    using L = ConvLayout<CIN, COUT>;
    static int per_sm = 0;  // CTAs per SM of this instance
    if (per_sm == 0) {
        const cudaError_t e = cudaFuncSetAttribute(conv3x3_tc_kernel<CIN, COUT>,
                                                   cudaFuncAttributeMaxDynamicSharedMemorySize, L::bytes);
        if (e != cudaSuccess) return e;
        per_sm = std::min(kConvCtasPerSm,
                          resident_ctas(reinterpret_cast<const void*>(conv3x3_tc_kernel<CIN, COUT>), kConvThreads,
                                        L::bytes));
    }
    PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
    if (!enc) return cudaErrorNotSupported;
    CUtensorMap map;
    const cuuint64_t dims[4] = {(cuuint64_t)CIN, (cuuint64_t)Wc, (cuuint64_t)Hc, (cuuint64_t)N};
    const cuuint64_t strides[3] = {(cuuint64_t)CIN * 2, (cuuint64_t)Wc * CIN * 2, (cuuint64_t)Hc * Wc * CIN * 2};
    const cuuint32_t box[4] = {8u, (cuuint32_t)kHaloW, (cuuint32_t)kHaloH, 1u};
    const cuuint32_t estr[4] = {1u, 1u, 1u, 1u};
    if (enc(&map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, const_cast<__nv_bfloat16*>(x), dims, strides, box, estr,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
        return cudaErrorInvalidValue;
    const long long tiles = (long long)N * ((Hc + kTileH - 1) / kTileH) * ((Wc + kTileW - 1) / kTileW);
    int grid = (int)std::min(tiles, (long long)per_sm * g_conv_sms);
    if (grid < 1) grid = 1;
    conv3x3_tc_kernel<CIN, COUT><<<grid, kConvThreads, L::bytes, s>>>(map, w, b, mask, relu, N, Hc, Wc, units, y16,
                                                                       y32, seeds, cm, err);
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
    int* units = nullptr;              // active tile list of the sparse forward (count first)
    int* err = nullptr;                // set by a device wait that gave up
};

namespace {

int woff_of(int l)
{
    int o = 0;
    for (int q = 0; q < l; ++q) o += wsize(q);
    return o;
}

// Layers 0..4.  With seeds the last layer's epilogue pools the per-MB seeds
// (with class maps: only MBs visible in one of them); otherwise its output
// goes to out32.
int forward(sme_seednet* s, const __nv_bfloat16* feat, int N, int Hc, int Wc, const int* units = nullptr,
            float* seeds = nullptr, const ClsMaps& cm = ClsMaps{})
{
    const ClsMaps none{};
    cudaStream_t st = s->stream;
    const float* b[kLayers];
    const __nv_bfloat16* w[kLayers];
    for (int l = 0; l < kLayers; ++l) {
        w[l] = s->w16 + woff_of(l);
        b[l] = s->master + loff(l) + wsize(l);
    }
    int* e = s->err;
    if (conv<16, 32>(feat, w[0], b[0], nullptr, 1, N, Hc, Wc, units, s->act[1], nullptr, nullptr, none, e, st) ||
        conv<32, 32>(s->act[1], w[1], b[1], nullptr, 1, N, Hc, Wc, units, s->act[2], nullptr, nullptr, none, e, st) ||
        conv<32, 32>(s->act[2], w[2], b[2], nullptr, 1, N, Hc, Wc, units, s->act[3], nullptr, nullptr, none, e, st) ||
        conv<32, 32>(s->act[3], w[3], b[3], nullptr, 1, N, Hc, Wc, units, s->act[4], nullptr, nullptr, none, e, st) ||
        conv<32, 16>(s->act[4], w[4], b[4], nullptr, 0, N, Hc, Wc, units, nullptr,
                     (seeds || cm.seed_rows) ? nullptr : s->out32, seeds,
                     cm, e, st))
        return SME_ERR_CUDA;
    return SME_OK;
}

int check_geom(sme_seednet* s, const void* feat, int N, int width, int height)
{
    if (!s || !feat || N < 1 || width <= 0 || height <= 0 || width % 16 || height % 16 || ((uintptr_t)feat & 15))
        return SME_ERR_ARG;
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
    const ClsMaps none{};
    // layer 4 (32 -> 16): weights from act[4] and d0; input gradient into d1 (masked by act[4])
    if (wgrad<32, 16>(s->act[4], s->d0, N, Hc, Wc, dw[4], db[4], s->sms, st) ||
        conv<16, 32>(s->d0, wt[4], nullptr, s->act[4], 0, N, Hc, Wc, nullptr, s->d1, nullptr, nullptr, none, s->err, st) ||
        wgrad<32, 32>(s->act[3], s->d1, N, Hc, Wc, dw[3], db[3], s->sms, st) ||
        conv<32, 32>(s->d1, wt[3], nullptr, s->act[3], 0, N, Hc, Wc, nullptr, s->d0, nullptr, nullptr, none, s->err, st) ||
        wgrad<32, 32>(s->act[2], s->d0, N, Hc, Wc, dw[2], db[2], s->sms, st) ||
        conv<32, 32>(s->d0, wt[2], nullptr, s->act[2], 0, N, Hc, Wc, nullptr, s->d1, nullptr, nullptr, none, s->err, st) ||
        wgrad<32, 32>(s->act[1], s->d1, N, Hc, Wc, dw[1], db[1], s->sms, st) ||
        conv<32, 32>(s->d1, wt[1], nullptr, s->act[1], 0, N, Hc, Wc, nullptr, s->d0, nullptr, nullptr, none, s->err, st) ||
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
         cudaMalloc(&s->units, (C / 16 + 1) * sizeof(int)) == cudaSuccess &&
         cudaMalloc(&s->err, sizeof(int)) == cudaSuccess && cudaMemset(s->err, 0, sizeof(int)) == cudaSuccess;
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
                    s->out32,  s->d0,   s->d1,     s->scal,   s->units, s->err};
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
    if (!s || !luma || !feat || ((uintptr_t)luma & 3) || ((uintptr_t)feat & 15) || width % 16 || height % 16 ||
        width <= 0 || height <= 0 || ref_frame < 0 ||
        cur_frame < 0 || n_pairs < 1 || n_pairs > 65535 || (subpel != 1 && subpel != 2) || (temporal && n_pairs != 1))
        return SME_ERR_ARG;
    const int cells = (width / 4) * (height / 4);
    features_kernel<<<dim3((cells + 127) / 128, n_pairs), 128, 0, s->stream>>>(
        luma, nullptr, width, height, ref_frame, cur_frame, temporal, nullptr, subpel,
        reinterpret_cast<__nv_bfloat16*>(feat));
    return cudaGetLastError() == cudaSuccess ? SME_OK : SME_ERR_CUDA;
}

int sme_seednet_features_table(sme_seednet* s, const uint8_t* const* frames, const sme_mv* const* temporal,
                               int n_pairs, int width, int height, int subpel, uint16_t* feat)
{
    if (!s || !frames || !feat || ((uintptr_t)feat & 15) || width % 16 || height % 16 || width <= 0 || height <= 0 ||
        n_pairs < 1 || n_pairs > 65535 || (subpel != 1 && subpel != 2))
        return SME_ERR_ARG;
    const int cells = (width / 4) * (height / 4);
    features_kernel<<<dim3((cells + 127) / 128, n_pairs), 128, 0, s->stream>>>(
        nullptr, frames, width, height, 0, 0, nullptr, temporal, subpel, reinterpret_cast<__nv_bfloat16*>(feat));
    return cudaGetLastError() == cudaSuccess ? SME_OK : SME_ERR_CUDA;
}

int sme_seednet_forward(sme_seednet* s, const uint16_t* feat, int n, int width, int height, float* seeds,
                        float* out_cells)
{
    int rc = check_geom(s, feat, n, width, height);
    if (rc) return rc;
    const int Hc = height / 4, Wc = width / 4;
    const __nv_bfloat16* f = reinterpret_cast<const __nv_bfloat16*>(feat);
    if (!out_cells) return seeds ? forward(s, f, n, Hc, Wc, nullptr, seeds) : SME_OK;  // seeds pooled in place
    if ((rc = forward(s, f, n, Hc, Wc))) return rc;
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

// The sparse forward for class maps given either way (see ClsMaps).  With
// contiguous seeds the MBs not evaluated get (0, 0); with seed rows they are
// left as they are.
static int forward_active(sme_seednet* s, const uint16_t* feat, int n, int width, int height, const ClsMaps& cm,
                          float* seeds)
{
    const int Hc = height / 4, Wc = width / 4, M = n * (Hc / 4) * (Wc / 4);
    const int TR = (Hc + kTileH - 1) / kTileH, TC = (Wc + kTileW - 1) / kTileW, T = n * TR * TC;
    if (cudaMemsetAsync(s->units, 0, sizeof(int), s->stream) != cudaSuccess) return SME_ERR_CUDA;
    active_tiles_kernel<<<(T + 127) / 128, 128, 0, s->stream>>>(cm, n, Wc / 4, Hc / 4, TR, TC, s->units);
    if (cudaGetLastError() != cudaSuccess ||
        (!cm.seed_rows && cudaMemsetAsync(seeds, 0, sizeof(float) * 2 * (size_t)M, s->stream) != cudaSuccess))
        return SME_ERR_CUDA;
    return forward(s, reinterpret_cast<const __nv_bfloat16*>(feat), n, Hc, Wc, s->units, seeds, cm);
}

int sme_seednet_forward_active(sme_seednet* s, const uint16_t* feat, int n, int width, int height,
                               const uint8_t* mb_class, int n_maps, long long map_stride, float* seeds)
{
    int rc = check_geom(s, feat, n, width, height);
    if (rc) return rc;
    const int M = n * (height / 16) * (width / 16);
    if (!mb_class || !seeds || n_maps < 1 || (n_maps > 1 && map_stride < M)) return SME_ERR_ARG;
    ClsMaps cm{};
    cm.cls = mb_class;
    cm.n_maps = n_maps;
    cm.stride = map_stride;
    cm.N = n;
    cm.M = (height / 16) * (width / 16);
    return forward_active(s, feat, n, width, height, cm, seeds);
}

int sme_seednet_forward_active_table(sme_seednet* s, const uint16_t* feat, int n, int width, int height,
                                     const uint8_t* const* rows, int n_maps, float* seeds, float* const* seed_rows)
{
    int rc = check_geom(s, feat, n, width, height);
    if (rc) return rc;
    if (!rows || (!seeds == !seed_rows) || n_maps < 1) return SME_ERR_ARG;
    ClsMaps cm{};
    cm.rows = rows;
    cm.seed_rows = seed_rows;
    cm.n_maps = n_maps;
    cm.N = n;
    cm.M = (height / 16) * (width / 16);
    return forward_active(s, feat, n, width, height, cm, seeds);
}

// One temporal field per scene from its VOPs' fields (the network input is
// shared by the VOPs of a scene): in scene q (blockIdx.y), MB m takes the
// vector of the first VOP j whose class row marks it non-transparent
// (fields[q][j][m]), else (0, 0).
__global__ void temporal_composite_kernel(const sme_mv* const* fields, const uint8_t* const* classes, int n_vops,
                                          int M, sme_mv* out)
{
    const int m = blockIdx.x * blockDim.x + threadIdx.x, q = blockIdx.y;
    if (m >= M) return;
    sme_mv t{0, 0};
    for (int j = 0; j < n_vops; ++j) {
        const uint8_t* c = classes[(size_t)q * n_vops + j];
        const sme_mv* f = fields[(size_t)q * n_vops + j];
        if (c && f && c[m] != 0) {
            t = f[m];
            break;
        }
    }
    out[(size_t)q * M + m] = t;
}

int sme_seednet_temporal_composite(sme_seednet* s, const sme_mv* const* fields, const uint8_t* const* classes,
                                   int n, int n_vops, int width, int height, sme_mv* out)
{
    if (!s || !fields || !classes || !out || n < 1 || n > 65535 || n_vops < 1 || width <= 0 || height <= 0 ||
        width % 16 || height % 16)
        return SME_ERR_ARG;
    const int M = (width / 16) * (height / 16);
    temporal_composite_kernel<<<dim3((M + 255) / 256, n), 256, 0, s->stream>>>(fields, classes, n_vops, M, out);
    return cudaGetLastError() == cudaSuccess ? SME_OK : SME_ERR_CUDA;
}

int sme_seednet_synchronize(sme_seednet* s)
{
    if (!s) return SME_ERR_ARG;
    int e = 0;
    if (cudaStreamSynchronize(s->stream) != cudaSuccess ||
        cudaMemcpy(&e, s->err, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess)
        return SME_ERR_CUDA;
    return e ? SME_ERR_TIMEOUT : SME_OK;
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
