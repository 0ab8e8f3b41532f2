// Exhaustive search (ES) on the GPU: for every 16x16 MB of every frame pair,
// the SAD at every vector of the valid set V and the first minimum in raster
// order (dy outer, dx inner).  This is the comparison method of the paper's
// experiments (Sec. 1, Table 1's ES row, Table 2), not part of the method
// itself: it gives the optimum that the block/pixel recursive search is
// judged against (search points and PSNR).
//
// One CTA per MB.  The reference window every vector of V can reach is
// staged in shared memory, at half-pel as the four MPEG-4 planes (integer,
// horizontal, vertical and diagonal half samples, rounding control 0), each
// row padded to whole 32-bit words, the planes 16 banks apart modulo 32 (the
// lanes of a warp read two planes at once: odd and even dx); each thread
// keeps the current block in registers.  Each thread takes whole positions:
// per block row it reads 5 aligned words of the plane once, shifts them into
// the 4 words under the block and adds __vsadu4 against the current row --
// 16 x 4 packed operations per position.
// The CTA's minimum is taken over (SAD << 32 | raster index), so ties go to
// the first position in raster order exactly as in the definition.
#include <cuda_runtime.h>
#include <stdint.h>

#include "sme_internal.h"

namespace sme {
namespace {

constexpr int kEsThreads = 256;

struct EsGeom {
    int W, H, S, h, rd, M, MBW;
};

// Words per plane: wh rows of pw words, rounded up to 16 modulo 32 words.
__host__ __device__ __forceinline__ int es_plane_words(int wh, int pw)
{
    const int n = wh * pw;
    return n + ((16 - n % 32) + 32) % 32;
}

__global__ void __launch_bounds__(kEsThreads) es_kernel(const uint8_t* __restrict__ luma, EsGeom g, sme_mv* mv,
                                                       uint32_t* sad_out)
{
    extern __shared__ __align__(16) uint32_t es_smem[];
    const int pair = blockIdx.y, mb = blockIdx.x;
    const int u = mb % g.MBW, v = mb / g.MBW, X0 = 16 * u, Y0 = 16 * v;
    const int h = g.h, S = g.S;
    const size_t FS = (size_t)g.W * g.H;
    const uint8_t* ref = luma + (size_t)pair * FS;
    const uint8_t* cur = luma + (size_t)(pair + g.rd) * FS;
    // V in MV units (Table 1's convention: displaced block inside the frame)
    const int lox = max(-S * h, -X0 * h), hix = min(S * h, (g.W - 16 - X0) * h);
    const int loy = max(-S * h, -Y0 * h), hiy = min(S * h, (g.H - 16 - Y0) * h);
    // Window of integer pixels every vector of V reads: the displaced block
    // at d = (q + f/2) px covers pixels X0 + q .. X0 + 15 + q + f, so x runs
    // from X0 + floor(lox / h) to X0 + 15 + ceil(hix / h) (inside the frame by
    // the definition of V); likewise for y.
    const int qlx = lox >= 0 ? lox / h : -((-lox + h - 1) / h), qly = loy >= 0 ? loy / h : -((-loy + h - 1) / h);
    const int wx0 = X0 + qlx, wy0 = Y0 + qly;
    const int ww = 16 + (hix + h - 1) / h - qlx, wh = 16 + (hiy + h - 1) / h - qly;
    const int pw = (ww + 3) / 4 + 2;  // words per plane row (+1 for unaligned reads, +1 slack)
    const int planes = h * h, pstride = es_plane_words(wh, pw);
    uint32_t* cur_s = es_smem;                 // 16 rows x 4 words
    uint32_t* win = es_smem + 64;              // planes x pstride words (rows of pw words)
    const int tid = threadIdx.x;
    // current block
    if (tid < 64) {
        const int r = tid >> 2, c = (tid & 3) * 4;
        cur_s[tid] = *reinterpret_cast<const uint32_t*>(cur + (size_t)(Y0 + r) * g.W + X0 + c);
    }
    // planes: byte (r, c) of plane (fy, fx) = sample at (wx0 + c + fx/2, wy0 + r + fy/2)
    uint8_t* winb = reinterpret_cast<uint8_t*>(win);
    for (int i = tid; i < planes * wh * pw * 4; i += blockDim.x) {
        const int p = i / (wh * pw * 4), rem = i - p * wh * pw * 4, r = rem / (pw * 4), c = rem - r * (pw * 4);
        uint8_t* dst = winb + (size_t)p * pstride * 4 + rem;
        const int fy = p >> 1, fx = p & 1;
        int val = 0;
        const int x = wx0 + c, y = wy0 + r;
        if (c < ww && x + fx < g.W && y + fy < g.H && x >= 0 && y >= 0) {
            const uint8_t* q = ref + (size_t)y * g.W + x;
            const int a = q[0];
            if (!fx && !fy) val = a;
            else if (fx && !fy) val = (a + q[1] + 1) >> 1;
            else if (!fx && fy) val = (a + q[g.W] + 1) >> 1;
            else val = (a + q[1] + q[g.W] + q[g.W + 1] + 2) >> 2;
        }
        *dst = (uint8_t)val;
    }
    __syncthreads();
    uint32_t cw[64];  // the current block, row-major words
#pragma unroll
    for (int i = 0; i < 64; ++i) cw[i] = cur_s[i];

    const int nx = hix - lox + 1, n = nx * (hiy - loy + 1);
    unsigned long long best = ~0ull;
    for (int idx = tid; idx < n; idx += blockDim.x) {
        const int dy = loy + idx / nx, dx = lox + idx % nx;
        // integer and half parts of the displaced block origin, in window coordinates
        const int fx = h == 2 ? (dx & 1) : 0, fy = h == 2 ? (dy & 1) : 0;
        const int qx = (dx - fx) / h, qy = (dy - fy) / h;
        const int c0 = X0 + qx - wx0, r0 = Y0 + qy - wy0;
        const uint32_t* plane = win + (size_t)(fy * 2 + fx) * pstride;
        const int w0 = c0 >> 2, sh = (c0 & 3) * 8;
        unsigned s = 0;
#pragma unroll
        for (int r = 0; r < 16; ++r) {
            const uint32_t* row = plane + (size_t)(r0 + r) * pw + w0;
            const unsigned a0 = row[0], a1 = row[1], a2 = row[2], a3 = row[3], a4 = row[4];
            s = __vsadu4(__funnelshift_r(a0, a1, sh), cw[4 * r]) + s;
            s = __vsadu4(__funnelshift_r(a1, a2, sh), cw[4 * r + 1]) + s;
            s = __vsadu4(__funnelshift_r(a2, a3, sh), cw[4 * r + 2]) + s;
            s = __vsadu4(__funnelshift_r(a3, a4, sh), cw[4 * r + 3]) + s;
        }
        const unsigned long long key = ((unsigned long long)s << 32) | (unsigned)idx;
        best = key < best ? key : best;
    }
    // CTA minimum of (SAD, raster index)
    for (int o = 16; o; o >>= 1) {
        const unsigned long long other = __shfl_xor_sync(0xffffffffu, best, o);
        best = other < best ? other : best;
    }
    __shared__ unsigned long long s_best[kEsThreads / 32];
    if ((tid & 31) == 0) s_best[tid >> 5] = best;
    __syncthreads();
    if (tid == 0) {
        unsigned long long b = s_best[0];
        for (int w = 1; w < (int)(blockDim.x >> 5); ++w) b = s_best[w] < b ? s_best[w] : b;
        const int idx = (int)(unsigned)b;
        const size_t o = (size_t)pair * g.M + mb;
        mv[o] = sme_mv{(int16_t)(lox + idx % nx), (int16_t)(loy + idx / nx)};
        if (sad_out) sad_out[o] = (uint32_t)(b >> 32);
    }
}

// The packed-SAD operation mix of the integer roofline (per 32-bit word: a
// funnel-shift alignment, a __vsadu4 absolute difference, an add), on 8
// register-resident chains per thread; chain k aligns its own value with its
// neighbour's, so nothing is loop-invariant.  Per step 24 operations.
__global__ void __launch_bounds__(256) packed_sad_rate_kernel(int iters, uint32_t* out)
{
    const uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
    uint32_t acc[8], z[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        acc[k] = t * 0x9E3779B9u + (uint32_t)k * 0x85EBCA6Bu;
        z[k] = t ^ ((uint32_t)k * 0x27D4EB2Du);
    }
    const int sh = (int)(t & 3u) * 8;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int k = 0; k < 8; ++k) acc[k] = __vsadu4(__funnelshift_r(acc[k], acc[(k + 1) & 7], sh), z[k]) + acc[k];
    }
    uint32_t r = 0;
#pragma unroll
    for (int k = 0; k < 8; ++k) r ^= acc[k];
    out[t] = r;
}

}  // namespace

cudaError_t launch_packed_sad_rate(int ctas_per_sm, int iters, uint32_t* out, cudaStream_t s, int* grid)
{
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    *grid = sms * ctas_per_sm;
    packed_sad_rate_kernel<<<*grid, 256, 0, s>>>(iters, out);
    return cudaGetLastError();
}

size_t es_smem_bytes(int S, int h)
{
    const int ww = 16 + 2 * S, pw = (ww + 3) / 4 + 2;  // the widest window: |d| <= S px both ways
    return (size_t)(64 + h * h * es_plane_words(ww, pw)) * 4;
}

cudaError_t launch_es(const uint8_t* luma, int W, int H, int S, int h, int rd, int pairs, sme_mv* mv, uint32_t* sad,
                      cudaStream_t s)
{
    EsGeom g{W, H, S, h, rd, (W / 16) * (H / 16), W / 16};
    const size_t smem = es_smem_bytes(S, h);
    if (smem > 48 * 1024) {
        const cudaError_t e = cudaFuncSetAttribute(es_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    es_kernel<<<dim3(g.M, pairs), kEsThreads, smem, s>>>(luma, g, mv, sad);
    return cudaGetLastError();
}

}  // namespace sme
