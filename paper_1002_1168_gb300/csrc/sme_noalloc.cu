// sme_estimate_sequence_noalloc: the whole-sequence estimate for callers that
// cannot allocate device memory.
//
// Some callers cannot call cudaMalloc: code that runs inside another
// framework's memory pool or a custom allocator that must own every device
// allocation, code that runs where allocation would synchronise the device
// at the wrong moment, or embedded/real-time users that forbid allocation
// after start-up.  The regular entry points keep their scratch (packed alpha,
// MB classes, ready words, wavefront schedule, status words) in buffers the
// context allocates; this entry point keeps the same scratch in one
// fixed-size array in device memory instead, so it needs no context and
// allocates nothing.  The caller still passes every input and output.
//
// The array is a file-scope __device__ variable of kScratchBytes: every GPU
// that loads the library holds it until the process exits.  Host code may not
// use the array's name as a device address (on the host it is only a
// stand-in), so the first call on each device looks the address up with
// cudaGetSymbolAddress (with that device current) and caches it; that first
// call should therefore come before any stream capture.  The cached address
// belongs to the device's primary context: a caller that resets the device
// (cudaDeviceReset) must not call this entry point again in the same process,
// because the array may then sit at another address.  All calls share the
// array and it keeps the previous call's contents: every part that must start
// at zero is cleared here, and calls that overlap on the GPU (for example on
// two streams at once) race on it.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <mutex>

#include "sme_internal.h"

namespace sme {
namespace {

constexpr size_t kScratchBytes = 4u << 20;  // 4 MiB
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

std::mutex g_setup_lock;
void* g_scratch_addr[kMaxDevices];
int g_sms[kMaxDevices];

size_t round256(size_t v) { return (v + 255) & ~(size_t)255; }

int check(const sme_params* p)
{
    if (!p) return SME_ERR_ARG;
    if (p->width <= 0 || p->height <= 0 || p->width % 16 || p->height % 16 || p->width > kMaxDim ||
        p->height > kMaxDim)
        return SME_ERR_SIZE;
    if (p->search_range < 1 || p->search_range > kMaxSearch) return SME_ERR_ARG;
    if (p->subpel != 1 && p->subpel != 2) return SME_ERR_ARG;
    if (!(p->theta > 0.0f) || !isfinite(p->theta)) return SME_ERR_ARG;
    if (!(p->epsilon > 0.0f) || !(p->epsilon <= 4.0f)) return SME_ERR_ARG;
    if (p->max_iters < 0 || p->max_iters > kMaxIters) return SME_ERR_ARG;
    if (p->ref_distance < 1) return SME_ERR_ARG;
    return SME_OK;
}

// Device-side wavefront order (the regular path builds the same order on the
// host): MBs sorted by step t = u + 2v + k, then by pair k, then by row v.
// One CTA: count the MBs of every step, prefix-sum, then list them.
__global__ void noalloc_schedule_kernel(const Geom g, int P, int T, int* offs, int* sched)
{
    for (int t = threadIdx.x; t < T; t += blockDim.x) {
        int c = 0;
        for (int k = 0; k < P && k <= t; ++k) {
            const int r = t - k, lo = r - g.MBW + 1;
            const int vmin = lo > 0 ? (lo + 1) / 2 : 0, vmax = min(g.MBH - 1, r / 2);
            if (vmax >= vmin) c += vmax - vmin + 1;
        }
        offs[t + 1] = c;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        offs[0] = 0;
        for (int t = 0; t < T; ++t) offs[t + 1] += offs[t];
    }
    __syncthreads();
    for (int t = threadIdx.x; t < T; t += blockDim.x) {
        int n = offs[t];
        for (int k = 0; k < P && k <= t; ++k) {
            const int r = t - k, lo = r - g.MBW + 1;
            const int vmin = lo > 0 ? (lo + 1) / 2 : 0, vmax = min(g.MBH - 1, r / 2);
            for (int v = vmin; v <= vmax; ++v) sched[n++] = k * g.M + v * g.MBW + (r - 2 * v);
        }
    }
}

// Looks up the array's device address once per device (with that device
// current) and caches it together with the SM count.
int setup(int dev, void** addr, int* sms)
{
    if (dev < 0 || dev >= kMaxDevices) return SME_ERR_CUDA;
    std::lock_guard<std::mutex> lk(g_setup_lock);
    if (!g_scratch_addr[dev]) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_scratch) != cudaSuccess || !p) {
            cudaGetLastError();
            return SME_ERR_CUDA;
        }
        int n = 0;
        if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n < 1) {
            cudaGetLastError();
            return SME_ERR_CUDA;
        }
        g_sms[dev] = n;
        g_scratch_addr[dev] = p;
    }
    *addr = g_scratch_addr[dev];
    *sms = g_sms[dev];
    return SME_OK;
}

}  // namespace
}  // namespace sme

using namespace sme;

extern "C" int sme_estimate_sequence_noalloc(const sme_params* p, const uint8_t* luma, const uint8_t* alpha,
                                             int n_frames, const sme_mv* temporal_in, const float* seed,
                                             const sme_outputs* out, void* cuda_stream)
{
    int rc = check(p);
    if (rc) return rc;
    if (!luma || !alpha || !out || !out->mv) return SME_ERR_ARG;
    if (((uintptr_t)luma & 15u) || ((uintptr_t)alpha & 15u)) return SME_ERR_ARG;
    if (seed && p->max_iters > kMaxSeededIters) return SME_ERR_ARG;
    const int rd = p->ref_distance;
    if (n_frames <= rd) return SME_ERR_ARG;

    Geom g;
    g.W = p->width;
    g.H = p->height;
    g.MBW = p->width / 16;
    g.MBH = p->height / 16;
    g.M = g.MBW * g.MBH;
    g.Wp = (((p->width + 31) / 32 + 1) + 3) & ~3;
    Method mth;
    mth.S = p->search_range;
    mth.h = p->subpel;
    mth.K = p->max_iters;
    mth.theta = p->theta;
    mth.eps = p->epsilon;
    mth.tt = 0;
    const int F = n_frames, P = n_frames - rd;
    const int T = (g.MBW - 1) + 2 * (g.MBH - 1) + P;  // wavefront steps
    const size_t PM = (size_t)P * g.M;

    // Layout of the fixed scratch; anything larger is rejected.
    const size_t o_status = 0;
    const size_t o_desc = o_status + round256(sizeof(DevStatus));
    const size_t o_packed = o_desc + round256(sizeof(SeqDesc));
    const size_t o_cls = o_packed + round256((size_t)F * g.H * g.Wp * sizeof(uint32_t));
    const size_t o_ready = o_cls + round256((size_t)F * g.M);
    const size_t o_sched = o_ready + round256(PM * sizeof(unsigned long long));
    const size_t o_offs = o_sched + round256(PM * sizeof(int));
    const size_t need = o_offs + round256(((size_t)T + 1) * sizeof(int));
    if (need > kScratchBytes) return SME_ERR_SCRATCH;

    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return SME_ERR_CUDA;
    // The array used is the current device's: a stream of another device
    // would run the kernels there against this device's address.
    int sdev = -1;
    if (cudaStreamGetDevice((cudaStream_t)cuda_stream, &sdev) != cudaSuccess) {
        cudaGetLastError();
        return SME_ERR_ARG;
    }
    if (sdev != dev) return SME_ERR_ARG;
    void* base = nullptr;
    if ((rc = setup(dev, &base, &sms))) return rc;
    int per_sm = 0;
    if (me_occupancy(mth.S, &per_sm) != cudaSuccess || per_sm < 1) return SME_ERR_CUDA;

    unsigned char* s = (unsigned char*)base;
    DevStatus* status = (DevStatus*)(s + o_status);
    SeqDesc* desc = (SeqDesc*)(s + o_desc);
    uint32_t* packed = (uint32_t*)(s + o_packed);
    uint8_t* cls = s + o_cls;
    unsigned long long* ready = (unsigned long long*)(s + o_ready);
    int* sched = (int*)(s + o_sched);
    int* offs = (int*)(s + o_offs);
    const cudaStream_t st = (cudaStream_t)cuda_stream;

    // Clear what must start at zero: status words and ready stamps.
    if (cudaMemsetAsync(status, 0, sizeof(DevStatus), st) != cudaSuccess ||
        cudaMemsetAsync(ready, 0, PM * sizeof(unsigned long long), st) != cudaSuccess)
        return SME_ERR_CUDA;
    noalloc_schedule_kernel<<<1, 256, 0, st>>>(g, P, T, offs, sched);
    if (cudaGetLastError() != cudaSuccess) return SME_ERR_CUDA;

    SeqDesc d{};
    d.luma = luma;
    d.alpha = alpha;
    d.packed_w = packed;
    d.cls_w = cls;
    d.packed = packed;
    d.cls = cls;
    d.temporal_in = temporal_in;
    d.seed = seed;
    d.mv = out->mv;
    d.cost = out->cost;
    d.disp = out->disp;
    d.iters = out->iters;
    d.npos = out->npos;
    d.out_cls = out->mb_class;
    d.sse_mb = out->sse_mb;
    d.sse = out->sse;
    d.pred = out->pred;
    d.W = g.W;
    d.H = g.H;
    d.MBW = g.MBW;
    d.MBH = g.MBH;
    d.M = g.M;
    d.Wp = g.Wp;
    d.P = P;
    d.rd = rd;
    d.F = F;
    d.gid_base = 0;

    ClassifyArgs ca{};
    ca.alpha = alpha;
    ca.n_frames = F;
    ca.cls = cls;
    ca.packed = packed;
    ca.status = status;
    ca.sse = out->sse;
    ca.n_sse = P;
    ca.desc_out = desc;
    ca.desc = d;
    if (launch_classify(g, ca, st) != cudaSuccess) return SME_ERR_CUDA;

    MeArgs a{};
    a.seqs = desc;
    a.sched = sched;
    a.sched_seq = nullptr;
    a.ready = ready;
    a.status = status;
    a.m = mth;
    a.total = (int)PM;
    a.fault_ticket = -1;
    a.speculate = 1;
    a.timeout_ns = kDefaultTimeoutNs;
    const long long cap = (long long)sms * per_sm;
    const long long want = ((long long)PM + kMeWarps - 1) / kMeWarps;
    const int grid = (int)(cap < want ? cap : want);
    if (launch_me(mth, a, grid, st) != cudaSuccess) return SME_ERR_CUDA;

    // Report a device-side failure of this call (synchronises the stream).
    int err = 0;
    if (cudaMemcpyAsync(&err, &status->err, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
        return SME_ERR_CUDA;
    return err ? err : SME_OK;
}
