// Internal declarations shared by the C-ABI layer (sme_api.cu) and the
// kernels (sme_kernels.cu).  Not part of the public interface.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/sme.h"

namespace sme {

constexpr int kMaxSearch = 64;
constexpr int kMaxIters = 16;
constexpr int kMaxDim = 8192;
// Evaluated-position log per MB: 5 block-recursive candidates plus, per
// pixel-recursive iteration, one proposal and eight neighbours.
constexpr int kMaxLog = 5 + 9 * kMaxIters;
constexpr long long kDefaultTimeoutNs = 1000000000LL;

// Device status words (ctx scratch).  `err` is sticky until read by
// sme_synchronize; `abort` and `ticket` are reset by the classify kernel at
// the start of every estimate.
struct DevStatus {
    unsigned ticket;
    unsigned abort;
    int err;
    unsigned pad;
};

// Geometry + method parameters as the kernels see them.
struct Geom {
    int W, H, M, MBW, MBH, Wp;  // Wp = packed alpha words per row
    int S, h, K;
    float theta, eps;
};

struct ClassifyArgs {
    const uint8_t* alpha;
    int n_frames;
    uint8_t* cls;        // [F][M]
    uint32_t* packed;    // [F][H][Wp]
    DevStatus* status;   // reset here when non-null
    unsigned long long* sse;  // [P] zeroed here when non-null
    int n_sse;
};

struct MeArgs {
    const uint8_t* luma;
    const uint32_t* packed;
    const uint8_t* cls;       // [F][M]
    const sme_mv* temporal_in;
    const float* seed;        // [P][M][2]
    sme_mv* mv;               // [P][M]
    uint32_t* cost;
    float* disp;
    uint8_t* iters;
    uint8_t* npos;
    uint8_t* out_cls;
    uint32_t* sse_mb;
    unsigned long long* sse;
    uint8_t* pred;
    const int* sched;         // ticket -> k*M + mb, ordered by wavefront step
    unsigned* ready;          // [P][M] epoch stamps
    DevStatus* status;
    unsigned epoch;
    int P, rd, total;
    int fault_ticket;
    long long timeout_ns;
};

struct CompArgs {
    const uint8_t* ref;
    const uint8_t* cur;
    const sme_mv* mv;
    uint8_t* pred;
    unsigned long long* sse;
    DevStatus* status;
};

struct QueryArgs {
    const uint8_t* ref;
    const uint8_t* cur;
    const uint32_t* pref;   // packed alpha of ref (may be null)
    const uint32_t* pcur;
    const int32_t* q;
    int n;
    uint32_t* tsad;
    uint32_t* ssad;
    float* delta;
    DevStatus* status;
};

// Launchers (sme_kernels.cu).  Return cudaSuccess or the launch error.
cudaError_t launch_classify(const Geom& g, const ClassifyArgs& a, cudaStream_t s);
cudaError_t launch_me(const Geom& g, const MeArgs& a, int grid, cudaStream_t s);
cudaError_t launch_compensate(const Geom& g, const CompArgs& a, cudaStream_t s);
cudaError_t launch_queries(const Geom& g, const QueryArgs& a, cudaStream_t s);
// Resident CTAs per SM of the persistent ME kernel for this geometry.
cudaError_t me_occupancy(const Geom& g, int* blocks_per_sm);
size_t me_smem_bytes(const Geom& g);

}  // namespace sme
