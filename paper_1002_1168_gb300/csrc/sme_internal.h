// Internal declarations shared by the C-ABI layer (sme_api.cu, sme_noalloc.cu)
// and the kernels (sme_kernels.cu).  Not part of the public interface.
#pragma once

#include <cuda.h>  // CUtensorMap (the layout only; no driver library is linked)
#include <cudaTypedefs.h>
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
// With seeds, an opaque MB whose seed wins runs two pixel-recursive searches
// into the same log (the seeded one and its plain fallback): 5 + 2 * 9 * K
// entries.  Seeds are therefore accepted only up to this iteration cap, at
// which both searches fit the log exactly.
constexpr int kMaxSeededIters = 8;
static_assert(5 + 2 * 9 * kMaxSeededIters <= kMaxLog, "seeded searches overrun the position log");
// Four vectors per MB: one log per 8x8 block, the 4 MB candidates plus the
// block's own steps.
static_assert(4 + 9 * kMaxIters <= kMaxLog, "block searches overrun the position log");
// The distinct-position count is stored in a byte and carried in the top 8
// bits of one 32-bit warp reduction: it must stay below 256.
static_assert(kMaxLog < 256, "distinct-position count does not fit its byte");
constexpr long long kDefaultTimeoutNs = 1000000000LL;
constexpr int kMeWarps = 8;        // warps (one MB each) per CTA of the per-MB ME kernel
// Warps per CTA of the sparse schedule's search build for `min_blocks` CTAs
// per SM: 4 for the five-CTA build, else kMeWarps.
__host__ __device__ constexpr int sparse_cta_warps(int min_blocks) { return min_blocks == 5 ? 4 : kMeWarps; }
constexpr int kClusterWarps = 12;  // warps (one MB each) per CTA of the cluster schedule
constexpr int kPairWarpsMax = 16;  // warps (MB rows) per CTA of the per-pair ME kernel

// ME schedules: one warp per MB with tickets in wavefront order, or one CTA
// per frame pair with one warp per MB row.
// kSchedSparse: a streaming pass finishes the transparent MBs, the per-MB
// search runs over a wavefront-ordered list of the others.
enum Schedule { kSchedAuto = 0, kSchedMB = 1, kSchedPair = 2, kSchedCluster = 3, kSchedSparse = 4 };
constexpr int kGroupMax = 64;     // VOPs sharing one luma in one streaming pass of the sparse schedule

// Device status words (scratch).  `err` is sticky until read by
// sme_synchronize; `abort` and `ticket` are reset by the classify kernel at
// the start of every estimate.
struct DevStatus {
    unsigned ticket;
    unsigned abort;
    int err;
    unsigned epoch;  // stamp of the current launch's ready words, bumped by classify
};

// Method parameters shared by every sequence of a launch.
struct Method {
    int S, h, K;
    float theta, eps;
    int tt;  // boundary MBs: T judged by texture against the shape winner of the others (Sec. 3.1 variant)
};

// Per-frame geometry.
struct Geom {
    int W, H, M, MBW, MBH, Wp;  // Wp = packed alpha words per row
};

// One sequence (one VOP) of an ME launch.  Global MB id of MB `mb` of pair k
// = gid_base + k*M + mb; ready words are indexed by global MB id.
struct SeqDesc {
    const uint8_t* luma;      // [F][H][W]
    const uint8_t* alpha;     // [F][H][W]
    uint32_t* packed_w;       // [F][H][Wp] (written by the classify launch)
    uint8_t* cls_w;           // [F][M]     (written by the classify launch)
    const uint32_t* packed;   // [F][H][Wp]
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
    unsigned long long* sse;  // [P]
    uint8_t* pred;
    int W, H, MBW, MBH, M, Wp, P, rd, F;
    int gid_base;
};

// Counters of the sparse schedule's list (scratch).
struct SparseCounters {
    unsigned total;   // non-transparent MBs listed (written by the scan launch)
    unsigned ticket;  // next list entry of the search launch
};

struct ClassifyArgs {
    const uint8_t* alpha;
    const uint8_t* const* frames;  // when non-null: frame f is frames[f] (NULL: an empty plane)
    int n_frames;
    uint8_t* cls;        // [F][M]
    uint32_t* packed;    // [F][H][Wp]
    DevStatus* status;   // reset here when non-null
    unsigned long long* sse;  // [P] zeroed here when non-null
    int n_sse;
    SeqDesc* desc_out;   // when non-null, block (0,0) stores `desc` there
    SeqDesc desc;
};

// Classification of many sequences in one launch: block (x, g) handles MB
// row x of global frame g = (sequence fseq[g], frame ffrm[g]).
struct ClassifyBatchArgs {
    const SeqDesc* seqs;
    const int* fseq;
    const int* ffrm;
    DevStatus* status;
};

// The sparse schedule's preparation launches (reset, streaming pass, scan,
// scatter) over `nseq` sequences grouped by shared luma.
struct SparseArgs {
    SeqDesc* seqs;             // [nseq] (device)
    SeqDesc* desc_dst;         // single-sequence path: where the reset launch stores the descriptor
    int nseq;
    const int* grp_first;      // [ngrp + 1]: group g = grp_members[grp_first[g] .. grp_first[g + 1]) (<= kGroupMax)
    const int* grp_members;    // sequence indices; the members of a group share luma, size and frames
    const int* gf_group;       // per (group, frame) block row of the streaming pass: its group
    const int* gf_frame;       //   and frame
    int n_gf, max_mbh;
    const long long* row_base; // [nseq]: rows (frame, MB row) of sequence q start here in rowcnt
    long long total_rows;
    unsigned* rowcnt;          // non-transparent MBs per row (0 for frames < ref_distance)
    int* first_step;           // [nseq]: first wavefront step with a non-transparent MB of each sequence
    unsigned* hist;            // [8 * (steps + 1)]: MBs per list key (one 32-byte sector each)
    unsigned* cursor;          // [8 * steps]: scatter cursor of each key
    int steps;                 // list keys (steps, or pair_keys * the largest pair count)
    int pair_keys;             // > 0: pair rounds -- key = k * pair_keys + u + 2v (pair k's MBs contiguous)
    unsigned* round_ticket;    // [rounds]: next entry of each pair round's search launch
    int rounds;
    int* list;                 // global MB ids of the non-transparent MBs, by step
    SparseCounters* ctr;
    DevStatus* status;
};

struct MeArgs {
    const SeqDesc* seqs;      // [nseq] in device memory
    const int* sched;         // per-MB schedule: ticket -> global MB id, by wavefront step
    const int* sched_seq;     // per-MB schedule: ticket -> sequence index (NULL: sequence 0)
    const int* unit_seq;      // per-pair schedule: ticket -> sequence (NULL: sequence 0)
    const int* unit_pair;     // per-pair schedule: ticket -> pair (NULL: pair = ticket)
    const CUtensorMap* tmaps; // per-pair schedule: luma tensor map per sequence (NULL: kernel parameter)
    int total_units;
    int mbw_max;
    unsigned long long* ready;  // [total] (epoch << 32) | packed vector (four-vector mode: block 0)
    unsigned long long* ready_a;   // four-vector mode, per-MB schedule: block 1 (for A)
    unsigned long long* ready_bc;  // four-vector mode, per-MB schedule: block 2 (for B, C)
    DevStatus* status;
    Method m;
    int total;
    int fault_ticket;
    int speculate;
    int pair_direct;          // per-pair schedule: transparent MBs skip the TMA staging
    int four_mv;              // per-pair schedule: four vectors per MB (8x8 blocks), outputs [P][M][4]
    long long timeout_ns;
    // cluster schedule (one sequence per cluster)
    const int* cl_items;      // [cluster][cl_cap] global MB ids, each CTA's list in wavefront order
    const int* cl_count;      // [cluster] items per CTA
    const int* cl_consumers;  // [total][4] consumer slot of each MB in the roles A, B, C, T (or -1)
    int cl_cap;
    // sparse schedule
    const int* list;          // global MB ids by wavefront step (sparse_scatter_kernel)
    const int* seq_base;      // [nseq] first global MB id of each sequence (ascending)
    int nseq;
    SparseCounters* ctr;
    // pair rounds: the launch searches pair `round` of every sequence only:
    // list entries [offs[8 * round * pair_keys], offs[8 * (round + 1) * pair_keys])
    int round;                // -1: the whole list
    int pair_keys, rounds;
    const unsigned* offs;     // exclusive list offset of each key (one 32-byte sector each)
    unsigned* round_ticket;   // [rounds]
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
cudaError_t launch_classify_batch(const ClassifyBatchArgs& a, int max_mbh, int total_frames, cudaStream_t s);
cudaError_t launch_me(const Method& m, const MeArgs& a, int grid, cudaStream_t s);
// Per-MB schedule in the four-vector mode (three ready arrays in MeArgs).
cudaError_t launch_me4(const Method& m, const MeArgs& a, int grid, cudaStream_t s);
cudaError_t me4_occupancy(int S, int* blocks_per_sm);
// `maps` points to 4 CUtensorMaps (128-byte aligned): luma window box, current
// block box, packed-alpha reference strip, packed-alpha current BAB.
cudaError_t launch_me_pair(const Method& m, const MeArgs& a, const void* maps, int nwarps, int grid, cudaStream_t s);
cudaError_t me_pair_occupancy(int S, int nwarps, int mbw_max, bool direct, bool four_mv, int* blocks_per_sm);
size_t me_pair_smem_bytes(int S, int nwarps, int mbw_max, bool four_mv = false);
// Boxes (elements wide, rows high) of the four TMA copies of the per-pair
// kernel: luma window, current block, packed-alpha reference strip (u32),
// packed-alpha current BAB (u32).
void pair_boxes(int S, unsigned (&box)[4][2]);
// Cluster schedule: dynamic shared memory of one CTA of `warps` warps for
// `cap` items per CTA; how many clusters of `cluster` such CTAs can be
// resident at once (0: none).
size_t me_cluster_smem_bytes(int S, int cap, int warps);
int me_cluster_fits(int S, int cap, int cluster, int warps);
cudaError_t launch_me_cluster(const Method& m, const MeArgs& a, int cluster, int warps, int helpers, cudaStream_t s);
cudaError_t launch_compensate(const Geom& g, const Method& m, const CompArgs& a, cudaStream_t s);
// Sparse schedule: preparation (desc: single-sequence descriptor stored by the
// reset launch, or NULL when a.seqs already holds the descriptors) and the search.
cudaError_t launch_sparse_prep(const SparseArgs& a, const SeqDesc* desc, cudaStream_t s);
// min_blocks selects the register budget of the search kernel (1, 2 or 3 CTAs per SM).
cudaError_t me_sparse_occupancy(int S, int min_blocks, int* blocks_per_sm, bool variants);
cudaError_t launch_me_sparse(const Method& m, const MeArgs& a, int grid, int min_blocks, cudaStream_t s);

// Exhaustive search over V for every MB of `pairs` frame pairs (sme_es.cu).
size_t es_smem_bytes(int S, int h);
cudaError_t launch_host_copy(void* dst, const void* src, size_t bytes, int num_sms, cudaStream_t s);
cudaError_t launch_packed_sad_rate(int ctas_per_sm, int iters, uint32_t* out, cudaStream_t s, int* grid);
cudaError_t launch_es(const uint8_t* luma, int W, int H, int S, int h, int rd, int pairs, sme_mv* mv, uint32_t* sad,
                      cudaStream_t s);

// cuTensorMapEncodeTiled of the installed driver (NULL if unavailable).
PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder();
cudaError_t launch_queries(const Geom& g, const Method& m, const QueryArgs& a, cudaStream_t s);
// Resident CTAs per SM of the persistent ME kernel for search range S.
cudaError_t me_occupancy(int S, int* blocks_per_sm, bool variants = false);
size_t me_smem_bytes(int S);

}  // namespace sme
