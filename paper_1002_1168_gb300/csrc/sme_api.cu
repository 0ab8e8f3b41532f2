// C ABI of the shape-adaptive motion estimation library (declared in
// include/sme.h): argument checks, context-owned device scratch, the
// wavefront schedule, and the launch sequence of each call.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <mutex>
#include <new>
#include <vector>

#include "sme_internal.h"

using namespace sme;

// cuTensorMapEncodeTiled from the driver, looked up once through the runtime
// (no link-time dependency on the driver library).
PFN_cuTensorMapEncodeTiled_v12000 sme::tensor_map_encoder()
{
    static std::once_flag once;
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    std::call_once(once, [] {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (PFN_cuTensorMapEncodeTiled_v12000)p;
        cudaGetLastError();
    });
    return fn;
}

namespace {

struct DevBuf {
    void* p = nullptr;
    size_t bytes = 0;
};

// Scratch of the sparse schedule (SME_SCHED_SPARSE): the luma groups of the
// streaming pass, the per-row counts, the per-step offsets and cursors, the
// list of non-transparent MBs and its counters.
struct SparseScratch {
    DevBuf grp_first, grp_members, gf_group, gf_frame, row_base, rowcnt, hist, cursor, list, ctr, seq_base, first,
        round_ticket;
    int n_gf = 0, max_mbh = 0, steps = 0, nseq = 0;
    int pair_keys = 0, rounds = 0;  // pair rounds: keys per pair (0: off), pairs of the longest sequence
    long long total_rows = 0;
    const void* key = nullptr;  // single-sequence path: the set-up is reused while (luma, F) stay the same
    int key_f = -1;
};

}  // namespace

struct sme_ctx {
    sme_params prm;
    Geom g;
    Method m;
    cudaStream_t stream = nullptr;
    int device = 0, num_sms = 0, me_blocks_per_sm = 0, smem_optin = 0;
    DevStatus* status = nullptr;
    DevBuf packed, cls, ready, sched, desc, qpacked, qcls;
    std::vector<int> sched_host;
    int sched_P = -1;
    int schedule = kSchedAuto, pair_warps = 0, mb_ctas_per_sm = 0, speculate = 1, cluster = 0, pair_direct = 1;
    int four_mv = 0;
    // cluster schedule: per-CTA item lists and consumer slots (rebuilt when P or the size changes)
    DevBuf cl_items, cl_count, cl_cons;
    int cl_P = -1, cl_C = 0, cl_cap = 0, cl_warps = 0, cl_resident = 0;
    int fault_ticket = -1;
    long long timeout_ns = kDefaultTimeoutNs;
    // pair interface
    DevBuf pair_luma, pair_alpha, temporal, last_mv, last_sse, seed_field;
    bool have_ref = false, have_cur = false, have_temporal = false, have_result = false, have_seed = false;
    // stage timing: three events per recorded call
    std::vector<cudaEvent_t> prof_ev;
    int prof_max = 0, prof_n = 0;
    // host-buffer interface
    DevBuf h_luma, h_alpha, h_tmp, h_seed, h_mv, h_cost, h_disp, h_iters, h_npos, h_cls, h_ssemb,
        h_sse, h_pred;
    int* h_err = nullptr;  // pinned host copy of the device error word (sme_synchronize)
    // host-buffer interface: the luma copy runs on a second stream while the
    // classification reads a pinned alpha in place
    cudaStream_t copy_stream = nullptr;
    cudaEvent_t copy_go = nullptr, copy_done = nullptr;
    SparseScratch sp;
};

namespace {

int cuda_status(cudaError_t e) { return e == cudaSuccess ? SME_OK : SME_ERR_CUDA; }

int ensure(DevBuf& b, size_t bytes, bool zero = false, cudaStream_t s = nullptr)
{
    if (bytes == 0) bytes = 16;
    if (b.bytes >= bytes) return SME_OK;
    if (b.p) cudaFree(b.p);
    b.p = nullptr;
    b.bytes = 0;
    if (cudaMalloc(&b.p, bytes) != cudaSuccess) {
        cudaGetLastError();
        return SME_ERR_NOMEM;
    }
    b.bytes = bytes;
    if (zero && cudaMemsetAsync(b.p, 0, bytes, s) != cudaSuccess) return SME_ERR_CUDA;
    return SME_OK;
}

void release(DevBuf& b)
{
    if (b.p) cudaFree(b.p);
    b.p = nullptr;
    b.bytes = 0;
}

bool aligned16(const void* p) { return ((uintptr_t)p & 15u) == 0; }

void release_sparse(SparseScratch& sp)
{
    DevBuf* bufs[] = {&sp.grp_first, &sp.grp_members, &sp.gf_group, &sp.gf_frame, &sp.row_base, &sp.rowcnt,
                      &sp.hist,      &sp.cursor,      &sp.list,     &sp.ctr,      &sp.seq_base, &sp.first,
                      &sp.round_ticket};
    for (DevBuf* b : bufs) release(*b);
    sp = SparseScratch{};
}

template <class T>
int upload(DevBuf& b, const std::vector<T>& v, cudaStream_t s)
{
    int rc = ensure(b, v.size() * sizeof(T));
    if (rc) return rc;
    return cudaMemcpyAsync(b.p, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice, s) == cudaSuccess
               ? SME_OK
               : SME_ERR_CUDA;
}

// Host set-up of the sparse schedule for sequences d (host copies of the
// descriptors, in launch order): sequences sharing one luma plane, size and
// frame count form a group (at most kGroupMax VOPs) whose co-located errors
// the streaming pass computes once; one block row per (group, frame).
int setup_sparse(SparseScratch& sp, const std::vector<SeqDesc>& d, cudaStream_t s, bool rounds = false)
{
    const int n = (int)d.size();
    std::vector<int> first, members, gfg, gff, base(n);
    std::vector<long long> rb(n);
    std::vector<int> gid_of(n, -1);
    long long rows = 0;
    int steps = 0, max_mbh = 0, pair_keys = 0, max_p = 0;
    for (int i = 0; i < n; ++i) {
        rb[i] = rows;
        rows += (long long)d[i].F * d[i].MBH;
        base[i] = d[i].gid_base;
        steps = std::max(steps, (d[i].MBW - 1) + 2 * (d[i].MBH - 1) + d[i].P);
        pair_keys = std::max(pair_keys, (d[i].MBW - 1) + 2 * (d[i].MBH - 1) + 1);
        max_p = std::max(max_p, d[i].P);
        max_mbh = std::max(max_mbh, d[i].MBH);
    }
    if (rounds) {
        if ((long long)pair_keys * max_p > (1LL << 26)) return SME_ERR_SIZE;
        steps = pair_keys * max_p;
    }
    for (int i = 0; i < n; ++i) {
        if (gid_of[i] >= 0) continue;
        const int g = (int)first.size();
        first.push_back((int)members.size());
        for (int j = i; j < n && (int)members.size() - first.back() < kGroupMax; ++j)
            if (gid_of[j] < 0 && d[j].luma == d[i].luma && d[j].W == d[i].W && d[j].H == d[i].H &&
                d[j].F == d[i].F && d[j].rd == d[i].rd) {
                gid_of[j] = g;
                members.push_back(j);
            }
        for (int f = 0; f < d[i].F; ++f) {
            gfg.push_back(g);
            gff.push_back(f);
        }
    }
    first.push_back((int)members.size());
    if (gfg.size() > 65535u * 1024u) return SME_ERR_SIZE;
    int rc;
    const size_t total = (size_t)d.back().gid_base + (size_t)d.back().P * d.back().M;
    if ((rc = upload(sp.grp_first, first, s)) || (rc = upload(sp.grp_members, members, s)) ||
        (rc = upload(sp.gf_group, gfg, s)) || (rc = upload(sp.gf_frame, gff, s)) || (rc = upload(sp.row_base, rb, s)) ||
        (rc = upload(sp.seq_base, base, s)) || (rc = ensure(sp.rowcnt, (size_t)rows * 4)) ||
        (rc = ensure(sp.hist, ((size_t)steps + 1) * 32)) || (rc = ensure(sp.cursor, (size_t)steps * 32)) ||
        (rc = ensure(sp.first, (size_t)n * 4)) || (rc = ensure(sp.round_ticket, (size_t)max_p * 4)) ||
        (rc = ensure(sp.list, total * 4)) || (rc = ensure(sp.ctr, sizeof(SparseCounters))))
        return rc;
    sp.n_gf = (int)gfg.size();
    sp.max_mbh = max_mbh;
    sp.steps = steps;
    sp.pair_keys = rounds ? pair_keys : 0;
    sp.rounds = max_p;
    sp.nseq = n;
    sp.total_rows = rows;
    return SME_OK;
}

SparseArgs sparse_args(const SparseScratch& sp, SeqDesc* seqs, DevStatus* status)
{
    SparseArgs a{};
    a.seqs = seqs;
    a.desc_dst = seqs;
    a.nseq = sp.nseq;
    a.grp_first = (const int*)sp.grp_first.p;
    a.grp_members = (const int*)sp.grp_members.p;
    a.gf_group = (const int*)sp.gf_group.p;
    a.gf_frame = (const int*)sp.gf_frame.p;
    a.n_gf = sp.n_gf;
    a.max_mbh = sp.max_mbh;
    a.row_base = (const long long*)sp.row_base.p;
    a.total_rows = sp.total_rows;
    a.rowcnt = (unsigned*)sp.rowcnt.p;
    a.hist = (unsigned*)sp.hist.p;
    a.first_step = (int*)sp.first.p;
    a.cursor = (unsigned*)sp.cursor.p;
    a.steps = sp.steps;
    a.pair_keys = sp.pair_keys;
    a.round_ticket = (unsigned*)sp.round_ticket.p;
    a.rounds = sp.rounds;
    a.list = (int*)sp.list.p;
    a.ctr = (SparseCounters*)sp.ctr.p;
    a.status = status;
    return a;
}

// The search launch of the sparse schedule: every CTA resident (the warps
// wait on each other), min_blocks selects the register budget.
int launch_sparse_search(const Method& m, MeArgs a, const SparseScratch& sp, int num_sms, int min_blocks,
                         cudaStream_t s, int round = -1)
{
    int per_sm = 0;
    if (me_sparse_occupancy(m.S, min_blocks, &per_sm, m.tt != 0) != cudaSuccess || per_sm < 1) return SME_ERR_CUDA;
    a.list = (const int*)sp.list.p;
    a.seq_base = (const int*)sp.seq_base.p;
    a.nseq = sp.nseq;
    a.ctr = (SparseCounters*)sp.ctr.p;
    a.round = round;
    a.pair_keys = sp.pair_keys;
    a.rounds = sp.rounds;
    a.offs = (const unsigned*)sp.hist.p;
    a.round_ticket = (unsigned*)sp.round_ticket.p;
    return cuda_status(launch_me_sparse(m, a, num_sms * per_sm, min_blocks, s));
}

int check_params(const sme_params* p)
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

Geom make_geom(const sme_params& p)
{
    Geom g;
    g.W = p.width;
    g.H = p.height;
    g.MBW = p.width / 16;
    g.MBH = p.height / 16;
    g.M = g.MBW * g.MBH;
    g.Wp = (((p.width + 31) / 32 + 1) + 3) & ~3;  // 16-byte rows (TMA)
    return g;
}

Method make_method(const sme_params& p)
{
    Method m;
    m.S = p.search_range;
    m.h = p.subpel;
    m.K = p.max_iters;
    m.theta = p.theta;
    m.eps = p.epsilon;
    m.tt = 0;
    return m;
}

// The per-pair kernel's four tensor maps of one sequence: the luma frames
// (u8 [F][H][W]) with the reference-window box and the current-block box, and
// the packed alpha (u32 [F][H][Wp]) with the reference-strip box and the
// current-BAB box.
struct alignas(128) MapSet {
    CUtensorMap m[4];
};

int encode_map(CUtensorMap* map, CUtensorMapDataType dt, const void* base, cuuint64_t w, cuuint64_t h,
               cuuint64_t f, cuuint64_t elem, const unsigned (&box)[2])
{
    PFN_cuTensorMapEncodeTiled_v12000 fn = tensor_map_encoder();
    if (!fn) return SME_ERR_CUDA;
    const cuuint64_t dims[3] = {w, h, f};
    const cuuint64_t strides[2] = {w * elem, w * h * elem};
    const cuuint32_t bx[3] = {box[0], box[1], 1u};
    const cuuint32_t estr[3] = {1u, 1u, 1u};
    const CUresult r = fn(map, dt, 3, const_cast<void*>(base), dims, strides, bx, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                          CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                          CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? SME_OK : SME_ERR_CUDA;
}

int encode_pair_maps(MapSet* ms, const uint8_t* luma, const uint32_t* packed, const Geom& g, int F, int S)
{
    unsigned box[4][2];
    pair_boxes(S, box);
    int rc;
    if ((rc = encode_map(&ms->m[0], CU_TENSOR_MAP_DATA_TYPE_UINT8, luma, g.W, g.H, F, 1, box[0])) ||
        (rc = encode_map(&ms->m[1], CU_TENSOR_MAP_DATA_TYPE_UINT8, luma, g.W, g.H, F, 1, box[1])) ||
        (rc = encode_map(&ms->m[2], CU_TENSOR_MAP_DATA_TYPE_UINT32, packed, g.Wp, g.H, F, 4, box[2])) ||
        (rc = encode_map(&ms->m[3], CU_TENSOR_MAP_DATA_TYPE_UINT32, packed, g.Wp, g.H, F, 4, box[3])))
        return rc;
    return SME_OK;
}

// Ticket order of the persistent launch: MB (u, v) of pair k becomes ready
// at wavefront step t = u + 2v + k (A, B, C of Fig. 3 sit at steps t-1,
// t-2, t-1 of the same pair; T is step t-1 of the previous pair), so listing
// MBs by increasing t puts every dependency before its dependents.
int build_schedule(sme_ctx* c, int P)
{
    if (c->sched_P == P) return SME_OK;
    const Geom& g = c->g;
    const size_t total = (size_t)P * g.M;
    if (total > (size_t)INT32_MAX) return SME_ERR_SIZE;
    try {
        c->sched_host.assign(total, 0);
    } catch (...) {
        return SME_ERR_NOMEM;
    }
    const int tmax = (g.MBW - 1) + 2 * (g.MBH - 1) + (P - 1);
    size_t n = 0;
    for (int t = 0; t <= tmax; ++t)
        for (int k = 0; k < P; ++k)
            for (int v = 0; v < g.MBH; ++v) {
                const int u = t - 2 * v - k;
                if (u < 0) break;
                if (u < g.MBW) c->sched_host[n++] = k * g.M + v * g.MBW + u;
            }
    if (n != total) return SME_ERR_STATE;
    int rc = ensure(c->sched, total * sizeof(int));
    if (rc) return rc;
    if (cudaMemcpyAsync(c->sched.p, c->sched_host.data(), total * sizeof(int), cudaMemcpyHostToDevice,
                        c->stream) != cudaSuccess)
        return SME_ERR_CUDA;
    c->sched_P = P;
    return SME_OK;
}

// Cluster schedule of P pairs: the MBs in wavefront order dealt round robin
// to the C CTAs of a cluster (item n -> CTA n % C, position n / C), and for
// every MB the slot of each MB that takes it as candidate A, B, C or T.
int build_cluster_schedule(sme_ctx* c, int P, int* C_out)
{
    const Geom& g = c->g;
    const long long total = (long long)P * g.M;
    const int want = c->cluster > 0 ? c->cluster : 16;
    int C = 0, cap = 0, nw = 0;
    for (int cs = want; cs >= 2 && !C; cs /= 2)
        for (int w = kClusterWarps; w >= 4 && !C; --w) {
            const long long cp = (total + cs - 1) / cs;
            const int resident = cp <= (1 << 18) ? me_cluster_fits(c->m.S, (int)cp, cs, w) : 0;
            if (resident > 0) {
                C = cs;
                cap = (int)cp;
                nw = w;
                c->cl_resident = resident;
            }
        }
    if (!C) return SME_ERR_SIZE;
    *C_out = C;
    c->cl_warps = nw;
    if (c->cl_P == P && c->cl_C == C) return SME_OK;
    int rc = build_schedule(c, P);  // the wavefront order
    if (rc) return rc;
    std::vector<int> items, count, where, cons;
    try {
        items.assign((size_t)C * cap, -1);
        count.assign(C, 0);
        where.assign(total, 0);
        cons.assign(4 * total, -1);
    } catch (...) {
        return SME_ERR_NOMEM;
    }
    for (long long n = 0; n < total; ++n) {
        const int gid = c->sched_host[n], r = (int)(n % C), slot = (int)(n / C);
        items[(size_t)r * cap + slot] = gid;
        ++count[r];
        where[gid] = (r << 20) | (4 * slot);
    }
    for (long long gid = 0; gid < total; ++gid) {
        const int k = (int)(gid / g.M), mb = (int)(gid - (long long)k * g.M), u = mb % g.MBW, v = mb / g.MBW;
        long long to[4] = {-1, -1, -1, -1};  // the MBs whose A, B, C, T this one is
        if (u + 1 < g.MBW) to[0] = gid + 1;
        if (v + 1 < g.MBH) to[1] = gid + g.MBW;
        if (v + 1 < g.MBH && u > 0) to[2] = gid + g.MBW - 1;
        if (k + 1 < P) to[3] = gid + g.M;
        for (int role = 0; role < 4; ++role)
            if (to[role] >= 0) cons[4 * gid + role] = where[to[role]] + role;
    }
    if ((rc = ensure(c->cl_items, items.size() * sizeof(int))) || (rc = ensure(c->cl_count, C * sizeof(int))) ||
        (rc = ensure(c->cl_cons, cons.size() * sizeof(int))))
        return rc;
    if (cudaMemcpy(c->cl_items.p, items.data(), items.size() * sizeof(int), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(c->cl_count.p, count.data(), C * sizeof(int), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(c->cl_cons.p, cons.data(), cons.size() * sizeof(int), cudaMemcpyHostToDevice) != cudaSuccess)
        return SME_ERR_CUDA;
    c->cl_P = P;
    c->cl_C = C;
    c->cl_cap = cap;
    return SME_OK;
}

// before_me: an event the motion-estimation launch waits for (after the
// classification has been queued), or NULL.
int run_sequence(sme_ctx* c, const uint8_t* luma, const uint8_t* alpha, int F, const sme_mv* temporal_in,
                 const float* seed, const sme_outputs* out, cudaEvent_t before_me = nullptr)
{
    const Geom& g = c->g;
    if (!luma || !alpha || !out || !out->mv) return SME_ERR_ARG;
    if (!aligned16(luma) || !aligned16(alpha)) return SME_ERR_ARG;
    if (seed && c->m.K > kMaxSeededIters) return SME_ERR_ARG;  // the position log's bound
    const int rd = c->prm.ref_distance;
    if (F <= rd) return SME_ERR_ARG;
    const int P = F - rd;
    const size_t total = (size_t)P * g.M;
    int rc;
    if ((rc = ensure(c->packed, (size_t)F * g.H * g.Wp * sizeof(uint32_t)))) return rc;
    if ((rc = ensure(c->cls, (size_t)F * g.M))) return rc;
    // the four-vector mode's per-MB schedule publishes three words per MB
    if ((rc = ensure(c->ready, (c->four_mv ? 3 : 1) * total * sizeof(unsigned long long), true, c->stream))) return rc;
    if ((rc = ensure(c->desc, sizeof(SeqDesc)))) return rc;
    // The per-MB schedule is the faster one on single sequences (measured on
    // CIF x 30 frames: 130 us vs 193 us per launch); the pair schedule is
    // chosen only on request, and always in the four-vector mode.
    if (c->four_mv && (seed || c->m.tt)) return SME_ERR_ARG;
    // four-vector mode: the pair schedule on request, else the per-MB one
    const bool pair = c->schedule == kSchedPair, cluster = !c->four_mv && c->schedule == kSchedCluster;
    const bool sparse = !c->four_mv && c->schedule == kSchedSparse;
    MapSet maps;
    memset(&maps, 0, sizeof(maps));
    int C = 0;
    if (pair) {
        if ((rc = encode_pair_maps(&maps, luma, (const uint32_t*)c->packed.p, g, F, c->m.S))) return rc;
    } else if (cluster) {
        if ((rc = build_cluster_schedule(c, P, &C))) return rc;
    } else if (!sparse && (rc = build_schedule(c, P))) {
        return rc;
    }

    SeqDesc d{};
    d.luma = luma;
    d.alpha = alpha;
    d.packed_w = (uint32_t*)c->packed.p;
    d.cls_w = (uint8_t*)c->cls.p;
    d.packed = (const uint32_t*)c->packed.p;
    d.cls = (const uint8_t*)c->cls.p;
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

    // The classify launch also stores the descriptor the ME launch reads.
    ClassifyArgs ca{};
    ca.alpha = alpha;
    ca.n_frames = F;
    ca.cls = (uint8_t*)c->cls.p;
    ca.packed = (uint32_t*)c->packed.p;
    ca.status = c->status;
    ca.sse = out->sse;
    ca.n_sse = P;
    ca.desc_out = (SeqDesc*)c->desc.p;
    ca.desc = d;
    cudaEvent_t* ev = nullptr;
    if (c->prof_n < c->prof_max) {
        ev = &c->prof_ev[3 * c->prof_n++];
        if (cudaEventRecord(ev[0], c->stream) != cudaSuccess) return SME_ERR_CUDA;
    }
    if (sparse) {
        // one sequence, one group: the set-up depends on the frame count only
        if (c->sp.key_f != F) {
            std::vector<SeqDesc> one(1, d);
            if ((rc = setup_sparse(c->sp, one, c->stream))) return rc;
            c->sp.key_f = F;
        }
        if (before_me && cudaStreamWaitEvent(c->stream, before_me, 0) != cudaSuccess) return SME_ERR_CUDA;
        if (launch_sparse_prep(sparse_args(c->sp, (SeqDesc*)c->desc.p, c->status), &d, c->stream) != cudaSuccess)
            return SME_ERR_CUDA;
    } else if (launch_classify(g, ca, c->stream) != cudaSuccess) {
        return SME_ERR_CUDA;
    }
    if (ev && cudaEventRecord(ev[1], c->stream) != cudaSuccess) return SME_ERR_CUDA;
    if (!sparse && before_me && cudaStreamWaitEvent(c->stream, before_me, 0) != cudaSuccess) return SME_ERR_CUDA;

    MeArgs a{};
    a.seqs = (const SeqDesc*)c->desc.p;
    a.sched = pair ? nullptr : (const int*)c->sched.p;
    a.sched_seq = nullptr;
    a.unit_seq = nullptr;
    a.unit_pair = nullptr;
    a.tmaps = nullptr;
    a.total_units = P;
    a.mbw_max = g.MBW;
    a.ready = (unsigned long long*)c->ready.p;
    a.ready_a = c->four_mv ? a.ready + total : nullptr;
    a.ready_bc = c->four_mv ? a.ready + 2 * total : nullptr;
    a.status = c->status;
    a.m = c->m;
    a.total = (int)total;
    a.fault_ticket = c->fault_ticket;
    a.speculate = c->speculate;
    a.pair_direct = c->four_mv ? 0 : c->pair_direct;
    a.four_mv = c->four_mv;
    a.timeout_ns = c->timeout_ns;
    if (sparse) {
        if ((rc = launch_sparse_search(c->m, a, c->sp, c->num_sms, c->mb_ctas_per_sm, c->stream))) return rc;
    } else if (cluster) {
        a.cl_items = (const int*)c->cl_items.p;
        a.cl_count = (const int*)c->cl_count.p;
        a.cl_consumers = (const int*)c->cl_cons.p;
        a.cl_cap = c->cl_cap;
        // helpers only in clusters that are resident together with the chain
        const int helpers = std::max(1, c->cl_resident - 1);
        if (launch_me_cluster(c->m, a, C, c->cl_warps, helpers, c->stream) != cudaSuccess) return SME_ERR_CUDA;
    } else if (pair) {
        int nw = c->pair_warps > 0 ? c->pair_warps : std::min(kPairWarpsMax, g.MBH);
        if (a.pair_direct && !a.four_mv) nw = std::min(nw, 8);  // the direct instantiation's bound
        while (nw > 1 && me_pair_smem_bytes(c->m.S, nw, g.MBW, c->four_mv != 0) > (size_t)c->smem_optin) --nw;
        int per_sm = 0;
        if (me_pair_occupancy(c->m.S, nw, g.MBW, a.pair_direct != 0, a.four_mv != 0, &per_sm) != cudaSuccess ||
            per_sm < 1)
            return SME_ERR_CUDA;
        const int grid = std::max(1, std::min(c->num_sms * per_sm, P));
        if (launch_me_pair(c->m, a, &maps, nw, grid, c->stream) != cudaSuccess) return SME_ERR_CUDA;
    } else {
        int resident = c->me_blocks_per_sm;
        if (c->four_mv && (me4_occupancy(c->m.S, &resident) != cudaSuccess || resident < 1)) return SME_ERR_CUDA;
        if (!c->four_mv && c->m.tt && (me_occupancy(c->m.S, &resident, true) != cudaSuccess || resident < 1))
            return SME_ERR_CUDA;
        const int per_sm = c->mb_ctas_per_sm > 0 ? std::min(c->mb_ctas_per_sm, resident) : resident;
        const long long cap = (long long)c->num_sms * per_sm;
        const long long want = ((long long)total + kMeWarps - 1) / kMeWarps;
        const int grid = (int)std::max(1LL, std::min<long long>(cap, want));
        if ((c->four_mv ? launch_me4(c->m, a, grid, c->stream) : launch_me(c->m, a, grid, c->stream)) != cudaSuccess)
            return SME_ERR_CUDA;
    }
    if (ev && cudaEventRecord(ev[2], c->stream) != cudaSuccess) return SME_ERR_CUDA;
    return SME_OK;
}

void profile_free(sme_ctx* c)
{
    for (cudaEvent_t e : c->prof_ev) cudaEventDestroy(e);
    c->prof_ev.clear();
    c->prof_max = c->prof_n = 0;
}

// The device-mapped address of a pinned (page-locked) host buffer, or NULL
// for any other pointer.  Kernels read and write such buffers in place, over
// the CPU-GPU link, instead of through a staging copy.
void* mapped_host(const void* p)
{
    cudaPointerAttributes at;
    if (!p || cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return at.type == cudaMemoryTypeHost ? at.devicePointer : nullptr;
}

int read_status(sme_ctx* c)
{
    int err = 0;
    if (cudaMemcpy(&err, &c->status->err, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess)
        return SME_ERR_CUDA;
    if (err) {
        if (cudaMemset(&c->status->err, 0, sizeof(int)) != cudaSuccess) return SME_ERR_CUDA;
        return err;
    }
    return SME_OK;
}

struct ExecCfg {
    int schedule, pair_warps, mb_ctas_per_sm, speculate, cluster, pair_direct;
};
// The cluster schedule runs single sequences only (the batch skips it).
const ExecCfg kTuneCandidates[] = {
    {kSchedMB, 0, 1, 1, 0, 1},       {kSchedMB, 0, 0, 1, 0, 1},       {kSchedMB, 0, 1, 0, 0, 1},
    {kSchedMB, 0, 0, 0, 0, 1},       {kSchedPair, 4, 0, 0, 0, 1},     {kSchedPair, 8, 0, 0, 0, 1},
    {kSchedPair, 4, 0, 0, 0, 0},     {kSchedPair, 8, 0, 0, 0, 0},
    {kSchedPair, 16, 0, 0, 0, 0},    {kSchedCluster, 0, 0, 1, 16, 1}, {kSchedCluster, 0, 0, 0, 16, 1},
    {kSchedCluster, 0, 0, 1, 8, 1},  {kSchedSparse, 0, 1, 0, 0, 1},   {kSchedSparse, 0, 2, 0, 0, 1},
    {kSchedSparse, 0, 3, 0, 0, 1},   {kSchedSparse, 0, 5, 0, 0, 1},
};

// Device time of `trials` back-to-back runs of `enqueue` (the minimum), ms;
// a negative value means the configuration failed.
template <class F>
float time_runs(cudaStream_t s, int trials, F enqueue)
{
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) return -1.0f;
    float best = -1.0f;
    for (int i = 0; i < trials; ++i) {
        if (cudaEventRecord(e0, s) != cudaSuccess || enqueue() != SME_OK || cudaEventRecord(e1, s) != cudaSuccess ||
            cudaEventSynchronize(e1) != cudaSuccess) {
            best = -1.0f;
            break;
        }
        float ms = 0.0f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (best < 0.0f || ms < best) best = ms;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaGetLastError();
    return best;
}

}  // namespace

extern "C" {

void sme_default_params(sme_params* p, int width, int height)
{
    if (!p) return;
    p->width = width;
    p->height = height;
    p->search_range = 16;
    p->subpel = 1;
    p->theta = 2.0f;
    p->epsilon = 1.0f;
    p->max_iters = 8;
    p->ref_distance = 1;
}

const char* sme_strerror(int s)
{
    switch (s) {
    case SME_OK: return "ok";
    case SME_ERR_ARG: return "invalid argument";
    case SME_ERR_SIZE: return "width/height must be positive multiples of 16 (at most 8192)";
    case SME_ERR_CUDA: return "CUDA runtime error";
    case SME_ERR_TIMEOUT: return "a bounded device wait gave up; results are incomplete";
    case SME_ERR_STATE: return "call made in the wrong state";
    case SME_ERR_NOMEM: return "allocation failed";
    case SME_ERR_RANGE: return "a supplied motion vector lies outside the valid set";
    case SME_ERR_SCRATCH: return "problem exceeds the fixed 4 MiB scratch of sme_estimate_sequence_noalloc";
    default: return "unknown status";
    }
}

int sme_packed_words(int width) { return width > 0 ? ((((width + 31) / 32 + 1) + 3) & ~3) : 0; }

int sme_create(sme_ctx** out, const sme_params* p, void* stream)
{
    if (!out) return SME_ERR_ARG;
    *out = nullptr;
    int rc = check_params(p);
    if (rc) return rc;
    sme_ctx* c = new (std::nothrow) sme_ctx();
    if (!c) return SME_ERR_NOMEM;
    c->prm = *p;
    c->g = make_geom(*p);
    c->m = make_method(*p);
    c->stream = (cudaStream_t)stream;
    if (cudaGetDevice(&c->device) != cudaSuccess ||
        cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, c->device) != cudaSuccess ||
        cudaDeviceGetAttribute(&c->smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, c->device) != cudaSuccess ||
        me_occupancy(c->m.S, &c->me_blocks_per_sm) != cudaSuccess || c->me_blocks_per_sm < 1) {
        cudaGetLastError();
        delete c;
        return SME_ERR_CUDA;
    }
    if (cudaMalloc(&c->status, sizeof(DevStatus)) != cudaSuccess ||
        cudaMemset(c->status, 0, sizeof(DevStatus)) != cudaSuccess ||
        cudaHostAlloc(&c->h_err, sizeof(int), cudaHostAllocDefault) != cudaSuccess) {
        cudaGetLastError();
        if (c->status) cudaFree(c->status);
        if (c->h_err) cudaFreeHost(c->h_err);
        delete c;
        return SME_ERR_NOMEM;
    }
    *out = c;
    return SME_OK;
}

int sme_destroy(sme_ctx* c)
{
    if (!c) return SME_ERR_ARG;
    cudaStreamSynchronize(c->stream);
    DevBuf* bufs[] = {&c->packed, &c->cls, &c->ready, &c->sched, &c->desc, &c->qpacked, &c->qcls,
                      &c->pair_luma, &c->pair_alpha, &c->temporal, &c->last_mv, &c->last_sse, &c->seed_field,
                      &c->h_luma, &c->h_alpha, &c->h_tmp, &c->h_seed, &c->h_mv, &c->h_cost,
                      &c->h_disp, &c->h_iters, &c->h_npos, &c->h_cls, &c->h_ssemb, &c->h_sse,
                      &c->h_pred, &c->cl_items, &c->cl_count, &c->cl_cons};
    for (DevBuf* b : bufs) release(*b);
    release_sparse(c->sp);
    profile_free(c);
    if (c->status) cudaFree(c->status);
    if (c->h_err) cudaFreeHost(c->h_err);
    if (c->copy_stream) {
        cudaStreamSynchronize(c->copy_stream);
        cudaStreamDestroy(c->copy_stream);
    }
    if (c->copy_go) cudaEventDestroy(c->copy_go);
    if (c->copy_done) cudaEventDestroy(c->copy_done);
    delete c;
    return SME_OK;
}

int sme_set_stream(sme_ctx* c, void* stream)
{
    if (!c) return SME_ERR_ARG;
    c->stream = (cudaStream_t)stream;
    return SME_OK;
}

int sme_synchronize(sme_ctx* c)
{
    if (!c) return SME_ERR_ARG;
    // the error word travels with the stream's work: one wait, not two
    if (cudaMemcpyAsync(c->h_err, &c->status->err, sizeof(int), cudaMemcpyDeviceToHost, c->stream) != cudaSuccess ||
        cudaStreamSynchronize(c->stream) != cudaSuccess)
        return SME_ERR_CUDA;
    const int err = *c->h_err;
    if (err) {
        if (cudaMemsetAsync(&c->status->err, 0, sizeof(int), c->stream) != cudaSuccess ||
            cudaStreamSynchronize(c->stream) != cudaSuccess)
            return SME_ERR_CUDA;
        return err;
    }
    return SME_OK;
}

int sme_classify(sme_ctx* c, const uint8_t* alpha, int n_frames, uint8_t* mb_class, uint32_t* packed)
{
    if (!c || !alpha || !mb_class || n_frames < 1 || !aligned16(alpha)) return SME_ERR_ARG;
    ClassifyArgs ca{};
    ca.alpha = alpha;
    ca.n_frames = n_frames;
    ca.cls = mb_class;
    ca.packed = packed;
    return cuda_status(launch_classify(c->g, ca, c->stream));
}

int sme_classify_table(sme_ctx* c, const uint8_t* const* frames, int n, uint8_t* mb_class)
{
    if (!c || !frames || !mb_class || n < 1 || n > 65535) return SME_ERR_ARG;
    ClassifyArgs ca{};
    ca.frames = frames;
    ca.n_frames = n;
    ca.cls = mb_class;
    return cuda_status(launch_classify(c->g, ca, c->stream));
}

int sme_estimate_sequence(sme_ctx* c, const uint8_t* luma, const uint8_t* alpha, int n_frames,
                          const sme_mv* temporal_in, const float* seed, const sme_outputs* out)
{
    if (!c) return SME_ERR_ARG;
    return run_sequence(c, luma, alpha, n_frames, temporal_in, seed, out);
}

int sme_estimate_sequence_host(sme_ctx* c, const uint8_t* luma, const uint8_t* alpha, int n_frames,
                               const sme_mv* temporal_in, const float* seed, const sme_outputs* out)
{
    if (!c || !luma || !alpha || !out || !out->mv) return SME_ERR_ARG;
    if (seed && c->m.K > kMaxSeededIters) return SME_ERR_ARG;
    const Geom& g = c->g;
    const int rd = c->prm.ref_distance;
    if (n_frames <= rd) return SME_ERR_ARG;
    const size_t FS = (size_t)g.W * g.H, P = (size_t)(n_frames - rd), PM = P * g.M;
    const size_t NB = c->four_mv ? 4 : 1;  // vectors per MB
    const cudaStream_t s = c->stream;
    int rc;
    // Luma is read many times (search windows): always copied.  Alpha is read
    // once, by the classification: read in place when it is pinned.  Outputs
    // other than the per-pair SSE (accumulated with atomics) are written in
    // place when pinned, else staged and copied back.
    const uint8_t* dalpha = (const uint8_t*)mapped_host(alpha);
    if ((rc = ensure(c->h_luma, FS * n_frames)) || (!dalpha && (rc = ensure(c->h_alpha, FS * n_frames))))
        return rc;
    cudaEvent_t luma_ready = nullptr;
    if (dalpha) {
        if (!c->copy_stream && (cudaStreamCreateWithFlags(&c->copy_stream, cudaStreamNonBlocking) != cudaSuccess ||
                                cudaEventCreateWithFlags(&c->copy_go, cudaEventDisableTiming) != cudaSuccess ||
                                cudaEventCreateWithFlags(&c->copy_done, cudaEventDisableTiming) != cudaSuccess))
            return SME_ERR_CUDA;
        // the copy waits for earlier work on the context's stream (which may still read h_luma)
        if (cudaEventRecord(c->copy_go, s) != cudaSuccess || cudaStreamWaitEvent(c->copy_stream, c->copy_go, 0) ||
            cudaMemcpyAsync(c->h_luma.p, luma, FS * n_frames, cudaMemcpyHostToDevice, c->copy_stream) ||
            cudaEventRecord(c->copy_done, c->copy_stream))
            return SME_ERR_CUDA;
        luma_ready = c->copy_done;
    } else if (cudaMemcpyAsync(c->h_luma.p, luma, FS * n_frames, cudaMemcpyHostToDevice, s) != cudaSuccess ||
               cudaMemcpyAsync(c->h_alpha.p, alpha, FS * n_frames, cudaMemcpyHostToDevice, s) != cudaSuccess) {
        return SME_ERR_CUDA;
    }
    if (!dalpha) dalpha = (const uint8_t*)c->h_alpha.p;
    const sme_mv* dtmp = nullptr;
    const float* dseed = nullptr;
    if (temporal_in) {
        if ((rc = ensure(c->h_tmp, NB * g.M * sizeof(sme_mv)))) return rc;
        if (cudaMemcpyAsync(c->h_tmp.p, temporal_in, NB * g.M * sizeof(sme_mv), cudaMemcpyHostToDevice, s))
            return SME_ERR_CUDA;
        dtmp = (const sme_mv*)c->h_tmp.p;
    }
    if (seed) {
        if ((rc = ensure(c->h_seed, PM * 2 * sizeof(float)))) return rc;
        if (cudaMemcpyAsync(c->h_seed.p, seed, PM * 2 * sizeof(float), cudaMemcpyHostToDevice, s))
            return SME_ERR_CUDA;
        dseed = (const float*)c->h_seed.p;
    }
    sme_outputs d{};
    struct Opt {
        void* host;
        DevBuf* buf;
        size_t bytes;
        void** dev;
        bool copy;  // staged (false: written in place)
    } opts[] = {
        {out->mv, &c->h_mv, NB * PM * sizeof(sme_mv), (void**)&d.mv},
        {out->cost, &c->h_cost, NB * PM * 4, (void**)&d.cost},
        {out->disp, &c->h_disp, NB * PM * 8, (void**)&d.disp},
        {out->iters, &c->h_iters, NB * PM, (void**)&d.iters},
        {out->npos, &c->h_npos, NB * PM, (void**)&d.npos},
        {out->mb_class, &c->h_cls, PM, (void**)&d.mb_class},
        {out->sse_mb, &c->h_ssemb, PM * 4, (void**)&d.sse_mb},
        {out->sse, &c->h_sse, P * 8, (void**)&d.sse},
        {out->pred, &c->h_pred, P * FS, (void**)&d.pred},
    };
    for (Opt& o : opts) {
        if (!o.host) continue;
        void* in_place = o.buf == &c->h_sse ? nullptr : mapped_host(o.host);
        o.copy = in_place == nullptr;
        if (in_place) {
            *o.dev = in_place;
            continue;
        }
        if ((rc = ensure(*o.buf, o.bytes))) return rc;
        *o.dev = o.buf->p;
    }
    rc = run_sequence(c, (const uint8_t*)c->h_luma.p, dalpha, n_frames, dtmp, dseed, &d, luma_ready);
    if (rc) return rc;
    for (Opt& o : opts)
        if (o.host && o.copy && cudaMemcpyAsync(o.host, *o.dev, o.bytes, cudaMemcpyDeviceToHost, s) != cudaSuccess)
            return SME_ERR_CUDA;
    return sme_synchronize(c);
}

int sme_set_reference(sme_ctx* c, const uint8_t* luma, const uint8_t* alpha)
{
    if (!c || !luma || !alpha) return SME_ERR_ARG;
    const size_t FS = (size_t)c->g.W * c->g.H;
    int rc;
    if ((rc = ensure(c->pair_luma, 2 * FS)) || (rc = ensure(c->pair_alpha, 2 * FS))) return rc;
    if (cudaMemcpyAsync(c->pair_luma.p, luma, FS, cudaMemcpyDeviceToDevice, c->stream) != cudaSuccess ||
        cudaMemcpyAsync(c->pair_alpha.p, alpha, FS, cudaMemcpyDeviceToDevice, c->stream) != cudaSuccess)
        return SME_ERR_CUDA;
    c->have_ref = true;
    return SME_OK;
}

int sme_set_current(sme_ctx* c, const uint8_t* luma, const uint8_t* alpha)
{
    if (!c || !luma || !alpha) return SME_ERR_ARG;
    const size_t FS = (size_t)c->g.W * c->g.H;
    int rc;
    if ((rc = ensure(c->pair_luma, 2 * FS)) || (rc = ensure(c->pair_alpha, 2 * FS))) return rc;
    if (cudaMemcpyAsync((uint8_t*)c->pair_luma.p + FS, luma, FS, cudaMemcpyDeviceToDevice, c->stream) ||
        cudaMemcpyAsync((uint8_t*)c->pair_alpha.p + FS, alpha, FS, cudaMemcpyDeviceToDevice, c->stream))
        return SME_ERR_CUDA;
    c->have_cur = true;
    return SME_OK;
}

int sme_estimate(sme_ctx* c, const sme_outputs* out)
{
    if (!c || c->four_mv) return SME_ERR_ARG;
    if (!c->have_ref || !c->have_cur) return SME_ERR_STATE;
    const Geom& g = c->g;
    int rc;
    if ((rc = ensure(c->last_mv, g.M * sizeof(sme_mv))) || (rc = ensure(c->last_sse, 8))) return rc;
    sme_outputs o = out ? *out : sme_outputs{};
    const bool user_mv = o.mv != nullptr, user_sse = o.sse != nullptr;
    if (!user_mv) o.mv = (sme_mv*)c->last_mv.p;
    if (!user_sse) o.sse = (unsigned long long*)c->last_sse.p;
    // The pair always has reference distance 1 inside the context buffers.
    const int rd = c->prm.ref_distance;
    c->prm.ref_distance = 1;
    rc = run_sequence(c, (const uint8_t*)c->pair_luma.p, (const uint8_t*)c->pair_alpha.p, 2,
                      c->have_temporal ? (const sme_mv*)c->temporal.p : nullptr,
                      c->have_seed ? (const float*)c->seed_field.p : nullptr, &o);
    c->prm.ref_distance = rd;
    if (rc) return rc;
    if (user_mv && cudaMemcpyAsync(c->last_mv.p, o.mv, g.M * sizeof(sme_mv), cudaMemcpyDeviceToDevice, c->stream))
        return SME_ERR_CUDA;
    if (user_sse && cudaMemcpyAsync(c->last_sse.p, o.sse, 8, cudaMemcpyDeviceToDevice, c->stream))
        return SME_ERR_CUDA;
    c->have_result = true;
    return SME_OK;
}

int sme_advance(sme_ctx* c)
{
    if (!c) return SME_ERR_ARG;
    if (!c->have_cur || !c->have_result) return SME_ERR_STATE;
    const Geom& g = c->g;
    const size_t FS = (size_t)g.W * g.H;
    int rc;
    if ((rc = ensure(c->temporal, g.M * sizeof(sme_mv)))) return rc;
    if (cudaMemcpyAsync(c->pair_luma.p, (uint8_t*)c->pair_luma.p + FS, FS, cudaMemcpyDeviceToDevice, c->stream) ||
        cudaMemcpyAsync(c->pair_alpha.p, (uint8_t*)c->pair_alpha.p + FS, FS, cudaMemcpyDeviceToDevice, c->stream) ||
        cudaMemcpyAsync(c->temporal.p, c->last_mv.p, g.M * sizeof(sme_mv), cudaMemcpyDeviceToDevice, c->stream))
        return SME_ERR_CUDA;
    c->have_temporal = true;
    c->have_cur = false;
    c->have_result = false;
    return SME_OK;
}

int sme_score(sme_ctx* c, double* psnr_db)
{
    if (!c || !psnr_db) return SME_ERR_ARG;
    if (!c->have_result) return SME_ERR_STATE;
    int rc = sme_synchronize(c);
    if (rc) return rc;
    unsigned long long sse = 0;
    if (cudaMemcpy(&sse, c->last_sse.p, 8, cudaMemcpyDeviceToHost) != cudaSuccess) return SME_ERR_CUDA;
    *psnr_db = sme_psnr(sse, c->g.W, c->g.H);
    return SME_OK;
}

int sme_get_temporal_field(sme_ctx* c, sme_mv* field)
{
    if (!c || !field) return SME_ERR_ARG;
    const size_t bytes = c->g.M * sizeof(sme_mv);
    if (!c->have_temporal) return cuda_status(cudaMemsetAsync(field, 0, bytes, c->stream));
    return cuda_status(cudaMemcpyAsync(field, c->temporal.p, bytes, cudaMemcpyDeviceToDevice, c->stream));
}

int sme_set_temporal_field(sme_ctx* c, const sme_mv* field)
{
    if (!c) return SME_ERR_ARG;
    if (!field) {
        c->have_temporal = false;
        return SME_OK;
    }
    const size_t bytes = c->g.M * sizeof(sme_mv);
    int rc = ensure(c->temporal, bytes);
    if (rc) return rc;
    if (cudaMemcpyAsync(c->temporal.p, field, bytes, cudaMemcpyDeviceToDevice, c->stream) != cudaSuccess)
        return SME_ERR_CUDA;
    c->have_temporal = true;
    return SME_OK;
}

int sme_set_seed_field(sme_ctx* c, const float* seed)
{
    if (!c) return SME_ERR_ARG;
    if (!seed) {
        c->have_seed = false;
        return SME_OK;
    }
    if (c->four_mv || c->m.K > kMaxSeededIters) return SME_ERR_ARG;
    const size_t bytes = (size_t)c->g.M * 2 * sizeof(float);
    int rc = ensure(c->seed_field, bytes);
    if (rc) return rc;
    if (cudaMemcpyAsync(c->seed_field.p, seed, bytes, cudaMemcpyDeviceToDevice, c->stream) != cudaSuccess)
        return SME_ERR_CUDA;
    c->have_seed = true;
    return SME_OK;
}

int sme_compensate(sme_ctx* c, const uint8_t* ref, const uint8_t* cur, const sme_mv* mv, uint8_t* pred,
                   unsigned long long* sse)
{
    if (!c || !ref || !cur || !mv || !sse) return SME_ERR_ARG;
    if (cudaMemsetAsync(sse, 0, sizeof(unsigned long long), c->stream) != cudaSuccess) return SME_ERR_CUDA;
    CompArgs a{ref, cur, mv, pred, sse, c->status};
    return cuda_status(launch_compensate(c->g, c->m, a, c->stream));
}

double sme_psnr(unsigned long long sse, int width, int height)
{
    if (sse == 0) return INFINITY;
    return 10.0 * log10(255.0 * 255.0 * (double)width * (double)height / (double)sse);
}

static int run_queries(sme_ctx* c, const uint8_t* ref, const uint8_t* cur, const uint8_t* aref,
                       const uint8_t* acur, const int32_t* q, int n, uint32_t* tsad, uint32_t* ssad,
                       float* delta)
{
    if (!c || !ref || !cur || !q || n < 0) return SME_ERR_ARG;
    const Geom& g = c->g;
    QueryArgs a{};
    a.ref = ref;
    a.cur = cur;
    a.q = q;
    a.n = n;
    a.tsad = tsad;
    a.ssad = ssad;
    a.delta = delta;
    a.status = c->status;
    if (ssad) {
        if (!aref || !acur || !aligned16(aref) || !aligned16(acur)) return SME_ERR_ARG;
        const size_t pw = (size_t)g.H * g.Wp;
        int rc;
        if ((rc = ensure(c->qpacked, 2 * pw * sizeof(uint32_t))) || (rc = ensure(c->qcls, 2 * (size_t)g.M)))
            return rc;
        uint32_t* pk = (uint32_t*)c->qpacked.p;
        uint8_t* cl = (uint8_t*)c->qcls.p;
        ClassifyArgs ca{};
        ca.n_frames = 1;
        ca.alpha = aref;
        ca.cls = cl;
        ca.packed = pk;
        if (launch_classify(g, ca, c->stream) != cudaSuccess) return SME_ERR_CUDA;
        ca.alpha = acur;
        ca.cls = cl + g.M;
        ca.packed = pk + pw;
        if (launch_classify(g, ca, c->stream) != cudaSuccess) return SME_ERR_CUDA;
        a.pref = pk;
        a.pcur = pk + pw;
    }
    return cuda_status(launch_queries(g, c->m, a, c->stream));
}

int sme_eval_costs(sme_ctx* c, const uint8_t* ref, const uint8_t* cur, const uint8_t* aref,
                   const uint8_t* acur, const int32_t* queries, int n, uint32_t* texture_sad,
                   uint32_t* shape_sad)
{
    return run_queries(c, ref, cur, aref, acur, queries, n, texture_sad, shape_sad, nullptr);
}

int sme_gradient_step(sme_ctx* c, const uint8_t* ref, const uint8_t* cur, const int32_t* queries, int n,
                      float* delta)
{
    if (!delta) return SME_ERR_ARG;
    return run_queries(c, ref, cur, nullptr, nullptr, queries, n, nullptr, nullptr, delta);
}

int sme_set_option(sme_ctx* c, int option, int value)
{
    if (!c) return SME_ERR_ARG;
    switch (option) {
    case SME_OPT_SCHEDULE:
        if (value != SME_SCHED_AUTO && value != SME_SCHED_MB && value != SME_SCHED_PAIR &&
            value != SME_SCHED_CLUSTER && value != SME_SCHED_SPARSE)
            return SME_ERR_ARG;
        c->schedule = value;
        return SME_OK;
    case SME_OPT_PAIR_WARPS:
        if (value < 0 || value > kPairWarpsMax) return SME_ERR_ARG;
        c->pair_warps = value;
        return SME_OK;
    case SME_OPT_MB_CTAS_PER_SM:
        if (value < 0 || value > 32) return SME_ERR_ARG;
        c->mb_ctas_per_sm = value;
        return SME_OK;
    case SME_OPT_SPECULATE:
        if (value != 0 && value != 1) return SME_ERR_ARG;
        c->speculate = value;
        return SME_OK;
    case SME_OPT_CLUSTER_SIZE:
        if (value != 0 && value != 2 && value != 4 && value != 8 && value != 16) return SME_ERR_ARG;
        c->cluster = value;
        return SME_OK;
    case SME_OPT_PAIR_DIRECT:
        if (value != 0 && value != 1) return SME_ERR_ARG;
        c->pair_direct = value;
        return SME_OK;
    case SME_OPT_FOUR_MV:
        if (value != 0 && value != 1) return SME_ERR_ARG;
        c->four_mv = value;
        return SME_OK;
    case SME_OPT_BOUNDARY_T_TEXTURE:
        if (value != 0 && value != 1) return SME_ERR_ARG;
        c->m.tt = value;
        return SME_OK;
    default:
        return SME_ERR_ARG;
    }
}

int sme_full_search(sme_ctx* c, const uint8_t* luma, int n_frames, sme_mv* mv, uint32_t* sad)
{
    if (!c || !luma || !mv || !aligned16(luma)) return SME_ERR_ARG;
    const int rd = c->prm.ref_distance;
    if (n_frames <= rd || n_frames - rd > 65535) return SME_ERR_ARG;
    if (es_smem_bytes(c->m.S, c->m.h) > (size_t)c->smem_optin) return SME_ERR_SIZE;
    return cuda_status(launch_es(luma, c->g.W, c->g.H, c->m.S, c->m.h, rd, n_frames - rd, mv, sad, c->stream));
}

int sme_packed_sad_rate_launch(int ctas_per_sm, int iters, uint32_t* out, void* cuda_stream, int* grid)
{
    if (ctas_per_sm < 1 || ctas_per_sm > 8 || iters < 1 || !out || !grid) return SME_ERR_ARG;
    return cuda_status(launch_packed_sad_rate(ctas_per_sm, iters, out, (cudaStream_t)cuda_stream, grid));
}

int sme_get_option(sme_ctx* c, int option, int* value)
{
    if (!c || !value) return SME_ERR_ARG;
    switch (option) {
    case SME_OPT_SCHEDULE: *value = c->schedule; return SME_OK;
    case SME_OPT_PAIR_WARPS: *value = c->pair_warps; return SME_OK;
    case SME_OPT_MB_CTAS_PER_SM: *value = c->mb_ctas_per_sm; return SME_OK;
    case SME_OPT_SPECULATE: *value = c->speculate; return SME_OK;
    case SME_OPT_CLUSTER_SIZE: *value = c->cluster; return SME_OK;
    case SME_OPT_PAIR_DIRECT: *value = c->pair_direct; return SME_OK;
    case SME_OPT_FOUR_MV: *value = c->four_mv; return SME_OK;
    case SME_OPT_BOUNDARY_T_TEXTURE: *value = c->m.tt; return SME_OK;
    default: return SME_ERR_ARG;
    }
}

int sme_autotune(sme_ctx* c, const uint8_t* luma, const uint8_t* alpha, int n_frames, const sme_outputs* out,
                 int trials)
{
    if (!c || trials < 1) return SME_ERR_ARG;
    int rc = run_sequence(c, luma, alpha, n_frames, nullptr, nullptr, out);  // validates, allocates
    if (rc) return rc;
    if ((rc = sme_synchronize(c))) return rc;
    float best = -1.0f;
    ExecCfg pick = {c->schedule, c->pair_warps, c->mb_ctas_per_sm, c->speculate, c->cluster, c->pair_direct};
    for (const ExecCfg& e : kTuneCandidates) {
        // the four-vector mode runs those on the per-MB schedule
        if (c->four_mv && (e.schedule == kSchedCluster || e.schedule == kSchedSparse)) continue;
        c->schedule = e.schedule;
        c->pair_warps = e.pair_warps;
        c->mb_ctas_per_sm = e.mb_ctas_per_sm;
        c->speculate = e.speculate;
        c->cluster = e.cluster;
        c->pair_direct = e.pair_direct;
        const float ms = time_runs(c->stream, trials, [&] {
            return run_sequence(c, luma, alpha, n_frames, nullptr, nullptr, out);
        });
        if (read_status(c) != SME_OK) continue;
        if (ms > 0.0f && (best < 0.0f || ms < best)) {
            best = ms;
            pick = e;
        }
    }
    c->schedule = pick.schedule;
    c->pair_warps = pick.pair_warps;
    c->mb_ctas_per_sm = pick.mb_ctas_per_sm;
    c->speculate = pick.speculate;
    c->cluster = pick.cluster;
    c->pair_direct = pick.pair_direct;
    return best > 0.0f ? SME_OK : SME_ERR_CUDA;
}

int sme_profile_begin(sme_ctx* c, int max_calls)
{
    if (!c || max_calls < 1 || max_calls > (1 << 20)) return SME_ERR_ARG;
    profile_free(c);
    try {
        c->prof_ev.assign(3 * (size_t)max_calls, nullptr);
    } catch (...) {
        return SME_ERR_NOMEM;
    }
    for (cudaEvent_t& e : c->prof_ev)
        if (cudaEventCreate(&e) != cudaSuccess) {
            profile_free(c);
            return SME_ERR_CUDA;
        }
    c->prof_max = max_calls;
    c->prof_n = 0;
    return SME_OK;
}

int sme_profile_end(sme_ctx* c, int* calls, double* classify_ms, double* me_ms)
{
    if (!c) return SME_ERR_ARG;
    double tc = 0.0, tm = 0.0;
    const int n = c->prof_n;
    if (n > 0 && cudaEventSynchronize(c->prof_ev[3 * (n - 1) + 2]) != cudaSuccess) return SME_ERR_CUDA;
    for (int i = 0; i < n; ++i) {
        float a = 0.0f, b = 0.0f;
        if (cudaEventElapsedTime(&a, c->prof_ev[3 * i], c->prof_ev[3 * i + 1]) != cudaSuccess ||
            cudaEventElapsedTime(&b, c->prof_ev[3 * i + 1], c->prof_ev[3 * i + 2]) != cudaSuccess)
            return SME_ERR_CUDA;
        tc += a;
        tm += b;
    }
    if (calls) *calls = n;
    if (classify_ms) *classify_ms = tc;
    if (me_ms) *me_ms = tm;
    profile_free(c);
    return SME_OK;
}

int sme_debug_set_fault(sme_ctx* c, int skip_ticket, long long timeout_ns)
{
    if (!c) return SME_ERR_ARG;
    c->fault_ticket = skip_ticket < 0 ? -1 : skip_ticket;
    c->timeout_ns = timeout_ns > 0 ? timeout_ns : kDefaultTimeoutNs;
    return SME_OK;
}

}  // extern "C"

// ====================================================================
// Batches of sequences
// ====================================================================
struct sme_batch {
    sme_params prm;
    Method m;
    cudaStream_t stream = nullptr, cap_stream = nullptr;
    int device = 0, num_sms = 0, smem_optin = 0, me_blocks_per_sm = 0;
    int n = 0, total_frames = 0, max_mbh = 0, mbw_max = 0, total_units = 0;
    long long total_mbs = 0;
    DevStatus* status = nullptr;
    DevBuf descs, packed, cls, ready, sched, sched_seq, unit_seq, unit_pair, fseq, ffrm, maps;
    SparseScratch sp;
    int four_mv = 0;              // four vectors per MB (Sec. 3.2): per-MB or staged per-pair schedule
    std::vector<size_t> cls_off;  // byte offset of each sequence's class map [F][M] in cls
    std::vector<SeqDesc> host_desc;  // the descriptors (device addresses, sizes) of every sequence
    // host-buffer uploads: copies spread over several streams (copy engines),
    // forked from and joined back to the batch's stream
    static constexpr int kCopyStreams = 4;
    cudaStream_t copy[kCopyStreams] = {};
    cudaEvent_t fork = nullptr, join[kCopyStreams] = {};
    ExecCfg cfg = {kSchedMB, 0, 0, 1, 0, 1};
    float tuned_ms = 0.0f;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
};

namespace {

// stage 1: the classification launch(es); stage 2: the motion search;
// 0: both; 3 + k: the search of pair round k (sparse schedule, pair rounds).
int batch_enqueue(sme_batch* b, cudaStream_t s, int stage = 0)
{
    if (b->cfg.schedule == kSchedCluster) return SME_ERR_ARG;  // single sequences only
    if (stage >= 3 && b->cfg.schedule != kSchedSparse) return SME_ERR_ARG;
    if (b->cfg.schedule == kSchedSparse) {
        if (stage <= 1 &&
            launch_sparse_prep(sparse_args(b->sp, (SeqDesc*)b->descs.p, b->status), nullptr, s) != cudaSuccess)
            return SME_ERR_CUDA;
        if (stage == 1) return SME_OK;
        MeArgs a{};
        a.seqs = (const SeqDesc*)b->descs.p;
        a.ready = (unsigned long long*)b->ready.p;
        a.status = b->status;
        a.m = b->m;
        a.total = (int)b->total_mbs;
        a.fault_ticket = -1;
        a.speculate = b->cfg.speculate;
        a.timeout_ns = kDefaultTimeoutNs;
        if (stage >= 3)  // one pair round
            return launch_sparse_search(b->m, a, b->sp, b->num_sms, b->cfg.mb_ctas_per_sm, s, stage - 3);
        if (!b->sp.pair_keys) return launch_sparse_search(b->m, a, b->sp, b->num_sms, b->cfg.mb_ctas_per_sm, s);
        for (int k = 0; k < b->sp.rounds; ++k)
            if (int rc = launch_sparse_search(b->m, a, b->sp, b->num_sms, b->cfg.mb_ctas_per_sm, s, k)) return rc;
        return SME_OK;
    }
    ClassifyBatchArgs ca{(const SeqDesc*)b->descs.p, (const int*)b->fseq.p, (const int*)b->ffrm.p, b->status};
    if (stage != 2 && launch_classify_batch(ca, b->max_mbh, b->total_frames, s) != cudaSuccess) return SME_ERR_CUDA;
    if (stage == 1) return SME_OK;
    MeArgs a{};
    a.seqs = (const SeqDesc*)b->descs.p;
    a.sched = (const int*)b->sched.p;
    a.sched_seq = (const int*)b->sched_seq.p;
    a.unit_seq = (const int*)b->unit_seq.p;
    a.unit_pair = (const int*)b->unit_pair.p;
    a.tmaps = (const CUtensorMap*)b->maps.p;
    a.total_units = b->total_units;
    a.mbw_max = b->mbw_max;
    a.ready = (unsigned long long*)b->ready.p;
    a.status = b->status;
    a.m = b->m;
    a.total = (int)b->total_mbs;
    a.fault_ticket = -1;
    a.speculate = b->cfg.speculate;
    a.pair_direct = b->four_mv ? 0 : b->cfg.pair_direct;
    a.four_mv = b->four_mv;
    a.timeout_ns = kDefaultTimeoutNs;
    if (b->four_mv) {  // three ready words per MB (blocks 0, 1, 2)
        a.ready_a = a.ready + b->total_mbs;
        a.ready_bc = a.ready + 2 * b->total_mbs;
    }
    if (b->cfg.schedule == kSchedPair) {
        int nw = b->cfg.pair_warps > 0 ? b->cfg.pair_warps : kPairWarpsMax;
        if (a.pair_direct) nw = std::min(nw, 8);  // the direct instantiation's bound
        while (nw > 1 && me_pair_smem_bytes(b->m.S, nw, b->mbw_max, b->four_mv != 0) > (size_t)b->smem_optin) --nw;
        int per_sm = 0;
        if (me_pair_occupancy(b->m.S, nw, b->mbw_max, a.pair_direct != 0, b->four_mv != 0, &per_sm) != cudaSuccess ||
            per_sm < 1)
            return SME_ERR_CUDA;
        const int grid = std::max(1, std::min(b->num_sms * per_sm, b->total_units));
        MapSet unused;
        memset(&unused, 0, sizeof(unused));
        return cuda_status(launch_me_pair(b->m, a, &unused, nw, grid, s));
    }
    int resident = b->me_blocks_per_sm;
    if (b->four_mv && (me4_occupancy(b->m.S, &resident) != cudaSuccess || resident < 1)) return SME_ERR_CUDA;
    const int per_sm = b->cfg.mb_ctas_per_sm > 0 ? std::min(b->cfg.mb_ctas_per_sm, resident) : resident;
    const long long want = (b->total_mbs + kMeWarps - 1) / kMeWarps;
    const int grid = (int)std::max(1LL, std::min<long long>((long long)b->num_sms * per_sm, want));
    return cuda_status(b->four_mv ? launch_me4(b->m, a, grid, s) : launch_me(b->m, a, grid, s));
}

void batch_drop_graph(sme_batch* b)
{
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    b->exec = nullptr;
    b->graph = nullptr;
}

// Capture one pass in a CUDA graph on the private stream; without a graph the
// batch simply launches directly.
void batch_capture(sme_batch* b)
{
    batch_drop_graph(b);
    if (cudaStreamBeginCapture(b->cap_stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
        cudaGetLastError();
        return;
    }
    const int rc = batch_enqueue(b, b->cap_stream);
    cudaGraph_t g = nullptr;
    const cudaError_t e = cudaStreamEndCapture(b->cap_stream, &g);
    if (rc != SME_OK || e != cudaSuccess || !g) {
        if (g) cudaGraphDestroy(g);
        cudaGetLastError();
        return;
    }
    if (cudaGraphInstantiate(&b->exec, g, 0) != cudaSuccess) {
        cudaGraphDestroy(g);
        b->exec = nullptr;
        cudaGetLastError();
        return;
    }
    b->graph = g;
}

int batch_read_status(sme_batch* b)
{
    int err = 0;
    if (cudaMemcpy(&err, &b->status->err, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) return SME_ERR_CUDA;
    if (err && cudaMemset(&b->status->err, 0, sizeof(int)) != cudaSuccess) return SME_ERR_CUDA;
    return err;
}

}  // namespace

extern "C" {

int sme_batch_create(sme_batch** out, const sme_params* p, const sme_sequence* seqs, int n, void* stream)
{
    if (!out || !seqs || n < 1) return SME_ERR_ARG;
    *out = nullptr;
    sme_params q = p ? *p : sme_params{};
    if (!p) return SME_ERR_ARG;
    q.width = seqs[0].width;
    q.height = seqs[0].height;
    int rc = check_params(&q);
    if (rc) return rc;
    const int rd = p->ref_distance;
    for (int i = 0; i < n; ++i) {
        const sme_sequence& x = seqs[i];
        if (x.width <= 0 || x.height <= 0 || x.width % 16 || x.height % 16 || x.width > kMaxDim ||
            x.height > kMaxDim)
            return SME_ERR_SIZE;
        if (!x.luma || !x.alpha || !x.out.mv || x.n_frames <= rd || !aligned16(x.luma) || !aligned16(x.alpha))
            return SME_ERR_ARG;
        if (x.seed && p->max_iters > kMaxSeededIters) return SME_ERR_ARG;
    }
    sme_batch* b = new (std::nothrow) sme_batch();
    if (!b) return SME_ERR_NOMEM;
    b->prm = *p;
    b->m = make_method(*p);
    b->stream = (cudaStream_t)stream;
    b->n = n;
    auto fail = [&](int code) {
        sme_batch_destroy(b);
        return code;
    };
    if (cudaGetDevice(&b->device) != cudaSuccess ||
        cudaDeviceGetAttribute(&b->num_sms, cudaDevAttrMultiProcessorCount, b->device) != cudaSuccess ||
        cudaDeviceGetAttribute(&b->smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, b->device) != cudaSuccess ||
        me_occupancy(b->m.S, &b->me_blocks_per_sm) != cudaSuccess || b->me_blocks_per_sm < 1 ||
        cudaStreamCreateWithFlags(&b->cap_stream, cudaStreamNonBlocking) != cudaSuccess) {
        cudaGetLastError();
        return fail(SME_ERR_CUDA);
    }
    if (cudaMalloc(&b->status, sizeof(DevStatus)) != cudaSuccess ||
        cudaMemset(b->status, 0, sizeof(DevStatus)) != cudaSuccess) {
        cudaGetLastError();
        return fail(SME_ERR_NOMEM);
    }
    // Geometry, scratch offsets and descriptors.
    std::vector<SeqDesc> d(n);
    size_t packed_words = 0, cls_bytes = 0;
    long long gid = 0;
    int max_steps = 0;
    std::vector<int> fseq, ffrm;
    for (int i = 0; i < n; ++i) {
        const sme_sequence& x = seqs[i];
        SeqDesc& e = d[i];
        e = SeqDesc{};
        e.W = x.width;
        e.H = x.height;
        e.MBW = x.width / 16;
        e.MBH = x.height / 16;
        e.M = e.MBW * e.MBH;
        e.Wp = (((x.width + 31) / 32 + 1) + 3) & ~3;
        e.F = x.n_frames;
        e.P = x.n_frames - rd;
        e.rd = rd;
        e.gid_base = (int)gid;
        gid += (long long)e.P * e.M;
        packed_words += (size_t)e.F * e.H * e.Wp;
        cls_bytes += (size_t)e.F * e.M;
        b->total_frames += e.F;
        b->max_mbh = std::max(b->max_mbh, e.MBH);
        b->mbw_max = std::max(b->mbw_max, e.MBW);
        b->total_units += e.P;
        max_steps = std::max(max_steps, (e.MBW - 1) + 2 * (e.MBH - 1) + e.P);
        for (int f = 0; f < e.F; ++f) {
            fseq.push_back(i);
            ffrm.push_back(f);
        }
    }
    if (gid > (long long)INT32_MAX) return fail(SME_ERR_SIZE);
    b->total_mbs = gid;
    if ((rc = ensure(b->packed, packed_words * 4)) || (rc = ensure(b->cls, cls_bytes)) ||
        (rc = ensure(b->ready, (size_t)gid * 8, true, nullptr)) || (rc = ensure(b->descs, sizeof(SeqDesc) * n)) ||
        (rc = ensure(b->fseq, fseq.size() * 4)) || (rc = ensure(b->ffrm, ffrm.size() * 4)) ||
        (rc = ensure(b->maps, sizeof(MapSet) * n)))
        return fail(rc);
    size_t po = 0, co = 0;
    std::vector<MapSet> maps(n);
    for (int i = 0; i < n; ++i) {
        const sme_sequence& x = seqs[i];
        SeqDesc& e = d[i];
        e.luma = x.luma;
        e.alpha = x.alpha;
        e.packed_w = (uint32_t*)b->packed.p + po;
        e.cls_w = (uint8_t*)b->cls.p + co;
        e.packed = e.packed_w;
        e.cls = e.cls_w;
        b->cls_off.push_back(co);
        e.temporal_in = x.temporal_in;
        e.seed = x.seed;
        e.mv = x.out.mv;
        e.cost = x.out.cost;
        e.disp = x.out.disp;
        e.iters = x.out.iters;
        e.npos = x.out.npos;
        e.out_cls = x.out.mb_class;
        e.sse_mb = x.out.sse_mb;
        e.sse = x.out.sse;
        e.pred = x.out.pred;
        po += (size_t)e.F * e.H * e.Wp;
        co += (size_t)e.F * e.M;
        Geom g{e.W, e.H, e.M, e.MBW, e.MBH, e.Wp};
        if ((rc = encode_pair_maps(&maps[i], x.luma, e.packed_w, g, e.F, b->m.S))) return fail(rc);
    }
    // Per-MB schedule: every MB of every sequence by wavefront step.
    std::vector<int> sched((size_t)gid), sseq((size_t)gid);
    size_t k = 0;
    for (int t = 0; t < max_steps; ++t)
        for (int i = 0; i < n; ++i) {
            const SeqDesc& e = d[i];
            for (int pr = 0; pr < e.P && pr <= t; ++pr)
                for (int v = 0; v < e.MBH; ++v) {
                    const int u = t - 2 * v - pr;
                    if (u < 0) break;
                    if (u < e.MBW) {
                        sched[k] = e.gid_base + pr * e.M + v * e.MBW + u;
                        sseq[k] = i;
                        ++k;
                    }
                }
        }
    if (k != (size_t)gid) return fail(SME_ERR_STATE);
    if ((rc = setup_sparse(b->sp, d, nullptr))) return fail(rc);
    b->host_desc = d;
    // Per-pair schedule: pair k of every sequence before pair k+1 of any.
    std::vector<int> useq, upair;
    int max_p = 0;
    for (const SeqDesc& e : d) max_p = std::max(max_p, e.P);
    for (int pr = 0; pr < max_p; ++pr)
        for (int i = 0; i < n; ++i)
            if (pr < d[i].P) {
                useq.push_back(i);
                upair.push_back(pr);
            }
    if ((rc = ensure(b->sched, sched.size() * 4)) || (rc = ensure(b->sched_seq, sseq.size() * 4)) ||
        (rc = ensure(b->unit_seq, useq.size() * 4)) || (rc = ensure(b->unit_pair, upair.size() * 4)))
        return fail(rc);
    if (cudaMemcpy(b->descs.p, d.data(), sizeof(SeqDesc) * n, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(b->maps.p, maps.data(), sizeof(MapSet) * n, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(b->fseq.p, fseq.data(), fseq.size() * 4, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(b->ffrm.p, ffrm.data(), ffrm.size() * 4, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(b->sched.p, sched.data(), sched.size() * 4, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(b->sched_seq.p, sseq.data(), sseq.size() * 4, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(b->unit_seq.p, useq.data(), useq.size() * 4, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(b->unit_pair.p, upair.data(), upair.size() * 4, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaDeviceSynchronize() != cudaSuccess) {
        cudaGetLastError();
        return fail(SME_ERR_CUDA);
    }
    *out = b;
    return SME_OK;
}

int sme_batch_tune(sme_batch* b, int trials)
{
    if (!b || trials < 1) return SME_ERR_ARG;
    batch_drop_graph(b);
    float best = -1.0f;
    ExecCfg pick = b->cfg;
    for (const ExecCfg& e : kTuneCandidates) {
        if (b->sp.pair_keys && e.schedule != kSchedSparse) continue;  // pair rounds: the sparse schedule only
        // four vectors per MB: the per-MB schedule and the staged per-pair one
        if (b->four_mv && (e.schedule == kSchedSparse || (e.schedule == kSchedPair && e.pair_direct))) continue;
        b->cfg = e;
        if (batch_enqueue(b, b->stream) != SME_OK || cudaStreamSynchronize(b->stream) != cudaSuccess) {
            cudaGetLastError();
            continue;
        }
        const float ms = time_runs(b->stream, trials, [&] { return batch_enqueue(b, b->stream); });
        if (batch_read_status(b) != SME_OK) continue;
        if (ms > 0.0f && (best < 0.0f || ms < best)) {
            best = ms;
            pick = e;
        }
    }
    b->cfg = pick;
    b->tuned_ms = best > 0.0f ? best : 0.0f;
    batch_capture(b);
    return best > 0.0f ? SME_OK : SME_ERR_CUDA;
}

int sme_batch_run(sme_batch* b)
{
    if (!b) return SME_ERR_ARG;
    if (b->exec) return cuda_status(cudaGraphLaunch(b->exec, b->stream));
    return batch_enqueue(b, b->stream);
}

int sme_batch_run_stage(sme_batch* b, int stage)
{
    if (!b || (stage != 1 && stage != 2)) return SME_ERR_ARG;
    return batch_enqueue(b, b->stream, stage);
}

int sme_batch_set_option(sme_batch* b, int option, int value)
{
    if (!b || option != SME_OPT_FOUR_MV || (value != 0 && value != 1)) return SME_ERR_ARG;
    if (value == b->four_mv) return SME_OK;
    if (value) {
        if (b->sp.pair_keys) return SME_ERR_ARG;
        for (const SeqDesc& d : b->host_desc)
            if (d.seed) return SME_ERR_ARG;  // as in sme_estimate_sequence: no seeds with four vectors
        // the per-MB schedule publishes three words per MB in this mode
        DevBuf bigger;
        if (int rc = ensure(bigger, 3 * (size_t)b->total_mbs * sizeof(unsigned long long), true, b->stream)) return rc;
        if (cudaStreamSynchronize(b->stream) != cudaSuccess) return SME_ERR_CUDA;
        release(b->ready);
        b->ready = bigger;
        b->cfg = ExecCfg{kSchedMB, 0, 0, 1, 0, 1};
    } else if (b->cfg.schedule == kSchedPair) {
        b->cfg.pair_direct = 1;
    }
    batch_drop_graph(b);
    b->tuned_ms = 0.0f;
    b->four_mv = value;
    return SME_OK;
}

int sme_batch_set_pair_rounds(sme_batch* b, int on)
{
    if (!b || (on != 0 && on != 1)) return SME_ERR_ARG;
    if (on && b->four_mv) return SME_ERR_ARG;
    if (on == (b->sp.pair_keys > 0)) return SME_OK;
    int rc = setup_sparse(b->sp, b->host_desc, b->stream, on != 0);
    if (rc) return rc;
    if (cudaStreamSynchronize(b->stream) != cudaSuccess) return SME_ERR_CUDA;
    batch_drop_graph(b);
    if (on) b->cfg = ExecCfg{kSchedSparse, 0, b->cfg.schedule == kSchedSparse ? b->cfg.mb_ctas_per_sm : 2, 0, 0, 1};
    return SME_OK;
}

int sme_batch_run_pair(sme_batch* b, int k)
{
    if (!b || !b->sp.pair_keys || k < 0 || k >= b->sp.rounds) return SME_ERR_ARG;
    return batch_enqueue(b, b->stream, 3 + k);
}

int sme_batch_upload(sme_batch* b, const sme_host_io* io, int n)
{
    if (!b || !io || n != b->n) return SME_ERR_ARG;
    for (int i = 0; i < n; ++i)
        if (!io[i].luma || !io[i].alpha) return SME_ERR_ARG;
    const int K = sme_batch::kCopyStreams;
    if (!b->fork) {
        if (cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming) != cudaSuccess) return SME_ERR_CUDA;
        for (int c = 0; c < K; ++c)
            if (cudaStreamCreateWithFlags(&b->copy[c], cudaStreamNonBlocking) != cudaSuccess ||
                cudaEventCreateWithFlags(&b->join[c], cudaEventDisableTiming) != cudaSuccess)
                return SME_ERR_CUDA;
    }
    // the copies start after the work already queued on the batch's stream
    // (which may still read the buffers) and the stream waits for all of them
    if (cudaEventRecord(b->fork, b->stream) != cudaSuccess) return SME_ERR_CUDA;
    for (int c = 0; c < K; ++c)
        if (cudaStreamWaitEvent(b->copy[c], b->fork, 0) != cudaSuccess) return SME_ERR_CUDA;
    const void* last_luma = nullptr;
    int next = 0;
    // A mapped pinned buffer is read by the SMs (on the batch's stream, after
    // the work queued there); any other buffer goes to the copy engines.
    auto copy = [&](void* dst, const void* src, size_t bytes) {
        const void* m = mapped_host(src);
        if (m && aligned16(m) && aligned16(dst) && bytes % 16 == 0)
            return launch_host_copy(dst, m, bytes, b->num_sms, b->stream) == cudaSuccess;
        return cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, b->copy[next++ % K]) == cudaSuccess;
    };
    for (int i = 0; i < n; ++i) {
        const SeqDesc& d = b->host_desc[i];
        const size_t bytes = (size_t)d.F * d.W * d.H;
        // a luma plane shared with the previous sequence (the same device
        // address: the VOPs of one scene) is copied once
        if (d.luma != last_luma && !copy((void*)d.luma, io[i].luma, bytes)) return SME_ERR_CUDA;
        last_luma = d.luma;
        if (!copy((void*)d.alpha, io[i].alpha, bytes)) return SME_ERR_CUDA;
    }
    for (int c = 0; c < K; ++c)
        if (cudaEventRecord(b->join[c], b->copy[c]) != cudaSuccess ||
            cudaStreamWaitEvent(b->stream, b->join[c], 0) != cudaSuccess)
            return SME_ERR_CUDA;
    return SME_OK;
}

int sme_batch_download(sme_batch* b, const sme_host_io* io, int n)
{
    if (!b || !io || n != b->n) return SME_ERR_ARG;
    for (int i = 0; i < n; ++i) {
        const SeqDesc& d = b->host_desc[i];
        const sme_outputs& h = io[i].out;
        const size_t PM = (size_t)d.P * d.M;
        const struct {
            void* host;
            const void* dev;
            size_t bytes;
        } f[] = {{h.mv, d.mv, PM * sizeof(sme_mv)}, {h.cost, d.cost, PM * 4},         {h.disp, d.disp, PM * 8},
                 {h.iters, d.iters, PM},            {h.npos, d.npos, PM},             {h.mb_class, d.out_cls, PM},
                 {h.sse_mb, d.sse_mb, PM * 4},      {h.sse, d.sse, (size_t)d.P * 8}, {h.pred, d.pred, (size_t)d.P * d.W * d.H}};
        for (const auto& x : f) {
            if (!x.host) continue;
            if (!x.dev) return SME_ERR_ARG;  // not requested at creation
            if (cudaMemcpyAsync(x.host, x.dev, x.bytes, cudaMemcpyDeviceToHost, b->stream) != cudaSuccess)
                return SME_ERR_CUDA;
        }
    }
    return SME_OK;
}

int sme_batch_class_map(sme_batch* b, int seq, const uint8_t** mb_class)
{
    if (!b || !mb_class || seq < 0 || seq >= b->n) return SME_ERR_ARG;
    *mb_class = (const uint8_t*)b->cls.p + b->cls_off[seq];
    return SME_OK;
}

int sme_batch_synchronize(sme_batch* b)
{
    if (!b) return SME_ERR_ARG;
    if (cudaStreamSynchronize(b->stream) != cudaSuccess) return SME_ERR_CUDA;
    return batch_read_status(b);
}

int sme_batch_config(sme_batch* b, int* schedule, int* param, int* flag, float* best_ms)
{
    if (!b) return SME_ERR_ARG;
    if (schedule) *schedule = b->cfg.schedule;
    if (param) *param = b->cfg.schedule == kSchedPair ? b->cfg.pair_warps : b->cfg.mb_ctas_per_sm;
    if (flag) *flag = b->cfg.schedule == kSchedPair ? b->cfg.pair_direct : b->cfg.speculate;
    if (best_ms) *best_ms = b->tuned_ms;
    return SME_OK;
}

int sme_batch_set_config(sme_batch* b, int schedule, int param, int flag)
{
    if (!b) return SME_ERR_ARG;
    ExecCfg e = {schedule, 0, 0, 1, 0, 1};
    if (flag != 0 && flag != 1) return SME_ERR_ARG;
    switch (schedule) {
    case kSchedMB:
        if (param < 0 || param > 32) return SME_ERR_ARG;
        e.mb_ctas_per_sm = param;
        e.speculate = flag;
        break;
    case kSchedSparse:
        if (param < 0 || param > 5 || param == 4) return SME_ERR_ARG;
        e.mb_ctas_per_sm = param;
        e.speculate = flag;
        break;
    case kSchedPair:
        if (param < 0 || param > kPairWarpsMax) return SME_ERR_ARG;
        e.pair_warps = param;
        e.pair_direct = flag;
        e.speculate = 0;
        break;
    default:
        return SME_ERR_ARG;  // the cluster schedule runs single sequences only
    }
    if (b->sp.pair_keys && schedule != kSchedSparse) return SME_ERR_ARG;  // pair rounds: sparse only
    if (b->four_mv && schedule == kSchedSparse) return SME_ERR_ARG;
    batch_drop_graph(b);
    b->cfg = e;
    b->tuned_ms = 0.0f;
    return SME_OK;
}

int sme_batch_destroy(sme_batch* b)
{
    if (!b) return SME_ERR_ARG;
    cudaStreamSynchronize(b->stream);
    batch_drop_graph(b);
    DevBuf* bufs[] = {&b->descs, &b->packed, &b->cls, &b->ready, &b->sched, &b->sched_seq, &b->unit_seq,
                      &b->unit_pair, &b->fseq, &b->ffrm, &b->maps};
    for (DevBuf* x : bufs) release(*x);
    release_sparse(b->sp);
    for (int c = 0; c < sme_batch::kCopyStreams; ++c) {
        if (b->copy[c]) {
            cudaStreamSynchronize(b->copy[c]);
            cudaStreamDestroy(b->copy[c]);
        }
        if (b->join[c]) cudaEventDestroy(b->join[c]);
    }
    if (b->fork) cudaEventDestroy(b->fork);
    if (b->status) cudaFree(b->status);
    if (b->cap_stream) cudaStreamDestroy(b->cap_stream);
    delete b;
    return SME_OK;
}

}  // extern "C"
