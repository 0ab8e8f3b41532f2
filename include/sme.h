/*
 * sme.h -- C ABI of the GB300 shape-adaptive motion estimation library.
 *
 * The library implements, on one GPU, the per-macroblock procedure of
 * Benboubker, Abdi and Ahaitouf, "Shape-Adaptive Motion Estimation Algorithm
 * for MPEG-4 Video Coding": classification of each 16x16 macroblock (MB) from
 * its binary alpha block (BAB) (Fig. 1, Sec. 3.1), the block recursive search
 * over the neighbour and temporal candidates A, B, C, T (Fig. 1, Fig. 3) with
 * a shape cost on boundary MBs and a texture (SAD) cost on opaque MBs, the
 * pixel recursive gradient search of Sec. 3.2 (Eqs. 2-5, Fig. 4) on opaque
 * MBs, and motion compensation with PSNR (Sec. 4).
 *
 * Conventions shared by every call
 *  - Frames are 8-bit, row-major, pitch = width bytes, frame after frame
 *    ([n_frames][height][width]); width and height are multiples of 16.
 *    Luma is gray level; alpha is 0 (outside the object) or nonzero (inside).
 *  - MB m = v * (width/16) + h is the MB at column h, row v.  M = MB count.
 *  - Vectors (sme_mv) are in units of 1/subpel pixel.  The prediction of
 *    current pixel p is reference(p + mv) (backward matching, Sec. 2).
 *  - Valid vectors V: the displaced 16x16 block lies inside the reference
 *    frame and |dx|, |dy| <= search_range * subpel.  Every vector the library
 *    returns lies in V; every candidate is clamped into V before use.
 *  - Pair k of a sequence uses frame k as reference and frame
 *    k + ref_distance as current; P = n_frames - ref_distance pairs.  The
 *    temporal candidate of pair k is the field of pair k-1 (temporal_in, or
 *    zero vectors, for pair 0).
 *  - Unless a call says "host", every data pointer is DEVICE memory owned by
 *    the caller, must stay valid until the work queued on the context's
 *    stream has finished, and is never freed or retained by the library.
 *    Frame pointers must be 16-byte aligned.
 *  - Calls are asynchronous on the context's stream unless they say they
 *    synchronise.  Argument errors are returned immediately; a device-side
 *    failure (a bounded wait that gave up) is reported by the next
 *    sme_synchronize (or by a synchronising call).
 *  - Every call returns an SME_* status; nothing throws or aborts.
 *  - One context serves one stream at a time; calls that overlap on the GPU
 *    through the same context race on its scratch buffers.
 */
#ifndef SME_H
#define SME_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
    SME_OK = 0,
    SME_ERR_ARG = 1,     /* null or out-of-range argument, misaligned pointer */
    SME_ERR_SIZE = 2,    /* width/height not a positive multiple of 16, or too large */
    SME_ERR_CUDA = 3,    /* a CUDA runtime call failed */
    SME_ERR_TIMEOUT = 4, /* a bounded device wait gave up (results are incomplete) */
    SME_ERR_STATE = 5,   /* call made in the wrong state (e.g. estimate before set_current) */
    SME_ERR_NOMEM = 6,   /* device or host allocation failed */
    SME_ERR_RANGE = 7,   /* a caller-supplied vector lies outside V */
    SME_ERR_SCRATCH = 8  /* problem larger than sme_estimate_sequence_noalloc's fixed scratch */
};

enum { SME_TRANSPARENT = 0, SME_OPAQUE = 1, SME_BOUNDARY = 2 };

typedef struct sme_ctx sme_ctx;

typedef struct {
    int width, height;  /* pixels, multiples of 16, 16..8192 */
    int search_range;   /* S in pixels, 1..64 (window (2S+1)^2, Eq. 6) */
    int subpel;         /* 1 = full-pel, 2 = half-pel (MPEG-4 bilinear, rounding control 0) */
    float theta;        /* Theta of Eq. 4 (gradient threshold), > 0; default 2 */
    float epsilon;      /* convergence factor of Eq. 2, (0, 4]; default 1 */
    int max_iters;      /* cap on pixel-recursive iterations, 0..16; default 8 */
    int ref_distance;   /* frames between reference and current, >= 1; default 1 */
} sme_params;

typedef struct {
    int16_t dx, dy;
} sme_mv;

/* Per-MB and per-pair results of an estimate.  `mv` is required; every other
 * pointer may be NULL.  Sizes are for P pairs of M MBs. */
typedef struct {
    sme_mv* mv;               /* [P][M] final vectors */
    uint32_t* cost;           /* [P][M] final cost: SAD (opaque) or alpha mismatches (boundary) */
    float* disp;              /* [P][M][2] last FP32 gradient update (pixels), Eq. 3; 0 if none */
    uint8_t* iters;           /* [P][M] pixel-recursive iterations run */
    uint8_t* npos;            /* [P][M] distinct vectors whose cost was evaluated (Table 1 unit) */
    uint8_t* mb_class;        /* [P][M] class of the current frame's MB (SME_TRANSPARENT...) */
    uint32_t* sse_mb;         /* [P][M] sum of squared prediction errors of the MB */
    unsigned long long* sse;  /* [P] whole-frame sum of squared prediction errors */
    uint8_t* pred;            /* [P][height][width] motion-compensated prediction */
} sme_outputs;

/* Fill *p with the defaults above for a width x height sequence. */
void sme_default_params(sme_params* p, int width, int height);

/* Static text for a status code. */
const char* sme_strerror(int status);

/* Create a context bound to the current CUDA device and to `cuda_stream`
 * (a cudaStream_t; NULL = the legacy default stream).  Allocates the
 * context's own device scratch (packed alpha, class map, ready flags),
 * grown on demand by later calls.  Returns SME_ERR_ARG/SIZE on bad params. */
int sme_create(sme_ctx** out, const sme_params* p, void* cuda_stream);

/* Free the context and its device scratch (synchronises its stream). */
int sme_destroy(sme_ctx* ctx);

/* Rebind the context to another stream. */
int sme_set_stream(sme_ctx* ctx, void* cuda_stream);

/* Wait for the context's stream, then report (and clear) a device-side
 * failure of the work queued since the previous sme_synchronize. */
int sme_synchronize(sme_ctx* ctx);

/* Fig. 1 "Block_Type": classify every MB of `n_frames` alpha frames.
 *   alpha    [n_frames][H][W] device, 16-byte aligned
 *   mb_class [n_frames][M] device out: 0 transparent (no pixel inside),
 *            1 opaque (all 256 inside), 2 boundary
 *   packed   optional device out [n_frames][H][sme_packed_words(W)] uint32:
 *            bit b of word k of a row = (alpha[32k+b] != 0); trailing words 0
 *            (at least one, rows padded to a multiple of 4 words). */
int sme_classify(sme_ctx* ctx, const uint8_t* alpha, int n_frames, uint8_t* mb_class,
                 uint32_t* packed);
/* Fig. 1 Block_Type of n frames gathered from anywhere, in one launch:
 * frames is a DEVICE array of n pointers to [height][width] alpha planes of
 * the context's size (each 16-byte aligned; a NULL entry stands for an empty
 * plane, every MB transparent); mb_class [n][M] (device out).  SME_ERR_ARG on
 * bad arguments. */
int sme_classify_table(sme_ctx* ctx, const uint8_t* const* frames, int n, uint8_t* mb_class);

/* Words per row of the packed alpha layout above. */
int sme_packed_words(int width);

/* The whole per-MB pass of Fig. 1 over a sequence (classification, block
 * recursive search, pixel recursive search, motion compensation and SSE),
 * for all P pairs in one persistent launch.
 *   luma, alpha  [n_frames][H][W] device
 *   temporal_in  [M] device or NULL: temporal candidates of pair 0
 *   seed         [P][M][2] device FP32 pixels or NULL: an extra candidate per
 *                MB evaluated after T (rounded to the MV grid, clamped to V).
 *                Accepted only with max_iters <= 8 (SME_ERR_ARG otherwise):
 *                an MB whose seed wins runs two pixel-recursive searches, and
 *                the per-MB record of evaluated positions holds both only up
 *                to that cap.
 *   out          outputs as described in sme_outputs (device pointers)
 * Needs n_frames > ref_distance. */
int sme_estimate_sequence(sme_ctx* ctx, const uint8_t* luma, const uint8_t* alpha, int n_frames,
                          const sme_mv* temporal_in, const float* seed, const sme_outputs* out);

/* Same as sme_estimate_sequence with every pointer (inputs and outputs) in
 * HOST memory, and synchronises before returning.  The luma frames are
 * copied to a context-owned device buffer.  A pinned (page-locked) alpha is
 * read in place by the classification, and pinned outputs other than sse are
 * written in place by the kernels over the CPU-GPU link; pageable ones go
 * through context-owned device buffers and copies.  The results are the same
 * either way. */
int sme_estimate_sequence_host(sme_ctx* ctx, const uint8_t* luma, const uint8_t* alpha,
                               int n_frames, const sme_mv* temporal_in, const float* seed,
                               const sme_outputs* out);

/* Stateful pair interface (Sec. 2 problem statement: find, for every block
 * of the current frame, the vector minimising the matching error against
 * the reference).  set_reference / set_current copy one luma + alpha frame
 * (device) into context-owned buffers.  sme_estimate runs one pair with the
 * context's temporal field as T and keeps the result; sme_advance makes the
 * current frame the reference and the result the temporal field.  sme_score
 * synchronises and returns the PSNR (dB) of the last estimate's prediction. */
int sme_set_reference(sme_ctx* ctx, const uint8_t* luma, const uint8_t* alpha);
int sme_set_current(sme_ctx* ctx, const uint8_t* luma, const uint8_t* alpha);
int sme_estimate(sme_ctx* ctx, const sme_outputs* out /* P = 1; may be NULL */);
int sme_advance(sme_ctx* ctx);
int sme_score(sme_ctx* ctx, double* psnr_db);
int sme_get_temporal_field(sme_ctx* ctx, sme_mv* field /* [M] device out */);
int sme_set_temporal_field(sme_ctx* ctx, const sme_mv* field /* [M] device, NULL = zeros */);
/* Seeds of the pair interface (the learned proposal; the paper's own seeds
 * are the neighbour and temporal vectors of Sec. 3.1): seed [M][2] device
 * FP32 pixels, copied into a context-owned buffer and used by every following
 * sme_estimate as the fifth candidate of each MB exactly as the `seed`
 * argument of sme_estimate_sequence (rounded to the MV grid, clamped to V,
 * plain search as fallback), until replaced, or cleared with NULL.
 * SME_ERR_ARG with max_iters > 8 or in the four-vector mode. */
int sme_set_seed_field(sme_ctx* ctx, const float* seed);

/* Motion compensation of one frame pair with a caller-supplied field (Sec. 4):
 * pred(p) = ref(p + mv(mb(p))) with half-sample interpolation, and the SSE
 * against cur.  Every vector must lie in V: otherwise the MB is skipped and
 * the next sme_synchronize returns SME_ERR_RANGE.
 *   ref, cur [H][W] device; mv [M] device; pred [H][W] device or NULL;
 *   sse one device unsigned long long (overwritten). */
int sme_compensate(sme_ctx* ctx, const uint8_t* ref, const uint8_t* cur, const sme_mv* mv,
                   uint8_t* pred, unsigned long long* sse);

/* PSNR in dB of an 8-bit width x height frame from its SSE (Sec. 4);
 * +infinity when sse == 0.  Host only. */
double sme_psnr(unsigned long long sse, int width, int height);

/* Cost queries through the same device code as the estimate.  queries is
 * [n][3] int32 device (mb, dx, dy) with (dx, dy) in V of that MB.  Outputs
 * [n] device, either may be NULL: the texture SAD of the 16x16 block
 * (Fig. 1 opaque branch) and the alpha mismatch count (boundary branch,
 * full-pel part trunc(d/subpel)).  ref/cur luma [H][W], aref/acur alpha. */
int sme_eval_costs(sme_ctx* ctx, const uint8_t* ref, const uint8_t* cur, const uint8_t* aref,
                   const uint8_t* acur, const int32_t* queries, int n, uint32_t* texture_sad,
                   uint32_t* shape_sad);

/* One FP32 gradient update (Eqs. 3-5) per query (mb, dx, dy) through the
 * same device code as the estimate; delta [n][2] device out, in pixels. */
int sme_gradient_step(sme_ctx* ctx, const uint8_t* ref, const uint8_t* cur,
                      const int32_t* queries, int n, float* delta);

/* Execution options (no counterpart in the paper: they choose how the
 * raster dependency of Fig. 1 is mapped onto the GPU, never what is computed;
 * every option gives bit-identical results).
 *   SME_OPT_SCHEDULE: SME_SCHED_PAIR -- one CTA per frame pair, one warp per
 *     MB row, the row above handed over in shared memory and the reference
 *     windows fetched by TMA; SME_SCHED_MB -- one warp per MB, tickets in
 *     wavefront order, every dependency through global memory;
 *     SME_SCHED_CLUSTER -- one thread-block cluster per sequence (single
 *     sequences only): the MBs dealt in wavefront order to the cluster's
 *     CTAs, every vector stored by its producer straight into the shared
 *     memory of the CTAs that consume it (distributed shared memory), so no
 *     dependency is polled through L2; SME_ERR_SIZE when the sequence needs
 *     more shared memory than a cluster has;
 *     SME_SCHED_SPARSE -- for inputs where most MBs are transparent: one
 *     streaming pass reads every alpha plane once, classifies and packs it
 *     and finishes the transparent MBs (Fig. 1 gives them (0,0); their
 *     co-located prediction error is computed once per luma plane shared
 *     by several VOPs), then the per-MB search runs over a list of the
 *     other MBs in wavefront order, taking a transparent neighbour's (0,0)
 *     from the class map without waiting (never speculatively);
 *     SME_OPT_MB_CTAS_PER_SM 2 or 3 selects the search kernel built for
 *     that many resident 8-warp CTAs per SM, 5 the one built for five
 *     4-warp CTAs per SM, else one 8-warp CTA;
 *     SME_SCHED_AUTO (default) -- chosen per workload.
 *   SME_OPT_PAIR_WARPS: warps (MB rows in flight) per CTA of the pair
 *     schedule, 1..16 (at most 8 used with SME_OPT_PAIR_DIRECT); 0
 *     (default) = automatic.
 *   SME_OPT_MB_CTAS_PER_SM: resident CTAs (8 MBs each) per SM of the per-MB
 *     schedule, 1..32, capped by occupancy; 0 (default) = as many as fit.
 *   SME_OPT_SPECULATE: 1 (default) = in the per-MB schedule, cost each
 *     candidate as soon as its vector arrives and take the first
 *     pixel-recursive step at the first costed position while the other
 *     candidates are awaited; 0 = do all of it after the last arrival.
 *   SME_OPT_CLUSTER_SIZE: CTAs per cluster of the cluster schedule, 2, 4, 8
 *     or 16; 0 (default) = 16, halved until the cluster fits.
 *   SME_OPT_PAIR_DIRECT: 1 (default) = in the pair schedule, runs of
 *     transparent MBs (known from the classification launch) are finished
 *     straight from global memory, four at a time, and only the other MBs
 *     are staged by TMA; 0 = every MB is staged.
 *   SME_OPT_FOUR_MV: 1 = four vectors per MB (Sec. 3.2: MPEG-4's four
 *     vectors per macroblock, the recursive search on 8x8 blocks).  The
 *     block recursive search stays at MB level (Fig. 1, 16x16 costs) and its
 *     winner starts the pixel recursive search of each 8x8 block
 *     b = 2*by + bx; the candidates of an MB are block 1 of the left MB (A),
 *     block 2 of the MBs above and above-right (B, C) and block 0 of the same
 *     MB in the previous field (T); boundary MBs give the winner to all four
 *     blocks, each costed by the alpha mismatches of its quadrant.  Changes
 *     the layout of the estimate outputs: mv, cost, iters, npos become
 *     [P][M][4] and disp [P][M][4][2] (block-major inside each MB);
 *     temporal_in becomes [M][4]; mb_class, sse_mb, sse, pred keep theirs.
 *     Runs on the per-MB schedule or the pair schedule with every MB staged
 *     (whatever SME_OPT_PAIR_DIRECT says); seeds and
 *     SME_OPT_BOUNDARY_T_TEXTURE are rejected (SME_ERR_ARG);
 *     sme_estimate_sequence* (batches: sme_batch_set_option).  0 (default)
 *     = one vector per MB.
 *   SME_OPT_BOUNDARY_T_TEXTURE: 1 = Sec. 3.1's prose for boundary MBs: the
 *     spatial candidates (and a seed) are judged by shape, the temporal one
 *     by texture -- the first strict minimum of the others by alpha
 *     mismatches is compared with T by 16x16 texture SAD and T is kept only
 *     if strictly lower; the reported cost is the alpha mismatch count of the
 *     vector kept.  0 (default) = Fig. 1: all candidates by shape.
 * Returns SME_ERR_ARG for an unknown option or value. */
enum {
    SME_OPT_SCHEDULE = 1,
    SME_OPT_PAIR_WARPS = 2,
    SME_OPT_MB_CTAS_PER_SM = 3,
    SME_OPT_SPECULATE = 4,
    SME_OPT_CLUSTER_SIZE = 5,
    SME_OPT_PAIR_DIRECT = 6,
    SME_OPT_FOUR_MV = 7,
    SME_OPT_BOUNDARY_T_TEXTURE = 8
};
enum { SME_SCHED_AUTO = 0, SME_SCHED_MB = 1, SME_SCHED_PAIR = 2, SME_SCHED_CLUSTER = 3, SME_SCHED_SPARSE = 4 };
int sme_set_option(sme_ctx* ctx, int option, int value);
/* Exhaustive search (the ES of Sec. 1 / Table 1 / Table 2, the comparison
 * method of the paper's experiments; not part of the method): for every MB
 * of every pair (frame k, frame k + ref_distance) of a [n_frames][H][W] luma
 * sequence (device, 16-byte aligned), the texture SAD at every vector of the
 * valid set V of the context's parameters (search range, subpel) and the
 * first minimum in raster order (dy outer, dx inner).  Every MB of the frame
 * grid, whatever its class.  mv [P][M] (device out), sad [P][M] (device out,
 * optional).  Asynchronous on the context's stream; SME_ERR_SIZE if the
 * search window does not fit in shared memory. */
int sme_full_search(sme_ctx* ctx, const uint8_t* luma, int n_frames, sme_mv* mv, uint32_t* sad);
/* Measurement helper (no counterpart in the paper): the device's rate of the
 * packed-SAD operation mix that the integer roofline of the search and of
 * the exhaustive search counts -- per 32-bit word of a row, one funnel-shift
 * alignment, one __vsadu4 absolute difference and one add -- on independent
 * register-resident chains over the whole GPU.  Launches ctas_per_sm (1..8)
 * CTAs of 256 threads per SM on cuda_stream, each thread running iters steps
 * of 8 chains (24 operations per step), and writes one word per thread to
 * out (device, [grid * 256] uint32) so that the work is kept; *grid (host)
 * receives the number of CTAs.  The caller times the launch on the stream:
 * operations = grid * 256 * iters * 24.  SME_ERR_ARG on other values. */
int sme_packed_sad_rate_launch(int ctas_per_sm, int iters, uint32_t* out, void* cuda_stream, int* grid);

/* The current value of an option (e.g. what sme_autotune chose). */
int sme_get_option(sme_ctx* ctx, int option, int* value);

/* Autotuner for a context: runs the estimate on the given sequence once per
 * candidate execution configuration (schedule, CTAs per SM, speculation,
 * pair-schedule warps -- see sme_set_option), `trials` times each, and keeps
 * the fastest by device time.  Every configuration computes bit-identical
 * results, so the choice changes only speed.  Arguments as for
 * sme_estimate_sequence; synchronises.  No counterpart in the paper. */
int sme_autotune(sme_ctx* ctx, const uint8_t* luma, const uint8_t* alpha, int n_frames,
                 const sme_outputs* out, int trials);

/* Batches: many independent sequences (each one VOP, Sec. 1: every object
 * is coded as its own plane) of uneven frame size and length, estimated by
 * one classification launch and one persistent ME launch whose tickets
 * interleave all sequences by wavefront step.  The method parameters
 * (search range, subpel, Theta, eps, max_iters, ref_distance) are shared;
 * width/height come from each sequence.  Every pointer in sme_sequence is
 * caller-owned device memory that must stay valid (and keep its address)
 * for the life of the batch, because sme_batch_run replays the same work.
 *   sme_batch_create   validates, allocates scratch, builds the schedule.
 *   sme_batch_tune     times the candidate execution configurations
 *                      (`trials` runs each), keeps the fastest, captures
 *                      the launches in a CUDA graph; synchronises.
 *   sme_batch_run      enqueues one pass over all sequences (graph replay
 *                      once tuned) on the batch's stream.
 *   sme_batch_synchronize  waits and reports a device-side failure.
 *   sme_batch_config   the configuration in use (schedule SME_SCHED_*,
 *                      its parameter: CTAs per SM for SME_SCHED_MB (0 = all
 *                      that fit) and SME_SCHED_SPARSE, or warps for
 *                      SME_SCHED_PAIR, speculation)
 *                      and the tuned time per run in ms (0 before tuning).
 *   sme_batch_set_config  sets the configuration instead of tuning: schedule
 *                      SME_SCHED_MB (param = CTAs per SM, 0..32, 0 = all that
 *                      fit; flag = speculation), SME_SCHED_PAIR (param =
 *                      warps per CTA, 0..16, 0 = automatic; flag = direct
 *                      transparent runs) or SME_SCHED_SPARSE (param 0..3 or 5:
 *                      2, 3 = the search kernel built for that many 8-warp
 *                      CTAs per SM, 5 = for five 4-warp CTAs; flag 0 or 1,
 *                      unused); drops a captured graph (later runs
 *                      launch directly until sme_batch_tune).  SME_ERR_ARG on
 *                      other values.
 * Results per sequence are exactly those of sme_estimate_sequence on it. */
typedef struct {
    int width, height, n_frames;
    const uint8_t* luma;        /* [n_frames][height][width] */
    const uint8_t* alpha;       /* [n_frames][height][width] */
    const sme_mv* temporal_in;  /* [M] or NULL */
    const float* seed;          /* [P][M][2] or NULL */
    sme_outputs out;
} sme_sequence;

typedef struct sme_batch sme_batch;

int sme_batch_create(sme_batch** out, const sme_params* p, const sme_sequence* seqs, int n,
                     void* cuda_stream);
int sme_batch_tune(sme_batch* b, int trials);
int sme_batch_run(sme_batch* b);
int sme_batch_synchronize(sme_batch* b);
/* The batch's execution configuration (after sme_batch_tune: the chosen
 * one): schedule (SME_SCHED_*), param (pair schedule: warps per CTA; per-MB
 * schedule: CTAs per SM, 0 = as many as fit), flag (pair schedule:
 * SME_OPT_PAIR_DIRECT; per-MB schedule: SME_OPT_SPECULATE) and the tuned time
 * of one run in ms (0 before tuning).  Any output pointer may be NULL. */
int sme_batch_config(sme_batch* b, int* schedule, int* param, int* flag, float* best_ms);
int sme_batch_set_config(sme_batch* b, int schedule, int param, int flag);
/* Two-stage run, for callers that compute seeds from the batch's own MB
 * classes (the learned proposal): sme_batch_run_stage(b, 1) enqueues the
 * classification (and, in the sparse schedule, the transparent MBs' results
 * and the list of the others); afterwards the class map of sequence `seq`,
 * [n_frames][M] uint8 on the device (classes of every frame, as sme_classify
 * writes them), is at the address sme_batch_class_map returns, valid until
 * the next run; seeds written before sme_batch_run_stage(b, 2), which
 * enqueues the search, are used by it.  Both launch directly on the batch's
 * stream (no graph; a caller may capture them).  SME_ERR_ARG on a bad stage
 * or sequence index. */
int sme_batch_run_stage(sme_batch* b, int stage);
int sme_batch_class_map(sme_batch* b, int seq, const uint8_t** mb_class);
/* Pair rounds (sparse schedule only), for callers whose seeds for pair k
 * depend on the field of pair k - 1 (the learned proposal with the previous
 * field as input): sme_batch_set_pair_rounds(b, 1) lists the non-transparent
 * MBs pair by pair (and selects the sparse schedule; synchronises), so that
 * after stage 1, sme_batch_run_pair(b, k) for k = 0, 1, ... (in this order,
 * each after the previous one on the batch's stream) searches pair k of every
 * sequence, its temporal candidates being the results of round k - 1; stage
 * 2 runs every round in order.  Results are those of sme_batch_run.
 * sme_batch_set_pair_rounds(b, 0) returns to the whole-list order.
 * SME_ERR_ARG for k outside [0, largest pair count) or without pair rounds;
 * other schedules are then rejected by sme_batch_set_config. */
int sme_batch_set_pair_rounds(sme_batch* b, int on);
int sme_batch_run_pair(sme_batch* b, int k);
/* Options of a batch: SME_OPT_FOUR_MV 1 = four vectors per MB for every
 * sequence (Sec. 3.2, as for a context: the outputs given at creation must
 * have the four-vector layout [P][M][4], temporal_in [M][4]); the batch then
 * runs the per-MB schedule or the staged per-pair one (tuned between them);
 * SME_ERR_ARG with seeds, pair rounds, another option or value. */
int sme_batch_set_option(sme_batch* b, int option, int value);
/* Host-memory inputs and outputs of a batch.  sme_batch_upload copies io[i]
 * (HOST luma and alpha, [n_frames][H][W] of sequence i; n = the batch's
 * sequence count) into the device buffers the batch was created with, on the
 * batch's stream; a luma plane that sequence i shares with sequence i - 1
 * (the same device address: the VOPs of one scene) is copied once.
 * A page-locked (pinned) host buffer whose device mapping, the device
 * buffer and the size are 16-byte aligned is copied by a kernel whose
 * threads read it through that mapping, over the whole GPU (on the
 * CPU-GPU link of a GB300 node this moves about 1.5 times the bytes per
 * second of the copy engines); any other buffer is copied with
 * cudaMemcpyAsync on four internal streams forked from and joined back to
 * the batch's stream.
 * sme_batch_download copies every non-NULL HOST pointer of io[i].out from
 * the matching device output of sequence i (SME_ERR_ARG if that output was
 * not requested at creation).  Both are asynchronous on the batch's stream
 * (page-locked host buffers let the copies run at link speed) and finish
 * by sme_batch_synchronize; upload -> run -> download -> synchronize is the
 * whole host-to-host pass. */
typedef struct {
    const uint8_t* luma;
    const uint8_t* alpha;
    sme_outputs out;
} sme_host_io;
int sme_batch_upload(sme_batch* b, const sme_host_io* io, int n);
int sme_batch_download(sme_batch* b, const sme_host_io* io, int n);
int sme_batch_destroy(sme_batch* b);

/* Learned seed proposal (no counterpart in the paper, whose seeds are the
 * neighbour and temporal vectors of Sec. 3.1): a 5-layer 3x3 convolutional
 * network, 32 channels, bfloat16 weights and activations with FP32
 * accumulation on tensor cores, on a quarter-resolution grid (cell = 4x4
 * pixels, MB = 4x4 cells).  Inputs per cell (16 channels, bfloat16): current
 * and reference mean luma /255 - 0.5, their difference, the temporal
 * candidate of the cell's MB in pixels / 16, zeros.  Output per MB: a seed
 * (dx, dy) in pixels = 8 x the mean of output channels 0, 1 over its cells;
 * pass the seeds to sme_estimate_sequence (`seed`), where they are a fifth
 * candidate with the plain search as fallback.
 *   Parameters (FP32, sme_seednet_param_count() floats): per layer the
 *   weights [cout][3][3][cin] then the biases [cout]; channels
 *   16, 32, 32, 32, 32, 16.  Training: Huber loss (1 px) between the seeds and
 *   labels (pixels) over the MBs with mask != 0, averaged; Adam (0.9, 0.999,
 *   1e-8) on FP32 master weights.
 *   sme_seednet_create    max_cells = largest n * (W/4) * (H/4) used later.
 *   sme_seednet_features  n_pairs frame pairs (ref_frame + q, cur_frame + q) of a
 *                         [F][H][W] luma sequence (device) -> feat
 *                         [n_pairs][H/4][W/4][16] bfloat16 (device, as uint16);
 *                         a temporal field is accepted only with n_pairs = 1.
 *                         The caller guarantees that frames ref_frame +
 *                         n_pairs - 1 and cur_frame + n_pairs - 1 exist (the
 *                         library does not know F); n_pairs <= 65535.
 *   sme_seednet_forward   n stacked feature grids -> seeds [n][M][2] FP32
 *                         pixels (device, optional) and the raw cell outputs
 *                         [n][H/4][W/4][16] FP32 (device, optional).
 *   sme_seednet_forward_active  seeds [n][M][2] (device) of the MBs that
 *                         use one, the non-transparent ones, equal bit for
 *                         bit to those of sme_seednet_forward; the other MBs
 *                         get (0, 0).  mb_class: n_maps class maps [n][M]
 *                         (device, as sme_classify writes them), map_stride
 *                         bytes apart (>= n*M when n_maps > 1): an MB is
 *                         non-transparent if it is so in any map (the VOPs of
 *                         one sequence share features, hence seeds).  The
 *                         layers are evaluated only on MBs within one MB of
 *                         such an MB (five 3x3 layers reach 5 cells: one MB
 *                         is 4 cells and the MB's own cells are the fifth).
 *   sme_seednet_forward_active_table  the same with the class maps given
 *                         as a DEVICE table rows [n_maps][n] of pointers to
 *                         [M] class rows (a NULL entry: every MB transparent),
 *                         so maps written elsewhere (sme_batch_class_map) are
 *                         read in place; the seeds go to `seeds` [n][M][2]
 *                         (the other MBs get (0, 0)) or, with seeds NULL, to
 *                         the DEVICE table seed_rows [n] of pointers to
 *                         [M][2] rows (the other MBs' entries untouched).
 *   sme_seednet_set_stream  stream of the network's later calls.
 *   sme_seednet_synchronize waits for the network's stream; SME_ERR_TIMEOUT
 *                         if a device-side wait of an earlier call gave up
 *                         (its outputs are then not valid).
 *   sme_seednet_gradients loss and parameter gradients (host out), no update.
 *   sme_seednet_train_step forward, loss, backward, one Adam step with rate lr;
 *                         loss (host out, optional) synchronises.
 * Sizes must be multiples of 16; SME_ERR_SIZE beyond max_cells. */
typedef struct sme_seednet sme_seednet;
int sme_seednet_param_count(void);
int sme_seednet_create(sme_seednet** out, int max_cells, void* cuda_stream);
int sme_seednet_destroy(sme_seednet* net);
int sme_seednet_set_params(sme_seednet* net, const float* params /* host */);
int sme_seednet_get_params(sme_seednet* net, float* params /* host */);
int sme_seednet_features(sme_seednet* net, const uint8_t* luma, int width, int height, int ref_frame,
                         int cur_frame, int n_pairs, const sme_mv* temporal /* [M] device or NULL */,
                         int subpel, uint16_t* feat);
/* The same features for n_pairs pairs gathered from anywhere, in one launch:
 * frames is a DEVICE array [n_pairs][2] of pointers to [height][width] luma
 * frames (reference, current; each 4-byte aligned); temporal is NULL or a
 * DEVICE array [n_pairs] of pointers to [M] temporal fields (a NULL entry:
 * zeros); feat as above. */
int sme_seednet_features_table(sme_seednet* net, const uint8_t* const* frames, const sme_mv* const* temporal,
                               int n_pairs, int width, int height, int subpel, uint16_t* feat);
/* One temporal field per scene for the network input, for n scenes of
 * n_vops VOPs each, from the VOPs' fields (DEVICE arrays [n][n_vops] of
 * pointers: fields[q][j] [M] vectors, classes[q][j] [M] MB classes, either
 * NULL for an absent VOP): MB m of scene q takes fields[q][j][m] of the
 * first VOP j whose class is not transparent there, else (0, 0); out [n][M]
 * device.  No counterpart in the paper. */
int sme_seednet_temporal_composite(sme_seednet* net, const sme_mv* const* fields, const uint8_t* const* classes,
                                   int n, int n_vops, int width, int height, sme_mv* out);
int sme_seednet_forward(sme_seednet* net, const uint16_t* feat, int n, int width, int height, float* seeds,
                        float* out_cells);
int sme_seednet_forward_active(sme_seednet* net, const uint16_t* feat, int n, int width, int height,
                               const uint8_t* mb_class, int n_maps, long long map_stride, float* seeds);
int sme_seednet_forward_active_table(sme_seednet* net, const uint16_t* feat, int n, int width, int height,
                                     const uint8_t* const* rows, int n_maps, float* seeds, float* const* seed_rows);
int sme_seednet_set_stream(sme_seednet* net, void* cuda_stream);
int sme_seednet_synchronize(sme_seednet* net);
int sme_seednet_gradients(sme_seednet* net, const uint16_t* feat, int n, int width, int height,
                          const float* labels /* [n][M][2] device */, const uint8_t* mask /* [n][M] device */,
                          float* grads /* host, param layout */, float* loss /* host */);
int sme_seednet_train_step(sme_seednet* net, const uint16_t* feat, int n, int width, int height,
                           const float* labels, const uint8_t* mask, float lr, float* loss /* host */);

/* Stage timing (tracing).  sme_profile_begin makes every following
 * sme_estimate_sequence* call record CUDA events around its two launches on
 * the context's stream (classification, then the persistent ME launch), for
 * up to max_calls calls.  sme_profile_end synchronises and returns the number
 * of calls recorded and the summed device time of each stage in ms, then
 * stops recording.  Any output pointer may be NULL. */
int sme_profile_begin(sme_ctx* ctx, int max_calls);
int sme_profile_end(sme_ctx* ctx, int* calls, double* classify_ms, double* me_ms);

/* The paper has no counterpart of this call: it exists for callers that
 * cannot allocate device memory (code running inside another framework's
 * memory pool or a custom allocator that must own every device allocation,
 * or real-time / embedded callers that forbid allocation after start-up).
 * It computes exactly what sme_estimate_sequence computes, for the params
 * given here, without a context: its scratch (packed alpha, MB classes, ready
 * words, schedule, status) lives in one fixed 4 MiB array in device memory
 * that every GPU loading this library holds until exit, and the call makes no
 * cudaMalloc, cudaFree or other allocating call.
 *   p            parameters as for sme_create
 *   luma, alpha  [n_frames][H][W] device, 16-byte aligned (caller-owned)
 *   temporal_in, seed, out   as for sme_estimate_sequence (device, caller-owned)
 *   cuda_stream  cudaStream_t to run on (NULL = legacy default stream)
 * Scratch needed: F*H*Wp*4 + F*M + 12*P*M + 4*(steps+1) + 512 bytes, each part
 * rounded up to 256, where Wp = sme_packed_words(W), steps = (W/16-1) + 2*(H/16-1)
 * + P and P = F - ref_distance; a problem that needs more than 4 MiB (for
 * example more than 221 CIF frames, or more than 11 frames of 1920x1088) returns
 * SME_ERR_SCRATCH before any GPU work.
 * The first call on each device looks up the array's device address (with
 * that device current) and should come before any stream capture; the
 * address is kept for the life of the device's primary context, so the call
 * must not be used again after a cudaDeviceReset in the same process.
 * cuda_stream must belong to the current device (SME_ERR_ARG otherwise).
 * Seeds are accepted with max_iters <= 8, as for sme_estimate_sequence.  The
 * call synchronises the stream and returns the device-side status of its own
 * work.  All calls share the array: calls that overlap on the GPU (e.g. on
 * two streams, or from two threads) race and must be serialised by the
 * caller. */
int sme_estimate_sequence_noalloc(const sme_params* p, const uint8_t* luma, const uint8_t* alpha,
                                  int n_frames, const sme_mv* temporal_in, const float* seed,
                                  const sme_outputs* out, void* cuda_stream);

/* Failure injection for tests.  With skip_ticket >= 0 the MB with index
 * k*M + m (pair k, MB m) of the next estimates never publishes its result to
 * global memory, so the MBs that wait on it there (all its dependants in the
 * per-MB schedule; the next pair's T candidate in the pair schedule) wait
 * until `timeout_ns` and the launch ends with SME_ERR_TIMEOUT.
 * skip_ticket = -1 restores normal operation; timeout_ns <= 0 restores the
 * default wait limit (1 s). */
int sme_debug_set_fault(sme_ctx* ctx, int skip_ticket, long long timeout_ns);

#ifdef __cplusplus
}
#endif

#endif /* SME_H */
