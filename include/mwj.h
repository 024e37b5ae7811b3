/*
 * mwj.h -- C ABI of the GB300 multiway (3-way) hash join library (libmwj.so).
 *
 * The library evaluates, on one CUDA device, the single-step 3-way joins of
 * "Efficient Multiway Hash Join on Reconfigurable Hardware" (arXiv 1905.13376):
 *
 *   linear  R(A,B) |x| S(B,C) |x| T(C,D)   (Section 4, Algorithm 1)
 *   cyclic  R(A,B) |x| S(B,C) |x| T(C,A)   (Section 5)
 *
 * and the cascade of two binary hash joins the paper measures them against
 * (Section 6.3); the star variant of the linear join (Section 6), the chain
 * of four relations and Flajolet-Martin sketches of the friends-of-friends-
 * of-friends query (Sections 4.1 and 7); a batched mode and a learned
 * planner.  Results follow bag semantics (duplicates are not removed,
 * Section 1, Example 1) and are exact: counts are 64-bit and wrap modulo 2^64.
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * - All data pointers are DEVICE pointers on the context's device unless a
 *   comment says otherwise.  The caller owns every input, output and
 *   workspace buffer; the library never frees or retains caller memory
 *   beyond the call.
 * - Relations are column pairs of int32 (structure of arrays).  Columns may
 *   alias (R, S and T may be the same arrays).  n is limited to
 *   [0, 2^31 - 1] tuples per relation.
 * - `stream` is a cudaStream_t passed as void*; NULL is the legacy default
 *   stream.  Calls are stream-ordered: argument errors are returned
 *   synchronously; errors detected on the device (an A value outside the
 *   group-by domain, too few output rows, a bounded wait that ran out) are
 *   recorded in the context's status word and returned by
 *   mwj_stream_status().  mwj_cascade_join and calls with shares == NULL
 *   synchronise `stream` once on the host (they read sizes back).
 * - The library allocates no device memory inside join calls: all scratch
 *   comes from the caller's workspace, sized by mwj_workspace_size().
 * - A context is used by one host thread at a time.
 */
#ifndef MWJ_H
#define MWJ_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    MWJ_OK = 0,
    MWJ_ERR_INVALID_ARG = 1,   /* NULL pointer, n < 0 or too large, share < 1, bad mode/kind */
    MWJ_ERR_DOMAIN = 2,        /* GROUP BY A: some a outside [0, a_domain) */
    MWJ_ERR_CAPACITY = 3,      /* MATERIALIZE: more rows than `capacity`; *n_rows holds the exact count */
    MWJ_ERR_WORKSPACE = 4,     /* workspace too small for this call */
    MWJ_ERR_CUDA = 5,          /* a CUDA runtime call failed; see mwj_last_error() */
    MWJ_ERR_TIMEOUT = 6,       /* a bounded device-side wait reached its iteration limit */
    MWJ_ERR_CHECK = 7,         /* an internal consistency check failed on the device */
    MWJ_ERR_UNIMPLEMENTED = 8
} mwj_status;

typedef enum {
    MWJ_COUNT = 0,             /* COUNT(*) of the join into *total */
    MWJ_COUNT_GROUP_BY_A = 1,  /* COUNT(*) GROUP BY A into group_counts[a], plus *total */
    MWJ_MATERIALIZE = 2        /* the joined tuples into rows, plus *n_rows and *total */
} mwj_mode;

typedef enum { MWJ_LINEAR = 0, MWJ_CYCLIC = 1, MWJ_STAR = 4 } mwj_kind;

/* One relation: n tuples (x[i], y[i]).  Linear: R = (a,b), S = (b,c),
 * T = (c,d).  Cyclic: R = (a,b), S = (b,c), T = (c,a).  Device, borrowed,
 * read-only. */
typedef struct {
    const int32_t *x;
    const int32_t *y;
    int64_t n;
} mwj_rel;

/* Bucket counts ("shares") of the top-level hash functions (Sections 4.1,
 * 5 and the analyses 4.2, 5.2).
 *   linear: s[0] = number of H(B) buckets of R and S; s[1] = number of g(C)
 *           buckets of S and T (1 = T's tile stays whole in L2, see
 *           mwj_join3_linear); s[2] = log2 of the slots of the on-chip R
 *           bucket table, 9..14 (0 or 1: the library default, 12); a bucket
 *           with more distinct B values than half the slots is processed in
 *           chunks.
 *   cyclic: s = {H(A), G(B), F(C)} bucket counts; tile (i,j,k) joins
 *           R_ij, S_jk and T_ki.
 * Every used entry must be >= 1.  A NULL share pointer asks the library's
 * cost-model planner to choose (mwj_plan_shares). */
typedef struct {
    int32_t s[3];
} mwj_shares;

typedef struct {
    mwj_mode mode;
    int64_t *total;          /* device, 1 element, always written (all modes) */
    int64_t *group_counts;   /* device, a_domain elements, overwritten (GROUP BY A) */
    int32_t a_domain;        /* GROUP BY A: every a of R must lie in [0, a_domain) */
    int32_t *rows;           /* device, capacity * arity int32, row-major (MATERIALIZE);
                                arity 4 (a,b,c,d) linear, 3 (a,b,c) cyclic; order unspecified */
    int64_t capacity;        /* rows available */
    int64_t *n_rows;         /* device, 1 element: exact number of result rows (MATERIALIZE) */
} mwj_out;

typedef struct {
    int32_t device;          /* CUDA device ordinal, -1 = current device */
    uint32_t seed;           /* seed of the hash functions (results do not depend on it) */
    int32_t smem_bytes;      /* shared memory per CTA for tiles, 0 = library default */
    int32_t load_pct;        /* maximum fill of on-chip hash tables in percent, 0 = default (50) */
    int64_t spin_limit;      /* iteration cap of bounded device waits, 0 = default */
} mwj_config;

typedef struct mwj_ctx mwj_ctx;

/* Create a context on cfg->device (or the current device when cfg == NULL or
 * device == -1).  Allocates the context's device status word and creates two
 * internal streams and their events (work a join call forks onto them is
 * joined back to the caller's stream within the call).  Returns MWJ_ERR_CUDA
 * if no usable sm_103 device is present. */
mwj_status mwj_create(mwj_ctx **ctx, const mwj_config *cfg);
mwj_status mwj_destroy(mwj_ctx *ctx);

/* Bytes of device workspace a call needs.  kind: MWJ_LINEAR / MWJ_CYCLIC /
 * MWJ_STAR for mwj_join3_*, or 2 + kind (linear or cyclic) for
 * mwj_cascade_join.  For the cascade the size
 * includes room for 2^24 rows of the intermediate relation I; the cascade
 * uses every byte it is given beyond its fixed part as room for I, at 12
 * bytes per row (linear), 20 (cyclic counts) or 24 (cyclic rows), and works
 * through I in chunks of that many rows. */
mwj_status mwj_workspace_size(mwj_ctx *ctx, int kind, mwj_rel R, mwj_rel S, mwj_rel T,
                              const mwj_shares *shares, mwj_mode mode, size_t *bytes);

/* Linear 3-way join R(A,B) S(B,C) T(C,D) in one step (Algorithm 1, Section 4).
 * Shares s[0] = s[1] = 1 with COUNT or GROUP BY A (the default for those
 * modes when shares == NULL): one bucket per side, nothing partitioned, the
 * held tables kept whole in the L2: T's table c -> deg_T(c) is built (on a
 * context stream) while S's weight table b -> w(b) is sized, a pass over S
 * adds w(b) += deg_T(c), and a pass over R adds cnt[a] += w(b) and
 * total += w(b).  Both tables are sized from HyperLogLog estimates of the
 * distinct keys; w(b) is exact to 2^64.
 * Otherwise R is partitioned by H(B), S by (H(B), g(C)), T by g(C); each CTA holds one
 * H(B) bucket's B values as an on-chip hash table while the other side of
 * that bucket streams past it, and T's tables are probed (its bucket images
 * when shares.s[1] > 1, one L2-resident table when shares.s[1] == 1).  For
 * MATERIALIZE the table holds R's bucket (Algorithm 1's roles); for COUNT and
 * GROUP BY A it holds S's bucket with w(b) = sum of deg_T(c) whenever
 * |S| <= 2 |R| (each R tuple is then read once), else R's.  For COUNT and
 * GROUP BY A, B keys heavy enough to unbalance the buckets (sampled) are
 * routed to one extra bucket that every CTA aggregates.  No intermediate
 * relation is materialised.  The call may run parts of its work on the
 * context's own streams; they are joined back to `stream` before it returns
 * (also on errors).  workspace: device, >= mwj_workspace_size(ctx,
 * MWJ_LINEAR, ...). */
mwj_status mwj_join3_linear(mwj_ctx *ctx, mwj_rel R, mwj_rel S, mwj_rel T,
                            const mwj_shares *shares, const mwj_out *out,
                            void *workspace, size_t ws_bytes, void *stream);

/* Cyclic 3-way join R(A,B) S(B,C) T(C,A) in one step (Section 5): tile
 * (i,j,k) of the share cube holds R_ij (H(a)=i, G(b)=j) and T_ki
 * (F(c)=k, H(a)=i) on chip while S_jk streams past them.  T's columns are
 * (c, a). */
mwj_status mwj_join3_cyclic(mwj_ctx *ctx, mwj_rel R, mwj_rel S, mwj_rel T,
                            const mwj_shares *shares, const mwj_out *out,
                            void *workspace, size_t ws_bytes, void *stream);

/* Star 3-way join R(A,B) S(B,C) T(C,D) (Section 6, "linear star 3-way
 * join"): the same query and outputs as mwj_join3_linear, planned for small
 * dimension relations R and T and a large fact relation S.  R is grouped by
 * h(B) and T by g(C) into bucket tables that stay on chip (L2 and L1); S is
 * read once, unpartitioned, each tuple looked up in both tables (twice for
 * MATERIALIZE: a counting pass, then the rows).  shares: s[0] = h(B) buckets
 * of R, s[1] = g(C) buckets of T (0 or shares == NULL: about 2048 tuples per
 * bucket); s[2] is ignored.  GROUP BY A checks the domain of A while it adds
 * R's groups (MWJ_ERR_DOMAIN from mwj_stream_status).
 * workspace: device, >= mwj_workspace_size(ctx, MWJ_STAR, ...). */
mwj_status mwj_join3_star(mwj_ctx *ctx, mwj_rel R, mwj_rel S, mwj_rel T, const mwj_shares *shares,
                          const mwj_out *out, void *workspace, size_t ws_bytes, void *stream);

/* Chain of four relations R(A,B) S(B,C) T(C,D) U(D,E), COUNT or COUNT
 * GROUP BY A (the "additional levels of hashing" of Section 7): one hash
 * level per join attribute.  U becomes an on-chip table of deg_U(d), T a
 * table of w_T(c) = sum of deg_U(d) over T's (c,d), and R and S are joined
 * on B as in mwj_join3_linear with w_T(c) in place of T's degree; no
 * intermediate relation is materialised.  shares: s[0] = H(B) buckets,
 * s[1] must be 1, s[2] = log2 of the on-chip table slots (as for the linear
 * join); NULL = the linear join's default.  MATERIALIZE is not offered
 * (MWJ_ERR_INVALID_ARG).  workspace: >= mwj_join4_workspace_size(...). */
mwj_status mwj_join4_workspace_size(mwj_ctx *ctx, mwj_rel R, mwj_rel S, mwj_rel T, mwj_rel U,
                                    const mwj_shares *shares, mwj_mode mode, size_t *bytes);
mwj_status mwj_join4_linear(mwj_ctx *ctx, mwj_rel R, mwj_rel S, mwj_rel T, mwj_rel U,
                            const mwj_shares *shares, const mwj_out *out, void *workspace,
                            size_t ws_bytes, void *stream);

/* Flajolet-Martin sketches of the distinct friends of friends of friends of
 * every A (Section 4.1's footnote; the approximate variant of Example 1):
 * D(a) = { d : (a,b) in R, (b,c) in S, (c,d) in T } is summarised by a PCSA
 * sketch of 16 bitmaps of 32 bits (value d sets bit rho(h div 16) of bitmap
 * h mod 16, h = MurmurHash3's fmix32(d xor 0x5BD1E995), rho = index of the
 * lowest 1 bit, 27 when h div 16 is 0); sketches are carried along the join
 * with OR as counts are with +.  sketches: device, 16-byte aligned,
 * a_domain x 16 uint32, overwritten (sketch of a at [16 a, 16 a + 16)); a
 * misaligned pointer is MWJ_ERR_INVALID_ARG.  estimates: device,
 * a_domain floats, or NULL: (16 / 0.77351) * 2^(mean over bitmaps of the
 * index of their lowest 0 bit).  Every a of R must lie in [0, a_domain)
 * (MWJ_ERR_DOMAIN from mwj_stream_status otherwise).  shares: s[0] = H(B)
 * buckets (NULL: ~16K S tuples per bucket); the other entries are ignored.
 * workspace: device, >= mwj_fm_workspace_size(...). */
mwj_status mwj_fm_workspace_size(mwj_ctx *ctx, mwj_rel R, mwj_rel S, mwj_rel T,
                                 const mwj_shares *shares, size_t *bytes);
mwj_status mwj_fm_linear(mwj_ctx *ctx, mwj_rel R, mwj_rel S, mwj_rel T, const mwj_shares *shares,
                         int32_t a_domain, uint32_t *sketches, float *estimates, void *workspace,
                         size_t ws_bytes, void *stream);

/* Cascade of binary hash joins (Section 6.3): I(A,B,C) = R join S is
 * materialised in the workspace (in chunks when it does not fit), then
 * I join T gives the same result as the 3-way join.  kind = MWJ_LINEAR or
 * MWJ_CYCLIC.  Synchronises `stream` on the host to size the chunks. */
mwj_status mwj_cascade_join(mwj_ctx *ctx, int kind, mwj_rel R, mwj_rel S, mwj_rel T,
                            const mwj_out *out, void *workspace, size_t ws_bytes,
                            void *stream);

/* The linear join (COUNT or COUNT GROUP BY A only) for callers that cannot
 * allocate device memory -- for example code running under another
 * runtime's allocator, or a plug-in whose host process owns every device
 * allocation.  It needs no context and no workspace: its scratch is a
 * fixed 24 MiB device array inside the library, present on every GPU that
 * loads the library until the process exits.  There is no counterpart in
 * the paper.
 *
 * Limits: at most 2^18 tuples per relation and shares with s[0]*s[1] <= 1024
 * (NULL shares: the library picks them); larger inputs return
 * MWJ_ERR_WORKSPACE (use mwj_join3_linear with a workspace instead).
 * out->mode must be MWJ_COUNT or MWJ_COUNT_GROUP_BY_A.
 * Runs on the current device and `stream`, then synchronises `stream` and
 * returns any device-side error (e.g. MWJ_ERR_DOMAIN) directly.
 * The first call on a device looks up the scratch array's device address;
 * make it before any stream capture.  The address is kept for the life of
 * the process: after cudaDeviceReset on a device the array lives at a new
 * address, so the entry point must not be called on that device again.  All calls share the one array: calls
 * that overlap on the GPU (other streams, other host threads) race, so the
 * caller must serialise them.  Scratch that must start at zero is cleared by
 * every call. */
mwj_status mwj_join3_linear_noalloc(mwj_rel R, mwj_rel S, mwj_rel T, const mwj_shares *shares,
                                    const mwj_out *out, void *stream);

/* Synchronise `stream`, return the first device-side error recorded since the
 * previous call (MWJ_OK if none) and clear it. */
mwj_status mwj_stream_status(mwj_ctx *ctx, void *stream);

/* Failure detection check: launch one CTA that waits, with the library's
 * bounded wait and at most `polls` polls (1 .. 2^24), on a barrier phase
 * that never completes, then records MWJ_ERR_TIMEOUT in the context's
 * status word and returns; the next mwj_stream_status reports it and the
 * context stays usable.  The joins' own waits give up the same way when a
 * copy does not land within the context's spin_limit.  Stream-ordered. */
mwj_status mwj_check_bounded_wait(mwj_ctx *ctx, int64_t polls, void *stream);

/* ---- batches of independent joins (COUNT(*) per query) -------------------
 * Thousands of small 3-way joins of uneven sizes, linear and cyclic mixed,
 * run by one persistent join kernel after one persistent partitioning kernel
 * (the paper's tiling applied per query; no counterpart for batching in the
 * paper).  mwj_batch_create plans every query (shares.s[0] == 0: the
 * library chooses the shares from the sizes) and fixes the relations'
 * device pointers; mwj_batch_launch enqueues the whole batch with no host
 * round trip, so launches after the first one on a given workspace can be
 * captured into a CUDA graph and replayed (the first launch on a workspace
 * uploads the plan's descriptors and must happen outside a capture).
 * counts: device, n int64 elements, overwritten with each query's COUNT(*).
 * Linear queries take at most 4096 H(B) buckets, cyclic ones x*y, y*z and
 * z*x at most 4096 each. */
typedef struct {
    int32_t kind;          /* MWJ_LINEAR or MWJ_CYCLIC */
    mwj_rel R, S, T;       /* device relations, as for mwj_join3_* */
    mwj_shares shares;     /* s[0] == 0: chosen by the library */
} mwj_query;

typedef struct mwj_batch mwj_batch;

mwj_status mwj_batch_create(mwj_ctx *ctx, const mwj_query *queries, int32_t n, mwj_batch **batch);
mwj_status mwj_batch_workspace_size(mwj_batch *batch, size_t *bytes);
mwj_status mwj_batch_shares(mwj_batch *batch, int32_t q, mwj_shares *shares);
mwj_status mwj_batch_launch(mwj_batch *batch, int64_t *counts, void *workspace, size_t ws_bytes,
                            void *stream);
mwj_status mwj_batch_destroy(mwj_batch *batch);

/* Batch planning rules (the autotuner's output; no counterpart in the
 * paper).  A query whose shares the library chooses falls in the size class
 * floor(log2(max(|R|, |S|, |T|))) of its kind; the rule of that class gives
 *   tuples_per_bucket  linear: about this many R tuples per H(B) bucket
 *                      (I = the power of two at or above |R| / it);
 *   table_factor       linear: slots of T's degree table per T tuple (the
 *                      power of two at or above factor x |T|: load factor
 *                      at most 1 / factor), 2 .. 8;
 *   fit_pct            cyclic: R_ij and T_ki may fill this percentage of a
 *                      tile's on-chip capacity when the cube shares are
 *                      searched (Section 5.2's z|R| + x|S| + y|T|), 10 .. 100.
 * A field <= 0 keeps the library's rule (8192 tuples, factor 2, 50 %).
 * mwj_batch_set_rules replaces the context's rules (n == 0 restores the
 * library's); mwj_batch_set_launch sets the CTAs per SM of the batch's
 * persistent partitioning and join launches (0: the library's choice, 3 and
 * the occupancy limit).  Batches created afterwards use them. */
typedef struct {
    int32_t kind;               /* MWJ_LINEAR or MWJ_CYCLIC */
    int32_t size_log2;          /* 0 .. 31 */
    int32_t tuples_per_bucket;
    int32_t table_factor;
    int32_t fit_pct;
} mwj_batch_rule;

mwj_status mwj_batch_set_rules(mwj_ctx *ctx, const mwj_batch_rule *rules, int32_t n);
mwj_status mwj_batch_set_launch(mwj_ctx *ctx, int32_t prep_ctas_per_sm, int32_t join_ctas_per_sm);

/* The shares the planner would choose for these relations (host result in
 * *shares), the ones a call with shares == NULL uses.  kind = MWJ_LINEAR,
 * MWJ_CYCLIC or MWJ_STAR.  Linear: {1, 1, 1} for COUNT and GROUP BY A (the
 * one-bucket plan), H(B) buckets from |R| for MATERIALIZE.  Synchronises
 * `stream`. */
mwj_status mwj_plan_shares(mwj_ctx *ctx, int kind, mwj_rel R, mwj_rel S, mwj_rel T,
                           mwj_mode mode, mwj_shares *shares, void *stream);

/* The alternative share vector a planner weighs against the default one
 * (host only, from the sizes).  Linear (Section 4.2): H(B) buckets of R and S
 * held in shared memory, ~32K R tuples each (the default for MATERIALIZE).
 * Cyclic (Section 5.2 with a third share): the cube tiling (x, y, z) that
 * minimises z|R| + x|S| + y|T| with R_ij and T_ki fitting a CTA's shared
 * memory, against the default (1, 1, z) in which R stays whole. */
mwj_status mwj_plan_shares_alt(mwj_ctx *ctx, int kind, mwj_rel R, mwj_rel S, mwj_rel T, mwj_shares *shares);

/* Human-readable text of the last error on this context (static storage of
 * the context; valid until the next call). */
const char *mwj_last_error(mwj_ctx *ctx);

/* Launch accounting and per-kernel timing, for benchmarks and profiles.  No
 * counterpart in the paper (its numbers come from a performance model).
 * mwj_set_profiling(ctx, 1) makes every kernel the context launches record a
 * CUDA event pair on its stream (a pool of 2^15 launches; later launches are
 * counted but not timed until mwj_reset_phase_times); while it is on, work a
 * call would overlap on the context's internal streams runs on the caller's
 * stream instead, so that each event pair times its kernel alone (the
 * results are the same; the call's total time is then that of the
 * serialised kernels).  mwj_launch_count
 * returns the number of kernels the context has launched since it was
 * created, whether or not profiling is on.  mwj_get_phase_times synchronises
 * on the recorded events and fills up to `max` entries of per-kernel-name
 * totals (milliseconds and launches; names stay valid until the next call on
 * the context); it returns the number of distinct kernel names, or -1 for a
 * NULL context. */
mwj_status mwj_set_profiling(mwj_ctx *ctx, int enable);
long long mwj_launch_count(mwj_ctx *ctx);
int mwj_get_phase_times(mwj_ctx *ctx, const char **names, double *ms, long long *launches,
                        int max);
mwj_status mwj_reset_phase_times(mwj_ctx *ctx);

/* ---- planning: features, cost model, learned planner ----------------------
 * A plan only chooses between the 3-way join and the cascade and scales the
 * shares; it never changes a result.
 *
 * mwj_features writes 24 floats (host) describing a join instance: log2 of
 * the three sizes, log2 of HyperLogLog distinct counts of R.x, R.y, S.y, T.y,
 * the cyclic flag, log2 of a sampled estimate of |R join S| (the exact R
 * degrees of evenly spaced S tuples, scaled), and sampled key-frequency
 * fractions (once / 2-7 / 8+ times in the sample) of R.y, S.x, S.y, T.x and
 * T.y (cyclic only).  workspace: device, >= mwj_features_workspace_size().
 * Synchronises `stream`.
 *
 * mwj_cost_model: from the features, log2 predicted seconds of the three
 * plans a planner chooses from: out3[0] the cascade, out3[1] the 3-way join
 * with the default shares, out3[2] with the alternative shares
 * (mwj_plan_shares_alt).  It restates the tuple counts of Sections 4.2, 5.2
 * and 6.3 (tuples read, the intermediate written and read back, wedge checks)
 * as HBM bytes, random lookups and on-chip probes, a phase costing its
 * slowest resource (the paper's Appendix A model), with hbm_gbs the HBM
 * bandwidth in GB/s and rates measured on this GPU.
 *
 * mwj_mlp_*: the planner's network, 24 -> 128 -> 128 -> 3 with ReLU, BF16
 * weights and activations, FP32 accumulation and FP32 Adam master weights
 * (mwj_mlp_num_params() floats in the layout W1[24][128], b1[128],
 * W2[128][128], b2[128], W3[128][3], b3[3]).  X: device B x 24 floats
 * (rounded to BF16 on entry), Y: device B x 3.  backward writes the FP32
 * gradient of sum M (Y - T)^2 * inv_count into grads (device,
 * mwj_mlp_num_params()) and the loss into *loss (device); adam applies one
 * Adam step (beta 0.9 / 0.999, eps 1e-8; step >= 1 is the bias-correction
 * count). */
size_t mwj_features_workspace_size(void);
mwj_status mwj_features(mwj_ctx *ctx, int kind, mwj_rel R, mwj_rel S, mwj_rel T, float *features,
                        void *workspace, size_t ws_bytes, void *stream);
mwj_status mwj_cost_model(const float *features, double hbm_gbs, double *out3);

typedef struct mwj_mlp mwj_mlp;
size_t mwj_mlp_num_params(void);
mwj_status mwj_mlp_create(mwj_ctx *ctx, mwj_mlp **mlp);
mwj_status mwj_mlp_destroy(mwj_mlp *mlp);
mwj_status mwj_mlp_set_params(mwj_mlp *mlp, const float *host_params);
mwj_status mwj_mlp_get_params(mwj_mlp *mlp, float *host_params);
mwj_status mwj_mlp_forward(mwj_mlp *mlp, const float *X, int32_t B, float *Y, void *stream);
mwj_status mwj_mlp_backward(mwj_mlp *mlp, const float *X, const float *T, const float *M, int32_t B,
                            float inv_count, float *grads, float *loss, void *stream);
mwj_status mwj_mlp_adam(mwj_mlp *mlp, const float *grads, float lr, int32_t step, void *stream);

/* Library version string, e.g. "mwj 0.1 sm_103a". */
const char *mwj_version(void);

#ifdef __cplusplus
}
#endif

#endif /* MWJ_H */
