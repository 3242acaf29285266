/*
 * sptrsv.h -- C ABI of the GB300 (sm_103a) sparse lower-triangular solve library.
 *
 * Solves L x = b for a sparse lower-triangular L in CSR (arXiv 2206.05843, Section II.A)
 * with the level-set method, either on L itself or after the paper's equation-rewriting
 * graph transformation (Section II.B, Section III), which moves rows of thin levels up
 * into earlier target levels so that the solve crosses fewer level barriers.
 *
 * Conventions for every entry point:
 *   - Pointers named *_dev are device pointers; *_host are host pointers.  Matrix and
 *     vector arguments are caller-owned; handles (levels, systems, batches, pickers)
 *     are library-owned and freed by their *_destroy function.
 *   - CSR: int32 row pointers (n+1) and column indices, columns strictly ascending in
 *     each row, the diagonal stored as the LAST entry of the row and non-zero
 *     (Algorithm 1 reads it at rowPtrL[i+1]-1).  Values float64 or float32.
 *   - Right-hand sides and solutions are column-major n x nrhs with leading dimension
 *     ld >= n; b and x must not overlap.
 *   - Levels are numbered from 0.
 *   - Calls are ordered on the given CUDA stream (NULL = the legacy default stream) and
 *     asynchronous unless they return host data, in which case they synchronize the
 *     stream before returning.
 *   - No C++ exception crosses this boundary.  On failure a status code is returned and
 *     sptrsv_last_error() holds a one-line message for the calling thread.
 *   - Every device-side wait is bounded; a wait that runs out sets the status
 *     SPTRSV_ERR_TIMEOUT and the kernel returns, leaving the CUDA context usable.
 *   - The persistent solve kernel is a cooperative launch, with thread-block clusters when its
 *     schedule has CLUSTER segments.  It checks its cluster shape on entry: a launch that runs
 *     without it (Nsight Compute runs cooperative launches so) stops at once and the status
 *     reads SPTRSV_ERR_CUDA.  The environment variable SPTRSV_PROFILE_LAUNCH=1, read once per
 *     process, drops the cooperative attribute from launches with clusters, so that such a
 *     profiler sees the kernel as it runs; the grid is sized from cluster occupancy either way.
 */
#ifndef SPTRSV_H
#define SPTRSV_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st* sptrsv_stream_t; /* same type as cudaStream_t */

typedef enum {
    SPTRSV_OK = 0,
    SPTRSV_ERR_INVALID = 1,     /* argument or CSR contract violated */
    SPTRSV_ERR_OOM = 2,         /* device or host allocation failed */
    SPTRSV_ERR_CUDA = 3,        /* a CUDA runtime call failed */
    SPTRSV_ERR_TIMEOUT = 4,     /* a bounded device wait ran out */
    SPTRSV_ERR_NUMERIC = 5,     /* rewrite growth guard tripped or non-finite value */
    SPTRSV_ERR_UNSUPPORTED = 6  /* valid request outside what this build supports */
} sptrsv_status;

enum { SPTRSV_F64 = 0, SPTRSV_F32 = 1 };

/* A lower-triangular CSR matrix in device memory (caller-owned). */
typedef struct {
    int64_t n;              /* rows = columns */
    int64_t nnz;            /* entries, diagonal included; rowptr[n] == nnz */
    const int32_t* rowptr;  /* device, n+1 */
    const int32_t* colidx;  /* device, nnz */
    const void* vals;       /* device, nnz values of type dtype */
    int32_t dtype;          /* SPTRSV_F64 or SPTRSV_F32 */
} sptrsv_csr;

typedef struct sptrsv_levels sptrsv_levels;
typedef struct sptrsv_system sptrsv_system;
typedef struct sptrsv_batch sptrsv_batch;
typedef struct sptrsv_picker sptrsv_picker;

/* ---------------------------------------------------------------------------------
 * Last error
 * ------------------------------------------------------------------------------- */

/* Copies the calling thread's last error message (NUL-terminated, truncated to len). */
sptrsv_status sptrsv_last_error(char* buf_host, size_t len);

/* ---------------------------------------------------------------------------------
 * Validation and level-set analysis (Section II.A, Fig. 1)
 * ------------------------------------------------------------------------------- */

/* Checks the CSR contract on the device.  Returns SPTRSV_OK or SPTRSV_ERR_INVALID
 * (message names the first offending row).  Synchronizes the stream. */
sptrsv_status sptrsv_validate(const sptrsv_csr* L, sptrsv_stream_t stream);

/* Level sets of DAG_L: a row without off-diagonal entries is on level 0, any other row
 * one level below its deepest dependency (Section II.A).  Validates L first.  Computes
 * level[n], the level pointer levelPtr[m+1], the rows of each level in ascending row
 * order levelRows[n], and per-level rows / nnz / cost with cost = 2*sum(nnz) - rows
 * (Section III).  *out is library-owned.  Synchronizes the stream (m is read back). */
sptrsv_status sptrsv_analyse(const sptrsv_csr* L, sptrsv_levels** out, sptrsv_stream_t stream);

typedef struct {
    int64_t n;           /* rows */
    int64_t m;           /* levels */
    int64_t nnz;         /* entries of the analysed structure, diagonal included */
    int64_t total_cost;  /* sum of level costs */
    double avg_cost;     /* avgLevelCost = total_cost / m (Section III) */
    int64_t max_width;   /* rows of the widest level */
} sptrsv_level_stats;

/* Host summary of an analysis.  No stream work. */
sptrsv_status sptrsv_levels_stats(const sptrsv_levels* lv, sptrsv_level_stats* out_host);

/* Copies the analysis to caller device buffers (any pointer may be NULL to skip):
 * level[n], level_ptr[m+1], level_rows[n] (int32) and per-level rows / nnz / cost
 * (int64, m each).  Stream-ordered. */
sptrsv_status sptrsv_levels_export(const sptrsv_levels* lv, int32_t* level_dev, int32_t* level_ptr_dev,
                                   int32_t* level_rows_dev, int64_t* rows_dev, int64_t* nnz_dev,
                                   int64_t* cost_dev, sptrsv_stream_t stream);

void sptrsv_levels_destroy(sptrsv_levels* lv);

/* ---------------------------------------------------------------------------------
 * Systems: what the solve runs on
 * ------------------------------------------------------------------------------- */

/* The plain level-set system of L: rows stored in level order, each normalised by its
 * diagonal.  *out is library-owned.  Synchronizes the stream. */
sptrsv_status sptrsv_system_plain(const sptrsv_csr* L, const sptrsv_levels* lv, sptrsv_system** out,
                                  sptrsv_stream_t stream);

enum {
    SPTRSV_STRATEGY_NONE = 0,    /* no rewriting: same as sptrsv_system_plain */
    SPTRSV_STRATEGY_NAIVE = 1,   /* Section III avgLevelCost strategy over thin levels */
    SPTRSV_STRATEGY_DEPTH_K = 2, /* fixed distance: each target takes the next k levels (Section III, manual approach) */
    SPTRSV_STRATEGY_LEARNED = 3, /* thin levels (Section III) merged into targets at depths a trained picker
                                    chooses per target (NAIVE without a picker) */
    SPTRSV_STRATEGY_CHOSEN = 4,  /* depth per target given by the caller */
    SPTRSV_STRATEGY_MANUAL = 5,  /* fixed distance k over thin levels only: the manual approach of the earlier work
                                    (nine levels folded into each tenth, Sections III and IV) */
    SPTRSV_STRATEGY_ROWCAP = 6,  /* the Section III walk over thin levels with a row count in place of avgLevelCost:
                                    a target takes rows while it holds at most k of them (k <= 0: 32, one warp's
                                    lanes -- the width of a level in the fast thin-level executor) */
    SPTRSV_STRATEGY_CHOSEN_THIN = 7 /* depth per target given by the caller, over thin levels only (cost below
                                       avgLevelCost, Section III): the plan family of the learned strategy */
};

typedef struct {
    int32_t kind;                  /* SPTRSV_STRATEGY_* */
    int32_t k;                     /* DEPTH_K / MANUAL: levels merged into each target; ROWCAP: rows a target may
                                      hold (<= 0: 32) */
    double nnz_growth_cap;         /* > 0: nnz(L') + nnz(E) <= cap * nnz(L); <= 0: no cap */
    double avg_override;           /* > 0: use this avgLevelCost instead of the computed one */
    double growth_guard;           /* > 0: fail with SPTRSV_ERR_NUMERIC if a rewritten coefficient exceeds it in magnitude */
    const sptrsv_picker* picker;   /* LEARNED */
    const int32_t* depth_of_target_host; /* CHOSEN, CHOSEN_THIN: depth for each level (m entries) when it is a target */
    const int32_t* depths_host;    /* LEARNED: candidates, a depth g >= 1 or a row budget -r (the largest depth whose
                                      window holds at most r rows); NULL = {1,2,4,8,16,32,-16,-32,-64} */
    int32_t n_depths;              /* entries of depths_host */
    const int64_t* injected_cost_dev; /* test hook (NULL normally): per-row cost on the target used by
                                         the planner instead of 2 * |dependencies after substitution| */
    int32_t max_deps;              /* per-row rule (Section III.A), > 0: a row moves only while it keeps fewer
                                      than max_deps dependencies after substitution */
    int64_t max_spread;            /* per-row rule (Section III.A, the cache-locality constraint), > 0: a row moves
                                      only while max - min of its dependencies is below max_spread.  A row that breaks
                                      a rule stops its group like a cost overflow (its level becomes the next target). */
    int32_t learned_mode;          /* LEARNED: 0 = the picker's plan, the naive plan, the ROWCAP plan (32 rows) and
                                      the plain (not rewritten) system are built and timed (one right-hand side)
                                      and the fastest is kept -- the paper's strategy, the executor-shaped plan and
                                      no rewrite are the fallbacks, the measured solve time decides; 1 = the
                                      picker's plan only */
    int32_t walk_parts;            /* planner walks (NAIVE, MANUAL, ROWCAP, CHOSEN(_THIN), LEARNED; with a cap or per-row
                                      rules): <= 1 one walk over all levels; P > 1 starts the walk at the beginning of
                                      each of P equal level ranges, one warp per range at the same time (Section III:
                                      the rewriting can also start at the end of the graph; P = 2 is both ends), the
                                      cap's allowance shared by the ranges in proportion to their entries */
} sptrsv_strategy;

/* Plans the rewrite with the strategy, rewrites the chosen rows (substitution of every
 * dependency on the target level or below it, then rearrangement into
 * x_r + sum c_rk x_k = sum e_rm b_m; Section II.B, Fig. 2), re-levels the result, drops
 * the emptied levels and stores it in level order.  *out is library-owned and solves
 * the ORIGINAL system L x = b.  Synchronizes the stream. */
sptrsv_status sptrsv_rewrite(const sptrsv_csr* L, const sptrsv_levels* lv, const sptrsv_strategy* strategy,
                             sptrsv_system** out, sptrsv_stream_t stream);

typedef struct {
    int64_t n, m;          /* rows, levels of the stored system */
    int64_t nnz_c;         /* stored off-diagonal coefficients (L' without its diagonal) */
    int64_t nnz_e;         /* stored b-coefficients of rewritten rows, diagonal term excluded */
    int64_t rows_moved;    /* rows rewritten to a higher level */
    int64_t stored_nnz;    /* nnz(L') + nnz(E explicit rows) as the planner counts it */
    int64_t nnz_l;         /* nnz(L) */
    int64_t segments;      /* solve schedule: wide levels + single-CTA runs */
    int64_t run_levels;    /* levels executed inside single-CTA runs */
    int32_t dtype;
    int32_t rewritten;
    double avg_cost;       /* avgLevelCost used by the planner (0 for plain) */
    int32_t block;         /* solve schedule: block size, */
    int32_t run_width;     /*   widest level inside a single-CTA run (0 auto, -1 none, -2 one launch per level), */
    int32_t lanes_per_row; /*   lanes per row (0 auto) */
    int32_t strategy_used; /* SPTRSV_STRATEGY_* of the stored plan (LEARNED resolves to CHOSEN, NAIVE, ROWCAP or NONE) */
    int32_t launches;      /* kernels one single-RHS solve launches with the current schedule (0 before the
                              first solve or tune) */
    int32_t ctas;          /* CTAs of the persistent solve kernel with the current schedule (SMs x CTAs per SM) */
    double candidate_us[4]; /* LEARNED with learned_mode 0: the measured solve time (us, one right-hand side,
                               default schedule) of each candidate -- the picker's plan, the naive plan, the ROWCAP
                               plan, the plain system -- in that order; 0 for every other system */
    int32_t cluster;       /* CTAs per thread-block cluster of the persistent solve (1: no CLUSTER segments) */
    int32_t cluster_setting; /* the system's cluster knob (0 automatic, 1 off, 2..16 CTAs) */
    int64_t cluster_levels; /* levels executed in CLUSTER segments */
    int64_t cluster_rows;  /* the system's widest-cluster-level knob (0 automatic) */
    int64_t tiled_levels;  /* WIDE levels whose coefficients stream through shared-memory tiles */
    int32_t tiles_setting; /* the system's tile knob (0 automatic, 1 never) */
    int32_t reserved0;
    int64_t shared_x_levels; /* CLUSTER levels whose x the next level reads from the cluster's shared memory */
    int32_t shared_x_setting; /* the system's shared-x knob (0 automatic, 1 never) */
    int32_t reserved1;
} sptrsv_system_info;

sptrsv_status sptrsv_system_info_get(const sptrsv_system* s, sptrsv_system_info* out_host);

/* Exports the system in the ORIGINAL row numbering to caller device buffers sized from
 * sptrsv_system_info_get (NULL skips an array):
 *   target[n]   level each row was planned onto (original level numbering; int32)
 *   level[n]    level of each row in the stored system (int32)
 *   cptr[n+1], ccol[nnz_c], cval[nnz_c]  off-diagonal coefficients c_rk (x_r + sum c_rk x_k),
 *               columns in original numbering, ascending within a row (int64 / int32 / dtype)
 *   dinv[n]     1 / L_rr (dtype)
 *   eptr[n+1], ecol[nnz_e], eval[nnz_e]  b-coefficients e_rm of rewritten rows, m != r (dtype)
 * Stream-ordered. */
sptrsv_status sptrsv_system_export(const sptrsv_system* s, int32_t* target_dev, int32_t* level_dev,
                                   int64_t* cptr_dev, int32_t* ccol_dev, void* cval_dev, void* dinv_dev,
                                   int64_t* eptr_dev, int32_t* ecol_dev, void* eval_dev, sptrsv_stream_t stream);

void sptrsv_system_destroy(sptrsv_system* s);

/* ---------------------------------------------------------------------------------
 * Solve (Algorithm 1 executed level by level; Section II.A, Section V)
 * ------------------------------------------------------------------------------- */

/* x = L^{-1} b for nrhs right-hand sides (column-major, leading dimension ld >= n) in the
 * system's value type.  One persistent kernel: wide levels are split over all CTAs and
 * handed over through device-wide per-CTA completion flags; runs of thin levels execute
 * inside one CTA.  Asynchronous; the status of the bounded waits is checked by the next
 * host-returning call or by sptrsv_solve_status. */
sptrsv_status sptrsv_solve(const sptrsv_system* s, const void* b_dev, void* x_dev, int32_t nrhs, int64_t ld,
                           sptrsv_stream_t stream);

/* Same as sptrsv_solve and, when stamps_dev is not NULL, records the %globaltimer
 * nanosecond at which each stored level finished (uint64, m entries).  Used to harvest
 * per-level times for the learned picker. */
sptrsv_status sptrsv_solve_timed(const sptrsv_system* s, const void* b_dev, void* x_dev, int32_t nrhs, int64_t ld,
                                 uint64_t* stamps_dev, sptrsv_stream_t stream);

/* A solve that allocates nothing, for callers that cannot call cudaMalloc when they
 * solve: real-time loops that must stay out of the allocator, processes whose device
 * memory a framework's caching allocator already holds, or plug-in code handed only its
 * inputs and outputs.  (The paper has no counterpart; this is an interface of the
 * library.)  Same arguments and result as sptrsv_solve, with the launches of the
 * system's current schedule (the persistent kernel, or one launch per level when the
 * system is tuned to run_width -2).  The solution scratch and the completion flags live
 * in one fixed 64 MiB device array of the library, so n * nrhs * sizeof(value) must not
 * exceed 64 MiB - 64 KiB (else SPTRSV_ERR_UNSUPPORTED).
 * The system must already hold a solve schedule for this nrhs: call sptrsv_solve once
 * with the same nrhs first (that call builds the schedule and may allocate); otherwise
 * SPTRSV_ERR_INVALID.  The first call on a device looks up the array's device address
 * and should come before any stream capture.  Every call on a device shares the array,
 * so calls that overlap on the GPU race: order them on one stream.  The bounded-wait
 * status goes to the system's status word (sptrsv_solve_status). */
sptrsv_status sptrsv_solve_noalloc(const sptrsv_system* s, const void* b_dev, void* x_dev, int32_t nrhs, int64_t ld,
                                   sptrsv_stream_t stream);

/* Synchronizes the stream and reports the device status word of the system's last
 * solve (SPTRSV_OK or SPTRSV_ERR_TIMEOUT), then clears it. */
sptrsv_status sptrsv_solve_status(const sptrsv_system* s, sptrsv_stream_t stream);

/* Test hook (the paper has no counterpart): the host block cutter of the single-CTA executor, on
 * host arrays, no device work.  level_ptr_host[m+1] and cptr_host[n+1] (n = level_ptr_host[m]) are
 * the level pointer and the coefficient row pointer of a system in stored (level) order; nrhs,
 * lanes_per_row and value_bytes (4 or 8) select the staging geometry, written to geometry_out[4] =
 * {stage rows, stage entries, ring rows, fast-block records} when not NULL.  Blocks go to
 * blocks_host[4 * capacity] as {first position, end position, first level, levels | flags} with
 * flags 1 << 30 (narrow), 1 << 29 (fast) and K (FMA steps per lane) in bits 26..28; *count_out
 * receives the number of blocks.  SPTRSV_ERR_INVALID when capacity is too small (count set),
 * SPTRSV_ERR_UNSUPPORTED when a row has more coefficients than a staging buffer holds. */
sptrsv_status sptrsv_debug_run_blocks(const int32_t* level_ptr_host, int64_t m, const int32_t* cptr_host,
                                      int32_t nrhs, int32_t lanes_per_row, int32_t value_bytes,
                                      int32_t* blocks_host, int64_t capacity, int64_t* count_out,
                                      int32_t* geometry_out);

/* Test hook for the bounded waits: the CTA that finishes schedule segment `segment`
 * does not publish it, so every wait on it runs out after timeout_ns.  segment < 0
 * disables the hook; timeout_ns <= 0 restores the default (2 s). */
sptrsv_status sptrsv_debug_set_wait(sptrsv_system* s, int64_t withhold_segment, int64_t timeout_ns);

/* Tuning knobs of one system (0 keeps the current value): block size of the persistent
 * kernel, widest level executed inside a single-CTA run (-1: no runs; -2: no persistent
 * kernel at all, one launch of a row-per-thread kernel per level), lanes per row. */
sptrsv_status sptrsv_system_tune(sptrsv_system* s, int32_t block, int32_t run_width, int32_t lanes_per_row);

/* Level-executor knobs of one system.  Levels wider than a single-CTA run and at most cluster_rows
 * rows (0: automatic, 16384) run as CLUSTER segments on the `cluster` CTAs of one thread-block
 * cluster (2..16; 0: automatic, 16; 1: no clusters), one cluster barrier per level instead of a
 * device-wide handoff.  tiles 0 (automatic): without clusters, WIDE levels of one right-hand side
 * stream their coefficients through shared memory in tiles (bulk copies, double-buffered) when
 * they fit; tiles 1: never.  shared_x 0 (automatic): CLUSTER segments of one right-hand side keep each
 * level's x in the shared memory of the CTA that computed it, where the next level reads it across
 * the cluster (the global copy is written after the level's barrier); shared_x 1: never.  Negative
 * values keep the current setting.  No stream work. */
sptrsv_status sptrsv_system_tune_cluster(sptrsv_system* s, int32_t cluster, int64_t cluster_rows, int32_t tiles,
                                         int32_t shared_x);

/* Autotuner: times candidate solves (b = 0) over lanes per row, the widest level executed
 * inside a single-CTA run and the level-executor knobs (clusters of 16 or 8 CTAs, with the
 * shared-x exchange on and off for one right-hand side, or none, with or without tiles; then
 * the widest cluster level), keeps the fastest for nrhs right-hand sides and caches the choice by the
 * system's signature (n, m, stored entries, nrhs, dtype).
 * *best_us_host (may be NULL) receives the best time.  Synchronizes the stream. */
sptrsv_status sptrsv_system_autotune(sptrsv_system* s, int32_t nrhs, double* best_us_host, sptrsv_stream_t stream);

/* ---------------------------------------------------------------------------------
 * Upper-triangular systems U x = b (the second triangular solve of an ILU preconditioner,
 * Section I), through the index reversal i -> n-1-i
 * ------------------------------------------------------------------------------- */

/* Writes the lower-triangular matrix of the reversed index order of U (CSR, columns
 * ascending, diagonal FIRST in each row) into caller device buffers of the same sizes:
 * rowptr (n+1), colidx (nnz), vals (nnz, U's dtype).  The result satisfies the CSR
 * contract of sptrsv_analyse when U is upper triangular with a non-zero diagonal (that
 * call validates it).  Stream-ordered. */
sptrsv_status sptrsv_upper_to_lower(const sptrsv_csr* U, int32_t* rowptr_dev, int32_t* colidx_dev, void* vals_dev,
                                    sptrsv_stream_t stream);

/* Re-indexes a system built from the reversed matrix so that it solves U x = b with b and
 * x in U's numbering (and its exports use that numbering).  Synchronizes the stream. */
sptrsv_status sptrsv_system_reverse_rows(sptrsv_system* s, sptrsv_stream_t stream);

/* ---------------------------------------------------------------------------------
 * Batched solve
 * ------------------------------------------------------------------------------- */

/* Groups `count` systems (each solved for nrhs[i] right-hand sides, ld = n) into one
 * persistent launch captured in a CUDA graph: every CTA takes whole work items, longest
 * first, and crosses levels with CTA barriers.  A work item is a system with all its
 * right-hand sides or a contiguous part of them (at most 8 parts), so that the parts of a heavy
 * system run on several CTAs at once.  Three split policies: 0 splits a system whose float64
 * work on one SM (about 0.25 ns x (stored entries + n) per right-hand side) exceeds both its
 * critical path (about 250 ns per level) and an even share of the batch per SM; 1 and 2 cut
 * into parts of at most 8 or 4 right-hand sides every system whose estimate exceeds 1.3 x the
 * batch's longest critical path.  Split policy, block size and lanes per row are autotuned by
 * timing candidate launches; the choice is cached by the batch signature.  Systems must
 * outlive the batch.  Synchronizes the stream. */
sptrsv_status sptrsv_batch_create(const sptrsv_system* const* systems_host, const int32_t* nrhs_host, int32_t count,
                                  sptrsv_batch** out, sptrsv_stream_t stream);

/* Solves every system of the batch: b_host[i] / x_host[i] are DEVICE pointers held in a
 * host array (column-major, ld = n_i).  Replays the captured graph. */
sptrsv_status sptrsv_batch_solve(sptrsv_batch* bt, const void* const* b_host, void* const* x_host,
                                 sptrsv_stream_t stream);

typedef struct {
    int32_t count, block, lanes_per_row, graph;
    double tuned_us;       /* best measured time of the autotuner */
    int32_t items;         /* work items (systems, or parts of their right-hand sides) */
    int32_t split_policy;  /* the autotuner's split policy: 0 by work, 1 and 2 parts of at most 8 and 4 */
} sptrsv_batch_info;

sptrsv_status sptrsv_batch_info_get(const sptrsv_batch* bt, sptrsv_batch_info* out_host);

void sptrsv_batch_destroy(sptrsv_batch* bt);

/* ---------------------------------------------------------------------------------
 * Learned rewrite picker: an MLP 12 -> 64 -> 64 -> 64 -> 1 (ReLU) with bfloat16 weights
 * and float32 accumulation that predicts the solve-time change of rewriting the next
 * g levels into a target level (the learned strategy the paper names as future work,
 * Conclusion).
 * ------------------------------------------------------------------------------- */

#define SPTRSV_PICKER_FEATURES 12
#define SPTRSV_PICKER_HIDDEN 64
#define SPTRSV_PICKER_PARAMS (12 * 64 + 64 + 64 * 64 + 64 + 64 * 64 + 64 + 64 + 1)

/* New picker with weights drawn from a seeded generator (Kaiming-uniform). */
sptrsv_status sptrsv_picker_create(uint64_t seed, sptrsv_picker** out);
void sptrsv_picker_destroy(sptrsv_picker* pk);

/* Flat float32 parameter vector (SPTRSV_PICKER_PARAMS entries, layer by layer: W1 row-major
 * [64][12], b1, W2 [64][64], b2, W3 [64][64], b3, W4 [1][64], b4) to or from the host. */
sptrsv_status sptrsv_picker_get_params(const sptrsv_picker* pk, float* params_host);
sptrsv_status sptrsv_picker_set_params(sptrsv_picker* pk, const float* params_host);

/* Input normalisation applied before layer 1: f' = (f - mean) / std (12 each). */
sptrsv_status sptrsv_picker_set_norm(sptrsv_picker* pk, const float* mean_host, const float* std_host,
                                     float target_scale);

/* Saves / loads weights, normalisation and optimiser state (binary with a text header). */
sptrsv_status sptrsv_picker_save(const sptrsv_picker* pk, const char* path);
sptrsv_status sptrsv_picker_load(sptrsv_picker* pk, const char* path);

/* Features of every candidate (target level t, candidate d) for t in [0, m):
 * feat_dev[(t * n_depths + d) * 12 + f] (float32).  A candidate is a depth g >= 1 (the window
 * t..t+g) or a row budget -r, which resolves per target to the largest depth whose window holds
 * at most r rows (0 when level t alone holds more); 0 is rejected.  Stream-ordered. */
sptrsv_status sptrsv_picker_features(const sptrsv_csr* L, const sptrsv_levels* lv, const int32_t* depths_host,
                                     int32_t n_depths, float* feat_dev, sptrsv_stream_t stream);

/* Predicted solve-time change (float32, in target units) for `count` feature rows.
 * bf16_weights != 0 uses the bfloat16 copy of the weights, else the float32 master. */
sptrsv_status sptrsv_picker_infer(const sptrsv_picker* pk, const float* feat_dev, int64_t count, float* out_dev,
                                  int32_t bf16_weights, sptrsv_stream_t stream);

/* Gradient of the mean squared error over `count` rows with respect to every parameter
 * (float32, SPTRSV_PICKER_PARAMS entries) and the loss; forward through the bfloat16 or
 * float32 weights.  Stream-ordered. */
sptrsv_status sptrsv_picker_grad(const sptrsv_picker* pk, const float* feat_dev, const float* target_dev,
                                 int64_t count, int32_t bf16_weights, float* grad_dev, float* loss_dev,
                                 sptrsv_stream_t stream);

/* One Adam step (beta1 0.9, beta2 0.999, eps 1e-8) on a mini-batch: gradient as above,
 * then the float32 master weights, their bfloat16 copy and the moments are updated on
 * the device.  loss_dev (may be NULL) receives the batch loss before the step. */
sptrsv_status sptrsv_picker_train_step(sptrsv_picker* pk, const float* feat_dev, const float* target_dev,
                                       int64_t count, float lr, float* loss_dev, sptrsv_stream_t stream);

#ifdef __cplusplus
}
#endif

#endif /* SPTRSV_H */
