// system.cuh -- the stored system and the solve schedule (internal).
#pragma once

#include "internal.cuh"

namespace sp {

// WIDE: one level over CTAs 0..w-1; RUN: staged blocks [y, z) on CTA 0; CLUSTER: levels [y, z), each
// split over the w CTAs of cluster 0.  The type is in the low byte of a segment's x; a WIDE or CLUSTER
// segment keeps its lanes per row in the next byte (0: the schedule's).
enum SegType : int { SEG_WIDE = 0, SEG_RUN = 1, SEG_CLUSTER = 2 };
constexpr int SEG_TYPE_MASK = 0xff, SEG_LPR_SHIFT = 8, SEG_LPR_MASK = 0xff;
// A cluster region: consecutive RUN and CLUSTER segments that the CTAs of cluster 0 execute with
// cluster barriers (barrier.cluster, ~0.4 us) between them instead of device-wide completion flags.
// Every segment of a region carries SEG_REGION; the first (SEG_FIRST) is entered through the flags
// of the segment before it, the last (SEG_LAST) publishes the flags for the segment after it.
constexpr int SEG_REGION = 1 << 16, SEG_FIRST = 1 << 17, SEG_LAST = 1 << 18;
// A WIDE segment of one right-hand side whose coefficients stream through shared memory in tiles of
// TILE_ROWS >> ((x >> SEG_TILE_SHIFT) & 3) rows (bulk copies, double-buffered): SEG_TILED
constexpr int SEG_TILED = 1 << 19, SEG_TILE_SHIFT = 20;
// A CLUSTER segment of one right-hand side whose levels keep their x in the CTAs' shared memory (a
// two-level ring), read across the cluster by the next level: SEG_DSM
constexpr int SEG_DSM = 1 << 22;
constexpr int TILE_ROWS = 512;   // rows of a tile at the largest size (one per thread of a 512-thread CTA)
constexpr int TILE_MAX = 64;     // tiles of one CTA's share of a level
constexpr int64_t TILE_SMEM_MAX = 100 * 1024;  // shared memory the two tile buffers may take (2 CTAs per SM)

__host__ __device__ inline size_t align16(size_t v) { return (v + 15) & ~(size_t)15; }
// bytes of one tile buffer holding `ecap` coefficients (columns, then values) of vb-byte values,
// with room for the 16-byte rounding of both bulk copies
__host__ __device__ inline size_t tile_buf_bytes(int64_t ecap, int vb) {
    return align16((size_t)(ecap + 4) * 4) + align16((size_t)(ecap + 4) * vb);
}

// rows a ROWCAP target holds by default: the lanes of one warp, the fast executor's level width
constexpr int ROWCAP_DEFAULT_ROWS = 32;

// CLUSTER segments (automatic settings): levels wider than a single-CTA run and at most
// CLUSTER_ROWS_DEFAULT rows run on a cluster of CLUSTER_DEFAULT CTAs; a stretch of fewer than
// CLUSTER_RUN_MIN thin levels next to such levels joins them
constexpr int CLUSTER_DEFAULT = 16;
constexpr int64_t CLUSTER_ROWS_DEFAULT = 16384;
constexpr int CLUSTER_RUN_MIN = 4;

// A segment of the persistent solve.  WIDE: one level split over CTAs 0..parts-1.
// RUN: consecutive thin levels executed by CTA 0 alone, staged block by block.
// CLUSTER: consecutive levels, each split in contiguous chunks over the CTAs of cluster 0.
// int4 layout: {type | flags, a, b, c}
//   WIDE   : a = level, b = rows per participating CTA, c = number of participating CTAs
//   RUN    : a = first block, b = end block, c = 0
//   CLUSTER: a = first level, b = end level, c = CTAs of the cluster
// A run block: int4 {first level, end level, narrow (all levels fit one warp), 0}

struct Schedule {
    int nrhs = -1, block = 0, run_width = 0, lpr = 0, grid = 0, ring_rows = 0;
    int csize = 1;          // CTAs per cluster of the launch (1: no cluster segments, plain launch)
    int cluster = 0;        // the system's cluster setting the schedule was built with
    int tiles = 0;          // the system's tile setting the schedule was built with
    int shared_x = 0;       // and its shared-x setting
    int64_t dsm_levels = 0; // levels of SEG_DSM segments
    int64_t cluster_rows = 0;  // widest level run as a CLUSTER level
    int64_t cluster_levels = 0;  // levels executed in CLUSTER segments
    int stage_rows = 0, stage_entries = 0;
    int pre = 0;       // a b-part kernel runs before the solve (rewritten rows in staged blocks)
    int tile_ecap = 0; // coefficients a tile buffer holds (0: no tiled WIDE segments)
    int runs = 0;      // RUN segments (0: the wide-only kernel variant, no shared memory)
    int64_t tiled_levels = 0;
    int pre_grid = 0;  // its CTAs
    int pre_cl = 0;    // the b-part kernel also covers the rows of CLUSTER segments (ranges after the run blocks)
    int dsm_cap = 0;   // rows per CTA and level of the SEG_DSM segments' shared-memory ring slots
    size_t smem = 0;
    int64_t run_levels = 0;
    std::vector<int4> h_segs, h_blocks;
    DevBuf<int4> segs, blocks;
};

// rows in the stored order ("positions"): perm[p] = original row; ccol holds positions
template <typename T>
struct SolveArgs {
    int64_t n;
    int nrhs;
    int64_t ld;
    const int32_t* __restrict__ perm;
    const int32_t* __restrict__ lptr;
    const int32_t* __restrict__ cptr;
    const int32_t* __restrict__ ccol;
    const T* __restrict__ cval;
    const T* __restrict__ dinv;
    const int32_t* __restrict__ eptr;  // nullptr when no row was rewritten
    const int32_t* __restrict__ ecol;
    const T* __restrict__ eval;
    const int4* __restrict__ segs;
    const int4* __restrict__ blocks;
    int nseg;
    const T* __restrict__ b;
    T* x;
    T* xp;  // solution in stored order, position-major: xp[p * nrhs + k]
    int* flags;
    int* status;
    unsigned long long* stamps;
    int withhold;
    int64_t timeout_ns;
    int ring_rows;  // power of two
    int lpr;        // lanes per row (power of two <= 32)
    int csize;      // CTAs per cluster (1: launched without clusters)
    int tile_ecap;  // coefficients one tile buffer holds (0: no tiled WIDE segments)
    int stage_rows, stage_entries;
    int pre;        // xp holds the b-parts of the staged blocks' rows (k_bparts ran first)
    int pre_cl;     // and of the CLUSTER segments' rows
    int dsm_cap;    // rows of one level a CTA keeps in shared memory in SEG_DSM segments (one ring slot)
};

}  // namespace sp

struct sptrsv_system {
    int64_t n = 0, m = 0;
    int dtype = SPTRSV_F64;
    int rewritten = 0;
    int strategy_used = 0;
    double cand_us[4] = {0, 0, 0, 0};  // LEARNED: measured time of each candidate (model, naive, rowcap, plain)
    sp::Levels lv;  // levels of the stored structure; lv.level_rows is perm, lv.pos its inverse
    sp::DevBuf<int32_t> cptr, ccol, eptr, ecol, target;
    sp::DevBuf<unsigned char> cval, eval, dinv;
    int64_t nnz_c = 0, nnz_e = 0, rows_moved = 0, stored_nnz = 0, nnz_l = 0;
    double avg = 0.0;
    // solve state
    int block = 512, run_width = 0, lpr = 0;  // 0: automatic
    int cluster = 0;          // CTAs of the cluster that runs mid-width levels: 0 automatic, 1 none, 2..16
    int tiles = 0;            // wide levels through shared-memory tiles: 0 automatic, 1 never
    int shared_x = 0;         // cluster levels exchange x through shared memory: 0 automatic, 1 never
    int64_t cluster_rows = 0; // widest level run on the cluster (0: automatic)
    sp::Schedule sched;
    std::vector<int32_t> h_cptr;  // host copy of cptr, for cutting run blocks
    sp::DevBuf<int> flags, status;
    sp::DevBuf<unsigned char> xp;
    int withhold = -1;
    int64_t timeout_ns = 0;
};

namespace sp {

// builds (or reuses) the schedule of a system for nrhs right-hand sides
sptrsv_status prepare_schedule(sptrsv_system* s, int nrhs);

// enqueues one solve (flags/status reset + persistent kernel) on the stream
sptrsv_status enqueue_solve(sptrsv_system* s, const void* b, void* x, int nrhs, int64_t ld,
                            unsigned long long* stamps, cudaStream_t st);

// fills the stored arrays of a system from L (rows that were not rewritten) and, when
// moved != nullptr, from the rewrite heap (rows with moved[r] != 0).  s->lv must hold
// the levels of the final structure.
struct RewriteHeap {
    const int32_t* moved = nullptr;
    const int64_t* c_off = nullptr;
    const int32_t* c_cnt = nullptr;
    const int64_t* e_off = nullptr;
    const int32_t* e_cnt = nullptr;
    const int32_t* col = nullptr;
    const double* val = nullptr;
};
sptrsv_status pack_system(sptrsv_system* s, const sptrsv_csr* L, const RewriteHeap* rw, cudaStream_t st);

// rewrite with a planner walk kind (1 naive, 2 fixed depth, 3 depth per target) -> new system
sptrsv_status rewrite_system(const sptrsv_csr* L, const Levels& lv, int kind, int k, const int32_t* dot_dev,
                             double avg_override, double cap, double guard, const int64_t* inj, int alpha, int64_t beta,
                             int parts, sptrsv_system** out, cudaStream_t st);

// median time of `reps` solves with b = 0 (one right-hand side), in microseconds
sptrsv_status time_solve_us(sptrsv_system* s, int reps, double* us, cudaStream_t st);

// the learned strategy (picker.cu): features -> MLP -> depth per target -> rewrite_system
sptrsv_status learned_rewrite(const sptrsv_csr* L, const sptrsv_levels* lv, const sptrsv_strategy* sg,
                              sptrsv_system** out, cudaStream_t st);

}  // namespace sp
