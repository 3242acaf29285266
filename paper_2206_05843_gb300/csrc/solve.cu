// solve.cu -- the persistent level-set solve (Algorithm 1 executed level by level).
//
// One launch walks the schedule.  A WIDE segment is one level whose rows are split in
// contiguous chunks over CTAs 0..parts-1; a CTA publishes the segment in its own
// completion flag (release) and the CTAs of the next segment wait (acquire, bounded)
// for the flags of exactly the CTAs that worked on the previous one.  A RUN segment is a
// chain of thin levels executed by CTA 0 alone: its rows, coefficients and the b-part
// of every row (dinv * b plus the rewritten rows' E * b) are staged into shared memory
// block by block, x of the run stays in a shared-memory ring, and consecutive levels are
// separated by a CTA (or warp) barrier instead of a device-wide handoff.
#include <algorithm>
#include <map>
#include <tuple>
#include <mutex>
#include <vector>

#include "solve_kernel.cuh"

namespace sp {
namespace {

template <typename T>
sptrsv_status launch_solve(sptrsv_system* s, const void* b, void* x, int nrhs, int64_t ld,
                           unsigned long long* stamps, cudaStream_t st) {
    Schedule& sc = s->sched;
    SolveArgs<T> a;
    a.n = s->n;
    a.nrhs = nrhs;
    a.ld = ld;
    a.perm = s->lv.level_rows.p;
    a.lptr = s->lv.level_ptr.p;
    a.cptr = s->cptr.p;
    a.ccol = s->ccol.p;
    a.cval = (const T*)s->cval.p;
    a.dinv = (const T*)s->dinv.p;
    a.eptr = s->nnz_e > 0 ? s->eptr.p : nullptr;
    a.ecol = s->ecol.p;
    a.eval = (const T*)s->eval.p;
    a.segs = sc.segs.p;
    a.blocks = sc.blocks.p;
    a.nseg = (int)sc.h_segs.size();
    a.b = (const T*)b;
    a.x = (T*)x;
    a.xp = (T*)s->xp.p;
    a.flags = s->flags.p;
    a.status = s->status.p;
    a.stamps = stamps;
    a.withhold = s->withhold;
    a.timeout_ns = s->timeout_ns > 0 ? s->timeout_ns : default_timeout_ns();
    a.ring_rows = sc.ring_rows;
    a.lpr = sc.lpr;
    a.stage_rows = sc.stage_rows;
    a.stage_entries = sc.stage_entries;
    a.pre = sc.pre;
    a.pre_cl = sc.pre_cl;
    a.csize = sc.csize;
    a.dsm_cap = sc.dsm_cap;
    a.tile_ecap = sc.tile_ecap;

    SP_CUDA(cudaMemsetAsync(s->flags.p, 0xff, (size_t)sc.grid * sizeof(int), st));
    SP_CUDA(cudaMemsetAsync(s->status.p, 0, sizeof(int), st));
    if (s->run_width == -2) {
        // one launch per level
        const std::vector<int32_t>& lp = s->lv.h_level_ptr;
        for (int64_t l = 0; l < s->m; ++l) {
            const int64_t rows = (int64_t)(lp[l + 1] - lp[l]) * nrhs;
            k_level<T><<<(unsigned)((rows + 255) / 256), 256, 0, st>>>(a, lp[l], lp[l + 1]);
            if (stamps) k_stamp<<<1, 32, 0, st>>>(stamps, l);
        }
        SP_CUDA(cudaGetLastError());
        return SPTRSV_OK;
    }
    if (a.nseg == 0) return SPTRSV_OK;
    if (sc.pre) k_bparts<T><<<sc.pre_grid, 256, 0, st>>>(a, (int)sc.h_blocks.size());
    SP_CUDA(k_solve_attrs<T>(sc.smem, sc.csize, sc.tile_ecap, sc.runs));  // systems may differ in their shared memory
    SP_CUDA(launch_k_solve<T>(a, sc.grid, sc.block, sc.smem, sc.csize, st, sc.runs));
    return SPTRSV_OK;
}

// CTAs of the persistent kernel that can be co-resident with the given block, shared memory and
// cluster size (cluster size 1: no clusters); 0 when the configuration does not fit.
template <typename T>
sptrsv_status solve_capacity(int block, size_t smem, int csize, int tiled, int64_t* ctas) {
    *ctas = 0;
    SP_CUDA(k_solve_attrs<T>(smem, csize, tiled));
    if (csize <= 1) {
        int occ = 0;
        SP_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_solve_fn<T>(k_mode(1, tiled)), block, smem));
        *ctas = (int64_t)device_sm_count() * occ;
        return SPTRSV_OK;
    }
    cudaLaunchConfig_t q = {};
    q.gridDim = dim3((unsigned)csize);
    q.blockDim = dim3((unsigned)block);
    q.dynamicSmemBytes = smem;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = (unsigned)csize;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    q.attrs = at;
    q.numAttrs = 1;
    int ncl = 0;
    if (cudaOccupancyMaxActiveClusters(&ncl, k_solve_fn<T>(KM_CLUSTER), &q) != cudaSuccess) {
        cudaGetLastError();  // a cluster size the device cannot place: no clusters
        ncl = 0;
    }
    *ctas = (int64_t)ncl * csize;
    return SPTRSV_OK;
}

int pow2_floor(int64_t v) {
    int p = 1;
    while ((int64_t)p * 2 <= v) p *= 2;
    return p;
}

}  // namespace

// Cuts levels [l_begin, l_end) into blocks that fit the staging area: whole levels while
// they fit, a level that does not fit is split by rows.  Runs of levels that qualify for the
// fast executor form fast blocks of whole levels; the block's FMA steps per lane K is the
// largest ceil(row length / lpr) of its levels (an upper bound: dependencies older than the
// ring are folded into the b-part at staging).  Returns 0, or -1 when a single row has more
// coefficients than the staging area holds.
int build_run_blocks(const int32_t* lp, const int32_t* cptr, int64_t l_begin, int64_t l_end, int stage_rows,
                     int stage_entries, int lpr, int nrhs, int fast_recs, std::vector<int4>& out) {
    const bool fast_on = fast_recs > 0 && nrhs <= FAST_MAX_RHS &&
                         (lpr == 1 || lpr == 2 || (lpr == 4 && nrhs == 1));
    int r2 = 1;  // right-hand sides rounded up to a power of two
    while (r2 < nrhs) r2 <<= 1;
    r2 /= fast_rhs_per_lane(nrhs);  // lanes of a row's right-hand sides
    // FMA steps a level needs in a fast block, or 0 when the level does not qualify
    auto fast_k = [&](int64_t l) -> int {
        if (!fast_on) return 0;
        const int64_t rows = lp[l + 1] - lp[l];
        if (rows * lpr * r2 > 32) return 0;
        int64_t mx = 0;
        for (int64_t i = lp[l]; i < lp[l + 1]; ++i) mx = std::max<int64_t>(mx, (int64_t)cptr[i + 1] - cptr[i]);
        const int64_t k = std::max<int64_t>(1, (mx + lpr - 1) / lpr);
        return k <= K_MAX ? (int)k : 0;
    };
    int64_t P = lp[l_begin];
    const int64_t Pend = lp[l_end];
    int64_t l = l_begin;
    int next_k = -1;  // fast_k of level l when already known
    while (P < Pend) {
        while (lp[l + 1] <= P) {
            ++l;
            next_k = -1;
        }
        if (P == lp[l]) {
            int k0 = next_k >= 0 ? next_k : fast_k(l);
            next_k = -1;
            if (k0 > 0) {
                // a fast block: whole levels while the records fit
                int K = k0;
                int64_t rows = lp[l + 1] - lp[l];
                int64_t l1 = l + 1;
                while (l1 < l_end) {
                    const int kl = fast_k(l1);
                    if (kl == 0) {
                        next_k = 0;
                        break;
                    }
                    const int64_t r = lp[l1 + 1] - lp[l1];
                    const int Kn = std::max(K, kl);
                    if (rows + r > stage_rows || (int64_t)Kn * lpr * (rows + r) > fast_recs) {
                        next_k = kl;
                        break;
                    }
                    rows += r;
                    K = Kn;
                    ++l1;
                }
                out.push_back(make_int4((int)P, (int)lp[l1], (int)l, (int)(l1 - l) | BLK_NARROW | BLK_FAST |
                                                                         (K << BLK_K_SHIFT)));
                P = lp[l1];
                l = l1;
                continue;
            }
        }
        const int64_t P0 = P, l0 = l;
        int64_t rows = 0, ents = 0, maxw = 0;
        int64_t lcur = l;
        while (P < Pend) {
            while (lp[lcur + 1] <= P) ++lcur;
            // a level that qualifies for a fast block starts a block of its own
            if (rows > 0 && fast_on && P == lp[lcur] && fast_k(lcur) > 0) break;
            const int64_t lend = lp[lcur + 1];
            const int64_t r = lend - P, e = (int64_t)cptr[lend] - cptr[P];
            if (rows + r <= stage_rows && ents + e <= stage_entries) {
                rows += r;
                ents += e;
                maxw = std::max(maxw, lend - std::max<int64_t>(lp[lcur], P0));
                P = lend;
                continue;
            }
            if (rows == 0) {
                // this level alone does not fit: take the rows that do
                int64_t q = P;
                while (q < lend && rows + 1 <= stage_rows && ents + (cptr[q + 1] - cptr[q]) <= stage_entries) {
                    ents += cptr[q + 1] - cptr[q];
                    ++rows;
                    ++q;
                }
                if (rows == 0) return -1;
                maxw = rows;
                P = q;
            }
            break;
        }
        int64_t l_last = l0;
        while (lp[l_last + 1] < P) ++l_last;
        const int nl = (int)(l_last - l0 + 1);
        const int narrow = maxw * lpr <= 32 ? BLK_NARROW : 0;
        out.push_back(make_int4((int)P0, (int)P, (int)l0, nl | narrow));
    }
    return 0;
}

sptrsv_status prepare_schedule(sptrsv_system* s, int nrhs) {
    Schedule& sc = s->sched;
    const int vb = s->dtype == SPTRSV_F64 ? 8 : 4;
    int lpr = s->lpr;
    if (lpr <= 0) {
        if (nrhs >= 2) lpr = std::min(32, pow2_floor(2 * nrhs - 1));
        else lpr = (s->n > 0 && (double)s->nnz_c / (double)s->n > 12.0) ? 4 : 1;
    }
    int block = s->block > 0 ? s->block : 512;
    block = std::max(32, std::min(512, block / 32 * 32));
    if (lpr > 32 || (lpr & (lpr - 1))) {
        set_error("lanes per row must be a power of two <= 32");
        return SPTRSV_ERR_INVALID;
    }
    if (sc.nrhs == nrhs && sc.lpr == lpr && sc.block == block && sc.run_width == s->run_width &&
        sc.cluster == s->cluster && sc.cluster_rows == s->cluster_rows && sc.tiles == s->tiles &&
        sc.shared_x == s->shared_x && sc.segs.p)
        return SPTRSV_OK;
    const int ngroups = block / lpr;
    // shared memory: two staging buffers + an x ring of at least twice the staged rows
    const RunGeom geo = run_geometry(nrhs, vb);
    const int stage_entries = geo.stage_entries, stage_rows = geo.stage_rows, ring_rows = geo.ring_rows;
    int run_width = s->run_width > 0 ? s->run_width : (s->run_width < 0 ? 0 : ngroups);
    run_width = std::min(run_width, stage_rows);
    const int64_t m = s->m;
    // row pointers of the stored coefficients (host copy) for cutting blocks
    if ((int64_t)s->h_cptr.size() != s->n + 1) {
        s->h_cptr.assign(s->n + 1, 0);
        SP_CUDA(cudaMemcpy(s->h_cptr.data(), s->cptr.p, (s->n + 1) * sizeof(int32_t), cudaMemcpyDeviceToHost));
    }
    const std::vector<int32_t>& hcptr = s->h_cptr;
    const std::vector<int32_t>& lp = s->lv.h_level_ptr;
    sc.h_segs.clear();
    sc.h_blocks.clear();
    sc.run_levels = 0;
    sc.tile_ecap = 0;
    sc.tiled_levels = 0;
    int64_t max_parts = 1;
    int sms = device_sm_count();
    // occupancy decides the number of CTAs that WIDE levels can be split over
    size_t smem = run_smem_bytes(vb, nrhs, RunGeom{ring_rows, stage_rows, stage_entries});
    int64_t gplain = 0, gcl = 0;
    int csize = s->cluster == 1 ? 1 : (s->cluster > 1 ? std::min(16, s->cluster) : CLUSTER_DEFAULT);
    const int64_t cl_rows = s->cluster_rows > 0 ? s->cluster_rows : CLUSTER_ROWS_DEFAULT;
    auto capacity = [&](size_t sm, int cs, int tiled, int64_t* out) -> sptrsv_status {
        return s->dtype == SPTRSV_F64 ? solve_capacity<double>(block, sm, cs, tiled, out)
                                      : solve_capacity<float>(block, sm, cs, tiled, out);
    };
    // wide levels of one right-hand side may stream their coefficients through shared memory
    // (two tile buffers; the kernel variant with tiled WIDE levels, so schedules with CLUSTER
    // segments do not tile), when that does not lower the number of co-resident CTAs
    bool tiles_ok = nrhs == 1 && block == TILE_ROWS && s->tiles != 1;
    const size_t smem_tiles = std::max(smem, (size_t)TILE_SMEM_MAX);
    if (tiles_ok) {
        int64_t g_run = 0, g_tiles = 0;
        SP_TRY(capacity(smem, 1, 0, &g_run));
        SP_TRY(capacity(smem_tiles, 1, 1, &g_tiles));
        tiles_ok = g_tiles == g_run;
    }
    SP_TRY(capacity(tiles_ok ? smem_tiles : smem, 1, tiles_ok ? 1 : 0, &gplain));
    if (csize > 1) SP_TRY(capacity(smem, csize, 0, &gcl));
    if (gplain < 1) {
        set_error("solve kernel does not fit an SM with block %d and %zu bytes of shared memory", block, smem);
        return SPTRSV_ERR_UNSUPPORTED;
    }
    if (gcl < csize) csize = 1;
    auto thin = [&](int64_t l) {
        return lp[l + 1] - lp[l] <= run_width && (int64_t)hcptr[lp[l + 1]] - hcptr[lp[l]] <= stage_entries;
    };
    // level kinds: 0 thin (single-CTA runs), 1 mid-width (cluster levels), 2 wide (all CTAs)
    std::vector<unsigned char> kind(m);
    bool any_mid = false;
    for (int64_t l = 0; l < m; ++l) {
        kind[l] = thin(l) ? 0 : (csize > 1 && lp[l + 1] - lp[l] <= cl_rows ? 1 : 2);
        any_mid |= kind[l] == 1;
    }
    if (any_mid) {
        // short stretches of thin levels next to cluster levels become cluster levels: a cluster
        // barrier per level costs less than entering and leaving a staged single-CTA run
        int64_t l = 0;
        while (l < m) {
            if (kind[l] != 0) { ++l; continue; }
            int64_t l1 = l;
            while (l1 < m && kind[l1] == 0) ++l1;
            const bool next_to_mid = (l > 0 && kind[l - 1] == 1) || (l1 < m && kind[l1] == 1);
            if (l1 - l < CLUSTER_RUN_MIN && next_to_mid)
                for (int64_t q = l; q < l1; ++q) kind[q] = 1;
            l = l1;
        }
    } else {
        csize = 1;
    }
    if (csize > 1) tiles_ok = false;
    // cluster levels of one right-hand side keep their x in shared memory (two ring slots of the
    // widest CTA share), when the larger shared memory still leaves a whole cluster co-resident;
    // their b-parts are then computed up front (pre_cl below: one right-hand side always qualifies)
    sc.dsm_cap = 0;
    size_t smem_cl = smem;
    if (csize > 1 && nrhs == 1 && s->shared_x != 1) {
        int64_t cap = 0;
        for (int64_t q = 0; q < m; ++q)
            if (kind[q] == 1) cap = std::max<int64_t>(cap, (lp[q + 1] - lp[q] + csize - 1) / csize);
        const size_t ring = align16((size_t)(2 * cap * vb));
        int64_t g2 = gcl;
        if (ring > smem) SP_TRY(capacity(ring, csize, 0, &g2));
        if (cap > 0 && g2 >= csize) {
            sc.dsm_cap = (int)cap;
            smem_cl = std::max(smem, ring);
            gcl = g2;
        }
    }
    const int64_t gmax = csize > 1 ? gcl : gplain;
    sc.cluster_levels = 0;
    sc.dsm_levels = 0;
    int64_t l = 0;
    while (l < m) {
        if (kind[l] == 1) {
            int64_t l1 = l, ents = 0;
            while (l1 < m && kind[l1] == 1) ++l1;
            ents = (int64_t)hcptr[lp[l1]] - hcptr[lp[l]];
            const int64_t rows = lp[l1] - lp[l];
            // lanes per row of the segment: two for single right-hand sides of 4 or more coefficients
            const int wl = (nrhs == 1 && lpr == 1 && ents >= 4 * rows) ? 2 : lpr;
            const int dsm = sc.dsm_cap > 0 ? SEG_DSM : 0;
            sc.h_segs.push_back(
                make_int4(SEG_CLUSTER | dsm | (wl == lpr ? 0 : wl << SEG_LPR_SHIFT), (int)l, (int)l1, csize));
            sc.cluster_levels += l1 - l;
            if (dsm) sc.dsm_levels += l1 - l;
            max_parts = std::max<int64_t>(max_parts, csize);
            l = l1;
            continue;
        }
        if (kind[l] == 0) {
            int64_t l1 = l;
            while (l1 < m && kind[l1] == 0) ++l1;
            int blk0 = (int)sc.h_blocks.size();
            if (build_run_blocks(lp.data(), hcptr.data(), l, l1, stage_rows, stage_entries, lpr, nrhs,
                                 fast_rec_capacity(vb, RunGeom{ring_rows, stage_rows, stage_entries}),
                                 sc.h_blocks) != 0) {
                set_error("schedule: a row has more coefficients than the staging area");
                return SPTRSV_ERR_UNSUPPORTED;
            }
            sc.h_segs.push_back(make_int4(SEG_RUN, blk0, (int)sc.h_blocks.size(), 0));
            sc.run_levels += l1 - l;
            l = l1;
        } else {
            int64_t w = lp[l + 1] - lp[l];
            // lanes per row of this level: with one lane per row, a moderately wide level of
            // longer rows takes two, halving each row's dependent float64 chain; very wide levels
            // keep one (they are bound by float64 issue, where the extra add costs)
            int wl = lpr;
            if (nrhs == 1 && lpr == 1 && w <= 65536 && (int64_t)hcptr[lp[l + 1]] - hcptr[lp[l]] >= 4 * w) wl = 2;
            const int64_t ng = block / wl;
            int64_t per = std::max<int64_t>((w + gmax - 1) / gmax, ng);
            int64_t parts = (w + per - 1) / per;
            if (per >= INT32_MAX) { set_error("level too wide"); return SPTRSV_ERR_UNSUPPORTED; }
            max_parts = std::max(max_parts, parts);
            int flags = SEG_WIDE | (wl == lpr ? 0 : wl << SEG_LPR_SHIFT);
            if (tiles_ok && wl == 1) {
                // the largest tile (512, 256 or 128 rows) whose coefficients fit a buffer in every tile
                for (int sh = 0; sh < 3; ++sh) {
                    const int64_t tr = TILE_ROWS >> sh;
                    if ((per + tr - 1) / tr > TILE_MAX) break;
                    int64_t emax = 0;
                    for (int64_t c = 0; c < parts; ++c) {  // tiles of every CTA's share
                        const int64_t s0 = lp[l] + c * per, s1 = std::min<int64_t>(lp[l + 1], s0 + per);
                        for (int64_t r0 = s0; r0 < s1; r0 += tr) {
                            const int64_t r1 = std::min(r0 + tr, s1);
                            emax = std::max<int64_t>(emax, (int64_t)hcptr[r1] - hcptr[r0]);
                        }
                    }
                    if (2 * tile_buf_bytes(emax, vb) <= (size_t)TILE_SMEM_MAX) {
                        flags |= SEG_TILED | (sh << SEG_TILE_SHIFT);
                        sc.tile_ecap = (int)std::max<int64_t>(sc.tile_ecap, std::max<int64_t>(emax, 16));
                        sc.tiled_levels += 1;
                        break;
                    }
                }
            }
            sc.h_segs.push_back(make_int4(flags, (int)l, (int)per, (int)parts));
            ++l;
        }
    }
    // cluster regions: maximal stretches of RUN and CLUSTER segments that hold a CLUSTER segment
    for (size_t i = 0; i < sc.h_segs.size();) {
        if ((sc.h_segs[i].x & SEG_TYPE_MASK) == SEG_WIDE) { ++i; continue; }
        size_t j = i;
        bool has_cl = false;
        while (j < sc.h_segs.size() && (sc.h_segs[j].x & SEG_TYPE_MASK) != SEG_WIDE)
            has_cl |= (sc.h_segs[j++].x & SEG_TYPE_MASK) == SEG_CLUSTER;
        if (has_cl) {
            for (size_t q = i; q < j; ++q) sc.h_segs[q].x |= SEG_REGION;
            sc.h_segs[i].x |= SEG_FIRST;
            sc.h_segs[j - 1].x |= SEG_LAST;
        }
        i = j;
    }
    // rewritten rows in thin levels: their b-parts (E rows) are computed up front by every
    // CTA, so that staging reads one value per row instead of walking the E row
    const bool small_rhs = nrhs * (int64_t)vb <= 64;
    const bool run_pre = s->nnz_e > 0 && !sc.h_blocks.empty();
    // the rows of CLUSTER segments too: a cluster row then reads one contiguous b-part instead of
    // gathering b through the permutation after the level's wait (ranges of at most 4,096 positions,
    // after the run blocks, so that the runs' block indices stay as they are)
    sc.pre_cl = 0;
    if (csize > 1 && small_rhs) {
        for (const int4& sg : sc.h_segs) {
            if ((sg.x & SEG_TYPE_MASK) != SEG_CLUSTER) continue;
            for (int64_t q = lp[sg.y]; q < lp[sg.z]; q += 4096) {
                sc.h_blocks.push_back(make_int4((int)q, (int)std::min<int64_t>(lp[sg.z], q + 4096), 0, 0));
                sc.pre_cl = 1;
            }
        }
    }
    sc.pre = small_rhs && (run_pre || sc.pre_cl) ? 1 : 0;
    sc.pre_grid = (int)std::min<int64_t>((int64_t)sc.h_blocks.size(), (int64_t)sms * 8);
    if (sc.h_blocks.empty()) sc.h_blocks.push_back(make_int4(0, 0, 0, 0));
    SP_TRY(sc.segs.alloc(std::max<size_t>(1, sc.h_segs.size())));
    SP_TRY(sc.blocks.alloc(sc.h_blocks.size()));
    if (!sc.h_segs.empty())
        SP_CUDA(cudaMemcpy(sc.segs.p, sc.h_segs.data(), sc.h_segs.size() * sizeof(int4), cudaMemcpyHostToDevice));
    SP_CUDA(cudaMemcpy(sc.blocks.p, sc.h_blocks.data(), sc.h_blocks.size() * sizeof(int4), cudaMemcpyHostToDevice));
    sc.grid = (int)std::min<int64_t>(gmax, max_parts);
    if (csize > 1) sc.grid = (int)std::min<int64_t>(gmax, (std::max<int64_t>(max_parts, csize) + csize - 1) / csize * csize);
    sc.csize = csize;
    sc.cluster = s->cluster;
    sc.cluster_rows = s->cluster_rows;
    sc.tiles = s->tiles;
    sc.shared_x = s->shared_x;
    sc.nrhs = nrhs;
    sc.lpr = lpr;
    sc.block = block;
    sc.run_width = s->run_width;
    sc.ring_rows = ring_rows;
    sc.stage_rows = stage_rows;
    sc.stage_entries = stage_entries;
    sc.runs = 0;
    for (const int4& sg : sc.h_segs) sc.runs += (sg.x & SEG_TYPE_MASK) == SEG_RUN;
    sc.smem = sc.tile_ecap > 0 ? std::max(smem, 2 * tile_buf_bytes(sc.tile_ecap, vb)) : (csize > 1 ? smem_cl : smem);
    if (csize == 1 && sc.tile_ecap == 0 && sc.runs == 0) sc.smem = 0;  // wide levels only: no staging
    SP_TRY(s->flags.ensure((size_t)std::max(1, sc.grid)));
    SP_TRY(s->status.ensure(1));
    return SPTRSV_OK;
}

sptrsv_status enqueue_solve(sptrsv_system* s, const void* b, void* x, int nrhs, int64_t ld,
                            unsigned long long* stamps, cudaStream_t st) {
    if (nrhs < 1 || nrhs > 1024 || ld < s->n || (s->n > 0 && (!b || !x))) {
        set_error("solve: bad arguments (nrhs=%d ld=%lld n=%lld)", nrhs, (long long)ld, (long long)s->n);
        return SPTRSV_ERR_INVALID;
    }
    if (s->n == 0) return SPTRSV_OK;
    SP_TRY(prepare_schedule(s, nrhs));
    const size_t vb = s->dtype == SPTRSV_F64 ? 8 : 4;
    if (s->xp.n < (size_t)s->n * nrhs * vb) SP_TRY(s->xp.alloc((size_t)s->n * nrhs * vb));
    if (s->dtype == SPTRSV_F64) return launch_solve<double>(s, b, x, nrhs, ld, stamps, st);
    return launch_solve<float>(s, b, x, nrhs, ld, stamps, st);
}

}  // namespace sp

namespace sp {
namespace {
struct TuneKey {
    int64_t n, m, nnz_c, nnz_e;
    int nrhs, dtype;
    bool operator<(const TuneKey& o) const {
        return std::tie(n, m, nnz_c, nnz_e, nrhs, dtype) < std::tie(o.n, o.m, o.nnz_c, o.nnz_e, o.nrhs, o.dtype);
    }
};
struct TuneVal {
    int block, run_width, lpr;
    double us;
    int cluster = 0;
    int64_t cluster_rows = 0;
    int tiles = 0;
    int shared_x = 0;
};
std::mutex g_stune_mu;
std::map<TuneKey, TuneVal> g_stune_cache;
}  // namespace
}  // namespace sp

extern "C" sptrsv_status sptrsv_system_autotune(sptrsv_system* s, int32_t nrhs, double* best_us,
                                                sptrsv_stream_t stream) {
    using namespace sp;
    if (!s || nrhs < 1) { set_error("system_autotune: bad argument"); return SPTRSV_ERR_INVALID; }
    cudaStream_t st = (cudaStream_t)stream;
    if (s->n == 0) {
        if (best_us) *best_us = 0;
        return SPTRSV_OK;
    }
    const TuneKey key{s->n, s->m, s->nnz_c, s->nnz_e, nrhs, s->dtype};
    {
        std::lock_guard<std::mutex> lk(g_stune_mu);
        auto f = g_stune_cache.find(key);
        if (f != g_stune_cache.end()) {
            s->block = f->second.block;
            s->run_width = f->second.run_width;
            s->lpr = f->second.lpr;
            s->cluster = f->second.cluster;
            s->cluster_rows = f->second.cluster_rows;
            s->tiles = f->second.tiles;
            s->shared_x = f->second.shared_x;
            if (best_us) *best_us = f->second.us;
            return prepare_schedule(s, nrhs);
        }
    }
    const size_t vb = s->dtype == SPTRSV_F64 ? 8 : 4;
    Scratch b, x;
    SP_TRY(b.alloc((size_t)s->n * nrhs * vb, st));
    SP_TRY(x.alloc((size_t)s->n * nrhs * vb, st));
    SP_CUDA(cudaMemsetAsync(b.p, 0, (size_t)s->n * nrhs * vb, st));
    std::vector<int> lprs;
    if (nrhs == 1) lprs = {1, 2, 4};
    else {
        int p = 1;
        while (p < nrhs && p < 32) p <<= 1;
        lprs = {std::max(1, p / 2), p};
        // one lane per row and right-hand side: thin levels run in the fast executor
        if (nrhs <= FAST_MAX_RHS && p / 2 > 1) lprs.push_back(1);
    }
    std::vector<int> widths = {0, 64, -1};
    if (s->m <= 256) widths.push_back(-2);  // one launch per level
    cudaEvent_t e0, e1;
    SP_CUDA(cudaEventCreate(&e0));
    SP_CUDA(cudaEventCreate(&e1));
    TuneVal best{512, 0, 0, 1e300};
    const int old_block = s->block, old_rw = s->run_width, old_lpr = s->lpr, old_cl = s->cluster, old_tl = s->tiles;
    const int old_sx = s->shared_x;
    s->shared_x = 0;
    const int64_t old_clr = s->cluster_rows;
    sptrsv_status rc = SPTRSV_OK;
    // best of 3 timed solves of the current settings, in microseconds
    auto time_current = [&](double* us) -> sptrsv_status {
        s->sched.nrhs = -1;
        SP_TRY(enqueue_solve(s, b.p, x.p, nrhs, s->n, nullptr, st));
        float bestms = 1e30f;
        for (int rep = 0; rep < 3; ++rep) {
            cudaEventRecord(e0, st);
            SP_TRY(enqueue_solve(s, b.p, x.p, nrhs, s->n, nullptr, st));
            cudaEventRecord(e1, st);
            cudaEventSynchronize(e1);
            float ms = 0;
            cudaEventElapsedTime(&ms, e0, e1);
            bestms = std::min(bestms, ms);
        }
        *us = bestms * 1e3;
        return SPTRSV_OK;
    };
    // lanes per row x widest single-CTA level x {no cluster with and without tiled wide levels,
    // a cluster of 16 or 8 CTAs for mid-width levels with and without the shared-x exchange};
    // then the widest cluster level for the best
    const int cls[][4] = {{1, 0, 0, 0}, {1, 0, 1, 0}, {16, 16384, 1, 0}, {8, 16384, 1, 0}, {16, 16384, 1, 1},
                          {8, 16384, 1, 1}};
    for (int lpr : lprs) {
        for (int rw : widths) {
            if (rw == -2 && lpr != lprs[0]) continue;
            for (const auto& c : cls) {
                if (rw == -2 && (c[0] != 1 || c[2] != 1)) continue;  // one launch per level: no clusters, no tiles
                if (nrhs > 1 && c[0] == 1 && c[2] == 0) continue;   // tiles are for one right-hand side
                if (nrhs > 1 && c[3] == 1) continue;                 // and the shared-x exchange
                s->block = 512;
                s->run_width = rw;
                s->lpr = lpr;
                s->cluster = c[0];
                s->cluster_rows = c[1];
                s->tiles = c[2];
                s->shared_x = c[3];
                double us = 0;
                rc = time_current(&us);
                if (rc != SPTRSV_OK) break;
                if (us < best.us) best = TuneVal{512, rw, lpr, us, c[0], c[1], c[2], c[3]};
            }
            if (rc != SPTRSV_OK) break;
        }
        if (rc != SPTRSV_OK) break;
    }
    if (rc == SPTRSV_OK && best.cluster > 1) {
        s->block = best.block;
        s->run_width = best.run_width;
        s->lpr = best.lpr;
        s->cluster = best.cluster;
        s->tiles = best.tiles;
        s->shared_x = best.shared_x;
        for (int64_t rows : {(int64_t)4096, (int64_t)65536}) {
            s->cluster_rows = rows;
            double us = 0;
            rc = time_current(&us);
            if (rc != SPTRSV_OK) break;
            if (us < best.us)
                best = TuneVal{best.block, best.run_width, best.lpr, us, best.cluster, rows, best.tiles, best.shared_x};
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc != SPTRSV_OK) {
        s->block = old_block;
        s->run_width = old_rw;
        s->lpr = old_lpr;
        s->cluster = old_cl;
        s->cluster_rows = old_clr;
        s->tiles = old_tl;
        s->shared_x = old_sx;
        s->sched.nrhs = -1;
        return rc;
    }
    SP_TRY(sptrsv_solve_status(s, stream));
    s->block = best.block;
    s->run_width = best.run_width;
    s->lpr = best.lpr;
    s->cluster = best.cluster;
    s->cluster_rows = best.cluster_rows;
    s->tiles = best.tiles;
    s->shared_x = best.shared_x;
    s->sched.nrhs = -1;
    {
        std::lock_guard<std::mutex> lk(g_stune_mu);
        g_stune_cache[key] = best;
    }
    if (best_us) *best_us = best.us;
    return prepare_schedule(s, nrhs);
}

namespace sp {
sptrsv_status time_solve_us(sptrsv_system* s, int reps, double* us, cudaStream_t st) {
    *us = 0;
    if (s->n == 0) return SPTRSV_OK;
    const size_t vb = s->dtype == SPTRSV_F64 ? 8 : 4;
    Scratch b, x;
    SP_TRY(b.alloc((size_t)s->n * vb, st));
    SP_TRY(x.alloc((size_t)s->n * vb, st));
    SP_CUDA(cudaMemsetAsync(b.p, 0, (size_t)s->n * vb, st));
    SP_TRY(enqueue_solve(s, b.p, x.p, 1, s->n, nullptr, st));
    cudaEvent_t e0, e1;
    SP_CUDA(cudaEventCreate(&e0));
    SP_CUDA(cudaEventCreate(&e1));
    std::vector<float> t;
    sptrsv_status rc = SPTRSV_OK;
    for (int r = 0; r < reps && rc == SPTRSV_OK; ++r) {
        cudaEventRecord(e0, st);
        rc = enqueue_solve(s, b.p, x.p, 1, s->n, nullptr, st);
        cudaEventRecord(e1, st);
        cudaEventSynchronize(e1);
        float ms = 0;
        cudaEventElapsedTime(&ms, e0, e1);
        t.push_back(ms);
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    SP_TRY(rc);
    std::sort(t.begin(), t.end());
    *us = t[t.size() / 2] * 1e3;
    return sptrsv_solve_status(s, st);
}
}  // namespace sp

// Test hook: the host block cutter on caller arrays (no device work).
extern "C" sptrsv_status sptrsv_debug_run_blocks(const int32_t* level_ptr_host, int64_t m, const int32_t* cptr_host,
                                                 int32_t nrhs, int32_t lanes_per_row, int32_t value_bytes,
                                                 int32_t* blocks_host, int64_t capacity, int64_t* count_out,
                                                 int32_t* geometry_out) {
    using namespace sp;
    if (!level_ptr_host || !cptr_host || !count_out || m < 0 || nrhs < 1 || lanes_per_row < 1 ||
        (value_bytes != 4 && value_bytes != 8)) {
        set_error("debug_run_blocks: invalid argument");
        return SPTRSV_ERR_INVALID;
    }
    const RunGeom g = run_geometry(nrhs, value_bytes);
    const int recs = fast_rec_capacity(value_bytes, g);
    if (geometry_out) {
        geometry_out[0] = g.stage_rows;
        geometry_out[1] = g.stage_entries;
        geometry_out[2] = g.ring_rows;
        geometry_out[3] = recs;
    }
    std::vector<int4> out;
    if (m > 0 && build_run_blocks(level_ptr_host, cptr_host, 0, m, g.stage_rows, g.stage_entries, lanes_per_row, nrhs,
                                  recs, out) != 0) {
        set_error("debug_run_blocks: a row has more coefficients than the staging area");
        return SPTRSV_ERR_UNSUPPORTED;
    }
    *count_out = (int64_t)out.size();
    if ((int64_t)out.size() > capacity || (!blocks_host && !out.empty())) {
        set_error("debug_run_blocks: %zu blocks, capacity %lld", out.size(), (long long)capacity);
        return SPTRSV_ERR_INVALID;
    }
    for (size_t i = 0; i < out.size(); ++i) {
        blocks_host[4 * i] = out[i].x;
        blocks_host[4 * i + 1] = out[i].y;
        blocks_host[4 * i + 2] = out[i].z;
        blocks_host[4 * i + 3] = out[i].w;
    }
    return SPTRSV_OK;
}
