// system.cu -- stored systems: level-ordered packing, export, and the system ABI.
//
// A stored system keeps every row in level order ("positions"), normalised so that
//   x_r = dinv_r * b_r + sum_m e_rm b_m - sum_k c_rk x_k
// with dinv_r = 1 / L_rr, c_rk = L_rk / L_rr for rows that kept their equation and the
// rearranged coefficients of Section II.B for rewritten rows (whose explicit E row holds
// the b-coefficients other than the diagonal one).  Dependency columns are stored as
// positions, so a level's rows and their coefficients are contiguous in memory.
#include <algorithm>
#include <cmath>

#include "system.cuh"

namespace sp {
namespace {

inline unsigned nblk(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

template <typename T>
__global__ void k_pack_counts(int64_t n, const int32_t* perm, const int32_t* rowptr, RewriteHeap rw,
                              int32_t* ccnt, int32_t* ecnt) {
    int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n) return;
    int32_t r = perm[p];
    bool mv = rw.moved && rw.moved[r];
    ccnt[p] = mv ? rw.c_cnt[r] : rowptr[r + 1] - rowptr[r] - 1;
    ecnt[p] = mv ? rw.e_cnt[r] : 0;
}

template <typename T>
__global__ void k_pack_fill(int64_t n, const int32_t* perm, const int32_t* pos, const int32_t* rowptr,
                            const int32_t* colidx, const T* vals, RewriteHeap rw, const int64_t* cptr64,
                            const int64_t* eptr64, int32_t* cptr, int32_t* ccol, T* cval, T* dinv, int32_t* eptr,
                            int32_t* ecol, T* eval) {
    int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p > n) return;
    cptr[p] = (int32_t)cptr64[p];
    eptr[p] = (int32_t)eptr64[p];
    if (p == n) return;
    int32_t r = perm[p];
    int64_t a = rowptr[r], e = rowptr[r + 1] - 1;
    double d = (double)vals[e];
    dinv[p] = (T)(1.0 / d);
    int64_t o = cptr64[p];
    if (rw.moved && rw.moved[r]) {
        int64_t h = rw.c_off[r];
        for (int32_t q = 0; q < rw.c_cnt[r]; ++q) {
            ccol[o + q] = pos[rw.col[h + q]];
            cval[o + q] = (T)rw.val[h + q];
        }
        int64_t he = rw.e_off[r], oe = eptr64[p];
        for (int32_t q = 0; q < rw.e_cnt[r]; ++q) {
            ecol[oe + q] = rw.col[he + q];
            eval[oe + q] = (T)rw.val[he + q];
        }
    } else {
        for (int64_t q = a; q < e; ++q) {
            ccol[o + (q - a)] = pos[colidx[q]];
            cval[o + (q - a)] = (T)((double)vals[q] / d);
        }
    }
}

// export in the original numbering
__global__ void k_export_counts(int64_t n, const int32_t* pos, const int32_t* cptr, const int32_t* eptr,
                                int32_t* ccnt, int32_t* ecnt) {
    int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n) return;
    int32_t p = pos[r];
    ccnt[r] = cptr[p + 1] - cptr[p];
    ecnt[r] = eptr ? eptr[p + 1] - eptr[p] : 0;
}

template <typename T>
__global__ void k_export_fill(int64_t n, const int32_t* pos, const int32_t* perm, const int32_t* cptr,
                              const int32_t* ccol, const T* cval, const T* dinv, const int32_t* eptr,
                              const int32_t* ecol, const T* eval, const int64_t* ocptr, const int64_t* oeptr,
                              int32_t* xccol, T* xcval, T* xdinv, int32_t* xecol, T* xeval) {
    int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n) return;
    int32_t p = pos[r];
    if (xdinv) xdinv[r] = dinv[p];
    int64_t o = ocptr[r];
    for (int32_t q = cptr[p]; q < cptr[p + 1]; ++q, ++o) {
        if (xccol) xccol[o] = perm[ccol[q]];
        if (xcval) xcval[o] = cval[q];
    }
    if (eptr) {
        int64_t oe = oeptr[r];
        for (int32_t q = eptr[p]; q < eptr[p + 1]; ++q, ++oe) {
            if (xecol) xecol[oe] = ecol[q];
            if (xeval) xeval[oe] = eval[q];
        }
    }
}

}  // namespace

sptrsv_status pack_system(sptrsv_system* s, const sptrsv_csr* L, const RewriteHeap* rwp, cudaStream_t st) {
    const int64_t n = s->n;
    RewriteHeap rw = rwp ? *rwp : RewriteHeap{};
    const size_t vb = s->dtype == SPTRSV_F64 ? 8 : 4;
    Scratch cc, ec, c64, e64;
    SP_TRY(cc.alloc((n + 1) * sizeof(int32_t), st));
    SP_TRY(ec.alloc((n + 1) * sizeof(int32_t), st));
    SP_TRY(c64.alloc((n + 1) * sizeof(int64_t), st));
    SP_TRY(e64.alloc((n + 1) * sizeof(int64_t), st));
    if (s->dtype == SPTRSV_F64)
        k_pack_counts<double><<<nblk(n, 256), 256, 0, st>>>(n, s->lv.level_rows.p, L->rowptr, rw, cc.as<int32_t>(),
                                                           ec.as<int32_t>());
    else
        k_pack_counts<float><<<nblk(n, 256), 256, 0, st>>>(n, s->lv.level_rows.p, L->rowptr, rw, cc.as<int32_t>(),
                                                          ec.as<int32_t>());
    SP_CUDA(cudaGetLastError());
    SP_TRY(scan_exclusive_i32_to_i64(cc.as<int32_t>(), c64.as<int64_t>(), n, st));
    SP_TRY(scan_exclusive_i32_to_i64(ec.as<int32_t>(), e64.as<int64_t>(), n, st));
    int64_t tot[2];
    SP_CUDA(cudaMemcpyAsync(&tot[0], c64.as<int64_t>() + n, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
    SP_CUDA(cudaMemcpyAsync(&tot[1], e64.as<int64_t>() + n, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
    SP_CUDA(cudaStreamSynchronize(st));
    if (tot[0] >= INT32_MAX || tot[1] >= INT32_MAX) {
        set_error("stored system has %lld / %lld entries; int32 offsets are exceeded", (long long)tot[0],
                  (long long)tot[1]);
        return SPTRSV_ERR_UNSUPPORTED;
    }
    s->nnz_c = tot[0];
    s->nnz_e = tot[1];
    SP_TRY(s->cptr.alloc(n + 1));
    SP_TRY(s->eptr.alloc(n + 1));
    SP_TRY(s->ccol.alloc(std::max<int64_t>(1, tot[0])));
    SP_TRY(s->cval.alloc(std::max<int64_t>(1, tot[0]) * vb));
    SP_TRY(s->ecol.alloc(std::max<int64_t>(1, tot[1])));
    SP_TRY(s->eval.alloc(std::max<int64_t>(1, tot[1]) * vb));
    SP_TRY(s->dinv.alloc(std::max<int64_t>(1, n) * vb));
    if (s->dtype == SPTRSV_F64)
        k_pack_fill<double><<<nblk(n + 1, 256), 256, 0, st>>>(
            n, s->lv.level_rows.p, s->lv.pos.p, L->rowptr, L->colidx, (const double*)L->vals, rw, c64.as<int64_t>(),
            e64.as<int64_t>(), s->cptr.p, s->ccol.p, (double*)s->cval.p, (double*)s->dinv.p, s->eptr.p, s->ecol.p,
            (double*)s->eval.p);
    else
        k_pack_fill<float><<<nblk(n + 1, 256), 256, 0, st>>>(
            n, s->lv.level_rows.p, s->lv.pos.p, L->rowptr, L->colidx, (const float*)L->vals, rw, c64.as<int64_t>(),
            e64.as<int64_t>(), s->cptr.p, s->ccol.p, (float*)s->cval.p, (float*)s->dinv.p, s->eptr.p, s->ecol.p,
            (float*)s->eval.p);
    SP_CUDA(cudaGetLastError());
    SP_CUDA(cudaStreamSynchronize(st));
    return SPTRSV_OK;
}

}  // namespace sp

using namespace sp;

extern "C" {

sptrsv_status sptrsv_system_plain(const sptrsv_csr* L, const sptrsv_levels* lvh, sptrsv_system** out,
                                  sptrsv_stream_t stream) {
    if (!L || !lvh || !out) { set_error("system_plain: null argument"); return SPTRSV_ERR_INVALID; }
    *out = nullptr;
    cudaStream_t st = (cudaStream_t)stream;
    const Levels& lv = lvh->lv;
    if (lv.n != L->n) { set_error("system_plain: levels belong to another matrix"); return SPTRSV_ERR_INVALID; }
    sptrsv_system* s = new (std::nothrow) sptrsv_system();
    if (!s) { set_error("host allocation failed"); return SPTRSV_ERR_OOM; }
    s->n = L->n;
    s->m = lv.m;
    s->dtype = L->dtype;
    s->nnz_l = L->nnz;
    s->stored_nnz = L->nnz;
    sptrsv_status rc = SPTRSV_OK;
    // copy the analysis (levels, level pointer, permutation, inverse) into the system
    auto copy_levels = [&]() -> sptrsv_status {
        Levels& d = s->lv;
        d.n = lv.n; d.m = lv.m; d.nnz = lv.nnz; d.total_cost = lv.total_cost; d.max_width = lv.max_width;
        d.avg = lv.avg;
        d.h_level_ptr = lv.h_level_ptr;
        d.h_lcost = lv.h_lcost;
        int64_t n1 = std::max<int64_t>(1, lv.n);
        SP_TRY(d.level.alloc(n1));
        SP_TRY(d.level_rows.alloc(n1));
        SP_TRY(d.pos.alloc(n1));
        SP_TRY(d.level_ptr.alloc(lv.m + 1));
        SP_CUDA(cudaMemcpyAsync(d.level.p, lv.level.p, n1 * 4, cudaMemcpyDeviceToDevice, st));
        SP_CUDA(cudaMemcpyAsync(d.level_rows.p, lv.level_rows.p, n1 * 4, cudaMemcpyDeviceToDevice, st));
        SP_CUDA(cudaMemcpyAsync(d.pos.p, lv.pos.p, n1 * 4, cudaMemcpyDeviceToDevice, st));
        SP_CUDA(cudaMemcpyAsync(d.level_ptr.p, lv.level_ptr.p, (lv.m + 1) * 4, cudaMemcpyDeviceToDevice, st));
        SP_TRY(s->target.alloc(n1));
        SP_CUDA(cudaMemcpyAsync(s->target.p, lv.level.p, n1 * 4, cudaMemcpyDeviceToDevice, st));
        return SPTRSV_OK;
    };
    rc = copy_levels();
    if (rc == SPTRSV_OK && L->n > 0) rc = pack_system(s, L, nullptr, st);
    if (rc != SPTRSV_OK) {
        delete s;
        return rc;
    }
    *out = s;
    return SPTRSV_OK;
}

sptrsv_status sptrsv_system_info_get(const sptrsv_system* s, sptrsv_system_info* o) {
    if (!s || !o) { set_error("system_info: null argument"); return SPTRSV_ERR_INVALID; }
    o->n = s->n;
    o->m = s->m;
    o->nnz_c = s->nnz_c;
    o->nnz_e = s->nnz_e;
    o->rows_moved = s->rows_moved;
    o->stored_nnz = s->stored_nnz;
    o->nnz_l = s->nnz_l;
    o->segments = (int64_t)s->sched.h_segs.size();
    o->run_levels = s->sched.run_levels;
    o->dtype = s->dtype;
    o->rewritten = s->rewritten;
    o->avg_cost = s->avg;
    o->block = s->block;
    o->run_width = s->run_width;
    o->lanes_per_row = s->lpr;
    o->strategy_used = s->strategy_used;
    const sp::Schedule& sc = s->sched;
    if (!sc.segs.p) o->launches = 0;
    else if (sc.run_width == -2) o->launches = (int32_t)s->m;
    else o->launches = sc.h_segs.empty() ? 0 : 1 + sc.pre;
    o->ctas = sc.segs.p ? sc.grid : 0;
    for (int i = 0; i < 4; ++i) o->candidate_us[i] = s->cand_us[i];
    o->cluster = sc.segs.p ? sc.csize : 1;
    o->cluster_setting = s->cluster;
    o->cluster_levels = sc.segs.p ? sc.cluster_levels : 0;
    o->cluster_rows = s->cluster_rows;
    o->tiled_levels = sc.segs.p ? sc.tiled_levels : 0;
    o->tiles_setting = s->tiles;
    o->reserved0 = 0;
    o->shared_x_levels = sc.segs.p ? sc.dsm_levels : 0;
    o->shared_x_setting = s->shared_x;
    o->reserved1 = 0;
    return SPTRSV_OK;
}

sptrsv_status sptrsv_system_export(const sptrsv_system* s, int32_t* target_dev, int32_t* level_dev, int64_t* cptr_dev,
                                   int32_t* ccol_dev, void* cval_dev, void* dinv_dev, int64_t* eptr_dev,
                                   int32_t* ecol_dev, void* eval_dev, sptrsv_stream_t stream) {
    if (!s) { set_error("system_export: null system"); return SPTRSV_ERR_INVALID; }
    cudaStream_t st = (cudaStream_t)stream;
    const int64_t n = s->n;
    if (n == 0) return SPTRSV_OK;
    if (target_dev) SP_CUDA(cudaMemcpyAsync(target_dev, s->target.p, n * 4, cudaMemcpyDeviceToDevice, st));
    if (level_dev) SP_CUDA(cudaMemcpyAsync(level_dev, s->lv.level.p, n * 4, cudaMemcpyDeviceToDevice, st));
    Scratch cc, ec, c64, e64;
    SP_TRY(cc.alloc((n + 1) * 4, st));
    SP_TRY(ec.alloc((n + 1) * 4, st));
    SP_TRY(c64.alloc((n + 1) * 8, st));
    SP_TRY(e64.alloc((n + 1) * 8, st));
    const int32_t* ep = s->nnz_e > 0 ? s->eptr.p : nullptr;
    k_export_counts<<<nblk(n, 256), 256, 0, st>>>(n, s->lv.pos.p, s->cptr.p, ep, cc.as<int32_t>(), ec.as<int32_t>());
    SP_CUDA(cudaGetLastError());
    SP_TRY(scan_exclusive_i32_to_i64(cc.as<int32_t>(), c64.as<int64_t>(), n, st));
    SP_TRY(scan_exclusive_i32_to_i64(ec.as<int32_t>(), e64.as<int64_t>(), n, st));
    if (cptr_dev) SP_CUDA(cudaMemcpyAsync(cptr_dev, c64.p, (n + 1) * 8, cudaMemcpyDeviceToDevice, st));
    if (eptr_dev) SP_CUDA(cudaMemcpyAsync(eptr_dev, e64.p, (n + 1) * 8, cudaMemcpyDeviceToDevice, st));
    if (s->dtype == SPTRSV_F64)
        k_export_fill<double><<<nblk(n, 256), 256, 0, st>>>(
            n, s->lv.pos.p, s->lv.level_rows.p, s->cptr.p, s->ccol.p, (const double*)s->cval.p,
            (const double*)s->dinv.p, ep, s->ecol.p, (const double*)s->eval.p, c64.as<int64_t>(), e64.as<int64_t>(),
            ccol_dev, (double*)cval_dev, (double*)dinv_dev, ecol_dev, (double*)eval_dev);
    else
        k_export_fill<float><<<nblk(n, 256), 256, 0, st>>>(
            n, s->lv.pos.p, s->lv.level_rows.p, s->cptr.p, s->ccol.p, (const float*)s->cval.p,
            (const float*)s->dinv.p, ep, s->ecol.p, (const float*)s->eval.p, c64.as<int64_t>(), e64.as<int64_t>(),
            ccol_dev, (float*)cval_dev, (float*)dinv_dev, ecol_dev, (float*)eval_dev);
    SP_CUDA(cudaGetLastError());
    return SPTRSV_OK;
}

void sptrsv_system_destroy(sptrsv_system* s) { delete s; }

sptrsv_status sptrsv_solve(const sptrsv_system* s, const void* b_dev, void* x_dev, int32_t nrhs, int64_t ld,
                           sptrsv_stream_t stream) {
    if (!s) { set_error("solve: null system"); return SPTRSV_ERR_INVALID; }
    return enqueue_solve(const_cast<sptrsv_system*>(s), b_dev, x_dev, nrhs, ld, nullptr, (cudaStream_t)stream);
}

sptrsv_status sptrsv_solve_timed(const sptrsv_system* s, const void* b_dev, void* x_dev, int32_t nrhs, int64_t ld,
                                 uint64_t* stamps_dev, sptrsv_stream_t stream) {
    if (!s) { set_error("solve: null system"); return SPTRSV_ERR_INVALID; }
    cudaStream_t st = (cudaStream_t)stream;
    if (stamps_dev && s->m > 0) SP_CUDA(cudaMemsetAsync(stamps_dev, 0, s->m * sizeof(uint64_t), st));
    return enqueue_solve(const_cast<sptrsv_system*>(s), b_dev, x_dev, nrhs, ld, (unsigned long long*)stamps_dev, st);
}

sptrsv_status sptrsv_solve_status(const sptrsv_system* s, sptrsv_stream_t stream) {
    if (!s) { set_error("solve_status: null system"); return SPTRSV_ERR_INVALID; }
    cudaStream_t st = (cudaStream_t)stream;
    SP_CUDA(cudaStreamSynchronize(st));
    if (!s->status.p) return SPTRSV_OK;
    int h = 0;
    SP_CUDA(cudaMemcpy(&h, s->status.p, sizeof(int), cudaMemcpyDeviceToHost));
    SP_CUDA(cudaMemset(s->status.p, 0, sizeof(int)));
    return map_dev_status(h, "solve");
}

sptrsv_status sptrsv_debug_set_wait(sptrsv_system* s, int64_t withhold_segment, int64_t timeout_ns) {
    if (!s) { set_error("debug_set_wait: null system"); return SPTRSV_ERR_INVALID; }
    s->withhold = withhold_segment < 0 || withhold_segment > INT32_MAX ? -1 : (int)withhold_segment;
    s->timeout_ns = timeout_ns > 0 ? timeout_ns : 0;
    return SPTRSV_OK;
}

sptrsv_status sptrsv_system_tune(sptrsv_system* s, int32_t block, int32_t run_width, int32_t lanes_per_row) {
    if (!s) { set_error("system_tune: null system"); return SPTRSV_ERR_INVALID; }
    if (lanes_per_row < 0 || lanes_per_row > 32 || (lanes_per_row & (lanes_per_row - 1))) {
        set_error("system_tune: lanes_per_row must be 0 or a power of two <= 32");
        return SPTRSV_ERR_INVALID;
    }
    if (block < 0 || block > 1024 || run_width < -2) { set_error("system_tune: bad block / run width"); return SPTRSV_ERR_INVALID; }
    if (block) s->block = block;
    if (run_width) s->run_width = run_width;
    if (lanes_per_row) s->lpr = lanes_per_row;
    s->sched.nrhs = -1;  // rebuild on the next solve
    return SPTRSV_OK;
}

sptrsv_status sptrsv_system_tune_cluster(sptrsv_system* s, int32_t cluster, int64_t cluster_rows, int32_t tiles,
                                         int32_t shared_x) {
    if (!s) { set_error("system_tune_cluster: null system"); return SPTRSV_ERR_INVALID; }
    if (cluster > 16) { set_error("system_tune_cluster: at most 16 CTAs per cluster"); return SPTRSV_ERR_INVALID; }
    if (tiles > 1) { set_error("system_tune_cluster: tiles must be 0 (automatic) or 1 (never)"); return SPTRSV_ERR_INVALID; }
    if (shared_x > 1) {
        set_error("system_tune_cluster: shared_x must be 0 (automatic) or 1 (never)");
        return SPTRSV_ERR_INVALID;
    }
    if (cluster >= 0) s->cluster = cluster;
    if (cluster_rows >= 0) s->cluster_rows = cluster_rows;
    if (tiles >= 0) s->tiles = tiles;
    if (shared_x >= 0) s->shared_x = shared_x;
    s->sched.nrhs = -1;  // rebuild on the next solve
    return SPTRSV_OK;
}

}  // extern "C"
