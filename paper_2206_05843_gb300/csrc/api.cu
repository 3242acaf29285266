// api.cu -- ABI entry points for validation and level-set analysis.
#include <cstring>

#include "internal.cuh"

using namespace sp;

extern "C" {

sptrsv_status sptrsv_last_error(char* buf, size_t len) {
    if (!buf || len == 0) return SPTRSV_ERR_INVALID;
    strncpy(buf, get_error(), len - 1);
    buf[len - 1] = '\0';
    return SPTRSV_OK;
}

sptrsv_status sptrsv_validate(const sptrsv_csr* L, sptrsv_stream_t stream) {
    return validate_csr(L, (cudaStream_t)stream);
}

sptrsv_status sptrsv_analyse(const sptrsv_csr* L, sptrsv_levels** out, sptrsv_stream_t stream) {
    if (!out) { set_error("analyse: null output"); return SPTRSV_ERR_INVALID; }
    *out = nullptr;
    cudaStream_t st = (cudaStream_t)stream;
    SP_TRY(validate_csr(L, st));
    sptrsv_levels* h = new (std::nothrow) sptrsv_levels();
    if (!h) { set_error("host allocation failed"); return SPTRSV_ERR_OOM; }
    DepCsr d;
    d.n = L->n;
    d.rowptr = L->rowptr;
    d.colidx = L->colidx;
    d.diag_last = 1;
    sptrsv_status rc = analyse_dep(d, h->lv, st);
    if (rc != SPTRSV_OK) {
        delete h;
        return rc;
    }
    *out = h;
    return SPTRSV_OK;
}

sptrsv_status sptrsv_levels_stats(const sptrsv_levels* h, sptrsv_level_stats* o) {
    if (!h || !o) { set_error("levels_stats: null argument"); return SPTRSV_ERR_INVALID; }
    o->n = h->lv.n;
    o->m = h->lv.m;
    o->nnz = h->lv.nnz;
    o->total_cost = h->lv.total_cost;
    o->avg_cost = h->lv.avg;
    o->max_width = h->lv.max_width;
    return SPTRSV_OK;
}

sptrsv_status sptrsv_levels_export(const sptrsv_levels* h, int32_t* level_dev, int32_t* level_ptr_dev,
                                   int32_t* level_rows_dev, int64_t* rows_dev, int64_t* nnz_dev, int64_t* cost_dev,
                                   sptrsv_stream_t stream) {
    if (!h) { set_error("levels_export: null levels"); return SPTRSV_ERR_INVALID; }
    cudaStream_t st = (cudaStream_t)stream;
    const Levels& lv = h->lv;
    const int64_t n = lv.n, m = lv.m;
    if (level_dev && n) SP_CUDA(cudaMemcpyAsync(level_dev, lv.level.p, n * 4, cudaMemcpyDeviceToDevice, st));
    if (level_ptr_dev) SP_CUDA(cudaMemcpyAsync(level_ptr_dev, lv.level_ptr.p, (m + 1) * 4, cudaMemcpyDeviceToDevice, st));
    if (level_rows_dev && n)
        SP_CUDA(cudaMemcpyAsync(level_rows_dev, lv.level_rows.p, n * 4, cudaMemcpyDeviceToDevice, st));
    if (rows_dev && m) SP_CUDA(cudaMemcpyAsync(rows_dev, lv.lrows.p, m * 8, cudaMemcpyDeviceToDevice, st));
    if (nnz_dev && m) SP_CUDA(cudaMemcpyAsync(nnz_dev, lv.lnnz.p, m * 8, cudaMemcpyDeviceToDevice, st));
    if (cost_dev && m) SP_CUDA(cudaMemcpyAsync(cost_dev, lv.lcost.p, m * 8, cudaMemcpyDeviceToDevice, st));
    return SPTRSV_OK;
}

void sptrsv_levels_destroy(sptrsv_levels* h) { delete h; }

}  // extern "C"
