// upper.cu -- upper-triangular systems U x = b (the second triangular solve of an ILU
// preconditioner, Section I) on the lower-triangular path.
//
// Reversing the index order, i -> n-1-i, turns U (diagonal first in each row) into a
// lower-triangular matrix with the diagonal last: row i of the reversed matrix is row
// n-1-i of U with its entries in reverse order and columns c -> n-1-c.  Its row
// pointers have a closed form, rowptr'[i] = nnz - rowptr[n-i], so no scan is needed.
// Analysis, rewriting and the solve then run unchanged on the reversed matrix, and
// sptrsv_system_reverse_rows re-indexes the stored system so that it reads b and writes
// x in U's own numbering.
#include "system.cuh"

namespace sp {
namespace {

inline unsigned nblk(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

template <typename T>
__global__ void k_upper_to_lower(int64_t n, int64_t nnz, const int32_t* urp, const int32_t* uci, const T* uv,
                                 int32_t* lrp, int32_t* lci, T* lv) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i > n) return;
    lrp[i] = (int32_t)(nnz - urp[n - i]);
    if (i == n) return;
    const int64_t r = n - 1 - i;
    const int64_t a = urp[r], e = urp[r + 1];
    int64_t o = nnz - urp[n - i];
    for (int64_t src = e - 1; src >= a; --src, ++o) {
        lci[o] = (int32_t)(n - 1 - uci[src]);
        lv[o] = uv[src];
    }
}

__global__ void k_reverse_index_values(int64_t count, int64_t n, int32_t* a) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < count) a[i] = (int32_t)(n - 1 - a[i]);
}

__global__ void k_reverse_order(int64_t n, const int32_t* in, int32_t* out) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = in[n - 1 - i];
}

__global__ void k_inverse(const int32_t* perm, int32_t* inv, int64_t n) {
    int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p < n) inv[perm[p]] = (int32_t)p;
}

}  // namespace
}  // namespace sp

using namespace sp;

extern "C" {

sptrsv_status sptrsv_upper_to_lower(const sptrsv_csr* U, int32_t* rowptr_dev, int32_t* colidx_dev, void* vals_dev,
                                    sptrsv_stream_t stream) {
    if (!U || U->n < 0 || U->nnz < U->n || U->n >= INT32_MAX || U->nnz >= INT32_MAX) {
        set_error("upper_to_lower: bad matrix");
        return SPTRSV_ERR_INVALID;
    }
    if (!rowptr_dev || (U->n > 0 && (!colidx_dev || !vals_dev || !U->rowptr || !U->colidx || !U->vals))) {
        set_error("upper_to_lower: null array");
        return SPTRSV_ERR_INVALID;
    }
    cudaStream_t st = (cudaStream_t)stream;
    const int64_t n = U->n;
    if (U->dtype == SPTRSV_F64)
        k_upper_to_lower<double><<<nblk(n + 1, 256), 256, 0, st>>>(n, U->nnz, U->rowptr, U->colidx,
                                                                  (const double*)U->vals, rowptr_dev, colidx_dev,
                                                                  (double*)vals_dev);
    else if (U->dtype == SPTRSV_F32)
        k_upper_to_lower<float><<<nblk(n + 1, 256), 256, 0, st>>>(n, U->nnz, U->rowptr, U->colidx,
                                                                 (const float*)U->vals, rowptr_dev, colidx_dev,
                                                                 (float*)vals_dev);
    else {
        set_error("upper_to_lower: unknown dtype %d", U->dtype);
        return SPTRSV_ERR_INVALID;
    }
    SP_CUDA(cudaGetLastError());
    return SPTRSV_OK;
}

sptrsv_status sptrsv_system_reverse_rows(sptrsv_system* s, sptrsv_stream_t stream) {
    if (!s) { set_error("system_reverse_rows: null system"); return SPTRSV_ERR_INVALID; }
    cudaStream_t st = (cudaStream_t)stream;
    const int64_t n = s->n;
    if (n == 0) return SPTRSV_OK;
    // rows of the stored order and the b columns of the E rows
    k_reverse_index_values<<<nblk(n, 256), 256, 0, st>>>(n, n, s->lv.level_rows.p);
    if (s->nnz_e > 0) k_reverse_index_values<<<nblk(s->nnz_e, 256), 256, 0, st>>>(s->nnz_e, n, s->ecol.p);
    k_inverse<<<nblk(n, 256), 256, 0, st>>>(s->lv.level_rows.p, s->lv.pos.p, n);
    // per-row arrays in the original numbering
    Scratch tmp;
    SP_TRY(tmp.alloc(n * sizeof(int32_t), st));
    for (int32_t* a : {s->lv.level.p, s->target.p}) {
        k_reverse_order<<<nblk(n, 256), 256, 0, st>>>(n, a, tmp.as<int32_t>());
        SP_CUDA(cudaMemcpyAsync(a, tmp.p, n * sizeof(int32_t), cudaMemcpyDeviceToDevice, st));
    }
    SP_CUDA(cudaGetLastError());
    SP_CUDA(cudaStreamSynchronize(st));
    return SPTRSV_OK;
}

}  // extern "C"
