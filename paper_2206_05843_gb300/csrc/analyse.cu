// analyse.cu -- CSR validation and level-set construction of DAG_L (Section II.A).
//
// Levels: level(i) = 0 for a row without dependencies, else 1 + max level of its
// dependencies.  The sweep is a persistent, ticketed kernel: each warp takes the next
// chunk of 32 consecutive rows, resolves dependencies outside the chunk by waiting
// (bounded) on their published levels, and dependencies inside the chunk through a
// 32-bit mask iterated in shared memory.  Tickets are handed out in row order, so every
// row a warp waits on belongs to a chunk that a running warp already owns.
#include <cstdarg>
#include <cstdio>

#include "internal.cuh"

namespace sp {
namespace {

// ---------------------------------------------------------------------------------
// validation
// ---------------------------------------------------------------------------------

template <typename T>
__global__ void k_validate(int64_t n, int64_t nnz, const int32_t* rowptr, const int32_t* colidx, const T* vals,
                           unsigned long long* first_bad) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int code = 0;
    int64_t a = rowptr[i], b = rowptr[i + 1];
    if (i == 0 && a != 0) code = 1;
    else if (b < a || b > nnz || a < 0) code = 1;
    else if (b == a) code = 2;
    else {
        int32_t prev = -1;
        for (int64_t k = a; k < b && !code; ++k) {
            int32_t c = colidx[k];
            if (c < 0 || c > i || c <= prev) code = 3;
            prev = c;
        }
        if (!code && colidx[b - 1] != i) code = 4;
        if (!code) {
            double d = (double)vals[b - 1];
            if (d == 0.0 || !isfinite(d)) code = 5;
        }
        for (int64_t k = a; k < b - 1 && !code; ++k)
            if (!isfinite((double)vals[k])) code = 6;
    }
    if (i == n - 1 && !code && b != nnz) code = 1;
    if (code) atomicMin(first_bad, ((unsigned long long)i << 4) | (unsigned long long)code);
}

// ---------------------------------------------------------------------------------
// level sweep
// ---------------------------------------------------------------------------------

constexpr int LV_THREADS = 256;
constexpr int LV_WARPS = LV_THREADS / 32;

__global__ void __launch_bounds__(LV_THREADS) k_levels(int64_t n, const int32_t* __restrict__ rowptr,
                                                       const int32_t* __restrict__ colidx, int diag_last,
                                                       int32_t* level, int* ticket, int* status, int* max_level,
                                                       int64_t timeout_ns) {
    __shared__ int32_t s_lev[LV_WARPS][32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t nchunks = (n + 31) / 32;
    int local_max = -1;
    while (true) {
        int c = 0;
        if (lane == 0) c = atomicAdd(ticket, 1);
        c = __shfl_sync(0xffffffffu, c, 0);
        if (c >= nchunks) break;
        const int64_t base = (int64_t)c * 32;
        const int64_t i = base + lane;
        const bool live = i < n;
        int ext = -1;
        unsigned inner = 0;
        bool failed = false;
        if (live) {
            int64_t a = rowptr[i], e = (int64_t)rowptr[i + 1] - diag_last;
            for (int64_t q = a; q < e; ++q) {
                int64_t j = colidx[q];
                if (j >= base) {
                    inner |= 1u << (unsigned)(j - base);
                } else {
                    int v = ld_acquire(level + j);
                    if (v < 0) {
                        uint64_t t0 = globaltimer();
                        unsigned spins = 0;
                        while ((v = ld_acquire(level + j)) < 0) {
                            if ((++spins & 63u) == 0) {
                                if (ld_volatile(status) != 0 || globaltimer() - t0 > (uint64_t)timeout_ns) {
                                    atomicCAS(status, 0, (int)DEV_TIMEOUT);
                                    failed = true;
                                    break;
                                }
                            }
                        }
                        if (failed) break;
                    }
                    ext = max(ext, v);
                }
            }
        }
        // resolve dependencies inside the chunk; each pass settles at least the lowest
        // unresolved row, so 32 passes bound the loop
        s_lev[warp][lane] = -1;
        __syncwarp();
        bool done = !live || failed;
        int mine = -1;
        for (int pass = 0; pass < 32; ++pass) {
            if (!done) {
                int mx = ext;
                bool ready = true;
                unsigned msk = inner;
                while (msk) {
                    int bpos = __ffs(msk) - 1;
                    msk &= msk - 1;
                    int v = s_lev[warp][bpos];
                    if (v < 0) { ready = false; break; }
                    mx = max(mx, v);
                }
                if (ready) {
                    mine = mx + 1;
                    s_lev[warp][lane] = mine;
                    done = true;
                }
            }
            __syncwarp();
            if (__all_sync(0xffffffffu, done)) break;
        }
        if (live && mine >= 0) {
            st_release(level + i, mine);
            local_max = max(local_max, mine);
        }
        if (__any_sync(0xffffffffu, failed)) break;
    }
    if (local_max >= 0) atomicMax(max_level, local_max);
}

__global__ void k_level_stats(int64_t n, const int32_t* rowptr, int diag_last, const int32_t* level,
                              int64_t* lrows, int64_t* lnnz, int64_t* lcost) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int64_t z = (int64_t)rowptr[i + 1] - rowptr[i] + (diag_last ? 0 : 1);  // entries incl. diagonal
    int l = level[i];
    atomicAdd((unsigned long long*)&lrows[l], 1ull);
    atomicAdd((unsigned long long*)&lnnz[l], (unsigned long long)z);
    atomicAdd((unsigned long long*)&lcost[l], (unsigned long long)(2 * z - 1));
}

__global__ void k_i64_to_i32(const int64_t* in, int32_t* out, int64_t n) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = (int32_t)in[i];
}

__global__ void k_iota(int32_t* out, int64_t n) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = (int32_t)i;
}

__global__ void k_inverse_perm(const int32_t* perm, int32_t* inv, int64_t n) {
    int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p < n) inv[perm[p]] = (int32_t)p;
}

inline unsigned blocks_for(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

}  // namespace

// ---------------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------------

static thread_local char g_err[1024] = "";

void set_error(const char* fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
}
const char* get_error() { return g_err; }

int device_sm_count() {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    return sms > 0 ? sms : 1;
}

int64_t default_timeout_ns() { return 2000000000ll; }

sptrsv_status map_dev_status(int code, const char* where) {
    switch (code) {
        case DEV_OK: return SPTRSV_OK;
        case DEV_TIMEOUT: set_error("%s: a bounded device wait ran out", where); return SPTRSV_ERR_TIMEOUT;
        case DEV_NUMERIC: set_error("%s: rewritten coefficient above the growth guard or not finite", where);
            return SPTRSV_ERR_NUMERIC;
        case DEV_OVERFLOW: set_error("%s: device scratch capacity exceeded", where); return SPTRSV_ERR_OOM;
        case DEV_LAUNCH: set_error("%s: the solve kernel ran without its thread-block clusters", where);
            return SPTRSV_ERR_CUDA;
        default: set_error("%s: invalid input detected on the device (code %d)", where, code);
            return SPTRSV_ERR_INVALID;
    }
}

sptrsv_status validate_csr(const sptrsv_csr* L, cudaStream_t st) {
    if (!L) { set_error("validate: null matrix"); return SPTRSV_ERR_INVALID; }
    if (L->n < 0 || L->nnz < L->n || L->n >= INT32_MAX || L->nnz >= INT32_MAX) {
        set_error("validate: bad sizes n=%lld nnz=%lld", (long long)L->n, (long long)L->nnz);
        return SPTRSV_ERR_INVALID;
    }
    if (L->dtype != SPTRSV_F64 && L->dtype != SPTRSV_F32) {
        set_error("validate: unknown dtype %d", L->dtype);
        return SPTRSV_ERR_INVALID;
    }
    if (L->n == 0) return SPTRSV_OK;
    if (!L->rowptr || !L->colidx || !L->vals) { set_error("validate: null array"); return SPTRSV_ERR_INVALID; }
    Scratch bad;
    SP_TRY(bad.alloc(sizeof(unsigned long long), st));
    SP_CUDA(cudaMemsetAsync(bad.p, 0xff, sizeof(unsigned long long), st));
    unsigned nb = blocks_for(L->n, 256);
    if (L->dtype == SPTRSV_F64)
        k_validate<double><<<nb, 256, 0, st>>>(L->n, L->nnz, L->rowptr, L->colidx, (const double*)L->vals,
                                               bad.as<unsigned long long>());
    else
        k_validate<float><<<nb, 256, 0, st>>>(L->n, L->nnz, L->rowptr, L->colidx, (const float*)L->vals,
                                              bad.as<unsigned long long>());
    SP_CUDA(cudaGetLastError());
    unsigned long long h = 0;
    SP_CUDA(cudaMemcpyAsync(&h, bad.p, sizeof(h), cudaMemcpyDeviceToHost, st));
    SP_CUDA(cudaStreamSynchronize(st));
    if (h != ~0ull) {
        static const char* what[] = {"", "bad row pointers", "empty row", "column out of range or not ascending",
                                     "diagonal missing or not last", "diagonal zero or not finite",
                                     "off-diagonal value not finite"};
        int code = (int)(h & 15);
        set_error("invalid CSR at row %lld: %s", (long long)(h >> 4), what[code < 7 ? code : 0]);
        return SPTRSV_ERR_INVALID;
    }
    return SPTRSV_OK;
}

sptrsv_status analyse_dep(const DepCsr& d, Levels& out, cudaStream_t st) {
    const int64_t n = d.n;
    out.n = n;
    SP_TRY(out.level.alloc(n > 0 ? n : 1));
    SP_TRY(out.level_rows.alloc(n > 0 ? n : 1));
    SP_TRY(out.pos.alloc(n > 0 ? n : 1));
    if (n == 0) {
        out.m = 0;
        SP_TRY(out.level_ptr.alloc(1));
        SP_CUDA(cudaMemsetAsync(out.level_ptr.p, 0, sizeof(int32_t), st));
        out.h_level_ptr.assign(1, 0);
        out.h_lcost.clear();
        out.nnz = 0; out.total_cost = 0; out.max_width = 0; out.avg = 0;
        SP_TRY(out.lrows.alloc(1)); SP_TRY(out.lnnz.alloc(1)); SP_TRY(out.lcost.alloc(1));
        return SPTRSV_OK;
    }
    Scratch ctl;  // ticket, status, max level
    SP_TRY(ctl.alloc(4 * sizeof(int), st));
    int* ticket = ctl.as<int>();
    int* status = ticket + 1;
    int* maxl = ticket + 2;
    SP_CUDA(cudaMemsetAsync(ctl.p, 0, 3 * sizeof(int), st));
    SP_CUDA(cudaMemsetAsync(maxl, 0xff, sizeof(int), st));
    SP_CUDA(cudaMemsetAsync(out.level.p, 0xff, (size_t)n * sizeof(int32_t), st));
    int occ = 0;
    SP_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_levels, LV_THREADS, 0));
    int64_t chunks = (n + 31) / 32;
    int64_t want = (chunks + LV_WARPS - 1) / LV_WARPS;
    int64_t grid = std::min<int64_t>((int64_t)device_sm_count() * std::max(occ, 1), want);
    k_levels<<<(unsigned)grid, LV_THREADS, 0, st>>>(n, d.rowptr, d.colidx, d.diag_last, out.level.p, ticket, status,
                                                   maxl, default_timeout_ns());
    SP_CUDA(cudaGetLastError());
    int h[3];
    SP_CUDA(cudaMemcpyAsync(h, ctl.p, 3 * sizeof(int), cudaMemcpyDeviceToHost, st));
    SP_CUDA(cudaStreamSynchronize(st));
    if (h[1] != 0) return map_dev_status(h[1], "analyse: level sweep");
    const int64_t m = (int64_t)h[2] + 1;
    out.m = m;
    SP_TRY(out.lrows.alloc(m));
    SP_TRY(out.lnnz.alloc(m));
    SP_TRY(out.lcost.alloc(m));
    SP_TRY(out.level_ptr.alloc(m + 1));
    SP_CUDA(cudaMemsetAsync(out.lrows.p, 0, m * sizeof(int64_t), st));
    SP_CUDA(cudaMemsetAsync(out.lnnz.p, 0, m * sizeof(int64_t), st));
    SP_CUDA(cudaMemsetAsync(out.lcost.p, 0, m * sizeof(int64_t), st));
    k_level_stats<<<blocks_for(n, 256), 256, 0, st>>>(n, d.rowptr, d.diag_last, out.level.p, out.lrows.p,
                                                       out.lnnz.p, out.lcost.p);
    SP_CUDA(cudaGetLastError());
    {
        Scratch lp64;
        SP_TRY(lp64.alloc((m + 1) * sizeof(int64_t), st));
        SP_TRY(scan_exclusive_i64(out.lrows.p, lp64.as<int64_t>(), m, st));
        k_i64_to_i32<<<blocks_for(m + 1, 256), 256, 0, st>>>(lp64.as<int64_t>(), out.level_ptr.p, m + 1);
        SP_CUDA(cudaGetLastError());
    }
    // rows ordered by level, ascending row index inside a level (stable sort)
    {
        Scratch idx, keys_out;
        SP_TRY(idx.alloc(n * sizeof(int32_t), st));
        SP_TRY(keys_out.alloc(n * sizeof(int32_t), st));
        k_iota<<<blocks_for(n, 256), 256, 0, st>>>(idx.as<int32_t>(), n);
        int bits = 1;
        while ((1ll << bits) < m) ++bits;
        SP_TRY(radix_sort_pairs(out.level.p, idx.as<int32_t>(), keys_out.as<int32_t>(), out.level_rows.p, n, bits, st));
        k_inverse_perm<<<blocks_for(n, 256), 256, 0, st>>>(out.level_rows.p, out.pos.p, n);
        SP_CUDA(cudaGetLastError());
    }
    out.h_level_ptr.resize(m + 1);
    out.h_lcost.resize(m);
    std::vector<int64_t> hrows(m), hnnz(m);
    SP_CUDA(cudaMemcpyAsync(out.h_level_ptr.data(), out.level_ptr.p, (m + 1) * sizeof(int32_t),
                            cudaMemcpyDeviceToHost, st));
    SP_CUDA(cudaMemcpyAsync(out.h_lcost.data(), out.lcost.p, m * sizeof(int64_t), cudaMemcpyDeviceToHost, st));
    SP_CUDA(cudaMemcpyAsync(hrows.data(), out.lrows.p, m * sizeof(int64_t), cudaMemcpyDeviceToHost, st));
    SP_CUDA(cudaMemcpyAsync(hnnz.data(), out.lnnz.p, m * sizeof(int64_t), cudaMemcpyDeviceToHost, st));
    SP_CUDA(cudaStreamSynchronize(st));
    int64_t tot = 0, nz = 0, mw = 0;
    for (int64_t l = 0; l < m; ++l) {
        tot += out.h_lcost[l];
        nz += hnnz[l];
        mw = std::max(mw, hrows[l]);
    }
    out.total_cost = tot;
    out.nnz = nz;
    out.max_width = mw;
    out.avg = m ? (double)tot / (double)m : 0.0;
    return SPTRSV_OK;
}

}  // namespace sp
