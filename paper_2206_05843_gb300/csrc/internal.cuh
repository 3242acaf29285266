// internal.cuh -- shared declarations of the sm_103a SpTRSV library (not part of the ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/sptrsv.h"

namespace sp {

// ---------------------------------------------------------------------------------
// error plumbing: every ABI entry point returns a status; the message is per thread
// ---------------------------------------------------------------------------------

void set_error(const char* fmt, ...);
const char* get_error();

#define SP_CUDA(call)                                                                   \
    do {                                                                                \
        cudaError_t e_ = (call);                                                        \
        if (e_ != cudaSuccess) {                                                        \
            ::sp::set_error("%s:%d %s: %s", __FILE__, __LINE__, #call, cudaGetErrorString(e_)); \
            return e_ == cudaErrorMemoryAllocation ? SPTRSV_ERR_OOM : SPTRSV_ERR_CUDA;  \
        }                                                                               \
    } while (0)

#define SP_TRY(expr)                              \
    do {                                          \
        sptrsv_status s_ = (expr);                \
        if (s_ != SPTRSV_OK) return s_;           \
    } while (0)

// device buffer owned by a handle; freed with cudaFree on destruction
template <typename T>
struct DevBuf {
    T* p = nullptr;
    size_t n = 0;
    DevBuf() = default;
    DevBuf(const DevBuf&) = delete;
    DevBuf& operator=(const DevBuf&) = delete;
    ~DevBuf() { release(); }
    void release() {
        if (p) cudaFree(p);
        p = nullptr;
        n = 0;
    }
    // allocates count elements plus 64 bytes of tail padding (bulk copies may round the
    // end of a range up to 16 bytes)
    sptrsv_status alloc(size_t count) {
        release();
        size_t bytes = count * sizeof(T) + 64;
        cudaError_t e = cudaMalloc((void**)&p, bytes);
        if (e != cudaSuccess) {
            p = nullptr;
            set_error("cudaMalloc(%zu bytes): %s", bytes, cudaGetErrorString(e));
            return e == cudaErrorMemoryAllocation ? SPTRSV_ERR_OOM : SPTRSV_ERR_CUDA;
        }
        n = count;
        return SPTRSV_OK;
    }
    sptrsv_status ensure(size_t count) { return count <= n && p ? SPTRSV_OK : alloc(count); }
    T* get() const { return p; }
};

// stream-ordered scratch (cudaMallocAsync) freed when the object goes out of scope
struct Scratch {
    void* p = nullptr;
    cudaStream_t st = nullptr;
    Scratch() = default;
    Scratch(const Scratch&) = delete;
    ~Scratch() {
        if (p) cudaFreeAsync(p, st);
    }
    sptrsv_status alloc(size_t bytes, cudaStream_t s) {
        if (p) cudaFreeAsync(p, st);
        p = nullptr;
        st = s;
        cudaError_t e = cudaMallocAsync(&p, bytes + 64, s);
        if (e != cudaSuccess) {
            p = nullptr;
            set_error("cudaMallocAsync(%zu bytes): %s", bytes, cudaGetErrorString(e));
            return e == cudaErrorMemoryAllocation ? SPTRSV_ERR_OOM : SPTRSV_ERR_CUDA;
        }
        return SPTRSV_OK;
    }
    template <typename T>
    T* as() const { return (T*)p; }
};

int device_sm_count();
int64_t default_timeout_ns();

// ---------------------------------------------------------------------------------
// device helpers
// ---------------------------------------------------------------------------------

#ifdef __CUDACC__
__device__ __forceinline__ int ld_acquire(const int* p) {
    int v;
    asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_release(int* p, int v) {
    asm volatile("st.release.gpu.global.b32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ int ld_volatile(const int* p) {
    int v;
    asm volatile("ld.volatile.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
// Cluster barrier, split: arrive (release: this thread's earlier writes become visible to the
// cluster) and wait (acquire).  Every thread of every CTA of the cluster must take both, in order.
__device__ __forceinline__ void cluster_arrive() { asm volatile("barrier.cluster.arrive.release;" ::: "memory"); }
__device__ __forceinline__ void cluster_wait() { asm volatile("barrier.cluster.wait.acquire;" ::: "memory"); }
__device__ __forceinline__ uint64_t globaltimer() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
// mbarrier and bulk-copy helpers (shared::cta addresses)
__device__ __forceinline__ uint32_t smem_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void mbar_init(uint64_t* m, int count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(m)), "r"(count) : "memory");
}
// makes initialised mbarriers visible to the bulk-copy unit
__device__ __forceinline__ void mbar_fence_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }
// one arrival that also expects `bytes` of bulk-copy transactions in the current phase
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* m, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(m)), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* m, uint32_t parity) {
    uint32_t done;
    asm volatile(
        "{ .reg .pred p; mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2; selp.u32 %0, 1, 0, p; }"
        : "=r"(done)
        : "r"(smem_addr(m)), "r"(parity)
        : "memory");
    return done != 0;
}
// global -> shared bulk copy (16-byte aligned addresses, size a multiple of 16) that completes
// its bytes on the mbarrier
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* m) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_addr(dst)),
                 "l"(src), "r"(bytes), "r"(smem_addr(m))
                 : "memory");
}

// Asks the TMA unit to bring [p, p + bytes) into L2 without waiting for it: the threads of
// the CTA issue one bulk prefetch per 4 KB piece.  Only the 16-byte aligned interior of the
// range is prefetched (the bulk copy's alignment rule), so nothing outside it is touched.
__device__ __forceinline__ void l2_prefetch(const void* p, int64_t bytes) {
    if (bytes <= 0) return;
    constexpr uint64_t PIECE = 4096;
    const uint64_t a = ((uint64_t)p + 15) & ~(uint64_t)15;
    const uint64_t e = ((uint64_t)p + (uint64_t)bytes) & ~(uint64_t)15;
    for (uint64_t q = a + (uint64_t)threadIdx.x * PIECE; q < e; q += (uint64_t)blockDim.x * PIECE) {
        const uint32_t n = (uint32_t)(e - q < PIECE ? e - q : PIECE);
        asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(q), "r"(n) : "memory");
    }
}
// waits for the mbarrier phase of the given parity; false when timeout_ns passes first
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* m, uint32_t parity, int64_t timeout_ns) {
    if (mbar_try_wait(m, parity)) return true;
    const uint64_t t0 = globaltimer();
    while (!mbar_try_wait(m, parity))
        if (globaltimer() - t0 > (uint64_t)timeout_ns) return false;
    return true;
}
#endif

// status words written by kernels (device int, 0 = ok)
// DEV_LAUNCH: a kernel found itself launched without the thread-block cluster shape it was built for
enum DevStatus : int { DEV_OK = 0, DEV_TIMEOUT = 1, DEV_NUMERIC = 2, DEV_OVERFLOW = 3, DEV_INVALID = 4, DEV_LAUNCH = 5 };

sptrsv_status map_dev_status(int code, const char* where);

// ---------------------------------------------------------------------------------
// primitives (prims.cu)
// ---------------------------------------------------------------------------------

// exclusive scan of n values into out[0..n]; out[n] = total.  in and out may alias.
sptrsv_status scan_exclusive_i64(const int64_t* in, int64_t* out, int64_t n, cudaStream_t st);
sptrsv_status scan_exclusive_i32(const int32_t* in, int32_t* out, int64_t n, cudaStream_t st);
// scan of int32 counts into int64 offsets
sptrsv_status scan_exclusive_i32_to_i64(const int32_t* in, int64_t* out, int64_t n, cudaStream_t st);

// stable sort of (key, value) pairs by key (keys in [0, 2^bits)); results in keys_out/vals_out
sptrsv_status radix_sort_pairs(const int32_t* keys_in, const int32_t* vals_in, int32_t* keys_out,
                               int32_t* vals_out, int64_t n, int bits, cudaStream_t st);

// ---------------------------------------------------------------------------------
// analysis (analyse.cu)
// ---------------------------------------------------------------------------------

// a dependency structure: row i depends on colidx[rowptr[i] .. rowptr[i+1] - diag_last)
struct DepCsr {
    int64_t n = 0;
    const int32_t* rowptr = nullptr;
    const int32_t* colidx = nullptr;
    int diag_last = 1;
};

struct Levels {
    int64_t n = 0, m = 0, nnz = 0, total_cost = 0, max_width = 0;
    double avg = 0.0;
    DevBuf<int32_t> level, level_ptr, level_rows, pos;
    DevBuf<int64_t> lrows, lnnz, lcost;
    std::vector<int32_t> h_level_ptr;
    std::vector<int64_t> h_lcost;
};

sptrsv_status validate_csr(const sptrsv_csr* L, cudaStream_t st);
sptrsv_status analyse_dep(const DepCsr& d, Levels& out, cudaStream_t st);

}  // namespace sp

// opaque handle types of the ABI
struct sptrsv_levels {
    sp::Levels lv;
};
