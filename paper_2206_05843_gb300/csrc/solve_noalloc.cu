// solve_noalloc.cu -- sptrsv_solve_noalloc: the persistent solve without any allocation.
//
// Some callers cannot call cudaMalloc at the moment they solve: real-time loops that must
// never enter the allocator (its latency is unbounded and it may synchronize the device),
// processes whose device memory a framework's caching allocator has already reserved in
// full, and plug-in code that is handed its inputs and outputs but no allocator.  The
// regular sptrsv_solve may allocate its scratch (the solution in stored order and the
// per-CTA completion flags) on first use; this entry point instead keeps that scratch in
// one file-scope device array of fixed size and calls no allocating routine at all.
//
// The array is shared by every call on a device and keeps the last call's contents:
// the completion flags are reset to "nothing published" (-1) at the start of each call,
// the solution scratch needs no reset because every entry is written before it is read.
// Calls that overlap on the GPU (on different streams, or from different threads) use
// the same array and race; order them on one stream.
#include <mutex>

#include "solve_kernel.cuh"

namespace sp {
namespace {

// 64 MiB: completion flags in the first 64 KiB (16,384 CTAs), the solution scratch after
// them.  Every GPU that loads the library holds this array until the process exits.
constexpr size_t NOALLOC_BYTES = (size_t)64 << 20;
constexpr size_t NOALLOC_FLAG_BYTES = (size_t)64 << 10;

static __device__ __align__(256) unsigned char g_noalloc_scratch[NOALLOC_BYTES];

constexpr int MAX_DEVICES = 128;
std::mutex g_setup_mu;
unsigned char* g_scratch_addr[MAX_DEVICES] = {};

// once per device, with that device current: the device address of the array (in host
// code the array's name is only a host-side stand-in) and the kernel attributes
sptrsv_status setup_device(unsigned char** out) {
    int dev = 0;
    SP_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= MAX_DEVICES) {
        set_error("solve_noalloc: device ordinal %d out of range", dev);
        return SPTRSV_ERR_UNSUPPORTED;
    }
    std::lock_guard<std::mutex> lk(g_setup_mu);
    if (!g_scratch_addr[dev]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) {
            set_error("solve_noalloc: cudaGetSymbolAddress failed: %s", cudaGetErrorString(e));
            return SPTRSV_ERR_CUDA;
        }
        g_scratch_addr[dev] = (unsigned char*)p;
    }
    *out = g_scratch_addr[dev];
    return SPTRSV_OK;
}

template <typename T>
sptrsv_status launch_noalloc(const sptrsv_system* s, const void* b, void* x, int nrhs, int64_t ld,
                             unsigned char* scratch, cudaStream_t st) {
    const Schedule& sc = s->sched;
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
    a.xp = (T*)(scratch + NOALLOC_FLAG_BYTES);
    a.flags = (int*)scratch;
    a.status = s->status.p;  // the system's status word, read by sptrsv_solve_status
    a.stamps = nullptr;
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
    SP_CUDA(cudaMemsetAsync(a.status, 0, sizeof(int), st));
    if (sc.run_width == -2) {
        // the system is tuned to one launch per level: the same launches as sptrsv_solve, with
        // the solution scratch in the static array (they use no completion flags)
        const std::vector<int32_t>& lp = s->lv.h_level_ptr;
        for (int64_t l = 0; l < s->m; ++l) {
            const int64_t rows = (int64_t)(lp[l + 1] - lp[l]) * nrhs;
            k_level<T><<<(unsigned)((rows + 255) / 256), 256, 0, st>>>(a, lp[l], lp[l + 1]);
        }
        SP_CUDA(cudaGetLastError());
        return SPTRSV_OK;
    }
    SP_CUDA(k_solve_attrs<T>(sc.smem, sc.csize, sc.tile_ecap, sc.runs));
    SP_CUDA(cudaMemsetAsync(a.flags, 0xff, (size_t)sc.grid * sizeof(int), st));
    if (a.nseg == 0) return SPTRSV_OK;
    if (sc.pre) k_bparts<T><<<sc.pre_grid, 256, 0, st>>>(a, (int)sc.h_blocks.size());
    SP_CUDA(launch_k_solve<T>(a, sc.grid, sc.block, sc.smem, sc.csize, st, sc.runs));
    return SPTRSV_OK;
}

}  // namespace
}  // namespace sp

using namespace sp;

extern "C" sptrsv_status sptrsv_solve_noalloc(const sptrsv_system* s, const void* b_dev, void* x_dev, int32_t nrhs,
                                              int64_t ld, sptrsv_stream_t stream) {
    if (!s) { set_error("solve_noalloc: null system"); return SPTRSV_ERR_INVALID; }
    if (nrhs < 1 || ld < s->n || (s->n > 0 && (!b_dev || !x_dev))) {
        set_error("solve_noalloc: bad arguments (nrhs=%d ld=%lld n=%lld)", nrhs, (long long)ld, (long long)s->n);
        return SPTRSV_ERR_INVALID;
    }
    if (s->n == 0) return SPTRSV_OK;
    const Schedule& sc = s->sched;
    if (sc.nrhs != nrhs || !sc.segs.p || !s->status.p) {
        set_error("solve_noalloc: the system has no solve schedule for nrhs=%d; run sptrsv_solve once with this "
                  "nrhs first (it builds the schedule, which allocates)", nrhs);
        return SPTRSV_ERR_INVALID;
    }
    const size_t vb = s->dtype == SPTRSV_F64 ? 8 : 4;
    const size_t need = (size_t)s->n * (size_t)nrhs * vb;
    if (need > NOALLOC_BYTES - NOALLOC_FLAG_BYTES || (size_t)sc.grid * sizeof(int) > NOALLOC_FLAG_BYTES) {
        set_error("solve_noalloc: needs %zu bytes of scratch (n=%lld x nrhs=%d x %zu bytes); the static area holds "
                  "%zu bytes", need, (long long)s->n, nrhs, vb, NOALLOC_BYTES - NOALLOC_FLAG_BYTES);
        return SPTRSV_ERR_UNSUPPORTED;
    }
    unsigned char* scratch = nullptr;
    SP_TRY(setup_device(&scratch));
    cudaStream_t st = (cudaStream_t)stream;
    if (s->dtype == SPTRSV_F64) return launch_noalloc<double>(s, b_dev, x_dev, nrhs, ld, scratch, st);
    return launch_noalloc<float>(s, b_dev, x_dev, nrhs, ld, scratch, st);
}
