// batch.cu -- many systems of uneven size, each with its own right-hand sides, solved in
// one persistent launch captured in a CUDA graph.
//
// Every CTA takes whole work items from a ticket in longest-first order and runs all of an
// item's levels with the single-CTA executor (run_exec.cuh): levels are separated by CTA
// barriers, never by device-wide handoffs, so items proceed independently.  An item is a
// system with all of its right-hand sides or, when their work outweighs both the system's
// critical path and an even share of the batch per SM, with a contiguous part of them (at most
// 8 parts): the parts of one system run on different CTAs at the same time.  float64 and
// float32 systems share the launch.  The block size and the lanes-per-row policy are chosen by
// timing candidate launches; the choice is cached by the batch signature.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <mutex>

#include "run_exec.cuh"

namespace sp {
namespace {

struct BatchItem {
    int64_t n;
    int32_t nrhs, dtype, lpr, blk0, blk1;
    int32_t ring_rows, stage_rows, stage_entries;
    int32_t sys;      // the system (index of its b and x pointers)
    int64_t rhs_off;  // its first right-hand side times n: element offset into the system's b and x
    const int32_t* perm;
    const int32_t* lptr;
    const int32_t* cptr;
    const int32_t* ccol;
    const int32_t* eptr;
    const int32_t* ecol;
    const void* cval;
    const void* dinv;
    const void* eval;
    void* xp;
};

template <typename T>
__device__ void run_item(const BatchItem& it, const int4* blocks, const void* b, void* x, unsigned char* smem) {
    SysView<T> v{it.nrhs,
                 it.n,
                 it.perm,
                 it.lptr,
                 it.cptr,
                 it.ccol,
                 (const T*)it.cval,
                 (const T*)it.dinv,
                 it.eptr,
                 it.ecol,
                 (const T*)it.eval,
                 (const T*)b,
                 (T*)x,
                 (T*)it.xp,
                 nullptr};
    const Lanes ln = make_lanes(it.lpr, it.nrhs);
    run_blocks(v, smem, RunGeom{it.ring_rows, it.stage_rows, it.stage_entries}, ln, blocks, it.blk0, it.blk1,
               []() { return true; }, nullptr);
}

__global__ void __launch_bounds__(512) k_batch(const BatchItem* items, const int4* blocks, const int32_t* order,
                                               const void* const* bptr, void* const* xptr, int nitems, int* ticket) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ int s_t;
    while (true) {
        __syncthreads();
        if (threadIdx.x == 0) s_t = atomicAdd(ticket, 1);
        __syncthreads();
        const int t = s_t;
        if (t >= nitems) break;
        const BatchItem it = items[order[t]];
        const int64_t off = it.rhs_off * (it.dtype == SPTRSV_F64 ? 8 : 4);
        const void* b = (const unsigned char*)bptr[it.sys] + off;
        void* x = (unsigned char*)xptr[it.sys] + off;
        if (it.dtype == SPTRSV_F64) run_item<double>(it, blocks, b, x, smem);
        else run_item<float>(it, blocks, b, x, smem);
    }
}

struct Tuned {
    int block, lpr_mode;
    double us;
    int policy = 0;  // split policy of the work items
};
std::mutex g_tune_mu;
std::map<std::vector<int64_t>, Tuned> g_tune_cache;

int lanes_for(int nrhs, double avg_row, int mode) {
    int lpr;
    // mode 3: lanes per row split only the coefficients; thin levels of several right-hand
    // sides then run in the fast executor (one lane per row and right-hand side)
    if (mode == 3) return avg_row > 12.0 ? 4 : 1;
    if (nrhs >= 2) {
        lpr = 1;
        while (lpr < nrhs && lpr < 32) lpr <<= 1;
    } else {
        lpr = avg_row > 12.0 ? 4 : 1;
    }
    if (mode == 1) lpr = std::max(1, lpr / 2);
    if (mode == 2) lpr = std::min(32, lpr * 2);
    return lpr;
}

RunGeom geom_for(int nrhs, int vb) { return run_geometry(nrhs, vb); }

}  // namespace
}  // namespace sp

using namespace sp;

struct sptrsv_batch {
    int count = 0;   // systems
    int nitems = 0;  // work items (systems or parts of their right-hand sides)
    int policy = 0;  // the split policy the items were made with
    std::vector<const sptrsv_system*> sys;
    std::vector<int32_t> nrhs;
    std::vector<std::vector<int32_t>> hcptr;
    std::vector<BatchItem> items;  // work items
    std::vector<int32_t> order;
    DevBuf<BatchItem> d_items;
    DevBuf<int4> d_blocks;
    DevBuf<int32_t> d_order;
    DevBuf<void*> d_io;  // b pointers then x pointers
    DevBuf<int> d_ticket;
    DevBuf<unsigned char> xp;
    void** h_io = nullptr;  // pinned staging of the pointer table
    size_t smem = 0;
    int block = 256, lpr_mode = 0, grid = 0;
    double tuned_us = 0;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    cudaStream_t cap_stream = nullptr;
    ~sptrsv_batch() {
        if (exec) cudaGraphExecDestroy(exec);
        if (graph) cudaGraphDestroy(graph);
        if (cap_stream) cudaStreamDestroy(cap_stream);
        if (h_io) cudaFreeHost(h_io);
    }
};

namespace sp {
namespace {

// items and blocks for one (block size, lanes mode) choice
sptrsv_status layout_batch(sptrsv_batch* bt, int lpr_mode) {
    std::vector<int4> blocks;
    size_t smem = 0;
    for (int i = 0; i < bt->nitems; ++i) {
        BatchItem& it = bt->items[i];
        const sptrsv_system* s = bt->sys[it.sys];
        const int vb = s->dtype == SPTRSV_F64 ? 8 : 4;
        const int nr = it.nrhs;
        RunGeom g = geom_for(nr, vb);
        const double avg_row = s->n ? (double)s->nnz_c / (double)s->n : 0.0;
        it.lpr = lanes_for(nr, avg_row, lpr_mode);
        it.ring_rows = g.ring_rows;
        it.stage_rows = g.stage_rows;
        it.stage_entries = g.stage_entries;
        it.blk0 = (int)blocks.size();
        if (s->m > 0 &&
            build_run_blocks(s->lv.h_level_ptr.data(), bt->hcptr[it.sys].data(), 0, s->m, g.stage_rows,
                             g.stage_entries, it.lpr, nr, fast_rec_capacity(vb, g), blocks) != 0) {
            set_error("batch: system %d has a row with more coefficients than the staging area", it.sys);
            return SPTRSV_ERR_UNSUPPORTED;
        }
        it.blk1 = (int)blocks.size();
        smem = std::max(smem, run_smem_bytes(vb, nr, g));
    }
    if (blocks.empty()) blocks.push_back(make_int4(0, 0, 0, 0));
    SP_TRY(bt->d_blocks.alloc(blocks.size()));
    SP_CUDA(cudaMemcpy(bt->d_blocks.p, blocks.data(), blocks.size() * sizeof(int4), cudaMemcpyHostToDevice));
    SP_CUDA(cudaMemcpy(bt->d_items.p, bt->items.data(), bt->nitems * sizeof(BatchItem), cudaMemcpyHostToDevice));
    bt->smem = smem;
    return SPTRSV_OK;
}

sptrsv_status launch_batch(sptrsv_batch* bt, int block, cudaStream_t st) {
    SP_CUDA(cudaFuncSetAttribute(k_batch, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bt->smem));
    int occ = 0;
    SP_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_batch, block, bt->smem));
    if (occ < 1) {
        set_error("batch kernel does not fit an SM (block %d, %zu bytes shared)", block, bt->smem);
        return SPTRSV_ERR_UNSUPPORTED;
    }
    int grid = std::min<int64_t>((int64_t)device_sm_count() * occ, bt->nitems);
    bt->grid = std::max(1, grid);
    SP_CUDA(cudaMemsetAsync(bt->d_ticket.p, 0, sizeof(int), st));
    k_batch<<<bt->grid, block, bt->smem, st>>>(bt->d_items.p, bt->d_blocks.p, bt->d_order.p,
                                               (const void* const*)bt->d_io.p, (void* const*)(bt->d_io.p + bt->count),
                                               bt->nitems, bt->d_ticket.p);
    SP_CUDA(cudaGetLastError());
    return SPTRSV_OK;
}

}  // namespace
}  // namespace sp

extern "C" {

sptrsv_status sptrsv_batch_create(const sptrsv_system* const* systems, const int32_t* nrhs, int32_t count,
                                  sptrsv_batch** out, sptrsv_stream_t stream) {
    if (!systems || !nrhs || !out || count < 1) { set_error("batch_create: bad arguments"); return SPTRSV_ERR_INVALID; }
    *out = nullptr;
    cudaStream_t st = (cudaStream_t)stream;
    SP_CUDA(cudaStreamSynchronize(st));
    sptrsv_batch* bt = new (std::nothrow) sptrsv_batch();
    if (!bt) { set_error("host allocation failed"); return SPTRSV_ERR_OOM; }
    auto fail = [&](sptrsv_status rc) {
        delete bt;
        return rc;
    };
    bt->count = count;
    bt->sys.assign(systems, systems + count);
    bt->nrhs.assign(nrhs, nrhs + count);
    bt->hcptr.resize(count);
    // b and x of every system (autotuning scratch), the critical path and the work of each
    std::vector<int64_t> boff(count + 1, 0);
    std::vector<double> crit(count), work(count);
    std::vector<int64_t> sig;
    for (int i = 0; i < count; ++i) {
        const sptrsv_system* s = systems[i];
        if (!s || nrhs[i] < 1 || nrhs[i] > 1024) return fail((set_error("batch_create: bad system or nrhs at %d", i), SPTRSV_ERR_INVALID));
        const int vb = s->dtype == SPTRSV_F64 ? 8 : 4;
        boff[i + 1] = boff[i] + ((int64_t)s->n * nrhs[i] * vb + 255) / 256 * 256;
        // critical path (about 250 ns a level) and float64 work on one SM (about two FMAs a
        // cycle, 0.25 ns each), in rough nanoseconds
        crit[i] = 250.0 * (double)s->m;
        work[i] = 0.25 * (double)(s->nnz_c + s->n + s->nnz_e) * nrhs[i];
        sig.push_back(s->n);
        sig.push_back(s->m);
        sig.push_back(s->nnz_c + s->nnz_e);
        sig.push_back(nrhs[i] * 2 + s->dtype);
        bt->hcptr[i].resize(s->n + 1);
        if (s->n > 0)
            if (cudaMemcpy(bt->hcptr[i].data(), s->cptr.p, (s->n + 1) * sizeof(int32_t), cudaMemcpyDeviceToHost) !=
                cudaSuccess)
                return fail((set_error("batch_create: copy failed"), SPTRSV_ERR_CUDA));
    }
    // work items: a system's right-hand sides split into at most 8 contiguous parts, so that the
    // parts of a heavy system run on several CTAs instead of one item queueing the batch.  Split
    // policy 0: when the system's float64 work exceeds both its critical path and an even share
    // of the batch per SM; 1 and 2: parts of at most 8 or 4 right-hand sides for every system
    // whose estimate exceeds 1.3 x the longest critical path of the batch (a thin level costs
    // more with more right-hand sides: about 10% per extra one).  The autotuner times the three.
    double total = 0, crit_max = 0;
    int64_t xcap = 0;
    for (int i = 0; i < count; ++i) {
        total += crit[i] + work[i];
        crit_max = std::max(crit_max, crit[i]);
        xcap += (int64_t)systems[i]->n * nrhs[i] * (systems[i]->dtype == SPTRSV_F64 ? 8 : 4);
    }
    xcap += (int64_t)256 * 8 * count;
    const double share = total / (double)device_sm_count();
    sptrsv_status rc;
    if ((rc = bt->xp.alloc(std::max<int64_t>(256, xcap))) != SPTRSV_OK) return fail(rc);
    if ((rc = bt->d_items.alloc((size_t)8 * count)) != SPTRSV_OK) return fail(rc);
    if ((rc = bt->d_order.alloc((size_t)8 * count)) != SPTRSV_OK) return fail(rc);
    auto make_items = [&](int policy) -> sptrsv_status {
        bt->items.clear();
        std::vector<double> cost;
        int64_t xoff = 0;
        for (int i = 0; i < count; ++i) {
            const sptrsv_system* s = systems[i];
            const int vb = s->dtype == SPTRSV_F64 ? 8 : 4;
            auto estimate = [&](int r) { return crit[i] * (1.0 + 0.1 * (r - 1)) + work[i] * r / nrhs[i]; };
            int parts = 1;
            if (nrhs[i] >= 2) {
                if (policy == 0) {
                    const double bar = std::max(crit[i], share);
                    if (work[i] > bar) parts = (int)std::min<double>({(double)nrhs[i], 8.0, std::ceil(work[i] / bar)});
                } else if (estimate(nrhs[i]) > 1.3 * crit_max) {
                    const int cap = policy == 1 ? 8 : 4;
                    parts = std::min(8, (nrhs[i] + cap - 1) / cap);
                }
            }
            const int per = (nrhs[i] + parts - 1) / parts;
            for (int k0 = 0; k0 < nrhs[i]; k0 += per) {
                BatchItem it{};
                it.sys = i;
                it.nrhs = std::min(per, nrhs[i] - k0);
                it.rhs_off = (int64_t)k0 * s->n;
                it.n = s->n;
                it.dtype = s->dtype;
                it.perm = s->lv.level_rows.p;
                it.lptr = s->lv.level_ptr.p;
                it.cptr = s->cptr.p;
                it.ccol = s->ccol.p;
                it.eptr = s->nnz_e > 0 ? s->eptr.p : nullptr;
                it.ecol = s->ecol.p;
                it.cval = s->cval.p;
                it.dinv = s->dinv.p;
                it.eval = s->eval.p;
                it.xp = bt->xp.p + xoff;
                xoff += ((int64_t)s->n * it.nrhs * vb + 255) / 256 * 256;
                bt->items.push_back(it);
                cost.push_back(estimate(it.nrhs));
            }
        }
        bt->nitems = (int)bt->items.size();
        bt->order.resize(bt->nitems);
        for (int i = 0; i < bt->nitems; ++i) bt->order[i] = i;
        std::stable_sort(bt->order.begin(), bt->order.end(), [&](int a, int b) { return cost[a] > cost[b]; });
        SP_CUDA(cudaMemcpy(bt->d_order.p, bt->order.data(), bt->nitems * sizeof(int32_t), cudaMemcpyHostToDevice));
        bt->policy = policy;
        return SPTRSV_OK;
    };
    if ((rc = bt->d_io.alloc(2 * count)) != SPTRSV_OK) return fail(rc);
    if ((rc = bt->d_ticket.alloc(1)) != SPTRSV_OK) return fail(rc);
    if (cudaMallocHost((void**)&bt->h_io, 2 * count * sizeof(void*)) != cudaSuccess)
        return fail((set_error("batch_create: pinned allocation failed"), SPTRSV_ERR_OOM));

    // autotune on zero right-hand sides (the time does not depend on the values)
    {
        DevBuf<unsigned char> tb, tx;
        if ((rc = tb.alloc(std::max<int64_t>(256, boff[count]))) != SPTRSV_OK) return fail(rc);
        if ((rc = tx.alloc(std::max<int64_t>(256, boff[count]))) != SPTRSV_OK) return fail(rc);
        cudaMemset(tb.p, 0, std::max<int64_t>(256, boff[count]));
        std::vector<void*> io(2 * count);
        for (int i = 0; i < count; ++i) {
            io[i] = tb.p + boff[i];
            io[count + i] = tx.p + boff[i];
        }
        if (cudaMemcpy(bt->d_io.p, io.data(), 2 * count * sizeof(void*), cudaMemcpyHostToDevice) != cudaSuccess)
            return fail((set_error("batch_create: copy failed"), SPTRSV_ERR_CUDA));
        Tuned best{256, 0, 1e30};
        bool cached = false;
        {
            std::lock_guard<std::mutex> lk(g_tune_mu);
            auto f = g_tune_cache.find(sig);
            if (f != g_tune_cache.end()) {
                best = f->second;
                cached = true;
            }
        }
        if (!cached) {
            cudaEvent_t e0, e1;
            cudaEventCreate(&e0);
            cudaEventCreate(&e1);
            std::vector<std::vector<int64_t>> seen;  // item sets already timed
            for (int policy = 0; policy < 3; ++policy) {
                if ((rc = make_items(policy)) != SPTRSV_OK) return fail(rc);
                std::vector<int64_t> key;
                for (const BatchItem& it : bt->items) key.push_back((int64_t)it.sys * 2048 + it.nrhs);
                if (std::find(seen.begin(), seen.end(), key) != seen.end()) continue;
                seen.push_back(key);
                for (int mode = 0; mode < 4; ++mode) {
                    if ((rc = layout_batch(bt, mode)) != SPTRSV_OK) return fail(rc);
                    for (int block : {128, 256, 512}) {
                        float best_ms = 1e30f;
                        for (int rep = 0; rep < 3; ++rep) {
                            cudaEventRecord(e0, st);
                            if ((rc = launch_batch(bt, block, st)) != SPTRSV_OK) return fail(rc);
                            cudaEventRecord(e1, st);
                            cudaEventSynchronize(e1);
                            float ms = 0;
                            cudaEventElapsedTime(&ms, e0, e1);
                            if (rep > 0) best_ms = std::min(best_ms, ms);
                        }
                        if (best_ms * 1e3 < best.us) best = Tuned{block, mode, best_ms * 1e3, policy};
                    }
                }
            }
            cudaEventDestroy(e0);
            cudaEventDestroy(e1);
            std::lock_guard<std::mutex> lk(g_tune_mu);
            g_tune_cache[sig] = best;
        }
        bt->block = best.block;
        bt->lpr_mode = best.lpr_mode;
        bt->tuned_us = best.us;
        if ((rc = make_items(best.policy)) != SPTRSV_OK) return fail(rc);
        if ((rc = layout_batch(bt, best.lpr_mode)) != SPTRSV_OK) return fail(rc);
        if (cudaStreamSynchronize(st) != cudaSuccess) return fail((set_error("batch_create: sync failed"), SPTRSV_ERR_CUDA));
    }
    // capture the solve (ticket reset + persistent kernel) in a graph
    if (cudaStreamCreateWithFlags(&bt->cap_stream, cudaStreamNonBlocking) != cudaSuccess)
        return fail((set_error("batch_create: stream creation failed"), SPTRSV_ERR_CUDA));
    if (cudaStreamBeginCapture(bt->cap_stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess)
        return fail((set_error("batch_create: capture failed"), SPTRSV_ERR_CUDA));
    rc = launch_batch(bt, bt->block, bt->cap_stream);
    cudaError_t ce = cudaStreamEndCapture(bt->cap_stream, &bt->graph);
    if (rc != SPTRSV_OK) return fail(rc);
    if (ce != cudaSuccess) return fail((set_error("batch_create: end capture: %s", cudaGetErrorString(ce)), SPTRSV_ERR_CUDA));
    ce = cudaGraphInstantiate(&bt->exec, bt->graph, 0);
    if (ce != cudaSuccess) return fail((set_error("batch_create: instantiate: %s", cudaGetErrorString(ce)), SPTRSV_ERR_CUDA));
    *out = bt;
    return SPTRSV_OK;
}

sptrsv_status sptrsv_batch_solve(sptrsv_batch* bt, const void* const* b, void* const* x, sptrsv_stream_t stream) {
    if (!bt || !b || !x) { set_error("batch_solve: null argument"); return SPTRSV_ERR_INVALID; }
    cudaStream_t st = (cudaStream_t)stream;
    // the pointer table is staged in pinned memory; wait for the previous copy to finish
    // reading it before overwriting
    SP_CUDA(cudaStreamSynchronize(st));
    for (int i = 0; i < bt->count; ++i) {
        bt->h_io[i] = const_cast<void*>(b[i]);
        bt->h_io[bt->count + i] = x[i];
    }
    SP_CUDA(cudaMemcpyAsync(bt->d_io.p, bt->h_io, 2 * bt->count * sizeof(void*), cudaMemcpyHostToDevice, st));
    SP_CUDA(cudaGraphLaunch(bt->exec, st));
    return SPTRSV_OK;
}

sptrsv_status sptrsv_batch_info_get(const sptrsv_batch* bt, sptrsv_batch_info* o) {
    if (!bt || !o) { set_error("batch_info: null argument"); return SPTRSV_ERR_INVALID; }
    o->count = bt->count;
    o->items = bt->nitems;
    o->split_policy = bt->policy;
    o->block = bt->block;
    o->lanes_per_row = bt->lpr_mode;
    o->graph = bt->exec != nullptr;
    o->tuned_us = bt->tuned_us;
    return SPTRSV_OK;
}

void sptrsv_batch_destroy(sptrsv_batch* bt) { delete bt; }

}  // extern "C"
