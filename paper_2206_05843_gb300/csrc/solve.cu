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

#include "system.cuh"

namespace sp {
namespace {

struct Lanes {
    int lpr, RL, EL, rl, el, chunks;
};

__device__ __forceinline__ Lanes make_lanes(int lpr, int nrhs) {
    Lanes l;
    l.lpr = lpr;
    int p2 = 1;
    while (p2 < nrhs && p2 < lpr) p2 <<= 1;
    l.RL = p2;
    l.EL = lpr / p2;
    int lg = threadIdx.x & (lpr - 1);
    l.rl = lg % l.RL;
    l.el = lg / l.RL;
    l.chunks = (nrhs + l.RL - 1) / l.RL;
    return l;
}

template <typename T>
__device__ __forceinline__ T group_reduce(T v, const Lanes& ln) {
    for (int o = ln.RL; o < ln.lpr; o <<= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// b-part of row p for right-hand side k, partial over this lane's share of the E row
template <typename T>
__device__ __forceinline__ T bpart(const SolveArgs<T>& a, int64_t p, int32_t row, int k, const Lanes& ln) {
    T acc = T(0);
    if (ln.el == 0) acc = a.dinv[p] * a.b[(int64_t)row + (int64_t)k * a.ld];
    if (a.eptr) {
        int e1 = a.eptr[p + 1];
        for (int q = a.eptr[p] + ln.el; q < e1; q += ln.EL)
            acc += a.eval[q] * a.b[(int64_t)a.ecol[q] + (int64_t)k * a.ld];
    }
    return acc;
}

// ---------------------------------------------------------------------------------
// bounded waits and publication
// ---------------------------------------------------------------------------------

template <typename T>
__device__ bool wait_segment(const SolveArgs<T>& a, int s) {
    if (s < 0) return true;
    int4 sg = a.segs[s];
    int parts = sg.x == SEG_WIDE ? sg.w : 1;
    bool failed = false;
    for (int t = threadIdx.x; t < parts && !failed; t += blockDim.x) {
        const int* f = a.flags + t;
        if (ld_acquire(f) >= s) continue;
        uint64_t t0 = globaltimer();
        unsigned spins = 0;
        while (ld_acquire(f) < s) {
            if ((++spins & 31u) == 0) {
                if (ld_volatile(a.status) != 0 || globaltimer() - t0 > (uint64_t)a.timeout_ns) {
                    atomicCAS(a.status, 0, (int)DEV_TIMEOUT);
                    failed = true;
                    break;
                }
            }
        }
    }
    return !__syncthreads_or(failed);
}

template <typename T>
__device__ __forceinline__ void publish(const SolveArgs<T>& a, int s) {
    __syncthreads();
    if (threadIdx.x == 0 && s != a.withhold) {
        __threadfence();
        st_release(a.flags + blockIdx.x, s);
    }
}

// ---------------------------------------------------------------------------------
// the kernel
// ---------------------------------------------------------------------------------

template <typename T>
__global__ void __launch_bounds__(1024) k_solve(SolveArgs<T> a) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int nrhs = a.nrhs;
    T* ring = (T*)smem;
    T* s_bp = ring + (size_t)a.ring_rows * nrhs;
    T* s_cval = s_bp + (size_t)a.stage_rows * nrhs;
    int32_t* s_ccol = (int32_t*)(s_cval + a.stage_entries);
    int32_t* s_cptr = s_ccol + a.stage_entries;
    int32_t* s_row = s_cptr + a.stage_rows + 1;

    const Lanes ln = make_lanes(a.lpr, nrhs);
    const int ngroups = blockDim.x / a.lpr;
    const int grp = threadIdx.x / a.lpr;
    const int G = gridDim.x, me = blockIdx.x;
    const int ring_mask = a.ring_rows - 1;

    for (int s = 0; s < a.nseg; ++s) {
        const int4 sg = a.segs[s];
        if (sg.x == SEG_WIDE) {
            if (me >= sg.w) continue;
            const int l = sg.y;
            const int64_t p0 = a.lptr[l], p1 = a.lptr[l + 1];
            const int64_t my0 = p0 + (int64_t)me * sg.z;
            const int64_t my1 = min(p1, my0 + (int64_t)sg.z);
            // independent part of the first row before the wait: b-part (dinv b + E b)
            const int64_t pf = my0 + grp;
            const bool act0 = pf < my1;
            const int32_t row0 = act0 ? a.perm[pf] : 0;
            T pre = T(0);
            if (act0 && ln.chunks == 1 && ln.rl < nrhs) pre = bpart(a, pf, row0, ln.rl, ln);
            if (!wait_segment(a, s - 1)) return;
            for (int64_t base = my0; base < my1; base += ngroups) {
                const int64_t p = base + grp;
                const bool act = p < my1;
                const int32_t row = act ? (base == my0 ? row0 : a.perm[p]) : 0;
                const int c0 = act ? a.cptr[p] : 0, c1 = act ? a.cptr[p + 1] : 0;
                for (int j = 0; j < ln.chunks; ++j) {
                    const int k = ln.rl + j * ln.RL;
                    const bool kv = act && k < nrhs;
                    T acc = T(0);
                    if (kv) {
                        acc = (base == my0 && ln.chunks == 1) ? pre : bpart(a, p, row, k, ln);
                        for (int q = c0 + ln.el; q < c1; q += ln.EL)
                            acc -= a.cval[q] * __ldcg(a.xp + (int64_t)a.ccol[q] * nrhs + k);
                    }
                    acc = group_reduce(acc, ln);
                    if (kv && ln.el == 0) {
                        __stcg(a.xp + p * nrhs + k, acc);
                        a.x[(int64_t)row + (int64_t)k * a.ld] = acc;
                    }
                }
            }
            publish(a, s);
            if (a.stamps && threadIdx.x == 0) atomicMax(a.stamps + l, (unsigned long long)globaltimer());
        } else {
            if (me != 0) continue;
            const int blk0 = sg.y, blk1 = sg.z;
            const int64_t run_p0 = a.lptr[a.blocks[blk0].x];
            bool waited = false;
            for (int blk = blk0; blk < blk1; ++blk) {
                const int4 bd = a.blocks[blk];
                const int64_t P0 = a.lptr[bd.x], P1 = a.lptr[bd.y];
                const int64_t Q0 = a.cptr[P0], Q1 = a.cptr[P1];
                const int rows = (int)(P1 - P0), ents = (int)(Q1 - Q0);
                __syncthreads();  // the previous block is done with the staging area
                for (int i = threadIdx.x; i <= rows; i += blockDim.x) {
                    s_cptr[i] = (int32_t)(a.cptr[P0 + i] - Q0);
                    if (i < rows) s_row[i] = a.perm[P0 + i];
                }
                for (int j = threadIdx.x; j < ents; j += blockDim.x) {
                    s_ccol[j] = a.ccol[Q0 + j];
                    s_cval[j] = a.cval[Q0 + j];
                }
                for (int base = 0; base < rows; base += ngroups) {
                    const int i = base + grp;
                    const bool act = i < rows;
                    const int32_t row = act ? a.perm[P0 + i] : 0;
                    for (int j = 0; j < ln.chunks; ++j) {
                        const int k = ln.rl + j * ln.RL;
                        const bool kv = act && k < nrhs;
                        T acc = kv ? bpart(a, P0 + i, row, k, ln) : T(0);
                        acc = group_reduce(acc, ln);
                        if (kv && ln.el == 0) s_bp[(size_t)i * nrhs + k] = acc;
                    }
                }
                if (!waited) {
                    // everything staged so far is independent of x: overlap it with the wait
                    if (!wait_segment(a, s - 1)) return;
                    waited = true;
                } else {
                    __syncthreads();
                }
                const bool narrow = bd.z != 0;
                if (narrow && threadIdx.x >= 32) continue;  // warp 0 alone runs this block
                for (int l = bd.x; l < bd.y; ++l) {
                    const int64_t lp0 = a.lptr[l], lp1 = a.lptr[l + 1];
                    const int64_t ring_lo = max(run_p0, lp1 - (int64_t)a.ring_rows);
                    for (int64_t base = lp0; base < lp1; base += ngroups) {
                        const int64_t p = base + grp;
                        const bool act = p < lp1;
                        const int i = (int)(p - P0);
                        const int c0 = act ? s_cptr[i] : 0, c1 = act ? s_cptr[i + 1] : 0;
                        for (int j = 0; j < ln.chunks; ++j) {
                            const int k = ln.rl + j * ln.RL;
                            const bool kv = act && k < nrhs;
                            T acc = T(0);
                            if (kv) {
                                if (ln.el == 0) acc = s_bp[(size_t)i * nrhs + k];
                                for (int q = c0 + ln.el; q < c1; q += ln.EL) {
                                    const int32_t d = s_ccol[q];
                                    const T xv = d >= ring_lo ? ring[(size_t)(d & ring_mask) * nrhs + k]
                                                              : __ldcg(a.xp + (int64_t)d * nrhs + k);
                                    acc -= s_cval[q] * xv;
                                }
                            }
                            acc = group_reduce(acc, ln);
                            if (kv && ln.el == 0) {
                                ring[(size_t)(p & ring_mask) * nrhs + k] = acc;
                                __stcg(a.xp + p * nrhs + k, acc);
                                a.x[(int64_t)s_row[i] + (int64_t)k * a.ld] = acc;
                            }
                        }
                    }
                    if (narrow) __syncwarp();
                    else __syncthreads();
                    if (a.stamps && threadIdx.x == 0) a.stamps[l] = globaltimer();
                }
            }
            publish(a, s);
        }
    }
}

__global__ void k_gather_level_entries(const int32_t* lptr, const int32_t* cptr, int64_t m, int64_t* out) {
    int64_t l = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (l <= m) out[l] = cptr[lptr[l]];
}

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

    SP_CUDA(cudaMemsetAsync(s->flags.p, 0xff, (size_t)sc.grid * sizeof(int), st));
    SP_CUDA(cudaMemsetAsync(s->status.p, 0, sizeof(int), st));
    if (a.nseg == 0) return SPTRSV_OK;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)sc.grid);
    cfg.blockDim = dim3((unsigned)sc.block);
    cfg.dynamicSmemBytes = sc.smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;  // all CTAs co-resident: waits always make progress
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    SP_CUDA(cudaLaunchKernelEx(&cfg, k_solve<T>, a));
    return SPTRSV_OK;
}

int pow2_floor(int64_t v) {
    int p = 1;
    while ((int64_t)p * 2 <= v) p *= 2;
    return p;
}

}  // namespace

sptrsv_status prepare_schedule(sptrsv_system* s, int nrhs) {
    Schedule& sc = s->sched;
    const int vb = s->dtype == SPTRSV_F64 ? 8 : 4;
    int lpr = s->lpr;
    if (lpr <= 0) {
        if (nrhs >= 2) lpr = std::min(32, pow2_floor(2 * nrhs - 1));
        else lpr = (s->n > 0 && (double)s->nnz_c / (double)s->n > 12.0) ? 4 : 1;
    }
    int block = s->block > 0 ? s->block : 512;
    block = std::max(32, std::min(1024, block / 32 * 32));
    if (lpr > 32 || (lpr & (lpr - 1))) {
        set_error("lanes per row must be a power of two <= 32");
        return SPTRSV_ERR_INVALID;
    }
    if (sc.nrhs == nrhs && sc.lpr == lpr && sc.block == block && sc.run_width == s->run_width && sc.segs.p)
        return SPTRSV_OK;
    const int ngroups = block / lpr;
    // shared memory: x ring (16 KB) + staging (32 KB)
    int ring_rows = pow2_floor(std::max<int64_t>(16, 16384 / ((int64_t)nrhs * vb)));
    int stage_entries = 1536;
    int stage_rows = (int)((32768 - (int64_t)stage_entries * (vb + 4)) / ((int64_t)nrhs * vb + 8));
    if (stage_rows < 16) {
        stage_entries = 256;
        stage_rows = std::max<int64_t>(16, (32768 - (int64_t)stage_entries * (vb + 4)) / ((int64_t)nrhs * vb + 8));
    }
    int run_width = s->run_width > 0 ? s->run_width : (s->run_width < 0 ? 0 : ngroups);
    run_width = std::min(run_width, stage_rows);
    const int64_t m = s->m;
    // entries per level (host copy)
    std::vector<int64_t> lent(m + 1, 0);
    if (m > 0) {
        Scratch tmp;
        SP_TRY(tmp.alloc((m + 1) * sizeof(int64_t), nullptr));
        k_gather_level_entries<<<(unsigned)((m + 1 + 255) / 256), 256>>>(s->lv.level_ptr.p, s->cptr.p, m,
                                                                         tmp.as<int64_t>());
        SP_CUDA(cudaGetLastError());
        SP_CUDA(cudaMemcpy(lent.data(), tmp.p, (m + 1) * sizeof(int64_t), cudaMemcpyDeviceToHost));
    }
    const std::vector<int32_t>& lp = s->lv.h_level_ptr;
    sc.h_segs.clear();
    sc.h_blocks.clear();
    sc.run_levels = 0;
    int64_t max_parts = 1;
    int sms = device_sm_count();
    // occupancy decides the number of CTAs that WIDE levels can be split over
    size_t smem = (size_t)ring_rows * nrhs * vb + (size_t)stage_rows * nrhs * vb + (size_t)stage_entries * (vb + 4) +
                  (size_t)(2 * stage_rows + 1) * 4;
    int occ = 0;
    if (s->dtype == SPTRSV_F64) {
        SP_CUDA(cudaFuncSetAttribute(k_solve<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        SP_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_solve<double>, block, smem));
    } else {
        SP_CUDA(cudaFuncSetAttribute(k_solve<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        SP_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_solve<float>, block, smem));
    }
    if (occ < 1) {
        set_error("solve kernel does not fit an SM with block %d and %zu bytes of shared memory", block, smem);
        return SPTRSV_ERR_UNSUPPORTED;
    }
    const int64_t gmax = (int64_t)sms * occ;
    int64_t l = 0;
    while (l < m) {
        int64_t w = lp[l + 1] - lp[l];
        int64_t e = lent[l + 1] - lent[l];
        bool thin = w <= run_width && e <= stage_entries;
        if (thin) {
            int blk0 = (int)sc.h_blocks.size();
            int64_t l1 = l;
            while (l1 < m) {
                int64_t w1 = lp[l1 + 1] - lp[l1];
                int64_t e1 = lent[l1 + 1] - lent[l1];
                if (!(w1 <= run_width && e1 <= stage_entries)) break;
                // a block: consecutive thin levels within the staging capacity
                int64_t b0 = l1, rows = 0, ents = 0, maxw = 0;
                while (l1 < m) {
                    int64_t w2 = lp[l1 + 1] - lp[l1];
                    int64_t e2 = lent[l1 + 1] - lent[l1];
                    if (!(w2 <= run_width && e2 <= stage_entries)) break;
                    if (rows + w2 > stage_rows || ents + e2 > stage_entries) break;
                    rows += w2;
                    ents += e2;
                    maxw = std::max(maxw, w2);
                    ++l1;
                }
                int narrow = maxw * lpr <= 32 ? 1 : 0;
                sc.h_blocks.push_back(make_int4((int)b0, (int)l1, narrow, 0));
            }
            sc.h_segs.push_back(make_int4(SEG_RUN, blk0, (int)sc.h_blocks.size(), 0));
            sc.run_levels += l1 - l;
            l = l1;
        } else {
            int64_t per = std::max<int64_t>((w + gmax - 1) / gmax, ngroups);
            int64_t parts = (w + per - 1) / per;
            if (per >= INT32_MAX) { set_error("level too wide"); return SPTRSV_ERR_UNSUPPORTED; }
            max_parts = std::max(max_parts, parts);
            sc.h_segs.push_back(make_int4(SEG_WIDE, (int)l, (int)per, (int)parts));
            ++l;
        }
    }
    if (sc.h_blocks.empty()) sc.h_blocks.push_back(make_int4(0, 0, 0, 0));
    SP_TRY(sc.segs.alloc(std::max<size_t>(1, sc.h_segs.size())));
    SP_TRY(sc.blocks.alloc(sc.h_blocks.size()));
    if (!sc.h_segs.empty())
        SP_CUDA(cudaMemcpy(sc.segs.p, sc.h_segs.data(), sc.h_segs.size() * sizeof(int4), cudaMemcpyHostToDevice));
    SP_CUDA(cudaMemcpy(sc.blocks.p, sc.h_blocks.data(), sc.h_blocks.size() * sizeof(int4), cudaMemcpyHostToDevice));
    sc.grid = (int)std::min<int64_t>(gmax, max_parts);
    sc.nrhs = nrhs;
    sc.lpr = lpr;
    sc.block = block;
    sc.run_width = s->run_width;
    sc.ring_rows = ring_rows;
    sc.stage_rows = stage_rows;
    sc.stage_entries = stage_entries;
    sc.smem = smem;
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
