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

#include "run_exec.cuh"

namespace sp {
namespace {

constexpr int PF = 6;  // coefficients of a wide-level row prefetched into registers before the wait

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

// b-part partial over this lane's share of the E row (lanes split the row)
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
// the kernel
// ---------------------------------------------------------------------------------

template <typename T>
__global__ void __launch_bounds__(512, 2) k_solve(SolveArgs<T> a) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int nrhs = a.nrhs;
    const Lanes ln = make_lanes(a.lpr, nrhs);
    const int ngroups = blockDim.x / a.lpr;
    const int grp = threadIdx.x / a.lpr;
    const int me = blockIdx.x;

    for (int s = 0; s < a.nseg; ++s) {
        const int4 sg = a.segs[s];
        if (sg.x == SEG_WIDE) {
            if (me >= sg.w) continue;
            const int l = sg.y;
            const int64_t p0 = a.lptr[l], p1 = a.lptr[l + 1];
            const int64_t my0 = p0 + (int64_t)me * sg.z;
            const int64_t my1 = min(p1, my0 + (int64_t)sg.z);
            // everything of the first row that does not depend on x, before the wait
            const int64_t pf = my0 + grp;
            const bool act0 = pf < my1;
            const bool single = ln.chunks == 1;
            const int32_t row0 = act0 ? a.perm[pf] : 0;
            const int f0 = act0 ? a.cptr[pf] : 0, f1 = act0 ? a.cptr[pf + 1] : 0;
            T pre = T(0);
            int32_t pcol[PF];
            T pval[PF];
#pragma unroll
            for (int u = 0; u < PF; ++u) {
                const int q = f0 + ln.el + u * ln.EL;
                const bool ok = single && q < f1;
                pcol[u] = ok ? a.ccol[q] : -1;
                pval[u] = ok ? a.cval[q] : T(0);
            }
            if (act0 && single && ln.rl < nrhs) pre = bpart(a, pf, row0, ln.rl, ln);
            if (!wait_segment(a, s - 1)) return;
            int64_t base = my0;
            const bool two = nrhs == 1 && a.lpr == 1;
            for (; base < my1; base += ngroups) {
                const int64_t p = base + grp;
                const bool act = p < my1;
                const bool first = base == my0;
                if (!first && two) break;  // the rest goes two rows per thread below
                const int32_t row = act ? (first ? row0 : a.perm[p]) : 0;
                const int c0 = act ? (first ? f0 : a.cptr[p]) : 0, c1 = act ? (first ? f1 : a.cptr[p + 1]) : 0;
                for (int j = 0; j < ln.chunks; ++j) {
                    const int k = ln.rl + j * ln.RL;
                    const bool kv = act && k < nrhs;
                    T acc = T(0);
                    if (kv) {
                        int q = c0 + ln.el;
                        if (first && single) {
                            acc = pre;
#pragma unroll
                            for (int u = 0; u < PF; ++u)
                                if (pcol[u] >= 0) acc -= pval[u] * __ldcg(a.xp + (int64_t)pcol[u] * nrhs + k);
                            q += PF * ln.EL;
                        } else {
                            acc = bpart(a, p, row, k, ln);
                        }
                        for (; q < c1; q += ln.EL) acc -= a.cval[q] * __ldcg(a.xp + (int64_t)a.ccol[q] * nrhs + k);
                    }
                    acc = group_reduce(acc, ln);
                    if (kv && ln.el == 0) {
                        __stcg(a.xp + p * nrhs + k, acc);
                        a.x[(int64_t)row + (int64_t)k * a.ld] = acc;
                    }
                }
            }
            // one right-hand side, a row per thread: two independent rows in flight
            for (; base < my1; base += 2 * ngroups) {
                const int64_t pa = base + grp, pb = pa + ngroups;
                const bool aa = pa < my1, ab = pb < my1;
                const int32_t ra = aa ? a.perm[pa] : 0, rb = ab ? a.perm[pb] : 0;
                const int ca0 = aa ? a.cptr[pa] : 0, ca1 = aa ? a.cptr[pa + 1] : 0;
                const int cb0 = ab ? a.cptr[pb] : 0, cb1 = ab ? a.cptr[pb + 1] : 0;
                T acc_a = aa ? a.dinv[pa] * a.b[ra] : T(0);
                T acc_b = ab ? a.dinv[pb] * a.b[rb] : T(0);
                if (a.eptr) {
                    const int ea0 = aa ? a.eptr[pa] : 0, ea1 = aa ? a.eptr[pa + 1] : 0;
                    const int eb0 = ab ? a.eptr[pb] : 0, eb1 = ab ? a.eptr[pb + 1] : 0;
                    for (int q = ea0; q < ea1; ++q) acc_a += a.eval[q] * a.b[a.ecol[q]];
                    for (int q = eb0; q < eb1; ++q) acc_b += a.eval[q] * a.b[a.ecol[q]];
                }
                const int la = ca1 - ca0, lb = cb1 - cb0;
                const int lmax = la > lb ? la : lb;
                for (int u = 0; u < lmax; ++u) {
                    T xa = T(0), xb = T(0), va = T(0), vb = T(0);
                    if (u < la) {
                        va = a.cval[ca0 + u];
                        xa = __ldcg(a.xp + a.ccol[ca0 + u]);
                    }
                    if (u < lb) {
                        vb = a.cval[cb0 + u];
                        xb = __ldcg(a.xp + a.ccol[cb0 + u]);
                    }
                    if (u < la) acc_a -= va * xa;
                    if (u < lb) acc_b -= vb * xb;
                }
                if (aa) {
                    __stcg(a.xp + pa, acc_a);
                    a.x[ra] = acc_a;
                }
                if (ab) {
                    __stcg(a.xp + pb, acc_b);
                    a.x[rb] = acc_b;
                }
            }
            publish(a, s);
            if (a.stamps && threadIdx.x == 0) atomicMax(a.stamps + l, (unsigned long long)globaltimer());
        } else {
            if (me != 0) continue;
            RunSmem<T> sm;
            sm.carve(smem, nrhs, RunGeom{a.ring_rows, a.stage_rows, a.stage_entries});
            SysView<T> v{nrhs,   a.ld,   a.perm, a.lptr, a.cptr, a.ccol, a.cval, a.dinv,
                         a.eptr, a.ecol, a.eval, a.b,    a.x,    a.xp};
            auto wait = [&]() { return wait_segment(a, s - 1); };
            if (!run_blocks(v, sm, ln, a.blocks, sg.y, sg.z, wait, a.stamps)) return;
            publish(a, s);
        }
    }
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

// Cuts levels [l_begin, l_end) into blocks that fit the staging area: whole levels while
// they fit, a level that does not fit is split by rows.  Returns 0, or -1 when a single
// row has more coefficients than the staging area holds.
int build_run_blocks(const int32_t* lp, const int32_t* cptr, int64_t l_begin, int64_t l_end, int stage_rows,
                     int stage_entries, int lpr, std::vector<int4>& out) {
    int64_t P = lp[l_begin];
    const int64_t Pend = lp[l_end];
    int64_t l = l_begin;
    while (P < Pend) {
        while (lp[l + 1] <= P) ++l;
        const int64_t P0 = P, l0 = l;
        int64_t rows = 0, ents = 0, maxw = 0;
        int64_t lcur = l;
        while (P < Pend) {
            while (lp[lcur + 1] <= P) ++lcur;
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
    if (sc.nrhs == nrhs && sc.lpr == lpr && sc.block == block && sc.run_width == s->run_width && sc.segs.p)
        return SPTRSV_OK;
    const int ngroups = block / lpr;
    // shared memory: staging (~32 KB) + an x ring of at least twice the staged rows
    int stage_entries = 1536;
    int stage_rows = (int)((32768 - (int64_t)stage_entries * (vb + 4)) / ((int64_t)nrhs * vb + 12));
    if (stage_rows < 16) {
        stage_entries = 256;
        stage_rows = (int)std::max<int64_t>(16, (32768 - (int64_t)stage_entries * (vb + 4)) / ((int64_t)nrhs * vb + 12));
    }
    int ring_rows = 16;
    while (ring_rows < 2 * stage_rows) ring_rows *= 2;
    int run_width = s->run_width > 0 ? s->run_width : (s->run_width < 0 ? 0 : ngroups);
    run_width = std::min(run_width, stage_rows);
    const int64_t m = s->m;
    // row pointers of the stored coefficients (host copy) for cutting blocks
    std::vector<int32_t> hcptr(s->n + 1, 0);
    SP_CUDA(cudaMemcpy(hcptr.data(), s->cptr.p, (s->n + 1) * sizeof(int32_t), cudaMemcpyDeviceToHost));
    const std::vector<int32_t>& lp = s->lv.h_level_ptr;
    sc.h_segs.clear();
    sc.h_blocks.clear();
    sc.run_levels = 0;
    int64_t max_parts = 1;
    int sms = device_sm_count();
    // occupancy decides the number of CTAs that WIDE levels can be split over
    size_t smem = run_smem_bytes(vb, nrhs, RunGeom{ring_rows, stage_rows, stage_entries});
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
    auto thin = [&](int64_t l) {
        return lp[l + 1] - lp[l] <= run_width && (int64_t)hcptr[lp[l + 1]] - hcptr[lp[l]] <= stage_entries;
    };
    int64_t l = 0;
    while (l < m) {
        if (thin(l)) {
            int64_t l1 = l;
            while (l1 < m && thin(l1)) ++l1;
            int blk0 = (int)sc.h_blocks.size();
            if (build_run_blocks(lp.data(), hcptr.data(), l, l1, stage_rows, stage_entries, lpr, sc.h_blocks) != 0) {
                set_error("schedule: a row has more coefficients than the staging area");
                return SPTRSV_ERR_UNSUPPORTED;
            }
            sc.h_segs.push_back(make_int4(SEG_RUN, blk0, (int)sc.h_blocks.size(), 0));
            sc.run_levels += l1 - l;
            l = l1;
        } else {
            int64_t w = lp[l + 1] - lp[l];
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
