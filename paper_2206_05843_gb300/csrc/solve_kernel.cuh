// solve_kernel.cuh -- the persistent level-set solve kernel (internal; included by the
// translation units that launch it, each of which instantiates its own copy).
//
// One launch walks the schedule.  A WIDE segment is one level whose rows are split in
// contiguous chunks over CTAs 0..parts-1; a CTA publishes the segment in its own
// completion flag (release) and the CTAs of the next segment wait (acquire, bounded)
// for the flags of exactly the CTAs that worked on the previous one.  A RUN segment is a
// chain of thin levels executed by CTA 0 alone with the staged single-CTA executor.
#pragma once

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
            SysView<T> v{nrhs,   a.ld,   a.perm, a.lptr, a.cptr, a.ccol, a.cval, a.dinv,
                         a.eptr, a.ecol, a.eval, a.b,    a.x,    a.xp};
            auto wait = [&]() { return wait_segment(a, s - 1); };
            if (!run_blocks(v, smem, RunGeom{a.ring_rows, a.stage_rows, a.stage_entries}, ln, a.blocks, sg.y, sg.z,
                            wait, a.stamps))
                return;
            publish(a, s);
        }
    }
}

}  // namespace
}  // namespace sp
