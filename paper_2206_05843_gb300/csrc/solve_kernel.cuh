// solve_kernel.cuh -- the persistent level-set solve kernel (internal; included by the
// translation units that launch it, each of which instantiates its own copy).
//
// One launch walks the schedule.  A WIDE segment is one level whose rows are split in
// contiguous chunks over CTAs 0..parts-1; a CTA publishes the segment in its own
// completion flag (release) and the CTAs of the next segment wait (acquire, bounded)
// for the flags of exactly the CTAs that worked on the previous one.  A RUN segment is a
// chain of thin levels executed by CTA 0 alone with the staged single-CTA executor.
#pragma once

#include <cstdlib>

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
    int parts = (sg.x & SEG_TYPE_MASK) == SEG_RUN ? 1 : sg.w;
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

// The barrier orders every thread's stores of the segment before thread 0's store; the
// release (cumulative, gpu scope) makes them visible to whoever acquires the flag.
template <typename T>
__device__ __forceinline__ void publish(const SolveArgs<T>& a, int s) {
    __syncthreads();
    if (threadIdx.x == 0 && s != a.withhold) st_release(a.flags + blockIdx.x, s);
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

// Wide level, several right-hand sides or several lanes per row: the first row of each
// thread is prepared (coefficients in registers, b-part) before the wait.
// PRE: the b-parts of these rows were computed before the solve (k_bparts) and sit in xp
template <typename T, typename WaitFn, bool PRE = false>
__device__ bool wide_rows_general(const SolveArgs<T>& a, const Lanes& ln, int ngroups, int grp, int64_t my0,
                                  int64_t my1, WaitFn wait) {
    const int nrhs = a.nrhs;
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
    if (act0 && single && ln.rl < nrhs)
        pre = PRE ? (ln.el == 0 ? __ldcg(a.xp + pf * nrhs + ln.rl) : T(0)) : bpart(a, pf, row0, ln.rl, ln);
    if (!wait()) return false;
    for (int64_t base = my0; base < my1; base += ngroups) {
        const int64_t p = base + grp;
        const bool act = p < my1;
        const bool first = base == my0;
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
                    acc = PRE ? (ln.el == 0 ? __ldcg(a.xp + p * nrhs + k) : T(0)) : bpart(a, p, row, k, ln);
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
    return true;
}

// Wide level, one right-hand side, one lane per row: the first row is prepared before
// the wait; coefficients come in chunks of four whose gathers are in flight together.
template <typename T, bool PRE = false>
__device__ __forceinline__ T row_1rhs(const SolveArgs<T>& a, int64_t p, int32_t row, int c0, int c1, T acc) {
    if (!PRE && a.eptr) {
        const int e1 = __ldcs(a.eptr + p + 1);
        for (int q = __ldcs(a.eptr + p); q < e1; q += 4) {
            int ec[4];
            T ev[4], bv[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const bool ok = q + u < e1;
                ec[u] = ok ? __ldcs(a.ecol + q + u) : 0;
                ev[u] = ok ? __ldcs(a.eval + q + u) : T(0);
            }
#pragma unroll
            for (int u = 0; u < 4; ++u) bv[u] = q + u < e1 ? a.b[ec[u]] : T(0);
#pragma unroll
            for (int u = 0; u < 4; ++u)
                if (q + u < e1) acc += ev[u] * bv[u];
        }
    }
    for (int q = c0; q < c1; q += 4) {
        int cc[4];
        T cv[4], xv[4];
        if ((q & 3) == 0 && q + 4 <= c1) {
            // four coefficients on a 16-byte boundary: vector loads (3 instructions, not 8)
            const int4 c4 = __ldcs((const int4*)(a.ccol + q));
            cc[0] = c4.x; cc[1] = c4.y; cc[2] = c4.z; cc[3] = c4.w;
            if (sizeof(T) == 8) {
                const double2 v0 = __ldcs((const double2*)(a.cval + q));
                const double2 v1 = __ldcs((const double2*)(a.cval + q + 2));
                cv[0] = (T)v0.x; cv[1] = (T)v0.y; cv[2] = (T)v1.x; cv[3] = (T)v1.y;
            } else {
                const float4 v = __ldcs((const float4*)(a.cval + q));
                cv[0] = (T)v.x; cv[1] = (T)v.y; cv[2] = (T)v.z; cv[3] = (T)v.w;
            }
        } else {
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const bool ok = q + u < c1;
                cc[u] = ok ? __ldcs(a.ccol + q + u) : 0;
                cv[u] = ok ? __ldcs(a.cval + q + u) : T(0);
            }
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) xv[u] = q + u < c1 ? __ldcg(a.xp + cc[u]) : T(0);
#pragma unroll
        for (int u = 0; u < 4; ++u)
            if (q + u < c1) acc -= cv[u] * xv[u];
    }
    return acc;
}

template <typename T, typename WaitFn, bool PRE = false>
__device__ bool wide_rows_1rhs(const SolveArgs<T>& a, int64_t my0, int64_t my1, WaitFn wait) {
    const int64_t pf = my0 + threadIdx.x;
    const bool act0 = pf < my1;
    const int32_t row0 = act0 ? __ldcs(a.perm + pf) : 0;
    const int f0 = act0 ? __ldcs(a.cptr + pf) : 0, f1 = act0 ? __ldcs(a.cptr + pf + 1) : 0;
    T pre = act0 ? (PRE ? __ldcg(a.xp + pf) : __ldcs(a.dinv + pf) * __ldcs(a.b + row0)) : T(0);
    int32_t pcol[PF];
    T pval[PF];
#pragma unroll
    for (int u = 0; u < PF; ++u) {
        const bool ok = f0 + u < f1;
        pcol[u] = ok ? __ldcs(a.ccol + f0 + u) : 0;
        pval[u] = ok ? __ldcs(a.cval + f0 + u) : T(0);
    }
    if (!wait()) return false;
    if (act0) {
        T xv[PF];
#pragma unroll
        for (int u = 0; u < PF; ++u) xv[u] = f0 + u < f1 ? __ldcg(a.xp + pcol[u]) : T(0);
        T acc = pre;
#pragma unroll
        for (int u = 0; u < PF; ++u)
            if (f0 + u < f1) acc -= pval[u] * xv[u];
        acc = row_1rhs<T, PRE>(a, pf, row0, f0 + PF < f1 ? f0 + PF : f1, f1, acc);
        __stcg(a.xp + pf, acc);
        a.x[row0] = acc;
    }
    for (int64_t p = pf + blockDim.x; p < my1; p += blockDim.x) {
        const int32_t row = __ldcs(a.perm + p);
        const T b0 = PRE ? __ldcg(a.xp + p) : __ldcs(a.dinv + p) * __ldcs(a.b + row);
        const T acc = row_1rhs<T, PRE>(a, p, row, __ldcs(a.cptr + p), __ldcs(a.cptr + p + 1), b0);
        __stcg(a.xp + p, acc);
        __stcs(a.x + row, acc);
    }
    return true;
}

// Wide level, one right-hand side, one lane per row, in the kernel variant for schedules without
// single-CTA runs (registers to spare): as wide_rows_1rhs for the first row; after it, a row's
// coefficients are loaded eight at a time (their gathers in flight together), and the next row's
// position data (perm, row pointers, 1 / L_rr) one row ahead, so that a row costs one round trip
// to memory less.
template <typename T>
__device__ __forceinline__ T row_1rhs8(const SolveArgs<T>& a, int c0, int c1, T acc) {
    for (int q = c0; q < c1; q += 8) {
        int cc[8];
        T cv[8], xv[8];
        if ((q & 3) == 0 && q + 8 <= c1) {
            const int4 i0 = __ldcs((const int4*)(a.ccol + q)), i1 = __ldcs((const int4*)(a.ccol + q + 4));
            cc[0] = i0.x; cc[1] = i0.y; cc[2] = i0.z; cc[3] = i0.w;
            cc[4] = i1.x; cc[5] = i1.y; cc[6] = i1.z; cc[7] = i1.w;
            if (sizeof(T) == 8) {
#pragma unroll
                for (int h = 0; h < 4; ++h) {
                    const double2 v = __ldcs((const double2*)(a.cval + q) + h);
                    cv[2 * h] = (T)v.x;
                    cv[2 * h + 1] = (T)v.y;
                }
            } else {
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const float4 v = __ldcs((const float4*)(a.cval + q) + h);
                    cv[4 * h] = (T)v.x; cv[4 * h + 1] = (T)v.y; cv[4 * h + 2] = (T)v.z; cv[4 * h + 3] = (T)v.w;
                }
            }
        } else {
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const bool ok = q + u < c1;
                cc[u] = ok ? __ldcs(a.ccol + q + u) : 0;
                cv[u] = ok ? __ldcs(a.cval + q + u) : T(0);
            }
        }
#pragma unroll
        for (int u = 0; u < 8; ++u) xv[u] = q + u < c1 ? __ldcg(a.xp + cc[u]) : T(0);
#pragma unroll
        for (int u = 0; u < 8; ++u)
            if (q + u < c1) acc -= cv[u] * xv[u];
    }
    return acc;
}

template <typename T, typename WaitFn>
__device__ bool wide_rows_1rhs_ilp(const SolveArgs<T>& a, int64_t my0, int64_t my1, WaitFn wait) {
    const int64_t pf = my0 + threadIdx.x;
    const bool act0 = pf < my1;
    const int32_t row0 = act0 ? __ldcs(a.perm + pf) : 0;
    const int f0 = act0 ? __ldcs(a.cptr + pf) : 0, f1 = act0 ? __ldcs(a.cptr + pf + 1) : 0;
    T pre = act0 ? __ldcs(a.dinv + pf) * __ldcs(a.b + row0) : T(0);
    int32_t pcol[PF];
    T pval[PF];
#pragma unroll
    for (int u = 0; u < PF; ++u) {
        const bool ok = f0 + u < f1;
        pcol[u] = ok ? __ldcs(a.ccol + f0 + u) : 0;
        pval[u] = ok ? __ldcs(a.cval + f0 + u) : T(0);
    }
    // the second row's position data, independent of x
    int64_t p = pf + blockDim.x;
    bool actn = p < my1;
    int32_t rown = actn ? __ldcs(a.perm + p) : 0;
    int c0n = actn ? __ldcs(a.cptr + p) : 0, c1n = actn ? __ldcs(a.cptr + p + 1) : 0;
    T din = actn ? __ldcs(a.dinv + p) : T(0);
    if (!wait()) return false;
    if (act0) {
        T xv[PF];
#pragma unroll
        for (int u = 0; u < PF; ++u) xv[u] = f0 + u < f1 ? __ldcg(a.xp + pcol[u]) : T(0);
        T acc = pre;
#pragma unroll
        for (int u = 0; u < PF; ++u)
            if (f0 + u < f1) acc -= pval[u] * xv[u];
        acc = row_1rhs(a, pf, row0, f0 + PF < f1 ? f0 + PF : f1, f1, acc);
        __stcg(a.xp + pf, acc);
        a.x[row0] = acc;
    }
    while (actn) {
        const int32_t row = rown;
        const int c0 = c0n, c1 = c1n;
        const T di = din;
        const T bv = __ldcs(a.b + row);
        const int64_t pn = p + blockDim.x;
        actn = pn < my1;
        if (actn) {
            rown = __ldcs(a.perm + pn);
            c0n = __ldcs(a.cptr + pn);
            c1n = __ldcs(a.cptr + pn + 1);
            din = __ldcs(a.dinv + pn);
        }
        T acc = di * bv;
        if (a.eptr) {
            const int e1 = __ldcs(a.eptr + p + 1);
            for (int q = __ldcs(a.eptr + p); q < e1; ++q) acc += __ldcs(a.eval + q) * a.b[__ldcs(a.ecol + q)];
        }
        acc = row_1rhs8(a, c0, c1, acc);
        __stcg(a.xp + p, acc);
        __stcs(a.x + row, acc);
        p = pn;
    }
    return true;
}

// One level per launch (the plain level-set solve): every row of the level is a thread,
// so the whole level is in flight at full occupancy.  Used when the schedule consists of
// a few wide levels, where one launch per level costs less than a device-wide handoff
// would save.
template <typename T>
__global__ void __launch_bounds__(256, 6) k_level(SolveArgs<T> a, int64_t p0, int64_t p1) {
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int nrhs = a.nrhs;
    const int64_t p = p0 + idx / nrhs;
    const int k = (int)(idx % nrhs);
    if (p >= p1) return;
    const int32_t row = __ldcs(a.perm + p);
    if (nrhs == 1) {
        const T acc = row_1rhs(a, p, row, __ldcs(a.cptr + p), __ldcs(a.cptr + p + 1), __ldcs(a.dinv + p) * __ldcs(a.b + row));
        __stcg(a.xp + p, acc);
        __stcs(a.x + row, acc);
        return;
    }
    T acc = a.dinv[p] * a.b[(int64_t)row + (int64_t)k * a.ld];
    if (a.eptr)
        for (int q = a.eptr[p]; q < a.eptr[p + 1]; ++q) acc += a.eval[q] * a.b[(int64_t)a.ecol[q] + (int64_t)k * a.ld];
    for (int q = a.cptr[p]; q < a.cptr[p + 1]; ++q) acc -= a.cval[q] * __ldcg(a.xp + (int64_t)a.ccol[q] * nrhs + k);
    __stcg(a.xp + p * nrhs + k, acc);
    a.x[(int64_t)row + (int64_t)k * a.ld] = acc;
}

// b-parts dinv_p b_row + E_p b of the rows of the staged blocks, written to xp (indexed like
// x) before the solve, so that staging reads one value per row instead of walking its E row.
// CTA me takes blocks me, me + gridDim.x, ...; a thread per row with at most LONG E entries
// (four in flight at a time), then a warp per longer row.
template <typename T>
__global__ void __launch_bounds__(256) k_bparts(SolveArgs<T> a, int nblocks) {
    constexpr int LONG = 64;
    const int me = blockIdx.x, parts = gridDim.x;
    const int nrhs = a.nrhs;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    for (int bi = me; bi < nblocks; bi += parts) {
        const int4 bd = a.blocks[bi];
        for (int64_t p = bd.x + threadIdx.x; p < bd.y; p += blockDim.x) {
            const int e0 = a.eptr ? a.eptr[p] : 0, e1 = a.eptr ? a.eptr[p + 1] : 0;
            if (e1 - e0 > LONG) continue;
            const int32_t row = a.perm[p];
            const T di = a.dinv[p];
            for (int k = 0; k < nrhs; ++k) {
                const int64_t ko = (int64_t)k * a.ld;
                T acc = di * a.b[(int64_t)row + ko];
                int q = e0;
                for (; q + 4 <= e1; q += 4) {
                    const int32_t c0 = a.ecol[q], c1 = a.ecol[q + 1], c2 = a.ecol[q + 2], c3 = a.ecol[q + 3];
                    const T v0 = a.eval[q], v1 = a.eval[q + 1], v2 = a.eval[q + 2], v3 = a.eval[q + 3];
                    const T b0 = a.b[c0 + ko], b1 = a.b[c1 + ko], b2 = a.b[c2 + ko], b3 = a.b[c3 + ko];
                    acc += v0 * b0;
                    acc += v1 * b1;
                    acc += v2 * b2;
                    acc += v3 * b3;
                }
                for (; q < e1; ++q) acc += a.eval[q] * a.b[a.ecol[q] + ko];
                __stcg(a.xp + p * nrhs + k, acc);
            }
        }
        for (int64_t base = bd.x + (int64_t)warp * 32; base < bd.y && a.eptr; base += (int64_t)nwarps * 32) {
            const int64_t pl = base + lane;
            const bool lng = pl < bd.y && a.eptr[pl + 1] - a.eptr[pl] > LONG;
            unsigned mk = __ballot_sync(0xffffffffu, lng);
            while (mk) {
                const int src = __ffs(mk) - 1;
                mk &= mk - 1;
                const int64_t p = base + src;
                const int e0 = a.eptr[p], e1 = a.eptr[p + 1];
                const int32_t row = a.perm[p];
                for (int k = 0; k < nrhs; ++k) {
                    const int64_t ko = (int64_t)k * a.ld;
                    T acc = T(0);
                    for (int q = e0 + lane; q < e1; q += 32) acc += a.eval[q] * a.b[a.ecol[q] + ko];
#pragma unroll
                    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
                    if (lane == 0) __stcg(a.xp + p * nrhs + k, a.dinv[p] * a.b[(int64_t)row + ko] + acc);
                }
            }
        }
    }
}

__global__ void k_stamp(unsigned long long* stamps, int64_t l) {
    if (threadIdx.x == 0) stamps[l] = globaltimer();
}

// ---------------------------------------------------------------------------------
// the kernel
// ---------------------------------------------------------------------------------

// ---------------------------------------------------------------------------------
// wide levels of one right-hand side with the coefficients streamed through shared memory
// ---------------------------------------------------------------------------------

// The CTA's share [my0, my1) of a level is cut into tiles of TR rows (one thread per row).  The
// columns and values of a tile are one contiguous range of the stored arrays; thread 0 copies it
// into one of two shared-memory buffers with two bulk copies on that buffer's mbarrier, two tiles
// ahead of the compute (the first two before the handoff wait, since they do not depend on x).
// A thread keeps its row's position data for the next tile in registers; x gathers read L2.
// the two buffers' mbarriers, the first coefficient of every tile of the CTA's share, and the
// buffers themselves (the dynamic shared memory, which RUN segments use for staging)
__shared__ __align__(8) uint64_t g_tile_mbar[2];
__shared__ int32_t g_tile_q[TILE_MAX + 1];
extern __shared__ __align__(16) unsigned char g_dyn_smem[];

struct TileCtx {
    uint32_t k;  // tile copies this CTA has issued so far (buffer k & 1, phase k >> 1)
};

template <typename T>
__device__ __forceinline__ void tile_issue(const SolveArgs<T>& a, int i, uint32_t slot) {
    constexpr int VA = 16 / (int)sizeof(T);  // values per 16 bytes
    const int q0 = g_tile_q[i], q1 = g_tile_q[i + 1];
    const int qa = q0 & ~3, qv = q0 & ~(VA - 1);  // 16-byte starts of the two copies
    const uint32_t cb = (uint32_t)align16((size_t)(q1 - qa) * 4);
    const uint32_t vbytes = (uint32_t)align16((size_t)(q1 - qv) * sizeof(T));
    unsigned char* base = g_dyn_smem + (size_t)slot * tile_buf_bytes(a.tile_ecap, (int)sizeof(T));
    uint64_t* m = g_tile_mbar + slot;
    mbar_arrive_expect_tx(m, cb + vbytes);
    if (cb) bulk_g2s(base, a.ccol + qa, cb, m);
    if (vbytes) bulk_g2s(base + align16((size_t)(a.tile_ecap + 4) * 4), a.cval + qv, vbytes, m);
}

// bounded wait for tile copies [i0, i1) that were issued and not yet consumed (after a failure)
template <typename T>
__device__ void tile_drain(const SolveArgs<T>& a, const TileCtx& c, int i0, int i1) {
    for (int i = i0; i < i1; ++i) {
        const uint32_t kk = c.k + (uint32_t)i;
        mbar_wait_bounded(g_tile_mbar + (kk & 1), (kk >> 1) & 1, a.timeout_ns);
    }
}

template <typename T, typename WaitFn>
__device__ bool wide_rows_tiled(const SolveArgs<T>& a, int64_t my0, int64_t my1, int TR, TileCtx& c, WaitFn wait) {
    constexpr int VA = 16 / (int)sizeof(T);
    const int t = threadIdx.x;
    const int nt = my1 > my0 ? (int)((my1 - my0 + TR - 1) / TR) : 0;  // the schedule keeps nt <= TILE_MAX
    for (int i = t; i <= nt; i += blockDim.x) g_tile_q[i] = a.cptr[min(my1, my0 + (int64_t)i * TR)];
    // the buffers may hold a single-CTA run's staging, written by the threads: order those writes
    // before the bulk copies that overwrite them
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
    const int pre_issued = nt < 2 ? nt : 2;
    if (t == 0)
        for (int i = 0; i < pre_issued; ++i) tile_issue(a, i, (c.k + i) & 1);
    // this thread's row of tile 0
    int64_t p = my0 + t;
    bool act = t < TR && p < my1;
    int32_t row = act ? __ldcs(a.perm + p) : 0;
    int f0 = act ? __ldcs(a.cptr + p) : 0, f1 = act ? __ldcs(a.cptr + p + 1) : 0;
    T di = act ? __ldcs(a.dinv + p) : T(0);
    if (!wait()) {
        tile_drain(a, c, 0, pre_issued);
        c.k += pre_issued;
        return false;
    }
    const size_t bb = tile_buf_bytes(a.tile_ecap, (int)sizeof(T));
    const size_t voff = align16((size_t)(a.tile_ecap + 4) * 4);
    for (int i = 0; i < nt; ++i) {
        const uint32_t kk = c.k + (uint32_t)i;
        const uint32_t slot = kk & 1;
        const T bv = act ? __ldcs(a.b + row) : T(0);
        // next tile's row
        const int64_t pn = p + TR;
        const bool actn = t < TR && pn < my1;
        const int32_t rown = actn ? __ldcs(a.perm + pn) : 0;
        const int f0n = actn ? __ldcs(a.cptr + pn) : 0, f1n = actn ? __ldcs(a.cptr + pn + 1) : 0;
        const T din = actn ? __ldcs(a.dinv + pn) : T(0);
        const bool got = mbar_wait_bounded(g_tile_mbar + slot, (kk >> 1) & 1, a.timeout_ns);
        if (got && act) {
            const int q0 = g_tile_q[i];
            const int32_t* cs = (const int32_t*)(g_dyn_smem + slot * bb) + (f0 - (q0 & ~3));
            const T* vs = (const T*)(g_dyn_smem + slot * bb + voff) + (f0 - (q0 & ~(VA - 1)));
            const int len = f1 - f0;
            T acc = di * bv;
            if (a.eptr) {
                const int e1 = a.eptr[p + 1];
                for (int q = a.eptr[p]; q < e1; ++q) acc += a.eval[q] * a.b[a.ecol[q]];
            }
            for (int u = 0; u < len; u += 4) {
                T xv[4];
#pragma unroll
                for (int j = 0; j < 4; ++j) xv[j] = u + j < len ? __ldcg(a.xp + cs[u + j]) : T(0);
#pragma unroll
                for (int j = 0; j < 4; ++j)
                    if (u + j < len) acc -= vs[u + j] * xv[j];
            }
            __stcg(a.xp + p, acc);
            __stcs(a.x + row, acc);
        }
        // every thread is done with the buffer before it is refilled; a copy that never completed
        // stops the CTA after its other copies in flight are waited for
        if (__syncthreads_or(!got)) {
            if (t == 0) atomicCAS(a.status, 0, (int)DEV_TIMEOUT);
            tile_drain(a, c, i, min(nt, i + 2));
            c.k += min(nt, i + 2);
            return false;
        }
        if (t == 0 && i + 2 < nt) tile_issue(a, i + 2, slot);
        p = pn;
        act = actn;
        row = rown;
        f0 = f0n;
        f1 = f1n;
        di = din;
    }
    c.k += nt;
    return true;
}

// the rows [my0, my1) of one level with lanes-per-row wl (0: the schedule's), `wait` taken after the
// first row's independent data is in registers
template <typename T, typename WaitFn, bool PRE = false>
__device__ __forceinline__ bool level_rows(const SolveArgs<T>& a, const Lanes& ln, int wl, int64_t my0, int64_t my1,
                                           WaitFn wait) {
    if (wl <= 0) wl = a.lpr;
    if (a.nrhs == 1 && wl == 1) return wide_rows_1rhs<T, WaitFn, PRE>(a, my0, my1, wait);
    if (wl == a.lpr)
        return wide_rows_general<T, WaitFn, PRE>(a, ln, (int)blockDim.x / a.lpr, (int)threadIdx.x / a.lpr, my0, my1,
                                                 wait);
    const Lanes lw = make_lanes(wl, a.nrhs);
    return wide_rows_general<T, WaitFn, PRE>(a, lw, (int)blockDim.x / wl, (int)threadIdx.x / wl, my0, my1, wait);
}

// Thread 0's L2 prefetch of the row data of a CLUSTER segment, PD levels ahead, in three steps over
// three levels: the level pointer of level l + PD (loaded), then the CTA's share of it -- its
// positions' arrays prefetched and its coefficient range loaded -- then that coefficient range
// prefetched.  Every value is used one level after its load, so thread 0 does not wait on it.
struct ClusterPrefetch {
    int64_t q_lo = 0, q_hi = 0;  // level pointer of the level two steps behind
    int c_lo = 0, c_hi = 0;      // coefficient range of the share one step behind
    bool have_q = false, have_c = false;
};
constexpr int CL_PD = 4;

__device__ __forceinline__ void l2_prefetch_1(const void* p, int64_t bytes) {
    // one thread: the 16-byte aligned interior of [p, p + bytes) in 4 KB pieces
    const uint64_t a0 = ((uint64_t)p + 15) & ~(uint64_t)15, e = ((uint64_t)p + (uint64_t)bytes) & ~(uint64_t)15;
    for (uint64_t q = a0; q < e; q += 4096) {
        const uint32_t n = (uint32_t)(e - q < 4096 ? e - q : 4096);
        asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(q), "r"(n) : "memory");
    }
}

template <typename T>
__device__ __forceinline__ void cluster_prefetch_step(const SolveArgs<T>& a, ClusterPrefetch& pf, int l, int lend,
                                                      int me) {
    if (pf.have_c && pf.c_hi > pf.c_lo) {
        l2_prefetch_1(a.ccol + pf.c_lo, (int64_t)(pf.c_hi - pf.c_lo) * 4);
        l2_prefetch_1(a.cval + pf.c_lo, (int64_t)(pf.c_hi - pf.c_lo) * (int64_t)sizeof(T));
    }
    pf.have_c = false;
    if (pf.have_q) {
        const int chunk = ((int)(pf.q_hi - pf.q_lo) + a.csize - 1) / a.csize;
        const int64_t s0 = min(pf.q_hi, pf.q_lo + (int64_t)me * chunk), s1 = min(pf.q_hi, s0 + chunk);
        if (s1 > s0) {
            l2_prefetch_1(a.perm + s0, (s1 - s0) * 4);
            l2_prefetch_1(a.cptr + s0, (s1 - s0 + 1) * 4);
            l2_prefetch_1(a.xp + s0 * a.nrhs, (s1 - s0) * a.nrhs * (int64_t)sizeof(T));
            pf.c_lo = a.cptr[s0];
            pf.c_hi = a.cptr[s1];
            pf.have_c = true;
        }
    }
    const int lq = l + CL_PD;
    pf.have_q = lq < lend;
    if (pf.have_q) {
        pf.q_lo = a.lptr[lq];
        pf.q_hi = a.lptr[lq + 1];
    }
}

// ---------------------------------------------------------------------------------
// CLUSTER segments with x in the cluster's shared memory
// ---------------------------------------------------------------------------------

// One CTA's share of level l: rows [my0, my1), chunks of ceil(width / csize) rows
struct ClShare {
    int64_t p0, my0, my1;
    int chunk;
};
template <typename T>
__device__ __forceinline__ ClShare cl_share(const SolveArgs<T>& a, int l, int me) {
    ClShare c;
    c.p0 = a.lptr[l];
    const int64_t p1 = a.lptr[l + 1];
    c.chunk = ((int)(p1 - c.p0) + a.csize - 1) / a.csize;
    c.my0 = min(p1, c.p0 + (int64_t)me * c.chunk);
    c.my1 = min(p1, c.my0 + c.chunk);
    return c;
}

// the x value of position q: from the shared memory of the CTA that computed it when q is on the previous
// level of the segment (owner (q - pp0) / pchunk, ring slot `slot`), else from L2
template <typename T>
__device__ __forceinline__ T cl_x(const SolveArgs<T>& a, int32_t q, bool prev_ok, int64_t pp0, int pchunk,
                                  uint32_t ring_base, int slot) {
    if (prev_ok && q >= pp0) {
        const int rel = (int)(q - pp0);
        const int owner = rel / pchunk;
        const uint32_t local = ring_base + (uint32_t)((slot * a.dsm_cap + (rel - owner * pchunk)) * (int)sizeof(T));
        uint32_t remote;
        asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(remote) : "r"(local), "r"(owner));
        if (sizeof(T) == 8) {
            double d;
            asm volatile("ld.shared::cluster.f64 %0, [%1];" : "=d"(d) : "r"(remote) : "memory");
            return (T)d;
        } else {
            float f;
            asm volatile("ld.shared::cluster.f32 %0, [%1];" : "=f"(f) : "r"(remote) : "memory");
            return (T)f;
        }
    }
    return __ldcg(a.xp + q);
}

// One CTA's share of a level from its two level pointers (registers, no loads)
struct DsmShare {
    int32_t p0, my0, my1, chunk;
};
__device__ __forceinline__ DsmShare dsm_share(int32_t l0, int32_t l1, int csize, int me) {
    DsmShare c;
    c.p0 = l0;
    c.chunk = (l1 - l0 + csize - 1) / csize;
    c.my0 = min(l1, l0 + me * c.chunk);
    c.my1 = min(l1, c.my0 + c.chunk);
    return c;
}

// the first row of a thread's share of a level, loaded ahead of the level's barrier in two stages:
// its row, row pointers and b-part two levels ahead, its first DSM_PF coefficients one level ahead
constexpr int DSM_PF = 4;
template <typename T>
struct DsmHead {
    int32_t p, row, f0, f1;
    T bp;
};
template <typename T>
struct DsmRow {
    DsmHead<T> h;
    int32_t pc[DSM_PF];
    T pv[DSM_PF];
};
template <typename T>
__device__ __forceinline__ DsmHead<T> dsm_load_head(const SolveArgs<T>& a, int32_t p, bool act) {
    DsmHead<T> h;
    h.p = act ? p : -1;
    h.row = act ? __ldcs(a.perm + p) : 0;
    h.f0 = act ? __ldcs(a.cptr + p) : 0;
    h.f1 = act ? __ldcs(a.cptr + p + 1) : 0;
    h.bp = act ? __ldcg(a.xp + p) : T(0);
    return h;
}
template <typename T>
__device__ __forceinline__ void dsm_load_coefs(const SolveArgs<T>& a, const DsmHead<T>& h, DsmRow<T>& r) {
    r.h = h;
#pragma unroll
    for (int j = 0; j < DSM_PF; ++j) {
        const bool ok = h.f0 + j < h.f1;
        r.pc[j] = ok ? __ldcs(a.ccol + h.f0 + j) : 0;
        r.pv[j] = ok ? __ldcs(a.cval + h.f0 + j) : T(0);
    }
}

// A whole SEG_DSM segment, levels [la, lb), for one CTA of cluster 0, one lane per row.  Level l: wait
// (the segment's entry, or the cluster barrier of level l-1); every row of the CTA's share reads its
// dependencies on level l-1 from the cluster's shared memory and older ones from L2 (four partial sums,
// so that a long row's float64 chain is a quarter as long), and leaves its x in this CTA's ring slot
// (l - la) & 1; arrive.  After the arrive (whose release would otherwise wait for these loads): the
// first row of level l+1 loads its first coefficients, the first row of level l+2 its row data, the
// level pointer of level l+4 comes in (so that no load waits on another one inside a level), the CTA's
// last thread prefetches the data of later levels to L2, and the level's x goes to xp and x in global
// memory -- the next level reads it from shared memory, later levels after later barriers.  On the
// segment's last level the global stores come before the arrive (the next segment reads global memory),
// and a closing cluster barrier at the region's end keeps every CTA until no other CTA reads its shared
// memory.  The rows' b-parts (E rows included) are in xp already (the schedule computes them up front
// for every CLUSTER segment of one right-hand side).  A dead CTA still takes every barrier.  Returns
// false when the entry wait ran out.
template <typename T, typename EnterFn>
__device__ bool cluster_segment_dsm(const SolveArgs<T>& a, int la, int lb, bool last, int me, bool dead,
                                    EnterFn enter) {
    const uint32_t ring_base = smem_addr(g_dyn_smem);
    T* ring = (T*)g_dyn_smem;
    const int t = threadIdx.x;
    const int cs = a.csize;
    const bool pf_thread = t == (int)blockDim.x - 1;
    ClusterPrefetch cpf;
    // level pointers lptr[l .. l+3] (entries past lb repeat lptr[lb]; they describe no rows)
    int32_t L0 = a.lptr[la], L1 = a.lptr[la + 1];
    int32_t L2 = la + 2 <= lb ? a.lptr[la + 2] : L1;
    int32_t L3 = la + 3 <= lb ? a.lptr[la + 3] : L2;
    DsmShare sh = dsm_share(L0, L1, cs, me);
    DsmRow<T> cur;
    dsm_load_coefs(a, dsm_load_head(a, sh.my0 + t, sh.my0 + t < sh.my1), cur);
    DsmShare sh1 = dsm_share(L1, L2, cs, me);
    DsmHead<T> nxt = dsm_load_head(a, sh1.my0 + t, la + 1 < lb && sh1.my0 + t < sh1.my1);
    int32_t L4 = la + 4 <= lb ? a.lptr[la + 4] : L3;
    if (pf_thread && !dead) cluster_prefetch_step(a, cpf, la, lb, me);
    int32_t pp0 = 0;
    int pchunk = 1;
    for (int l = la; l < lb; ++l) {
        const int slot = (l - la) & 1;
        if (l == la) dead = !enter() || dead;
        else cluster_wait();
        const bool prev_ok = l > la;
        if (!dead) {
            // the thread's rows of the share: the first from registers, the others loaded here
            for (int32_t q = sh.my0 + t; q < sh.my1; q += blockDim.x) {
                const bool first = q == cur.h.p;
                const int32_t r = first ? cur.h.row : __ldcs(a.perm + q);
                const int c0 = first ? cur.h.f0 : __ldcs(a.cptr + q), c1 = first ? cur.h.f1 : __ldcs(a.cptr + q + 1);
                T sum[4] = {first ? cur.h.bp : __ldcg(a.xp + q), T(0), T(0), T(0)};
                int u = c0;
                if (first) {
                    T xv[DSM_PF];
#pragma unroll
                    for (int j = 0; j < DSM_PF; ++j)
                        xv[j] = c0 + j < c1 ? cl_x(a, cur.pc[j], prev_ok, pp0, pchunk, ring_base, slot ^ 1) : T(0);
#pragma unroll
                    for (int j = 0; j < DSM_PF; ++j)
                        if (c0 + j < c1) sum[j & 3] -= cur.pv[j] * xv[j];
                    u = c0 + DSM_PF;
                }
                for (; u < c1; u += 4) {
                    int32_t cc[4];
                    T cv[4], xv[4];
#pragma unroll
                    for (int j = 0; j < 4; ++j) {
                        const bool ok = u + j < c1;
                        cc[j] = ok ? __ldcs(a.ccol + u + j) : 0;
                        cv[j] = ok ? __ldcs(a.cval + u + j) : T(0);
                    }
#pragma unroll
                    for (int j = 0; j < 4; ++j)
                        xv[j] = u + j < c1 ? cl_x(a, cc[j], prev_ok, pp0, pchunk, ring_base, slot ^ 1) : T(0);
#pragma unroll
                    for (int j = 0; j < 4; ++j)
                        if (u + j < c1) sum[j] -= cv[j] * xv[j];
                }
                const T acc = (sum[0] + sum[1]) + (sum[2] + sum[3]);
                ring[slot * a.dsm_cap + (q - sh.my0)] = acc;
                if (l + 1 == lb) {  // the segment's last level: global memory before the arrive
                    __stcg(a.xp + q, acc);
                    a.x[r] = acc;
                }
            }
        }
        if (l + 1 < lb || !last) cluster_arrive();
        // loads for later levels, independent of x
        const int32_t p_l = cur.h.p, row_l = cur.h.row;
        dsm_load_coefs(a, nxt, cur);  // level l+1
        const DsmShare sh2 = dsm_share(L2, L3, cs, me);
        nxt = dsm_load_head(a, sh2.my0 + t, l + 2 < lb && sh2.my0 + t < sh2.my1);  // level l+2
        const int32_t L5 = l + 5 <= lb ? a.lptr[l + 5] : L4;
        if (pf_thread && !dead && l + 1 < lb) cluster_prefetch_step(a, cpf, l + 1, lb, me);
        if (!dead && l + 1 < lb) {
            // this thread's own values of the level (no other thread wrote them)
            for (int32_t q = sh.my0 + t; q < sh.my1; q += blockDim.x) {
                const T v = ring[slot * a.dsm_cap + (q - sh.my0)];
                __stcg(a.xp + q, v);
                __stcs(a.x + (q == p_l ? row_l : __ldcs(a.perm + q)), v);
            }
        }
        if (a.stamps && t == 0 && !dead) atomicMax(a.stamps + l, (unsigned long long)globaltimer());
        pp0 = sh.p0;
        pchunk = max(1, sh.chunk);
        sh = dsm_share(L1, L2, cs, me);
        L1 = L2;
        L2 = L3;
        L3 = L4;
        L4 = L5;
    }
    if (last) {
        // no CTA leaves while another may still read its ring
        cluster_arrive();
        cluster_wait();
    }
    return !dead;
}

// A CTA whose bounded wait ran out ("dead": the status word is set) does no more work and no more
// flag waits, and publishes nothing, so that the CTAs waiting on it run out too; inside a cluster
// region it still takes every cluster barrier, so that no CTA of its cluster waits on it forever.
// No CTA returns early.
// kernel variants (one register allocation each): plain, plain with tiled WIDE levels, cluster, and
// WIDE levels only (no single-CTA runs, no shared memory)
enum KMode : int { KM_PLAIN = 0, KM_TILED = 1, KM_CLUSTER = 2, KM_WIDE = 3 };

template <typename T, int MODE>
__global__ void __launch_bounds__(512, MODE == 2 ? 1 : 2) k_solve(SolveArgs<T> a) {
    constexpr bool CL = MODE == KM_CLUSTER;
    constexpr bool TL = MODE == KM_TILED;
    constexpr bool WO = MODE == KM_WIDE;
    unsigned char* smem = g_dyn_smem;
    const int nrhs = a.nrhs;
    const Lanes ln = make_lanes(a.lpr, nrhs);
    const int me = blockIdx.x;
    TileCtx tc{0u};
    if (TL && a.tile_ecap > 0) {
        if (threadIdx.x == 0) {
            mbar_init(&g_tile_mbar[0], 1);
            mbar_init(&g_tile_mbar[1], 1);
            mbar_fence_init();
        }
        __syncthreads();
    }
    if constexpr (!CL) {
        // no CLUSTER segments: a CTA whose bounded wait runs out returns
        for (int s = 0; s < a.nseg; ++s) {
            const int4 sg = a.segs[s];
            const int wl = (sg.x >> SEG_LPR_SHIFT) & SEG_LPR_MASK;
            if ((sg.x & SEG_TYPE_MASK) == SEG_WIDE) {
                if (me >= sg.w) continue;
                const int l = sg.y;
                const int64_t p0 = a.lptr[l], p1 = a.lptr[l + 1];
                const int64_t my0 = p0 + (int64_t)me * sg.z;
                const int64_t my1 = min(p1, my0 + (int64_t)sg.z);
                auto w = [&]() { return wait_segment(a, s - 1); };
                bool ok;
                if constexpr (TL) {
                    ok = (sg.x & SEG_TILED)
                             ? wide_rows_tiled(a, my0, my1, TILE_ROWS >> ((sg.x >> SEG_TILE_SHIFT) & 3), tc, w)
                             : level_rows(a, ln, wl, my0, my1, w);
                } else if constexpr (WO) {
                    ok = (nrhs == 1 && (wl == 1 || (wl == 0 && a.lpr == 1))) ? wide_rows_1rhs_ilp(a, my0, my1, w)
                                                                             : level_rows(a, ln, wl, my0, my1, w);
                } else {
                    ok = level_rows(a, ln, wl, my0, my1, w);
                }
                if (!ok) return;
                publish(a, s);
                if (a.stamps && threadIdx.x == 0) atomicMax(a.stamps + l, (unsigned long long)globaltimer());
            } else {
                if (WO || me != 0) continue;  // the wide-only variant never holds a run
                SysView<T> v{nrhs,   a.ld,   a.perm, a.lptr, a.cptr, a.ccol, a.cval,
                             a.dinv, a.eptr, a.ecol, a.eval, a.b,    a.x,    a.xp,
                             a.pre ? a.xp : nullptr};
                auto wait = [&]() { return wait_segment(a, s - 1); };
                if (!run_blocks(v, smem, RunGeom{a.ring_rows, a.stage_rows, a.stage_entries}, ln, a.blocks, sg.y,
                                sg.z, wait, a.stamps))
                    return;
                publish(a, s);
            }
        }
    } else {
        // the cluster shape the schedule was built for: CTAs csize apart form one cluster.  A launch
        // without it (every CTA sees the same) records the error and ends before any CTA touches
        // another's shared memory or waits at a cluster barrier
        unsigned ncta, crank;
        asm volatile("mov.u32 %0, %%cluster_nctarank;" : "=r"(ncta));
        asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(crank));
        if (__syncthreads_or((int)ncta != a.csize || (int)crank != me % a.csize)) {
            if (threadIdx.x == 0) atomicCAS(a.status, 0, (int)DEV_LAUNCH);
            return;
        }
        const bool cluster0 = me < a.csize;  // cluster 0: CTAs 0 .. csize-1 of the 1-D grid
        bool dead = false;
        for (int s = 0; s < a.nseg; ++s) {
            const int4 sg = a.segs[s];
            const int type = sg.x & SEG_TYPE_MASK;
            const int wl = (sg.x >> SEG_LPR_SHIFT) & SEG_LPR_MASK;
            const bool region = CL && (sg.x & SEG_REGION) != 0;
            const bool first = (sg.x & SEG_FIRST) != 0, last = (sg.x & SEG_LAST) != 0;
            if (region ? !cluster0 : (dead || (type == SEG_WIDE ? me >= sg.w : me != 0))) continue;
            if (type == SEG_RUN) {
                // entry: the cluster barrier of the previous segment inside a region, else its flags
                const bool barrier_entry = region && !first;
                const bool was_dead = dead;
                auto w = [&a, s, barrier_entry, was_dead]() -> bool {
                    if (barrier_entry) {
                        cluster_wait();
                        return !was_dead;
                    }
                    return was_dead ? false : wait_segment(a, s - 1);
                };
                bool ok;
                if (me == 0) {
                    SysView<T> v{nrhs,   a.ld,   a.perm, a.lptr, a.cptr, a.ccol, a.cval,
                                 a.dinv, a.eptr, a.ecol, a.eval, a.b,    a.x,    a.xp,
                                 a.pre ? a.xp : nullptr};
                    ok = was_dead ? (w(), false)
                                  : run_blocks(v, smem, RunGeom{a.ring_rows, a.stage_rows, a.stage_entries}, ln, a.blocks,
                                               sg.y, sg.z, w, a.stamps);
                } else {
                    ok = barrier_entry ? w() : !was_dead;  // other CTAs of the cluster: the barrier only
                }
                if (!ok) dead = true;
                if (region && !last) cluster_arrive();
            } else if (type == SEG_CLUSTER && (sg.x & SEG_DSM)) {
                // the whole segment with x in the cluster's shared memory
                const bool was_dead = dead;
                auto enter = [&a, s, first, was_dead]() -> bool {
                    if (!first) {
                        cluster_wait();
                        return !was_dead;
                    }
                    return was_dead ? false : wait_segment(a, s - 1);
                };
                dead = !cluster_segment_dsm<T>(a, sg.y, sg.z, last, me, dead, enter);
            } else {
                // WIDE: one level over CTAs 0..parts-1; CLUSTER: levels [y, z), each over the cluster
                const int la = sg.y, lb = CL && type == SEG_CLUSTER ? sg.z : sg.y + 1;
                ClusterPrefetch cpf;
                for (int l = la; l < lb; ++l) {
                    if (type == SEG_CLUSTER && threadIdx.x == 0 && !dead) cluster_prefetch_step(a, cpf, l, lb, me);
                    const bool barrier_entry = l != la || (region && !first);
                    const bool was_dead = dead;
                    auto w = [&a, s, barrier_entry, was_dead]() -> bool {
                        if (barrier_entry) {
                            cluster_wait();
                            return !was_dead;
                        }
                        return was_dead ? false : wait_segment(a, s - 1);
                    };
                    const int64_t p0 = a.lptr[l], p1 = a.lptr[l + 1];
                    const int chunk = type == SEG_WIDE ? sg.z : ((int)(p1 - p0) + a.csize - 1) / a.csize;
                    const int64_t my0 = min(p1, p0 + (int64_t)me * chunk), my1 = min(p1, my0 + chunk);
                    const bool ok = was_dead ? (w(), false)
                                    : (type == SEG_CLUSTER && a.pre_cl)
                                        ? level_rows<T, decltype(w), true>(a, ln, wl, my0, my1, w)
                                        : level_rows(a, ln, wl, my0, my1, w);
                    if (!ok) dead = true;
                    else if (a.stamps && threadIdx.x == 0) atomicMax(a.stamps + l, (unsigned long long)globaltimer());
                    if (region && (l + 1 < lb || !last)) cluster_arrive();
                }
            }
            // completion flags: outside regions after every segment, else after the region's last one
            // (by the CTAs that worked on it: all of a CLUSTER segment, CTA 0 of a RUN)
            if (!dead && (!region || last) && (type != SEG_RUN || me == 0)) publish(a, s);
        }
    }
}

// Kernel attributes of the k_solve instantiation a launch with csize CTAs per cluster uses
// the variant a schedule runs: cluster when it has CLUSTER segments, tiled when it has tiled WIDE
// segments, else plain
inline int k_mode(int csize, int tile_ecap, int runs = 1) {
    return csize > 1 ? KM_CLUSTER : (tile_ecap > 0 ? KM_TILED : (runs == 0 ? KM_WIDE : KM_PLAIN));
}

template <typename T>
const void* k_solve_fn(int mode) {
    switch (mode) {
        case KM_CLUSTER: return (const void*)k_solve<T, KM_CLUSTER>;
        case KM_TILED: return (const void*)k_solve<T, KM_TILED>;
        case KM_WIDE: return (const void*)k_solve<T, KM_WIDE>;
        default: return (const void*)k_solve<T, KM_PLAIN>;
    }
}

template <typename T>
cudaError_t k_solve_attrs(size_t smem, int csize, int tile_ecap, int runs = 1) {
    const void* fn = k_solve_fn<T>(k_mode(csize, tile_ecap, runs));
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess && csize > 8) e = cudaFuncSetAttribute(fn, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    return e;
}

// Launches k_solve for a prepared schedule: cooperative (all CTAs co-resident, so every bounded
// wait can succeed), and with the schedule's cluster size when it has CLUSTER segments.
template <typename T>
cudaError_t launch_k_solve(const SolveArgs<T>& a, int grid, int block, size_t smem, int csize, cudaStream_t st,
                           int runs = 1) {
    // SPTRSV_PROFILE_LAUNCH=1: launches with clusters go out without the cooperative attribute, for
    // profilers that run cooperative launches without their cluster shape (the kernel detects that
    // and stops with an error); the grid is sized from cluster occupancy either way, so every CTA of
    // it is resident on an otherwise idle GPU
    static const bool profile_launch = [] {
        const char* e = std::getenv("SPTRSV_PROFILE_LAUNCH");
        return e && e[0] == '1';
    }();
    const int mode = k_mode(csize, a.tile_ecap, runs);
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)grid);
    cfg.blockDim = dim3((unsigned)block);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[2];
    int na = 0;
    if (csize <= 1 || !profile_launch) {
        attr[na].id = cudaLaunchAttributeCooperative;
        attr[na].val.cooperative = 1;
        ++na;
    }
    if (csize > 1) {
        attr[na].id = cudaLaunchAttributeClusterDimension;
        attr[na].val.clusterDim.x = (unsigned)csize;
        attr[na].val.clusterDim.y = 1;
        attr[na].val.clusterDim.z = 1;
        ++na;
    }
    cfg.attrs = attr;
    cfg.numAttrs = na;
    if (mode == KM_CLUSTER) return cudaLaunchKernelEx(&cfg, k_solve<T, KM_CLUSTER>, a);
    if (mode == KM_TILED) return cudaLaunchKernelEx(&cfg, k_solve<T, KM_TILED>, a);
    if (mode == KM_WIDE) return cudaLaunchKernelEx(&cfg, k_solve<T, KM_WIDE>, a);
    return cudaLaunchKernelEx(&cfg, k_solve<T, KM_PLAIN>, a);
}

}  // namespace
}  // namespace sp
