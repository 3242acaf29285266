// run_exec.cuh -- single-CTA executor of a chain of levels (internal).
//
// Used for runs of thin levels inside the persistent solve and for whole matrices in
// the batched solve.  On GB300 a float64 warp instruction occupies its sub-partition's
// FP64 pipe for about 64 cycles, so a thin level costs at least (dependent FMAs) x 31 ns;
// the level loop therefore touches nothing but shared memory:
//   stage A (independent of x): rows of the block, its level pointers and the b-part of
//           every row (dinv_r b_r plus the rewritten rows' E row times b);
//   stage B (after every x the block reads from outside the ring is final): each
//           coefficient whose dependency is older than the ring window is applied to the
//           b-part right away; the others are compacted with their ring slot, or, in a
//           fast block, laid out as one record per lane and FMA step (below);
//   compute: per level, rows read x only from the shared-memory ring;
//   write-out: the block's x leaves the ring once, coalesced.
//
// Fast blocks.  An SM runs at most four float64 warp instructions at a time, each for ~64
// cycles, and a predicated-off one still takes its slot.  A fast block (every level within
// 32 lanes of rows x right-hand sides x lanes per row, at most K_MAX FMAs per lane) runs exactly K
// FMAs per lane and level, K fixed for the block: the staging pads each lane to K records
// (coefficient, ring slot) with (0, zero slot), and warp 0 runs a branch-free loop whose
// per-level metadata is loaded one level ahead.
#pragma once

#include "system.cuh"

namespace sp {

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

// the arrays of one stored system as the executors read them
template <typename T>
struct SysView {
    int nrhs;
    int64_t ld;
    const int32_t* __restrict__ perm;
    const int32_t* __restrict__ lptr;
    const int32_t* __restrict__ cptr;
    const int32_t* __restrict__ ccol;
    const T* __restrict__ cval;
    const T* __restrict__ dinv;
    const int32_t* __restrict__ eptr;  // nullptr: no rewritten row
    const int32_t* __restrict__ ecol;
    const T* __restrict__ eval;
    const T* __restrict__ b;
    T* x;
    T* xp;  // x in stored order, position-major: xp[p * nrhs + k]
    const T* bpre;  // b-parts computed before the solve, indexed like xp; nullptr: staging computes them
};

// b-part of row p for right-hand side k: dinv_p b_row + sum over the E row
template <typename T>
__device__ __forceinline__ T bpart_full(const SysView<T>& v, int64_t p, int32_t row, int k) {
    T acc = v.dinv[p] * v.b[(int64_t)row + (int64_t)k * v.ld];
    if (v.eptr) {
        const int e1 = v.eptr[p + 1];
        for (int q = v.eptr[p]; q < e1; ++q) acc += v.eval[q] * v.b[(int64_t)v.ecol[q] + (int64_t)k * v.ld];
    }
    return acc;
}

struct RunGeom {
    int ring_rows, stage_rows, stage_entries;
};

// One staging buffer: 32 KB.  Two CTAs per SM (the persistent kernel's occupancy, which its
// registers set) then leave about a third of the unified L1 / shared array to L1, which the
// wide levels' per-lane vector loads use to merge the halves of each sector: larger buffers
// (44 KB) shortened the thin-level block turnover but made wide levels slower (w2: 228 ->
// 390 us) for the smaller L1.
constexpr int64_t STAGE_BYTES = 32768;
constexpr int STAGE_ENTRIES = 1536;

// staging geometry for nrhs right-hand sides of vb-byte values: rows and coefficients of one
// buffer, and an x ring of at least twice the staged rows
inline RunGeom run_geometry(int nrhs, int vb) {
    RunGeom g;
    g.stage_entries = STAGE_ENTRIES;
    g.stage_rows = (int)((STAGE_BYTES - (int64_t)g.stage_entries * (vb + 4)) / ((int64_t)nrhs * vb + 12));
    if (g.stage_rows < 16) {
        g.stage_entries = 256;
        g.stage_rows =
            (int)std::max<int64_t>(16, (STAGE_BYTES - (int64_t)g.stage_entries * (vb + 4)) / ((int64_t)nrhs * vb + 12));
    }
    g.ring_rows = 16;
    while (g.ring_rows < 2 * g.stage_rows) g.ring_rows *= 2;
    return g;
}

inline size_t run_stage_bytes(int vb, int nrhs, const RunGeom& g) {
    return (size_t)g.stage_rows * nrhs * vb + (size_t)g.stage_entries * (vb + 4) + (size_t)(3 * g.stage_rows + 2) * 4;
}

// the ring holds ring_rows x nrhs values plus RING_PAD spare values: two extra slots (rows) of
// nrhs <= 32 values each -- the zero slot ring_rows (read by the padding records of fast
// blocks, always 0) and the dummy slot ring_rows + 1 (written by their idle lanes)
constexpr int RING_PAD = 64;
constexpr int FAST_MAX_RHS = RING_PAD / 2;

// the x ring plus two staging buffers (one is filled while the other is computed)
inline size_t run_smem_bytes(int vb, int nrhs, const RunGeom& g) {
    return ((size_t)g.ring_rows * nrhs + RING_PAD) * vb + 2 * ((run_stage_bytes(vb, nrhs, g) + 15) / 16 * 16);
}

// one FMA step of one lane of a fast block: the coefficient and the ring slot of its
// dependency, kept as two arrays (T and 16-bit slot; a ring of at most 32,766 rows plus the zero
// and dummy slots) in the area of the compacted coefficients
__host__ __device__ inline int fast_rec_capacity(int vb, const RunGeom& g) {
    const int64_t bytes = (int64_t)g.stage_entries * (vb + 4) - 16;
    return bytes > 0 ? (int)(bytes / (vb + 2)) : 0;
}

template <typename T>
struct RunSmem {
    T* ring;
    T* bp;
    T* cval;
    int32_t* cslot;
    T* rcv;           // fast blocks: record coefficients (aliases cval / cslot)
    uint16_t* rslot;  //   and record ring slots
    int32_t* cptr;
    int32_t* row;
    int32_t* lp;
    RunGeom g;
    int zero_slot;    // ring slot (row) whose nrhs values are always 0
    int dummy_slot;   // ring slot (row) that idle lanes write
    // buffer 0 or 1 of the staging area; the ring is shared
    __device__ void carve(unsigned char* base, int nrhs, RunGeom geo, int buf = 0) {
        g = geo;
        ring = (T*)base;
        zero_slot = g.ring_rows;
        dummy_slot = g.ring_rows + 1;
        const size_t vb = sizeof(T);
        const size_t stage = ((size_t)g.stage_rows * nrhs * vb + (size_t)g.stage_entries * (vb + 4) +
                              (size_t)(3 * g.stage_rows + 2) * 4 + 15) / 16 * 16;
        bp = (T*)(base + ((size_t)g.ring_rows * nrhs + RING_PAD) * vb + buf * stage);
        cval = bp + (size_t)g.stage_rows * nrhs;
        cslot = (int32_t*)(cval + g.stage_entries);
        rcv = (T*)(((uintptr_t)cval + 15) & ~(uintptr_t)15);
        rslot = (uint16_t*)(rcv + fast_rec_capacity((int)vb, g));
        cptr = cslot + g.stage_entries;
        row = cptr + g.stage_rows + 1;
        lp = row + g.stage_rows;
    }
};

// A block is a range of positions [P0, P1) covering nl consecutive levels from l0 (the
// first and last of them possibly in part: the rows of one level are independent, so a
// level too large for the staging area is split over consecutive blocks; fast blocks hold
// whole levels).  int4 {P0, P1, l0, nl | flags}
constexpr int BLK_NARROW = 1 << 30;   // every level of the block fits 32 lanes
constexpr int BLK_FAST = 1 << 29;     // fast block (narrow, one right-hand side, records)
constexpr int BLK_K_SHIFT = 26;       // FMA steps per lane and level of a fast block, 1..K_MAX
constexpr int BLK_NL_MASK = (1 << 26) - 1;
constexpr int K_MAX = 4;

// stage A: rows, level pointers (relative to P0) and the b-part; thread per row
// a group of threads that stages a block: all threads of the CTA (barrier 0) or the
// warps after warp 0 (named barrier 1) while warp 0 computes the previous block
struct Grp {
    int tid, nthr, bar;
    __device__ void sync() const {
        if (bar == 0) __syncthreads();
        else asm volatile("bar.sync 1, %0;" ::"r"(nthr) : "memory");
    }
};

__device__ __forceinline__ Grp grp_all() { return Grp{(int)threadIdx.x, (int)blockDim.x, 0}; }
__device__ __forceinline__ Grp grp_stagers() { return Grp{(int)threadIdx.x - 32, (int)blockDim.x - 32, 1}; }

template <typename T>
__device__ void run_stage_a(const SysView<T>& v, RunSmem<T>& sm, int l0, int nl, int64_t P0, int64_t P1,
                            const Grp& G) {
    const int nrhs = v.nrhs;
    const int rows = (int)(P1 - P0);
    for (int li = G.tid; li <= nl; li += G.nthr) {
        int64_t q = li == nl ? P1 : (int64_t)v.lptr[l0 + li];
        q = q < P0 ? P0 : (q > P1 ? P1 : q);
        sm.lp[li] = (int32_t)(q - P0);
    }
    // a thread per (row, right-hand side): b-part t = i * nrhs + k
    for (int t = G.tid; t < rows * nrhs; t += G.nthr) {
        const int i = t / nrhs, k = t - i * nrhs;
        const int64_t p = P0 + i;
        const int32_t row = v.perm[p];
        if (k == 0) sm.row[i] = row;
        sm.bp[t] = v.bpre ? __ldcg(v.bpre + p * nrhs + k) : bpart_full(v, p, row, k);
    }
}

// stage B: fold coefficients of dependencies older than the ring window into the
// b-part; compact the others with their ring slots.  The folding uses stage A's mapping of
// threads to b-parts (row with one right-hand side, (row, right-hand side) with several), so
// the b-parts need no barrier in between.
template <typename T>
__device__ void run_stage_b_fast(const SysView<T>& v, RunSmem<T>& sm, int64_t P0, int rows, int64_t ring_lo,
                                 const Grp& G, int nl, int K, int lpr) {
    const int mask = sm.g.ring_rows - 1;
    const int nrhs = v.nrhs;
    const int steps = K * lpr;  // records per row
    G.sync();                   // the level pointers and b-parts of stage A, written by other threads
    for (int i = G.tid; i < rows; i += G.nthr) {
        // level of row i: the last li with lp[li] <= i
        int lo = 0, hi = nl - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (sm.lp[mid] <= i) lo = mid;
            else hi = mid - 1;
        }
        const int lb = sm.lp[lo], le = sm.lp[lo + 1];
        const int nlanes = (le - lb) * lpr;
        // records of level lo start at K * lpr * lb; step u of lane (g * lpr + e) at u * nlanes + lane
        const size_t r0 = (size_t)K * lpr * lb + (size_t)(i - lb) * lpr;  // this row's first record
        const int64_t p = P0 + i;
        const int q0 = v.cptr[p], q1 = v.cptr[p + 1];
        // a fast row has at most K * lpr entries: its loads go out QC at a time
        constexpr int QC = 8;
        T bp = sm.bp[(size_t)i * nrhs];
        int j = 0;
        for (int qb = q0; qb < q1; qb += QC) {
            int32_t dd[QC];
            T cc[QC];
#pragma unroll
            for (int u = 0; u < QC; ++u) {
                const bool ok = qb + u < q1;
                dd[u] = ok ? v.ccol[qb + u] : -1;
                cc[u] = ok ? v.cval[qb + u] : T(0);
            }
#pragma unroll
            for (int u = 0; u < QC; ++u) {
                if (qb + u >= q1) break;
                const int32_t d = dd[u];
                if (d >= ring_lo) {
                    if (j < steps) {
                        const size_t e = r0 + (size_t)(j / lpr) * nlanes + (j % lpr);
                        sm.rcv[e] = cc[u];
                        sm.rslot[e] = (uint16_t)(d & mask);
                    }
                    ++j;
                } else {
                    bp -= cc[u] * __ldcg(v.xp + (int64_t)d * nrhs);
                }
            }
        }
        for (; j < steps; ++j) {
            const size_t e = r0 + (size_t)(j / lpr) * nlanes + (j % lpr);
            sm.rcv[e] = T(0);
            sm.rslot[e] = (uint16_t)sm.zero_slot;
        }
        sm.bp[(size_t)i * nrhs] = bp;
    }
    if (nrhs > 1) {
        // the other right-hand sides of the folded dependencies, a thread per (row, right-hand
        // side); the first one (k = 0) was folded above by the thread of the row
        G.sync();
        for (int t = G.tid; t < rows * nrhs; t += G.nthr) {
            const int i = t / nrhs, k = t - i * nrhs;
            if (k == 0) continue;
            const int64_t p = P0 + i;
            const int q0 = v.cptr[p], q1 = v.cptr[p + 1];
            T acc = sm.bp[t];
            for (int q = q0; q < q1; ++q) {
                const int32_t d = v.ccol[q];
                if (d < ring_lo) acc -= v.cval[q] * __ldcg(v.xp + (int64_t)d * nrhs + k);
            }
            sm.bp[t] = acc;
        }
    }
    G.sync();
}

template <typename T>
__device__ void run_stage_b(const SysView<T>& v, RunSmem<T>& sm, int64_t P0, int rows, int64_t ring_lo,
                            const Grp& G, int nl, int blk_flags, int lpr) {
    if (blk_flags & BLK_FAST) {
        run_stage_b_fast(v, sm, P0, rows, ring_lo, G, nl, (blk_flags >> BLK_K_SHIFT) & 7, lpr);
        return;
    }
    const int nrhs = v.nrhs;
    const int mask = sm.g.ring_rows - 1;
    if (nrhs == 1) {
        for (int i = G.tid; i < rows; i += G.nthr) {
            const int64_t p = P0 + i;
            const int q0 = v.cptr[p], q1 = v.cptr[p + 1];
            int near = 0;
            for (int q = q0; q < q1; ++q) {
                const int32_t d = v.ccol[q];
                if (d >= ring_lo) ++near;
                else sm.bp[i] -= v.cval[q] * __ldcg(v.xp + d);
            }
            sm.cptr[i + 1] = near;
        }
    } else {
        // near counts a thread per row; the folding a thread per (row, right-hand side), the
        // mapping of stage A, so that neighbouring lanes read neighbouring values of x
        for (int i = G.tid; i < rows; i += G.nthr) {
            const int64_t p = P0 + i;
            const int q0 = v.cptr[p], q1 = v.cptr[p + 1];
            int near = 0;
            for (int q = q0; q < q1; ++q) near += v.ccol[q] >= ring_lo;
            sm.cptr[i + 1] = near;
        }
        for (int t = G.tid; t < rows * nrhs; t += G.nthr) {
            const int i = t / nrhs, k = t - i * nrhs;
            const int64_t p = P0 + i;
            const int q0 = v.cptr[p], q1 = v.cptr[p + 1];
            T acc = sm.bp[t];
            for (int q = q0; q < q1; ++q) {
                const int32_t d = v.ccol[q];
                if (d < ring_lo) acc -= v.cval[q] * __ldcg(v.xp + (int64_t)d * nrhs + k);
            }
            sm.bp[t] = acc;
        }
    }
    G.sync();
    // inclusive scan of the near counts by the group's first warp
    if (G.tid < 32) {
        const int lane = G.tid;
        int carry = 0;
        for (int base = 0; base < rows; base += 32) {
            const int i = base + lane;
            int x = i < rows ? sm.cptr[i + 1] : 0;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                int y = __shfl_up_sync(0xffffffffu, x, o);
                if (lane >= o) x += y;
            }
            if (i < rows) sm.cptr[i + 1] = x + carry;
            carry += __shfl_sync(0xffffffffu, x, 31);
        }
        if (lane == 0) sm.cptr[0] = 0;
    }
    G.sync();
    for (int i = G.tid; i < rows; i += G.nthr) {
        const int64_t p = P0 + i;
        const int q0 = v.cptr[p], q1 = v.cptr[p + 1];
        int o = sm.cptr[i];
        for (int q = q0; q < q1; ++q) {
            const int32_t d = v.ccol[q];
            if (d >= ring_lo) {
                sm.cslot[o] = d & mask;
                sm.cval[o] = v.cval[q];
                ++o;
            }
        }
    }
    G.sync();
}

// Fast block compute, warp 0.  Lane ((g * R2 + k) * LPR + e) of a level takes row g of the
// level, right-hand side k (R2: nrhs rounded up to a power of two) and the row's FMA steps
// e, e + LPR, ...: K records (shared by the row's right-hand sides), its row's b-part on e = 0,
// the ring load of each dependency, K float64 FMAs, log2(LPR) shuffle adds, one store.  The
// records of level li + 1 are loaded while level li computes (two register sets, alternating),
// and the level pointers two levels ahead.
template <typename T, int K, int RPL>
struct FastOps {
    int slot[K];  // ring slot (row) of each step's dependency
    T cv[K];
    T bp[RPL];
    int out[RPL];  // ring elements the lane writes
};

struct FastLane {
    int g, k, e, nrhs;  // row in the level, first right-hand side, coefficient lane, right-hand sides
};

// MR: several right-hand sides, RPL of them per lane (lane = (g * r2 / RPL + k / RPL) * LPR + e);
// otherwise one (lane = g * LPR + e)
template <typename T, int LPR, int K, bool MR, int RPL>
__device__ __forceinline__ void fast_load(const RunSmem<T>& sm, const FastLane& fl, int64_t P0, int mask, int lb,
                                          int le, FastOps<T, K, RPL>& o) {
    const int nr = MR ? fl.nrhs : 1;
    const int rows = le - lb;
    const int nrec = rows * LPR;  // record lanes of the level (one per row and coefficient lane)
    const bool act = fl.g < rows && (!MR || fl.k < fl.nrhs);
    const size_t r0 = (size_t)K * LPR * lb + fl.g * LPR + fl.e;
#pragma unroll
    for (int u = 0; u < K; ++u) {
        if (act) {
            o.slot[u] = sm.rslot[r0 + u * nrec];
            o.cv[u] = sm.rcv[r0 + u * nrec];
        } else {
            o.slot[u] = sm.zero_slot;
            o.cv[u] = T(0);
        }
    }
    const int i = lb + fl.g;
    const bool head = act && fl.e == 0;
#pragma unroll
    for (int j = 0; j < RPL; ++j) {
        const int k = MR ? fl.k + j : 0;
        const bool hj = head && k < nr;
        o.bp[j] = hj ? sm.bp[(size_t)i * nr + k] : T(0);
        o.out[j] = hj ? (int)((P0 + i) & mask) * nr + k : sm.dummy_slot * nr + j;
    }
}

template <typename T, int LPR, int K, bool MR, int RPL>
__device__ __forceinline__ void fast_level(RunSmem<T>& sm, const FastLane& fl, const FastOps<T, K, RPL>& o) {
    const int nr = MR ? fl.nrhs : 1;
    T acc[RPL];
#pragma unroll
    for (int j = 0; j < RPL; ++j) {
        // a right-hand side past nrhs reads the zero slot's values (its k stays below 32)
        const int k = MR ? min(fl.k + j, fl.nrhs - 1) : 0;
        T xv[K];
#pragma unroll
        for (int u = 0; u < K; ++u) xv[u] = sm.ring[o.slot[u] * nr + k];
        acc[j] = o.bp[j];
#pragma unroll
        for (int u = 0; u < K; ++u) acc[j] -= o.cv[u] * xv[u];
    }
#pragma unroll
    for (int j = 0; j < RPL; ++j) {
#pragma unroll
        for (int sh = 1; sh < LPR; sh <<= 1) acc[j] += __shfl_xor_sync(0xffffffffu, acc[j], sh);
        sm.ring[o.out[j]] = acc[j];
    }
    __syncwarp();
}

template <typename T, int LPR, int K, bool MR, int RPL>
__device__ void run_compute_fast(RunSmem<T>& sm, int nrhs, int64_t P0, int l0, int nl, unsigned long long* stamps) {
    if (threadIdx.x >= 32) return;
    const int mask = sm.g.ring_rows - 1;
    FastLane fl;
    fl.nrhs = nrhs;
    int r2 = 1;
    if (MR)
        while (r2 < nrhs) r2 <<= 1;
    const int kl = MR ? r2 / RPL : 1;  // lanes of a row's right-hand sides
    fl.e = (int)threadIdx.x & (LPR - 1);
    fl.k = MR ? (((int)threadIdx.x / LPR) % kl) * RPL : 0;
    fl.g = (int)threadIdx.x / (LPR * kl);
    auto lpb = [&](int li) { return li < nl ? sm.lp[li] : 0; };
    auto lpe = [&](int li) { return li < nl ? sm.lp[li + 1] : 0; };
    FastOps<T, K, RPL> oa, ob;
    int b1 = lpb(1), e1 = lpe(1), b2 = lpb(2), e2 = lpe(2);
    fast_load<T, LPR, K, MR, RPL>(sm, fl, P0, mask, lpb(0), lpe(0), oa);
    for (int li = 0; li < nl; li += 2) {
        const int b3 = lpb(li + 3), e3 = lpe(li + 3);
        fast_load<T, LPR, K, MR, RPL>(sm, fl, P0, mask, b1, e1, ob);
        fast_level<T, LPR, K, MR, RPL>(sm, fl, oa);
        if (stamps && threadIdx.x == 0) stamps[l0 + li] = globaltimer();
        if (li + 1 >= nl) break;
        const int b4 = lpb(li + 4), e4 = lpe(li + 4);
        fast_load<T, LPR, K, MR, RPL>(sm, fl, P0, mask, b2, e2, oa);
        fast_level<T, LPR, K, MR, RPL>(sm, fl, ob);
        if (stamps && threadIdx.x == 0) stamps[l0 + li + 1] = globaltimer();
        b1 = b3; e1 = e3; b2 = b4; e2 = e4;
    }
}

template <typename T, int LPR, bool MR, int RPL>
__device__ void run_compute_fast_k(RunSmem<T>& sm, int nrhs, int K, int64_t P0, int l0, int nl,
                                   unsigned long long* stamps) {
    switch (K) {
        case 1: run_compute_fast<T, LPR, 1, MR, RPL>(sm, nrhs, P0, l0, nl, stamps); break;
        case 2: run_compute_fast<T, LPR, 2, MR, RPL>(sm, nrhs, P0, l0, nl, stamps); break;
        case 3: run_compute_fast<T, LPR, 3, MR, RPL>(sm, nrhs, P0, l0, nl, stamps); break;
        default: run_compute_fast<T, LPR, 4, MR, RPL>(sm, nrhs, P0, l0, nl, stamps); break;
    }
}

// right-hand sides per lane of a fast block: one up to 16, two above
__host__ __device__ inline int fast_rhs_per_lane(int nrhs) { return nrhs > 16 ? 2 : 1; }

template <typename T>
__device__ void run_compute_fast_any(RunSmem<T>& sm, int lpr, int nrhs, int K, int64_t P0, int l0, int nl,
                                     unsigned long long* stamps) {
    if (nrhs == 1) {
        if (lpr == 1) run_compute_fast_k<T, 1, false, 1>(sm, 1, K, P0, l0, nl, stamps);
        else if (lpr == 2) run_compute_fast_k<T, 2, false, 1>(sm, 1, K, P0, l0, nl, stamps);
        else run_compute_fast_k<T, 4, false, 1>(sm, 1, K, P0, l0, nl, stamps);
    } else if (fast_rhs_per_lane(nrhs) == 1) {
        if (lpr == 1) run_compute_fast_k<T, 1, true, 1>(sm, nrhs, K, P0, l0, nl, stamps);
        else run_compute_fast_k<T, 2, true, 1>(sm, nrhs, K, P0, l0, nl, stamps);
    } else {
        if (lpr == 1) run_compute_fast_k<T, 1, true, 2>(sm, nrhs, K, P0, l0, nl, stamps);
        else run_compute_fast_k<T, 2, true, 2>(sm, nrhs, K, P0, l0, nl, stamps);
    }
}

// the level loop of one staged block; narrow blocks run on warp 0 alone
template <typename T>
__device__ void run_compute(const SysView<T>& v, RunSmem<T>& sm, const Lanes& ln, bool narrow, int64_t P0, int l0,
                            int nl, unsigned long long* stamps) {
    if (narrow && threadIdx.x >= 32) return;
    const int nrhs = v.nrhs;
    const int mask = sm.g.ring_rows - 1;
    const int ng = (narrow ? 32 : (int)blockDim.x) / ln.lpr;
    const int grp = threadIdx.x / ln.lpr;
    for (int li = 0; li < nl; ++li) {
        const int lb = sm.lp[li], le = sm.lp[li + 1];
        for (int base = lb; base < le; base += ng) {
            const int i = base + grp;
            const bool act = i < le;
            const int c0 = act ? sm.cptr[i] : 0, c1 = act ? sm.cptr[i + 1] : 0;
            const int slot = (int)((P0 + i) & mask);
            for (int j = 0; j < ln.chunks; ++j) {
                const int k = ln.rl + j * ln.RL;
                const bool kv = act && k < nrhs;
                T acc = T(0);
                if (kv) {
                    if (ln.el == 0) acc = sm.bp[(size_t)i * nrhs + k];
                    for (int q = c0 + ln.el; q < c1; q += ln.EL) acc -= sm.cval[q] * sm.ring[(size_t)sm.cslot[q] * nrhs + k];
                }
                acc = group_reduce(acc, ln);
                if (kv && ln.el == 0) sm.ring[(size_t)slot * nrhs + k] = acc;
            }
        }
        if (narrow) __syncwarp();
        else __syncthreads();
        if (stamps && threadIdx.x == 0) stamps[l0 + li] = globaltimer();
    }
}

// x of the block leaves the ring: coalesced into xp, scattered into the caller's x
template <typename T>
__device__ void run_write_out(const SysView<T>& v, const RunSmem<T>& sm, int64_t P0, int rows, const Grp& G) {
    const int nrhs = v.nrhs;
    const int mask = sm.g.ring_rows - 1;
    const int total = rows * nrhs;
    for (int t = G.tid; t < total; t += G.nthr) {
        const int i = t / nrhs, k = t - i * nrhs;
        const T val = sm.ring[(size_t)((P0 + i) & mask) * nrhs + k];
        __stcg(v.xp + (P0 + i) * nrhs + k, val);
        v.x[(int64_t)sm.row[i] + (int64_t)k * v.ld] = val;
    }
}

// Runs blocks [blk0, blk1).  `wait` is called once, after the first block's stage A.
// Iteration of block i (buffer i % 2): compute block i; meanwhile -- when block i is a fast
// block, on warps 1.. while warp 0 computes; otherwise on all threads, before and after the
// compute -- write block i-1's x out of the ring and stage block i+1 into the other buffer.
// Stage B of block i+1 reads from xp only x older than the ring window, which lies in
// blocks <= i-1 (two blocks fit the ring), written out just before.
// The stored arrays of a run of blocks are contiguous (positions [Pa, Pb), coefficients
// [cptr[Pa], cptr[Pb])): one bulk L2 prefetch per array as the run starts, each capped, so that
// staging reads L2 instead of DRAM.  Runs of one block skip it.
constexpr int64_t RUN_PREFETCH_CAP = 24ll << 20;  // bytes per array

template <typename T>
__device__ void prefetch_run(const SysView<T>& v, int64_t Pa, int64_t Pb) {
    auto cap = [](int64_t b) { return b < RUN_PREFETCH_CAP ? b : RUN_PREFETCH_CAP; };
    const int64_t qa = v.cptr[Pa], qb = v.cptr[Pb];
    l2_prefetch(v.perm + Pa, cap((Pb - Pa) * 4));
    l2_prefetch(v.cptr + Pa, cap((Pb - Pa + 1) * 4));
    l2_prefetch(v.ccol + qa, cap((qb - qa) * 4));
    l2_prefetch(v.cval + qa, cap((qb - qa) * (int64_t)sizeof(T)));
    if (v.bpre) {
        l2_prefetch(v.bpre + Pa * v.nrhs, cap((Pb - Pa) * v.nrhs * (int64_t)sizeof(T)));
    } else {
        l2_prefetch(v.dinv + Pa, cap((Pb - Pa) * (int64_t)sizeof(T)));
        if (v.eptr) {
            const int64_t ea = v.eptr[Pa], eb = v.eptr[Pb];
            l2_prefetch(v.eptr + Pa, cap((Pb - Pa + 1) * 4));
            l2_prefetch(v.ecol + ea, cap((eb - ea) * 4));
            l2_prefetch(v.eval + ea, cap((eb - ea) * (int64_t)sizeof(T)));
        }
    }
}

template <typename T, typename WaitFn>
__device__ bool run_blocks(const SysView<T>& v, unsigned char* smem, RunGeom geo, const Lanes& ln, const int4* blocks,
                           int blk0, int blk1, WaitFn wait, unsigned long long* stamps) {
    if (blk0 >= blk1) return wait();
    const int64_t run_p0 = blocks[blk0].x;
    const int R = geo.ring_rows;
    if (blk1 - blk0 > 1) prefetch_run(v, run_p0, (int64_t)blocks[blk1 - 1].y);
    {
        RunSmem<T> s0;
        s0.carve(smem, v.nrhs, geo, 0);
        if (threadIdx.x < RING_PAD) s0.ring[(size_t)s0.zero_slot * v.nrhs + threadIdx.x] = T(0);
        const int4 bd = blocks[blk0];
        __syncthreads();
        run_stage_a(v, s0, bd.z, bd.w & BLK_NL_MASK, bd.x, bd.y, grp_all());
        if (!wait()) return false;
        run_stage_b(v, s0, bd.x, bd.y - bd.x, max(run_p0, (int64_t)bd.y - R), grp_all(), bd.w & BLK_NL_MASK, bd.w,
                    ln.lpr);
    }
    for (int blk = blk0; blk < blk1; ++blk) {
        const int par = (blk - blk0) & 1;
        RunSmem<T> cur, oth;
        cur.carve(smem, v.nrhs, geo, par);
        oth.carve(smem, v.nrhs, geo, par ^ 1);
        const int4 bd = blocks[blk];
        const int64_t P0 = bd.x;
        const int nl = bd.w & BLK_NL_MASK;
        const bool narrow = (bd.w & BLK_NARROW) != 0;
        const bool fast = (bd.w & BLK_FAST) != 0;
        const bool prev = blk > blk0;
        const bool next = blk + 1 < blk1;
        const bool overlap = fast && blockDim.x > 32 && (prev || next);
        if (overlap) {
            if (threadIdx.x < 32) {
                run_compute_fast_any(cur, ln.lpr, v.nrhs, (bd.w >> BLK_K_SHIFT) & 7, P0, bd.z, nl, stamps);
            } else {
                const Grp G = grp_stagers();
                if (prev) {
                    const int4 bp = blocks[blk - 1];
                    run_write_out(v, oth, bp.x, (int)(bp.y - bp.x), G);
                    G.sync();
                }
                if (next) {
                    const int4 bn = blocks[blk + 1];
                    run_stage_a(v, oth, bn.z, bn.w & BLK_NL_MASK, bn.x, bn.y, G);
                    run_stage_b(v, oth, bn.x, bn.y - bn.x, max(run_p0, (int64_t)bn.y - R), G, bn.w & BLK_NL_MASK,
                                bn.w, ln.lpr);
                }
            }
        } else {
            if (prev) {
                const int4 bp = blocks[blk - 1];
                run_write_out(v, oth, bp.x, (int)(bp.y - bp.x), grp_all());
            }
            if (fast) {
                if (threadIdx.x < 32)
                    run_compute_fast_any(cur, ln.lpr, v.nrhs, (bd.w >> BLK_K_SHIFT) & 7, P0, bd.z, nl, stamps);
            } else {
                run_compute(v, cur, ln, narrow, P0, bd.z, nl, stamps);
            }
            __syncthreads();
            if (next) {
                const int4 bn = blocks[blk + 1];
                run_stage_a(v, oth, bn.z, bn.w & BLK_NL_MASK, bn.x, bn.y, grp_all());
                run_stage_b(v, oth, bn.x, bn.y - bn.x, max(run_p0, (int64_t)bn.y - R), grp_all(), bn.w & BLK_NL_MASK,
                            bn.w, ln.lpr);
            }
        }
        __syncthreads();
    }
    {
        RunSmem<T> last;
        last.carve(smem, v.nrhs, geo, (blk1 - 1 - blk0) & 1);
        const int4 bl = blocks[blk1 - 1];
        run_write_out(v, last, bl.x, (int)(bl.y - bl.x), grp_all());
        __syncthreads();
    }
    return true;
}

// host: cuts levels [l_begin, l_end) into staged blocks; levels that qualify (lpr 1, 2 or 4 for
// one right-hand side, 1 or 2 for several; rows x lpr x nrhs rounded up to a power of two /
// right-hand sides per lane at most 32 lanes; at most K_MAX FMA steps per lane) go to fast
// blocks of at most fast_recs records (0: no fast blocks)
int build_run_blocks(const int32_t* lp, const int32_t* cptr, int64_t l_begin, int64_t l_end, int stage_rows,
                     int stage_entries, int lpr, int nrhs, int fast_recs, std::vector<int4>& out);

}  // namespace sp
