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
//           b-part right away; the others are compacted with their ring slot;
//   compute: per level, rows read x only from the shared-memory ring;
//   write-out: the block's x leaves the ring once, coalesced.
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

inline size_t run_stage_bytes(int vb, int nrhs, const RunGeom& g) {
    return (size_t)g.stage_rows * nrhs * vb + (size_t)g.stage_entries * (vb + 4) + (size_t)(3 * g.stage_rows + 2) * 4;
}

// the x ring plus two staging buffers (one is filled while the other is computed)
inline size_t run_smem_bytes(int vb, int nrhs, const RunGeom& g) {
    return (size_t)g.ring_rows * nrhs * vb + 2 * ((run_stage_bytes(vb, nrhs, g) + 15) / 16 * 16);
}

template <typename T>
struct RunSmem {
    T* ring;
    T* bp;
    T* cval;
    int32_t* cslot;
    int32_t* cptr;
    int32_t* row;
    int32_t* lp;
    RunGeom g;
    // buffer 0 or 1 of the staging area; the ring is shared
    __device__ void carve(unsigned char* base, int nrhs, RunGeom geo, int buf = 0) {
        g = geo;
        ring = (T*)base;
        const size_t vb = sizeof(T);
        const size_t stage = ((size_t)g.stage_rows * nrhs * vb + (size_t)g.stage_entries * (vb + 4) +
                              (size_t)(3 * g.stage_rows + 2) * 4 + 15) / 16 * 16;
        bp = (T*)(base + (size_t)g.ring_rows * nrhs * vb + buf * stage);
        cval = bp + (size_t)g.stage_rows * nrhs;
        cslot = (int32_t*)(cval + g.stage_entries);
        cptr = cslot + g.stage_entries;
        row = cptr + g.stage_rows + 1;
        lp = row + g.stage_rows;
    }
};

// A block is a range of positions [P0, P1) covering nl consecutive levels from l0 (the
// first and last of them possibly in part: the rows of one level are independent, so a
// level too large for the staging area is split over consecutive blocks).
// int4 {P0, P1, l0, nl | narrow << 30}
constexpr int BLK_NARROW = 1 << 30;

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
    for (int i = G.tid; i < rows; i += G.nthr) {
        const int64_t p = P0 + i;
        const int32_t row = v.perm[p];
        sm.row[i] = row;
        for (int k = 0; k < nrhs; ++k) sm.bp[(size_t)i * nrhs + k] = bpart_full(v, p, row, k);
    }
}

// stage B: fold coefficients of dependencies older than the ring window into the
// b-part; compact the others with their ring slots.  Same thread-to-row mapping as
// stage A, so the b-part needs no barrier in between.
template <typename T>
__device__ void run_stage_b(const SysView<T>& v, RunSmem<T>& sm, int64_t P0, int rows, int64_t ring_lo,
                            const Grp& G) {
    const int nrhs = v.nrhs;
    const int mask = sm.g.ring_rows - 1;
    for (int i = G.tid; i < rows; i += G.nthr) {
        const int64_t p = P0 + i;
        const int q0 = v.cptr[p], q1 = v.cptr[p + 1];
        int near = 0;
        for (int q = q0; q < q1; ++q) {
            const int32_t d = v.ccol[q];
            if (d >= ring_lo) {
                ++near;
            } else {
                const T c = v.cval[q];
                for (int k = 0; k < nrhs; ++k)
                    sm.bp[(size_t)i * nrhs + k] -= c * __ldcg(v.xp + (int64_t)d * nrhs + k);
            }
        }
        sm.cptr[i + 1] = near;
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

// Narrow block, one right-hand side, LPR lanes per row (LPR = 1, 2 or 4): every lane
// holds up to NK of its row's coefficients (entries el, el+LPR, ...) and their ring slots
// in registers, read for the next level while the current level computes; the lanes of
// a row combine their partial sums with shuffles.  A level costs its ring loads plus
// ceil(deps / LPR) dependent float64 FMAs and log2(LPR) adds.
constexpr int NK = 4;  // coefficients per lane held in registers

template <typename T>
struct RowRegs {
    int i, c0, c1;
    bool act;
    T bp;
    int slot[NK];
};

template <typename T, int LPR>
__device__ __forceinline__ void load_row_regs(const RunSmem<T>& sm, int lb, int le, RowRegs<T>& r) {
    const int el = (int)threadIdx.x & (LPR - 1);
    r.i = lb + (int)threadIdx.x / LPR;
    r.act = r.i < le;
    r.c0 = r.act ? sm.cptr[r.i] : 0;
    r.c1 = r.act ? sm.cptr[r.i + 1] : 0;
    r.bp = (r.act && el == 0) ? sm.bp[r.i] : T(0);
#pragma unroll
    for (int u = 0; u < NK; ++u) {
        const int q = r.c0 + el + u * LPR;
        r.slot[u] = q < r.c1 ? sm.cslot[q] : 0;
    }
}

template <typename T, int LPR>
__device__ void run_compute_narrow(RunSmem<T>& sm, int64_t P0, int l0, int nl, unsigned long long* stamps) {
    if (threadIdx.x >= 32) return;
    const int mask = sm.g.ring_rows - 1;
    const int el = (int)threadIdx.x & (LPR - 1);
    RowRegs<T> cur, nxt;
    load_row_regs<T, LPR>(sm, sm.lp[0], sm.lp[1], cur);
    for (int li = 0; li < nl; ++li) {
        if (li + 1 < nl) load_row_regs<T, LPR>(sm, sm.lp[li + 1], sm.lp[li + 2], nxt);
        T acc = cur.bp;
        if (cur.act) {
            T xv[NK], cv[NK];
#pragma unroll
            for (int u = 0; u < NK; ++u) {
                const int q = cur.c0 + el + u * LPR;
                xv[u] = sm.ring[cur.slot[u]];
                cv[u] = q < cur.c1 ? sm.cval[q] : T(0);
            }
#pragma unroll
            for (int u = 0; u < NK; ++u)
                if (cur.c0 + el + u * LPR < cur.c1) acc -= cv[u] * xv[u];
            for (int q = cur.c0 + el + NK * LPR; q < cur.c1; q += LPR) acc -= sm.cval[q] * sm.ring[sm.cslot[q]];
        }
#pragma unroll
        for (int o = 1; o < LPR; o <<= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        if (cur.act && el == 0) sm.ring[(int)((P0 + cur.i) & mask)] = acc;
        __syncwarp();
        if (stamps && threadIdx.x == 0) stamps[l0 + li] = globaltimer();
        cur = nxt;
    }
}

template <typename T>
__device__ __forceinline__ bool narrow_fast(const Lanes& ln, int nrhs) {
    return nrhs == 1 && (ln.lpr == 1 || ln.lpr == 2 || ln.lpr == 4);
}

template <typename T>
__device__ void run_compute_narrow_any(RunSmem<T>& sm, const Lanes& ln, int64_t P0, int l0, int nl,
                                       unsigned long long* stamps) {
    if (ln.lpr == 1) run_compute_narrow<T, 1>(sm, P0, l0, nl, stamps);
    else if (ln.lpr == 2) run_compute_narrow<T, 2>(sm, P0, l0, nl, stamps);
    else run_compute_narrow<T, 4>(sm, P0, l0, nl, stamps);
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
__device__ void run_write_out(const SysView<T>& v, RunSmem<T>& sm, int64_t P0, int rows) {
    const int nrhs = v.nrhs;
    const int mask = sm.g.ring_rows - 1;
    const int total = rows * nrhs;
    for (int t = threadIdx.x; t < total; t += blockDim.x) {
        const int i = t / nrhs, k = t - i * nrhs;
        const T val = sm.ring[(size_t)((P0 + i) & mask) * nrhs + k];
        __stcg(v.xp + (P0 + i) * nrhs + k, val);
        v.x[(int64_t)sm.row[i] + (int64_t)k * v.ld] = val;
    }
}

// Runs blocks [blk0, blk1).  `wait` is called once, after the first block's stage A.
// Iteration of block i: compute block i (buffer i % 2) while -- when block i is narrow and
// single-RHS -- warps 1.. stage block i+1 into the other buffer; then every thread writes
// block i's x out of the ring.  Block i+1's stage B reads x only of blocks <= i-1 (a
// dependency inside block i is always inside the ring window), which iteration i-1
// wrote out.
template <typename T, typename WaitFn>
__device__ bool run_blocks(const SysView<T>& v, unsigned char* smem, RunGeom geo, const Lanes& ln, const int4* blocks,
                           int blk0, int blk1, WaitFn wait, unsigned long long* stamps) {
    if (blk0 >= blk1) return wait();
    const int64_t run_p0 = blocks[blk0].x;
    const int R = geo.ring_rows;
    {
        RunSmem<T> s0;
        s0.carve(smem, v.nrhs, geo, 0);
        const int4 bd = blocks[blk0];
        __syncthreads();
        run_stage_a(v, s0, bd.z, bd.w & (BLK_NARROW - 1), bd.x, bd.y, grp_all());
        if (!wait()) return false;
        run_stage_b(v, s0, bd.x, bd.y - bd.x, max(run_p0, (int64_t)bd.y - R), grp_all());
    }
    for (int blk = blk0; blk < blk1; ++blk) {
        const int par = (blk - blk0) & 1;
        RunSmem<T> cur;
        cur.carve(smem, v.nrhs, geo, par);
        const int4 bd = blocks[blk];
        const int64_t P0 = bd.x;
        const int nl = bd.w & (BLK_NARROW - 1);
        const bool narrow = (bd.w & BLK_NARROW) != 0;
        const bool next = blk + 1 < blk1;
        const bool fast = narrow && narrow_fast<T>(ln, v.nrhs);
        const bool overlap = fast && next && blockDim.x > 32;
        if (!overlap || threadIdx.x < 32) {
            if (fast) run_compute_narrow_any(cur, ln, P0, bd.z, nl, stamps);
            else run_compute(v, cur, ln, narrow, P0, bd.z, nl, stamps);
        }
        if (!overlap) __syncthreads();
        if (next && (!overlap || threadIdx.x >= 32)) {
            // stage the next block into the other buffer
            RunSmem<T> nx;
            nx.carve(smem, v.nrhs, geo, par ^ 1);
            const int4 bn = blocks[blk + 1];
            const Grp G = overlap ? grp_stagers() : grp_all();
            run_stage_a(v, nx, bn.z, bn.w & (BLK_NARROW - 1), bn.x, bn.y, G);
            run_stage_b(v, nx, bn.x, bn.y - bn.x, max(run_p0, (int64_t)bn.y - R), G);
        }
        if (overlap) __syncthreads();
        run_write_out(v, cur, P0, (int)(bd.y - bd.x));
        __syncthreads();
    }
    return true;
}

// host: cuts levels [l_begin, l_end) into staged blocks
int build_run_blocks(const int32_t* lp, const int32_t* cptr, int64_t l_begin, int64_t l_end, int stage_rows,
                     int stage_entries, int lpr, std::vector<int4>& out);

}  // namespace sp
