// rewrite.cu -- equation rewriting (Section II.B, Fig. 2) and its planners (Section III).
//
// Planning decides the level each row moves to (its target):
//   * a single-warp walk over the levels in order for the naive avgLevelCost strategy
//     and for any strategy under an nnz cap.  Inside a source level the 32 lanes cost up
//     to 32 candidate rows in parallel (the symbolic union of the substituted
//     dependencies), then one greedy prefix in ascending row order decides which rows
//     move: the paper's "threads compute costs, one thread inserts" (Section III);
//   * a parallel map level -> target for fixed depths without a cap.
// Rewriting then runs in rounds of depth d = level - target: every row of depth d only
// substitutes rows of smaller depth in its group, so all rows of one depth are rewritten
// in parallel.  A rewritten row is assembled from its own entries and the current
// equations of its substituted dependencies, sorted by column (stable), and rearranged
// by one division by its diagonal.  The arithmetic is written with explicit
// round-to-nearest operations in the same order as the serial oracle, so the stored
// coefficients are reproducible bit for bit in float64.
#include <algorithm>
#include <cmath>

#include "system.cuh"

namespace sp {

// kinds of the walk
// CHOSEN_THIN: the learned strategy's plan -- thin levels only (Section III), each target
// taking its own number of following levels.  ROWCAP: the NAIVE walk with the number of rows on
// the target (at most k) in place of avgLevelCost -- a level of the fast executor holds at
// most 32 lanes, so the cap shapes the plan for it
enum { WALK_NAIVE = 1, WALK_DEPTH = 2, WALK_CHOSEN = 3, WALK_MANUAL = 4, WALK_CHOSEN_THIN = 5, WALK_ROWCAP = 6 };

namespace {

inline unsigned nblk(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

__device__ __forceinline__ int64_t warp_incl_scan(int64_t v) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int64_t y = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += y;
    }
    return v;
}

// in-place heap sort of an int32 range (rows of the planner can hold thousands of entries)
__device__ void heap_sort_i32(int32_t* a, int n) {
    auto sift = [&](int root, int end) {
        while (true) {
            int child = 2 * root + 1;
            if (child >= end) break;
            if (child + 1 < end && a[child] < a[child + 1]) ++child;
            if (a[root] >= a[child]) break;
            int32_t t = a[root];
            a[root] = a[child];
            a[child] = t;
            root = child;
        }
    };
    for (int i = n / 2 - 1; i >= 0; --i) sift(i, n);
    for (int end = n - 1; end > 0; --end) {
        int32_t t = a[0];
        a[0] = a[end];
        a[end] = t;
        sift(0, end);
    }
}

// sort + unique of an int32 range in global memory; returns the new length
__device__ int sort_unique(int32_t* a, int len) {
    if (len <= 32) {
        for (int i = 1; i < len; ++i) {
            int32_t v = a[i];
            int j = i - 1;
            while (j >= 0 && a[j] > v) {
                a[j + 1] = a[j];
                --j;
            }
            a[j + 1] = v;
        }
    } else {
        heap_sort_i32(a, len);
    }
    int w = 0;
    for (int i = 0; i < len; ++i)
        if (w == 0 || a[w - 1] != a[i]) a[w++] = a[i];
    return w;
}

// entries of one candidate set the warp sorts together in shared memory
constexpr int WALK_SORT_CAP = 512;

// The warp sorts and de-duplicates len <= WALK_SORT_CAP values in shared memory sv[0, len) together:
// each lane ranks its entries against all the others -- an entry is kept when no earlier entry has its
// value, and goes to the place given by the number of distinct smaller values -- and the sorted
// distinct values go to dst (global memory).  Returns the new length on every lane.  Called by the
// whole warp.
__device__ int warp_sort_unique_smem(const int32_t* sv, int len, int32_t* sk, int32_t* dst) {
    const int lane = threadIdx.x & 31;
    for (int i = lane; i < len; i += 32) {
        const int32_t v = sv[i];
        int dup = 0;
        for (int k = 0; k < i; ++k) dup |= sv[k] == v;
        sk[i] = !dup;
    }
    __syncwarp();
    int kept = 0;
    for (int i = lane; i < len; i += 32) {
        if (!sk[i]) continue;
        const int32_t v = sv[i];
        int pos = 0;
        for (int k = 0; k < len; ++k) pos += (sk[k] && sv[k] < v) ? 1 : 0;
        dst[pos] = v;
        ++kept;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) kept += __shfl_xor_sync(0xffffffffu, kept, o);
    __syncwarp();
    return kept;
}

struct WalkArgs {
    int64_t n, m, nnzL;
    const int32_t* rowptr;
    const int32_t* colidx;
    const int32_t* level;
    const int32_t* lptr;
    const int32_t* lrows;
    const int64_t* lcost;
    int kind, k;
    double avg;
    const int64_t* part_limit;  // per level range: entries its moves may add (INT64_MAX: no cap)
    const int32_t* dot;  // depth of target (CHOSEN)
    const int64_t* inj;  // injected costs (test hook)
    int alpha;           // per-row rules (Section III.A): dependencies after substitution < alpha
    int64_t beta;        //   and max - min dependency < beta (0: off)
    int32_t* target;     // current level of every row (init: level)
    int64_t* row_cost;
    int64_t* d_off;
    int32_t* d_len;
    int64_t* e_off;
    int32_t* e_len;
    int32_t* pool;
    int64_t pool_cap;   // entries of the pool of one level range
    int64_t* info;  // per level range: moved, entries added, targets
    int* status;
};

// One warp walks the levels of one range in order: range w = levels [w*m/P, (w+1)*m/P) of P = gridDim.x
// ranges, from a fresh start (the walk started at several places, Section III; P = 1 is the single
// walk).  A range only rewrites rows of its own levels, and substitution never reaches below a
// target, so it reads nothing another range writes that could change its decisions: a dependency
// in an earlier range sits on a level below the range's targets whatever its own range did.
// Candidate sets of a chunk of at most 4 rows (thin levels: mostly 1 or 2) are gathered and sorted by
// the whole warp, one row after the other (warp_sort_unique_smem); larger chunks take a row per lane.
__global__ void __launch_bounds__(32) k_plan_walk(WalkArgs a) {
    extern __shared__ int32_t walk_smem[];  // 3 x WALK_SORT_CAP: D values, E values, keep flags
    const int lane = threadIdx.x;
    const int w = blockIdx.x, P = gridDim.x;
    const int64_t s_begin = a.m * w / P, s_end = a.m * (w + 1) / P;
    const int64_t limit = a.part_limit[w];
    int32_t* const pool = a.pool + (int64_t)w * a.pool_cap;
    int t = -1;
    int64_t cur = 0, stored = 0, moved = 0, targets = 0, top = 0;
    for (int64_t s = s_begin; s < s_end; ++s) {
        const int64_t ls = a.lcost[s];
        const bool eligible = (a.kind == WALK_NAIVE || a.kind == WALK_MANUAL || a.kind == WALK_CHOSEN_THIN ||
                               a.kind == WALK_ROWCAP)
                                  ? ((double)ls < a.avg)
                                  : true;
        const bool rowcap = a.kind == WALK_ROWCAP;
        if (!eligible) {
            t = -1;
            continue;
        }
        if (t < 0 || ((a.kind == WALK_DEPTH || a.kind == WALK_MANUAL) && s - t > a.k) ||
            ((a.kind == WALK_CHOSEN || a.kind == WALK_CHOSEN_THIN) && s - t > a.dot[t])) {
            t = (int)s;
            cur = rowcap ? (int64_t)(a.lptr[s + 1] - a.lptr[s]) : ls;
            targets++;
            top = 0;
            continue;
        }
        const int64_t A = a.lptr[s], Bn = a.lptr[s + 1];
        for (int64_t base = A; base < Bn; base += 32) {
            const int nvalid = (int)(Bn - base < 32 ? Bn - base : 32);
            const bool coop = nvalid <= 4;  // warp-uniform
            const int64_t idx = base + lane;
            const bool valid = idx < Bn;
            const int32_t r = valid ? a.lrows[idx] : 0;
            const int64_t q0 = valid ? a.rowptr[r] : 0, q1 = valid ? (int64_t)a.rowptr[r + 1] - 1 : 0;
            // upper bounds of the candidate sets
            int64_t ubD = 0, ubE = valid ? 1 : 0;
            for (int64_t q = q0; q < q1; ++q) {
                const int32_t j = a.colidx[q];
                if (a.target[j] >= t) {
                    const bool mj = a.level[j] != t;  // moved into this group earlier
                    ubD += mj ? a.d_len[j] : (a.rowptr[j + 1] - a.rowptr[j] - 1);
                    ubE += mj ? a.e_len[j] : 1;
                } else {
                    ubD += 1;
                }
            }
            const int64_t ub = ubD + ubE;
            const int64_t incl = warp_incl_scan(ub);
            const int64_t off = incl - ub;
            const int64_t total = __shfl_sync(0xffffffffu, incl, 31);
            if (top + total > a.pool_cap) {
                if (lane == 0) atomicCAS(a.status, 0, (int)DEV_OVERFLOW);
                return;
            }
            int32_t* Dp = pool + top + off;
            int32_t* Ep = Dp + ubD;
            int nd = 0, ne = 0;
            if (valid && !coop) {
                for (int64_t q = q0; q < q1; ++q) {
                    const int32_t j = a.colidx[q];
                    if (a.target[j] >= t) {
                        if (a.level[j] != t) {
                            const int64_t o = a.d_off[j];
                            for (int u = 0; u < a.d_len[j]; ++u) Dp[nd++] = pool[o + u];
                            const int64_t oe = a.e_off[j];
                            for (int u = 0; u < a.e_len[j]; ++u) Ep[ne++] = pool[oe + u];
                        } else {
                            for (int64_t u = a.rowptr[j]; u < (int64_t)a.rowptr[j + 1] - 1; ++u) Dp[nd++] = a.colidx[u];
                            Ep[ne++] = j;
                        }
                    } else {
                        Dp[nd++] = j;
                    }
                }
                Ep[ne++] = r;
                nd = sort_unique(Dp, nd);
                ne = sort_unique(Ep, ne);
            }
            if (coop) {
                // rows one after the other, each gathered by the whole warp: dependency by dependency,
                // the same lists in the same order as the lane-per-row concatenation above, into shared
                // memory (sets of at most WALK_SORT_CAP entries; a longer one is gathered by its lane into
                // the pool), then sorted and de-duplicated into the pool
                int32_t* sD = walk_smem;
                int32_t* sE = walk_smem + WALK_SORT_CAP;
                int32_t* sK = walk_smem + 2 * WALK_SORT_CAP;
                for (int L = 0; L < nvalid; ++L) {
                    int32_t* dl = (int32_t*)__shfl_sync(0xffffffffu, (unsigned long long)Dp, L);
                    int32_t* el = (int32_t*)__shfl_sync(0xffffffffu, (unsigned long long)Ep, L);
                    const int32_t rl = __shfl_sync(0xffffffffu, r, L);
                    const int64_t a0 = __shfl_sync(0xffffffffu, q0, L), a1 = __shfl_sync(0xffffffffu, q1, L);
                    const int64_t uD = __shfl_sync(0xffffffffu, ubD, L), uE = __shfl_sync(0xffffffffu, ubE, L);
                    int dn = 0, en = 0;
                    if (uD <= WALK_SORT_CAP && uE <= WALK_SORT_CAP) {
                        for (int64_t q = a0; q < a1; ++q) {
                            const int32_t j = a.colidx[q];
                            if (a.target[j] >= t) {
                                if (a.level[j] != t) {
                                    const int64_t o = a.d_off[j], oe = a.e_off[j];
                                    const int ld = a.d_len[j], le = a.e_len[j];
                                    for (int u = lane; u < ld; u += 32) sD[dn + u] = pool[o + u];
                                    for (int u = lane; u < le; u += 32) sE[en + u] = pool[oe + u];
                                    dn += ld;
                                    en += le;
                                } else {
                                    const int64_t b0 = a.rowptr[j], b1 = (int64_t)a.rowptr[j + 1] - 1;
                                    for (int64_t u = b0 + lane; u < b1; u += 32) sD[dn + (int)(u - b0)] = a.colidx[u];
                                    dn += (int)(b1 - b0);
                                    if (lane == 0) sE[en] = j;
                                    ++en;
                                }
                            } else {
                                if (lane == 0) sD[dn] = j;
                                ++dn;
                            }
                        }
                        if (lane == 0) sE[en] = rl;
                        ++en;
                        __syncwarp();
                        dn = warp_sort_unique_smem(sD, dn, sK, dl);
                        en = warp_sort_unique_smem(sE, en, sK, el);
                    } else {
                        if (lane == L) {
                            for (int64_t q = a0; q < a1; ++q) {
                                const int32_t j = a.colidx[q];
                                if (a.target[j] >= t) {
                                    if (a.level[j] != t) {
                                        const int64_t o = a.d_off[j];
                                        for (int u = 0; u < a.d_len[j]; ++u) dl[dn++] = pool[o + u];
                                        const int64_t oe = a.e_off[j];
                                        for (int u = 0; u < a.e_len[j]; ++u) el[en++] = pool[oe + u];
                                    } else {
                                        for (int64_t u = a.rowptr[j]; u < (int64_t)a.rowptr[j + 1] - 1; ++u)
                                            dl[dn++] = a.colidx[u];
                                        el[en++] = j;
                                    }
                                } else {
                                    dl[dn++] = j;
                                }
                            }
                            el[en++] = rl;
                            dn = sort_unique(dl, dn);
                            en = sort_unique(el, en);
                        }
                        __syncwarp();
                        dn = __shfl_sync(0xffffffffu, dn, L);
                        en = __shfl_sync(0xffffffffu, en, L);
                    }
                    if (lane == L) {
                        nd = dn;
                        ne = en;
                    }
                }
            }
            const int64_t c = valid ? (a.inj ? a.inj[r] : 2 * (int64_t)nd) : 0;
            const int64_t growth = valid ? (int64_t)nd + ne - (q1 - q0) : 0;
            const int64_t pc = warp_incl_scan(rowcap ? (valid ? 1 : 0) : c);
            const int64_t pg = warp_incl_scan(growth);
            bool rules = true;
            if (valid && a.alpha > 0 && nd >= a.alpha) rules = false;
            if (valid && a.beta > 0 && nd > 1 && (int64_t)Dp[nd - 1] - (int64_t)Dp[0] >= a.beta) rules = false;
            // a rule broken by an earlier lane stops the prefix there, like a cost overflow
            const unsigned badrule = __ballot_sync(0xffffffffu, !rules);
            const int first_bad = badrule ? __ffs(badrule) - 1 : 32;
            const bool pass = (a.kind != WALK_NAIVE || (double)(cur + pc) <= a.avg) && (!rowcap || cur + pc <= a.k) &&
                              (limit == INT64_MAX || stored + pg <= limit) && lane < first_bad;
            const unsigned failmask = __ballot_sync(0xffffffffu, valid && !pass);
            const int first = failmask ? __ffs(failmask) - 1 : 32;
            const int acc_n = min(first, nvalid);
            if (lane < acc_n) {
                a.target[r] = t;
                a.row_cost[r] = c;
                a.d_off[r] = top + off;
                a.d_len[r] = nd;
                a.e_off[r] = top + off + ubD;
                a.e_len[r] = ne;
            }
            if (acc_n > 0) {
                cur += __shfl_sync(0xffffffffu, pc, acc_n - 1);
                stored += __shfl_sync(0xffffffffu, pg, acc_n - 1);
                top += __shfl_sync(0xffffffffu, off, acc_n - 1) + __shfl_sync(0xffffffffu, ub, acc_n - 1);
                moved += acc_n;
            }
            __syncwarp();
            if (first < nvalid) {
                // this level becomes the next target with the rows it still holds
                t = (int)s;
                targets++;
                top = 0;
                int64_t rest = 0;
                for (int64_t i2 = A + lane; i2 < Bn; i2 += 32) {
                    const int32_t r2 = a.lrows[i2];
                    if (a.target[r2] == s) rest += rowcap ? 1 : a.row_cost[r2];
                }
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) rest += __shfl_xor_sync(0xffffffffu, rest, o);
                cur = rest;
                break;
            }
        }
        __syncwarp();
    }
    if (lane == 0) {
        a.info[3 * w] = moved;
        a.info[3 * w + 1] = stored;
        a.info[3 * w + 2] = targets;
    }
}

__global__ void k_init_walk(int64_t n, const int32_t* rowptr, const int32_t* level, int32_t* target,
                            int64_t* row_cost) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    target[i] = level[i];
    row_cost[i] = 2 * ((int64_t)rowptr[i + 1] - rowptr[i]) - 1;
}

// fixed depths without a cap: every level maps to its target independently of the rows (over all
// levels for DEPTH and CHOSEN; over thin levels, cost below avgLevelCost, for MANUAL and CHOSEN_THIN,
// where a level that is not thin keeps its rows and ends the group)
__global__ void k_level_targets(int64_t m, int kind, int k, const int32_t* dot, const int64_t* lcost, double avg,
                                int parts, int32_t* ltarget) {
    if (blockIdx.x != 0 || threadIdx.x != 0) return;
    const bool thin_only = kind == WALK_MANUAL || kind == WALK_CHOSEN_THIN;
    const bool by_dot = kind == WALK_CHOSEN || kind == WALK_CHOSEN_THIN;
    int64_t t = -1;
    int w = 0;  // level range (the walk restarts at the first level of every range)
    for (int64_t s = 0; s < m; ++s) {
        while (w + 1 < parts && s == m * (w + 1) / parts) {
            ++w;
            t = -1;
        }
        if (thin_only && !((double)lcost[s] < avg)) {
            t = -1;
            ltarget[s] = (int32_t)s;
            continue;
        }
        if (t < 0 || (!by_dot && s - t > k) || (by_dot && s - t > dot[t])) t = s;
        ltarget[s] = (int32_t)t;
    }
}

__global__ void k_map_targets(int64_t n, const int32_t* level, const int32_t* ltarget, int32_t* target) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) target[i] = ltarget[level[i]];
}

__global__ void k_depths(int64_t n, const int32_t* level, const int32_t* target, int32_t* moved, int* maxd,
                         unsigned long long* nmoved) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int d = level[i] - target[i];
    moved[i] = d > 0 ? 1 : 0;
    if (d > 0) {
        atomicMax(maxd, d);
        atomicAdd(nmoved, 1ull);
    }
}

// ---------------------------------------------------------------------------------
// substitution rounds
// ---------------------------------------------------------------------------------

template <typename T>
struct FillArgs {
    int64_t n;
    const int32_t* rowptr;
    const int32_t* colidx;
    const T* vals;
    const int32_t* level;
    const int32_t* target;
    const int32_t* moved;
    int64_t* c_off;
    int32_t* c_cnt;
    int64_t* e_off;
    int32_t* e_cnt;
    int32_t* hcol;
    double* hval;
    int64_t* ub;  // per row: upper bound of C + E entries in this depth round (0 for other rows)
    int64_t* ubc;
    int32_t* tcol;  // per-round temporary of the merge sort (same offsets as the round's rows)
    double* tval;
    double guard;
    int* status;
};

template <typename T>
__global__ void k_fill_size(FillArgs<T> a, int d) {
    int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= a.n) return;
    if (a.level[r] - a.target[r] != d) {
        a.ub[r] = 0;
        return;
    }
    const int t = a.target[r];
    int64_t uc = 0, ue = 0;
    for (int64_t q = a.rowptr[r]; q < (int64_t)a.rowptr[r + 1] - 1; ++q) {
        const int32_t j = a.colidx[q];
        if (a.target[j] >= t) {
            uc += a.moved[j] ? a.c_cnt[j] : (a.rowptr[j + 1] - a.rowptr[j] - 1);
            ue += 1 + (a.moved[j] ? a.e_cnt[j] : 0);
        } else {
            uc += 1;
        }
    }
    a.ub[r] = uc + ue;
    a.ubc[r] = uc;
}

// Stable sort of (col, val) pairs by col -- insertion sort for short rows, a bottom-up
// merge sort through the temporary arrays for long ones -- then equal columns are summed
// in their original order (the order the serial rewrite adds them in).
__device__ int sort_merge(int32_t* c, double* v, int32_t* tc, double* tv, int len) {
    if (len <= 32) {
        for (int i = 1; i < len; ++i) {
            int32_t ci = c[i];
            double vi = v[i];
            int j = i - 1;
            while (j >= 0 && c[j] > ci) {
                c[j + 1] = c[j];
                v[j + 1] = v[j];
                --j;
            }
            c[j + 1] = ci;
            v[j + 1] = vi;
        }
    } else {
        int32_t *sc = c, *dc = tc;
        double *sv = v, *dv = tv;
        for (int w = 1; w < len; w *= 2) {
            for (int lo = 0; lo < len; lo += 2 * w) {
                const int mid = min(lo + w, len), hi = min(lo + 2 * w, len);
                int i = lo, j = mid, o = lo;
                while (i < mid && j < hi) {
                    if (sc[j] < sc[i]) { dc[o] = sc[j]; dv[o++] = sv[j++]; }
                    else { dc[o] = sc[i]; dv[o++] = sv[i++]; }
                }
                while (i < mid) { dc[o] = sc[i]; dv[o++] = sv[i++]; }
                while (j < hi) { dc[o] = sc[j]; dv[o++] = sv[j++]; }
            }
            int32_t* t1 = sc; sc = dc; dc = t1;
            double* t2 = sv; sv = dv; dv = t2;
        }
        if (sc != c)
            for (int i = 0; i < len; ++i) { c[i] = sc[i]; v[i] = sv[i]; }
    }
    int w = 0;
    for (int i = 0; i < len; ++i) {
        if (w > 0 && c[w - 1] == c[i]) {
            v[w - 1] = __dadd_rn(v[w - 1], v[i]);
        } else {
            c[w] = c[i];
            v[w] = v[i];
            ++w;
        }
    }
    return w;
}

template <typename T>
__global__ void k_fill(FillArgs<T> a, int d, const int64_t* off, int64_t heap_base) {
    int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= a.n) return;
    if (a.level[r] - a.target[r] != d) return;
    const int t = a.target[r];
    const int64_t o = heap_base + off[r];
    const int64_t uc = a.ubc[r];
    int32_t* cc = a.hcol + o;
    double* cv = a.hval + o;
    int32_t* ec = cc + uc;
    double* ev = cv + uc;
    int nc = 0, ne = 0;
    const int64_t q0 = a.rowptr[r], q1 = (int64_t)a.rowptr[r + 1] - 1;
    const double drr = (double)a.vals[q1];
    for (int64_t q = q0; q < q1; ++q) {
        const int32_t j = a.colidx[q];
        const double aj = (double)a.vals[q];
        if (a.target[j] < t) {
            cc[nc] = j;
            cv[nc++] = aj;
            continue;
        }
        if (a.moved[j]) {
            // j's rearranged equation: x_j = sum_m e_jm b_m - sum_k c_jk x_k, e_jj = 1 / L_jj
            const int64_t hj = a.c_off[j];
            for (int u = 0; u < a.c_cnt[j]; ++u) {
                cc[nc] = a.hcol[hj + u];
                cv[nc++] = __dmul_rn(-aj, a.hval[hj + u]);
            }
            const int64_t he = a.e_off[j];
            for (int u = 0; u < a.e_cnt[j]; ++u) {
                ec[ne] = a.hcol[he + u];
                ev[ne++] = __dmul_rn(-aj, a.hval[he + u]);
            }
            const double ejj = __ddiv_rn(1.0, (double)a.vals[(int64_t)a.rowptr[j + 1] - 1]);
            ec[ne] = j;
            ev[ne++] = __dmul_rn(-aj, ejj);
        } else {
            // j keeps its original equation: x_j = (b_j - sum_k L_jk x_k) / L_jj
            const int64_t p1 = (int64_t)a.rowptr[j + 1] - 1;
            const double dj = (double)a.vals[p1];
            for (int64_t u = a.rowptr[j]; u < p1; ++u) {
                cc[nc] = a.colidx[u];
                cv[nc++] = __dmul_rn(-aj, __ddiv_rn((double)a.vals[u], dj));
            }
            ec[ne] = j;
            ev[ne++] = __ddiv_rn(-aj, dj);
        }
    }
    int32_t* tc = a.tcol + off[r];
    double* tv = a.tval + off[r];
    nc = sort_merge(cc, cv, tc, tv, nc);
    ne = sort_merge(ec, ev, tc + uc, tv + uc, ne);
    bool bad = false;
    for (int i = 0; i < nc; ++i) {
        cv[i] = __ddiv_rn(cv[i], drr);
        if (!isfinite(cv[i]) || (a.guard > 0 && fabs(cv[i]) > a.guard)) bad = true;
    }
    for (int i = 0; i < ne; ++i) {
        ev[i] = __ddiv_rn(ev[i], drr);
        if (!isfinite(ev[i]) || (a.guard > 0 && fabs(ev[i]) > a.guard)) bad = true;
    }
    if (bad) atomicCAS(a.status, 0, (int)DEV_NUMERIC);
    a.c_off[r] = o;
    a.c_cnt[r] = nc;
    a.e_off[r] = o + uc;
    a.e_cnt[r] = ne;
}

__global__ void k_narrow(const int64_t* in, int32_t* out, int64_t n) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i <= n) out[i] = (int32_t)in[i];
}

// dependency structure of the rewritten system (original numbering, no diagonal)
__global__ void k_dep_counts(int64_t n, const int32_t* rowptr, const int32_t* moved, const int32_t* c_cnt,
                             int32_t* cnt) {
    int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r < n) cnt[r] = moved[r] ? c_cnt[r] : rowptr[r + 1] - rowptr[r] - 1;
}

__global__ void k_dep_fill(int64_t n, const int32_t* rowptr, const int32_t* colidx, const int32_t* moved,
                           const int64_t* c_off, const int32_t* c_cnt, const int32_t* hcol, const int32_t* dptr,
                           int32_t* dcol) {
    int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n) return;
    int64_t o = dptr[r];
    if (moved[r]) {
        for (int u = 0; u < c_cnt[r]; ++u) dcol[o + u] = hcol[c_off[r] + u];
    } else {
        for (int64_t q = rowptr[r]; q < (int64_t)rowptr[r + 1] - 1; ++q) dcol[o++] = colidx[q];
    }
}

}  // namespace

// ---------------------------------------------------------------------------------
// host orchestration
// ---------------------------------------------------------------------------------

struct PlanOut {
    int64_t moved = 0, stored = -1, targets = 0;
};

// plans targets[n] (device) for the given walk kind; returns planner bookkeeping
sptrsv_status plan_targets(const sptrsv_csr* L, const Levels& lv, int kind, int k, const int32_t* dot_dev,
                           double avg, double cap, const int64_t* inj, int alpha, int64_t beta, int parts,
                           int32_t* target, PlanOut& po, cudaStream_t st) {
    const int64_t n = L->n, m = lv.m;
    // the row walk is needed where the rows decide (cost or row budget, the nnz cap, the per-row rules)
    const bool walk = kind == WALK_NAIVE || kind == WALK_ROWCAP || cap > 0 || inj || alpha > 0 || beta > 0;
    if (!walk) {
        Scratch lt;
        SP_TRY(lt.alloc(std::max<int64_t>(1, m) * sizeof(int32_t), st));
        k_level_targets<<<1, 1, 0, st>>>(m, kind, k, dot_dev, lv.lcost.p, avg, (int)std::max<int64_t>(1, parts),
                                          lt.as<int32_t>());
        k_map_targets<<<nblk(n, 256), 256, 0, st>>>(n, lv.level.p, lt.as<int32_t>(), target);
        SP_CUDA(cudaGetLastError());
        return SPTRSV_OK;
    }
    parts = (int)std::max<int64_t>(1, std::min<int64_t>(parts, std::max<int64_t>(1, m)));
    Scratch rc, doff, dlen, eoff, elen, info, status, plim;
    SP_TRY(rc.alloc(n * 8, st));
    SP_TRY(doff.alloc(n * 8, st));
    SP_TRY(dlen.alloc(n * 4, st));
    SP_TRY(eoff.alloc(n * 8, st));
    SP_TRY(elen.alloc(n * 4, st));
    SP_TRY(info.alloc((size_t)parts * 3 * 8, st));
    SP_TRY(status.alloc(sizeof(int), st));
    SP_TRY(plim.alloc((size_t)parts * 8, st));
    // the nnz cap's allowance, shared by the level ranges in proportion to their entries
    std::vector<int64_t> h_plim(parts, INT64_MAX);
    if (cap > 0) {
        const int64_t allowance = (int64_t)std::floor(cap * (double)L->nnz) - L->nnz;
        std::vector<int64_t> h_lnnz(std::max<int64_t>(1, m));
        SP_CUDA(cudaMemcpyAsync(h_lnnz.data(), lv.lnnz.p, m * 8, cudaMemcpyDeviceToHost, st));
        SP_CUDA(cudaStreamSynchronize(st));
        for (int w = 0; w < parts; ++w) {
            int64_t z = 0;
            for (int64_t l = m * w / parts; l < m * (w + 1) / parts; ++l) z += h_lnnz[l];
            h_plim[w] = L->nnz > 0 ? allowance * z / L->nnz : 0;
        }
    }
    SP_CUDA(cudaMemcpyAsync(plim.p, h_plim.data(), (size_t)parts * 8, cudaMemcpyHostToDevice, st));
    int64_t cap_pool = std::max<int64_t>(1 << 20, (cap > 0 ? 2 : 16) * L->nnz / parts * (parts > 1 ? 2 : 1));
    for (int attempt = 0; attempt < 6; ++attempt) {
        Scratch pool;
        SP_TRY(pool.alloc((size_t)cap_pool * parts * sizeof(int32_t), st));
        SP_CUDA(cudaMemsetAsync(status.p, 0, sizeof(int), st));
        k_init_walk<<<nblk(n, 256), 256, 0, st>>>(n, L->rowptr, lv.level.p, target, rc.as<int64_t>());
        WalkArgs a;
        a.n = n;
        a.m = m;
        a.nnzL = L->nnz;
        a.rowptr = L->rowptr;
        a.colidx = L->colidx;
        a.level = lv.level.p;
        a.lptr = lv.level_ptr.p;
        a.lrows = lv.level_rows.p;
        a.lcost = lv.lcost.p;
        a.kind = kind;
        a.k = k;
        a.avg = avg;
        a.part_limit = plim.as<int64_t>();
        a.dot = dot_dev;
        a.inj = inj;
        a.alpha = alpha;
        a.beta = beta;
        a.target = target;
        a.row_cost = rc.as<int64_t>();
        a.d_off = doff.as<int64_t>();
        a.d_len = dlen.as<int32_t>();
        a.e_off = eoff.as<int64_t>();
        a.e_len = elen.as<int32_t>();
        a.pool = pool.as<int32_t>();
        a.pool_cap = cap_pool;
        a.info = info.as<int64_t>();
        a.status = status.as<int>();
        k_plan_walk<<<parts, 32, 3 * WALK_SORT_CAP * sizeof(int32_t), st>>>(a);
        SP_CUDA(cudaGetLastError());
        int hs = 0;
        std::vector<int64_t> hi((size_t)parts * 3);
        SP_CUDA(cudaMemcpyAsync(&hs, status.p, sizeof(int), cudaMemcpyDeviceToHost, st));
        SP_CUDA(cudaMemcpyAsync(hi.data(), info.p, (size_t)parts * 3 * 8, cudaMemcpyDeviceToHost, st));
        SP_CUDA(cudaStreamSynchronize(st));
        if (hs == DEV_OVERFLOW) {
            cap_pool *= 4;
            continue;
        }
        if (hs != 0) return map_dev_status(hs, "rewrite: planner");
        po.moved = 0;
        po.stored = L->nnz;
        po.targets = 0;
        for (int w = 0; w < parts; ++w) {
            po.moved += hi[3 * w];
            po.stored += hi[3 * w + 1];
            po.targets += hi[3 * w + 2];
        }
        return SPTRSV_OK;
    }
    set_error("rewrite: planner scratch exceeded %lld entries", (long long)cap_pool);
    return SPTRSV_ERR_OOM;
}

template <typename T>
sptrsv_status rewrite_rows(const sptrsv_csr* L, const Levels& lv, const int32_t* target, double guard,
                           sptrsv_system* s, cudaStream_t st) {
    const int64_t n = L->n;
    Scratch moved, ctl, c_off, c_cnt, e_off, e_cnt, ub, ubc, off;
    SP_TRY(moved.alloc(n * 4, st));
    SP_TRY(ctl.alloc(32, st));
    SP_TRY(c_off.alloc(n * 8, st));
    SP_TRY(c_cnt.alloc(n * 4, st));
    SP_TRY(e_off.alloc(n * 8, st));
    SP_TRY(e_cnt.alloc(n * 4, st));
    SP_TRY(ub.alloc(n * 8, st));
    SP_TRY(ubc.alloc(n * 8, st));
    SP_TRY(off.alloc((n + 1) * 8, st));
    SP_CUDA(cudaMemsetAsync(ctl.p, 0, 32, st));
    int* maxd = ctl.as<int>();
    unsigned long long* nmv = (unsigned long long*)(ctl.as<char>() + 8);
    int* status = ctl.as<int>() + 4;
    SP_CUDA(cudaMemsetAsync(c_cnt.p, 0, n * 4, st));
    SP_CUDA(cudaMemsetAsync(e_cnt.p, 0, n * 4, st));
    k_depths<<<nblk(n, 256), 256, 0, st>>>(n, lv.level.p, target, moved.as<int32_t>(), maxd, nmv);
    SP_CUDA(cudaGetLastError());
    int64_t h[2];
    SP_CUDA(cudaMemcpyAsync(h, ctl.p, 16, cudaMemcpyDeviceToHost, st));
    SP_CUDA(cudaStreamSynchronize(st));
    const int maxdepth = (int)(h[0] & 0xffffffff);
    s->rows_moved = (int64_t)h[1];

    // heap of rewritten rows: grows between rounds
    DevBuf<int32_t> hcol;
    DevBuf<double> hval;
    int64_t heap_top = 0, heap_cap = std::max<int64_t>(1024, n / 4);
    SP_TRY(hcol.alloc(heap_cap));
    SP_TRY(hval.alloc(heap_cap));
    FillArgs<T> a;
    a.n = n;
    a.rowptr = L->rowptr;
    a.colidx = L->colidx;
    a.vals = (const T*)L->vals;
    a.level = lv.level.p;
    a.target = target;
    a.moved = moved.as<int32_t>();
    a.c_off = c_off.as<int64_t>();
    a.c_cnt = c_cnt.as<int32_t>();
    a.e_off = e_off.as<int64_t>();
    a.e_cnt = e_cnt.as<int32_t>();
    a.ub = ub.as<int64_t>();
    a.ubc = ubc.as<int64_t>();
    a.guard = guard;
    a.status = status;
    for (int d = 1; d <= maxdepth; ++d) {
        k_fill_size<T><<<nblk(n, 256), 256, 0, st>>>(a, d);
        SP_CUDA(cudaGetLastError());
        SP_TRY(scan_exclusive_i64(ub.as<int64_t>(), off.as<int64_t>(), n, st));
        int64_t tot = 0;
        SP_CUDA(cudaMemcpyAsync(&tot, off.as<int64_t>() + n, 8, cudaMemcpyDeviceToHost, st));
        SP_CUDA(cudaStreamSynchronize(st));
        if (heap_top + tot > heap_cap) {
            int64_t nc = std::max<int64_t>(2 * heap_cap, heap_top + tot + 1024);
            DevBuf<int32_t> c2;
            DevBuf<double> v2;
            SP_TRY(c2.alloc(nc));
            SP_TRY(v2.alloc(nc));
            if (heap_top) {
                SP_CUDA(cudaMemcpyAsync(c2.p, hcol.p, heap_top * 4, cudaMemcpyDeviceToDevice, st));
                SP_CUDA(cudaMemcpyAsync(v2.p, hval.p, heap_top * 8, cudaMemcpyDeviceToDevice, st));
                SP_CUDA(cudaStreamSynchronize(st));
            }
            std::swap(hcol.p, c2.p);
            std::swap(hcol.n, c2.n);
            std::swap(hval.p, v2.p);
            std::swap(hval.n, v2.n);
            heap_cap = nc;
        }
        a.hcol = hcol.p;
        a.hval = hval.p;
        Scratch tcol, tval;
        SP_TRY(tcol.alloc(std::max<int64_t>(1, tot) * sizeof(int32_t), st));
        SP_TRY(tval.alloc(std::max<int64_t>(1, tot) * sizeof(double), st));
        a.tcol = tcol.as<int32_t>();
        a.tval = tval.as<double>();
        k_fill<T><<<nblk(n, 128), 128, 0, st>>>(a, d, off.as<int64_t>(), heap_top);
        SP_CUDA(cudaGetLastError());
        heap_top += tot;
    }
    int hs = 0;
    SP_CUDA(cudaMemcpyAsync(&hs, status, sizeof(int), cudaMemcpyDeviceToHost, st));
    SP_CUDA(cudaStreamSynchronize(st));
    if (hs != 0) return map_dev_status(hs, "rewrite");

    // dependency structure of the rewritten rows -> levels of the stored system
    Scratch dcnt, dptr64, dptr, dcol;
    SP_TRY(dcnt.alloc((n + 1) * 4, st));
    SP_TRY(dptr64.alloc((n + 1) * 8, st));
    SP_TRY(dptr.alloc((n + 1) * 4, st));
    k_dep_counts<<<nblk(n, 256), 256, 0, st>>>(n, L->rowptr, moved.as<int32_t>(), c_cnt.as<int32_t>(),
                                               dcnt.as<int32_t>());
    SP_CUDA(cudaGetLastError());
    SP_TRY(scan_exclusive_i32_to_i64(dcnt.as<int32_t>(), dptr64.as<int64_t>(), n, st));
    int64_t ndeps = 0;
    SP_CUDA(cudaMemcpyAsync(&ndeps, dptr64.as<int64_t>() + n, 8, cudaMemcpyDeviceToHost, st));
    SP_CUDA(cudaStreamSynchronize(st));
    if (ndeps >= INT32_MAX) {
        set_error("rewritten system has %lld dependencies; int32 offsets are exceeded", (long long)ndeps);
        return SPTRSV_ERR_UNSUPPORTED;
    }
    k_narrow<<<nblk(n + 1, 256), 256, 0, st>>>(dptr64.as<int64_t>(), dptr.as<int32_t>(), n);
    SP_TRY(dcol.alloc(std::max<int64_t>(1, ndeps) * 4, st));
    k_dep_fill<<<nblk(n, 256), 256, 0, st>>>(n, L->rowptr, L->colidx, moved.as<int32_t>(), c_off.as<int64_t>(),
                                             c_cnt.as<int32_t>(), hcol.p, dptr.as<int32_t>(), dcol.as<int32_t>());
    SP_CUDA(cudaGetLastError());
    DepCsr dep;
    dep.n = n;
    dep.rowptr = dptr.as<int32_t>();
    dep.colidx = dcol.as<int32_t>();
    dep.diag_last = 0;
    SP_TRY(analyse_dep(dep, s->lv, st));
    s->m = s->lv.m;
    RewriteHeap rw;
    rw.moved = moved.as<int32_t>();
    rw.c_off = c_off.as<int64_t>();
    rw.c_cnt = c_cnt.as<int32_t>();
    rw.e_off = e_off.as<int64_t>();
    rw.e_cnt = e_cnt.as<int32_t>();
    rw.col = hcol.p;
    rw.val = hval.p;
    SP_TRY(pack_system(s, L, &rw, st));
    return SPTRSV_OK;
}

sptrsv_status rewrite_system(const sptrsv_csr* L, const Levels& lv, int kind, int k, const int32_t* dot_dev,
                             double avg_override, double cap, double guard, const int64_t* inj, int alpha, int64_t beta,
                             int parts, sptrsv_system** out, cudaStream_t st) {
    const int64_t n = L->n;
    sptrsv_system* s = new (std::nothrow) sptrsv_system();
    if (!s) { set_error("host allocation failed"); return SPTRSV_ERR_OOM; }
    s->n = n;
    s->dtype = L->dtype;
    s->nnz_l = L->nnz;
    s->rewritten = 1;
    const double avg = avg_override > 0 ? avg_override : lv.avg;
    s->avg = avg;
    auto fail = [&](sptrsv_status rc) {
        delete s;
        return rc;
    };
    sptrsv_status rc = s->target.alloc(std::max<int64_t>(1, n));
    if (rc != SPTRSV_OK) return fail(rc);
    PlanOut po;
    if (n > 0) {
        rc = plan_targets(L, lv, kind, k, dot_dev, avg, cap, inj, alpha, beta, parts, s->target.p, po, st);
        if (rc != SPTRSV_OK) return fail(rc);
        rc = L->dtype == SPTRSV_F64 ? rewrite_rows<double>(L, lv, s->target.p, guard, s, st)
                                    : rewrite_rows<float>(L, lv, s->target.p, guard, s, st);
        if (rc != SPTRSV_OK) return fail(rc);
    } else {
        DepCsr dep;
        rc = analyse_dep(dep, s->lv, st);
        if (rc != SPTRSV_OK) return fail(rc);
    }
    // nnz(L') + nnz(E explicit rows): off-diagonal coefficients, diagonals, and for
    // rewritten rows their E row including its diagonal term
    s->stored_nnz = s->nnz_c + n + s->nnz_e + s->rows_moved;
    if (po.stored >= 0 && po.stored != s->stored_nnz) {
        set_error("rewrite: planner counted %lld stored entries, the rewrite produced %lld", (long long)po.stored,
                  (long long)s->stored_nnz);
        return fail(SPTRSV_ERR_CUDA);
    }
    *out = s;
    return SPTRSV_OK;
}

}  // namespace sp

using namespace sp;

extern "C" sptrsv_status sptrsv_rewrite(const sptrsv_csr* L, const sptrsv_levels* lvh, const sptrsv_strategy* sg,
                                        sptrsv_system** out, sptrsv_stream_t stream) {
    if (!L || !lvh || !sg || !out) { set_error("rewrite: null argument"); return SPTRSV_ERR_INVALID; }
    *out = nullptr;
    cudaStream_t st = (cudaStream_t)stream;
    const Levels& lv = lvh->lv;
    if (lv.n != L->n) { set_error("rewrite: levels belong to another matrix"); return SPTRSV_ERR_INVALID; }
    int kind = sg->kind;
    if (kind == SPTRSV_STRATEGY_NONE) return sptrsv_system_plain(L, lvh, out, stream);
    if (kind == SPTRSV_STRATEGY_LEARNED) {
        if (!sg->picker) {
            kind = SPTRSV_STRATEGY_NAIVE;  // the paper's strategy is the fallback without a model
        } else {
            return learned_rewrite(L, lvh, sg, out, st);
        }
    }
    if ((kind == SPTRSV_STRATEGY_DEPTH_K || kind == SPTRSV_STRATEGY_MANUAL) && sg->k < 0) {
        set_error("rewrite: depth k < 0");
        return SPTRSV_ERR_INVALID;
    }
    Scratch dot;
    const int32_t* dot_dev = nullptr;
    if (kind == SPTRSV_STRATEGY_CHOSEN || kind == SPTRSV_STRATEGY_CHOSEN_THIN) {
        if (!sg->depth_of_target_host) { set_error("rewrite: CHOSEN needs depth_of_target"); return SPTRSV_ERR_INVALID; }
        SP_TRY(dot.alloc(std::max<int64_t>(1, lv.m) * 4, st));
        SP_CUDA(cudaMemcpyAsync(dot.p, sg->depth_of_target_host, lv.m * 4, cudaMemcpyHostToDevice, st));
        dot_dev = dot.as<int32_t>();
    }
    int wk = kind == SPTRSV_STRATEGY_NAIVE ? WALK_NAIVE : kind == SPTRSV_STRATEGY_DEPTH_K ? WALK_DEPTH
           : kind == SPTRSV_STRATEGY_CHOSEN ? WALK_CHOSEN : kind == SPTRSV_STRATEGY_MANUAL ? WALK_MANUAL
           : kind == SPTRSV_STRATEGY_ROWCAP ? WALK_ROWCAP : kind == SPTRSV_STRATEGY_CHOSEN_THIN ? WALK_CHOSEN_THIN : 0;
    if (!wk) { set_error("rewrite: unknown strategy %d", kind); return SPTRSV_ERR_INVALID; }
    const int k = kind == SPTRSV_STRATEGY_ROWCAP && sg->k <= 0 ? ROWCAP_DEFAULT_ROWS : sg->k;
    sptrsv_status rc = rewrite_system(L, lv, wk, k, dot_dev, sg->avg_override, sg->nnz_growth_cap,
                                      sg->growth_guard, sg->injected_cost_dev, sg->max_deps, sg->max_spread,
                                      sg->walk_parts, out, st);
    if (rc == SPTRSV_OK) (*out)->strategy_used = kind;
    return rc;
}
