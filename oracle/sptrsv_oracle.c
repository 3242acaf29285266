/*
 * sptrsv_oracle.c -- plain serial CPU oracle for the SpTRSV hot path.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library calls, links or loads this
 * file; only the tests, the smoke check and the benchmark's CPU-baseline leg use it.
 * It shares no code, header or constant with the CUDA path.
 *
 * Everything here is the most direct restatement of the paper that still runs on the
 * full workloads: one core, fp64, plain multiply and add (compile with
 * -ffp-contract=off so that no fused multiply-add creeps in), no blocking or reordering
 * beyond what the definitions state.
 *
 *   orc_validate          the CSR contract of Algorithm 1 (diagonal last in the row).
 *   orc_forward_subst     Algorithm 1 (Section II.A): x_i = (b_i - sum_j L_ij x_j) / L_ii.
 *   orc_levels            level sets of DAG_L (Section II.A): a row without off-diagonal
 *                         entries is on level 0, any other row one level below its
 *                         deepest dependency.
 *   orc_level_stats       row cost 2*nnz-1 and level cost 2*sum(nnz)-n (Section III).
 *   orc_plan              the rewrite planner of Section III: the naive avgLevelCost
 *                         strategy, the fixed-distance ("every k levels into the next
 *                         target") strategy, the manual strategy (fixed distance over thin
 *                         levels), per-target depths chosen by a caller (over all levels or
 *                         thin levels only), the row-capped walk (a row count in place of
 *                         avgLevelCost), the nnz cap and the per-row rules of Section III.A.
 *                         Pinned by the Section III costMap example and structural
 *                         identities; on general inputs beyond those its choices are parity
 *                         unpinned against the paper (Table I needs datasets that are missing).
 *   orc_rewrite           equation rewriting with rearrangement (Section II.B, Fig. 2):
 *                         substitute every dependency that sits on the target level or
 *                         below it by its own equation, then group the coefficients of
 *                         each unknown and of each b entry.
 *   orc_solve_rewritten   forward substitution of the rewritten equations.
 *
 * Readings where the paper is silent or garbled: 0-based levels, rewritten-row cost
 * 2*|deps|, greedy prefix stop rule, fixed average, fat levels break a run, structural (not
 * numerical) fill, the nnz cap and the per-row rules checked in planning order.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------------------- */
/* validation                                                                       */
/* ------------------------------------------------------------------------------- */

/* Returns 0 when the CSR matrix is lower triangular with ascending columns and a
 * non-zero finite diagonal stored last in every row; otherwise a positive code and the
 * first offending row in *bad_row.
 * codes: 1 bad row pointers, 2 empty row, 3 column out of range / not ascending,
 *        4 diagonal missing or not last, 5 diagonal zero or non-finite,
 *        6 non-finite off-diagonal value. */
int orc_validate(int64_t n, const int32_t* rowptr, const int32_t* colidx, const double* vals,
                 int64_t* bad_row) {
    *bad_row = -1;
    if (rowptr[0] != 0) { *bad_row = 0; return 1; }
    for (int64_t i = 0; i < n; ++i) {
        int64_t a = rowptr[i], b = rowptr[i + 1];
        if (b < a) { *bad_row = i; return 1; }
        if (b == a) { *bad_row = i; return 2; }
        for (int64_t k = a; k < b; ++k) {
            int64_t c = colidx[k];
            if (c < 0 || c > i) { *bad_row = i; return 3; }
            if (k > a && colidx[k - 1] >= c) { *bad_row = i; return 3; }
        }
        if (colidx[b - 1] != i) { *bad_row = i; return 4; }
        double d = vals[b - 1];
        if (d == 0.0 || !isfinite(d)) { *bad_row = i; return 5; }
        for (int64_t k = a; k < b - 1; ++k)
            if (!isfinite(vals[k])) { *bad_row = i; return 6; }
    }
    return 0;
}

/* ------------------------------------------------------------------------------- */
/* Algorithm 1                                                                      */
/* ------------------------------------------------------------------------------- */

/* Serial forward substitution for one right-hand side.  The garbled accumulator of
 * the printed algorithm is read as one scalar partial sum over the off-diagonal
 * entries; the diagonal is the last entry of the row. */
void orc_forward_subst(int64_t n, const int32_t* rowptr, const int32_t* colidx,
                       const double* vals, const double* b, double* x) {
    for (int64_t i = 0; i < n; ++i) {
        double sum = 0.0;
        int64_t last = (int64_t)rowptr[i + 1] - 1;
        for (int64_t j = rowptr[i]; j < last; ++j) sum += vals[j] * x[colidx[j]];
        x[i] = (b[i] - sum) / vals[last];
    }
}

/* Same with float values promoted to double (used to score float32 batches). */
void orc_forward_subst_f32vals(int64_t n, const int32_t* rowptr, const int32_t* colidx,
                               const float* vals, const double* b, double* x) {
    for (int64_t i = 0; i < n; ++i) {
        double sum = 0.0;
        int64_t last = (int64_t)rowptr[i + 1] - 1;
        for (int64_t j = rowptr[i]; j < last; ++j) sum += (double)vals[j] * x[colidx[j]];
        x[i] = (b[i] - sum) / (double)vals[last];
    }
}

/* ------------------------------------------------------------------------------- */
/* level sets                                                                        */
/* ------------------------------------------------------------------------------- */

/* level(i) = 0 when row i has no dependency, else 1 + max level of its dependencies.
 * diag_last != 0: the last entry of each row is the diagonal and is skipped; otherwise
 * every entry of the row is a dependency.  Returns the number of levels m. */
int32_t orc_levels(int64_t n, const int32_t* rowptr, const int32_t* colidx, int diag_last,
                   int32_t* level) {
    int32_t m = 0;
    for (int64_t i = 0; i < n; ++i) {
        int64_t end = (int64_t)rowptr[i + 1] - (diag_last ? 1 : 0);
        int32_t lv = 0;
        for (int64_t k = rowptr[i]; k < end; ++k) {
            int32_t d = level[colidx[k]] + 1;
            if (d > lv) lv = d;
        }
        level[i] = lv;
        if (lv + 1 > m) m = lv + 1;
    }
    return n > 0 ? m : 0;
}

/* Per level: number of rows, number of nonzeros (diagonal included), and the cost
 * 2*sum(nnz) - rows, i.e. the sum of the row costs 2*nnz-1 (Section III). */
void orc_level_stats(int64_t n, const int32_t* rowptr, const int32_t* level, int32_t m,
                     int64_t* rows, int64_t* nnz, int64_t* cost) {
    for (int32_t l = 0; l < m; ++l) rows[l] = nnz[l] = cost[l] = 0;
    for (int64_t i = 0; i < n; ++i) {
        int64_t z = (int64_t)rowptr[i + 1] - rowptr[i];
        rows[level[i]] += 1;
        nnz[level[i]] += z;
        cost[level[i]] += 2 * z - 1;
    }
}

/* ------------------------------------------------------------------------------- */
/* small sorted integer sets                                                         */
/* ------------------------------------------------------------------------------- */

typedef struct { int32_t* v; int32_t len, cap; } iset;

static void iset_reserve(iset* s, int32_t cap) {
    if (s->cap >= cap) return;
    int32_t nc = s->cap ? s->cap : 4;
    while (nc < cap) nc *= 2;
    s->v = (int32_t*)realloc(s->v, sizeof(int32_t) * (size_t)nc);
    s->cap = nc;
}

/* insert keeping ascending order and no duplicates */
static void iset_add(iset* s, int32_t x) {
    int32_t lo = 0, hi = s->len;
    while (lo < hi) {
        int32_t mid = (lo + hi) / 2;
        if (s->v[mid] < x) lo = mid + 1; else hi = mid;
    }
    if (lo < s->len && s->v[lo] == x) return;
    iset_reserve(s, s->len + 1);
    memmove(s->v + lo + 1, s->v + lo, sizeof(int32_t) * (size_t)(s->len - lo));
    s->v[lo] = x;
    s->len++;
}

static void iset_free(iset* s) { free(s->v); s->v = NULL; s->len = s->cap = 0; }

/* ------------------------------------------------------------------------------- */
/* the planner (Section III)                                                          */
/* ------------------------------------------------------------------------------- */

/* strategy kinds */
#define ORC_NAIVE 1   /* avgLevelCost over thin levels */
#define ORC_DEPTH 2   /* fixed distance: target every (k+1)-th level, k levels merged in */
#define ORC_CHOSEN 3  /* per-target depth given by the caller (learned picker) */
#define ORC_MANUAL 4  /* fixed distance over thin levels only: nine levels folded into each tenth,
                         applied to the levels cheaper than avgLevelCost (Section IV) */
#define ORC_CHOSEN_THIN 5  /* per-target depth over thin levels only: the learned picker's
                              depth choice within the thin-level rule of Section III */
#define ORC_ROWCAP 6  /* thin levels, rows moved into a target while it holds at most k rows:
                         the Section III walk with a row count in place of avgLevelCost */

/*
 * Walk the levels in order and decide, row by row, the level each row moves to.
 *
 * State of the walk: the current target t (or none), the cost accumulated on t, and
 * for every row its current level, its current dependency set D and the support of its
 * b-coefficients E (which rows of b its rewritten equation reads; {r} for rows that
 * were not rewritten).
 *
 * For a row r of a source level s the planner substitutes, once, every dependency j
 * whose current level is >= t: D' = union over deps j of (curlev(j) >= t ? D(j) : {j}),
 * E' = {r} union E(j) over the substituted j.  Its cost on t is 2*|D'| (rearranged, no
 * division; Section III and the Table I discussion), or the injected cost when a test
 * supplies one.  Growth of the stored system: the row's entries become |D'|+1 in L'
 * plus |E'| in E instead of |D|+1.
 *
 * NAIVE: levels with cost < avgLevelCost are thin, the average is computed once over
 *   the original levels and kept fixed.  The first thin level of a run is the target;
 *   rows of the following thin levels are moved in ascending row order while
 *   cur + c <= avg; the first row that does not fit (or that the nnz cap rejects)
 *   makes its own level the new target, holding its remaining rows.  A level that is
 *   not thin ends the run and keeps its rows.
 * DEPTH / CHOSEN: every level is eligible; a level s joins target t while
 *   s - t <= depth(t) (depth k for DEPTH, depth_of_target[t] for CHOSEN), otherwise s
 *   becomes the next target.  The nnz cap rejects rows as in NAIVE.
 * MANUAL: thin levels are eligible as in NAIVE, levels join a target by distance as in
 *   DEPTH (no cost rule).
 * CHOSEN_THIN: thin levels are eligible as in NAIVE, levels join a target by its own
 *   distance depth_of_target[t] as in CHOSEN (no cost rule).
 * ROWCAP: NAIVE with the number of rows on the target in place of the cost: thin levels are
 *   eligible, rows of the following thin levels move while the target holds fewer than k
 *   rows; the first row that does not fit (or breaks the cap or a per-row rule) makes its
 *   own level the new target, holding its remaining rows.
 *
 * inputs : lower-triangular CSR (diagonal last), level[n], m, kind, k, avg_override
 *          (<= 0: computed), cap_ratio (<= 0: no cap), injected_cost (NULL: computed),
 *          depth_of_target[m] (CHOSEN and CHOSEN_THIN only)
 * outputs: target[n] (the level each row ends up on, in the original numbering),
 *          row_cost[n] (cost of each row on its final level under the planner's model),
 *          info[6] = {rows moved, nnz(L') + nnz(E explicit) after planning, nnz(L),
 *                     number of non-empty levels, avg*1e6 rounded, number of targets}
 * returns 0, or -1 on allocation failure.
 */
int orc_plan_rules(int64_t n, const int32_t* rowptr, const int32_t* colidx, const int32_t* level,
                   int32_t m, int kind, int32_t k, double avg_override, double cap_ratio,
                   const int64_t* injected_cost, const int32_t* depth_of_target, int32_t alpha,
                   int64_t beta, int32_t* target, int64_t* row_cost, int64_t* info);

int orc_plan_parts(int64_t n, const int32_t* rowptr, const int32_t* colidx, const int32_t* level,
                   int32_t m, int kind, int32_t k, double avg_override, double cap_ratio,
                   const int64_t* injected_cost, const int32_t* depth_of_target, int32_t alpha,
                   int64_t beta, int32_t parts, int32_t* target, int64_t* row_cost, int64_t* info);

int orc_plan(int64_t n, const int32_t* rowptr, const int32_t* colidx, const int32_t* level,
             int32_t m, int kind, int32_t k, double avg_override, double cap_ratio,
             const int64_t* injected_cost, const int32_t* depth_of_target,
             int32_t* target, int64_t* row_cost, int64_t* info) {
    return orc_plan_rules(n, rowptr, colidx, level, m, kind, k, avg_override, cap_ratio, injected_cost,
                          depth_of_target, 0, 0, target, row_cost, info);
}

/* The planner with the per-row rules of Section III.A: a row may move only while its
 * dependency count after substitution is below alpha (alpha > 0) and its dependencies
 * lie within a distance beta of each other, max - min < beta (beta > 0: the
 * cache-locality constraint).  A row that breaks a rule is treated like one that does
 * not fit the cost: its level becomes the next target. */
int orc_plan_rules(int64_t n, const int32_t* rowptr, const int32_t* colidx, const int32_t* level,
                   int32_t m, int kind, int32_t k, double avg_override, double cap_ratio,
                   const int64_t* injected_cost, const int32_t* depth_of_target, int32_t alpha,
                   int64_t beta, int32_t* target, int64_t* row_cost, int64_t* info) {
    return orc_plan_parts(n, rowptr, colidx, level, m, kind, k, avg_override, cap_ratio, injected_cost,
                          depth_of_target, alpha, beta, 1, target, row_cost, info);
}

/* The walk started at several places at once (Section III: since emptied levels are removed only
 * when the process ends, the rewriting can also start at the end of the graph while it runs from
 * the beginning).  The levels are cut into `parts` consecutive ranges, range i = levels
 * [i*m/parts, (i+1)*m/parts); every range is walked by the rule above from a fresh start (no
 * target carried in), ranges in ascending order.  parts = 2 is the walk from both ends.  The nnz
 * cap's allowance, floor(cap*nnz(L)) - nnz(L), is shared: range i may add at most
 * allowance * nnz(rows of range i) / nnz(L) entries (integer division).  Substitution never
 * reaches below a target, so what a range decides does not depend on the other ranges. */
int orc_plan_parts(int64_t n, const int32_t* rowptr, const int32_t* colidx, const int32_t* level,
                   int32_t m, int kind, int32_t k, double avg_override, double cap_ratio,
                   const int64_t* injected_cost, const int32_t* depth_of_target, int32_t alpha,
                   int64_t beta, int32_t parts, int32_t* target, int64_t* row_cost, int64_t* info) {
    if (parts < 1) parts = 1;
    int64_t* lrows = (int64_t*)calloc((size_t)m + 1, sizeof(int64_t));
    int64_t* lcost = (int64_t*)calloc((size_t)m + 1, sizeof(int64_t));
    int64_t* lptr = (int64_t*)calloc((size_t)m + 2, sizeof(int64_t));
    int64_t* byl = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
    int32_t* curlev = (int32_t*)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
    iset* D = (iset*)calloc((size_t)(n > 0 ? n : 1), sizeof(iset));
    iset* E = (iset*)calloc((size_t)(n > 0 ? n : 1), sizeof(iset));
    if (!lrows || !lcost || !lptr || !byl || !curlev || !D || !E) return -1;

    int64_t nnzL = rowptr[n];
    for (int64_t i = 0; i < n; ++i) {
        int64_t z = (int64_t)rowptr[i + 1] - rowptr[i];
        lrows[level[i]] += 1;
        lcost[level[i]] += 2 * z - 1;
        row_cost[i] = 2 * z - 1;
        target[i] = level[i];
        curlev[i] = level[i];
        iset_reserve(&D[i], (int32_t)(z - 1));
        for (int64_t q = rowptr[i]; q < rowptr[i + 1] - 1; ++q) D[i].v[D[i].len++] = colidx[q];
        iset_add(&E[i], (int32_t)i);
    }
    /* rows bucketed by level, ascending row index within a level */
    for (int32_t l = 0; l < m; ++l) lptr[l + 1] = lptr[l] + lrows[l];
    {
        int64_t* fill = (int64_t*)malloc(sizeof(int64_t) * (size_t)(m + 1));
        for (int32_t l = 0; l <= m; ++l) fill[l] = lptr[l];
        for (int64_t i = 0; i < n; ++i) byl[fill[level[i]]++] = i;
        free(fill);
    }
    double total_cost = 0.0;
    for (int32_t l = 0; l < m; ++l) total_cost += (double)lcost[l];
    double avg = avg_override > 0.0 ? avg_override : (m > 0 ? total_cost / (double)m : 0.0);
    int64_t limit = cap_ratio > 0.0 ? (int64_t)floor(cap_ratio * (double)nnzL) : INT64_MAX;
    int64_t allowance = limit - nnzL; /* entries the whole plan may add */
    int64_t stored = nnzL; /* nnz(L') + nnz(E explicit rows) */
    int64_t moved = 0, targets = 0;

    iset Dn = {0}, En = {0};
    int32_t t = -1;
    int64_t cur = 0;
    int32_t part = -1;
    int64_t part_stored = 0, part_limit = INT64_MAX; /* growth of the current range and its share */
    for (int32_t s = 0; s < m; ++s) {
        if (part + 1 < parts && (int64_t)s == (int64_t)m * (part + 1) / parts) {
            /* a range starts (the last of several that start here when parts > m: the others are
             * empty): fresh walk, its share of the cap's allowance */
            while (part + 1 < parts && (int64_t)s == (int64_t)m * (part + 1) / parts) part++;
            t = -1;
            cur = 0;
            part_stored = 0;
            if (limit != INT64_MAX) {
                int64_t z = 0, lend = (int64_t)m * (part + 1) / parts;
                for (int64_t q = lptr[s]; q < lptr[lend]; ++q) {
                    int64_t r = byl[q];
                    z += (int64_t)rowptr[r + 1] - rowptr[r];
                }
                part_limit = nnzL > 0 ? allowance * z / nnzL : 0;
            }
        }
        int eligible = (kind == ORC_NAIVE || kind == ORC_MANUAL || kind == ORC_CHOSEN_THIN || kind == ORC_ROWCAP)
                           ? ((double)lcost[s] < avg) : 1;
        if (!eligible) { t = -1; continue; }
        if (t < 0) { t = s; cur = kind == ORC_ROWCAP ? (int64_t)(lptr[s + 1] - lptr[s]) : lcost[s]; targets++; continue; }
        if ((kind == ORC_DEPTH || kind == ORC_MANUAL) && s - t > k) { t = s; cur = lcost[s]; targets++; continue; }
        if ((kind == ORC_CHOSEN || kind == ORC_CHOSEN_THIN) && s - t > depth_of_target[t]) {
            t = s; cur = lcost[s]; targets++; continue;
        }
        for (int64_t q = lptr[s]; q < lptr[s + 1]; ++q) {
            int64_t r = byl[q];
            /* substitute every dependency on the target level or below it, until none
             * is left (one pass suffices: substituted equations only reach rows above
             * the target) */
            Dn.len = 0; En.len = 0;
            for (int32_t a = 0; a < D[r].len; ++a) iset_add(&Dn, D[r].v[a]);
            iset_add(&En, (int32_t)r);
            int changed = 1;
            while (changed) {
                changed = 0;
                for (int32_t a = 0; a < Dn.len; ++a) {
                    int32_t j = Dn.v[a];
                    if (curlev[j] >= t) {
                        memmove(Dn.v + a, Dn.v + a + 1, sizeof(int32_t) * (size_t)(Dn.len - a - 1));
                        Dn.len--;
                        for (int32_t b2 = 0; b2 < D[j].len; ++b2) iset_add(&Dn, D[j].v[b2]);
                        for (int32_t b2 = 0; b2 < E[j].len; ++b2) iset_add(&En, E[j].v[b2]);
                        changed = 1;
                        break;
                    }
                }
            }
            int64_t c = injected_cost ? injected_cost[r] : 2 * (int64_t)Dn.len;
            int64_t growth = (int64_t)Dn.len + (int64_t)En.len - (int64_t)D[r].len;
            int fits_cost = (kind == ORC_NAIVE) ? ((double)(cur + c) <= avg) : (kind == ORC_ROWCAP) ? (cur + 1 <= k) : 1;
            int fits_cap = limit == INT64_MAX || (part_stored + growth <= part_limit);
            int fits_rules = 1;
            if (alpha > 0 && Dn.len >= alpha) fits_rules = 0;
            if (beta > 0 && Dn.len > 1 && (int64_t)Dn.v[Dn.len - 1] - (int64_t)Dn.v[0] >= beta) fits_rules = 0;
            if (fits_cost && fits_cap && fits_rules) {
                target[r] = t;
                curlev[r] = t;
                row_cost[r] = c;
                cur += kind == ORC_ROWCAP ? 1 : c;
                stored += growth;
                part_stored += growth;
                moved++;
                iset tmp = D[r]; D[r] = Dn; Dn = tmp;
                tmp = E[r]; E[r] = En; En = tmp;
            } else {
                /* this level becomes the next target with the rows it still holds */
                t = s;
                targets++;
                cur = 0;
                for (int64_t q2 = lptr[s]; q2 < lptr[s + 1]; ++q2) {
                    int64_t r2 = byl[q2];
                    if (curlev[r2] == s) cur += kind == ORC_ROWCAP ? 1 : row_cost[r2];
                }
                break;
            }
        }
    }
    /* count non-empty levels after the moves */
    int64_t nonempty = 0;
    {
        char* used = (char*)calloc((size_t)m + 1, 1);
        for (int64_t i = 0; i < n; ++i) used[target[i]] = 1;
        for (int32_t l = 0; l < m; ++l) nonempty += used[l];
        free(used);
    }
    info[0] = moved;
    info[1] = stored;
    info[2] = nnzL;
    info[3] = nonempty;
    info[4] = (int64_t)llround(avg * 1e6);
    info[5] = targets;
    iset_free(&Dn); iset_free(&En);
    for (int64_t i = 0; i < n; ++i) { iset_free(&D[i]); iset_free(&E[i]); }
    free(D); free(E); free(lrows); free(lcost); free(lptr); free(byl); free(curlev);
    return 0;
}

/* ------------------------------------------------------------------------------- */
/* equation rewriting with rearrangement (Section II.B)                               */
/* ------------------------------------------------------------------------------- */

/* sparse accumulator: ascending columns with coefficients */
typedef struct { int32_t* c; double* v; int32_t len, cap; } sacc;

static void sacc_reserve(sacc* s, int32_t cap) {
    if (s->cap >= cap) return;
    int32_t nc = s->cap ? s->cap : 8;
    while (nc < cap) nc *= 2;
    s->c = (int32_t*)realloc(s->c, sizeof(int32_t) * (size_t)nc);
    s->v = (double*)realloc(s->v, sizeof(double) * (size_t)nc);
    s->cap = nc;
}

/* coefficient of column x += a; a new column is inserted even when a is zero, so the
 * structure is the symbolic union of the substituted equations */
static void sacc_add(sacc* s, int32_t x, double a) {
    int32_t lo = 0, hi = s->len;
    while (lo < hi) {
        int32_t mid = (lo + hi) / 2;
        if (s->c[mid] < x) lo = mid + 1; else hi = mid;
    }
    if (lo < s->len && s->c[lo] == x) { s->v[lo] += a; return; }
    sacc_reserve(s, s->len + 1);
    memmove(s->c + lo + 1, s->c + lo, sizeof(int32_t) * (size_t)(s->len - lo));
    memmove(s->v + lo + 1, s->v + lo, sizeof(double) * (size_t)(s->len - lo));
    s->c[lo] = x;
    s->v[lo] = a;
    s->len++;
}

static void sacc_remove_at(sacc* s, int32_t at) {
    memmove(s->c + at, s->c + at + 1, sizeof(int32_t) * (size_t)(s->len - at - 1));
    memmove(s->v + at, s->v + at + 1, sizeof(double) * (size_t)(s->len - at - 1));
    s->len--;
}

static void sacc_free(sacc* s) { free(s->c); free(s->v); s->c = NULL; s->v = NULL; s->len = s->cap = 0; }

/* Result of a rewrite: for every row r (original numbering)
 *   moved[r]            1 when r was rewritten to a higher level
 *   C row  cptr/ccol/cval  the coefficients of the unknowns x_k it still reads;
 *                        raw L_rk for rows that were not rewritten, rearranged c_rk for
 *                        rewritten rows
 *   dval[r]             L_rr for rows that were not rewritten, 1 for rewritten rows
 *                        (the division is folded into the coefficients)
 *   E row  eptr/ecol/eval  rewritten rows only: b'_r = sum_m e_rm b_m (diagonal e_rr
 *                        included); empty for the other rows
 * so that every row reads  x_r = (b'_r - sum_k c_rk x_k) / dval[r]  with b'_r = b_r
 * for rows that were not rewritten. */
typedef struct {
    int64_t n;
    int64_t *cptr, *eptr;
    int32_t *ccol, *ecol, *moved;
    double *cval, *eval, *dval;
} orc_system;

void orc_system_free(orc_system* s) {
    if (!s) return;
    free(s->cptr); free(s->eptr); free(s->ccol); free(s->ecol); free(s->moved);
    free(s->cval); free(s->eval); free(s->dval);
    free(s);
}

int64_t orc_system_nnz_c(const orc_system* s) { return s->cptr[s->n]; }
int64_t orc_system_nnz_e(const orc_system* s) { return s->eptr[s->n]; }

void orc_system_copy(const orc_system* s, int64_t* cptr, int32_t* ccol, double* cval, double* dval,
                     int64_t* eptr, int32_t* ecol, double* eval, int32_t* moved) {
    int64_t n = s->n;
    memcpy(cptr, s->cptr, sizeof(int64_t) * (size_t)(n + 1));
    memcpy(eptr, s->eptr, sizeof(int64_t) * (size_t)(n + 1));
    memcpy(ccol, s->ccol, sizeof(int32_t) * (size_t)s->cptr[n]);
    memcpy(cval, s->cval, sizeof(double) * (size_t)s->cptr[n]);
    memcpy(ecol, s->ecol, sizeof(int32_t) * (size_t)s->eptr[n]);
    memcpy(eval, s->eval, sizeof(double) * (size_t)s->eptr[n]);
    memcpy(dval, s->dval, sizeof(double) * (size_t)n);
    memcpy(moved, s->moved, sizeof(int32_t) * (size_t)n);
}

/*
 * Rewrite every row r whose target[r] is above its level: while its equation reads an
 * unknown x_j whose current level is >= target[r], replace x_j by x_j's own equation
 * (Fig. 2), then rearrange into the form x_r + sum_k c_rk x_k = sum_m e_rm b_m by
 * dividing through by L_rr.  Rows are processed in ascending index so that the
 * equation of every dependency is final when it is substituted.
 * Returns NULL on allocation failure.
 */
orc_system* orc_rewrite(int64_t n, const int32_t* rowptr, const int32_t* colidx,
                        const double* vals, const int32_t* level, const int32_t* target) {
    orc_system* S = (orc_system*)calloc(1, sizeof(orc_system));
    if (!S) return NULL;
    S->n = n;
    S->cptr = (int64_t*)calloc((size_t)n + 1, sizeof(int64_t));
    S->eptr = (int64_t*)calloc((size_t)n + 1, sizeof(int64_t));
    S->moved = (int32_t*)calloc((size_t)(n > 0 ? n : 1), sizeof(int32_t));
    S->dval = (double*)calloc((size_t)(n > 0 ? n : 1), sizeof(double));
    /* per-row storage while building (rows are read back when substituted) */
    sacc* C = (sacc*)calloc((size_t)(n > 0 ? n : 1), sizeof(sacc));
    sacc* Ev = (sacc*)calloc((size_t)(n > 0 ? n : 1), sizeof(sacc));
    if (!S->cptr || !S->eptr || !S->moved || !S->dval || !C || !Ev) return NULL;

    sacc a = {0}, f = {0};
    for (int64_t r = 0; r < n; ++r) {
        int64_t lo = rowptr[r], hi = (int64_t)rowptr[r + 1] - 1;
        double drr = vals[hi];
        if (target[r] >= level[r]) {
            /* row keeps its original equation */
            sacc_reserve(&C[r], (int32_t)(hi - lo));
            for (int64_t q = lo; q < hi; ++q) { C[r].c[C[r].len] = colidx[q]; C[r].v[C[r].len++] = vals[q]; }
            S->dval[r] = drr;
            continue;
        }
        int32_t t = target[r];
        a.len = 0; f.len = 0;
        for (int64_t q = lo; q < hi; ++q) sacc_add(&a, colidx[q], vals[q]);
        sacc_add(&f, (int32_t)r, 1.0);
        int changed = 1;
        while (changed) {
            changed = 0;
            for (int32_t p = 0; p < a.len; ++p) {
                int32_t j = a.c[p];
                if (target[j] < t) continue; /* current level of j is target[j] */
                double aj = a.v[p];
                sacc_remove_at(&a, p);
                /* x_j = (sum_m e_jm b_m - sum_k c_jk x_k) / dval_j, with e_jj = 1 for rows
                 * that kept their equation */
                double dj = S->dval[j];
                for (int32_t u = 0; u < C[j].len; ++u) sacc_add(&a, C[j].c[u], -aj * (C[j].v[u] / dj));
                if (S->moved[j]) {
                    for (int32_t u = 0; u < Ev[j].len; ++u) sacc_add(&f, Ev[j].c[u], -aj * Ev[j].v[u]);
                } else {
                    sacc_add(&f, j, -aj / dj);
                }
                changed = 1;
                break;
            }
        }
        /* rearrange: divide through by the diagonal */
        sacc_reserve(&C[r], a.len);
        for (int32_t p = 0; p < a.len; ++p) { C[r].c[p] = a.c[p]; C[r].v[p] = a.v[p] / drr; }
        C[r].len = a.len;
        sacc_reserve(&Ev[r], f.len);
        for (int32_t p = 0; p < f.len; ++p) { Ev[r].c[p] = f.c[p]; Ev[r].v[p] = f.v[p] / drr; }
        Ev[r].len = f.len;
        S->dval[r] = 1.0;
        S->moved[r] = 1;
    }
    sacc_free(&a); sacc_free(&f);
    for (int64_t r = 0; r < n; ++r) {
        S->cptr[r + 1] = S->cptr[r] + C[r].len;
        S->eptr[r + 1] = S->eptr[r] + (S->moved[r] ? Ev[r].len : 0);
    }
    S->ccol = (int32_t*)malloc(sizeof(int32_t) * (size_t)(S->cptr[n] + 1));
    S->cval = (double*)malloc(sizeof(double) * (size_t)(S->cptr[n] + 1));
    S->ecol = (int32_t*)malloc(sizeof(int32_t) * (size_t)(S->eptr[n] + 1));
    S->eval = (double*)malloc(sizeof(double) * (size_t)(S->eptr[n] + 1));
    if (!S->ccol || !S->cval || !S->ecol || !S->eval) return NULL;
    for (int64_t r = 0; r < n; ++r) {
        memcpy(S->ccol + S->cptr[r], C[r].c, sizeof(int32_t) * (size_t)C[r].len);
        memcpy(S->cval + S->cptr[r], C[r].v, sizeof(double) * (size_t)C[r].len);
        if (S->moved[r]) {
            memcpy(S->ecol + S->eptr[r], Ev[r].c, sizeof(int32_t) * (size_t)Ev[r].len);
            memcpy(S->eval + S->eptr[r], Ev[r].v, sizeof(double) * (size_t)Ev[r].len);
        }
        sacc_free(&C[r]);
        sacc_free(&Ev[r]);
    }
    free(C); free(Ev);
    return S;
}

/* Levels of a rewritten system: rows whose equations read no unknown are on level 0,
 * any other row one level below its deepest remaining dependency. */
int32_t orc_system_levels(const orc_system* s, int32_t* level) {
    int32_t m = 0;
    for (int64_t i = 0; i < s->n; ++i) {
        int32_t lv = 0;
        for (int64_t q = s->cptr[i]; q < s->cptr[i + 1]; ++q) {
            int32_t d = level[s->ccol[q]] + 1;
            if (d > lv) lv = d;
        }
        level[i] = lv;
        if (lv + 1 > m) m = lv + 1;
    }
    return s->n > 0 ? m : 0;
}

/* Forward substitution of the rewritten equations for one right-hand side. */
void orc_solve_rewritten(const orc_system* s, const double* b, double* x) {
    for (int64_t r = 0; r < s->n; ++r) {
        double rhs;
        if (s->moved[r]) {
            rhs = 0.0;
            for (int64_t q = s->eptr[r]; q < s->eptr[r + 1]; ++q) rhs += s->eval[q] * b[s->ecol[q]];
        } else {
            rhs = b[r];
        }
        double sum = 0.0;
        for (int64_t q = s->cptr[r]; q < s->cptr[r + 1]; ++q) sum += s->cval[q] * x[s->ccol[q]];
        x[r] = (rhs - sum) / s->dval[r];
    }
}

/* ------------------------------------------------------------------------------- */
/* backward substitution (upper-triangular U x = b, diagonal FIRST in each row)      */
/* ------------------------------------------------------------------------------- */

/* x_i = (b_i - sum_{j>i} U_ij x_j) / U_ii for i = n-1 down to 0. */
void orc_backward_subst(int64_t n, const int32_t* rowptr, const int32_t* colidx, const double* vals,
                        const double* b, double* x) {
    for (int64_t i = n - 1; i >= 0; --i) {
        double sum = 0.0;
        int64_t first = rowptr[i];
        for (int64_t j = first + 1; j < rowptr[i + 1]; ++j) sum += vals[j] * x[colidx[j]];
        x[i] = (b[i] - sum) / vals[first];
    }
}
