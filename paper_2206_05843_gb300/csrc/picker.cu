// picker.cu -- the learned rewrite picker: features, MLP inference and training kernels,
// and the learned strategy (predicted solve-time change -> depth per target level).
//
// The paper leaves the choice of rows and rewriting distance to a fixed rule and names a
// learned strategy as future work (Conclusion).  Here a small MLP (12 -> 64 -> 64 -> 64 ->
// 1, ReLU, bfloat16 weights, float32 accumulation) predicts the change in solve time of
// rewriting the g levels after a target level t into t; the planner then walks the levels
// and gives each target the depth with the lowest prediction (0 when none is negative),
// under the same nnz cap as the naive strategy.
#include <cuda_bf16.h>

#include <cmath>
#include <cstdio>
#include <cstring>
#include <random>
#include <string>
#include <thread>
#include <vector>

#include "system.cuh"

namespace sp {
namespace {

constexpr int NF = SPTRSV_PICKER_FEATURES;  // 12
constexpr int NH = SPTRSV_PICKER_HIDDEN;    // 64
constexpr int NP = SPTRSV_PICKER_PARAMS;    // 9217
constexpr int OW1 = 0, OB1 = OW1 + NH * NF, OW2 = OB1 + NH, OB2 = OW2 + NH * NH, OW3 = OB2 + NH,
              OB3 = OW3 + NH * NH, OW4 = OB3 + NH, OB4 = OW4 + NH;
constexpr int ACT = NF + 3 * NH;  // stored activations per sample: x0, h1, h2, h3
constexpr int DZ = 3 * NH + 1;    // stored gradients per sample: dz1, dz2, dz3, dy

inline unsigned nblk(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

// ---------------------------------------------------------------------------------
// features
// ---------------------------------------------------------------------------------

__global__ void k_level_aggr(int64_t n, const int32_t* rowptr, const int32_t* colidx, const int32_t* level,
                             int* maxdeg, unsigned long long* twohop) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int64_t a = rowptr[i], e = (int64_t)rowptr[i + 1] - 1;
    int64_t two = 0;
    for (int64_t q = a; q < e; ++q) {
        const int32_t j = colidx[q];
        two += (int64_t)rowptr[j + 1] - rowptr[j] - 1;
    }
    const int l = level[i];
    atomicMax(maxdeg + l, (int)(e - a));
    atomicAdd(twohop + l, (unsigned long long)two);
}

__global__ void k_thin_flags(int64_t m, const int64_t* cost, double avg, int64_t* thin) {
    int64_t l = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (l < m) thin[l] = (double)cost[l] < avg ? 1 : 0;
}

struct FeatArgs {
    int64_t m;
    const int64_t *prow, *pnnz, *pcost, *ptwo, *pthin;  // exclusive prefix sums over levels (m+1)
    const int64_t* rows;
    const int* maxdeg;
    const int32_t* depths;
    int nd;
    double avg;
    float* out;
    int32_t* gsel;  // depth each candidate resolves to (may be null)
};

// A candidate is a depth g >= 1 or a row budget -r: the largest depth whose window t..t+g holds at
// most r rows (0 when level t alone holds more) -- a binary search on the level-row prefix sums
__device__ int candidate_depth(const int64_t* prow, int64_t m, int64_t t, int c) {
    if (c >= 1) return c;
    const int64_t r = -(int64_t)c;
    if (prow[t + 1] - prow[t] > r) return 0;
    int64_t lo = t, hi = m - 1;  // largest e in [t, m-1] with prow[e+1] - prow[t] <= r
    while (lo < hi) {
        const int64_t mid = (lo + hi + 1) >> 1;
        if (prow[mid + 1] - prow[t] <= r) lo = mid;
        else hi = mid - 1;
    }
    return (int)(lo - t);
}

__global__ void k_features(FeatArgs a) {
    int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= a.m * a.nd) return;
    const int64_t t = idx / a.nd;
    const int g = candidate_depth(a.prow, a.m, t, a.depths[idx % a.nd]);
    if (a.gsel) a.gsel[idx] = g;
    const int64_t te = min(t + (int64_t)g, a.m - 1);
    auto sum = [&](const int64_t* p, int64_t lo, int64_t hi) { return hi >= lo ? p[hi + 1] - p[lo] : (int64_t)0; };
    const double rW = (double)sum(a.prow, t, te), nW = (double)sum(a.pnnz, t, te);
    const double rS = (double)sum(a.prow, t + 1, te), nS = (double)sum(a.pnnz, t + 1, te);
    int mx = 0;
    for (int64_t l = t + 1; l <= te; ++l) mx = max(mx, a.maxdeg[l]);
    float* f = a.out + idx * NF;
    f[0] = (float)log2(1.0 + g);
    f[1] = (float)log2(1.0 + rW);
    f[2] = (float)log2(1.0 + nW);
    f[3] = (float)log2(1.0 + rS / (double)(te - t > 1 ? te - t : 1));
    f[4] = (float)((nS - rS) / fmax(1.0, rS));
    f[5] = (float)mx;
    f[6] = (float)log2(1.0 + (double)sum(a.ptwo, t + 1, te));
    f[7] = (float)log2(1.0 + (double)a.rows[t]);
    f[8] = t > 0 ? (float)log2(1.0 + (double)a.rows[t - 1]) : 0.0f;
    f[9] = te + 1 < a.m ? (float)log2(1.0 + (double)a.rows[te + 1]) : 0.0f;
    f[10] = (float)((double)sum(a.pcost, t, te) / a.avg);
    f[11] = (float)((double)sum(a.pthin, t, te) / (double)(te - t + 1));
}

// ---------------------------------------------------------------------------------
// MLP
// ---------------------------------------------------------------------------------

// parameters into shared memory as float (bfloat16 weights are widened exactly)
template <bool BF16>
__device__ void load_params(float* sp, const float* p32, const __nv_bfloat16* p16) {
    for (int i = threadIdx.x; i < NP; i += blockDim.x) sp[i] = BF16 ? __bfloat162float(p16[i]) : p32[i];
    __syncthreads();
}

template <bool BF16>
__global__ void __launch_bounds__(128) k_mlp_forward(const float* p32, const __nv_bfloat16* p16, const float* norm,
                                                     const float* X, int64_t N, float* y, float* act) {
    extern __shared__ float sp[];
    load_params<BF16>(sp, p32, p16);
    for (int64_t n = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; n < N; n += (int64_t)gridDim.x * blockDim.x) {
        float x0[NF], h1[NH], h2[NH];
#pragma unroll
        for (int i = 0; i < NF; ++i) x0[i] = (X[n * NF + i] - norm[i]) / norm[NF + i];
#pragma unroll
        for (int j = 0; j < NH; ++j) {
            float z = sp[OB1 + j];
#pragma unroll
            for (int i = 0; i < NF; ++i) z = fmaf(sp[OW1 + j * NF + i], x0[i], z);
            h1[j] = fmaxf(z, 0.0f);
        }
#pragma unroll
        for (int j = 0; j < NH; ++j) {
            float z = sp[OB2 + j];
#pragma unroll
            for (int i = 0; i < NH; ++i) z = fmaf(sp[OW2 + j * NH + i], h1[i], z);
            h2[j] = fmaxf(z, 0.0f);
        }
        float out = sp[OB4];
        if (act) {
            float* A = act + n * ACT;
            for (int i = 0; i < NF; ++i) A[i] = x0[i];
            for (int i = 0; i < NH; ++i) A[NF + i] = h1[i];
            for (int i = 0; i < NH; ++i) A[NF + NH + i] = h2[i];
        }
#pragma unroll
        for (int j = 0; j < NH; ++j) {
            float z = sp[OB3 + j];
#pragma unroll
            for (int i = 0; i < NH; ++i) z = fmaf(sp[OW3 + j * NH + i], h2[i], z);
            const float h3 = fmaxf(z, 0.0f);
            out = fmaf(sp[OW4 + j], h3, out);
            if (act) act[n * ACT + NF + 2 * NH + j] = h3;
        }
        y[n] = out;
    }
}

// per-sample backward: dz for every hidden layer and dy
template <bool BF16>
__global__ void __launch_bounds__(128) k_mlp_backward_rows(const float* p32, const __nv_bfloat16* p16, const float* norm,
                                                           const float* y, const float* target, int64_t N,
                                                           const float* act, float* dz, float* resid2) {
    extern __shared__ float sp[];
    load_params<BF16>(sp, p32, p16);
    const float ts = norm[2 * NF];
    for (int64_t n = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; n < N; n += (int64_t)gridDim.x * blockDim.x) {
        const float* A = act + n * ACT;
        const float r = y[n] - target[n] / ts;
        resid2[n] = r * r;
        const float dy = 2.0f * r / (float)N;
        float dz3[NH];
        float* D = dz + n * DZ;
#pragma unroll
        for (int i = 0; i < NH; ++i) {
            dz3[i] = A[NF + 2 * NH + i] > 0.0f ? dy * sp[OW4 + i] : 0.0f;
            D[2 * NH + i] = dz3[i];
        }
#pragma unroll 1
        for (int j = 0; j < NH; ++j) {
            float s = 0.0f;
#pragma unroll
            for (int i = 0; i < NH; ++i) s = fmaf(dz3[i], sp[OW3 + i * NH + j], s);
            D[NH + j] = A[NF + NH + j] > 0.0f ? s : 0.0f;  // dz2
        }
        float dz2[NH];
#pragma unroll
        for (int i = 0; i < NH; ++i) dz2[i] = D[NH + i];
#pragma unroll 1
        for (int j = 0; j < NH; ++j) {
            float s = 0.0f;
#pragma unroll
            for (int i = 0; i < NH; ++i) s = fmaf(dz2[i], sp[OW2 + i * NH + j], s);
            D[j] = A[NF + j] > 0.0f ? s : 0.0f;  // dz1
        }
        D[3 * NH] = dy;
    }
}

// gradient of every parameter: a sum over the samples in a fixed order (deterministic)
__global__ void k_mlp_param_grads(int64_t N, const float* act, const float* dz, float* grad) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= NP) return;
    int dz_off, a_off;  // dz column and activation column (-1: bias)
    if (k < OB1) { dz_off = k / NF; a_off = k % NF; }
    else if (k < OW2) { dz_off = k - OB1; a_off = -1; }
    else if (k < OB2) { dz_off = NH + (k - OW2) / NH; a_off = NF + (k - OW2) % NH; }
    else if (k < OW3) { dz_off = NH + (k - OB2); a_off = -1; }
    else if (k < OB3) { dz_off = 2 * NH + (k - OW3) / NH; a_off = NF + NH + (k - OW3) % NH; }
    else if (k < OW4) { dz_off = 2 * NH + (k - OB3); a_off = -1; }
    else if (k < OB4) { dz_off = 3 * NH; a_off = NF + 2 * NH + (k - OW4); }
    else { dz_off = 3 * NH; a_off = -1; }
    float s = 0.0f;
    for (int64_t n = 0; n < N; ++n) {
        const float d = dz[n * DZ + dz_off];
        s = a_off < 0 ? s + d : fmaf(d, act[n * ACT + a_off], s);
    }
    grad[k] = s;
}

__global__ void k_sum_mean(const float* v, int64_t N, float* out) {
    __shared__ float red[256];
    float s = 0.0f;
    for (int64_t i = threadIdx.x; i < N; i += blockDim.x) s += v[i];
    red[threadIdx.x] = s;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = red[0] / (float)N;
}

__global__ void k_adam(float* p, float* m, float* v, const float* g, __nv_bfloat16* p16, float lr, float c1, float c2) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= NP) return;
    const float gk = g[k];
    const float mk = 0.9f * m[k] + 0.1f * gk;
    const float vk = 0.999f * v[k] + 0.001f * gk * gk;
    m[k] = mk;
    v[k] = vk;
    const float pk = p[k] - lr * (mk / c1) / (sqrtf(vk / c2) + 1e-8f);
    p[k] = pk;
    p16[k] = __float2bfloat16_rn(pk);
}

__global__ void k_to_bf16(const float* p, __nv_bfloat16* p16) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < NP) p16[k] = __float2bfloat16_rn(p[k]);
}

// depth per level: the candidate with the lowest predicted change, 0 if none is negative
// (gsel: the depth each candidate resolves to)
__global__ void k_choose_depths(int64_t m, const float* pred, const int32_t* gsel, int nd, int32_t* dot) {
    int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= m) return;
    int best = 0;
    float bv = 0.0f;
    for (int d = 0; d < nd; ++d) {
        const float v = pred[t * nd + d];
        if (v < bv) {
            bv = v;
            best = gsel[t * nd + d];
        }
    }
    dot[t] = best;
}

// fixed depths and row budgets (negative: a target takes levels while it holds at most r rows)
constexpr int DEFAULT_DEPTHS[] = {1, 2, 4, 8, 16, 32, -16, -32, -64};

}  // namespace
}  // namespace sp

using namespace sp;

struct sptrsv_picker {
    DevBuf<float> p, m, v, norm, grad, loss;
    DevBuf<__nv_bfloat16> p16;
    int64_t step = 0;
    float h_norm[2 * NF + 1];
};

namespace sp {
namespace {

sptrsv_status upload_norm(sptrsv_picker* pk) {
    SP_CUDA(cudaMemcpy(pk->norm.p, pk->h_norm, sizeof(pk->h_norm), cudaMemcpyHostToDevice));
    return SPTRSV_OK;
}

size_t param_smem() { return (size_t)NP * sizeof(float); }

sptrsv_status forward(const sptrsv_picker* pk, const float* X, int64_t N, float* y, float* act, int bf16,
                      cudaStream_t st) {
    const size_t sm = param_smem();
    unsigned grid = (unsigned)std::min<int64_t>(nblk(N, 128), (int64_t)device_sm_count() * 8);
    if (grid == 0) return SPTRSV_OK;
    if (bf16) {
        SP_CUDA(cudaFuncSetAttribute(k_mlp_forward<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
        k_mlp_forward<true><<<grid, 128, sm, st>>>(pk->p.p, pk->p16.p, pk->norm.p, X, N, y, act);
    } else {
        SP_CUDA(cudaFuncSetAttribute(k_mlp_forward<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
        k_mlp_forward<false><<<grid, 128, sm, st>>>(pk->p.p, pk->p16.p, pk->norm.p, X, N, y, act);
    }
    SP_CUDA(cudaGetLastError());
    return SPTRSV_OK;
}

sptrsv_status grad_impl(const sptrsv_picker* pk, const float* X, const float* t, int64_t N, int bf16, float* grad,
                        float* loss, cudaStream_t st) {
    if (N <= 0) { set_error("picker: empty batch"); return SPTRSV_ERR_INVALID; }
    Scratch y, act, dz, r2;
    SP_TRY(y.alloc(N * 4, st));
    SP_TRY(act.alloc(N * ACT * 4, st));
    SP_TRY(dz.alloc(N * DZ * 4, st));
    SP_TRY(r2.alloc(N * 4, st));
    SP_TRY(forward(pk, X, N, y.as<float>(), act.as<float>(), bf16, st));
    const size_t sm = param_smem();
    unsigned grid = (unsigned)std::min<int64_t>(nblk(N, 128), (int64_t)device_sm_count() * 8);
    if (bf16) {
        SP_CUDA(cudaFuncSetAttribute(k_mlp_backward_rows<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
        k_mlp_backward_rows<true><<<grid, 128, sm, st>>>(pk->p.p, pk->p16.p, pk->norm.p, y.as<float>(), t, N,
                                                         act.as<float>(), dz.as<float>(), r2.as<float>());
    } else {
        SP_CUDA(cudaFuncSetAttribute(k_mlp_backward_rows<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
        k_mlp_backward_rows<false><<<grid, 128, sm, st>>>(pk->p.p, pk->p16.p, pk->norm.p, y.as<float>(), t, N,
                                                          act.as<float>(), dz.as<float>(), r2.as<float>());
    }
    k_mlp_param_grads<<<nblk(NP, 128), 128, 0, st>>>(N, act.as<float>(), dz.as<float>(), grad);
    if (loss) k_sum_mean<<<1, 256, 0, st>>>(r2.as<float>(), N, loss);
    SP_CUDA(cudaGetLastError());
    return SPTRSV_OK;
}

// per-level aggregates, prefix sums and the feature kernel
sptrsv_status features_impl(const sptrsv_csr* L, const Levels& lv, const int32_t* depths_host, int nd, float* out,
                            int32_t* gsel, cudaStream_t st) {
    const int64_t n = L->n, m = lv.m;
    if (m == 0) return SPTRSV_OK;
    Scratch maxdeg, two, thin, pre, dep;
    SP_TRY(maxdeg.alloc(m * 4, st));
    SP_TRY(two.alloc(m * 8, st));
    SP_TRY(thin.alloc(m * 8, st));
    SP_TRY(pre.alloc(5 * (m + 1) * 8, st));
    SP_TRY(dep.alloc(nd * 4, st));
    SP_CUDA(cudaMemsetAsync(maxdeg.p, 0, m * 4, st));
    SP_CUDA(cudaMemsetAsync(two.p, 0, m * 8, st));
    SP_CUDA(cudaMemcpyAsync(dep.p, depths_host, nd * 4, cudaMemcpyHostToDevice, st));
    k_level_aggr<<<nblk(n, 256), 256, 0, st>>>(n, L->rowptr, L->colidx, lv.level.p, maxdeg.as<int>(),
                                                two.as<unsigned long long>());
    k_thin_flags<<<nblk(m, 256), 256, 0, st>>>(m, lv.lcost.p, lv.avg, thin.as<int64_t>());
    SP_CUDA(cudaGetLastError());
    int64_t* P = pre.as<int64_t>();
    SP_TRY(scan_exclusive_i64(lv.lrows.p, P, m, st));
    SP_TRY(scan_exclusive_i64(lv.lnnz.p, P + (m + 1), m, st));
    SP_TRY(scan_exclusive_i64(lv.lcost.p, P + 2 * (m + 1), m, st));
    SP_TRY(scan_exclusive_i64(two.as<int64_t>(), P + 3 * (m + 1), m, st));
    SP_TRY(scan_exclusive_i64(thin.as<int64_t>(), P + 4 * (m + 1), m, st));
    FeatArgs a;
    a.m = m;
    a.prow = P;
    a.pnnz = P + (m + 1);
    a.pcost = P + 2 * (m + 1);
    a.ptwo = P + 3 * (m + 1);
    a.pthin = P + 4 * (m + 1);
    a.rows = lv.lrows.p;
    a.maxdeg = maxdeg.as<int>();
    a.depths = dep.as<int32_t>();
    a.nd = nd;
    a.avg = lv.avg;
    a.out = out;
    a.gsel = gsel;
    k_features<<<nblk(m * nd, 256), 256, 0, st>>>(a);
    SP_CUDA(cudaGetLastError());
    SP_CUDA(cudaStreamSynchronize(st));  // the scratch above is released after the kernel
    return SPTRSV_OK;
}

}  // namespace

sptrsv_status learned_rewrite(const sptrsv_csr* L, const sptrsv_levels* lvh, const sptrsv_strategy* sg,
                              sptrsv_system** out, cudaStream_t st) {
    const Levels& lv = lvh->lv;
    const int32_t* depths = sg->depths_host && sg->n_depths > 0 ? sg->depths_host : DEFAULT_DEPTHS;
    const int nd = sg->depths_host && sg->n_depths > 0 ? sg->n_depths : (int)(sizeof(DEFAULT_DEPTHS) / sizeof(int));
    const int64_t m = lv.m;
    Scratch feat, pred, dot, gsel;
    SP_TRY(feat.alloc(std::max<int64_t>(1, m * nd) * NF * 4, st));
    SP_TRY(pred.alloc(std::max<int64_t>(1, m * nd) * 4, st));
    SP_TRY(dot.alloc(std::max<int64_t>(1, m) * 4, st));
    SP_TRY(gsel.alloc(std::max<int64_t>(1, m * nd) * 4, st));
    SP_TRY(features_impl(L, lv, depths, nd, feat.as<float>(), gsel.as<int32_t>(), st));
    SP_TRY(forward(sg->picker, feat.as<float>(), m * nd, pred.as<float>(), nullptr, 1, st));
    if (m > 0) k_choose_depths<<<nblk(m, 256), 256, 0, st>>>(m, pred.as<float>(), gsel.as<int32_t>(), nd, dot.as<int32_t>());
    SP_CUDA(cudaGetLastError());
    if (sg->learned_mode == 1) {
        sptrsv_system* model = nullptr;
        SP_TRY(rewrite_system(L, lv, 5 /* depth per thin target */, 0, dot.as<int32_t>(), sg->avg_override,
                              sg->nnz_growth_cap, sg->growth_guard, nullptr, sg->max_deps, sg->max_spread,
                              sg->walk_parts, &model, st));
        model->strategy_used = SPTRSV_STRATEGY_CHOSEN;
        *out = model;
        return SPTRSV_OK;
    }
    // Candidates: the model's plan, the paper's naive strategy, the plan shaped for the fast executor
    // (targets of at most one warp's rows) and no rewrite; the measured solve time decides.  The three
    // plans are independent (each planner walk is one warp for the length of the level sequence), so
    // they are built at the same time, each by a host thread on a stream of its own.
    constexpr int NC = 4;
    sptrsv_system* cand[NC] = {nullptr, nullptr, nullptr, nullptr};
    sptrsv_status crc[NC] = {SPTRSV_OK, SPTRSV_OK, SPTRSV_OK, SPTRSV_OK};
    std::string cerr[NC];
    int dev = 0;
    SP_CUDA(cudaGetDevice(&dev));
    cudaEvent_t ready;
    SP_CUDA(cudaEventCreateWithFlags(&ready, cudaEventDisableTiming));
    SP_CUDA(cudaEventRecord(ready, st));  // the depths per target are on `st`
    const int kinds[3] = {5 /* depth per thin target */, 1 /* naive */, 6 /* rowcap */};
    const int used[3] = {SPTRSV_STRATEGY_CHOSEN, SPTRSV_STRATEGY_NAIVE, SPTRSV_STRATEGY_ROWCAP};
    std::vector<std::thread> workers;
    for (int i = 0; i < 3; ++i) {
        workers.emplace_back([&, i]() {
            cudaStream_t ws = nullptr;
            sptrsv_status rc = SPTRSV_OK;
            if (cudaSetDevice(dev) != cudaSuccess || cudaStreamCreateWithFlags(&ws, cudaStreamNonBlocking) != cudaSuccess ||
                cudaStreamWaitEvent(ws, ready, 0) != cudaSuccess) {
                set_error("learned strategy: stream setup failed");
                rc = SPTRSV_ERR_CUDA;
            } else {
                rc = rewrite_system(L, lv, kinds[i], kinds[i] == 6 ? ROWCAP_DEFAULT_ROWS : 0,
                                    kinds[i] == 5 ? dot.as<int32_t>() : nullptr, sg->avg_override, sg->nnz_growth_cap,
                                    sg->growth_guard, nullptr, sg->max_deps, sg->max_spread, sg->walk_parts, &cand[i],
                                    ws);
                if (rc == SPTRSV_OK && cudaStreamSynchronize(ws) != cudaSuccess) {
                    set_error("learned strategy: candidate plan failed");
                    rc = SPTRSV_ERR_CUDA;
                }
            }
            if (ws) cudaStreamDestroy(ws);
            crc[i] = rc;
            if (rc != SPTRSV_OK) cerr[i] = get_error();
            else cand[i]->strategy_used = used[i];
        });
    }
    crc[3] = sptrsv_system_plain(L, lvh, &cand[3], st);
    if (crc[3] == SPTRSV_OK) cand[3]->strategy_used = SPTRSV_STRATEGY_NONE;
    else cerr[3] = get_error();
    for (auto& w : workers) w.join();
    cudaEventDestroy(ready);
    sptrsv_status rc = SPTRSV_OK;
    for (int i = 0; i < NC; ++i)
        if (crc[i] != SPTRSV_OK && rc == SPTRSV_OK) {
            rc = crc[i];
            set_error("%s", cerr[i].c_str());
        }
    if (rc != SPTRSV_OK) {
        for (sptrsv_system* c : cand)
            if (c) sptrsv_system_destroy(c);
        return rc;
    }
    double t[NC] = {0, 0, 0, 0};
    for (int i = 0; i < NC && rc == SPTRSV_OK; ++i) rc = time_solve_us(cand[i], 5, &t[i], st);
    if (rc != SPTRSV_OK) {
        for (sptrsv_system* c : cand) sptrsv_system_destroy(c);
        return rc;
    }
    int best = 0;
    for (int i = 1; i < NC; ++i)
        if (t[i] < t[best]) best = i;
    for (int i = 0; i < NC; ++i)
        if (i != best) sptrsv_system_destroy(cand[i]);
    for (int i = 0; i < NC; ++i) cand[best]->cand_us[i] = t[i];
    *out = cand[best];
    return SPTRSV_OK;
}

}  // namespace sp

extern "C" {

sptrsv_status sptrsv_picker_create(uint64_t seed, sptrsv_picker** out) {
    if (!out) { set_error("picker_create: null output"); return SPTRSV_ERR_INVALID; }
    *out = nullptr;
    sptrsv_picker* pk = new (std::nothrow) sptrsv_picker();
    if (!pk) { set_error("host allocation failed"); return SPTRSV_ERR_OOM; }
    auto fail = [&](sptrsv_status rc) {
        delete pk;
        return rc;
    };
    sptrsv_status rc;
    if ((rc = pk->p.alloc(NP)) || (rc = pk->m.alloc(NP)) || (rc = pk->v.alloc(NP)) || (rc = pk->grad.alloc(NP)) ||
        (rc = pk->norm.alloc(2 * NF + 1)) || (rc = pk->loss.alloc(1)) || (rc = pk->p16.alloc(NP)))
        return fail(rc);
    // Kaiming-uniform weights, zero biases, from a seeded generator
    std::vector<float> h(NP, 0.0f);
    std::mt19937_64 gen(seed);
    auto fill = [&](int off, int fan_out, int fan_in) {
        std::uniform_real_distribution<double> u(-std::sqrt(6.0 / fan_in), std::sqrt(6.0 / fan_in));
        for (int i = 0; i < fan_out * fan_in; ++i) h[off + i] = (float)u(gen);
    };
    fill(OW1, NH, NF);
    fill(OW2, NH, NH);
    fill(OW3, NH, NH);
    fill(OW4, 1, NH);
    if (cudaMemcpy(pk->p.p, h.data(), NP * 4, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemset(pk->m.p, 0, NP * 4) != cudaSuccess || cudaMemset(pk->v.p, 0, NP * 4) != cudaSuccess)
        return fail((set_error("picker_create: copy failed"), SPTRSV_ERR_CUDA));
    for (int i = 0; i < NF; ++i) {
        pk->h_norm[i] = 0.0f;
        pk->h_norm[NF + i] = 1.0f;
    }
    pk->h_norm[2 * NF] = 1.0f;
    if ((rc = upload_norm(pk)) != SPTRSV_OK) return fail(rc);
    k_to_bf16<<<nblk(NP, 256), 256>>>(pk->p.p, pk->p16.p);
    if (cudaDeviceSynchronize() != cudaSuccess) return fail((set_error("picker_create: kernel failed"), SPTRSV_ERR_CUDA));
    *out = pk;
    return SPTRSV_OK;
}

void sptrsv_picker_destroy(sptrsv_picker* pk) { delete pk; }

sptrsv_status sptrsv_picker_get_params(const sptrsv_picker* pk, float* params) {
    if (!pk || !params) { set_error("picker_get_params: null argument"); return SPTRSV_ERR_INVALID; }
    SP_CUDA(cudaDeviceSynchronize());
    SP_CUDA(cudaMemcpy(params, pk->p.p, NP * 4, cudaMemcpyDeviceToHost));
    return SPTRSV_OK;
}

sptrsv_status sptrsv_picker_set_params(sptrsv_picker* pk, const float* params) {
    if (!pk || !params) { set_error("picker_set_params: null argument"); return SPTRSV_ERR_INVALID; }
    SP_CUDA(cudaDeviceSynchronize());
    SP_CUDA(cudaMemcpy(pk->p.p, params, NP * 4, cudaMemcpyHostToDevice));
    k_to_bf16<<<nblk(NP, 256), 256>>>(pk->p.p, pk->p16.p);
    SP_CUDA(cudaDeviceSynchronize());
    return SPTRSV_OK;
}

sptrsv_status sptrsv_picker_set_norm(sptrsv_picker* pk, const float* mean, const float* stdv, float target_scale) {
    if (!pk || !mean || !stdv || !(target_scale > 0)) { set_error("picker_set_norm: bad argument"); return SPTRSV_ERR_INVALID; }
    for (int i = 0; i < NF; ++i) {
        if (!(stdv[i] > 0)) { set_error("picker_set_norm: std must be positive"); return SPTRSV_ERR_INVALID; }
        pk->h_norm[i] = mean[i];
        pk->h_norm[NF + i] = stdv[i];
    }
    pk->h_norm[2 * NF] = target_scale;
    SP_CUDA(cudaDeviceSynchronize());
    return upload_norm(pk);
}

sptrsv_status sptrsv_picker_save(const sptrsv_picker* pk, const char* path) {
    if (!pk || !path) { set_error("picker_save: null argument"); return SPTRSV_ERR_INVALID; }
    std::vector<float> p(NP), m(NP), v(NP);
    SP_CUDA(cudaDeviceSynchronize());
    SP_CUDA(cudaMemcpy(p.data(), pk->p.p, NP * 4, cudaMemcpyDeviceToHost));
    SP_CUDA(cudaMemcpy(m.data(), pk->m.p, NP * 4, cudaMemcpyDeviceToHost));
    SP_CUDA(cudaMemcpy(v.data(), pk->v.p, NP * 4, cudaMemcpyDeviceToHost));
    FILE* f = fopen(path, "wb");
    if (!f) { set_error("picker_save: cannot open %s", path); return SPTRSV_ERR_INVALID; }
    fprintf(f, "SPTRSV-PICKER 1 features %d hidden %d params %d step %lld\n", NF, NH, NP, (long long)pk->step);
    bool ok = fwrite(pk->h_norm, sizeof(float), 2 * NF + 1, f) == (size_t)(2 * NF + 1) &&
              fwrite(p.data(), 4, NP, f) == (size_t)NP && fwrite(m.data(), 4, NP, f) == (size_t)NP &&
              fwrite(v.data(), 4, NP, f) == (size_t)NP;
    ok = (fclose(f) == 0) && ok;
    if (!ok) { set_error("picker_save: write failed"); return SPTRSV_ERR_INVALID; }
    return SPTRSV_OK;
}

sptrsv_status sptrsv_picker_load(sptrsv_picker* pk, const char* path) {
    if (!pk || !path) { set_error("picker_load: null argument"); return SPTRSV_ERR_INVALID; }
    FILE* f = fopen(path, "rb");
    if (!f) { set_error("picker_load: cannot open %s", path); return SPTRSV_ERR_INVALID; }
    int nf = 0, nh = 0, np = 0;
    long long step = 0;
    char line[256];
    bool ok = fgets(line, sizeof(line), f) &&
              sscanf(line, "SPTRSV-PICKER 1 features %d hidden %d params %d step %lld", &nf, &nh, &np, &step) == 4 &&
              nf == NF && nh == NH && np == NP;
    std::vector<float> norm(2 * NF + 1), p(NP), m(NP), v(NP);
    ok = ok && fread(norm.data(), 4, 2 * NF + 1, f) == (size_t)(2 * NF + 1) && fread(p.data(), 4, NP, f) == (size_t)NP &&
         fread(m.data(), 4, NP, f) == (size_t)NP && fread(v.data(), 4, NP, f) == (size_t)NP;
    fclose(f);
    if (!ok) { set_error("picker_load: %s is not a picker file of this architecture", path); return SPTRSV_ERR_INVALID; }
    memcpy(pk->h_norm, norm.data(), sizeof(pk->h_norm));
    pk->step = step;
    SP_CUDA(cudaDeviceSynchronize());
    SP_CUDA(cudaMemcpy(pk->p.p, p.data(), NP * 4, cudaMemcpyHostToDevice));
    SP_CUDA(cudaMemcpy(pk->m.p, m.data(), NP * 4, cudaMemcpyHostToDevice));
    SP_CUDA(cudaMemcpy(pk->v.p, v.data(), NP * 4, cudaMemcpyHostToDevice));
    SP_TRY(upload_norm(pk));
    k_to_bf16<<<nblk(NP, 256), 256>>>(pk->p.p, pk->p16.p);
    SP_CUDA(cudaDeviceSynchronize());
    return SPTRSV_OK;
}

sptrsv_status sptrsv_picker_features(const sptrsv_csr* L, const sptrsv_levels* lv, const int32_t* depths, int32_t nd,
                                     float* feat, sptrsv_stream_t stream) {
    if (!L || !lv || !depths || nd < 1 || !feat) { set_error("picker_features: bad argument"); return SPTRSV_ERR_INVALID; }
    for (int d = 0; d < nd; ++d)
        if (depths[d] == 0) { set_error("picker_features: a candidate is a depth >= 1 or a row budget < 0"); return SPTRSV_ERR_INVALID; }
    return features_impl(L, lv->lv, depths, nd, feat, nullptr, (cudaStream_t)stream);
}

sptrsv_status sptrsv_picker_infer(const sptrsv_picker* pk, const float* feat, int64_t count, float* out, int32_t bf16,
                                  sptrsv_stream_t stream) {
    if (!pk || (count > 0 && (!feat || !out)) || count < 0) { set_error("picker_infer: bad argument"); return SPTRSV_ERR_INVALID; }
    return forward(pk, feat, count, out, nullptr, bf16, (cudaStream_t)stream);
}

sptrsv_status sptrsv_picker_grad(const sptrsv_picker* pk, const float* feat, const float* target, int64_t count,
                                 int32_t bf16, float* grad, float* loss, sptrsv_stream_t stream) {
    if (!pk || !feat || !target || !grad) { set_error("picker_grad: bad argument"); return SPTRSV_ERR_INVALID; }
    return grad_impl(pk, feat, target, count, bf16, grad, loss, (cudaStream_t)stream);
}

sptrsv_status sptrsv_picker_train_step(sptrsv_picker* pk, const float* feat, const float* target, int64_t count,
                                       float lr, float* loss, sptrsv_stream_t stream) {
    if (!pk || !feat || !target) { set_error("picker_train_step: bad argument"); return SPTRSV_ERR_INVALID; }
    cudaStream_t st = (cudaStream_t)stream;
    SP_TRY(grad_impl(pk, feat, target, count, 1, pk->grad.p, loss, st));
    pk->step += 1;
    const float c1 = 1.0f - std::pow(0.9f, (float)pk->step), c2 = 1.0f - std::pow(0.999f, (float)pk->step);
    k_adam<<<nblk(NP, 256), 256, 0, st>>>(pk->p.p, pk->m.p, pk->v.p, pk->grad.p, pk->p16.p, lr, c1, c2);
    SP_CUDA(cudaGetLastError());
    return SPTRSV_OK;
}

}  // extern "C"
