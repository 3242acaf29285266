// prims.cu -- device-wide exclusive scan and stable LSD radix sort (own kernels).
#include "internal.cuh"

namespace sp {
namespace {

constexpr int SCAN_THREADS = 256;
constexpr int SCAN_ITEMS = 8;
constexpr int SCAN_TILE = SCAN_THREADS * SCAN_ITEMS;

template <typename T>
__device__ T block_exclusive_scan(T v, T* total, T* warp_tmp) {
    // warp inclusive scan
    int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    T x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        T y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) warp_tmp[warp] = x;
    __syncthreads();
    if (warp == 0) {
        int nw = blockDim.x >> 5;
        T w = lane < nw ? warp_tmp[lane] : T(0);
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            T y = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += y;
        }
        if (lane < nw) warp_tmp[lane] = w;  // inclusive per warp
    }
    __syncthreads();
    T before = warp ? warp_tmp[warp - 1] : T(0);
    T tot = warp_tmp[(blockDim.x >> 5) - 1];
    __syncthreads();
    *total = tot;
    return before + x - v;
}

template <typename Tin, typename Tout>
__global__ void k_tile_reduce(const Tin* in, int64_t n, Tout* sums) {
    __shared__ Tout tmp[32];
    int64_t base = (int64_t)blockIdx.x * SCAN_TILE;
    Tout s = 0;
    for (int i = 0; i < SCAN_ITEMS; ++i) {
        int64_t idx = base + (int64_t)i * SCAN_THREADS + threadIdx.x;
        if (idx < n) s += (Tout)in[idx];
    }
    Tout total;
    block_exclusive_scan<Tout>(s, &total, tmp);
    if (threadIdx.x == 0) sums[blockIdx.x] = total;
}

// single-block exclusive scan of `count` values in place; writes the grand total at sums[count]
template <typename T>
__global__ void k_scan_small(T* sums, int64_t count) {
    __shared__ T tmp[32];
    __shared__ T carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (int64_t base = 0; base < count; base += blockDim.x) {
        int64_t idx = base + threadIdx.x;
        T v = idx < count ? sums[idx] : T(0);
        T total;
        T ex = block_exclusive_scan<T>(v, &total, tmp);
        T c = carry;
        if (idx < count) sums[idx] = ex + c;
        __syncthreads();
        if (threadIdx.x == 0) carry = c + total;
        __syncthreads();
    }
    if (threadIdx.x == 0) sums[count] = carry;
}

template <typename Tin, typename Tout>
__global__ void k_tile_scan(const Tin* in, Tout* out, int64_t n, const Tout* offsets) {
    __shared__ Tout tmp[32];
    int64_t base = (int64_t)blockIdx.x * SCAN_TILE + (int64_t)threadIdx.x * SCAN_ITEMS;
    Tout v[SCAN_ITEMS];
    Tout s = 0;
#pragma unroll
    for (int i = 0; i < SCAN_ITEMS; ++i) {
        int64_t idx = base + i;
        v[i] = idx < n ? (Tout)in[idx] : Tout(0);
        s += v[i];
    }
    Tout total;
    Tout ex = block_exclusive_scan<Tout>(s, &total, tmp) + offsets[blockIdx.x];
#pragma unroll
    for (int i = 0; i < SCAN_ITEMS; ++i) {
        int64_t idx = base + i;
        if (idx < n) out[idx] = ex;
        ex += v[i];
    }
    if (blockIdx.x == gridDim.x - 1 && threadIdx.x == 0) out[n] = offsets[gridDim.x];
}

template <typename Tin, typename Tout>
sptrsv_status scan_impl(const Tin* in, Tout* out, int64_t n, cudaStream_t st) {
    if (n <= 0) {
        SP_CUDA(cudaMemsetAsync(out, 0, sizeof(Tout), st));
        return SPTRSV_OK;
    }
    int64_t tiles = (n + SCAN_TILE - 1) / SCAN_TILE;
    Scratch sums;
    SP_TRY(sums.alloc((tiles + 1) * sizeof(Tout), st));
    // the in-place case (in == out) reads every input before any tile writes: the
    // reduce pass reads all inputs, the scan pass re-reads a tile before writing it
    k_tile_reduce<Tin, Tout><<<(unsigned)tiles, SCAN_THREADS, 0, st>>>(in, n, sums.as<Tout>());
    k_scan_small<Tout><<<1, 1024, 0, st>>>(sums.as<Tout>(), tiles);
    k_tile_scan<Tin, Tout><<<(unsigned)tiles, SCAN_THREADS, 0, st>>>(in, out, n, sums.as<Tout>());
    SP_CUDA(cudaGetLastError());
    return SPTRSV_OK;
}

// ---------------------------------------------------------------------------------
// stable LSD radix sort, 8-bit digits
// ---------------------------------------------------------------------------------

constexpr int RS_THREADS = 256;
constexpr int RS_ROUNDS = 16;
constexpr int RS_TILE = RS_THREADS * RS_ROUNDS;
constexpr int RS_WARPS = RS_THREADS / 32;

__global__ void k_radix_hist(const int32_t* keys, int64_t n, int shift, int32_t* hist, int nblocks) {
    __shared__ int32_t h[256];
    h[threadIdx.x] = 0;
    __syncthreads();
    int64_t base = (int64_t)blockIdx.x * RS_TILE;
    for (int j = 0; j < RS_ROUNDS; ++j) {
        int64_t idx = base + (int64_t)j * RS_THREADS + threadIdx.x;
        if (idx < n) atomicAdd(&h[(keys[idx] >> shift) & 255], 1);
    }
    __syncthreads();
    // digit-major layout so that one linear scan yields global offsets
    hist[(int64_t)threadIdx.x * nblocks + blockIdx.x] = h[threadIdx.x];
}

__global__ void k_radix_scatter(const int32_t* keys, const int32_t* vals, int32_t* keys_out, int32_t* vals_out,
                                int64_t n, int shift, const int32_t* offsets, int nblocks) {
    __shared__ int32_t run_cnt[256];
    __shared__ int32_t warp_cnt[RS_WARPS][256];
    __shared__ int32_t round_tot[256];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    run_cnt[tid] = 0;
    const int32_t my_off = offsets[(int64_t)tid * nblocks + blockIdx.x];
    __shared__ int32_t base_off[256];
    base_off[tid] = my_off;
    int64_t base = (int64_t)blockIdx.x * RS_TILE;
    const unsigned lt_mask = (1u << lane) - 1u;
    for (int j = 0; j < RS_ROUNDS; ++j) {
        if (base + (int64_t)j * RS_THREADS >= n) break;  // uniform over the block
        for (int w = 0; w < RS_WARPS; ++w) warp_cnt[w][tid] = 0;
        __syncthreads();
        int64_t idx = base + (int64_t)j * RS_THREADS + tid;
        bool valid = idx < n;
        int32_t k = valid ? keys[idx] : 0;
        int32_t v = valid ? vals[idx] : 0;
        int d = valid ? ((k >> shift) & 255) : 256 + lane;
        unsigned peers = __match_any_sync(0xffffffffu, d);
        int rank = __popc(peers & lt_mask);
        int leader = __ffs(peers) - 1;
        if (valid && lane == leader) warp_cnt[warp][d] = __popc(peers);
        __syncthreads();
        {
            int acc = 0;
            for (int w = 0; w < RS_WARPS; ++w) {
                int c = warp_cnt[w][tid];
                warp_cnt[w][tid] = acc;
                acc += c;
            }
            round_tot[tid] = acc;
        }
        __syncthreads();
        if (valid) {
            int64_t pos = (int64_t)base_off[d] + run_cnt[d] + warp_cnt[warp][d] + rank;
            keys_out[pos] = k;
            vals_out[pos] = v;
        }
        __syncthreads();
        run_cnt[tid] += round_tot[tid];
        __syncthreads();
    }
}

}  // namespace

sptrsv_status scan_exclusive_i64(const int64_t* in, int64_t* out, int64_t n, cudaStream_t st) {
    return scan_impl<int64_t, int64_t>(in, out, n, st);
}
sptrsv_status scan_exclusive_i32(const int32_t* in, int32_t* out, int64_t n, cudaStream_t st) {
    return scan_impl<int32_t, int32_t>(in, out, n, st);
}
sptrsv_status scan_exclusive_i32_to_i64(const int32_t* in, int64_t* out, int64_t n, cudaStream_t st) {
    return scan_impl<int32_t, int64_t>(in, out, n, st);
}

sptrsv_status radix_sort_pairs(const int32_t* keys_in, const int32_t* vals_in, int32_t* keys_out,
                               int32_t* vals_out, int64_t n, int bits, cudaStream_t st) {
    if (n <= 0) return SPTRSV_OK;
    if (bits < 1) bits = 1;
    int passes = (bits + 7) / 8;
    int64_t nb64 = (n + RS_TILE - 1) / RS_TILE;
    if (nb64 * 256 >= (int64_t)INT32_MAX) {
        set_error("radix sort: %lld elements exceed the int32 histogram", (long long)n);
        return SPTRSV_ERR_UNSUPPORTED;
    }
    int nb = (int)nb64;
    Scratch hist, tk, tv;
    SP_TRY(hist.alloc(((size_t)nb * 256 + 1) * sizeof(int32_t), st));
    SP_TRY(tk.alloc((size_t)n * sizeof(int32_t), st));
    SP_TRY(tv.alloc((size_t)n * sizeof(int32_t), st));
    // ping-pong so that the last pass lands in keys_out / vals_out
    const int32_t* src_k = keys_in;
    const int32_t* src_v = vals_in;
    for (int p = 0; p < passes; ++p) {
        bool to_out = ((passes - 1 - p) % 2) == 0;
        int32_t* dk = to_out ? keys_out : tk.as<int32_t>();
        int32_t* dv = to_out ? vals_out : tv.as<int32_t>();
        k_radix_hist<<<nb, RS_THREADS, 0, st>>>(src_k, n, 8 * p, hist.as<int32_t>(), nb);
        SP_TRY(scan_exclusive_i32(hist.as<int32_t>(), hist.as<int32_t>(), (int64_t)nb * 256, st));
        k_radix_scatter<<<nb, RS_THREADS, 0, st>>>(src_k, src_v, dk, dv, n, 8 * p, hist.as<int32_t>(), nb);
        SP_CUDA(cudaGetLastError());
        src_k = dk;
        src_v = dv;
    }
    return SPTRSV_OK;
}

}  // namespace sp
