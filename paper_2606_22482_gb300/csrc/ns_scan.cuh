// ns_scan.cuh -- device-wide exclusive scan and small-key stable counting sort.
//
// Both are deterministic (no floating point, fixed reduction order) so that plans come out
// bit-identical run to run.  Inputs are produced by functors, outputs consumed by functors, so
// callers fuse the element work into the scan passes instead of materialising temporaries.
#pragma once

#include "ns_internal.cuh"

namespace ns {

constexpr int kScanThreads = 256;
constexpr int kScanItems = 8;

template <class T>
__device__ __forceinline__ T warp_incl_scan(T v)
{
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        T y = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += y;
    }
    return v;
}

template <class T>
__device__ __forceinline__ T warp_sum(T v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Exclusive block scan of one value per thread; returns the prefix, *total gets the block sum.
template <class T, int NT>
__device__ __forceinline__ T block_excl_scan(T v, T* total, T* smem /* NT/32 + 1 */)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    T inc = warp_incl_scan(v);
    if (lane == 31) smem[warp] = inc;
    __syncthreads();
    if (warp == 0) {
        T w = lane < NT / 32 ? smem[lane] : T(0);
        T wi = warp_incl_scan(w);
        if (lane < NT / 32) smem[lane] = wi - w;
        if (lane == NT / 32 - 1) smem[NT / 32] = wi;
    }
    __syncthreads();
    T r = inc - v + smem[warp];
    *total = smem[NT / 32];
    __syncthreads();
    return r;
}

template <class T, class Load, int ITEMS>
__global__ void __launch_bounds__(kScanThreads) k_scan_reduce(Load load, int64_t n, T* partial)
{
    __shared__ T sm[kScanThreads / 32 + 1];
    const int64_t base = (int64_t)blockIdx.x * (kScanThreads * ITEMS);
    T acc = 0;
#pragma unroll
    for (int j = 0; j < ITEMS; ++j) {
        int64_t i = base + (int64_t)j * kScanThreads + threadIdx.x;
        if (i < n) acc += load(i);
    }
    T tot;
    block_excl_scan<T, kScanThreads>(acc, &tot, sm);
    if (threadIdx.x == 0) partial[blockIdx.x] = tot;
}

// single block: exclusive scan of the block partials in place, total to *total_out
template <class T>
__global__ void __launch_bounds__(1024) k_scan_partials(T* partial, int64_t nb, T* total_out)
{
    __shared__ T sm[1024 / 32 + 1];
    T carry = 0;
    for (int64_t b0 = 0; b0 < nb; b0 += 1024) {
        int64_t b = b0 + threadIdx.x;
        T v = b < nb ? partial[b] : T(0);
        T tot;
        T ex = block_excl_scan<T, 1024>(v, &tot, sm);
        if (b < nb) partial[b] = carry + ex;
        carry += tot;
    }
    if (threadIdx.x == 0 && total_out) *total_out = carry;
}

// warp-striped items: warp w of the block owns 32 * ITEMS consecutive items, lane l item
// j * 32 + l of them, so every load of the Load functor is coalesced.  Prefixes come from a warp
// scan per item row, carried across rows, then across the block's warps.
template <class T, class Load, class Store, int ITEMS>
__global__ void __launch_bounds__(kScanThreads) k_scan_down(Load load, Store store, int64_t n,
                                                            const T* partial)
{
    constexpr int NW = kScanThreads / 32;
    __shared__ T wsum[NW + 1];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t wbase = (int64_t)blockIdx.x * (kScanThreads * ITEMS) + (int64_t)warp * (32 * ITEMS);
    T v[ITEMS];
#pragma unroll
    for (int j = 0; j < ITEMS; ++j) {
        const int64_t i = wbase + j * 32 + lane;
        v[j] = i < n ? load(i) : T(0);
    }
    T ex[ITEMS];
    T run = 0;
#pragma unroll
    for (int j = 0; j < ITEMS; ++j) {
        const T inc = warp_incl_scan(v[j]);
        ex[j] = run + inc - v[j];
        run += __shfl_sync(0xffffffffu, inc, 31);
    }
    if (lane == 0) wsum[warp] = run;
    __syncthreads();
    if (warp == 0) {
        const T w = lane < NW ? wsum[lane] : T(0);
        const T wi = warp_incl_scan(w);
        if (lane < NW) wsum[lane] = wi - w;
    }
    __syncthreads();
    const T pre = wsum[warp] + partial[blockIdx.x];
#pragma unroll
    for (int j = 0; j < ITEMS; ++j) {
        const int64_t i = wbase + j * 32 + lane;
        if (i < n) store(i, pre + ex[j], v[j]);
    }
}

// Scratch for device_scan: one partial per kScanThreads items (enough for any items per thread).
inline int64_t scan_partials(int64_t n) { return ceil_div(n > 0 ? n : 1, kScanThreads); }

// Exclusive scan: store(i, prefix_i, value_i) for i in [0, n); *total_out (device) = sum.
// The reduce pass sums items in a different grouping than the down pass, which is fine for
// integers (exact).  ITEMS items per thread: 8 for cheap loads over long ranges, 1 where each
// load is a chain of dependent reads over a short range (more threads hide the latency).
template <class T, class Load, class Store, int ITEMS = kScanItems>
ns_status_t device_scan(Load load, Store store, int64_t n, T* partial, T* total_out,
                        cudaStream_t s)
{
    const int64_t nb = ceil_div(n > 0 ? n : 1, kScanThreads * ITEMS);
    if (n <= 0) {
        if (total_out) NS_CUDA_TRY(cudaMemsetAsync(total_out, 0, sizeof(T), s));
        return NS_OK;
    }
    k_scan_reduce<T, Load, ITEMS><<<(unsigned)nb, kScanThreads, 0, s>>>(load, n, partial);
    NS_LAUNCH_CHECK();
    k_scan_partials<T><<<1, 1024, 0, s>>>(partial, nb, total_out);
    NS_LAUNCH_CHECK();
    k_scan_down<T, Load, Store, ITEMS><<<(unsigned)nb, kScanThreads, 0, s>>>(load, store, n, partial);
    NS_LAUNCH_CHECK();
    return NS_OK;
}

// ---------------------------------------------------------------------------------------------
// stable counting sort by a small key (0 .. kSortBuckets-1), DESCENDING key order, ties by index
// ---------------------------------------------------------------------------------------------
constexpr int kSortBuckets = 64;
constexpr int kSortThreads = 1024;

template <class KeyF>
__global__ void __launch_bounds__(kSortThreads) k_bucket_hist(KeyF key, int64_t n, int32_t* hist)
{
    __shared__ int32_t h[kSortBuckets];
    if (threadIdx.x < kSortBuckets) h[threadIdx.x] = 0;
    __syncthreads();
    int64_t i = (int64_t)blockIdx.x * kSortThreads + threadIdx.x;
    if (i < n) atomicAdd(&h[key(i)], 1);
    __syncthreads();
    if (threadIdx.x < kSortBuckets) hist[(int64_t)blockIdx.x * kSortBuckets + threadIdx.x] = h[threadIdx.x];
}

// offsets in (bucket descending, block ascending) order
__global__ void k_bucket_offsets(int32_t* hist, int64_t nblocks);

template <class KeyF, class Emit>
__global__ void __launch_bounds__(kSortThreads) k_bucket_scatter(KeyF key, Emit emit, int64_t n,
                                                                 const int32_t* offs)
{
    __shared__ int32_t wcnt[kSortThreads / 32][kSortBuckets];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int t = threadIdx.x; t < (kSortThreads / 32) * kSortBuckets; t += kSortThreads)
        (&wcnt[0][0])[t] = 0;
    __syncthreads();
    int64_t i = (int64_t)blockIdx.x * kSortThreads + threadIdx.x;
    int b = i < n ? key(i) : -1;
    unsigned peers = __match_any_sync(0xffffffffu, b);
    int rank_in_warp = __popc(peers & ((1u << lane) - 1u));
    if (b >= 0 && rank_in_warp == 0) wcnt[warp][b] = __popc(peers);
    __syncthreads();
    if (b >= 0) {
        int before = 0;
        for (int w = 0; w < warp; ++w) before += wcnt[w][b];
        emit(i, (int64_t)offs[(int64_t)blockIdx.x * kSortBuckets + b] + before + rank_in_warp);
    }
}

template <class KeyF, class Emit>
ns_status_t bucket_sort_desc(KeyF key, Emit emit, int64_t n, int32_t* hist /* nblocks*64 */,
                             cudaStream_t s)
{
    if (n <= 0) return NS_OK;
    const int64_t nb = ceil_div(n, kSortThreads);
    k_bucket_hist<KeyF><<<(unsigned)nb, kSortThreads, 0, s>>>(key, n, hist);
    NS_LAUNCH_CHECK();
    k_bucket_offsets<<<1, 1024, 0, s>>>(hist, nb);
    NS_LAUNCH_CHECK();
    k_bucket_scatter<KeyF, Emit><<<(unsigned)nb, kSortThreads, 0, s>>>(key, emit, n, hist);
    NS_LAUNCH_CHECK();
    return NS_OK;
}

inline int64_t bucket_hist_size(int64_t n) { return ceil_div(n > 0 ? n : 1, kSortThreads) * kSortBuckets; }

// binary search: largest k in [0, count) with arr[k] <= key; 0 if none (arr[0] <= key assumed)
__device__ __forceinline__ int64_t upper_minus_one(const int32_t* arr, int64_t count, int64_t key)
{
    int64_t lo = 0, hi = count;
    while (hi - lo > 1) {
        int64_t mid = lo + ((hi - lo) >> 1);
        if ((int64_t)__ldg(arr + mid) <= key) lo = mid;
        else hi = mid;
    }
    return lo;
}

}  // namespace ns
