// Device-wide exclusive scan of int32 (deterministic: fixed-order block reduce, one-CTA scan of
// the block sums, block-local scan plus offset). Used for edge numbering (Sec. 3.2: enumerate the
// non-zeros of the upper triangle of E), vertex buckets and crease-list compaction (Sec. 3.3,
// "count then fill").
#include "common.cuh"
#include "internal.h"

namespace alsub {

namespace {

constexpr int kScanThreads = 512;
constexpr int kItems = 8;                         // per thread
constexpr int kTile = kScanThreads * kItems;      // 4096 elements per CTA

__device__ __forceinline__ int warp_incl_scan(int v) {
    int lane = threadIdx.x & 31;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int t = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += t;
    }
    return v;
}

// Exclusive scan of one value per thread across the CTA; returns the CTA total in *tot.
__device__ int block_excl_scan(int v, int *tot) {
    __shared__ int warp_sums[kScanThreads / 32 + 1];
    int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    int inc = warp_incl_scan(v);
    if (lane == 31) warp_sums[w] = inc;
    __syncthreads();
    if (w == 0) {
        int s = lane < kScanThreads / 32 ? warp_sums[lane] : 0;
        int si = warp_incl_scan(s);
        if (lane < kScanThreads / 32) warp_sums[lane] = si - s;
        if (lane == kScanThreads / 32 - 1) warp_sums[kScanThreads / 32] = si;  // total
    }
    __syncthreads();
    int res = warp_sums[w] + inc - v;
    if (tot) *tot = warp_sums[kScanThreads / 32];
    __syncthreads();
    return res;
}

__device__ __forceinline__ long long limit_of(long long n, const int *n_dev) {
    if (!n_dev) return n;
    long long d = *n_dev;
    return d < n ? (d < 0 ? 0 : d) : n;
}

__global__ void k_tile_sums(const int *__restrict__ in, long long n, const int *n_dev, int *sums) {
    long long lim = limit_of(n, n_dev);
    long long base = (long long)blockIdx.x * kTile + (long long)threadIdx.x * kItems;
    int s = 0;
#pragma unroll
    for (int i = 0; i < kItems; i++) s += (base + i < lim) ? in[base + i] : 0;
    int tot;
    block_excl_scan(s, &tot);
    if (threadIdx.x == 0) sums[blockIdx.x] = tot;
}

// One CTA scans the tile sums in place (any count, looping over chunks).
__global__ void k_scan_sums(int *sums, int nt, int *total) {
    __shared__ int carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (int base = 0; base < nt; base += kScanThreads) {
        int i = base + threadIdx.x;
        int v = i < nt ? sums[i] : 0;
        int tot;
        int ex = block_excl_scan(v, &tot);
        if (i < nt) sums[i] = ex + carry;
        __syncthreads();
        if (threadIdx.x == 0) carry += tot;
        __syncthreads();
    }
    if (threadIdx.x == 0 && total) *total = carry;
}

__global__ void k_scan_tiles(const int *__restrict__ in, int *out, long long n, const int *n_dev,
                             const int *sums) {
    long long lim = limit_of(n, n_dev);
    long long base = (long long)blockIdx.x * kTile + (long long)threadIdx.x * kItems;
    int v[kItems];
    int s = 0;
#pragma unroll
    for (int i = 0; i < kItems; i++) {
        v[i] = (base + i < lim) ? in[base + i] : 0;
        s += v[i];
    }
    int ex = block_excl_scan(s, nullptr) + sums[blockIdx.x];
#pragma unroll
    for (int i = 0; i < kItems; i++) {
        if (base + i < n) out[base + i] = ex;
        ex += v[i];
    }
}

// Small inputs: one CTA scans the whole array in tiles, carrying the running total.
constexpr long long kSmallScan = 1 << 14;

__global__ void __launch_bounds__(kScanThreads) k_scan_single(const int *__restrict__ in, int *out,
                                                              long long n, const int *n_dev, int *total) {
    __shared__ int carry;
    const long long lim = limit_of(n, n_dev);
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (long long base0 = 0; base0 < n; base0 += kTile) {
        const long long base = base0 + (long long)threadIdx.x * kItems;
        int v[kItems];
        int s = 0;
#pragma unroll
        for (int i = 0; i < kItems; i++) {
            v[i] = (base + i < lim) ? in[base + i] : 0;
            s += v[i];
        }
        int tot;
        int ex = block_excl_scan(s, &tot) + carry;
#pragma unroll
        for (int i = 0; i < kItems; i++) {
            if (base + i < n) out[base + i] = ex;
            ex += v[i];
        }
        __syncthreads();
        if (threadIdx.x == 0) carry += tot;
        __syncthreads();
    }
    if (threadIdx.x == 0 && total) *total = carry;
}

}  // namespace

size_t scan_tmp_bytes(long long n) {
    long long nt = (n + kTile - 1) / kTile;
    return sizeof(int) * (size_t)(nt < 1 ? 1 : nt);
}

int scan_exclusive(const int *in, int *out, long long n, int *total, const int *n_dev, void *tmp,
                   cudaStream_t s) {
    if (n <= 0) {
        if (total) cudaMemsetAsync(total, 0, sizeof(int), s);
        return 0;
    }
    if (n <= kSmallScan) {
        k_scan_single<<<1, kScanThreads, 0, s>>>(in, out, n, n_dev, total);
        return 1;
    }
    int nt = (int)((n + kTile - 1) / kTile);
    int *sums = (int *)tmp;
    k_tile_sums<<<nt, kScanThreads, 0, s>>>(in, n, n_dev, sums);
    k_scan_sums<<<1, kScanThreads, 0, s>>>(sums, nt, total);
    k_scan_tiles<<<nt, kScanThreads, 0, s>>>(in, out, n, n_dev, sums);
    return 3;
}

}  // namespace alsub
