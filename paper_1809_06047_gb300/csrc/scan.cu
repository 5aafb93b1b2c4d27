// Device-wide exclusive scan (deterministic: fixed-order block reduce, one-CTA scan of the block
// sums, block-local scan plus offset; inputs up to 65536 elements in one CTA). Used for edge numbering (Sec. 3.2:
// enumerate the non-zeros of the upper triangle of E), vertex buckets, crease-list compaction and
// the row offsets of the subdivision operators (Sec. 3.6, count then fill).
#include "common.cuh"
#include "internal.h"

namespace alsub {

namespace {

constexpr int kScanThreads = 512;
constexpr int kItems = 8;                         // per thread
constexpr int kTile = kScanThreads * kItems;      // 4096 elements per CTA

template <class T>
__device__ __forceinline__ T warp_incl_scan(T v) {
    int lane = threadIdx.x & 31;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        T t = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += t;
    }
    return v;
}

// Exclusive scan of one value per thread across the CTA; the CTA total goes to *tot.
template <class T>
__device__ T block_excl_scan(T v, T *tot) {
    __shared__ T warp_sums[kScanThreads / 32 + 1];
    int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    T inc = warp_incl_scan(v);
    if (lane == 31) warp_sums[w] = inc;
    __syncthreads();
    if (w == 0) {
        T s = lane < kScanThreads / 32 ? warp_sums[lane] : T(0);
        T si = warp_incl_scan(s);
        if (lane < kScanThreads / 32) warp_sums[lane] = si - s;
        if (lane == kScanThreads / 32 - 1) warp_sums[kScanThreads / 32] = si;
    }
    __syncthreads();
    T res = warp_sums[w] + inc - v;
    if (tot) *tot = warp_sums[kScanThreads / 32];
    __syncthreads();
    return res;
}

__device__ __forceinline__ long long limit_of(long long n, const int *n_dev) {
    if (!n_dev) return n;
    long long d = *n_dev;
    return d < n ? (d < 0 ? 0 : d) : n;
}

template <class T>
__global__ void k_tile_sums(const int *__restrict__ in, long long n, const int *n_dev, T *sums) {
    pdl_wait();
    pdl_trigger();
    long long lim = limit_of(n, n_dev);
    long long base = (long long)blockIdx.x * kTile + (long long)threadIdx.x * kItems;
    T s = 0;
#pragma unroll
    for (int i = 0; i < kItems; i++) s += (base + i < lim) ? (T)in[base + i] : T(0);
    T tot;
    block_excl_scan<T>(s, &tot);
    if (threadIdx.x == 0) sums[blockIdx.x] = tot;
}

// One CTA scans the tile sums in place (any count, looping over chunks).
template <class T>
__global__ void k_scan_sums(T *sums, int nt, T *total) {
    pdl_wait();
    pdl_trigger();
    __shared__ T carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (int base = 0; base < nt; base += kScanThreads) {
        int i = base + threadIdx.x;
        T v = i < nt ? sums[i] : T(0);
        T tot;
        T ex = block_excl_scan<T>(v, &tot);
        if (i < nt) sums[i] = ex + carry;
        __syncthreads();
        if (threadIdx.x == 0) carry += tot;
        __syncthreads();
    }
    if (threadIdx.x == 0 && total) *total = carry;
}

template <class T>
__global__ void k_scan_tiles(const int *__restrict__ in, T *out, long long n, const int *n_dev,
                             const T *sums) {
    pdl_wait();
    pdl_trigger();
    long long lim = limit_of(n, n_dev);
    long long base = (long long)blockIdx.x * kTile + (long long)threadIdx.x * kItems;
    T v[kItems];
    T s = 0;
#pragma unroll
    for (int i = 0; i < kItems; i++) {
        v[i] = (base + i < lim) ? (T)in[base + i] : T(0);
        s += v[i];
    }
    T ex = block_excl_scan<T>(s, (T *)nullptr) + sums[blockIdx.x];
#pragma unroll
    for (int i = 0; i < kItems; i++) {
        if (base + i < n) out[base + i] = ex;
        ex += v[i];
    }
}

// Up to kBlockScanMax elements in one 1024-thread CTA and one launch. Warp w owns a contiguous
// segment and reads it 32 consecutive elements at a time (coalesced): pass 1 sums the segment,
// one scan of the 32 segment sums gives each warp its offset, pass 2 (from L1) scans each group
// of 32 with shuffles and carries the running total across the groups.
constexpr int kBlockScanThreads = 1024;
constexpr long long kBlockScanMax = 1 << 16;

template <class T>
__global__ void __launch_bounds__(kBlockScanThreads) k_scan_block(const int *__restrict__ in, T *out,
                                                                  long long n, const int *n_dev, T *total) {
    pdl_wait();
    pdl_trigger();
    __shared__ T wsum[kBlockScanThreads / 32 + 1];
    const long long lim = limit_of(n, n_dev);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const long long seg = ((n + 32 * 32 - 1) / (32 * 32)) * 32;      // multiple of 32
    const long long b = (long long)w * seg, e = b + seg < n ? b + seg : n;
    T sum = 0;
#pragma unroll 8
    for (long long i = b + lane; i < e; i += 32) sum += i < lim ? (T)in[i] : T(0);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
    if (lane == 0) wsum[w] = sum;
    __syncthreads();
    if (w == 0) {
        const T x = wsum[lane];                                       // exactly 32 warps
        const T xi = warp_incl_scan(x);
        wsum[lane] = xi - x;
        if (lane == 31) wsum[32] = xi;
    }
    __syncthreads();
    T carry = wsum[w];
#pragma unroll 4
    for (long long i0 = b; i0 < e; i0 += 32) {
        const long long i = i0 + lane;
        const T v = (i < e && i < lim) ? (T)in[i] : T(0);
        const T inc = warp_incl_scan(v);
        if (i < e) out[i] = carry + inc - v;
        carry += __shfl_sync(0xffffffffu, inc, 31);
    }
    if (threadIdx.x == 0 && total) *total = wsum[32];
}

template <class T>
int scan_impl(const int *in, T *out, long long n, T *total, const int *n_dev, void *tmp, cudaStream_t s) {
    if (n <= 0) {
        if (total) cudaMemsetAsync(total, 0, sizeof(T), s);
        return 0;
    }
    if (n <= kBlockScanMax) {
        launch_pdl(k_scan_block<T>, 1, kBlockScanThreads, s, in, out, n, n_dev, total);
        return 1;
    }
    int nt = (int)((n + kTile - 1) / kTile);
    T *sums = (T *)tmp;
    launch_pdl(k_tile_sums<T>, nt, kScanThreads, s, in, n, n_dev, sums);
    launch_pdl(k_scan_sums<T>, 1, kScanThreads, s, sums, nt, total);
    launch_pdl(k_scan_tiles<T>, nt, kScanThreads, s, in, out, n, n_dev, sums);
    return 3;
}

}  // namespace

size_t scan_tmp_bytes(long long n) {
    long long nt = (n + kTile - 1) / kTile;
    return sizeof(long long) * (size_t)(nt < 1 ? 1 : nt);
}

int scan_exclusive(const int *in, int *out, long long n, int *total, const int *n_dev, void *tmp,
                   cudaStream_t s) {
    return scan_impl<int>(in, out, n, total, n_dev, tmp, s);
}

int scan_exclusive64(const int *in, long long *out, long long n, long long *total, void *tmp,
                     cudaStream_t s) {
    return scan_impl<long long>(in, out, n, total, nullptr, tmp, s);
}

}  // namespace alsub
