// Exclusive prefix sum over int64 counts (the "count" half of Sec. 4.1's two
// passes turned into row pointers).  Three deterministic phases: per-tile
// sums, one block scanning the tile sums, per-tile scan plus carry-in.
#include <mutex>

#include "cih_internal.h"

namespace cih {
namespace {

constexpr int kScanThreads = 512;
constexpr int kScanItems = 8;
constexpr int kScanTile = kScanThreads * kScanItems;

__device__ __forceinline__ int64_t warp_incl(int64_t v)
{
    int lane = threadIdx.x & 31;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        int64_t o = __shfl_up_sync(0xffffffffu, v, d);
        if (lane >= d) v += o;
    }
    return v;
}

// exclusive scan of one value per thread across the block; total = block sum
__device__ int64_t block_excl(int64_t v, int64_t &total)
{
    constexpr int NW = kScanThreads / 32;
    __shared__ int64_t ws[NW];
    __shared__ int64_t tot;
    int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    int64_t inc = warp_incl(v);
    if (lane == 31) ws[wid] = inc;
    __syncthreads();
    if (wid == 0) {
        int64_t s = lane < NW ? ws[lane] : 0;
        int64_t si = warp_incl(s);
        if (lane < NW) ws[lane] = si - s;
        if (lane == NW - 1) tot = si;
    }
    __syncthreads();
    int64_t res = ws[wid] + inc - v;
    total = tot;
    __syncthreads();
    return res;
}

__global__ void k_tile_sums(const int64_t *data, int64_t n, int64_t *sums)
{
    int64_t base = (int64_t)blockIdx.x * kScanTile;
    int64_t acc = 0;
    for (int k = 0; k < kScanItems; ++k) {
        int64_t i = base + (int64_t)k * kScanThreads + threadIdx.x;
        if (i < n) acc += data[i];
    }
    __shared__ int64_t red[kScanThreads / 32];
    for (int d = 16; d > 0; d >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, d);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x < 32) {
        int64_t v = threadIdx.x < kScanThreads / 32 ? red[threadIdx.x] : 0;
        for (int d = 16; d > 0; d >>= 1) v += __shfl_down_sync(0xffffffffu, v, d);
        if (threadIdx.x == 0) sums[blockIdx.x] = v;
    }
}

// one block: exclusive scan of the tile sums in chunks, running carry;
// the grand total goes to data[n]
__global__ void k_scan_sums(int64_t *sums, int64_t nt, int64_t *data, int64_t n)
{
    __shared__ int64_t carry_s;
    if (threadIdx.x == 0) carry_s = 0;
    __syncthreads();
    for (int64_t c0 = 0; c0 < nt; c0 += kScanThreads) {
        int64_t i = c0 + threadIdx.x;
        int64_t v = i < nt ? sums[i] : 0;
        int64_t total = 0;
        int64_t ex = block_excl(v, total);
        int64_t carry = carry_s;
        if (i < nt) sums[i] = carry + ex;
        __syncthreads();
        if (threadIdx.x == 0) carry_s = carry + total;
        __syncthreads();
    }
    if (threadIdx.x == 0) data[n] = carry_s;
}

__global__ void k_tile_scan(int64_t *data, int64_t n, const int64_t *sums)
{
    int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
    int64_t v[kScanItems];
    int64_t loc = 0;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        int64_t i = base + k;
        v[k] = i < n ? data[i] : 0;
        loc += v[k];
    }
    int64_t total = 0;
    int64_t ex = block_excl(loc, total) + sums[blockIdx.x];
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        int64_t i = base + k;
        if (i < n) data[i] = ex;
        ex += v[k];
    }
}

}  // namespace

int64_t scan_scratch_needed(int64_t n)
{
    return (n + kScanTile - 1) / kScanTile + 1;
}

int exclusive_scan_i64(int64_t *data, int64_t n, int64_t *block_sums, int64_t block_sums_len,
                       cudaStream_t st)
{
    int64_t nt = (n + kScanTile - 1) / kScanTile;
    if (block_sums_len < nt) return fail(CIH_ERR_ARG, "scan scratch too small");
    if (nt > INT32_MAX) return fail(CIH_ERR_UNSUPPORTED, "scan too long");
    count_launches(nt > 0 ? 3 : 1);
    if (nt > 0) k_tile_sums<<<(unsigned)nt, kScanThreads, 0, st>>>(data, n, block_sums);
    k_scan_sums<<<1, kScanThreads, 0, st>>>(block_sums, nt, data, n);
    if (nt > 0) k_tile_scan<<<(unsigned)nt, kScanThreads, 0, st>>>(data, n, block_sums);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "scan");
    return CIH_OK;
}

// ---------------------------------------------------------------- no-allocation variant
//
// The same scan with its tile sums in a fixed device array that lives in this
// library's module instead of caller or library allocations.  Every call on a
// device uses the same array; phase 1 rewrites every tile sum the call reads, so
// nothing has to be cleared between calls, but two calls whose work overlaps on
// the GPU (different streams, or host threads) race on it.

namespace {

constexpr int64_t kStaticTileSums = 16384;                 // 128 KiB on every device that loads the library
static __device__ __align__(256) int64_t g_static_tile_sums[kStaticTileSums];

// device address of the array, resolved once per device with that device current
// (the cached address does not survive a reset of that device's primary context)
int static_tile_sums(int device, int64_t **out)
{
    static std::mutex mu;
    static int64_t *addr[64] = {};
    if (device < 0 || device >= 64) return fail(CIH_ERR_UNSUPPORTED, "device index above 63");
    std::lock_guard<std::mutex> lock(mu);
    if (!addr[device]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_static_tile_sums);
        if (e != cudaSuccess) return cuda_fail(e, "static scan scratch: cudaGetSymbolAddress");
        addr[device] = (int64_t *)p;
    }
    *out = addr[device];
    return CIH_OK;
}

}  // namespace

}  // namespace cih

extern "C" int cih_rowptr_scan_static(const int64_t *counts_dev, int64_t n, int64_t *rowptr_dev, void *stream)
{
    using namespace cih;
    if (n < 0 || !rowptr_dev || (n > 0 && !counts_dev)) return fail(CIH_ERR_ARG, "NULL array or negative length");
    if (n > kStaticTileSums * kScanTile)
        return fail(CIH_ERR_CAPACITY, "rowptr_scan_static: more than 67108864 rows (16384 tiles of 4096)");
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
    int64_t *sums = nullptr;
    int rc = static_tile_sums(dev, &sums);
    if (rc) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    if (n > 0 && counts_dev != rowptr_dev) {
        // in place, or disjoint: the copy below must not read what it has written
        const uintptr_t c0 = (uintptr_t)counts_dev, c1 = c0 + sizeof(int64_t) * (uint64_t)n;
        const uintptr_t r0 = (uintptr_t)rowptr_dev, r1 = r0 + sizeof(int64_t) * ((uint64_t)n + 1);
        if (c0 < r1 && r0 < c1) return fail(CIH_ERR_ARG, "rowptr_scan_static: counts and rowptr partly overlap");
        e = cudaMemcpyAsync(rowptr_dev, counts_dev, sizeof(int64_t) * n, cudaMemcpyDeviceToDevice, st);
        if (e != cudaSuccess) return cuda_fail(e, "rowptr_scan_static: copy counts");
    }
    return exclusive_scan_i64(rowptr_dev, n, sums, kStaticTileSums, st);
}

