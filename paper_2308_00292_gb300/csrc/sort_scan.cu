// sort_scan.cu -- device-wide exclusive scan and a stable LSD radix sort of
// (Morton key, index) pairs, used to order the points along the Z-curve
// before the tree is built (Step 0 of Sec. 3.4).
#include "dmk_internal.h"

namespace dmk {

namespace {

constexpr int kScanThreads = 512;
constexpr int kScanItems = 4;
constexpr int kScanTile = kScanThreads * kScanItems;

__device__ __forceinline__ int32_t block_excl_scan(int32_t v, int32_t *s_warp, int32_t *total) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int32_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) s_warp[warp] = x;
    __syncthreads();
    if (warp == 0) {
        int nw = blockDim.x >> 5;
        int32_t w = lane < nw ? s_warp[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int32_t y = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += y;
        }
        if (lane < nw) s_warp[lane] = w;
    }
    __syncthreads();
    int32_t before = (warp > 0 ? s_warp[warp - 1] : 0) + x - v;
    if (total) *total = s_warp[(blockDim.x >> 5) - 1];
    __syncthreads();
    return before;
}

__global__ void k_tile_sums(const int32_t *in, int64_t n, int32_t *sums) {
    __shared__ int32_t s_warp[32];
    int64_t base = (int64_t)blockIdx.x * kScanTile;
    int32_t acc = 0;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        int64_t i = base + (int64_t)threadIdx.x * kScanItems + k;
        if (i < n) acc += in[i];
    }
    int32_t tot;
    block_excl_scan(acc, s_warp, &tot);
    if (threadIdx.x == 0) sums[blockIdx.x] = tot;
}

__global__ void k_scan_sums(int32_t *sums, int64_t m, int32_t *d_total) {
    __shared__ int32_t s_warp[32];
    __shared__ int32_t carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (int64_t b = 0; b < m; b += blockDim.x) {
        int64_t i = b + threadIdx.x;
        int32_t v = i < m ? sums[i] : 0;
        int32_t tot;
        int32_t ex = block_excl_scan(v, s_warp, &tot);
        if (i < m) sums[i] = ex + carry;
        __syncthreads();
        if (threadIdx.x == 0) carry += tot;
        __syncthreads();
    }
    if (threadIdx.x == 0 && d_total) *d_total = carry;
}

__global__ void k_scan_apply(const int32_t *in, int32_t *out, int64_t n, const int32_t *sums) {
    __shared__ int32_t s_warp[32];
    int64_t base = (int64_t)blockIdx.x * kScanTile;
    int32_t v[kScanItems];
    int32_t acc = 0;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        int64_t i = base + (int64_t)threadIdx.x * kScanItems + k;
        v[k] = i < n ? in[i] : 0;
        acc += v[k];
    }
    int32_t ex = block_excl_scan(acc, s_warp, nullptr) + sums[blockIdx.x];
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        int64_t i = base + (int64_t)threadIdx.x * kScanItems + k;
        if (i < n) out[i] = ex;
        ex += v[k];
    }
}

}  // namespace

size_t scan_tmp_bytes(int64_t n) {
    int64_t tiles = (n + kScanTile - 1) / kScanTile;
    return (size_t)(tiles + 1) * sizeof(int32_t);
}

void scan_exclusive_i32(const int32_t *d_in, int32_t *d_out, int64_t n, int32_t *d_total,
                        void *tmp, size_t tmp_bytes, cudaStream_t st) {
    int64_t tiles = (n + kScanTile - 1) / kScanTile;
    if (tiles == 0) {
        if (d_total) cudaMemsetAsync(d_total, 0, sizeof(int32_t), st);
        return;
    }
    (void)tmp_bytes;
    int32_t *sums = static_cast<int32_t *>(tmp);
    ::dmk::launch_tick();
    k_tile_sums<<<(unsigned)tiles, kScanThreads, 0, st>>>(d_in, n, sums);
    ::dmk::launch_tick();
    k_scan_sums<<<1, 1024, 0, st>>>(sums, tiles, d_total);
    ::dmk::launch_tick();
    k_scan_apply<<<(unsigned)tiles, kScanThreads, 0, st>>>(d_in, d_out, n, sums);
}

// ---------------------------------------------------------------- radix sort
namespace {

constexpr int kRThreads = 256;
constexpr int kRRounds = 16;
constexpr int kRTile = kRThreads * kRRounds;  // keys per block
constexpr int kRWarps = kRThreads / 32;

__global__ void __launch_bounds__(kRThreads) k_radix_hist(const uint64_t *keys, int64_t n, int shift,
                                                          int32_t *counts, int nblocks) {
    __shared__ int32_t s_hist[256];
    s_hist[threadIdx.x] = 0;
    __syncthreads();
    int64_t base = (int64_t)blockIdx.x * kRTile;
    for (int r = 0; r < kRRounds; ++r) {
        int64_t i = base + (int64_t)r * kRThreads + threadIdx.x;
        if (i < n) atomicAdd(&s_hist[(keys[i] >> shift) & 255u], 1);
    }
    __syncthreads();
    counts[(int64_t)threadIdx.x * nblocks + blockIdx.x] = s_hist[threadIdx.x];
}

__global__ void __launch_bounds__(kRThreads) k_radix_scatter(const uint64_t *keys, const uint32_t *vals, int64_t n,
                                                             int shift, const int32_t *offsets, int nblocks,
                                                             uint64_t *okeys, uint32_t *ovals) {
    __shared__ int32_t s_off[256];
    __shared__ int32_t s_cnt[kRWarps][256];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    s_off[threadIdx.x] = offsets[(int64_t)threadIdx.x * nblocks + blockIdx.x];
    for (int k = lane; k < 256; k += 32) s_cnt[warp][k] = 0;
    __syncthreads();
    const unsigned lt_mask = (1u << lane) - 1u;
    int64_t base = (int64_t)blockIdx.x * kRTile;
    for (int r = 0; r < kRRounds; ++r) {
        int64_t i = base + (int64_t)r * kRThreads + threadIdx.x;
        bool valid = i < n;
        uint64_t key = valid ? keys[i] : 0;
        uint32_t val = valid ? vals[i] : 0;
        int d = valid ? (int)((key >> shift) & 255u) : 256;
        unsigned peers = __match_any_sync(0xffffffffu, d);
        int lrank = __popc(peers & lt_mask);
        if (valid && lrank == 0) s_cnt[warp][d] = __popc(peers);
        __syncthreads();
        {
            int t = threadIdx.x;  // one digit per thread
            int32_t run = s_off[t];
#pragma unroll
            for (int w = 0; w < kRWarps; ++w) {
                int32_t c = s_cnt[w][t];
                s_cnt[w][t] = run;
                run += c;
            }
            s_off[t] = run;
        }
        __syncthreads();
        if (valid) {
            int32_t pos = s_cnt[warp][d] + lrank;
            okeys[pos] = key;
            ovals[pos] = val;
        }
        __syncwarp();
        for (int k = lane; k < 256; k += 32) s_cnt[warp][k] = 0;
        __syncwarp();
    }
}

}  // namespace

size_t radix_tmp_bytes(int64_t n) {
    int64_t nblocks = (n + kRTile - 1) / kRTile;
    int64_t m = 256 * nblocks;
    return (size_t)m * sizeof(int32_t) * 2 + scan_tmp_bytes(m) + 64;
}

void radix_sort_pairs(uint64_t *keys, uint32_t *vals, uint64_t *keys_alt, uint32_t *vals_alt,
                      int64_t n, int bits, void *tmp, size_t tmp_bytes, cudaStream_t st,
                      uint64_t **keys_out, uint32_t **vals_out) {
    int64_t nblocks = (n + kRTile - 1) / kRTile;
    uint64_t *kin = keys, *kout = keys_alt;
    uint32_t *vin = vals, *vout = vals_alt;
    if (n > 0) {
        int64_t m = 256 * nblocks;
        int32_t *counts = static_cast<int32_t *>(tmp);
        int32_t *offs = counts + m;
        void *stmp = offs + m;
        size_t stmp_bytes = tmp_bytes - (size_t)m * sizeof(int32_t) * 2;
        for (int shift = 0; shift < bits; shift += 8) {
            ::dmk::launch_tick();
            k_radix_hist<<<(unsigned)nblocks, kRThreads, 0, st>>>(kin, n, shift, counts, (int)nblocks);
            scan_exclusive_i32(counts, offs, m, nullptr, stmp, stmp_bytes, st);
            ::dmk::launch_tick();
            k_radix_scatter<<<(unsigned)nblocks, kRThreads, 0, st>>>(kin, vin, n, shift, offs, (int)nblocks, kout,
                                                                      vout);
            std::swap(kin, kout);
            std::swap(vin, vout);
        }
    }
    *keys_out = kin;
    *vals_out = vin;
}

}  // namespace dmk
