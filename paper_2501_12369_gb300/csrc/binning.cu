// Steps 2 and 3: tile/depth key duplication and the radix sort of those keys, plus the
// per-tile ranges.  This is the tile-based rasterization with a bounding box that the paper
// keeps from 3DGS (Sec. A.3); the paper prints none of it, so the design here is GB300's:
//
//   k_block_sums / k_scan_block_sums  scan of tiles_touched (2048 splats per CTA, then one
//                                      CTA over the CTA sums; no inter-CTA waiting)
//   k_duplicate                        per CTA: block scan -> per-splat offsets in shared
//                                      memory, then a load-balanced flat loop over the CTA's
//                                      instances (binary search for the owning splat), so
//                                      consecutive threads write consecutive keys
//   k_sort_hist / k_hist_scan          one read of the keys for the digit histograms of all
//                                      passes, then per-pass exclusive scans
//   k_onesweep (one launch per pass)   LSD onesweep pass: warp-level multisplit ranking with
//                                      match.any, decoupled look-back across partitions
//                                      (bounded spins), staging in shared memory so global
//                                      writes go out in digit runs
//   k_ranges                           [start, end) of each tile from adjacent keys
//
// Keys are tile << 32 | bits(depth) with depth > 0, so the unsigned order is (tile, depth);
// only the low 32 + ceil(log2(tiles)) bits are sorted.  Each pass is stable, so equal keys
// keep their emission order, which is ascending splat index.
#include <algorithm>
#include <utility>

#include "kernels.cuh"

namespace darb {

namespace {

constexpr uint32_t kFlagLocal = 1u << 30;
constexpr uint32_t kFlagIncl = 2u << 30;
constexpr uint32_t kCountMask = (1u << 30) - 1;
constexpr int kSpinLimit = 1 << 22;  // x >= 64 ns sleep: a few hundred ms at most

__device__ __forceinline__ uint32_t lanemask_lt() {
    uint32_t m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

__device__ __forceinline__ uint32_t ld_relaxed(const uint32_t *p) {
    return *reinterpret_cast<const volatile uint32_t *>(p);
}
__device__ __forceinline__ void st_relaxed(uint32_t *p, uint32_t v) {
    *reinterpret_cast<volatile uint32_t *>(p) = v;
}

// Exclusive scan of one value per thread over a CTA of NT threads.  s_warp holds NT/32
// entries.  Returns the exclusive prefix; total receives the CTA sum.
template <int NT, typename T>
__device__ __forceinline__ T block_exclusive_scan(T v, T *s_warp, T &total) {
    constexpr int NW = NT / 32;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    T x = v;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        const T y = __shfl_up_sync(0xffffffffu, x, off);
        if (lane >= off) x += y;
    }
    if (lane == 31) s_warp[warp] = x;
    __syncthreads();
    if (warp == 0) {
        T w = lane < NW ? s_warp[lane] : T(0);
        T incl = w;
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const T y = __shfl_up_sync(0xffffffffu, incl, off);
            if (lane >= off) incl += y;
        }
        if (lane < NW) s_warp[lane] = incl - w;
        if (lane == NW - 1) s_warp[NW] = incl;
    }
    __syncthreads();
    const T res = s_warp[warp] + x - v;
    total = s_warp[NW];
    __syncthreads();
    return res;
}

__global__ void __launch_bounds__(kScanThreads)
k_block_sums(int n, const uint32_t *__restrict__ tiles, uint32_t *__restrict__ sums) {
    __shared__ uint32_t s_warp[kScanThreads / 32 + 1];
    const int base = blockIdx.x * kScanTile;
    uint32_t s = 0;
#pragma unroll
    for (int j = 0; j < kScanItems; ++j) {
        const int idx = base + j * kScanThreads + threadIdx.x;
        if (idx < n) s += tiles[idx];
    }
    uint32_t total;
    block_exclusive_scan<kScanThreads>(s, s_warp, total);
    if (threadIdx.x == 0) sums[blockIdx.x] = total;
}

__global__ void __launch_bounds__(1024)
k_scan_block_sums(int nb, const uint32_t *__restrict__ sums, unsigned long long *__restrict__ offsets,
                  uint32_t *num_instances, uint32_t *status, unsigned long long capacity) {
    __shared__ unsigned long long s_warp[1024 / 32 + 1];
    unsigned long long carry = 0;
    for (int chunk = 0; chunk < nb; chunk += 1024) {
        const int idx = chunk + threadIdx.x;
        const unsigned long long v = idx < nb ? sums[idx] : 0ull;
        unsigned long long total;
        const unsigned long long ex = block_exclusive_scan<1024>(v, s_warp, total);
        if (idx < nb) offsets[idx] = carry + ex;
        carry += total;
    }
    if (threadIdx.x == 0) {
        num_instances[0] = carry > 0xffffffffull ? 0xffffffffu : (uint32_t)carry;
        if (carry > capacity) atomicExch(status, (uint32_t)DARB_ERR_CAPACITY);
    }
}

__global__ void __launch_bounds__(kScanThreads)
k_duplicate(int n, const uint32_t *__restrict__ tiles, const unsigned long long *__restrict__ block_offsets,
            const int4 *__restrict__ rect, const float *__restrict__ depth, int tiles_x,
            unsigned long long capacity, uint64_t *__restrict__ keys, uint32_t *__restrict__ vals) {
    __shared__ uint32_t s_off[kScanTile + 1];
    __shared__ uint32_t s_warp[kScanThreads / 32 + 1];
    const int base = blockIdx.x * kScanTile;
    const int t = threadIdx.x;
    uint32_t c[kScanItems], sum = 0;
#pragma unroll
    for (int j = 0; j < kScanItems; ++j) {
        const int idx = base + t * kScanItems + j;
        c[j] = idx < n ? tiles[idx] : 0u;
        sum += c[j];
    }
    uint32_t total;
    uint32_t ex = block_exclusive_scan<kScanThreads>(sum, s_warp, total);
#pragma unroll
    for (int j = 0; j < kScanItems; ++j) {
        s_off[t * kScanItems + j] = ex;
        ex += c[j];
    }
    __syncthreads();
    const unsigned long long gbase = block_offsets[blockIdx.x];
    const int nloc = min(kScanTile, n - base);
    for (uint32_t k = t; k < total; k += kScanThreads) {
        // owning splat: the largest s with s_off[s] <= k (it has >= 1 instance)
        int lo = 0, hi = nloc - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (s_off[mid] <= k) lo = mid;
            else hi = mid - 1;
        }
        const uint32_t l = k - s_off[lo];
        const int4 r = __ldg(rect + base + lo);
        const int w = r.z - r.x + 1;
        const int ty = r.y + (int)(l / (uint32_t)w), tx = r.x + (int)(l % (uint32_t)w);
        const uint64_t key = ((uint64_t)(uint32_t)(ty * tiles_x + tx) << 32) | __float_as_uint(__ldg(depth + base + lo));
        const unsigned long long dst = gbase + k;
        if (dst < capacity) {
            keys[dst] = key;
            vals[dst] = (uint32_t)(base + lo);
        }
    }
}

__global__ void __launch_bounds__(256)
k_sort_hist(const uint64_t *__restrict__ keys, const uint32_t *num, unsigned long long cap, int passes,
            uint32_t *__restrict__ hist) {
    __shared__ uint32_t s_h[kMaxPasses * 256];
    for (int i = threadIdx.x; i < passes * 256; i += 256) s_h[i] = 0;
    __syncthreads();
    const unsigned long long M = min((unsigned long long)*num, cap);
    const int lane = threadIdx.x & 31;
    for (unsigned long long b = (unsigned long long)blockIdx.x * 256; b < M; b += (unsigned long long)gridDim.x * 256) {
        const unsigned long long i = b + threadIdx.x;
        const bool valid = i < M;
        const uint64_t k = valid ? keys[i] : 0ull;
        for (int p = 0; p < passes; ++p) {
            const uint32_t d = valid ? (uint32_t)(k >> (8 * p)) & 255u : 256u;
            const uint32_t peers = __match_any_sync(0xffffffffu, d);
            if (valid && lane == __ffs(peers) - 1) atomicAdd(&s_h[p * 256 + d], (uint32_t)__popc(peers));
        }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < passes * 256; i += 256)
        if (s_h[i]) atomicAdd(&hist[i], s_h[i]);
}

__global__ void __launch_bounds__(256) k_hist_scan(const uint32_t *__restrict__ hist, uint32_t *__restrict__ base) {
    __shared__ uint32_t s_warp[256 / 32 + 1];
    const int p = blockIdx.x;
    uint32_t total;
    const uint32_t ex = block_exclusive_scan<256>(hist[p * 256 + threadIdx.x], s_warp, total);
    base[p * 256 + threadIdx.x] = ex;
}

// One LSD pass over the 8-bit digit at `shift`.  Stable.
__global__ void __launch_bounds__(kSortThreads)
k_onesweep(const uint64_t *__restrict__ kin, const uint32_t *__restrict__ vin, uint64_t *__restrict__ kout,
           uint32_t *__restrict__ vout, const uint32_t *num, unsigned long long cap, int shift,
           const uint32_t *__restrict__ digit_base, uint32_t *lookback, uint32_t *part_counter, uint32_t *status) {
    extern __shared__ __align__(16) unsigned char smem[];
    uint64_t *s_k = reinterpret_cast<uint64_t *>(smem);
    uint32_t *s_v = reinterpret_cast<uint32_t *>(smem + (size_t)kSortTile * 8);
    constexpr int NW = kSortThreads / 32;
    __shared__ uint32_t s_wh[NW][256];
    __shared__ uint32_t s_cta_excl[256];
    __shared__ uint32_t s_gbase[256];
    __shared__ uint32_t s_warp[NW + 1];
    __shared__ uint32_t s_part;

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (tid == 0) s_part = atomicAdd(part_counter, 1u);
    for (int i = tid; i < NW * 256; i += kSortThreads) (&s_wh[0][0])[i] = 0;
    __syncthreads();
    const uint32_t M = (uint32_t)min((unsigned long long)*num, cap);
    const uint32_t part = s_part;
    const uint32_t n_parts = (M + kSortTile - 1) / kSortTile;
    if (part >= n_parts) return;
    const uint32_t base = part * kSortTile;

    uint64_t k[kSortItems];
    uint32_t v[kSortItems], rk[kSortItems];
#pragma unroll
    for (int it = 0; it < kSortItems; ++it) {
        const uint32_t idx = base + warp * (32 * kSortItems) + it * 32 + lane;
        if (idx < M) {
            k[it] = kin[idx];
            v[it] = vin[idx];
        } else {
            k[it] = ~0ull;  // digit 255, ranked after every valid key of the partition
            v[it] = 0;
        }
    }
    const uint32_t lt = lanemask_lt();
#pragma unroll
    for (int it = 0; it < kSortItems; ++it) {
        const uint32_t d = (uint32_t)(k[it] >> shift) & 255u;
        const uint32_t peers = __match_any_sync(0xffffffffu, d);
        const uint32_t prev = s_wh[warp][d];
        rk[it] = prev + __popc(peers & lt);
        __syncwarp();
        if (lane == 31 - __clz(peers)) s_wh[warp][d] = prev + __popc(peers);
        __syncwarp();
    }
    __syncthreads();

    // thread = digit: per-warp exclusive offsets, CTA count, decoupled look-back
    const int dg = tid;
    uint32_t cnt = 0;
#pragma unroll
    for (int w = 0; w < NW; ++w) {
        const uint32_t c = s_wh[w][dg];
        s_wh[w][dg] = cnt;
        cnt += c;
    }
    uint32_t *mine = lookback + (size_t)part * 256 + dg;
    uint32_t excl = 0;
    if (part == 0) {
        st_relaxed(mine, kFlagIncl | cnt);
    } else {
        st_relaxed(mine, kFlagLocal | cnt);
        int p = (int)part - 1;
        int spins = 0, ns = 64;
        while (true) {
            const uint32_t s = ld_relaxed(lookback + (size_t)p * 256 + dg);
            const uint32_t f = s & ~kCountMask;
            if (f == 0) {
                if (++spins > kSpinLimit) {
                    atomicExch(status, (uint32_t)DARB_ERR_TIMEOUT);
                    break;
                }
                __nanosleep(ns);
                ns = min(ns * 2, 1024);
                continue;
            }
            excl += s & kCountMask;
            if (f == kFlagIncl || p == 0) break;
            --p;
        }
        st_relaxed(mine, kFlagIncl | ((excl + cnt) & kCountMask));
    }
    s_gbase[dg] = digit_base[dg] + excl;
    uint32_t tot;
    s_cta_excl[dg] = block_exclusive_scan<kSortThreads>(cnt, s_warp, tot);
    __syncthreads();

#pragma unroll
    for (int it = 0; it < kSortItems; ++it) {
        const uint32_t d = (uint32_t)(k[it] >> shift) & 255u;
        const uint32_t pos = s_cta_excl[d] + s_wh[warp][d] + rk[it];
        s_k[pos] = k[it];
        s_v[pos] = v[it];
    }
    __syncthreads();
    const uint32_t nvalid = min((uint32_t)kSortTile, M - base);
    for (uint32_t j = tid; j < nvalid; j += kSortThreads) {
        const uint64_t kk = s_k[j];
        const uint32_t d = (uint32_t)(kk >> shift) & 255u;
        const uint32_t dst = s_gbase[d] + (j - s_cta_excl[d]);
        kout[dst] = kk;
        vout[dst] = s_v[j];
    }
}

__global__ void __launch_bounds__(256)
k_ranges(const uint64_t *__restrict__ keys, const uint32_t *num, unsigned long long cap, uint32_t *__restrict__ ranges) {
    const unsigned long long M = min((unsigned long long)*num, cap);
    for (unsigned long long i = (unsigned long long)blockIdx.x * 256 + threadIdx.x; i < M;
         i += (unsigned long long)gridDim.x * 256) {
        const uint32_t t = (uint32_t)(keys[i] >> 32);
        if (i == 0 || (uint32_t)(keys[i - 1] >> 32) != t) ranges[2 * (size_t)t] = (uint32_t)i;
        if (i == M - 1 || (uint32_t)(keys[i + 1] >> 32) != t) ranges[2 * (size_t)t + 1] = (uint32_t)(i + 1);
    }
}

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

}  // namespace

size_t sort_workspace_bytes(int n, uint64_t capacity, int passes) {
    const size_t nb = (size_t)(n + kScanTile - 1) / kScanTile;
    const size_t n_parts = (capacity + kSortTile - 1) / kSortTile;
    size_t b = 0;
    b += align256(capacity * 8);
    b += align256(capacity * 4);
    b += align256(nb * 4);
    b += align256(nb * 8);
    b += (size_t)kMaxPasses * 256 * 4 * 2;
    b += (size_t)passes * n_parts * 256 * 4;
    b += align256((size_t)kMaxPasses * 4);
    return b + 256;
}

SortWorkspace carve_sort_workspace(void *base, int n, uint64_t capacity, int passes) {
    const size_t nb = (size_t)(n + kScanTile - 1) / kScanTile;
    const size_t n_parts = (capacity + kSortTile - 1) / kSortTile;
    unsigned char *p = reinterpret_cast<unsigned char *>(base);
    SortWorkspace w;
    w.keys_alt = reinterpret_cast<uint64_t *>(p);
    p += align256(capacity * 8);
    w.vals_alt = reinterpret_cast<uint32_t *>(p);
    p += align256(capacity * 4);
    w.block_sums = reinterpret_cast<uint32_t *>(p);
    p += align256(nb * 4);
    w.block_offsets = reinterpret_cast<uint32_t *>(p);
    p += align256(nb * 8);
    unsigned char *zero0 = p;
    w.hist = reinterpret_cast<uint32_t *>(p);
    p += (size_t)kMaxPasses * 256 * 4;
    w.digit_base = reinterpret_cast<uint32_t *>(p);
    p += (size_t)kMaxPasses * 256 * 4;
    w.lookback = reinterpret_cast<uint32_t *>(p);
    p += (size_t)passes * n_parts * 256 * 4;
    w.part_counter = reinterpret_cast<uint32_t *>(p);
    p += (size_t)kMaxPasses * 4;
    w.zero_bytes = (size_t)(p - zero0);
    return w;
}

cudaError_t launch_count_instances(int n, const uint32_t *tiles_touched, const SortWorkspace &ws,
                                   uint32_t *num_instances, uint32_t *status, uint64_t capacity,
                                   cudaStream_t st) {
    const int nb = (n + kScanTile - 1) / kScanTile;
    if (nb > 0) k_block_sums<<<nb, kScanThreads, 0, st>>>(n, tiles_touched, ws.block_sums);
    k_scan_block_sums<<<1, 1024, 0, st>>>(nb, ws.block_sums, reinterpret_cast<unsigned long long *>(ws.block_offsets),
                                          num_instances, status, (unsigned long long)capacity);
    return cudaGetLastError();
}

cudaError_t launch_duplicate_and_sort(int n, const uint32_t *tiles_touched, const int4 *rect,
                                      const float *depth, int tiles_x, int tile_bits,
                                      uint64_t capacity, uint64_t grid_instances,
                                      const SortWorkspace &ws, uint64_t *keys, uint32_t *values,
                                      uint32_t *ranges, const uint32_t *num_instances,
                                      uint32_t *status, cudaStream_t st) {
    const int bits = 32 + tile_bits;
    const int passes = (bits + 7) / 8;
    const int nb = (n + kScanTile - 1) / kScanTile;
    // the last pass must land in (keys, values)
    uint64_t *ka = (passes % 2 == 0) ? keys : ws.keys_alt;
    uint32_t *va = (passes % 2 == 0) ? values : ws.vals_alt;
    uint64_t *kb = (passes % 2 == 0) ? ws.keys_alt : keys;
    uint32_t *vb = (passes % 2 == 0) ? ws.vals_alt : values;
    if (nb > 0)
        k_duplicate<<<nb, kScanThreads, 0, st>>>(n, tiles_touched, reinterpret_cast<const unsigned long long *>(ws.block_offsets),
                                                 rect, depth, tiles_x, (unsigned long long)capacity, ka, va);
    if (grid_instances == 0) return cudaGetLastError();
    const int hist_blocks = (int)std::min<uint64_t>((grid_instances + 255) / 256, 152 * 8);
    k_sort_hist<<<hist_blocks, 256, 0, st>>>(ka, num_instances, (unsigned long long)capacity, passes, ws.hist);
    k_hist_scan<<<passes, 256, 0, st>>>(ws.hist, ws.digit_base);
    const int smem = kSortTile * 12;
    cudaError_t e = cudaFuncSetAttribute(k_onesweep, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    const unsigned n_parts = (unsigned)((grid_instances + kSortTile - 1) / kSortTile);
    const size_t lb_stride = (size_t)((capacity + kSortTile - 1) / kSortTile) * 256;
    for (int p = 0; p < passes; ++p) {
        k_onesweep<<<n_parts, kSortThreads, smem, st>>>(ka, va, kb, vb, num_instances, (unsigned long long)capacity,
                                                        8 * p, ws.digit_base + p * 256, ws.lookback + p * lb_stride,
                                                        ws.part_counter + p, status);
        std::swap(ka, kb);
        std::swap(va, vb);
    }
    const int rblocks = (int)std::min<uint64_t>((grid_instances + 255) / 256, 152 * 16);
    k_ranges<<<rblocks, 256, 0, st>>>(ka, num_instances, (unsigned long long)capacity, ranges);
    return cudaGetLastError();
}

}  // namespace darb
