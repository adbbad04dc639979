// Steps 2 and 3: tile/depth key duplication and the radix sort of those keys, plus the
// per-tile ranges.  This is the tile-based rasterization with a bounding box that the paper
// keeps from 3DGS (Sec. A.3); the paper prints none of it, so the design here is GB300's.
//
// The result is fixed: every (splat, member tile) instance -- the member tiles being, per tile
// row of the splat's rectangle, the run its ellipse reaches (see span_row) -- ordered by
// key = tile << 32 | bits(depth) (depth > 0, so the unsigned order is (tile, depth)), equal keys
// in ascending splat index.  Two strategies produce it bit for bit:
//
// DARB_SORT_DEPTH_THEN_TILE (default)
//   k_vis_count, k_depth_compact          the visible splats' depth keys in index order, with
//                                         their digit histograms
//   4 x k_onesweep<u32>                   sort them by depth bits (stable, so equal depths keep
//                                         index order): N-sized, cheap
//   k_block_sums / k_scan_block_sums      scan of tiles_touched in that depth order
//   k_tile_diff / k_tile_setup            per-tile instance counts from the row runs (a row-wise
//                                         difference array, 2 atomics per run) -> the tile
//                                         ranges and the digit bases of the tile passes
//   k_splat_offsets                       per-position instance offsets (depth order) and the
//                                         first and last owner of every sort partition
//   k_dup_sweep                           emit (tile id, splat) per instance in depth order, each
//                                         CTA a fixed range of instances (near splats are the
//                                         largest, so splitting by splats would be unbalanced),
//                                         and sort that partition by the first tile digit at once
//   (p - 1) x k_onesweep<u32>             the remaining stable LSD passes over the 32-bit tile ids
//                                         (p = 2 at 1080p with 16- or 32-pixel tiles); the last
//                                         writes only the values
//   k_keys64 (optional)                   the 64-bit keys, when the caller asks for them
//   About 20 bytes of HBM traffic per instance at p = 2.  (With the reduce-then-scan passes,
//   k_duplicate_balanced writes the instances and the first pass reads them back.)
//
// DARB_SORT_KEYS64
//   k_duplicate (64-bit keys in splat order), k_sort_hist, k_hist_scan, 6 x k_onesweep<u64>
//   over the low 32 + ceil(log2 tiles) bits, k_ranges.  About 170 bytes per instance.
//
// k_onesweep is one LSD pass: unordered per-warp digit counts published at once (so successors
// can look back early), stable warp-level ranking (peers by one ballot per digit bit, or by
// match.any), decoupled look-back across partitions claimed in launch order (spins bounded; on
// timeout the status word is set and successors are released), and staging in shared memory so
// the scatter leaves in digit runs.
#include <algorithm>
#include <mutex>
#include <utility>

#include "kernels.cuh"

namespace darb {

namespace {

constexpr uint32_t kFlagLocal = 1u << 30;
constexpr uint32_t kFlagIncl = 2u << 30;
constexpr uint32_t kCountMask = (1u << 30) - 1;
#ifndef DARB_SPIN_LIMIT
#define DARB_SPIN_LIMIT (1 << 22)  // with the 512 ns back-off: about two seconds at most
#endif
constexpr int kSpinLimit = DARB_SPIN_LIMIT;
#ifndef DARB_LOOKBACK_WINDOW
#define DARB_LOOKBACK_WINDOW 8  // predecessor statuses a digit's look-back reads per round trip
#endif
constexpr int kLookbackWindow = DARB_LOOKBACK_WINDOW;
constexpr size_t kMaxDiffSmem = 96 * 1024;  // tile difference array privatised per CTA up to this size
constexpr size_t kMaxSetupSmem = 160 * 1024;  // tile counts + difference array staged in shared memory up to this
constexpr int kDupItems = 16;
static_assert(kScanThreads * kDupItems == kSortTile, "a duplicate CTA must cover exactly one sort partition");
constexpr int kDupTile = kScanThreads * kDupItems;  // instances per balanced duplicate CTA

__device__ __forceinline__ uint32_t lanemask_lt() {
    uint32_t m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

// Lanes of the warp whose digit equals this lane's digit, from one ballot per digit bit.
__device__ __forceinline__ uint32_t match_digit(uint32_t d, int bits) {
    uint32_t peers = 0xffffffffu;
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        if (i < bits) {
            const bool b = (d >> i) & 1u;
            const uint32_t bal = __ballot_sync(0xffffffffu, b);
            peers &= b ? bal : ~bal;
        }
    }
    return peers;
}

__device__ __forceinline__ uint32_t ld_relaxed(const uint32_t *p) {
    return *reinterpret_cast<const volatile uint32_t *>(p);
}
__device__ __forceinline__ void st_relaxed(uint32_t *p, uint32_t v) {
    *reinterpret_cast<volatile uint32_t *>(p) = v;
}

// ---------------------------------------------------------------------------- chained scans
//
// A single-pass exclusive scan over partitions taken in launch order (each CTA claims the next
// index from a counter, so every predecessor of a partition is already running): a partition
// publishes its own total, sums its predecessors' published words back to the nearest inclusive
// prefix, and publishes its own inclusive prefix.  One 64-bit word per partition, zeroed before
// the launch: bits 62-63 the state (1: the partition's total, 2: the inclusive prefix through
// it), bits 0-61 the value.
constexpr unsigned long long kChainOwn = 1ull << 62, kChainIncl = 2ull << 62, kChainVal = (1ull << 62) - 1;
// The visible count with the compaction, and the instance offsets with M, each as one chained
// pass (1), or each as block sums, a one-CTA scan of them and the pass itself (0).
#ifndef DARB_CHAINED_SCANS
#define DARB_CHAINED_SCANS 1
#endif

__device__ __forceinline__ unsigned long long ld_relaxed64(const unsigned long long *p) {
    return *reinterpret_cast<const volatile unsigned long long *>(p);
}
__device__ __forceinline__ void st_relaxed64(unsigned long long *p, unsigned long long v) {
    *reinterpret_cast<volatile unsigned long long *>(p) = v;
}

// The next partition index from counter, for the whole CTA.
__device__ __forceinline__ int claim_partition(uint32_t *counter, int *s_part) {
    if (threadIdx.x == 0) *s_part = (int)atomicAdd(counter, 1u);
    __syncthreads();
    return *s_part;
}

// By the 32 lanes of warp 0: the sum over the partitions before `part` (whose own total is
// `total`), 32 predecessors per round.  A predecessor not published after kSpinLimit polls sets
// DARB_ERR_TIMEOUT in *status and ends the wait with the sum found so far.
__device__ __forceinline__ unsigned long long chain_exclusive(unsigned long long *chain, int part,
                                                              unsigned long long total, uint32_t *status) {
    const int lane = threadIdx.x & 31;
    if (part == 0) {
        if (lane == 0) st_relaxed64(chain, kChainIncl | (total & kChainVal));
        return 0ull;
    }
    if (lane == 0) st_relaxed64(chain + part, kChainOwn | (total & kChainVal));
    unsigned long long excl = 0;
    int p = part - 1, spins = 0, ns = 32;
    while (p >= 0) {
        const int idx = p - lane;  // lane l reads predecessor p - l; before partition 0: an inclusive 0
        const unsigned long long w = idx >= 0 ? ld_relaxed64(chain + idx) : kChainIncl;
        const uint32_t incl = __ballot_sync(0xffffffffu, (w & ~kChainVal) == kChainIncl);
        const uint32_t ready = __ballot_sync(0xffffffffu, (w & ~kChainVal) != 0ull);
        // the lanes up to the nearest inclusive prefix (all 32 when none is in this window)
        const uint32_t upto = incl ? ((incl & (0u - incl)) << 1) - 1u : 0xffffffffu;
        if ((ready & upto) != upto) {  // a predecessor has not published yet: poll again
            if (++spins > kSpinLimit) {
                if (lane == 0) atomicExch(status, (uint32_t)DARB_ERR_TIMEOUT);
                break;
            }
            if (spins > 16) {
                __nanosleep(ns);
                ns = min(ns * 2, 512);
            }
            continue;
        }
        unsigned long long v = ((upto >> lane) & 1u) ? (w & kChainVal) : 0ull;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        excl += v;
        if (incl) break;
        p -= 32;
    }
    if (lane == 0) st_relaxed64(chain + part, kChainIncl | ((excl + total) & kChainVal));
    return excl;
}

// Exclusive scan of one value per thread over a CTA of NT threads.  s_warp holds NT/32 + 1
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

struct PassSpec {
    int shift[kMaxPasses];
    int bits[kMaxPasses];
    int passes;
};

// ---------------------------------------------------------------------------- scan of tiles_touched

// Per-CTA sums of tiles_touched over kScanTile positions; order (if given) maps positions to splats.
__global__ void __launch_bounds__(kScanThreads)
k_block_sums(int n, const uint32_t *__restrict__ tiles, const uint32_t *__restrict__ order,
             const uint32_t *__restrict__ n_vis, uint32_t *__restrict__ sums) {
    pdl_entry();
    __shared__ uint32_t s_warp[kScanThreads / 32 + 1];
    const int base = blockIdx.x * kScanTile;
    const int m = n_vis ? (int)min(*n_vis, (uint32_t)n) : n;  // positions past the visible ones hold no instance
    uint32_t s = 0;
#pragma unroll
    for (int j = 0; j < kScanItems; ++j) {
        const int idx = base + j * kScanThreads + threadIdx.x;
        if (idx < m) s += tiles[order ? order[idx] : idx];
    }
    uint32_t total;
    block_exclusive_scan<kScanThreads>(s, s_warp, total);
    if (threadIdx.x == 0) sums[blockIdx.x] = total;
}

__global__ void __launch_bounds__(1024)
k_scan_block_sums(int nb, const uint32_t *__restrict__ sums, unsigned long long *__restrict__ offsets,
                  uint32_t *num_instances, uint32_t *status, unsigned long long capacity) {
    pdl_entry();
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

// Block scan of the CTA's kScanTile counts into s_off (exclusive, s_off[kScanTile] = total).
__device__ __forceinline__ uint32_t cta_offsets(int n, int base, const uint32_t *__restrict__ tiles,
                                                const uint32_t *__restrict__ order, uint32_t *s_off,
                                                uint32_t *s_id, uint32_t *s_warp) {
    const int t = threadIdx.x;
    uint32_t c[kScanItems], sum = 0;
#pragma unroll
    for (int j = 0; j < kScanItems; ++j) {
        const int idx = base + t * kScanItems + j;
        uint32_t id = (uint32_t)idx;
        c[j] = 0u;
        if (idx < n) {
            if (order) id = order[idx];
            c[j] = tiles[id];
        }
        if (s_id) s_id[t * kScanItems + j] = id;
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
    return total;
}

// Position in [0, nloc) of the splat owning CTA-local instance k: the largest s with s_off[s] <= k.
__device__ __forceinline__ int owner_of(const uint32_t *s_off, int nloc, uint32_t k) {
    int lo = 0, hi = nloc - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (s_off[mid] <= k) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// ---------------------------------------------------------------------------- duplication

// 64-bit keys in splat order (strategy KEYS64).
__global__ void __launch_bounds__(kScanThreads)
k_duplicate(int n, const uint32_t *__restrict__ tiles, const unsigned long long *__restrict__ block_offsets,
            const int4 *__restrict__ rect, const float2 *__restrict__ mean2d, const float4 *__restrict__ conic_o,
            SpanCtx sc, const float *__restrict__ depth, int tiles_x,
            unsigned long long capacity, uint64_t *__restrict__ keys, uint32_t *__restrict__ vals) {
    pdl_entry();
    __shared__ uint32_t s_off[kScanTile + 1];
    __shared__ uint32_t s_warp[kScanThreads / 32 + 1];
    const int base = blockIdx.x * kScanTile;
    const uint32_t total = cta_offsets(n, base, tiles, nullptr, s_off, nullptr, s_warp);
    const unsigned long long gbase = block_offsets[blockIdx.x];
    const int nloc = min(kScanTile, n - base);
    for (uint32_t k = threadIdx.x; k < total; k += kScanThreads) {
        const int s = owner_of(s_off, nloc, k);
        const uint32_t l = k - s_off[s];
        const uint32_t t = instance_tile(__ldg(mean2d + base + s), __ldg(conic_o + base + s), __ldg(rect + base + s), l,
                                         tiles_x, sc);
        const uint64_t key = ((uint64_t)t << 32) | __float_as_uint(__ldg(depth + base + s));
        const unsigned long long dst = gbase + k;
        if (dst < capacity) {
            keys[dst] = key;
            vals[dst] = (uint32_t)(base + s);
        }
    }
}

// Per-position instance offsets in depth order: offs[j] = sum of tiles_touched over positions < j.
// With bounds (max_parts entries), also the owners of every kSortTile-instance partition p:
// bounds[p].x owns its first instance p * kSortTile, bounds[p].y its last, min(M, (p + 1) *
// kSortTile) - 1 -- each position writes the partitions whose first or last instance it owns.
__global__ void __launch_bounds__(kScanThreads)
k_splat_offsets(int n, const uint32_t *__restrict__ order, const uint32_t *__restrict__ tiles,
                const uint32_t *__restrict__ n_vis,
                const unsigned long long *__restrict__ block_offsets, const uint32_t *__restrict__ num,
                uint32_t *__restrict__ offs, uint2 *__restrict__ bounds, uint32_t max_parts) {
    pdl_entry();
    __shared__ uint32_t s_off[kScanTile + 1];
    __shared__ uint32_t s_warp[kScanThreads / 32 + 1];
    const int base = blockIdx.x * kScanTile;
    // with n_vis, only the visible splats' positions (the ones that own instances) are needed
    const int m = n_vis ? (int)min(*n_vis, (uint32_t)n) : n;
    if (base >= m) {  // a block of culled positions (uniform over the CTA: no barrier is skipped)
        if (blockIdx.x == 0 && threadIdx.x == 0) offs[n] = *num;
        return;
    }
    const uint32_t total = cta_offsets(m, base, tiles, order, s_off, nullptr, s_warp);
    const uint32_t gbase = (uint32_t)block_offsets[blockIdx.x];
    const uint32_t M = *num;
    constexpr uint32_t T = kSortTile;
    for (int j = threadIdx.x; j < kScanTile; j += kScanThreads) {
        if (base + j >= m) continue;
        const uint32_t o0 = gbase + s_off[j];
        offs[base + j] = o0;
        const uint32_t o1 = gbase + (j + 1 < kScanTile ? s_off[j + 1] : total);
        if (!bounds || o1 <= o0) continue;
        for (uint32_t p = (o0 + T - 1) / T; p < (o1 + T - 1) / T && p < max_parts; ++p) bounds[p].x = (uint32_t)(base + j);
        for (uint32_t p = (o0 + 1 + T - 1) / T - 1; p + 1 <= o1 / T && p < max_parts; ++p)
            bounds[p].y = (uint32_t)(base + j);
        if (o1 == M && (M - 1) / T < max_parts) bounds[(M - 1) / T].y = (uint32_t)(base + j);
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) offs[n] = M;
}

// k_block_sums, k_scan_block_sums and k_splat_offsets in one pass: each CTA claims the next
// kScanTile positions, scans their instance counts, takes their global offset from a chained scan
// over the blocks before it, and writes the offsets and partition owners as k_splat_offsets
// does.  Every visible splat owns at least one instance (the preprocessing culls a splat that
// reaches no tile), so the block holding the last visible position n_vis - 1 holds the last
// instance: it writes M (num, clamped to 32 bits; DARB_ERR_CAPACITY in status above capacity),
// offs[n] = M and the owner of M's last partition.
__global__ void __launch_bounds__(kScanThreads)
k_splat_offsets_chained(int n, const uint32_t *__restrict__ order, const uint32_t *__restrict__ tiles,
                        const uint32_t *__restrict__ n_vis, unsigned long long *chain, uint32_t *claim,
                        uint32_t *__restrict__ num, uint32_t *status, unsigned long long capacity,
                        uint32_t *__restrict__ offs, uint2 *__restrict__ bounds, uint32_t max_parts) {
    pdl_entry();
    __shared__ uint32_t s_off[kScanTile + 1];
    __shared__ uint32_t s_warp[kScanThreads / 32 + 1];
    __shared__ int s_part;
    __shared__ unsigned long long s_g;
    const int m = (int)min(*n_vis, (uint32_t)n);
    const int part = claim_partition(claim, &s_part);
    const int base = part * kScanTile;
    if (m == 0) {  // no visible splat: no instance
        if (part == 0 && threadIdx.x == 0) {
            *num = 0u;
            offs[n] = 0u;
        }
        return;
    }
    if (base >= m) return;  // culled positions only (uniform over the CTA; it publishes nothing, and
                            // no block below m looks back past it)
    const uint32_t total = cta_offsets(m, base, tiles, order, s_off, nullptr, s_warp);
    if (threadIdx.x < 32) {
        const unsigned long long e = chain_exclusive(chain, part, total, status);
        if (threadIdx.x == 0) s_g = e;
    }
    __syncthreads();
    const unsigned long long g = s_g;
    const bool last = base + kScanTile >= m;
    const unsigned long long M = g + total;  // the instance count, in the last block
    if (last && threadIdx.x == 0) {
        *num = M > 0xffffffffull ? 0xffffffffu : (uint32_t)M;
        if (M > capacity) atomicExch(status, (uint32_t)DARB_ERR_CAPACITY);
        offs[n] = (uint32_t)M;
    }
    const uint32_t gbase = (uint32_t)g;
    constexpr uint32_t T = kSortTile;
    for (int j = threadIdx.x; j < kScanTile; j += kScanThreads) {
        if (base + j >= m) continue;
        const uint32_t o0 = gbase + s_off[j];
        offs[base + j] = o0;
        const uint32_t o1 = gbase + (j + 1 < kScanTile ? s_off[j + 1] : total);
        if (!bounds || o1 <= o0) continue;
        for (uint32_t p = (o0 + T - 1) / T; p < (o1 + T - 1) / T && p < max_parts; ++p) bounds[p].x = (uint32_t)(base + j);
        for (uint32_t p = (o0 + 1 + T - 1) / T - 1; p + 1 <= o1 / T && p < max_parts; ++p)
            bounds[p].y = (uint32_t)(base + j);
        if (last && base + j == m - 1 && (o1 - 1) / T < max_parts) bounds[(o1 - 1) / T].y = (uint32_t)(base + j);
    }
}

// Largest s in [0, n) with offs[s] <= target (offs non-decreasing, offs[0] = 0), by warp 0 of
// the CTA with 32-way probes.  Returns the result to every thread of the CTA.
__device__ __forceinline__ int cta_upper_owner(const uint32_t *__restrict__ offs, int n, uint32_t target, int *s_res) {
    if (threadIdx.x < 32) {
        const int lane = threadIdx.x;
        int a = 0, b = n;  // answer in [a, b)
        while (b - a > 32) {
            const int step = (b - a + 31) / 32;
            const int p = a + lane * step;
            const bool ok = p < b && offs[p] <= target;
            const uint32_t bal = __ballot_sync(0xffffffffu, ok);
            const int j = 31 - __clz(bal);  // offs[a] <= target always holds, so bal != 0
            a = a + j * step;
            b = min(b, a + step);
        }
        const int p = a + lane;
        const bool ok = p < b && offs[p] <= target;
        const uint32_t bal = __ballot_sync(0xffffffffu, ok);
        if (lane == 0) *s_res = a + 31 - __clz(bal);
    }
    __syncthreads();
    return *s_res;
}

// The instances [lo, hi) of one partition, owner by owner (owners first .. first + count - 1 in
// depth order): the thread that takes an owner computes its ellipse's row runs once and, at the
// first position of every run inside the partition (clipped to lo), records the run's tile id
// at that position and the splat id and sets the position's bit in `mark` (cleared by the
// caller).  Every instance then finds its run start in `mark` without recomputing the ellipse.
// The row runs of the splats whose runs are not packed (rectangles of more than 8 rows or 15
// columns), recorded once by k_tile_diff, which computes them anyway, so that the duplication
// reads them instead of recomputing the ellipse row by row.  off[id] is the first entry of
// splat id's rectangle rows (one entry per row, c0 | c1 << 16, c0 > c1 for a row without
// member tiles), or kNoTable when the table was full; only unpacked visible splats have one.
constexpr uint32_t kNoTable = 0xffffffffu;
constexpr uint32_t kRowEmpty = 0x0000ffffu;  // c0 = 65535 > c1 = 0
struct RunTable {
    uint32_t *off;
    uint32_t *tab;
    uint32_t *count;  // entries handed out (zeroed per call)
    uint32_t cap;
};

template <int NT>
__device__ __forceinline__ void partition_runs(int first, int count, uint32_t lo, uint32_t hi,
                                               const uint32_t *__restrict__ offs, const uint32_t *__restrict__ order,
                                               const int4 *__restrict__ rect, const uint64_t *__restrict__ runs,
                                               const float2 *__restrict__ mean2d, const float4 *__restrict__ conic_o,
                                               const SpanCtx &sc, const RunTable &rt, int tiles_x, uint32_t *s_base,
                                               uint32_t *s_val, uint32_t *mark, uint16_t *s_q, int *s_qn) {
    auto mark_run = [&](uint32_t id, uint32_t j, uint32_t w, int ty, int c0) {  // run [j, j + w) of id's instances
        const uint32_t q = max(j, lo), pos = q - lo;
        s_base[pos] = (uint32_t)(ty * tiles_x + c0) + (q - j);
        s_val[pos] = id;
        atomicOr(&mark[pos >> 5], 1u << (pos & 31));
    };
    // owners with packed runs: one thread each (at most 8 rows, decoded from one word); owners
    // whose runs are in the run table are queued for the warps
    for (int o = threadIdx.x; o < count; o += NT) {
        const uint32_t id = order[first + o];
        const uint64_t pk = __ldg(runs + id);
        if (pk == kRunsUnpacked && rt.tab) {
            s_q[atomicAdd(s_qn, 1)] = (uint16_t)o;
            continue;
        }
        uint32_t j = offs[first + o];
        const int4 r = __ldg(rect + id);
        for_each_run(pk, mean2d, conic_o, id, r, sc, [&](int ty, int c0, int c1) {
            const uint32_t w = (uint32_t)(c1 - c0 + 1);
            if (j + w > lo) mark_run(id, j, w, ty, c0);
            j += w;
            return j < hi;
        });
    }
    if (!rt.tab) return;  // uniform: a kernel argument
    __syncthreads();
    // queued owners: a warp each, one rectangle row per lane, rows read from the run table in
    // parallel and placed by a warp prefix sum of their lengths
    const int nq = *s_qn, lane = threadIdx.x & 31;
    for (int k = (int)(threadIdx.x >> 5); k < nq; k += NT / 32) {
        const int o = s_q[k];
        const uint32_t id = order[first + o];
        const int4 r = __ldg(rect + id);
        const uint32_t tb = __ldg(rt.off + id);
        uint32_t carry = offs[first + o];
        if (tb == kNoTable) {  // the table was full: one lane computes this owner's runs
            if (lane == 0)
                for_each_run(kRunsUnpacked, mean2d, conic_o, id, r, sc, [&](int ty, int c0, int c1) {
                    const uint32_t w = (uint32_t)(c1 - c0 + 1);
                    if (carry + w > lo) mark_run(id, carry, w, ty, c0);
                    carry += w;
                    return carry < hi;
                });
            continue;
        }
        const int rows = r.w - r.y + 1;
        for (int r0 = 0; r0 < rows && carry < hi; r0 += 32) {  // carry is the same in every lane
            const int k2 = r0 + lane;
            const uint32_t e = k2 < rows ? __ldg(rt.tab + tb + (uint32_t)k2) : kRowEmpty;
            const int c0 = (int)(e & 0xffffu), c1 = (int)(e >> 16);
            const uint32_t w = c0 <= c1 ? (uint32_t)(c1 - c0 + 1) : 0u;
            uint32_t x = w;
#pragma unroll
            for (int sh = 1; sh < 32; sh <<= 1) {
                const uint32_t y = __shfl_up_sync(0xffffffffu, x, sh);
                if (lane >= sh) x += y;
            }
            const uint32_t start = carry + x - w;
            if (w && start < hi && start + w > lo) mark_run(id, start, w, r.y + k2, c0);
            carry += __shfl_sync(0xffffffffu, x, 31);
        }
    }
}

// Tile id and splat id of partition position pos, from the nearest run start at or before it.
__device__ __forceinline__ void partition_lookup(uint32_t pos, const uint32_t *s_base, const uint32_t *s_val,
                                                 const uint32_t *mark, uint32_t &key, uint32_t &val) {
    int w = (int)(pos >> 5);
    uint32_t m = mark[w] & (0xffffffffu >> (31 - (pos & 31)));
    while (m == 0 && w > 0) m = mark[--w];
    if (m == 0) {  // unreachable: position 0 always starts a run
        key = 0xffffffffu;
        val = 0;
        return;
    }
    const uint32_t q = (uint32_t)w * 32 + 31 - __clz(m);
    key = s_base[q] + (pos - q);
    val = s_val[q];
}

// 32-bit tile ids in depth order (strategy DEPTH_THEN_TILE), balanced over instances: CTA c
// emits instances [c * kDupTile, (c + 1) * kDupTile).  Lane-major order within each warp's
// chunk keeps the writes coalesced.
// A CTA's instance range is exactly one sort partition (kDupTile == kSortTile), so the CTA also
// writes that partition's histogram of the first tile-pass digit (tile & (2^bits1 - 1)) into
// ph[d * n_parts + partition].
__global__ void __launch_bounds__(kScanThreads)
k_duplicate_balanced(int n, const uint32_t *__restrict__ order, const uint32_t *__restrict__ offs,
                     const int4 *__restrict__ rect, const uint64_t *__restrict__ runs, const float2 *__restrict__ mean2d,
                     const float4 *__restrict__ conic_o, SpanCtx sc, RunTable rt, int tiles_x,
                     const uint32_t *__restrict__ num,
                     unsigned long long cap, uint32_t *__restrict__ keys, uint32_t *__restrict__ vals, int bits1,
                     uint32_t n_parts, uint32_t *__restrict__ ph) {
    pdl_entry();
    __shared__ uint32_t s_base[kDupTile];
    __shared__ uint32_t s_val[kDupTile];
    __shared__ uint32_t s_mark[kDupTile / 32];
    __shared__ uint32_t s_h[256];
    __shared__ int s_res[2];
    __shared__ uint16_t s_q[kDupTile];
    __shared__ int s_qn;
    if (threadIdx.x == 0) s_qn = 0;  // ordered before partition_runs by cta_upper_owner's barriers
    const unsigned long long Mfull = *num;
    if (Mfull > cap) return;  // overflow: nothing is emitted (status already set)
    const uint32_t M = (uint32_t)Mfull;
    const uint32_t lo = blockIdx.x * (uint32_t)kDupTile;
    const uint32_t radix1 = 1u << bits1, mask1 = radix1 - 1u;
    for (int i = threadIdx.x; i < 256; i += kScanThreads) s_h[i] = 0;
    for (int i = threadIdx.x; i < kDupTile / 32; i += kScanThreads) s_mark[i] = 0;
    if (lo >= M) {  // an empty partition (capacity-sized grid): zero histogram
        for (uint32_t d = threadIdx.x; d < radix1; d += kScanThreads) ph[(size_t)d * n_parts + blockIdx.x] = 0;
        return;
    }
    const uint32_t hi = min(M, lo + (uint32_t)kDupTile);
    const int first = cta_upper_owner(offs, n, lo, &s_res[0]);
    const int last = cta_upper_owner(offs, n, hi - 1, &s_res[1]);
    const int count = min(last - first + 1, kDupTile);  // every owner has >= 1 instance
    partition_runs<kScanThreads>(first, count, lo, hi, offs, order, rect, runs, mean2d, conic_o, sc, rt, tiles_x,
                                 s_base, s_val, s_mark, s_q, &s_qn);
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint32_t wbase = lo + (uint32_t)warp * (32 * kDupItems);
#pragma unroll 4
    for (int it = 0; it < kDupItems; ++it) {
        const uint32_t k = wbase + it * 32 + lane;
        if (k >= hi) break;
        uint32_t tile, id;
        partition_lookup(k - lo, s_base, s_val, s_mark, tile, id);
        keys[k] = tile;
        vals[k] = id;
        atomicAdd(&s_h[tile & mask1], 1u);  // neighbouring lanes hold neighbouring tiles: few conflicts
    }
    __syncthreads();
    for (uint32_t d = threadIdx.x; d < radix1; d += kScanThreads) ph[(size_t)d * n_parts + blockIdx.x] = s_h[d];
}

// Tile coverage as a row-wise difference array: +1 at the first and -1 past the last member
// tile of each row run of each visible splat, so that prefix sums along the rows give the
// number of instances of every tile.  The splats are order[0, *n_vis) when the visible ones
// have been compacted (order and n_vis given), else all n with the culled ones skipped.  With
// SMEM each CTA accumulates a private copy in shared memory (grid-stride over splats) and adds
// its non-zero entries to the global array once.
#ifndef DARB_TILE_DIFF_THREADS
#define DARB_TILE_DIFF_THREADS 256  // small CTAs fit beside the depth passes' CTAs on the side stream
#endif
#ifdef DARB_TILE_DIFF_MIN_CTAS
#define DARB_TILE_DIFF_BOUNDS __launch_bounds__(DARB_TILE_DIFF_THREADS, DARB_TILE_DIFF_MIN_CTAS)
#else
#define DARB_TILE_DIFF_BOUNDS __launch_bounds__(DARB_TILE_DIFF_THREADS)
#endif
template <bool SMEM>
__global__ void DARB_TILE_DIFF_BOUNDS
k_tile_diff(int n, const uint32_t *__restrict__ order, const uint32_t *__restrict__ n_vis,
            const int *__restrict__ radius, const int4 *__restrict__ rect, const uint64_t *__restrict__ runs,
            const float2 *__restrict__ mean2d, const float4 *__restrict__ conic_o, SpanCtx sc, RunTable rt,
            int tiles_x, int diff_size, int *__restrict__ diff) {
    pdl_entry();
    extern __shared__ int s_diff[];
    int *d = SMEM ? s_diff : diff;
    if (SMEM) {
        for (int i = threadIdx.x; i < diff_size; i += blockDim.x) s_diff[i] = 0;
        __syncthreads();
    }
    const int w1 = tiles_x + 1;
    const int m = n_vis ? (int)min(*n_vis, (uint32_t)n) : n;
    const int lane = threadIdx.x & 31;
    auto add = [&](int ty, int c0, int c1) {  // one run of member tiles: +1 at c0, -1 after c1
        atomicAdd(&d[ty * w1 + c0], 1);
        atomicAdd(&d[ty * w1 + c1 + 1], -1);
    };
    // whole warps iterate together (the rows of a large rectangle are shared by the warp)
    for (int k0 = blockIdx.x * blockDim.x + (int)(threadIdx.x & ~31u); k0 < m; k0 += gridDim.x * blockDim.x) {
        const int k = k0 + lane;
        int i = 0;
        bool live = false;
        if (k < m) {
            i = order ? (int)order[k] : k;
            live = n_vis != nullptr || radius[i] != 0;  // the compacted order holds visible splats only
        }
        int4 r = make_int4(0, 0, 0, 0);
        uint64_t pk = kRunsUnpacked;
        if (live) {
            r = rect[i];
            pk = runs[i];
        }
        if (live && pk != kRunsUnpacked) for_each_packed_run(pk, r, [&](int ty, int c0, int c1) {
                add(ty, c0, c1);
                return true;
            });
        // run-table entries for the warp's unpacked splats: one reservation per warp (a prefix
        // sum of their row counts), not one atomic on the shared counter per splat
        const bool big = live && pk == kRunsUnpacked;
        uint32_t my_rows = big ? (uint32_t)(r.w - r.y + 1) : 0u, my_pre = my_rows;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, my_pre, o);
            if (lane >= o) my_pre += y;
        }
        const uint32_t warp_rows = __shfl_sync(0xffffffffu, my_pre, 31);
        uint32_t warp_base = 0;
        if (rt.tab && lane == 0 && warp_rows) warp_base = atomicAdd(rt.count, warp_rows);
        warp_base = __shfl_sync(0xffffffffu, warp_base, 0);
        my_pre = warp_base + my_pre - my_rows;  // this lane's first entry
        for (uint32_t bm = __ballot_sync(0xffffffffu, big); bm; bm &= bm - 1) {
            const int src = __ffs(bm) - 1;
            const int iL = __shfl_sync(0xffffffffu, i, src);
            const float2 mu = mean2d[iL];
            const float4 co = conic_o[iL];
            const int4 rL = rect[iL];
            // the rows' runs go to the run table too, for the duplication (every row, the empty
            // ones marked; each lane writes the rows it computes, so no two lanes share an entry)
            const uint32_t rows = (uint32_t)(rL.w - rL.y + 1);
            const uint32_t base = __shfl_sync(0xffffffffu, my_pre, src);
            const bool keep = rt.tab && (unsigned long long)base + rows <= rt.cap;
            if (keep)
                for (uint32_t k = lane; k < rows; k += 32) rt.tab[base + k] = kRowEmpty;
            warp_runs(mu.x, mu.y, co.x, co.y, co.z, rL, sc, [&](int ty, int c0, int c1, uint32_t) {
                add(ty, c0, c1);
                if (keep) rt.tab[base + (uint32_t)(ty - rL.y)] = (uint32_t)c0 | ((uint32_t)c1 << 16);
            });
            if (rt.tab && lane == 0) rt.off[iL] = keep ? base : kNoTable;
        }
    }
    if (SMEM) {
        __syncthreads();
        // each CTA starts its flush at a different entry, so that concurrent CTAs add to
        // different addresses rather than queueing on the same ones
        const int rot = (int)(((long long)blockIdx.x * diff_size) / gridDim.x);
        for (int k = threadIdx.x; k < diff_size; k += blockDim.x) {
            const int i = k + rot < diff_size ? k + rot : k + rot - diff_size;
            if (s_diff[i]) atomicAdd(&diff[i], s_diff[i]);
        }
    }
}

// ---------------------------------------------------------------------------- histograms

// Digit histograms of all passes in one read of the keys (M = min(*num, cap), or cap if num is null).
template <typename K>
__global__ void __launch_bounds__(256)
k_sort_hist(const K *__restrict__ keys, const uint32_t *num, unsigned long long cap, PassSpec ps,
            uint32_t *__restrict__ hist) {
    pdl_entry();
    __shared__ uint32_t s_h[kMaxPasses * 256];
    for (int i = threadIdx.x; i < ps.passes * 256; i += 256) s_h[i] = 0;
    __syncthreads();
    const unsigned long long M = num ? min((unsigned long long)*num, cap) : cap;
    const int lane = threadIdx.x & 31;
    for (unsigned long long b = (unsigned long long)blockIdx.x * 256; b < M; b += (unsigned long long)gridDim.x * 256) {
        const unsigned long long i = b + threadIdx.x;
        const bool valid = i < M;
        const K k = valid ? keys[i] : K(0);
        for (int p = 0; p < ps.passes; ++p) {
            const uint32_t d = valid ? (uint32_t)(k >> ps.shift[p]) & ((1u << ps.bits[p]) - 1u) : 256u;
            const uint32_t peers = __match_any_sync(0xffffffffu, d);
            if (valid && lane == __ffs(peers) - 1) atomicAdd(&s_h[p * 256 + d], (uint32_t)__popc(peers));
        }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < ps.passes * 256; i += 256)
        if (s_h[i]) atomicAdd(&hist[i], s_h[i]);
}

__global__ void __launch_bounds__(256) k_hist_scan(const uint32_t *__restrict__ hist, uint32_t *__restrict__ base) {
    pdl_entry();
    __shared__ uint32_t s_warp[256 / 32 + 1];
    const int p = blockIdx.x;
    uint32_t total;
    const uint32_t ex = block_exclusive_scan<256>(hist[p * 256 + threadIdx.x], s_warp, total);
    base[p * 256 + threadIdx.x] = ex;
}

// Per-tile instance counts (2D prefix of the difference array) -> ranges [start, end) and the
// digit bases of the tile passes.  One CTA.  After a capacity overflow every range is empty.
// One CTA: prefix sums of the per-row difference array (a warp per row, in shared memory when
// it fits) give the per-tile instance counts, then
// their exclusive scan gives the ranges and a histogram of each tile-pass digit the passes'
// digit bases.  With SMEM the difference array is staged into shared memory first.
template <bool SMEM>
__global__ void __launch_bounds__(1024)
k_tile_setup(int tiles_x, int tiles_y, const int *__restrict__ diff_g, uint32_t *__restrict__ counts_g,
             const uint32_t *num, unsigned long long capacity, PassSpec ps, uint32_t *__restrict__ ranges,
             uint32_t *__restrict__ digit_base) {
    pdl_entry();
    extern __shared__ uint32_t s_dyn[];
    __shared__ uint32_t s_h[kMaxPasses * 256];
    __shared__ unsigned long long s_warp[1024 / 32 + 1];
    __shared__ uint32_t s_warp32[1024 / 32 + 1];
    const int w1 = tiles_x + 1, n_tiles = tiles_x * tiles_y;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int *diff = diff_g;
    uint32_t *counts = counts_g;
    if (SMEM) {
        counts = s_dyn;
        int *d = reinterpret_cast<int *>(s_dyn + n_tiles);
        for (int i = threadIdx.x; i < w1 * (tiles_y + 1); i += 1024) d[i] = diff_g[i];
        diff = d;
    }
    for (int i = threadIdx.x; i < kMaxPasses * 256; i += 1024) s_h[i] = 0;
    __syncthreads();
    (void)num;
    for (int y = warp; y < tiles_y; y += 32) {  // prefix along x
        uint32_t carry = 0;
        for (int x0 = 0; x0 < tiles_x; x0 += 32) {
            const int x = x0 + lane;
            uint32_t v = x < tiles_x ? (uint32_t)diff[y * w1 + x] : 0u;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t u = __shfl_up_sync(0xffffffffu, v, o);
                if (lane >= o) v += u;
            }
            if (x < tiles_x) counts[y * tiles_x + x] = carry + v;
            carry += __shfl_sync(0xffffffffu, v, 31);
        }
    }
    __syncthreads();

    // M from the counts themselves (the sum of the member tiles, as the scan of tiles_touched
    // finds it), so that this kernel need not wait for that scan
    unsigned long long part = 0, M;
    for (int t = threadIdx.x; t < n_tiles; t += 1024) part += counts[t];
    block_exclusive_scan<1024>(part, s_warp, M);
    const bool overflow = M > capacity;
    unsigned long long carry = 0;
    for (int chunk = 0; chunk < n_tiles; chunk += 1024) {
        const int t = chunk + threadIdx.x;
        const uint32_t c = t < n_tiles ? counts[t] : 0u;
        unsigned long long total;
        const unsigned long long ex = carry + block_exclusive_scan<1024>((unsigned long long)c, s_warp, total);
        if (t < n_tiles) {
            // an empty tile's run is [0, 0), as the other strategy and the oracle write it
            ranges[2 * (size_t)t] = (overflow || c == 0) ? 0u : (uint32_t)ex;
            ranges[2 * (size_t)t + 1] = (overflow || c == 0) ? 0u : (uint32_t)(ex + c);
            if (c) {
#pragma unroll
                for (int p = 0; p < kMaxPasses; ++p)
                    if (p < ps.passes)
                        atomicAdd(&s_h[p * 256 + (((uint32_t)t >> ps.shift[p]) & ((1u << ps.bits[p]) - 1u))], c);
            }
        }
        carry += total;
    }
    __syncthreads();
    for (int p = 0; p < ps.passes; ++p) {
        const uint32_t v = threadIdx.x < 256 ? s_h[p * 256 + threadIdx.x] : 0u;
        uint32_t total;
        const uint32_t ex = block_exclusive_scan<1024>(v, s_warp32, total);
        if (threadIdx.x < 256) digit_base[p * 256 + threadIdx.x] = ex;
    }
}

// ---------------------------------------------------------------------------- reduce-then-scan passes
//
// One LSD pass without inter-CTA waiting: k_part_hist writes each partition's digit histogram
// digit-major (ph[d * n_parts + partition]), the three k_scan_* kernels turn that table into
// exclusive offsets -- digit-major order makes each entry the global output position of the
// partition's first key with that digit -- and k_downsweep ranks and scatters each partition.

constexpr int kScanBlock = 4096;  // values per CTA of the table scan (1024 threads x 4)

// The depth-then-tile strategy sorts with onesweep passes (1) or reduce-then-scan passes (0).
#ifndef DARB_PASS_ONESWEEP
#define DARB_PASS_ONESWEEP 1
#endif
constexpr bool kPassOnesweep = DARB_PASS_ONESWEEP != 0;

// Per-tile counts right after the depth compaction, over the visible splats in index order (1),
// or after the depth sort, in depth order (0).
#ifndef DARB_TILE_COUNTS_EARLY
#define DARB_TILE_COUNTS_EARLY 1
#endif
constexpr bool kTileCountsEarly = DARB_TILE_COUNTS_EARLY != 0;

// The duplication takes the runs of unpacked splats from the table k_tile_diff records, a warp
// per splat (1), or recomputes them, a thread per splat (0).
#ifndef DARB_RUN_TABLE
#define DARB_RUN_TABLE 1
#endif
constexpr bool kRunTable = DARB_RUN_TABLE != 0;

// CTAs per SM of the tile difference array (each privatises the array in shared memory and
// adds it to the global one at the end).
#ifndef DARB_TILE_DIFF_CTAS_PER_SM
#define DARB_TILE_DIFF_CTAS_PER_SM 4  // beside the depth passes, 256 threads: 4 -> 0.353 ms (8: 0.359; 1024 x 2: 0.371)
#endif

// Resident CTAs per SM the one-pass sort kernels are compiled for (their register budget).
#ifndef DARB_SORT_CTAS_PER_SM
#define DARB_SORT_CTAS_PER_SM 3
#endif
constexpr int kSortCtasPerSm = DARB_SORT_CTAS_PER_SM;

// Peer masks by match.any or by one ballot per digit bit (the default: the ballots measured
// faster, 0.462 -> 0.436 ms for the sort stage at 3M splats / 1080p).
#ifndef DARB_PEERS_BY_MATCH
#define DARB_PEERS_BY_MATCH 0
#endif
constexpr bool PEERS_BY_MATCH = DARB_PEERS_BY_MATCH != 0;


template <typename K>
__global__ void __launch_bounds__(kSortThreads)
k_part_hist(const K *__restrict__ keys, const uint32_t *num, unsigned long long cap, int shift, int bits,
            uint32_t n_parts, uint32_t *__restrict__ ph) {
    pdl_entry();
    __shared__ uint32_t s_h[256];
    const uint32_t radix = 1u << bits, mask = radix - 1u;
    for (int i = threadIdx.x; i < 256; i += kSortThreads) s_h[i] = 0;
    __syncthreads();
    const unsigned long long Mfull = num ? (unsigned long long)*num : cap;
    const uint32_t M = Mfull > cap ? 0u : (uint32_t)Mfull;
    const uint32_t base = blockIdx.x * (uint32_t)kSortTile;
    const int lane = threadIdx.x & 31;
    K kk[kSortItems];  // all loads in flight before the first warp vote
#pragma unroll
    for (int it = 0; it < kSortItems; ++it) {
        const uint32_t idx = base + it * kSortThreads + threadIdx.x;
        kk[it] = idx < M ? keys[idx] : K(0);
    }
#pragma unroll
    for (int it = 0; it < kSortItems; ++it) {
        const bool valid = base + it * kSortThreads + threadIdx.x < M;
        const uint32_t d = valid ? (uint32_t)(kk[it] >> shift) & mask : 0u;
        const uint32_t peers = (PEERS_BY_MATCH ? __match_any_sync(0xffffffffu, d) : match_digit(d, bits)) &
                               __ballot_sync(0xffffffffu, valid);
        if (valid && lane == __ffs(peers) - 1) atomicAdd(&s_h[d], (uint32_t)__popc(peers));
    }
    __syncthreads();
    for (uint32_t d = threadIdx.x; d < radix; d += kSortThreads) ph[(size_t)d * n_parts + blockIdx.x] = s_h[d];
}

__global__ void __launch_bounds__(1024)
k_scan_reduce(const uint32_t *__restrict__ data, unsigned long long count, uint32_t *__restrict__ sums) {
    pdl_entry();
    __shared__ uint32_t s_warp[1024 / 32 + 1];
    const unsigned long long base = (unsigned long long)blockIdx.x * kScanBlock;
    uint32_t v = 0;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const unsigned long long i = base + (unsigned long long)j * 1024 + threadIdx.x;
        if (i < count) v += data[i];
    }
    uint32_t total;
    block_exclusive_scan<1024>(v, s_warp, total);
    if (threadIdx.x == 0) sums[blockIdx.x] = total;
}

__global__ void __launch_bounds__(1024) k_scan_top(uint32_t *__restrict__ sums, int nb) {
    pdl_entry();
    __shared__ uint32_t s_warp[1024 / 32 + 1];
    uint32_t carry = 0;
    for (int chunk = 0; chunk < nb; chunk += 1024) {
        const int i = chunk + threadIdx.x;
        const uint32_t v = i < nb ? sums[i] : 0u;
        uint32_t total;
        const uint32_t ex = block_exclusive_scan<1024>(v, s_warp, total);
        if (i < nb) sums[i] = carry + ex;
        carry += total;
    }
}

__global__ void __launch_bounds__(1024)
k_scan_apply(uint32_t *__restrict__ data, unsigned long long count, const uint32_t *__restrict__ sums) {
    pdl_entry();
    __shared__ uint32_t s_warp[1024 / 32 + 1];
    const unsigned long long base = (unsigned long long)blockIdx.x * kScanBlock + (unsigned long long)threadIdx.x * 4;
    uint32_t v[4], sum = 0;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        v[j] = base + j < count ? data[base + j] : 0u;
        sum += v[j];
    }
    uint32_t total;
    uint32_t ex = block_exclusive_scan<1024>(sum, s_warp, total) + sums[blockIdx.x];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        if (base + j < count) data[base + j] = ex;
        ex += v[j];
    }
}

// Rank and scatter one partition with known per-digit global offsets (no look-back).
template <typename K, bool WRITE_KEYS>
__global__ void __launch_bounds__(kSortThreads, kSortCtasPerSm)
k_downsweep(const K *__restrict__ kin, const uint32_t *__restrict__ vin, K *__restrict__ kout,
            uint32_t *__restrict__ vout, const uint32_t *num, unsigned long long cap, int shift, int bits,
            const uint32_t *__restrict__ offsets, uint32_t n_parts) {
    pdl_entry();
    extern __shared__ __align__(16) unsigned char smem[];
    uint32_t *s_v = reinterpret_cast<uint32_t *>(smem);
    K *s_k = reinterpret_cast<K *>(smem + (size_t)kSortTile * 4);
    uint8_t *s_d = reinterpret_cast<uint8_t *>(smem + (size_t)kSortTile * 4);
    constexpr int NW = kSortThreads / 32;
    __shared__ uint32_t s_wh[NW][256];
    __shared__ uint32_t s_gbase[256];
    __shared__ uint32_t s_warp[NW + 1];

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const uint32_t radix = 1u << bits, mask = radix - 1u;
    if (num && (unsigned long long)*num > cap) return;  // overflow: sort nothing
    const uint32_t M = (uint32_t)(num ? min((unsigned long long)*num, cap) : cap);
    const uint32_t part = blockIdx.x;
    const uint32_t base = part * kSortTile;
    if (base >= M) return;
    for (int i = tid; i < NW * 256; i += kSortThreads) (&s_wh[0][0])[i] = 0;
    __syncthreads();

    K k[kSortItems];
    uint32_t v[kSortItems], rk[kSortItems];
#pragma unroll
    for (int it = 0; it < kSortItems; ++it) {
        const uint32_t idx = base + warp * (32 * kSortItems) + it * 32 + lane;
        if (idx < M) {
            k[it] = kin[idx];
            v[it] = vin ? vin[idx] : idx;
        } else {
            k[it] = ~K(0);  // the top digit, ranked after every valid key of the partition
            v[it] = 0;
        }
    }
    const uint32_t lt = lanemask_lt();
    // per-warp counts; each item's stable rank among the warp's items of its digit
#pragma unroll
    for (int it = 0; it < kSortItems; ++it) {
        const uint32_t d = (uint32_t)(k[it] >> shift) & mask;
        const uint32_t peers = PEERS_BY_MATCH ? __match_any_sync(0xffffffffu, d) : match_digit(d, bits);
        const int leader = __ffs(peers) - 1;
        uint32_t old = 0;
        if (lane == leader) old = atomicAdd(&s_wh[warp][d], (uint32_t)__popc(peers));
        rk[it] = __shfl_sync(0xffffffffu, old, leader) + __popc(peers & lt);
    }
    __syncthreads();
    const uint32_t dg = (uint32_t)tid;
    uint32_t cnt = 0;
    if (dg < radix) {
#pragma unroll
        for (int w = 0; w < NW; ++w) cnt += s_wh[w][dg];
    }
    uint32_t tot;
    const uint32_t cex = block_exclusive_scan<kSortThreads>(cnt, s_warp, tot);
    if (dg < radix) {
        // per-warp running positions start at the CTA offset of the digit plus earlier warps' counts
        uint32_t run = cex;
#pragma unroll
        for (int w = 0; w < NW; ++w) {
            const uint32_t c = s_wh[w][dg];
            s_wh[w][dg] = run;
            run += c;
        }
        s_gbase[dg] = offsets[(size_t)dg * n_parts + part] - cex;  // global = this + local position
    }
    __syncthreads();
#pragma unroll
    for (int it = 0; it < kSortItems; ++it) {
        const uint32_t d = (uint32_t)(k[it] >> shift) & mask;
        const uint32_t pos = s_wh[warp][d] + rk[it];
        if (WRITE_KEYS) s_k[pos] = k[it];
        else s_d[pos] = (uint8_t)d;
        s_v[pos] = v[it];
    }
    __syncthreads();
    const uint32_t nvalid = min((uint32_t)kSortTile, M - base);
    for (uint32_t j = tid; j < nvalid; j += kSortThreads) {
        uint32_t d;
        K kk = K(0);
        if (WRITE_KEYS) {
            kk = s_k[j];
            d = (uint32_t)(kk >> shift) & mask;
        } else {
            d = s_d[j];
        }
        const uint32_t dst = s_gbase[d] + j;
        if (WRITE_KEYS) kout[dst] = kk;
        vout[dst] = s_v[j];
    }
}

// ---------------------------------------------------------------------------- onesweep

template <typename K, bool WRITE_KEYS>
struct Staging {
    static constexpr size_t bytes = (size_t)kSortTile * ((WRITE_KEYS ? sizeof(K) : 1) + 4);
};

// Dynamic shared memory of the fused duplicate + first pass: the staging arrays, which also
// hold the partition's run starts (tile ids, splat ids and the kDupTile-bit mark) while the
// instances are generated.
template <bool WRITE_KEYS>
struct DupStaging {
    static constexpr size_t owners = (size_t)(2 * kDupTile + kDupTile / 32 + 4) * 4 + (size_t)kDupTile * 2;
    static constexpr size_t bytes = Staging<uint32_t, WRITE_KEYS>::bytes > owners ? Staging<uint32_t, WRITE_KEYS>::bytes
                                                                                   : owners;
};

struct SweepSmem {
    uint32_t wh[kSortThreads / 32][256];
    uint32_t cta_excl[256];
    uint32_t gbase[256];
    uint32_t warp[kSortThreads / 32 + 1];
    uint32_t part;
    int res[2];
};

// Claims this CTA's partition (in launch order, so that look-back only waits on CTAs that
// have started) and clears the per-warp digit counters.
__device__ __forceinline__ uint32_t sweep_begin(SweepSmem &sm, uint32_t *part_counter) {
    if (threadIdx.x == 0) sm.part = atomicAdd(part_counter, 1u);
    for (int i = threadIdx.x; i < (kSortThreads / 32) * 256; i += kSortThreads) (&sm.wh[0][0])[i] = 0;
    __syncthreads();
    return sm.part;
}

// Steps 1-4 of one stable LSD pass for a partition whose items are in registers (item `it` of
// lane l in warp w is input position base + w * 32 * kSortItems + it * 32 + l; invalid items
// carry the all-ones key): ranking, look-back for the digits' global bases, and the scatter.
// Staging may alias memory the caller used before, as long as its last read precedes this
// call's first barrier.
template <typename K, bool WRITE_KEYS>
__device__ __forceinline__ void sweep_partition(SweepSmem &sm, unsigned char *smem, const K (&k)[kSortItems],
                                                const uint32_t (&v)[kSortItems], uint32_t part, uint32_t base,
                                                uint32_t M, int shift, int bits,
                                                const uint32_t *__restrict__ digit_base, uint32_t *lookback,
                                                uint32_t *status, K *__restrict__ kout, uint32_t *__restrict__ vout) {
    uint32_t *s_v = reinterpret_cast<uint32_t *>(smem);
    K *s_k = reinterpret_cast<K *>(smem + (size_t)kSortTile * 4);
    uint8_t *s_d = reinterpret_cast<uint8_t *>(smem + (size_t)kSortTile * 4);
    constexpr int NW = kSortThreads / 32;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const uint32_t radix = 1u << bits, mask = radix - 1u;
    uint32_t rk[kSortItems];
    const uint32_t lt = lanemask_lt();
    // 1) Per-warp digit counts (one shared-memory atomic per group of equal digits).  The
    //    atomic's old value, broadcast to the group, plus the lower lanes of the group give each
    //    item's stable rank among the warp's items of its digit (item-major, lane-minor order).
#pragma unroll
    for (int it = 0; it < kSortItems; ++it) {
        const uint32_t d = (uint32_t)(k[it] >> shift) & mask;
        const uint32_t peers = PEERS_BY_MATCH ? __match_any_sync(0xffffffffu, d) : match_digit(d, bits);
        const int leader = __ffs(peers) - 1;
        uint32_t old = 0;
        if (lane == leader) old = atomicAdd(&sm.wh[warp][d], (uint32_t)__popc(peers));
        rk[it] = __shfl_sync(0xffffffffu, old, leader) + __popc(peers & lt);
    }
    __syncthreads();

    // 2) thread = digit: per-warp exclusive offsets and the CTA count, published at once so that
    //    successors can look back while this CTA is still ranking
    const uint32_t dg = (uint32_t)tid;
    uint32_t cnt = 0;
    uint32_t *mine = lookback + (size_t)part * radix + dg;
    if (dg < radix) {
#pragma unroll
        for (int w = 0; w < NW; ++w) {
            const uint32_t c = sm.wh[w][dg];
            sm.wh[w][dg] = cnt;
            cnt += c;
        }
        st_relaxed(mine, (part == 0 ? kFlagIncl : kFlagLocal) | cnt);
    }
    uint32_t tot;
    const uint32_t cex = block_exclusive_scan<kSortThreads>(cnt, sm.warp, tot);
    if (dg < radix) sm.cta_excl[dg] = cex;
    __syncthreads();

    // 3) staging at the CTA-local sorted position: the digit's CTA offset, the warp's offset
    //    within the digit, the item's rank within the warp (stable: input order)
#pragma unroll
    for (int it = 0; it < kSortItems; ++it) {
        const uint32_t d = (uint32_t)(k[it] >> shift) & mask;
        const uint32_t pos = sm.cta_excl[d] + sm.wh[warp][d] + rk[it];
        if (WRITE_KEYS) s_k[pos] = k[it];
        else s_d[pos] = (uint8_t)d;
        s_v[pos] = v[it];
    }

    // 4) decoupled look-back for the global base of each digit, 8 predecessors per round trip
    if (dg < radix) {
        uint32_t excl = 0;
        if (part > 0) {
            int p = (int)part - 1;
            bool found = false;
            while (!found) {
                const int nwin = min(kLookbackWindow, p + 1);
                uint32_t st[kLookbackWindow];
#pragma unroll
                for (int j = 0; j < kLookbackWindow; ++j)
                    st[j] = j < nwin ? ld_relaxed(lookback + (size_t)(p - j) * radix + dg) : 0u;
#pragma unroll
                for (int j = 0; j < kLookbackWindow; ++j) {
                    if (found || j >= nwin) break;
                    uint32_t sv = st[j];
                    int spins = 0, ns = 32;
                    while ((sv & ~kCountMask) == 0) {  // not published yet: wait for this one
                        if (++spins > kSpinLimit) {
                            atomicExch(status, (uint32_t)DARB_ERR_TIMEOUT);
                            sv = kFlagIncl;
                            break;
                        }
                        if (spins > 16) {  // poll busily at first, then back off
                            __nanosleep(ns);
                            ns = min(ns * 2, 512);
                        }
                        sv = ld_relaxed(lookback + (size_t)(p - j) * radix + dg);
                    }
                    excl += sv & kCountMask;
                    found = (sv & ~kCountMask) == kFlagIncl;
                }
                p -= nwin;
                if (p < 0) found = true;  // partition 0 publishes an inclusive count at once
            }
            st_relaxed(mine, kFlagIncl | ((excl + cnt) & kCountMask));
        }
        sm.gbase[dg] = digit_base[dg] + excl;
    }
    __syncthreads();
    const uint32_t nvalid = min((uint32_t)kSortTile, M - base);
    for (uint32_t j = tid; j < nvalid; j += kSortThreads) {
        uint32_t d;
        K kk = K(0);
        if (WRITE_KEYS) {
            kk = s_k[j];
            d = (uint32_t)(kk >> shift) & mask;
        } else {
            d = s_d[j];
        }
        const uint32_t dst = sm.gbase[d] + (j - sm.cta_excl[d]);
        if (dst < M) {  // always true for consistent digit bases; guards the buffers if they are not
            if (WRITE_KEYS) kout[dst] = kk;
            vout[dst] = s_v[j];
        }
    }
}

// One stable LSD pass over the digit of `bits` bits at `shift`.  M = min(*num, cap), or cap if
// num is null.  vin may be null: values are then the input positions (iota).
template <typename K, bool WRITE_KEYS>
__global__ void __launch_bounds__(kSortThreads, kSortCtasPerSm)
k_onesweep(const K *__restrict__ kin, const uint32_t *__restrict__ vin, K *__restrict__ kout,
           uint32_t *__restrict__ vout, const uint32_t *num, unsigned long long cap, int shift, int bits,
           const uint32_t *__restrict__ digit_base, uint32_t *lookback, uint32_t *part_counter, uint32_t *status) {
    pdl_entry();
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ SweepSmem sm;
    // After a capacity overflow the instance buffers hold only part of the instances while the
    // digit bases count all of them: sort nothing (the caller sees DARB_ERR_CAPACITY).
    if (num && (unsigned long long)*num > cap) return;
    const uint32_t part = sweep_begin(sm, part_counter);
    const uint32_t M = (uint32_t)(num ? min((unsigned long long)*num, cap) : cap);
    const uint32_t n_parts = (M + kSortTile - 1) / kSortTile;
    if (part >= n_parts) return;
    const uint32_t base = part * kSortTile;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    K k[kSortItems];
    uint32_t v[kSortItems];
#pragma unroll
    for (int it = 0; it < kSortItems; ++it) {
        const uint32_t idx = base + warp * (32 * kSortItems) + it * 32 + lane;
        if (idx < M) {
            k[it] = kin[idx];
            v[it] = vin ? vin[idx] : idx;
        } else {
            k[it] = ~K(0);  // the top digit, ranked after every valid key of the partition
            v[it] = 0;
        }
    }
    sweep_partition<K, WRITE_KEYS>(sm, smem, k, v, part, base, M, shift, bits, digit_base, lookback, status, kout,
                                   vout);
}

// The balanced duplication fused with the first tile pass: each CTA generates one partition
// of instances (tile id, splat) in depth order straight into registers -- the owner of
// instance j is the last depth-ordered splat whose offset is <= j -- and sorts it by the first
// tile digit, so the unsorted instances never go through HBM.
template <bool WRITE_KEYS>
__global__ void __launch_bounds__(kSortThreads, kSortCtasPerSm)
k_dup_sweep(int n, const uint32_t *__restrict__ order, const uint32_t *__restrict__ offs, const uint2 *__restrict__ bounds,
            const int4 *__restrict__ rect, const uint64_t *__restrict__ runs, const float2 *__restrict__ mean2d,
            const float4 *__restrict__ conic_o,
            SpanCtx sc, RunTable rt, int tiles_x, const uint32_t *num, unsigned long long cap, int bits,
            const uint32_t *__restrict__ digit_base, uint32_t *lookback, uint32_t *part_counter, uint32_t *status,
            uint32_t *__restrict__ kout, uint32_t *__restrict__ vout) {
    pdl_entry();
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ SweepSmem sm;
    if ((unsigned long long)*num > cap) return;  // overflow: nothing is emitted (status already set)
    const uint32_t part = sweep_begin(sm, part_counter);
    const uint32_t M = *num;
    const uint32_t n_parts = (M + kSortTile - 1) / kSortTile;
    if (part >= n_parts) return;
    const uint32_t lo = part * kSortTile, hi = min(M, lo + (uint32_t)kSortTile);
    uint32_t *s_base = reinterpret_cast<uint32_t *>(smem);
    uint32_t *s_val = s_base + kDupTile;
    uint32_t *s_mark = s_val + kDupTile;
    int *s_qn = reinterpret_cast<int *>(s_mark + kDupTile / 32);
    uint16_t *s_q = reinterpret_cast<uint16_t *>(s_qn + 4);
    for (int i = threadIdx.x; i < kDupTile / 32; i += kSortThreads) s_mark[i] = 0;
    if (threadIdx.x == 0) *s_qn = 0;
    const uint2 fl = bounds[part];
    const int first = (int)fl.x, count = min((int)fl.y - (int)fl.x + 1, kDupTile);  // every owner has >= 1 instance
    __syncthreads();
    partition_runs<kSortThreads>(first, count, lo, hi, offs, order, rect, runs, mean2d, conic_o, sc, rt, tiles_x,
                                 s_base, s_val, s_mark, s_q, s_qn);
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint32_t wbase = lo + (uint32_t)warp * (32 * kSortItems);
    uint32_t kk[kSortItems], vv[kSortItems];
#pragma unroll
    for (int it = 0; it < kSortItems; ++it) {
        const uint32_t j = wbase + it * 32 + lane;
        if (j < hi) {
            partition_lookup(j - lo, s_base, s_val, s_mark, kk[it], vv[it]);
        } else {
            kk[it] = 0xffffffffu;
            vv[it] = 0;
        }
    }
    __syncthreads();  // the staging arrays below reuse the run starts' memory
    sweep_partition<uint32_t, WRITE_KEYS>(sm, smem, kk, vv, part, lo, M, 0, bits, digit_base, lookback, status, kout,
                                          vout);
}

__global__ void __launch_bounds__(256)
k_ranges(const uint64_t *__restrict__ keys, const uint32_t *num, unsigned long long cap, uint32_t *__restrict__ ranges) {
    pdl_entry();
    if ((unsigned long long)*num > cap) return;  // overflow: ranges stay empty
    const unsigned long long M = *num;
    for (unsigned long long i = (unsigned long long)blockIdx.x * 256 + threadIdx.x; i < M;
         i += (unsigned long long)gridDim.x * 256) {
        const uint32_t t = (uint32_t)(keys[i] >> 32);
        if (i == 0 || (uint32_t)(keys[i - 1] >> 32) != t) ranges[2 * (size_t)t] = (uint32_t)i;
        if (i == M - 1 || (uint32_t)(keys[i + 1] >> 32) != t) ranges[2 * (size_t)t + 1] = (uint32_t)(i + 1);
    }
}

// Depth keys of the visible splats only, compacted in index order (so the depth sort, being
// stable, keeps equal depths in index order): k_vis_count counts each kScanTile block's visible
// splats, k_scan_block_sums turns the counts into block offsets and the total n_vis, and
// k_depth_compact writes (depth bits, index) of the visible splats to [0, n_vis).  Every later
// step reads the sorted order only below n_vis (the culled splats own no instance).
__global__ void __launch_bounds__(kScanThreads)
k_vis_count(int n, const int *__restrict__ radius, uint32_t *__restrict__ block_counts) {
    pdl_entry();
    __shared__ uint32_t s_warp[kScanThreads / 32 + 1];
    const int base = blockIdx.x * kScanTile;
    uint32_t c = 0;
#pragma unroll
    for (int j = 0; j < kScanItems; ++j) {
        const int i = base + j * kScanThreads + threadIdx.x;
        c += (i < n && radius[i] != 0) ? 1u : 0u;
    }
    uint32_t total;
    block_exclusive_scan<kScanThreads>(c, s_warp, total);
    if (threadIdx.x == 0) block_counts[blockIdx.x] = total;
}

// Depth digits at or above this bit are histogrammed with match.any aggregation, the lower ones
// with one shared-memory atomic per key.
#ifndef DARB_DEPTH_HIST_MATCH_SHIFT
#define DARB_DEPTH_HIST_MATCH_SHIFT 32  // every digit by plain atomics (16: 0.404, 8: 0.410 ms bin_sort)
#endif
__global__ void __launch_bounds__(kScanThreads)
k_depth_compact(int n, const int *__restrict__ radius, const float *__restrict__ depth,
                const unsigned long long *__restrict__ block_offsets, uint32_t *__restrict__ keys,
                uint32_t *__restrict__ ids0, PassSpec ps, uint32_t *__restrict__ hist) {
    pdl_entry();
    static_assert(kScanItems == 8, "two 16-byte loads per thread");
    __shared__ uint32_t s_warp[kScanThreads / 32 + 1];
    __shared__ uint32_t s_h[kMaxPasses * 256];
    for (int i = threadIdx.x; i < ps.passes * 256; i += kScanThreads) s_h[i] = 0;  // ordered by the scan
    const int base = blockIdx.x * kScanTile;
    const int i0 = base + (int)threadIdx.x * kScanItems;  // this thread's kScanItems consecutive splats
    const int lane = threadIdx.x & 31;
    int rad[kScanItems];
    uint32_t key[kScanItems];
    if (i0 + kScanItems <= n) {  // radius and depth are 16-byte aligned, i0 a multiple of 8
        const int4 r0 = *reinterpret_cast<const int4 *>(radius + i0), r1 = *reinterpret_cast<const int4 *>(radius + i0 + 4);
        const uint4 d0 = *reinterpret_cast<const uint4 *>(depth + i0), d1 = *reinterpret_cast<const uint4 *>(depth + i0 + 4);
        rad[0] = r0.x; rad[1] = r0.y; rad[2] = r0.z; rad[3] = r0.w;
        rad[4] = r1.x; rad[5] = r1.y; rad[6] = r1.z; rad[7] = r1.w;
        key[0] = d0.x; key[1] = d0.y; key[2] = d0.z; key[3] = d0.w;
        key[4] = d1.x; key[5] = d1.y; key[6] = d1.z; key[7] = d1.w;
    } else {
#pragma unroll
        for (int j = 0; j < kScanItems; ++j) {
            const bool valid = i0 + j < n;
            rad[j] = valid ? radius[i0 + j] : 0;
            key[j] = valid ? __float_as_uint(depth[i0 + j]) : 0u;
        }
    }
    uint32_t nv = 0;
#pragma unroll
    for (int j = 0; j < kScanItems; ++j) nv += (i0 + j < n && rad[j] != 0) ? 1u : 0u;
    uint32_t t;
    const uint32_t ex = block_exclusive_scan<kScanThreads>(nv, s_warp, t);
    uint32_t pv = (uint32_t)block_offsets[blockIdx.x] + ex;
#pragma unroll
    for (int j = 0; j < kScanItems; ++j) {
        const int i = i0 + j;
        const bool valid = i < n, v = valid && rad[j] != 0;
        if (v) {
            keys[pv] = key[j];
            ids0[pv] = (uint32_t)i;
            ++pv;
        }
#pragma unroll
        for (int p = 0; p < kMaxPasses; ++p) {  // digit histograms of the visible keys
            if (p >= ps.passes) break;
            const uint32_t d = v ? (key[j] >> ps.shift[p]) & ((1u << ps.bits[p]) - 1u) : 0xffffffffu;
            if (ps.shift[p] < DARB_DEPTH_HIST_MATCH_SHIFT) {  // spread digits: rare collisions in a warp
                if (v) atomicAdd(&s_h[p * 256 + d], 1u);
            } else {  // exponent side: few distinct digits, so a warp's equal digits add once
                const uint32_t peers = __match_any_sync(0xffffffffu, d);
                if (v && lane == __ffs(peers) - 1) atomicAdd(&s_h[p * 256 + d], (uint32_t)__popc(peers));
            }
        }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < ps.passes * 256; i += kScanThreads)
        if (s_h[i]) atomicAdd(&hist[i], s_h[i]);
}

// k_vis_count, k_scan_block_sums and k_depth_compact in one pass: each CTA claims the next
// kScanTile block of splats, counts its visible ones, takes their offset from a chained scan over
// the blocks before it, and writes their (depth bits, index) records and the digit histograms.
// The block holding splat n - 1 writes the visible count.
__global__ void __launch_bounds__(kScanThreads)
k_depth_compact_chained(int n, const int *__restrict__ radius, const float *__restrict__ depth,
                        unsigned long long *chain, uint32_t *claim, uint32_t *__restrict__ keys,
                        uint32_t *__restrict__ ids0, PassSpec ps, uint32_t *__restrict__ hist,
                        uint32_t *__restrict__ n_vis, uint32_t *status) {
    pdl_entry();
    static_assert(kScanItems == 8, "two 16-byte loads per thread");
    __shared__ uint32_t s_warp[kScanThreads / 32 + 1];
    __shared__ uint32_t s_h[kMaxPasses * 256];
    __shared__ int s_part;
    __shared__ unsigned long long s_base;
    for (int i = threadIdx.x; i < ps.passes * 256; i += kScanThreads) s_h[i] = 0;  // ordered by the claim
    const int part = claim_partition(claim, &s_part);
    const int base = part * kScanTile;
    const int i0 = base + (int)threadIdx.x * kScanItems;  // this thread's kScanItems consecutive splats
    const int lane = threadIdx.x & 31;
    int rad[kScanItems];
    uint32_t key[kScanItems];
    if (i0 + kScanItems <= n) {  // radius and depth are 16-byte aligned, i0 a multiple of 8
        const int4 r0 = *reinterpret_cast<const int4 *>(radius + i0), r1 = *reinterpret_cast<const int4 *>(radius + i0 + 4);
        const uint4 d0 = *reinterpret_cast<const uint4 *>(depth + i0), d1 = *reinterpret_cast<const uint4 *>(depth + i0 + 4);
        rad[0] = r0.x; rad[1] = r0.y; rad[2] = r0.z; rad[3] = r0.w;
        rad[4] = r1.x; rad[5] = r1.y; rad[6] = r1.z; rad[7] = r1.w;
        key[0] = d0.x; key[1] = d0.y; key[2] = d0.z; key[3] = d0.w;
        key[4] = d1.x; key[5] = d1.y; key[6] = d1.z; key[7] = d1.w;
    } else {
#pragma unroll
        for (int j = 0; j < kScanItems; ++j) {
            const bool valid = i0 + j < n;
            rad[j] = valid ? radius[i0 + j] : 0;
            key[j] = valid ? __float_as_uint(depth[i0 + j]) : 0u;
        }
    }
    uint32_t nv = 0;
#pragma unroll
    for (int j = 0; j < kScanItems; ++j) nv += (i0 + j < n && rad[j] != 0) ? 1u : 0u;
    uint32_t t;
    const uint32_t ex = block_exclusive_scan<kScanThreads>(nv, s_warp, t);
    if (threadIdx.x < 32) {
        const unsigned long long e = chain_exclusive(chain, part, t, status);
        if (threadIdx.x == 0) {
            s_base = e;
            if (base + kScanTile >= n) *n_vis = (uint32_t)(e + t);
        }
    }
    __syncthreads();
    uint32_t pv = (uint32_t)s_base + ex;
#pragma unroll
    for (int j = 0; j < kScanItems; ++j) {
        const int i = i0 + j;
        const bool valid = i < n, v = valid && rad[j] != 0;
        if (v) {
            keys[pv] = key[j];
            ids0[pv] = (uint32_t)i;
            ++pv;
        }
#pragma unroll
        for (int p = 0; p < kMaxPasses; ++p) {  // digit histograms of the visible keys
            if (p >= ps.passes) break;
            const uint32_t d = v ? (key[j] >> ps.shift[p]) & ((1u << ps.bits[p]) - 1u) : 0xffffffffu;
            if (ps.shift[p] < DARB_DEPTH_HIST_MATCH_SHIFT) {  // spread digits: rare collisions in a warp
                if (v) atomicAdd(&s_h[p * 256 + d], 1u);
            } else {  // exponent side: few distinct digits, so a warp's equal digits add once
                const uint32_t peers = __match_any_sync(0xffffffffu, d);
                if (v && lane == __ffs(peers) - 1) atomicAdd(&s_h[p * 256 + d], (uint32_t)__popc(peers));
            }
        }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < ps.passes * 256; i += kScanThreads)
        if (s_h[i]) atomicAdd(&hist[i], s_h[i]);
}

__global__ void __launch_bounds__(256)
k_depth_keys(int n, const int *__restrict__ radius, const float *__restrict__ depth, uint32_t *__restrict__ keys) {
    pdl_entry();
    const int i = blockIdx.x * 256 + threadIdx.x;
    if (i < n) keys[i] = radius[i] > 0 ? __float_as_uint(depth[i]) : 0xffffffffu;
}

// 64-bit keys of the sorted instances, one CTA per tile.
__global__ void __launch_bounds__(256)
k_keys64(const uint32_t *__restrict__ ranges, const uint32_t *__restrict__ vals, const float *__restrict__ depth,
         int n, uint64_t *__restrict__ keys) {
    pdl_entry();
    const uint32_t t = blockIdx.x;
    const uint32_t a = ranges[2 * t], b = ranges[2 * t + 1];
    for (uint32_t i = a + threadIdx.x; i < b; i += 256) {
        const uint32_t v = vals[i];
        keys[i] = ((uint64_t)t << 32) | (v < (uint32_t)n ? __float_as_uint(depth[v]) : 0u);
    }
}

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

PassSpec split_bits(int total_bits) {
    PassSpec ps{};
    const int tb = std::max(total_bits, 1);
    ps.passes = (tb + 7) / 8;
    int shift = 0;
    for (int p = 0; p < ps.passes; ++p) {
        const int b = (tb - shift + (ps.passes - p) - 1) / (ps.passes - p);
        ps.shift[p] = shift;
        ps.bits[p] = b;
        shift += b;
    }
    return ps;
}

// One reduce-then-scan pass.  ph: partition histograms (filled here unless hist_ready); table
// scan sums in `sums`.  n_parts = ceil(grid / kSortTile).
template <typename K, bool WK>
cudaError_t launch_rts_pass(const K *kin, const uint32_t *vin, K *kout, uint32_t *vout, const uint32_t *num,
                            unsigned long long cap, uint64_t grid, int shift, int bits, uint32_t *ph,
                            uint32_t *sums, bool hist_ready, cudaStream_t st) {
    const uint32_t n_parts = (uint32_t)((grid + kSortTile - 1) / kSortTile);
    if (n_parts == 0) return cudaSuccess;
    if (!hist_ready) launch_k(k_part_hist<K>, n_parts, kSortThreads, 0, st, kin, num, cap, shift, bits, n_parts, ph);
    const unsigned long long count = (unsigned long long)n_parts << bits;
    const int nb = (int)((count + kScanBlock - 1) / kScanBlock);
    launch_k(k_scan_reduce, nb, 1024, 0, st, ph, count, sums);
    launch_k(k_scan_top, 1, 1024, 0, st, sums, nb);
    launch_k(k_scan_apply, nb, 1024, 0, st, ph, count, sums);
    const size_t smem = Staging<K, WK>::bytes;
    cudaError_t e = cudaFuncSetAttribute(k_downsweep<K, WK>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    launch_k(k_downsweep<K, WK>, n_parts, kSortThreads, smem, st, kin, vin, kout, vout, num, cap, shift, bits, ph,
             n_parts);
    return cudaGetLastError();
}

template <typename K, bool WK>
cudaError_t launch_pass(const K *kin, const uint32_t *vin, K *kout, uint32_t *vout, const uint32_t *num,
                        unsigned long long cap, uint64_t grid_instances, int shift, int bits, const uint32_t *base,
                        uint32_t *lookback, uint32_t *counter, uint32_t *status, cudaStream_t st) {
    const size_t smem = Staging<K, WK>::bytes;
    cudaError_t e = cudaFuncSetAttribute(k_onesweep<K, WK>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const unsigned n_parts = (unsigned)((grid_instances + kSortTile - 1) / kSortTile);
    if (n_parts == 0) return cudaSuccess;
    launch_k(k_onesweep<K, WK>, n_parts, kSortThreads, smem, st, kin, vin, kout, vout, num, cap, shift, bits, base,
             lookback, counter, status);
    return cudaGetLastError();
}

}  // namespace

// ---------------------------------------------------------------------------- workspace

namespace {
// Entries of the run table: at most a quarter of the instance capacity, at least 64k.  A
// splat whose rows no longer fit is marked and its runs are recomputed by the duplication.
#ifndef DARB_RUN_TABLE_MAX
#define DARB_RUN_TABLE_MAX 0xffffffffu  // a test build caps it to reach the recomputing fallback
#endif
uint64_t run_table_entries(uint64_t capacity) {
    return std::min<uint64_t>(std::max<uint64_t>(capacity / 4, 1u << 16), DARB_RUN_TABLE_MAX);
}

struct Layout {
    size_t total;
    size_t off[24];
};

// Offsets of the workspace regions.  Regions 0..9 are data; [zero_begin, zero_end) is zeroed per call.
Layout layout(int n, uint64_t capacity, int tiles_x, int tiles_y, int strategy, int tile_bits) {
    const int n_tiles = tiles_x * tiles_y;
    const size_t nb = (size_t)(n + kScanTile - 1) / kScanTile;
    const size_t parts_cap = (capacity + kSortTile - 1) / kSortTile;
    const size_t parts_n = ((size_t)n + kSortTile - 1) / kSortTile;
    Layout L{};
    size_t b = 0;
    auto put = [&](int i, size_t bytes) {
        L.off[i] = b;
        b += align256(bytes);
    };
    if (strategy == DARB_SORT_KEYS64) {
        const int passes = (32 + tile_bits + 7) / 8;
        put(0, capacity * 8);  // keys_alt
        put(1, capacity * 4);  // vals_alt
        put(2, 0);
        put(3, 0);
        put(4, 0);
        put(5, 0);
        put(6, nb * 4);        // block sums
        put(7, nb * 8);        // block offsets
        put(8, 0);
        put(15, 0);
        put(16, 0);
        put(17, 0);
        put(18, 0);
        put(19, 0);
        put(20, 0);
        put(21, 0);
        put(22, 0);
        put(23, 0);
        put(9, (size_t)kMaxPasses * 256 * 4);  // digit bases
        put(10, (size_t)kMaxPasses * 256 * 4); // --- zeroed from here: histograms
        put(11, (size_t)passes * parts_cap * 256 * 4);  // look-back
        put(12, 0);
        put(13, (size_t)kMaxPasses * 4 * 2);   // partition counters
    } else {
        const int passes = split_bits(tile_bits).passes;
        put(0, capacity * 4);  // tile keys A
        put(1, capacity * 4);  // values A
        put(2, capacity * 4);  // tile keys B
        put(3, capacity * 4);  // values B
        put(4, (size_t)n * 4 * 2);  // depth keys ping-pong
        put(5, (size_t)n * 4 * 3);  // compacted ids, then the depth values ping-pong (sorted order ends here)
        put(6, nb * 4);
        put(7, nb * 8);
        put(8, (size_t)kMaxPasses * 256 * 4);  // tile digit bases
        put(9, (size_t)kMaxPasses * 256 * 4);  // depth digit bases
        put(15, ((size_t)n + 1) * 4);           // per-position instance offsets in depth order
        put(16, (size_t)n_tiles * 4);           // per-tile instance counts
        put(20, parts_cap * 8);                 // first and last owner of every tile-pass partition
        put(21, (size_t)n * 4);                 // run-table slot of every splat
        put(22, (size_t)run_table_entries(capacity) * 4);  // run table
        put(11, parts_cap * 256 * 4);           // tile-pass partition histograms / offsets
        put(12, parts_n * 256 * 4);             // depth-pass partition histograms / offsets
        put(17, ((std::max(parts_cap, parts_n) * 256 + 4095) / 4096 + 1) * 4);  // table-scan block sums
        // --- zeroed per call: histograms (+ spare), the tile difference array, onesweep look-backs
        put(10, (size_t)2 * kMaxPasses * 256 * 4 + (size_t)(tiles_x + 1) * (tiles_y + 1) * 4);
        put(18, kPassOnesweep ? (size_t)passes * parts_cap * 256 * 4 : 0);  // tile-pass look-back
        put(19, kPassOnesweep ? (size_t)4 * parts_n * 256 * 4 : 0);         // depth-pass look-back
        put(23, kPassOnesweep ? nb * 8 * 2 : 0);  // chained-scan words: the compaction's, the offsets'
        // onesweep partition counters, visible count, run-table fill, the chained scans' claims
        put(13, (size_t)(kMaxPasses * 2 + 4) * 4);
    }
    L.off[14] = b;
    L.total = b + 256;
    return L;
}
}  // namespace

int sort_tile_bits(int n_tiles) { return log2_ceil((uint32_t)n_tiles); }

namespace {
// k_tile_diff over the visible splats (order: their ids, n_vis: their count; null: every splat)
// and k_tile_setup: per-tile instance counts -> ranges and the tile passes' digit bases.
cudaError_t launch_tile_counts(int n, const uint32_t *order, const uint32_t *n_vis, const ProjectedIn &proj,
                               const SpanCtx &sc, const RunTable &rt, int tiles_x, int tiles_y, int *diff,
                               uint32_t *counts,
                               const BinOut &out, unsigned long long cap, const PassSpec &tps, uint32_t *tbase,
                               cudaStream_t st) {
    const int n_tiles = tiles_x * tiles_y;
    if (n > 0) {
        const int diff_size = (tiles_x + 1) * (tiles_y + 1);
        const size_t smem = (size_t)diff_size * 4;
        if (smem <= kMaxDiffSmem) {
            const cudaError_t e =
                cudaFuncSetAttribute(k_tile_diff<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            if (e != cudaSuccess) return e;
            const int blocks = std::min((n + DARB_TILE_DIFF_THREADS - 1) / DARB_TILE_DIFF_THREADS,
                                        DARB_TILE_DIFF_CTAS_PER_SM * kGridSms);
            launch_k(k_tile_diff<true>, blocks, DARB_TILE_DIFF_THREADS, smem, st, n, order, n_vis, proj.radius, proj.tile_rect,
                     proj.tile_runs, proj.mean2d, proj.conic_o, sc, rt, tiles_x, diff_size, diff);
        } else {
            launch_k(k_tile_diff<false>, (n + DARB_TILE_DIFF_THREADS - 1) / DARB_TILE_DIFF_THREADS,
                     DARB_TILE_DIFF_THREADS, 0, st, n, order, n_vis, proj.radius, proj.tile_rect,
                     proj.tile_runs, proj.mean2d, proj.conic_o, sc, rt, tiles_x, diff_size, diff);
        }
    }
    const size_t setup_smem = ((size_t)n_tiles + (size_t)(tiles_x + 1) * (tiles_y + 1)) * 4;
    if (setup_smem <= kMaxSetupSmem) {
        const cudaError_t e =
            cudaFuncSetAttribute(k_tile_setup<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)setup_smem);
        if (e != cudaSuccess) return e;
        launch_k(k_tile_setup<true>, 1, 1024, setup_smem, st, tiles_x, tiles_y, diff, counts, out.num_instances, cap,
                 tps, out.ranges, tbase);
    } else {
        launch_k(k_tile_setup<false>, 1, 1024, 0, st, tiles_x, tiles_y, diff, counts, out.num_instances, cap, tps,
                 out.ranges, tbase);
    }
    return cudaGetLastError();
}
}  // namespace

size_t sort_workspace_bytes(int n, uint64_t capacity, int tiles_x, int tiles_y, int strategy) {
    return layout(n, capacity, tiles_x, tiles_y, strategy, sort_tile_bits(tiles_x * tiles_y)).total;
}

namespace {
// The side stream of a device that takes the per-tile counts beside the depth passes, and its
// fork / join events; created on first use, kept for the process.
struct SortSide {
    std::mutex mu;
    bool ready = false;
    cudaStream_t s = nullptr;
    cudaEvent_t fork = nullptr, join = nullptr;
};
constexpr int kMaxDevicesSort = 64;
SortSide g_sort_side[kMaxDevicesSort];

cudaError_t sort_side_init(SortSide &P) {
    if (P.ready) return cudaSuccess;
    cudaError_t e = cudaStreamCreateWithFlags(&P.s, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&P.fork, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&P.join, cudaEventDisableTiming);
    if (e == cudaSuccess) P.ready = true;
    return e;
}

// Makes st wait for the side stream's work once, on every way out of the launcher.
struct SideJoin {
    cudaStream_t st = nullptr;
    cudaEvent_t ev = nullptr;
    bool pending = false;
    cudaError_t join() {
        if (!pending) return cudaSuccess;
        pending = false;
        return cudaStreamWaitEvent(st, ev, 0);
    }
    ~SideJoin() { join(); }
};
}  // namespace

// Per-tile counts beside the depth passes (1), or in line on the caller's stream (0).
#ifndef DARB_TILE_COUNTS_FORK
#define DARB_TILE_COUNTS_FORK 1
#endif

cudaError_t launch_bin_sort(int n, const ProjectedIn &proj, int tiles_x, int tiles_y, const SpanCtx &sc,
                            uint64_t capacity,
                            int strategy, void *workspace, const BinOut &out, uint64_t *num_instances_host,
                            bool *capacity_exceeded, cudaStream_t st, bool allow_fork) {
    const int n_tiles = tiles_x * tiles_y;
    const int tile_bits = sort_tile_bits(n_tiles);
    const Layout L = layout(n, capacity, tiles_x, tiles_y, strategy, tile_bits);
    unsigned char *w = reinterpret_cast<unsigned char *>(
        (reinterpret_cast<uintptr_t>(workspace) + 255) & ~(uintptr_t)255);
    auto at = [&](int i) { return reinterpret_cast<void *>(w + L.off[i]); };
    const int nb = (n + kScanTile - 1) / kScanTile;
    const unsigned long long cap = capacity;
    *capacity_exceeded = false;
    cudaError_t e;
#define TRY(x)                          \
    do {                                \
        e = (x);                        \
        if (e != cudaSuccess) return e; \
    } while (0)
    TRY(launch_zero(st, at(10), L.off[14] - L.off[10], out.status, sizeof(uint32_t), out.ranges,
                    (size_t)n_tiles * 2 * sizeof(uint32_t)));
    uint32_t *block_sums = reinterpret_cast<uint32_t *>(at(6));
    auto *block_off = reinterpret_cast<unsigned long long *>(at(7));
    uint32_t *counters = reinterpret_cast<uint32_t *>(at(13));
    // chained-scan words (zeroed with the counters): the compaction's nb, then the offsets' nb
    unsigned long long *chains = reinterpret_cast<unsigned long long *>(at(23));

    if (strategy == DARB_SORT_KEYS64) {
        if (nb > 0) launch_k(k_block_sums, nb, kScanThreads, 0, st, n, proj.tiles_touched, nullptr, nullptr, block_sums);
        launch_k(k_scan_block_sums, 1, 1024, 0, st, nb, block_sums, block_off, out.num_instances, out.status, cap);
        TRY(cudaGetLastError());
        uint64_t grid = capacity;
        if (num_instances_host) {
            uint32_t M = 0;
            TRY(cudaMemcpyAsync(&M, out.num_instances, 4, cudaMemcpyDeviceToHost, st));
            TRY(cudaStreamSynchronize(st));
            *num_instances_host = M;
            if (M > capacity) {
                *capacity_exceeded = true;
                return cudaSuccess;
            }
            grid = M;
        }
        const int passes = (32 + tile_bits + 7) / 8;
        uint64_t *ka = (passes % 2 == 0) ? out.keys : reinterpret_cast<uint64_t *>(at(0));
        uint32_t *va = (passes % 2 == 0) ? out.values : reinterpret_cast<uint32_t *>(at(1));
        uint64_t *kb = (passes % 2 == 0) ? reinterpret_cast<uint64_t *>(at(0)) : out.keys;
        uint32_t *vb = (passes % 2 == 0) ? reinterpret_cast<uint32_t *>(at(1)) : out.values;
        if (nb > 0)
            launch_k(k_duplicate, nb, kScanThreads, 0, st, n, proj.tiles_touched, block_off, proj.tile_rect,
                     proj.mean2d, proj.conic_o, sc, proj.depth, tiles_x, cap, ka, va);
        if (grid == 0) return cudaGetLastError();
        PassSpec ps{};
        ps.passes = passes;
        for (int p = 0; p < passes; ++p) {
            ps.shift[p] = 8 * p;
            ps.bits[p] = 8;
        }
        uint32_t *hist = reinterpret_cast<uint32_t *>(at(10));
        uint32_t *dbase = reinterpret_cast<uint32_t *>(at(9));
        const int hb = (int)std::min<uint64_t>((grid + 255) / 256, kGridSms * 8);
        launch_k(k_sort_hist<uint64_t>, hb, 256, 0, st, ka, out.num_instances, cap, ps, hist);
        launch_k(k_hist_scan, passes, 256, 0, st, hist, dbase);
        TRY(cudaGetLastError());
        const size_t lb_stride = ((capacity + kSortTile - 1) / kSortTile) * 256;
        uint32_t *lb = reinterpret_cast<uint32_t *>(at(11));
        for (int p = 0; p < passes; ++p) {
            TRY((launch_pass<uint64_t, true>(ka, va, kb, vb, out.num_instances, cap, grid, 8 * p, 8, dbase + p * 256,
                                             lb + p * lb_stride, counters + p, out.status, st)));
            std::swap(ka, kb);
            std::swap(va, vb);
        }
        const int rb = (int)std::min<uint64_t>((grid + 255) / 256, kGridSms * 16);
        launch_k(k_ranges, rb, 256, 0, st, ka, out.num_instances, cap, out.ranges);
        return cudaGetLastError();
    }

    // DEPTH_THEN_TILE
    const PassSpec tps = split_bits(tile_bits);
    int *diff = reinterpret_cast<int *>(at(10)) + 2 * kMaxPasses * 256;
    uint32_t *counts = reinterpret_cast<uint32_t *>(at(16));
    uint32_t *tbase = reinterpret_cast<uint32_t *>(at(8));
    bool tile_counts_done = false;
    // the side stream of this device, held (with its mutex) until the launcher returns
    SortSide *side = nullptr;
    std::unique_lock<std::mutex> side_lock;
    SideJoin side_join;  // declared after the lock: it joins before the lock is released
    if (allow_fork && DARB_TILE_COUNTS_FORK && kTileCountsEarly && kPassOnesweep && n > 0) {
        int dev = 0;
        TRY(cudaGetDevice(&dev));
        if (dev >= 0 && dev < kMaxDevicesSort) {
            side_lock = std::unique_lock<std::mutex>(g_sort_side[dev].mu);
            TRY(sort_side_init(g_sort_side[dev]));
            side = &g_sort_side[dev];
        }
    }
    const RunTable rt{reinterpret_cast<uint32_t *>(at(21)), kRunTable ? reinterpret_cast<uint32_t *>(at(22)) : nullptr,
                      counters + 2 * kMaxPasses + 1, (uint32_t)run_table_entries(capacity)};
    // 1) depth order of the splats (4 stable 8-bit passes over N keys)
    uint32_t *kbuf[2] = {reinterpret_cast<uint32_t *>(at(4)), reinterpret_cast<uint32_t *>(at(4)) + n};
    // vbuf[0]: the compacted visible ids in index order, which the per-tile counts read on the
    // side stream while the depth passes run, so the passes' values alternate between vbuf[1]
    // and vbuf[2] and never overwrite it
    uint32_t *vbuf[3] = {reinterpret_cast<uint32_t *>(at(5)), reinterpret_cast<uint32_t *>(at(5)) + n,
                         reinterpret_cast<uint32_t *>(at(5)) + 2 * (size_t)n};
    const uint32_t *order = nullptr;  // sorted splat ids
    const uint32_t *n_vis_dev = nullptr;  // visible count, when order starts with exactly the visible splats
    uint32_t *sums = reinterpret_cast<uint32_t *>(at(17));
    if (n > 0) {
        const PassSpec dps = split_bits(32);
        uint32_t *dph = reinterpret_cast<uint32_t *>(at(12));
        uint32_t *dbase = reinterpret_cast<uint32_t *>(at(9));
        const uint32_t *n_vis = nullptr;  // keys sorted: all n, or the visible n_vis (device)
        const uint32_t *vin = nullptr;    // first pass: values are the splat indices
        if (kPassOnesweep) {
            uint32_t *nv = counters + 2 * kMaxPasses;
            uint32_t *dhist = reinterpret_cast<uint32_t *>(at(10)) + kMaxPasses * 256;
            if (DARB_CHAINED_SCANS) {  // visible count, its scan and the compaction in one chained pass
                launch_k(k_depth_compact_chained, nb, kScanThreads, 0, st, n, proj.radius, proj.depth, chains,
                         counters + 2 * kMaxPasses + 2, kbuf[0], vbuf[0], dps, dhist, nv, out.status);
            } else {
                launch_k(k_vis_count, nb, kScanThreads, 0, st, n, proj.radius, block_sums);
                launch_k(k_scan_block_sums, 1, 1024, 0, st, nb, block_sums, block_off, nv, out.status,
                         (unsigned long long)n);
                launch_k(k_depth_compact, nb, kScanThreads, 0, st, n, proj.radius, proj.depth, block_off, kbuf[0],
                         vbuf[0], dps, dhist);
            }
            n_vis = nv;
            n_vis_dev = nv;
            vin = vbuf[0];
            launch_k(k_hist_scan, dps.passes, 256, 0, st, dhist, dbase);
            if (kTileCountsEarly) {
                // the per-tile counts need no depth order: walk the visible splats in index order
                // (coalesced reads) before the depth passes overwrite this compacted list; on the
                // side stream they run beside the (latency-bound) depth passes
                cudaStream_t ts = st;
                if (side) {
                    TRY(cudaEventRecord(side->fork, st));
                    TRY(cudaStreamWaitEvent(side->s, side->fork, 0));
                    ts = side->s;
                }
                TRY(launch_tile_counts(n, vbuf[0], nv, proj, sc, rt, tiles_x, tiles_y, diff, counts, out, cap, tps,
                                       tbase, ts));
                if (side) {
                    TRY(cudaEventRecord(side->join, side->s));
                    side_join.st = st;
                    side_join.ev = side->join;
                    side_join.pending = true;
                }
                tile_counts_done = true;
            }
        } else {
            launch_k(k_depth_keys, (n + 255) / 256, 256, 0, st, n, proj.radius, proj.depth, kbuf[0]);
        }
        TRY(cudaGetLastError());
        uint32_t *lbd = reinterpret_cast<uint32_t *>(at(19));
        const size_t lbd_stride = (((size_t)n + kSortTile - 1) / kSortTile) * 256;
        int cur = 0;
        for (int p = 0; p < dps.passes; ++p) {
            const int nxt = 1 - cur;
            const bool last = p == dps.passes - 1;
            uint32_t *vout = vbuf[1 + (p & 1)];
            if (kPassOnesweep) {
                if (last)
                    TRY((launch_pass<uint32_t, false>(kbuf[cur], vin, nullptr, vout, n_vis, (unsigned long long)n,
                                                      (uint64_t)n, dps.shift[p], dps.bits[p], dbase + p * 256,
                                                      lbd + p * lbd_stride, counters + kMaxPasses + p, out.status, st)));
                else
                    TRY((launch_pass<uint32_t, true>(kbuf[cur], vin, kbuf[nxt], vout, n_vis, (unsigned long long)n,
                                                     (uint64_t)n, dps.shift[p], dps.bits[p], dbase + p * 256,
                                                     lbd + p * lbd_stride, counters + kMaxPasses + p, out.status, st)));
            } else {
                if (last)
                    TRY((launch_rts_pass<uint32_t, false>(kbuf[cur], vin, nullptr, vout, nullptr,
                                                          (unsigned long long)n, (uint64_t)n, dps.shift[p], dps.bits[p],
                                                          dph, sums, false, st)));
                else
                    TRY((launch_rts_pass<uint32_t, true>(kbuf[cur], vin, kbuf[nxt], vout, nullptr,
                                                         (unsigned long long)n, (uint64_t)n, dps.shift[p], dps.bits[p],
                                                         dph, sums, false, st)));
            }
            vin = vout;
            cur = nxt;
        }
        order = vin;
    }
    // 2) scan of tiles_touched in depth order (with the onesweep passes: chained, in step 4)
    uint32_t *offs = reinterpret_cast<uint32_t *>(at(15));
    uint2 *bounds = kPassOnesweep ? reinterpret_cast<uint2 *>(at(20)) : nullptr;
    const uint32_t max_parts = (uint32_t)((capacity + kSortTile - 1) / kSortTile);
    const bool chained = DARB_CHAINED_SCANS && kPassOnesweep && n_vis_dev;
    if (chained) {
        // 4, ahead) per-position offsets and owners, M and the capacity check in one chained pass
        if (nb > 0)
            launch_k(k_splat_offsets_chained, nb, kScanThreads, 0, st, n, order, proj.tiles_touched, n_vis_dev,
                     chains + nb, counters + 2 * kMaxPasses + 3, out.num_instances, out.status, cap, offs, bounds,
                     max_parts);
    } else {
        if (nb > 0)
            launch_k(k_block_sums, nb, kScanThreads, 0, st, n, proj.tiles_touched, order, n_vis_dev, block_sums);
        launch_k(k_scan_block_sums, 1, 1024, 0, st, nb, block_sums, block_off, out.num_instances, out.status, cap);
    }
    TRY(cudaGetLastError());
    uint64_t grid = capacity;
    if (num_instances_host) {
        uint32_t M = 0;
        TRY(cudaMemcpyAsync(&M, out.num_instances, 4, cudaMemcpyDeviceToHost, st));
        TRY(cudaStreamSynchronize(st));
        *num_instances_host = M;
        if (M > capacity) {
            *capacity_exceeded = true;
            return cudaSuccess;
        }
        grid = M;
    }
    // 3) per-tile counts from the rectangles -> ranges and tile-pass digit bases (done above
    //    when the compacted index order was available)
    if (!tile_counts_done)
        TRY(launch_tile_counts(n, n_vis_dev ? order : nullptr, n_vis_dev, proj, sc, rt, tiles_x, tiles_y, diff,
                               counts, out, cap, tps, tbase, st));
    // 4) per-position offsets, then the balanced duplication in depth order
    uint32_t *tk_a = reinterpret_cast<uint32_t *>(at(0)), *tv_a = reinterpret_cast<uint32_t *>(at(1));
    uint32_t *tk_b = reinterpret_cast<uint32_t *>(at(2)), *tv_b = reinterpret_cast<uint32_t *>(at(3));
    if (nb > 0 && !chained)
        launch_k(k_splat_offsets, nb, kScanThreads, 0, st, n, order, proj.tiles_touched, n_vis_dev, block_off,
                 out.num_instances,
                 offs, bounds, max_parts);
    TRY(side_join.join());  // the duplication needs the tile counts' ranges, digit bases and run table
    uint32_t *tph = reinterpret_cast<uint32_t *>(at(11));
    const uint32_t n_parts = (uint32_t)((grid + kSortTile - 1) / kSortTile);
    uint32_t *lb = reinterpret_cast<uint32_t *>(at(18));
    const size_t lb_stride = ((capacity + kSortTile - 1) / kSortTile) * 256;
    if (grid > 0 && kPassOnesweep) {
        // 5) duplication fused with the first tile pass, then the remaining stable LSD passes;
        //    the last writes only the output values
        const bool last0 = tps.passes == 1;
        uint32_t *k0 = last0 ? nullptr : tk_b, *v0 = last0 ? out.values : tv_b;
        const size_t smem = last0 ? DupStaging<false>::bytes : DupStaging<true>::bytes;
        if (last0) {
            TRY(cudaFuncSetAttribute(k_dup_sweep<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
            launch_k(k_dup_sweep<false>, n_parts, kSortThreads, smem, st, n, order, offs, bounds, proj.tile_rect,
                     proj.tile_runs, proj.mean2d, proj.conic_o, sc, rt, tiles_x, out.num_instances, cap, tps.bits[0],
                     tbase, lb, counters, out.status, k0, v0);
        } else {
            TRY(cudaFuncSetAttribute(k_dup_sweep<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
            launch_k(k_dup_sweep<true>, n_parts, kSortThreads, smem, st, n, order, offs, bounds, proj.tile_rect,
                     proj.tile_runs, proj.mean2d, proj.conic_o, sc, rt, tiles_x, out.num_instances, cap, tps.bits[0],
                     tbase, lb, counters, out.status, k0, v0);
        }
        TRY(cudaGetLastError());
        uint32_t *ka = tk_b, *va = tv_b, *kb = tk_a, *vb = tv_a;
        for (int p = 1; p < tps.passes; ++p) {
            const bool last = p == tps.passes - 1;
            if (last)
                TRY((launch_pass<uint32_t, false>(ka, va, nullptr, out.values, out.num_instances, cap, grid,
                                                  tps.shift[p], tps.bits[p], tbase + p * 256, lb + p * lb_stride,
                                                  counters + p, out.status, st)));
            else
                TRY((launch_pass<uint32_t, true>(ka, va, kb, vb, out.num_instances, cap, grid, tps.shift[p],
                                                 tps.bits[p], tbase + p * 256, lb + p * lb_stride, counters + p,
                                                 out.status, st)));
            std::swap(ka, kb);
            std::swap(va, vb);
        }
    } else if (grid > 0) {
        // reduce-then-scan passes: the duplication also writes the first pass's histograms
        if (n > 0)
            launch_k(k_duplicate_balanced, n_parts, kScanThreads, 0, st, n, order, offs, proj.tile_rect,
                     proj.tile_runs, proj.mean2d, proj.conic_o, sc, rt, tiles_x, out.num_instances, cap, tk_a, tv_a,
                     tps.bits[0], n_parts, tph);
        else
            TRY(cudaMemsetAsync(tph, 0, ((size_t)n_parts << tps.bits[0]) * 4, st));
        TRY(cudaGetLastError());
        uint32_t *ka = tk_a, *va = tv_a, *kb = tk_b, *vb = tv_b;
        for (int p = 0; p < tps.passes; ++p) {
            const bool last = p == tps.passes - 1;
            uint32_t *kout = last ? nullptr : kb;
            uint32_t *vout = last ? out.values : vb;
            const bool ready = p == 0;
            if (last)
                TRY((launch_rts_pass<uint32_t, false>(ka, va, kout, vout, out.num_instances, cap, grid,
                                                      tps.shift[p], tps.bits[p], tph, sums, ready, st)));
            else
                TRY((launch_rts_pass<uint32_t, true>(ka, va, kout, vout, out.num_instances, cap, grid,
                                                     tps.shift[p], tps.bits[p], tph, sums, ready, st)));
            if (!last) {
                std::swap(ka, kb);
                std::swap(va, vb);
            }
        }
    }
    if (grid > 0) {
        if (out.keys) launch_k(k_keys64, n_tiles, 256, 0, st, out.ranges, out.values, proj.depth, n, out.keys);
        TRY(cudaGetLastError());
    }
    return cudaSuccess;
#undef TRY
}

}  // namespace darb

#ifdef DARB_TEST_HOOKS
// Test-only entry point, compiled into a separate test build of the library (with a short
// DARB_SPIN_LIMIT) and declared nowhere else: one onesweep pass whose single CTA finds the
// partition counter preset to 1, so it sorts partition 1 while partition 0 is never processed.
// Its look-back therefore waits on statuses that nothing publishes, gives up after
// DARB_SPIN_LIMIT polls, sets DARB_ERR_TIMEOUT in the status word and finishes its pass (every
// store stays inside the 2-partition buffers).  ws: device, 16-byte aligned, at least
// darb_test_lookback_timeout_bytes(); *status_host receives the status word after the stream
// has been synchronised.
extern "C" size_t darb_test_lookback_timeout_bytes(void) {
    return (2 * (size_t)darb::kSortTile * 2 + 256 + 2 * 256 + 4) * sizeof(uint32_t);
}

extern "C" darb_status darb_test_lookback_timeout(void *ws, size_t ws_bytes, uint32_t *status_host,
                                                  darb_stream stream) {
    using namespace darb;
    const size_t need = darb_test_lookback_timeout_bytes();
    if (!ws || ws_bytes < need || !status_host || (reinterpret_cast<uintptr_t>(ws) & 15u)) return DARB_ERR_INVALID_ARG;
    const size_t n = 2 * (size_t)kSortTile;
    uint32_t *kin = static_cast<uint32_t *>(ws), *vout = kin + n, *digit_base = vout + n;
    uint32_t *lookback = digit_base + 256, *words = lookback + 2 * 256;  // words: counter, status
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    if (cudaMemsetAsync(ws, 0, need, st) != cudaSuccess) return DARB_ERR_CUDA;
    if (cudaMemsetAsync(words, 1, 1, st) != cudaSuccess) return DARB_ERR_CUDA;  // counter = 1 (little endian)
    const size_t smem = Staging<uint32_t, false>::bytes;
    if (cudaFuncSetAttribute(k_onesweep<uint32_t, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
        cudaSuccess)
        return DARB_ERR_CUDA;
    launch_k(k_onesweep<uint32_t, false>, 1, kSortThreads, smem, st, (const uint32_t *)kin, (const uint32_t *)nullptr,
             (uint32_t *)nullptr, vout, (const uint32_t *)nullptr, (unsigned long long)n, 0, 8,
             (const uint32_t *)digit_base, lookback, words, words + 1);
    if (cudaGetLastError() != cudaSuccess) return DARB_ERR_CUDA;
    if (cudaMemcpyAsync(status_host, words + 1, 4, cudaMemcpyDeviceToHost, st) != cudaSuccess) return DARB_ERR_CUDA;
    return cudaStreamSynchronize(st) == cudaSuccess ? DARB_OK : DARB_ERR_CUDA;
}
#endif
