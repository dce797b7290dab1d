// rt_common.cu -- error reporting, device allocation, radix sort and scan.
#include "rt_internal.cuh"

#include <atomic>
#include <mutex>

namespace rr {

// ---------------------------------------------------------------------------
// errors (thread-local message)
// ---------------------------------------------------------------------------
static thread_local std::string g_err;

void set_error(const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_err = buf;
}

void clear_error() { g_err.clear(); }

rt_status cuda_status(cudaError_t e, const char* what) {
    if (e == cudaSuccess) return RT_OK;
    set_error("%s failed: %s", what, cudaGetErrorString(e));
    if (e == cudaErrorMemoryAllocation) return RT_ERR_OOM;
    return RT_ERR_CUDA;
}

// ---------------------------------------------------------------------------
// allocation: cudaMallocAsync on the call's stream, or a user hook
// ---------------------------------------------------------------------------
static std::mutex g_alloc_mu;
static rt_alloc_fn g_alloc = nullptr;
static rt_free_fn g_free = nullptr;
static void* g_ctx = nullptr;

// The stream-ordered pool would hand memory back to the driver at every
// synchronisation; keeping it makes repeated traces allocation-free.
static void keep_pool_memory() {
    static std::mutex mu;
    static bool done[64] = {};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return;
    std::lock_guard<std::mutex> lk(mu);
    if (done[dev]) return;
    cudaMemPool_t pool;
    if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
        uint64_t keep = UINT64_MAX;
        cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
    }
    cudaGetLastError();
    done[dev] = true;
}

thread_local bool g_alloc_misaligned = false;

bool last_alloc_misaligned() { return g_alloc_misaligned; }

void* dev_alloc(size_t bytes, cudaStream_t s) {
    rt_alloc_fn a;
    rt_free_fn f;
    void* ctx;
    {
        std::lock_guard<std::mutex> lk(g_alloc_mu);
        a = g_alloc;
        f = g_free;
        ctx = g_ctx;
    }
    g_alloc_misaligned = false;
    if (a) {
        void* p = a(bytes, (void*)s, ctx);
        // the kernels use 16- and 32-byte vector accesses: a block that is not
        // 256-byte aligned goes back to its owner before any kernel sees it
        if (p && ((uintptr_t)p & 255u)) {
            if (f) f(p, (void*)s, ctx);
            g_alloc_misaligned = true;
            return nullptr;
        }
        return p;
    }
    keep_pool_memory();
    void* p = nullptr;
    if (cudaMallocAsync(&p, bytes, s) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return p;
}

void dev_free(void* p, cudaStream_t s) {
    if (!p) return;
    rt_free_fn f;
    void* ctx;
    {
        std::lock_guard<std::mutex> lk(g_alloc_mu);
        f = g_free;
        ctx = g_ctx;
    }
    if (f) {
        f(p, (void*)s, ctx);
        return;
    }
    cudaFreeAsync(p, s);
}

static std::atomic<long long> g_launches{0};
void note_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }
long long launch_count() { return g_launches.load(std::memory_order_relaxed); }

int device_sm_count() {
    int dev = 0, n = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    return n > 0 ? n : 1;
}

// ---------------------------------------------------------------------------
// exclusive scan of uint32 (three phases: tile sums, scan of sums, apply)
// ---------------------------------------------------------------------------
static constexpr int SCAN_THREADS = 512;
static constexpr int SCAN_ITEMS = 8;
static constexpr int SCAN_TILE = SCAN_THREADS * SCAN_ITEMS;

__device__ __forceinline__ uint32_t warp_incl_scan(uint32_t v) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t y = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += y;
    }
    return v;
}

// block-wide exclusive scan; every thread receives the block total in `total`
template <int THREADS>
__device__ uint32_t block_excl_scan(uint32_t v, uint32_t& total) {
    constexpr int W = THREADS / 32;
    static_assert(W <= 32, "block too large");
    __shared__ uint32_t warp_sums[W];
    __shared__ uint32_t s_total;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t incl = warp_incl_scan(v);
    if (lane == 31) warp_sums[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        uint32_t w = (lane < W) ? warp_sums[lane] : 0u;
        uint32_t wi = warp_incl_scan(w);
        if (lane < W) warp_sums[lane] = wi - w;
        if (lane == 31) s_total = wi;
    }
    __syncthreads();
    uint32_t r = warp_sums[warp] + incl - v;
    total = s_total;
    __syncthreads();
    return r;
}

__global__ void k_scan_tiles(const uint32_t* __restrict__ in, int64_t n, uint32_t* __restrict__ tile_sums) {
    uint32_t tot;
    int64_t base = (int64_t)blockIdx.x * SCAN_TILE + (int64_t)threadIdx.x * SCAN_ITEMS;
    uint32_t s = 0;
#pragma unroll
    for (int k = 0; k < SCAN_ITEMS; k++) {
        int64_t i = base + k;
        if (i < n) s += in[i];
    }
    block_excl_scan<SCAN_THREADS>(s, tot);
    if (threadIdx.x == 0) tile_sums[blockIdx.x] = tot;
}

// scan of the tile sums by one block (sequential chunks per thread)
__global__ void k_scan_sums(uint32_t* sums, int64_t m, uint32_t* total_dev) {
    uint32_t tot;
    int64_t per = (m + SCAN_THREADS - 1) / SCAN_THREADS;
    int64_t b = (int64_t)threadIdx.x * per, e = b + per < m ? b + per : m;
    uint32_t s = 0;
    for (int64_t i = b; i < e; i++) s += sums[i];
    uint32_t off = block_excl_scan<SCAN_THREADS>(s, tot);
    for (int64_t i = b; i < e; i++) {
        uint32_t x = sums[i];
        sums[i] = off;
        off += x;
    }
    if (threadIdx.x == 0 && total_dev) *total_dev = tot;
}

__global__ void k_scan_apply(const uint32_t* __restrict__ in, uint32_t* __restrict__ out, int64_t n,
                             const uint32_t* __restrict__ tile_off) {
    uint32_t tot;
    int64_t base = (int64_t)blockIdx.x * SCAN_TILE + (int64_t)threadIdx.x * SCAN_ITEMS;
    uint32_t v[SCAN_ITEMS];
    uint32_t s = 0;
#pragma unroll
    for (int k = 0; k < SCAN_ITEMS; k++) {
        int64_t i = base + k;
        v[k] = (i < n) ? in[i] : 0u;
        s += v[k];
    }
    uint32_t off = block_excl_scan<SCAN_THREADS>(s, tot) + tile_off[blockIdx.x];
#pragma unroll
    for (int k = 0; k < SCAN_ITEMS; k++) {
        int64_t i = base + k;
        if (i < n) out[i] = off;
        off += v[k];
    }
}

size_t scan_temp_bytes(int64_t n) {
    int64_t tiles = (n + SCAN_TILE - 1) / SCAN_TILE;
    return (size_t)(tiles + 1) * sizeof(uint32_t);
}

rt_status exclusive_scan_u32(const uint32_t* in, uint32_t* out, int64_t n, uint32_t* total_dev, void* temp,
                             cudaStream_t s) {
    if (n <= 0) {
        if (total_dev) RR_CUDA(cudaMemsetAsync(total_dev, 0, sizeof(uint32_t), s));
        return RT_OK;
    }
    int64_t tiles = (n + SCAN_TILE - 1) / SCAN_TILE;
    uint32_t* sums = (uint32_t*)temp;
    RR_LAUNCH(k_scan_tiles, (unsigned)tiles, SCAN_THREADS, 0, s, in, n, sums);
    RR_LAUNCH(k_scan_sums, 1, SCAN_THREADS, 0, s, sums, tiles, total_dev);
    RR_LAUNCH(k_scan_apply, (unsigned)tiles, SCAN_THREADS, 0, s, in, out, n, sums);
    RR_CUDA(cudaGetLastError());
    return RT_OK;
}

// ---------------------------------------------------------------------------
// stable LSD radix sort, 8-bit digits, one scatter launch per pass
//   * one launch counts the digits of every pass at once (global histograms);
//   * per pass, one scatter launch: blocks take tile indices in launch order
//     from an atomic counter and publish their tile's digit counts.  Each
//     digit's offset is the sum of the earlier tiles' counts:
//       - up to DIRECT_MAX_TILES tiles, every tile also sets a ready flag; a
//         block waits for the earlier tiles' flags (one per thread) and sums
//         their counts with independent loads;
//       - beyond, by decoupled look-back (Merrill & Garland 2016; the
//         single-pass radix sort of Adinets & Merrill 2022): walk back over
//         the earlier tiles adding their counts until one that already
//         published its inclusive prefix.
//     Keys are ranked inside the tile with __match_any_sync per warp,
//     keeping the input order among equal digits, so every pass is stable.
// A tile index goes only to a block that is running, and every block
// publishes its counts before it waits, so each wait ends; the wait is
// bounded all the same: past the limit the block counts that tile's digit
// itself from the keys, which gives the same number.
// Look-back words (64-bit): bits 63-62 state (1 counts of the tile, 2
// inclusive prefix), bits 61-58 the pass, bits 57-0 the count.  Ready flags
// hold the pass + 1, so a flag left by the previous pass is not taken.
// ---------------------------------------------------------------------------
static constexpr int SORT_THREADS = 256;
static constexpr int SORT_WARPS = SORT_THREADS / 32;
// keys per thread: 15 (3840-key tiles) for large sorts, 8 (2048-key tiles)
// up to SORT_SMALL keys, where shorter per-tile chains pay more than fewer tiles
static constexpr int SORT_ITEMS_LARGE = 15, SORT_ITEMS_SMALL = 8;
static constexpr int64_t SORT_SMALL = 262144;
static int64_t sort_tile(int64_t n) { return SORT_THREADS * (int64_t)(n <= SORT_SMALL ? SORT_ITEMS_SMALL : SORT_ITEMS_LARGE); }
static constexpr int RADIX = 256;
static constexpr int SORT_MAX_PASSES = 8;
static constexpr uint64_t LB_AGG = 1ull << 62, LB_INC = 2ull << 62, LB_COUNT = (1ull << 58) - 1;
static constexpr int LB_SPIN = 1 << 14;
static constexpr int LB_WINDOW = 8;
static constexpr int DIRECT_MAX_TILES = 256;  // up to this many tiles the prefix is summed directly

__global__ void __launch_bounds__(SORT_THREADS) k_sort_hist(const uint64_t* __restrict__ keys, int64_t n,
                                                            int begin_bit, int passes,
                                                            uint32_t* __restrict__ counts) {
    __shared__ uint32_t h[SORT_MAX_PASSES * RADIX];
    for (int i = threadIdx.x; i < SORT_MAX_PASSES * RADIX; i += SORT_THREADS) h[i] = 0;
    __syncthreads();
    for (int64_t i = (int64_t)blockIdx.x * SORT_THREADS + threadIdx.x; i < n; i += (int64_t)gridDim.x * SORT_THREADS) {
        const uint64_t k = keys[i];
        for (int p = 0; p < passes; p++) atomicAdd(&h[p * RADIX + ((uint32_t)(k >> (begin_bit + 8 * p)) & 0xFFu)], 1u);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < passes * RADIX; i += SORT_THREADS)
        if (h[i]) atomicAdd(&counts[i], h[i]);
}

__device__ __forceinline__ uint64_t ld_volatile_u64(const uint64_t* p) {
    uint64_t v;
    asm volatile("ld.volatile.global.u64 %0, [%1];\n" : "=l"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ uint32_t ld_volatile_u32(const uint32_t* p) {
    uint32_t v;
    asm volatile("ld.volatile.global.u32 %0, [%1];\n" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void st_volatile_u64(uint64_t* p, uint64_t v) {
    asm volatile("st.volatile.global.u64 [%0], %1;\n" ::"l"(p), "l"(v) : "memory");
}

// digit d's count in tile j, recounted from the keys (the bounded wait's fallback)
__device__ uint64_t tile_digit_count(const uint64_t* __restrict__ kin, int64_t n, int64_t j, int64_t tile_keys,
                                     int shift, uint32_t d) {
    uint64_t c = 0;
    const int64_t lo = j * tile_keys, hi = lo + tile_keys < n ? lo + tile_keys : n;
    for (int64_t i = lo; i < hi; i++) c += ((uint32_t)(kin[i] >> shift) & 0xFFu) == d;
    return c;
}

template <int SORT_ITEMS>
__global__ void __launch_bounds__(SORT_THREADS) k_sort_scatter(const uint64_t* __restrict__ kin,
                                                               const uint32_t* __restrict__ vin,
                                                               uint64_t* __restrict__ kout,
                                                               uint32_t* __restrict__ vout, int64_t n, int shift,
                                                               int pass, const uint32_t* __restrict__ counts,
                                                               uint64_t* __restrict__ look,
                                                               uint32_t* __restrict__ rows,
                                                               uint32_t* __restrict__ ready,
                                                               uint32_t* __restrict__ tile_ctr, int64_t tiles) {
    __shared__ uint32_t whist[SORT_WARPS][RADIX];
    __shared__ uint64_t boff[RADIX];
    __shared__ uint32_t wsum[SORT_WARPS];
    __shared__ uint32_t s_tile;
    __shared__ uint32_t late[DIRECT_MAX_TILES / 32];  // tiles whose counts did not appear in time
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int i = threadIdx.x; i < SORT_WARPS * RADIX; i += SORT_THREADS) (&whist[0][0])[i] = 0;
    if (threadIdx.x == 0) s_tile = atomicAdd(tile_ctr, 1u);
    // exclusive prefix of the global digit counts (thread d: digit d)
    const uint32_t d = threadIdx.x;
    const uint32_t gc = counts[d];
    uint32_t incl = gc;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
    }
    if (lane == 31) wsum[warp] = incl;
    __syncthreads();
    uint32_t gbase = incl - gc;
    for (int w = 0; w < warp; w++) gbase += wsum[w];
    const int64_t tile = s_tile;
    constexpr int64_t SORT_TILE = SORT_THREADS * SORT_ITEMS;
    const int64_t wbase = tile * SORT_TILE + (int64_t)warp * 32 * SORT_ITEMS;
    uint64_t k[SORT_ITEMS];
    uint32_t v[SORT_ITEMS], rank[SORT_ITEMS], dig[SORT_ITEMS];
    // all loads first: the warp synchronisations of the ranking below would
    // otherwise keep each load behind the previous item's ranking
#pragma unroll
    for (int it = 0; it < SORT_ITEMS; it++) {
        const int64_t idx = wbase + it * 32 + lane;
        k[it] = idx < n ? kin[idx] : 0ull;
        v[it] = idx < n ? vin[idx] : 0u;
    }
#pragma unroll
    for (int it = 0; it < SORT_ITEMS; it++) {
        const bool valid = wbase + it * 32 + lane < n;
        const uint32_t dd = valid ? ((uint32_t)(k[it] >> shift) & 0xFFu) : 0xFFFFFFFFu;
        dig[it] = dd;
        const uint32_t peers = __match_any_sync(0xffffffffu, dd);
        const uint32_t below = peers & ((1u << lane) - 1u);
        uint32_t r = 0;
        if (valid) r = whist[warp][dd] + __popc(below);
        rank[it] = r;
        __syncwarp();
        if (valid && below == 0) whist[warp][dd] += __popc(peers);
        __syncwarp();
    }
    __syncthreads();
    // this tile's count of digit d; offsets of the warps inside the tile
    uint32_t cnt = 0;
#pragma unroll
    for (int w = 0; w < SORT_WARPS; w++) {
        const uint32_t c = whist[w][d];
        whist[w][d] = cnt;
        cnt += c;
    }
    uint64_t excl = 0;
    if (tiles <= DIRECT_MAX_TILES) {
        // few tiles: publish this tile's counts and a ready flag, wait for the
        // earlier tiles' flags (one per thread, in parallel), then sum their
        // counts with independent loads
        if (d < DIRECT_MAX_TILES / 32) late[d] = 0;
        __stcg(rows + tile * RADIX + d, cnt);
        __syncthreads();
        if (threadIdx.x == 0) {
            __threadfence();
            atomicExch(ready + tile, (uint32_t)pass + 1u);
        }
        for (int64_t i = threadIdx.x; i < tile; i += SORT_THREADS) {
            bool ok = false;
            for (int spin = 0; spin < LB_SPIN && !ok; spin++)
                ok = ld_volatile_u32(ready + i) == (uint32_t)pass + 1u;
            if (!ok) atomicOr(&late[i >> 5], 1u << (i & 31));
        }
        __threadfence();
        __syncthreads();
        uint32_t part[4] = {0u, 0u, 0u, 0u};
        int64_t i = 0;
        for (; i + 4 <= tile; i += 4) {
#pragma unroll
            for (int q = 0; q < 4; q++) {
                const uint32_t c = __ldcg(rows + (i + q) * RADIX + d);
                part[q] += (late[(i + q) >> 5] >> ((i + q) & 31)) & 1u ? 0u : c;
            }
        }
        for (; i < tile; i++) {
            const uint32_t c = __ldcg(rows + i * RADIX + d);
            part[0] += (late[i >> 5] >> (i & 31)) & 1u ? 0u : c;
        }
        excl = (uint64_t)part[0] + part[1] + part[2] + part[3];
        for (int64_t w = 0; w * 32 < tile; w++) {
            uint32_t bits = late[w];
            while (bits) {  // counts that were not published in time: recount them
                const int b = __ffs(bits) - 1;
                bits &= bits - 1;
                const int64_t j = w * 32 + b;
                if (j < tile) excl += tile_digit_count(kin, n, j, SORT_TILE, shift, d);
            }
        }
    } else {
        const uint64_t tag = (uint64_t)pass << 58;
        uint64_t* mine = look + tile * RADIX + d;
        st_volatile_u64(mine, (tile == 0 ? LB_INC : LB_AGG) | tag | cnt);
        // look back LB_WINDOW tiles at a time (independent loads), nearest first
        bool found = false;
        for (int64_t j0 = tile - 1; j0 >= 0 && !found; j0 -= LB_WINDOW) {
            uint64_t win[LB_WINDOW];
#pragma unroll
            for (int q = 0; q < LB_WINDOW; q++) win[q] = j0 - q >= 0 ? ld_volatile_u64(look + (j0 - q) * RADIX + d) : 0ull;
#pragma unroll
            for (int q = 0; q < LB_WINDOW; q++) {
                const int64_t j = j0 - q;
                if (found || j < 0) break;
                uint64_t x = win[q];
                bool ok = (x >> 62) != 0 && ((x >> 58) & 15u) == (uint64_t)pass;
                for (int spin = 0; !ok && spin < LB_SPIN; spin++) {
                    x = ld_volatile_u64(look + j * RADIX + d);
                    ok = (x >> 62) != 0 && ((x >> 58) & 15u) == (uint64_t)pass;
                }
                if (!ok) {  // not published in time: count it here
                    excl += tile_digit_count(kin, n, j, SORT_TILE, shift, d);
                    continue;
                }
                excl += x & LB_COUNT;
                found = (x >> 62) == 2;
            }
        }
        if (tile != 0) st_volatile_u64(mine, LB_INC | tag | (excl + cnt));
    }
    boff[d] = (uint64_t)gbase + excl;
    __syncthreads();
#pragma unroll
    for (int it = 0; it < SORT_ITEMS; it++) {
        const uint32_t dd = dig[it];
        if (dd != 0xFFFFFFFFu) {
            const uint64_t pos = boff[dd] + whist[warp][dd] + rank[it];
            if (pos < (uint64_t)n) {  // always, for consistent counts
                kout[pos] = k[it];
                vout[pos] = v[it];
            }
        }
    }
}

// scratch: global digit counts of every pass, the passes' tile counters and
// one look-back word per (tile, digit), reused by the passes (tagged)
static size_t sort_counts_bytes() { return sizeof(uint32_t) * SORT_MAX_PASSES * RADIX + 256; }

// For up to DIRECT_MAX_TILES tiles the 32-bit counts and ready flags serve;
// beyond that the 64-bit look-back words.
static size_t sort_lookback_bytes(int64_t tiles) {
    tiles = std::max<int64_t>(tiles, 1);
    if (tiles <= DIRECT_MAX_TILES)
        return sizeof(uint32_t) * RADIX * (size_t)tiles + ((sizeof(uint32_t) * (size_t)tiles + 255) & ~(size_t)255);
    return sizeof(uint64_t) * RADIX * (size_t)tiles;
}

size_t sort_temp_bytes(int64_t n) {
    const int64_t tiles = (n + sort_tile(n) - 1) / sort_tile(n);
    return sort_counts_bytes() + sort_lookback_bytes(tiles) + 256;
}

rt_status radix_sort_pairs(uint64_t* keys, uint32_t* vals, uint64_t* keys_alt, uint32_t* vals_alt, int64_t n,
                           int begin_bit, int end_bit, void* temp, cudaStream_t s) {
    if (n <= 1 || end_bit <= begin_bit) return RT_OK;
    if (n > (int64_t)0xFFFFFFFF) {
        set_error("radix sort of %lld keys exceeds 32-bit positions", (long long)n);
        return RT_ERR_INVALID_ARG;
    }
    const int passes = (end_bit - begin_bit + 7) / 8;
    if (passes > SORT_MAX_PASSES || begin_bit < 0 || begin_bit + 8 * passes > 64) {
        set_error("radix sort: bit range [%d, %d) not supported", begin_bit, end_bit);
        return RT_ERR_INVALID_ARG;
    }
    const int64_t tiles = (n + sort_tile(n) - 1) / sort_tile(n);
    uint32_t* counts = (uint32_t*)temp;                                // [passes][256]
    uint32_t* tile_ctr = counts + SORT_MAX_PASSES * RADIX;              // [passes]
    char* lb = (char*)temp + sort_counts_bytes();
    uint64_t* look = (uint64_t*)lb;                                     // [tiles][256], many tiles
    uint32_t* ready = (uint32_t*)lb;                                    // [tiles], few tiles
    uint32_t* rows = (uint32_t*)(lb + ((sizeof(uint32_t) * (size_t)tiles + 255) & ~(size_t)255));  // [tiles][256]
    RR_CUDA(cudaMemsetAsync(temp, 0, sort_temp_bytes(n), s));
    const int hist_grid = (int)std::min<int64_t>((n + SORT_THREADS - 1) / SORT_THREADS, 2 * (int64_t)device_sm_count());
    RR_LAUNCH(k_sort_hist, hist_grid, SORT_THREADS, 0, s, keys, n, begin_bit, passes, counts);
    uint64_t *ki = keys, *ko = keys_alt;
    uint32_t *vi = vals, *vo = vals_alt;
    for (int p = 0; p < passes; p++) {
        if (n <= SORT_SMALL)
            RR_LAUNCH(k_sort_scatter<SORT_ITEMS_SMALL>, (unsigned)tiles, SORT_THREADS, 0, s, ki, vi, ko, vo, n,
                      begin_bit + 8 * p, p, counts + p * RADIX, look, rows, ready, tile_ctr + p, tiles);
        else
            RR_LAUNCH(k_sort_scatter<SORT_ITEMS_LARGE>, (unsigned)tiles, SORT_THREADS, 0, s, ki, vi, ko, vo, n,
                      begin_bit + 8 * p, p, counts + p * RADIX, look, rows, ready, tile_ctr + p, tiles);
        RR_CUDA(cudaGetLastError());
        std::swap(ki, ko);
        std::swap(vi, vo);
    }
    if (passes & 1) {
        RR_CUDA(cudaMemcpyAsync(keys, ki, sizeof(uint64_t) * n, cudaMemcpyDeviceToDevice, s));
        RR_CUDA(cudaMemcpyAsync(vals, vi, sizeof(uint32_t) * n, cudaMemcpyDeviceToDevice, s));
    }
    return RT_OK;
}

// ---------------------------------------------------------------------------
// L2 read bandwidth probe (roofline denominator): every block streams an
// L2-resident buffer with 128-bit loads that bypass L1 (ld.global.cg)
// ---------------------------------------------------------------------------
__global__ void k_l2_read(const float4* __restrict__ buf, int64_t n4, int reps, float* __restrict__ sink) {
    float a = 0.f, b = 0.f, c = 0.f, d = 0.f;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int r = 0; r < reps; r++) {
        for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n4; i += stride) {
            float4 v = __ldcg(buf + i);
            a += v.x;
            b += v.y;
            c += v.z;
            d += v.w;
        }
    }
    if (a + b + c + d == -1.0f) sink[0] = a;  // never true for the zero-filled buffer; keeps the loads
}

static rt_status measure_l2_impl(double* gbs, cudaStream_t s) {
    if (!gbs) {
        set_error("rt_measure_l2_bandwidth: null output");
        return RT_ERR_INVALID_ARG;
    }
    const int64_t bytes = 32ll << 20;  // 32 MiB: well inside the L2
    const int64_t n4 = bytes / 16;
    const int reps = 64;  // 2 GiB of L2 reads per launch, about 0.15 ms
    Arena ar(s);
    float4* buf;
    float* sink;
    RR_TRY(ar.alloc(&buf, n4));
    RR_TRY(ar.alloc(&sink, 1));
    RR_CUDA(cudaMemsetAsync(buf, 0, bytes, s));
    const int grid = device_sm_count() * 4;
    cudaEvent_t e0, e1;
    RR_CUDA(cudaEventCreate(&e0));
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        RR_CUDA(cudaGetLastError());
    }
    // keep the L2 busy for at least 200 ms first, so that a cold GPU has
    // raised its clocks, then keep the best of 10 launches
    float warm = 0.f, best = 1e30f;
    for (int k = 0; k < 4000 && warm < 200.f; k++) {
        cudaEventRecord(e0, s);
        RR_LAUNCH(k_l2_read, grid, 512, 0, s, buf, n4, reps, sink);
        cudaEventRecord(e1, s);
        cudaEventSynchronize(e1);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        warm += ms;
    }
    for (int k = 0; k < 10; k++) {
        cudaEventRecord(e0, s);
        RR_LAUNCH(k_l2_read, grid, 512, 0, s, buf, n4, reps, sink);
        cudaEventRecord(e1, s);
        cudaEventSynchronize(e1);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (ms > 0.f && ms < best) best = ms;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    RR_CUDA(cudaGetLastError());
    *gbs = (double)bytes * reps / (best * 1e-3) / 1e9;
    return RT_OK;
}

}  // namespace rr

// ---------------------------------------------------------------------------
// C ABI: misc
// ---------------------------------------------------------------------------
extern "C" const char* rt_last_error(void) { return rr::g_err.c_str(); }

extern "C" int32_t rt_api_version(void) { return RT_API_VERSION; }

extern "C" int64_t rt_launch_count(void) { return rr::launch_count(); }

extern "C" rt_status rt_measure_l2_bandwidth(double* read_gbs, void* stream) {
    rr::clear_error();
    return rr::measure_l2_impl(read_gbs, (cudaStream_t)stream);
}

extern "C" rt_status rt_set_allocator(rt_alloc_fn alloc, rt_free_fn free_fn, void* ctx) {
    if ((alloc == nullptr) != (free_fn == nullptr)) {
        rr::set_error("rt_set_allocator: give both functions or neither");
        return RT_ERR_INVALID_ARG;
    }
    std::lock_guard<std::mutex> lk(rr::g_alloc_mu);
    rr::g_alloc = alloc;
    rr::g_free = free_fn;
    rr::g_ctx = ctx;
    return RT_OK;
}
