// rt_noalloc.cu -- rt_rir_static: the histogram step without device allocation.
//
// Some callers cannot allocate device memory while they run: a real-time
// auralisation loop that re-bins image sources for a moving listener on an
// audio deadline (a device allocation can block on the driver and on other
// streams), or a host application that reserves all of its GPU memory up
// front and forbids allocation afterwards.  rt_rir_static bins image sources
// exactly like rt_rir, but its sort scratch is a file-scope __device__ array
// of fixed size, so the call makes no cudaMalloc / cudaFree / cudaMallocAsync
// and calls no allocating library routine.  The caller passes the inputs and
// the zero-filled-by-this-call output buffer.
//
// Costs and rules of the static scratch:
//   - every GPU that loads the library holds RT_RIR_STATIC_SCRATCH_BYTES
//     (about 12.3 MB) for the life of the process;
//   - all calls share it and it keeps the last call's contents: two calls
//     whose GPU work overlaps (different streams, or different host threads
//     on one device) race and corrupt each other's result; serialise them;
//   - nothing in it needs to start at zero: every launch writes what it
//     later reads;
//   - the first call on a device looks up the array's device address
//     (cudaGetSymbolAddress) once for that device.  With lazy module loading
//     (the default) that lookup is what loads this library's device code on
//     the device, so the first call may make the driver allocate and may
//     block: real-time callers make one warm-up call (n = 0 is enough)
//     before their deadline loop, and before capturing the stream into a
//     CUDA graph;
//   - the address is cached for the life of the process; cudaDeviceReset
//     (or a release of the primary context) unloads the module, after which
//     the cached address is stale and later calls are invalid.
#include "rt_internal.cuh"

#include <mutex>

namespace rr {

// the kernels of rt_rir.cu that this step reuses unchanged
__global__ void k_bin_sum(const uint64_t* __restrict__ keys, const uint32_t* __restrict__ vals, int64_t n,
                          const double* __restrict__ energy, uint64_t sentinel, int64_t n_bins,
                          float* __restrict__ H);

static constexpr int64_t STATIC_MAX = RT_RIR_STATIC_MAX_SOURCES;
static constexpr size_t SORT_TILE_KEYS = 2048;  // sizing unit of the radix-sort scratch below
static constexpr size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }
static constexpr size_t OFF_KEYS = 0;
static constexpr size_t OFF_KEYS_ALT = OFF_KEYS + align256(sizeof(uint64_t) * STATIC_MAX);
static constexpr size_t OFF_VALS = OFF_KEYS_ALT + align256(sizeof(uint64_t) * STATIC_MAX);
static constexpr size_t OFF_VALS_ALT = OFF_VALS + align256(sizeof(uint32_t) * STATIC_MAX);
static constexpr size_t OFF_SORT = OFF_VALS_ALT + align256(sizeof(uint32_t) * STATIC_MAX);
// radix-sort scratch: 1 KB per 2048 keys plus 64 KB, above what the sort asks
// for (8 KB of digit counts and 2 KB of look-back words per 3840-key tile;
// checked against sort_temp_bytes at run time)
static constexpr size_t SORT_BYTES =
    align256(sizeof(uint32_t) * 256 * ((STATIC_MAX + SORT_TILE_KEYS - 1) / SORT_TILE_KEYS)) + 65536;
static constexpr size_t SCRATCH_BYTES = OFF_SORT + SORT_BYTES;
static_assert(SCRATCH_BYTES == RT_RIR_STATIC_SCRATCH_BYTES, "header constant out of date");

static __device__ __align__(256) unsigned char g_rir_scratch[SCRATCH_BYTES];

// device address of g_rir_scratch, looked up once per device
static std::mutex g_mu;
static void* g_addr[64] = {};

static rt_status scratch_address(void** out) {
    int dev = 0;
    RR_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) {
        set_error("rt_rir_static: device index %d out of range", dev);
        return RT_ERR_INVALID_ARG;
    }
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_addr[dev]) {
        void* p = nullptr;
        RR_CUDA(cudaGetSymbolAddress(&p, g_rir_scratch));
        g_addr[dev] = p;
    }
    *out = g_addr[dev];
    return RT_OK;
}

// keys (receiver, bin) of valid sources; anything out of range -> sentinel
__global__ void k_bin_keys_checked(const double* __restrict__ t, const int32_t* __restrict__ rcv, int64_t n,
                                   int32_t n_rcv, double fs, int64_t n_bins, uint64_t* __restrict__ keys,
                                   uint32_t* __restrict__ vals, uint64_t sentinel) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double x = floor(t[i] * fs);
    int32_t r = rcv[i];
    uint64_t key = sentinel;
    if (x >= 0.0 && x < (double)n_bins && r >= 0 && r < n_rcv) key = (uint64_t)r * (uint64_t)n_bins + (uint64_t)x;
    keys[i] = key;
    vals[i] = (uint32_t)i;
}

static rt_status rir_static_impl(const double* time, const int32_t* rcv, const double* energy, int64_t n,
                                 int32_t n_rcv, double fs, int64_t n_bins, float* hist, cudaStream_t s) {
    if (n < 0 || n_rcv < 1 || !(fs > 0) || n_bins < 1 || !hist || (n > 0 && (!time || !rcv || !energy))) {
        set_error("rt_rir_static: need n >= 0, n_rcv >= 1, fs > 0, n_bins >= 1 and non-null arrays");
        return RT_ERR_INVALID_ARG;
    }
    if (n > STATIC_MAX) {
        set_error("rt_rir_static: %lld image sources exceed the static scratch limit of %lld "
                  "(use rt_rir, which allocates)", (long long)n, (long long)STATIC_MAX);
        return RT_ERR_INVALID_ARG;
    }
    if ((int64_t)n_rcv * RT_N_BANDS * n_bins > ((int64_t)1 << 36) || n_bins > ((int64_t)1 << 40)) {
        set_error("rt_rir_static: %lld bins too many", (long long)n_bins);
        return RT_ERR_INVALID_ARG;
    }
    void* base = nullptr;
    RR_TRY(scratch_address(&base));
    unsigned char* b = (unsigned char*)base;
    uint64_t* keys = (uint64_t*)(b + OFF_KEYS);
    uint64_t* keys_alt = (uint64_t*)(b + OFF_KEYS_ALT);
    uint32_t* vals = (uint32_t*)(b + OFF_VALS);
    uint32_t* vals_alt = (uint32_t*)(b + OFF_VALS_ALT);
    void* sort_tmp = b + OFF_SORT;
    if (sort_temp_bytes(n) > SORT_BYTES) {
        set_error("rt_rir_static: internal scratch layout too small");
        return RT_ERR_INTERNAL;
    }
    RR_CUDA(cudaMemsetAsync(hist, 0, sizeof(float) * (size_t)n_rcv * RT_N_BANDS * (size_t)n_bins, s));
    if (n == 0) return RT_OK;
    const uint64_t sentinel = (uint64_t)n_rcv * (uint64_t)n_bins;
    int bits = 1;
    while (bits < 64 && (sentinel >> bits) != 0) bits++;
    const unsigned grid = (unsigned)((n + 255) / 256);
    RR_LAUNCH(k_bin_keys_checked, grid, 256, 0, s, time, rcv, n, n_rcv, fs, n_bins, keys, vals, sentinel);
    RR_CUDA(cudaGetLastError());
    RR_TRY(radix_sort_pairs(keys, vals, keys_alt, vals_alt, n, 0, ((bits + 7) / 8) * 8, sort_tmp, s));
    RR_LAUNCH(k_bin_sum, grid, 256, 0, s, keys, vals, n, energy, sentinel, n_bins, hist);
    RR_CUDA(cudaGetLastError());
    return RT_OK;
}

}  // namespace rr

extern "C" rt_status rt_rir_static(const double* time, const int32_t* rcv, const double* energy, int64_t n,
                                   int32_t n_rcv, double fs, int64_t n_bins, float* hist, void* stream) {
    rr::NvtxRange nvtx_range("rt_rir_static");
    rr::clear_error();
    return rr::rir_static_impl(time, rcv, energy, n, n_rcv, fs, n_bins, hist, (cudaStream_t)stream);
}
