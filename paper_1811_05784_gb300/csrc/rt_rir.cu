// rt_rir.cu -- rt_rir: 8-band energy impulse responses from image sources.
//
// Each image source arrives at t_s = d_s / c and carries E_s(f) (paper
// Sec. 1.4, eq. 19); the response of receiver k in band f is the histogram
// H[k][f][floor(t_s fs)] += E_s(f).  To make the sums independent of thread
// timing, image sources are radix-sorted by (receiver, bin) and every bin is
// summed in FP64 by one thread in that fixed order; the result is stored as
// float32.
#include "rt_internal.cuh"

#include <algorithm>
#include <cmath>

namespace rr {

// latest arrival: block maximum first, one atomic per block (times are >= 0,
// so their bit patterns order like the values)
__global__ void k_max_time(const double* __restrict__ t, int64_t n, unsigned long long* out) {
    __shared__ unsigned long long wmax[8];
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    unsigned long long v = i < n ? (unsigned long long)__double_as_longlong(fmax(t[i], 0.0)) : 0ull;
    for (int o = 16; o > 0; o >>= 1) {
        unsigned long long y = __shfl_down_sync(0xffffffffu, v, o);
        v = y > v ? y : v;
    }
    if ((threadIdx.x & 31) == 0) wmax[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < (int)(blockDim.x >> 5); w++) v = wmax[w] > v ? wmax[w] : v;
        atomicMax(out, v);
    }
}

__global__ void k_bin_keys(const double* __restrict__ t, const int32_t* __restrict__ rcv, int64_t n, double fs,
                           int64_t n_bins, uint64_t* __restrict__ keys, uint32_t* __restrict__ vals,
                           uint64_t sentinel) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double x = floor(t[i] * fs);
    uint64_t key = sentinel;
    if (x >= 0.0 && x < (double)n_bins) key = (uint64_t)rcv[i] * (uint64_t)n_bins + (uint64_t)x;
    keys[i] = key;
    vals[i] = (uint32_t)i;
}

// one thread per run of equal keys (started at a head), FP64 sums in order
__global__ void k_bin_sum(const uint64_t* __restrict__ keys, const uint32_t* __restrict__ vals, int64_t n,
                          const double* __restrict__ energy, uint64_t sentinel, int64_t n_bins,
                          float* __restrict__ H) {
    int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    uint64_t k = keys[j];
    if (k == sentinel || (j > 0 && keys[j - 1] == k)) return;
    double acc[RT_N_BANDS];
#pragma unroll
    for (int f = 0; f < RT_N_BANDS; f++) acc[f] = 0.0;
    for (int64_t e = j; e < n && keys[e] == k; e++) {
        const double* E = energy + 8 * (int64_t)vals[e];
#pragma unroll
        for (int f = 0; f < RT_N_BANDS; f++) acc[f] += E[f];
    }
    int64_t rcv = (int64_t)(k / (uint64_t)n_bins), bin = (int64_t)(k % (uint64_t)n_bins);
#pragma unroll
    for (int f = 0; f < RT_N_BANDS; f++) H[(rcv * RT_N_BANDS + f) * n_bins + bin] = (float)acc[f];
}

static unsigned grid_of(int64_t n, int threads) { return (unsigned)((n + threads - 1) / threads); }

static rt_status rir_impl(const rt_image_sources* is, double fs, double duration, cudaStream_t s, rt_response** out) {
    if (!is || !out || !(fs > 0)) {
        set_error("rt_rir: need an image-source handle, fs > 0 and an output pointer");
        return RT_ERR_INVALID_ARG;
    }
    *out = nullptr;
    const int64_t n = is->v.n;
    const int R = is->n_rcv;
    Arena tmp(s), keep(s);
    int64_t n_bins = 1;
    if (duration > 0) {
        n_bins = (int64_t)std::ceil(duration * fs);
    } else if (n > 0) {
        unsigned long long* d_max;
        RR_TRY(tmp.alloc(&d_max, 1));
        RR_CUDA(cudaMemsetAsync(d_max, 0, sizeof(unsigned long long), s));
        RR_LAUNCH(k_max_time, grid_of(n, 256), 256, 0, s, is->v.time, n, d_max);
        RR_CUDA(cudaGetLastError());
        unsigned long long bits = 0;
        RR_CUDA(cudaMemcpyAsync(&bits, d_max, sizeof bits, cudaMemcpyDeviceToHost, s));
        RR_CUDA(cudaStreamSynchronize(s));
        double tmax;
        memcpy(&tmax, &bits, sizeof tmax);
        n_bins = (int64_t)std::floor(tmax * fs) + 1;
    }
    if (n_bins < 1) n_bins = 1;
    const int64_t total = (int64_t)std::max(R, 1) * RT_N_BANDS * n_bins;
    if (n_bins > ((int64_t)1 << 40) || total > ((int64_t)1 << 36)) {
        set_error("rt_rir: %lld bins too many", (long long)n_bins);
        return RT_ERR_INVALID_ARG;
    }
    float* H;
    RR_TRY(keep.alloc(&H, total));
    RR_CUDA(cudaMemsetAsync(H, 0, sizeof(float) * total, s));
    if (n > 0 && R > 0) {
        const uint64_t sentinel = (uint64_t)R * (uint64_t)n_bins;
        int bits = 1;
        while (bits < 64 && (sentinel >> bits) != 0) bits++;
        uint64_t *keys, *keys_alt;
        uint32_t *vals, *vals_alt;
        void* sort_tmp;
        RR_TRY(tmp.alloc(&keys, n));
        RR_TRY(tmp.alloc(&keys_alt, n));
        RR_TRY(tmp.alloc(&vals, n));
        RR_TRY(tmp.alloc(&vals_alt, n));
        RR_TRY(tmp.alloc((char**)&sort_tmp, sort_temp_bytes(n)));
        RR_LAUNCH(k_bin_keys, grid_of(n, 256), 256, 0, s, is->v.time, is->v.rcv, n, fs, n_bins, keys, vals, sentinel);
        RR_CUDA(cudaGetLastError());
        RR_TRY(radix_sort_pairs(keys, vals, keys_alt, vals_alt, n, 0, ((bits + 7) / 8) * 8, sort_tmp, s));
        RR_LAUNCH(k_bin_sum, grid_of(n, 256), 256, 0, s, keys, vals, n, is->v.energy, sentinel, n_bins, H);
        RR_CUDA(cudaGetLastError());
    }
    rt_response* r = new rt_response();
    r->stream = s;
    r->v.n_rcv = R;
    r->v.n_bins = n_bins;
    r->v.fs = fs;
    r->v.data = H;
    r->owned = keep.release();
    *out = r;
    return RT_OK;
}

}  // namespace rr

extern "C" rt_status rt_rir(const rt_image_sources* is, double fs, double duration, void* stream,
                            rt_response** out) {
    rr::NvtxRange nvtx_range("rt_rir");
    rr::clear_error();
    return rr::rir_impl(is, fs, duration, (cudaStream_t)stream, out);
}

extern "C" rt_status rt_response_get(const rt_response* rir, rt_response_view* out) {
    if (!rir || !out) {
        rr::set_error("rt_response_get: null argument");
        return RT_ERR_INVALID_ARG;
    }
    *out = rir->v;
    return RT_OK;
}

extern "C" rt_status rt_response_download(const rt_response* rir, float* dst, void* stream) {
    rr::clear_error();
    if (!rir || !dst) {
        rr::set_error("rt_response_download: null argument");
        return RT_ERR_INVALID_ARG;
    }
    cudaStream_t s = (cudaStream_t)stream;
    size_t bytes = sizeof(float) * (size_t)std::max(rir->v.n_rcv, 1) * RT_N_BANDS * (size_t)rir->v.n_bins;
    RR_CUDA(cudaMemcpyAsync(dst, rir->v.data, bytes, cudaMemcpyDeviceToHost, s));
    RR_CUDA(cudaStreamSynchronize(s));
    return RT_OK;
}

extern "C" void rt_response_free(rt_response* rir) {
    if (!rir) return;
    for (void* p : rir->owned) rr::dev_free(p, rir->stream);
    delete rir;
}
