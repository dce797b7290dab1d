// rt_post.cu -- what the impulse responses feed: room-acoustic parameters of
// the energy histograms and the pressure response synthesised over the 8
// octave bands (Sec. 1.4: p = sqrt(E) per image source, FIR filters per band;
// Sec. 4: EDT, T30, SPL, C80, D50, Ts).
//
//   k_room_params   one block per (band, receiver): a chunked FP64 suffix scan
//                   gives the Schroeder curve, one more pass accumulates the
//                   least-squares sums of the three decay fits and the sums of
//                   C80, D50, Ts; fixed chunking and reduction order.
//   k_octave        the 8 linear-phase octave band-pass filters (windowed sinc).
//   k_pressure      one thread per output sample: the image sources of its
//                   receiver whose filter reaches it (sorted by arrival bin,
//                   found by binary search), summed in FP64 in sorted order.
#include "rt_internal.cuh"

#include <cmath>

namespace rr {

static constexpr int PP_THREADS = 1024;
static constexpr int N_PARAMS = 7;

template <typename T>
__device__ T block_sum(T v, T* red) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    __syncthreads();
    if (lane == 0) red[warp] = v;
    __syncthreads();
    T r = 0;
    if (warp == 0) {
        r = lane < (int)(blockDim.x >> 5) ? red[lane] : (T)0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) r += __shfl_down_sync(0xffffffffu, r, o);
        if (lane == 0) red[0] = r;
    }
    __syncthreads();
    r = red[0];
    __syncthreads();
    return r;
}

// slope of the least-squares line through the points, -60 / slope as a
// decay time; NaN when fewer than 2 points or the curve never gets that low
__device__ double fit_decay(double n, double st, double sl, double stt, double stl, bool reached) {
    if (!reached || n < 2.0) return nan("");
    const double den = n * stt - st * st;
    if (!(den > 0.0)) return nan("");
    const double slope = (n * stl - st * sl) / den;
    return slope < 0.0 ? -60.0 / slope : nan("");
}

__global__ void __launch_bounds__(PP_THREADS) k_room_params(const float* __restrict__ H, int64_t n_bins,
                                                             double fs, double* __restrict__ out) {
    __shared__ double red[32];
    __shared__ double scan[PP_THREADS];
    __shared__ long long bred[32];
    const int band = blockIdx.x, rcv = blockIdx.y;
    const float* e = H + ((int64_t)rcv * RT_N_BANDS + band) * n_bins;
    const int64_t per = (n_bins + PP_THREADS - 1) / PP_THREADS;
    const int64_t b_lo = (int64_t)threadIdx.x * per, b_hi = b_lo + per < n_bins ? b_lo + per : n_bins;
    // chunk sums and the first non-empty bin
    double cs = 0.0;
    long long first = LLONG_MAX;
    for (int64_t b = b_lo; b < b_hi; b++) {
        const double v = (double)e[b];
        cs += v;
        if (v > 0.0 && first == LLONG_MAX) first = b;
    }
    // suffix offsets: energy of all later chunks (a block scan from the end)
    scan[threadIdx.x] = cs;
    __syncthreads();
    for (int o = 1; o < PP_THREADS; o <<= 1) {
        const double add = threadIdx.x + o < PP_THREADS ? scan[threadIdx.x + o] : 0.0;
        __syncthreads();
        scan[threadIdx.x] += add;
        __syncthreads();
    }
    const double total = scan[0];
    // energy of the later chunks: the next thread's inclusive suffix (no
    // subtraction, which would cancel deep in the decay)
    const double suffix = threadIdx.x + 1 < PP_THREADS ? scan[threadIdx.x + 1] : 0.0;
    // the first non-empty bin of the whole histogram
    {
        long long f = first;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) f = min(f, __shfl_down_sync(0xffffffffu, f, o));
        if ((threadIdx.x & 31) == 0) bred[threadIdx.x >> 5] = f;
        __syncthreads();
        if (threadIdx.x < 32) {
            long long g = bred[threadIdx.x];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) g = min(g, __shfl_down_sync(0xffffffffu, g, o));
            if (threadIdx.x == 0) bred[0] = g;
        }
        __syncthreads();
        first = bred[0];
        __syncthreads();
    }
    double* o = out + ((int64_t)rcv * RT_N_BANDS + band) * N_PARAMS;
    if (!(total > 0.0)) {
        if (threadIdx.x == 0)
            for (int k = 0; k < N_PARAMS; k++) o[k] = nan("");
        return;
    }
    const long long n80 = (long long)ceil(0.08 * fs), n50 = (long long)ceil(0.05 * fs);
    // one pass from the end of the chunk: S[b], L[b], fit sums of the three ranges
    const double lo_db[3] = {-10.0, -25.0, -35.0}, hi_db[3] = {0.0, -5.0, -5.0};
    double fn[3] = {0, 0, 0}, ft[3] = {0, 0, 0}, fl[3] = {0, 0, 0}, ftt[3] = {0, 0, 0}, ftl[3] = {0, 0, 0};
    double reach[3] = {0, 0, 0};
    double early80 = 0.0, late80 = 0.0, early50 = 0.0, tsum = 0.0;
    double S = suffix;
    for (int64_t b = b_hi - 1; b >= b_lo; b--) {
        const double v = (double)e[b];
        S += v;
        // S <= E exactly: a rounding above it (at the direct sound) reads 0 dB
        const double L = S > 0.0 ? fmin(10.0 * log10(S / total), 0.0) : -INFINITY;
        const double t = (double)b / fs;
        const bool fit = b >= first;  // decay fits from the direct sound on
#pragma unroll
        for (int k = 0; k < 3; k++) {
            if (fit && isfinite(L) && L <= lo_db[k]) reach[k] = 1.0;
            if (fit && L <= hi_db[k] && L >= lo_db[k]) {
                fn[k] += 1.0;
                ft[k] += t;
                fl[k] += L;
                ftt[k] += t * t;
                ftl[k] += t * L;
            }
        }
        const long long rel = b - first;
        if (rel < n80)
            early80 += v;
        else
            late80 += v;
        if (rel < n50) early50 += v;
        tsum += ((double)rel + 0.5) / fs * v;
    }
    double acc[20];
    for (int k = 0; k < 3; k++) {
        acc[5 * k] = fn[k];
        acc[5 * k + 1] = ft[k];
        acc[5 * k + 2] = fl[k];
        acc[5 * k + 3] = ftt[k];
        acc[5 * k + 4] = ftl[k];
    }
    acc[15] = early80;
    acc[16] = early50;
    acc[17] = tsum;
    acc[18] = late80;
    acc[19] = reach[0] + 2.0 * reach[1] + 4.0 * reach[2];  // bit k: reached the lower limit of fit k
    double tot[19];
    for (int k = 0; k < 19; k++) tot[k] = block_sum<double>(acc[k], red);
    // flags: any thread that reached each level
    int fl_bits = (int)acc[19];
    fl_bits = __reduce_or_sync(0xffffffffu, (unsigned)fl_bits);
    if ((threadIdx.x & 31) == 0) bred[threadIdx.x >> 5] = fl_bits;
    __syncthreads();
    if (threadIdx.x == 0) {
        int any = 0;
        for (int w = 0; w < PP_THREADS / 32; w++) any |= (int)bred[w];
        for (int k = 0; k < 3; k++)
            o[k] = fit_decay(tot[5 * k], tot[5 * k + 1], tot[5 * k + 2], tot[5 * k + 3], tot[5 * k + 4],
                             (any >> k) & 1);
        o[3] = tot[18] > 0.0 ? 10.0 * log10(tot[15] / tot[18]) : INFINITY;
        o[4] = tot[16] / total;
        o[5] = tot[17] / total;
        o[6] = 10.0 * log10(total);
    }
}

// octave band f: Hann-windowed difference of two ideal low-pass sincs
__global__ void k_octave(double fs, int n_taps, double* __restrict__ g) {
    const int n = blockIdx.x * blockDim.x + threadIdx.x, f = blockIdx.y;
    if (n >= n_taps) return;
    const double D = 0.5 * (n_taps - 1);
    const double fc = 62.5 * exp2((double)f);
    const double lo = fc * 0.70710678118654752, hi = fc * 1.4142135623730951;
    const double x = (double)n - D;
    auto lp = [&](double F) {
        const double a = 2.0 * F / fs * x;
        return a == 0.0 ? 2.0 * F / fs : 2.0 * F / fs * sinpi(a) / (3.14159265358979323846 * a);
    };
    const double w = 0.5 * (1.0 - cospi(2.0 * (double)n / (double)(n_taps - 1)));
    g[(int64_t)f * n_taps + n] = w * (lp(hi) - lp(lo));
}

__global__ void k_pressure_keys(const int32_t* __restrict__ rcv, const double* __restrict__ time, int64_t n,
                                double fs, uint64_t* __restrict__ keys, uint32_t* __restrict__ vals) {
    const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n) return;
    const double b = floor(time[s] * fs);
    const uint64_t bin = b < 0.0 ? 0ull : (b > 4294967295.0 ? 0xFFFFFFFFull : (uint64_t)b);
    keys[s] = ((uint64_t)(uint32_t)rcv[s] << 32) | bin;
    vals[s] = (uint32_t)s;
}

// first index in [lo, hi) whose key is >= k
__device__ __forceinline__ int64_t lower_bound(const uint64_t* a, int64_t lo, int64_t hi, uint64_t k) {
    while (lo < hi) {
        const int64_t mid = lo + ((hi - lo) >> 1);
        if (a[mid] < k)
            lo = mid + 1;
        else
            hi = mid;
    }
    return lo;
}

// amplitudes sqrt(E_s(f)) in sorted order
__global__ void k_amplitudes(const uint32_t* __restrict__ order, int64_t n, const double* __restrict__ energy,
                             double* __restrict__ amp) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n * RT_N_BANDS) return;
    const int64_t s = i / RT_N_BANDS;
    const int f = (int)(i % RT_N_BANDS);
    amp[i] = sqrt(energy[(int64_t)order[s] * RT_N_BANDS + f]);
}

__global__ void k_pressure(const uint64_t* __restrict__ keys, int64_t n, const double* __restrict__ amp,
                           const double* __restrict__ g, int n_taps, int64_t n_out, float* __restrict__ out) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int rcv = blockIdx.y;
    if (t >= n_out) return;
    const int64_t D = (n_taps - 1) / 2;
    const uint64_t base = (uint64_t)(uint32_t)rcv << 32;
    const int64_t first_bin = t - D > 0 ? t - D : 0;
    int64_t s = lower_bound(keys, 0, n, base | (uint64_t)first_bin);
    const uint64_t last = base | (uint64_t)(t + D < 0xFFFFFFFFll ? t + D : 0xFFFFFFFFll);
    double acc = 0.0;
    for (; s < n && keys[s] <= last; s++) {
        const int64_t j = t - (int64_t)(keys[s] & 0xFFFFFFFFull) + D;  // filter tap, 0 .. n_taps - 1
        const double* as = amp + s * RT_N_BANDS;
#pragma unroll
        for (int f = 0; f < RT_N_BANDS; f++) acc += as[f] * g[(int64_t)f * n_taps + j];
    }
    out[(int64_t)rcv * n_out + t] = (float)acc;
}

}  // namespace rr

extern "C" rt_status rt_room_parameters(const float* H, int32_t n_rcv, int64_t n_bins, double fs, double* out,
                                        void* stream) {
    rr::NvtxRange nvtx_range("rt_room_parameters");
    rr::clear_error();
    if (!H || !out || n_rcv <= 0 || n_rcv > 65535 || n_bins <= 0 || !(fs > 0.0)) {
        rr::set_error("rt_room_parameters: need histograms, 0 < n_rcv <= 65535, n_bins > 0, fs > 0");
        return RT_ERR_INVALID_ARG;
    }
    cudaStream_t s = (cudaStream_t)stream;
    rr::Arena tmp(s);
    double* d_out;
    const int64_t n_out = (int64_t)n_rcv * RT_N_BANDS * rr::N_PARAMS;
    RR_TRY(tmp.alloc(&d_out, n_out));
    RR_LAUNCH(rr::k_room_params, dim3(RT_N_BANDS, n_rcv), rr::PP_THREADS, 0, s, H, n_bins, fs, d_out);
    RR_CUDA(cudaGetLastError());
    RR_CUDA(cudaMemcpyAsync(out, d_out, sizeof(double) * n_out, cudaMemcpyDeviceToHost, s));
    RR_CUDA(cudaStreamSynchronize(s));
    return RT_OK;
}

extern "C" rt_status rt_pressure_rir(const rt_image_sources* is, double fs, int64_t n_out, int32_t n_taps,
                                     float* out, void* stream) {
    rr::NvtxRange nvtx_range("rt_pressure_rir");
    rr::clear_error();
    if (!is || !out || !(fs > 0.0) || n_out <= 0 || n_out > 0x7FFFFFFFll || n_taps < 3 || n_taps % 2 == 0 ||
        n_taps > (1 << 20)) {
        rr::set_error("rt_pressure_rir: need image sources, fs > 0, 0 < n_out < 2^31, odd 3 <= n_taps <= 2^20");
        return RT_ERR_INVALID_ARG;
    }
    cudaStream_t s = (cudaStream_t)stream;
    const int64_t n = is->v.n;
    const int R = is->n_rcv;
    rr::Arena tmp(s);
    double* g;
    RR_TRY(tmp.alloc(&g, (int64_t)RT_N_BANDS * n_taps));
    RR_LAUNCH(rr::k_octave, dim3((n_taps + 255) / 256, RT_N_BANDS), 256, 0, s, fs, n_taps, g);
    uint64_t *keys = nullptr, *keys_alt = nullptr;
    uint32_t *vals = nullptr, *vals_alt = nullptr;
    double* amp = nullptr;
    if (n > 0) {
        RR_TRY(tmp.alloc(&keys, n));
        RR_TRY(tmp.alloc(&keys_alt, n));
        RR_TRY(tmp.alloc(&vals, n));
        RR_TRY(tmp.alloc(&vals_alt, n));
        void* sort_tmp;
        RR_TRY(tmp.alloc((char**)&sort_tmp, rr::sort_temp_bytes(n)));
        RR_LAUNCH(rr::k_pressure_keys, (unsigned)((n + 255) / 256), 256, 0, s, is->v.rcv, is->v.time, n, fs, keys,
                  vals);
        RR_TRY(rr::radix_sort_pairs(keys, vals, keys_alt, vals_alt, n, 0, 64, sort_tmp, s));
        RR_TRY(tmp.alloc(&amp, n * RT_N_BANDS));
        RR_LAUNCH(rr::k_amplitudes, (unsigned)((n * RT_N_BANDS + 255) / 256), 256, 0, s, vals, n, is->v.energy, amp);
    }
    RR_LAUNCH(rr::k_pressure, dim3((unsigned)((n_out + 255) / 256), (unsigned)R), 256, 0, s, keys, n, amp, g,
              (int)n_taps, n_out, out);
    RR_CUDA(cudaGetLastError());
    RR_CUDA(cudaStreamSynchronize(s));
    return RT_OK;
}
