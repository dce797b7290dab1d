// rt_surrogate.cu -- surrogate-tail mode: the learned late reverberation
// behind the C ABI (no counterpart in the paper; the method itself stays the
// fallback and the reference the predictions are measured against).
//
// A room (one source, one receiver sphere) is traced twice with few rays: a
// 0-50 ms trace (1 ms bins) and a 2 s tail probe (10 ms bins).  With the
// room's descriptors and the specular tail prior (rt_tail_prior) they form the
// network input; an ensemble of rt_mlp networks predicts the 8-band energy
// decay of the tail (50 ms - 2 s in 10 ms bins) as a correction to a base
// curve; a gate sends a room to full tracing when its descriptors leave the
// training range or the prediction disagrees with the traced early part or
// the probe.  Everything below runs on the device; the host only loops over
// batches of rooms and reads the gate's verdicts.
//
// Layouts (per room, float, row-major):
//   desc   [47]      log10 V, log10 S, area-weighted mean alpha [8], log10 of
//                    the share of S facing x / y / z (+1e-6), log10 of the
//                    energy-decay rate of each axis group [3][8] (+1e-6), air
//                    rate c beta [8], log10 r, log10 (V / bounding-box volume)
//   early  [8][50]   energy per 1 ms bin, 0-50 ms
//   probe  [8][195]  energy per 10 ms bin, 50 ms - 2 s, of the tail probe
//   *_db   [8][195]  tail decay curve: 10 log10 of the energy still to arrive
//                    from each bin start (backward sum) + 1e-30
//   target form      per band the curve's first value, then its decay
//                    relative to it clamped at -50 dB
//   X      [951]     desc, 10 log10 (early + 1e-10), and the probe's minus the
//                    prior's decay in target form at 63 bins per band (every
//                    bin below 300 ms, then every 50 ms)
//   env    [8][200]  energy per 10 ms bin, 0-2 s: traced 0-50 ms + the tail
#include "rt_internal.cuh"

#include <algorithm>
#include <cmath>
#include <cstring>
#include <numeric>
#include <random>
#include <vector>

namespace rr {
namespace sur {

constexpr int N_DESC = RT_SUR_N_DESC;
constexpr int N_EARLY = RT_SUR_N_EARLY;
constexpr int N_TAIL = RT_SUR_N_TAIL;
constexpr int N_ENV = RT_SUR_N_ENV;
constexpr int FIRST_TAIL = N_ENV - N_TAIL;  // 5: the tail starts at 50 ms
constexpr int N_PROBE = 63;
constexpr int N_FEAT = RT_SUR_N_FEAT;
constexpr int N_IN = (N_FEAT + 31) / 32 * 32;  // 960
constexpr int N_HIDDEN = 512;
constexpr int N_OUT_RAW = 8 * N_TAIL;            // 1560
constexpr int N_OUT = (N_OUT_RAW + 31) / 32 * 32;  // 1568
constexpr int X_EARLY = N_DESC;                  // 47
constexpr int X_PROBE = N_DESC + 8 * N_EARLY;    // 447
constexpr int BASE_PROBE_BINS = 20;  // the base curve follows the probe for the first 200 ms of the tail
constexpr double REL_FLOOR_DB = 50.0;
constexpr double FLOOR = 1e-30;
constexpr double FLOOR_IN = 1e-10;
constexpr double EARLY_S = 0.05, EARLY_FS = 1000.0, TAIL_FS = 100.0, DURATION = 2.0;
constexpr int PRIOR_NODES = 64;
constexpr int FULL_BOUNCES = 768;
constexpr int EARLY_BOUNCES = 64;
static_assert(X_PROBE + 8 * N_PROBE == N_FEAT, "feature layout");

// bins of the tail read by the features and the probe gate: every bin up to
// 300 ms of the tail, then every 50 ms
__host__ __device__ __forceinline__ int probe_bin(int j) { return j < 30 ? j : 30 + 5 * (j - 30); }

// loss weight of output k of a band: the level at 50 ms (x9) and the first
// 300 ms of the decay (x4) decide the early decay time
__host__ __device__ __forceinline__ double loss_weight(int k) { return k == 0 ? 9.0 : (k < 30 ? 4.0 : 1.0); }

// target form of a decay curve (in place is not allowed: d and t differ)
__device__ __forceinline__ void to_targets(const double* d, double* t) {
    t[0] = d[0];
    for (int k = 1; k < N_TAIL; k++) t[k] = fmax(d[k] - d[0], -REL_FLOOR_DB);
}

// backward-integrated tail energy in dB
__device__ __forceinline__ void tail_edc_db(const float* e, double* d) {
    double acc = 0.0;
    for (int k = N_TAIL - 1; k >= 0; k--) {
        acc += (double)e[k];
        d[k] = 10.0 * log10(acc + FLOOR);
    }
}

// per-bin energy of a (predicted) decay curve, made non-increasing first
__device__ __forceinline__ double edc_bin_energy(const double* edc_db, int k) {
    // e_j = min over i <= j of 10^(edc_i / 10): the running minimum
    double run = INFINITY, ek = 0.0, en = 0.0;
    for (int j = 0; j <= k + 1 && j < N_TAIL; j++) {
        run = fmin(run, pow(10.0, edc_db[j] / 10.0));
        if (j == k) ek = run;
        if (j == k + 1) en = run;
    }
    if (k + 1 >= N_TAIL) en = 0.0;
    return fmax(ek - en, 0.0);
}

// ---------------------------------------------------------------------------
// descriptors: one block per room, FP64 sums over its triangles
// ---------------------------------------------------------------------------
struct DescRoom {
    const float4* tris;         // tree order: v0 (w = id), v1 (w = surface), v2
    const int32_t* mat_of_surf;
    const float* alpha;         // [n_mat][8] the room's absorption table
    int64_t n_tris;
    double volume, radius;
};

constexpr int DESC_THREADS = 256;
constexpr int DESC_SUMS = 1 + 8 + 3 + 24;  // S, area alpha [8], area per axis [3], area loss [3][8]

__global__ void __launch_bounds__(DESC_THREADS) k_descriptors(const DescRoom* __restrict__ rooms, const double* __restrict__ beta,
                                                            double c, float* __restrict__ desc) {
    const DescRoom rm = rooms[blockIdx.x];
    double acc[DESC_SUMS];
    for (int k = 0; k < DESC_SUMS; k++) acc[k] = 0.0;
    double lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
    for (int64_t t = threadIdx.x; t < rm.n_tris; t += blockDim.x) {
        const float4 A = rm.tris[3 * t], B = rm.tris[3 * t + 1], C = rm.tris[3 * t + 2];
        const double ax = A.x, ay = A.y, az = A.z;
        const double ux = B.x - ax, uy = B.y - ay, uz = B.z - az;
        const double vx = C.x - ax, vy = C.y - ay, vz = C.z - az;
        const double n[3] = {uy * vz - uz * vy, uz * vx - ux * vz, ux * vy - uy * vx};
        const double area = 0.5 * sqrt(n[0] * n[0] + n[1] * n[1] + n[2] * n[2]);
        int axis = 0;
        if (fabs(n[1]) > fabs(n[axis])) axis = 1;
        if (fabs(n[2]) > fabs(n[axis])) axis = 2;
        const int mat = rm.mat_of_surf[__float_as_int(B.w)];
        acc[0] += area;
        acc[9 + axis] += area;
        for (int f = 0; f < 8; f++) {
            const double al = (double)rm.alpha[8 * mat + f];
            acc[1 + f] += area * al;
            acc[12 + 8 * axis + f] += area * -log(fmin(fmax(1.0 - al, 1e-6), 1.0));
        }
        const float4 P[3] = {A, B, C};
        for (int v = 0; v < 3; v++) {
            lo[0] = fmin(lo[0], (double)P[v].x), hi[0] = fmax(hi[0], (double)P[v].x);
            lo[1] = fmin(lo[1], (double)P[v].y), hi[1] = fmax(hi[1], (double)P[v].y);
            lo[2] = fmin(lo[2], (double)P[v].z), hi[2] = fmax(hi[2], (double)P[v].z);
        }
    }
    // block reduction: warps first, then one row per warp in shared memory
    __shared__ double red[DESC_THREADS / 32][DESC_SUMS + 6];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int k = 0; k < DESC_SUMS; k++)
        for (int o = 16; o > 0; o >>= 1) acc[k] += __shfl_down_sync(0xffffffffu, acc[k], o);
    for (int k = 0; k < 3; k++)
        for (int o = 16; o > 0; o >>= 1) {
            lo[k] = fmin(lo[k], __shfl_down_sync(0xffffffffu, lo[k], o));
            hi[k] = fmax(hi[k], __shfl_down_sync(0xffffffffu, hi[k], o));
        }
    if (lane == 0) {
        for (int k = 0; k < DESC_SUMS; k++) red[warp][k] = acc[k];
        for (int k = 0; k < 3; k++) red[warp][DESC_SUMS + k] = lo[k], red[warp][DESC_SUMS + 3 + k] = hi[k];
    }
    __syncthreads();
    if (threadIdx.x != 0) return;
    for (int w = 1; w < DESC_THREADS / 32; w++) {
        for (int k = 0; k < DESC_SUMS; k++) red[0][k] += red[w][k];
        for (int k = 0; k < 3; k++) {
            red[0][DESC_SUMS + k] = fmin(red[0][DESC_SUMS + k], red[w][DESC_SUMS + k]);
            red[0][DESC_SUMS + 3 + k] = fmax(red[0][DESC_SUMS + 3 + k], red[w][DESC_SUMS + 3 + k]);
        }
    }
    const double* s = red[0];
    const double S = s[0], V = rm.volume;
    float* o = desc + (int64_t)blockIdx.x * N_DESC;
    o[0] = (float)log10(V);
    o[1] = (float)log10(S);
    for (int f = 0; f < 8; f++) o[2 + f] = (float)(s[1 + f] / S);
    for (int k = 0; k < 3; k++) o[10 + k] = (float)log10(s[9 + k] / S + 1e-6);
    for (int k = 0; k < 24; k++) o[13 + k] = (float)log10(c * s[12 + k] / (2.0 * V) + 1e-6);
    for (int f = 0; f < 8; f++) o[37 + f] = (float)(c * beta[f]);
    o[45] = (float)log10(rm.radius);
    double box = 1.0;
    for (int k = 0; k < 3; k++) box *= s[DESC_SUMS + 3 + k] - s[DESC_SUMS + k];
    o[46] = (float)log10(V / box);
}

// inputs of rt_tail_prior from the descriptors: per-axis rates, air rates and
// the diffuse level pi r^2 c dt / V of the measurement sphere
__global__ void k_prior_inputs(const float* __restrict__ desc, int n, double c, float* __restrict__ rates,
                               float* __restrict__ air, float* __restrict__ level) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float* d = desc + (int64_t)i * N_DESC;
    for (int k = 0; k < 24; k++) rates[24 * (int64_t)i + k] = (float)fmax(pow(10.0, (double)d[13 + k]) - 1e-6, 0.0);
    for (int f = 0; f < 8; f++) air[8 * (int64_t)i + f] = d[37 + f];
    const double r = pow(10.0, (double)d[45]);
    level[i] = (float)(3.14159265358979323846 * r * r * c / TAIL_FS / pow(10.0, (double)d[0]));
}

// prior energies [n][8][195] -> prior decay curves [n][8][195] (in place is fine: one thread per band)
__global__ void k_energy_to_db(const float* __restrict__ e, int n, float* __restrict__ db) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= 8 * n) return;
    double d[N_TAIL];
    tail_edc_db(e + (int64_t)i * N_TAIL, d);
    for (int k = 0; k < N_TAIL; k++) db[(int64_t)i * N_TAIL + k] = (float)d[k];
}

// features and base curve: one thread per (room, band)
__global__ void k_features(const float* __restrict__ desc, const float* __restrict__ early,
                           const float* __restrict__ probe, const float* __restrict__ prior_db, int n,
                           float* __restrict__ X, float* __restrict__ base_db) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= 8 * n) return;
    const int room = i / 8, f = i % 8;
    double pd[N_TAIL], a[N_TAIL], b[N_TAIL];
    tail_edc_db(probe + (int64_t)i * N_TAIL, pd);
    to_targets(pd, a);
    for (int k = 0; k < N_TAIL; k++) pd[k] = prior_db[(int64_t)i * N_TAIL + k];
    to_targets(pd, b);
    float* x = X + (int64_t)room * N_FEAT;
    if (f == 0)
        for (int k = 0; k < N_DESC; k++) x[k] = desc[(int64_t)room * N_DESC + k];
    for (int k = 0; k < N_EARLY; k++)
        x[X_EARLY + f * N_EARLY + k] = (float)(10.0 * log10((double)early[(int64_t)i * N_EARLY + k] + FLOOR_IN));
    for (int j = 0; j < N_PROBE; j++) x[X_PROBE + f * N_PROBE + j] = (float)(a[probe_bin(j)] - b[probe_bin(j)]);
    // base: the probe's level and decay over the first BASE_PROBE_BINS bins,
    // then the prior's decay joined without a step; back to a decay curve
    double t[N_TAIL];
    const int K = BASE_PROBE_BINS;
    for (int k = 0; k < N_TAIL; k++) t[k] = k < K ? a[k] : b[k] - b[K - 1] + a[K - 1];
    float* o = base_db + (int64_t)i * N_TAIL;
    o[0] = (float)t[0];
    for (int k = 1; k < N_TAIL; k++) o[k] = (float)(t[0] + fmin(fmax(t[k], -REL_FLOOR_DB), 0.0));
}

// -- prediction ---------------------------------------------------------------
// normalised network input [n][960]: (X - mean) / std, zero padding
__global__ void k_norm_x(const float* __restrict__ X, int64_t rows, const float* __restrict__ mean,
                         const float* __restrict__ std_, float* __restrict__ out) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= rows * N_IN) return;
    const int64_t r = i / N_IN;
    const int c = (int)(i % N_IN);
    out[i] = c < N_FEAT ? (X[r * N_FEAT + c] - mean[c]) / std_[c] : 0.f;
}

// ensemble mean of the networks' outputs (target form, normalised), plus the
// base curve in target form, back to a decay curve: one thread per (room, band)
__global__ void k_predict_db(const float* __restrict__ Y, int n_nets, int64_t n, const float* __restrict__ y_mean,
                             const float* __restrict__ y_std, const float* __restrict__ base_db, int residual,
                             float* __restrict__ pred_db) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= 8 * n) return;
    const int64_t room = i / 8;
    const int f = (int)(i % 8);
    double b[N_TAIL], t[N_TAIL];
    if (residual) {
        double bd[N_TAIL];
        for (int k = 0; k < N_TAIL; k++) bd[k] = base_db[i * N_TAIL + k];
        to_targets(bd, b);
    }
    for (int k = 0; k < N_TAIL; k++) {
        const int col = f * N_TAIL + k;
        double y = 0.0;
        for (int m = 0; m < n_nets; m++) y += Y[((int64_t)m * n + room) * N_OUT + col];
        y = y / n_nets * y_std[col] + y_mean[col];
        t[k] = residual ? y + b[k] : y;
    }
    float* o = pred_db + i * N_TAIL;
    o[0] = (float)t[0];
    for (int k = 1; k < N_TAIL; k++) o[k] = (float)(t[0] + fmin(fmax(t[k], -REL_FLOOR_DB), 0.0));
}

// -- gate ----------------------------------------------------------------------
// per room: inside the training range (2 % margin), the join gap (largest over
// bands with traced energy in 40-50 ms of |predicted 50-60 ms - traced
// 40-50 ms| in dB; 0 when no band has traced energy there: the early trace
// then says nothing about the join, and the probe gap still checks the
// level) and the probe
// gap (largest over bands of the RMS between the predicted and the probe's
// decay in target form at the probe bins)
__global__ void k_gate(const float* __restrict__ desc, const float* __restrict__ X, const float* __restrict__ pred_db,
                       const float* __restrict__ prior_db, int n, const float* __restrict__ lo,
                       const float* __restrict__ hi, float* __restrict__ gaps, int32_t* __restrict__ in_range) {
    const int room = blockIdx.x * blockDim.x + threadIdx.x;
    if (room >= n) return;
    int ok = 1;
    for (int k = 0; k < N_DESC; k++) {
        const float span = hi[k] - lo[k], d = desc[(int64_t)room * N_DESC + k];
        if (!(d >= lo[k] - 0.02f * span && d <= hi[k] + 0.02f * span)) ok = 0;
    }
    in_range[room] = ok;
    const float* x = X + (int64_t)room * N_FEAT;
    double join = -1.0, probe = 0.0;
    for (int f = 0; f < 8; f++) {
        const float* pd = pred_db + ((int64_t)room * 8 + f) * N_TAIL;
        double p[N_TAIL], q[N_TAIL], tp[N_TAIL], tq[N_TAIL];
        for (int k = 0; k < N_TAIL; k++) p[k] = pd[k], q[k] = prior_db[((int64_t)room * 8 + f) * N_TAIL + k];
        double traced = 0.0;
        for (int k = 40; k < 50; k++) traced += pow(10.0, (double)x[X_EARLY + f * N_EARLY + k] / 10.0) - FLOOR_IN;
        if (traced > 0.5 * FLOOR_IN) {
            const double pred0 = 10.0 * log10(edc_bin_energy(p, 0) + FLOOR_IN);
            join = fmax(join, fabs(pred0 - 10.0 * log10(traced)));
        }
        to_targets(p, tp);
        to_targets(q, tq);
        double ss = 0.0;
        for (int j = 0; j < N_PROBE; j++) {
            const double d = (tp[probe_bin(j)] - tq[probe_bin(j)]) - (double)x[X_PROBE + f * N_PROBE + j];
            ss += d * d;
        }
        probe = fmax(probe, sqrt(ss / N_PROBE));
    }
    gaps[2 * room] = join < 0.0 ? 0.0f : (float)join;  // no traced 40-50 ms energy: nothing to join against
    gaps[2 * room + 1] = (float)probe;
}

// -- envelopes -------------------------------------------------------------------
// env [n][8][200]: the traced 0-50 ms summed into 10 ms bins, then the tail
// (per-bin energies, or a decay curve in dB turned into per-bin energies)
__global__ void k_envelope(const float* __restrict__ early, const float* __restrict__ tail, int tail_is_db, int n,
                           float* __restrict__ env) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= 8 * (int64_t)n) return;
    float* o = env + i * N_ENV;
    for (int b = 0; b < FIRST_TAIL; b++) {
        double s = 0.0;
        for (int k = 0; k < 10; k++) s += (double)early[i * N_EARLY + 10 * b + k];
        o[b] = (float)s;
    }
    const float* t = tail + i * N_TAIL;
    if (!tail_is_db) {
        for (int k = 0; k < N_TAIL; k++) o[FIRST_TAIL + k] = t[k];
        return;
    }
    double run = INFINITY, prev = 0.0;
    for (int k = 0; k < N_TAIL; k++) {
        run = fmin(run, pow(10.0, (double)t[k] / 10.0));
        if (k > 0) o[FIRST_TAIL + k - 1] = (float)fmax(prev - run, 0.0);
        prev = run;
    }
    o[FIRST_TAIL + N_TAIL - 1] = (float)fmax(prev, 0.0);
}

// full-trace histograms [n][8][200] (10 ms) -> tail decay curves [n][8][195]
__global__ void k_hist_tail_db(const float* __restrict__ hist, int n, float* __restrict__ db) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= 8 * (int64_t)n) return;
    double d[N_TAIL];
    tail_edc_db(hist + i * N_ENV + FIRST_TAIL, d);
    for (int k = 0; k < N_TAIL; k++) db[i * N_TAIL + k] = (float)d[k];
}

// copy rows [n][8][w] from a batch histogram whose bins start at `first`
__global__ void k_copy_bins(const float* __restrict__ src, int src_bins, int first, int n, int w,
                            float* __restrict__ dst) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= 8 * (int64_t)n * w) return;
    const int64_t row = i / w;
    const int k = (int)(i % w);
    dst[i] = src[row * src_bins + first + k];
}

// -- training ------------------------------------------------------------------
// residual targets in target form: targets(edc) - targets(base)  [n][1560]
__global__ void k_residual_targets(const float* __restrict__ edc_db, const float* __restrict__ base_db, int64_t n,
                                   int residual, float* __restrict__ Y) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= 8 * n) return;
    double d[N_TAIL], t[N_TAIL], bd[N_TAIL], tb[N_TAIL];
    for (int k = 0; k < N_TAIL; k++) d[k] = edc_db[i * N_TAIL + k], bd[k] = base_db[i * N_TAIL + k];
    to_targets(d, t);
    to_targets(bd, tb);
    for (int k = 0; k < N_TAIL; k++) Y[i * N_TAIL + k] = (float)(residual ? t[k] - tb[k] : t[k]);
}

// column mean and standard deviation (FP64, two passes) over the listed rows;
// std + 1e-6, divided by sqrt(w) for the output columns
__global__ void k_col_stats(const float* __restrict__ A, int cols, const int32_t* __restrict__ rows, int n_rows,
                            int weighted, float* __restrict__ mean, float* __restrict__ std_) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= cols) return;
    double s = 0.0;
    for (int r = 0; r < n_rows; r++) s += (double)A[(int64_t)rows[r] * cols + c];
    const double m = s / n_rows;
    double v = 0.0;
    for (int r = 0; r < n_rows; r++) {
        const double d = (double)A[(int64_t)rows[r] * cols + c] - m;
        v += d * d;
    }
    double sd = sqrt(v / n_rows) + 1e-6;
    if (weighted) sd /= sqrt(loss_weight(c % N_TAIL));
    mean[c] = (float)m;
    std_[c] = (float)sd;
}

// counter-based generator (splitmix64 steps): index and normal draws of a batch
__host__ __device__ __forceinline__ uint64_t mix64(uint64_t z) {
    z += 0x9E3779B97F4A7C15ULL;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

// one training batch: rows drawn from the training list, normalised inputs
// with Gaussian noise (Box-Muller) on the feature columns, normalised targets
__global__ void k_batch(const float* __restrict__ X, const float* __restrict__ Y, const int32_t* __restrict__ rows,
                        int n_rows, const float* __restrict__ xm, const float* __restrict__ xs,
                        const float* __restrict__ ym, const float* __restrict__ ys, int batch, uint64_t key,
                        float noise, float* __restrict__ xb, float* __restrict__ yb) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t nx = (int64_t)batch * N_IN, ny = (int64_t)batch * N_OUT;
    if (i >= nx + ny) return;
    if (i < nx) {
        const int b = (int)(i / N_IN), c = (int)(i % N_IN);
        const int32_t r = rows[mix64(key ^ (uint64_t)b) % (uint64_t)n_rows];
        float v = 0.f;
        if (c < N_FEAT) {
            v = (X[(int64_t)r * N_FEAT + c] - xm[c]) / xs[c];
            if (noise > 0.f) {
                const uint64_t h = mix64(mix64(key + 0x5851F42D4C957F2DULL) ^ (uint64_t)i);
                const double u1 = ((h >> 11) + 1.0) * (1.0 / 9007199254740993.0);
                const double u2 = (double)(mix64(h) >> 11) * (1.0 / 9007199254740992.0);
                v += noise * (float)(sqrt(-2.0 * log(u1)) * cos(6.283185307179586 * u2));
            }
        }
        xb[i] = v;
    } else {
        const int64_t j = i - nx;
        const int b = (int)(j / N_OUT), c = (int)(j % N_OUT);
        const int32_t r = rows[mix64(key ^ (uint64_t)b) % (uint64_t)n_rows];
        yb[j] = c < N_OUT_RAW ? (Y[(int64_t)r * N_OUT_RAW + c] - ym[c]) / ys[c] : 0.f;
    }
}

// rows of a list, normalised (validation set)
__global__ void k_norm_rows(const float* __restrict__ A, int cols, int cols_pad, const int32_t* __restrict__ rows,
                            int n_rows, const float* __restrict__ m, const float* __restrict__ sd,
                            float* __restrict__ out) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (int64_t)n_rows * cols_pad) return;
    const int64_t r = i / cols_pad;
    const int c = (int)(i % cols_pad);
    out[i] = c < cols ? (A[(int64_t)rows[r] * cols + c] - m[c]) / sd[c] : 0.f;
}

// squared error over the real output columns, partial sums per block
__global__ void k_sq_err(const float* __restrict__ y, const float* __restrict__ t, int64_t rows,
                         double* __restrict__ part) {
    __shared__ double red[256];
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    double e = 0.0;
    if (i < rows * N_OUT && (int)(i % N_OUT) < N_OUT_RAW) {
        const double d = (double)y[i] - (double)t[i];
        e = d * d;
    }
    red[threadIdx.x] = e;
    __syncthreads();
    for (int s = 128; s > 0; s >>= 1) {
        if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.x] = red[0];
}

// gather rows of a [*][cols] array
__global__ void k_gather_rows(const float* __restrict__ A, int cols, const int32_t* __restrict__ rows, int n_rows,
                              float* __restrict__ out) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (int64_t)n_rows * cols) return;
    out[i] = A[(int64_t)rows[i / cols] * cols + i % cols];
}

}  // namespace sur
}  // namespace rr

// ---------------------------------------------------------------------------
// the model
// ---------------------------------------------------------------------------
// statistics block (device float): feature mean / std, output mean / std,
// descriptor range of the training rooms
namespace rr {
namespace sur {
constexpr int ST_XM = 0, ST_XS = N_FEAT, ST_YM = 2 * N_FEAT, ST_YS = 2 * N_FEAT + N_OUT_RAW,
              ST_LO = 2 * N_FEAT + 2 * N_OUT_RAW, ST_HI = ST_LO + N_DESC, ST_N = ST_HI + N_DESC;

// descriptor range over listed rows: one thread per column
__global__ void k_desc_range(const float* __restrict__ desc, const int32_t* __restrict__ rows, int n_rows,
                             float* __restrict__ lo, float* __restrict__ hi) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= N_DESC) return;
    float a = INFINITY, b = -INFINITY;
    for (int r = 0; r < n_rows; r++) {
        const float v = desc[(int64_t)rows[r] * N_DESC + c];
        a = fminf(a, v), b = fmaxf(b, v);
    }
    lo[c] = a, hi[c] = b;
}
}  // namespace sur
}  // namespace rr

struct rt_surrogate {
    std::vector<rt_mlp*> nets;
    float* stats = nullptr;   // device [ST_N]
    float join_db = 9.f, probe_db = 9.f;
    int32_t residual = 1;
    std::vector<float> history;  // (member, step, validation loss) triples
    std::vector<void*> owned;
    cudaStream_t stream = nullptr;
    ~rt_surrogate() {
        for (rt_mlp* m : nets) rt_mlp_free(m);
        for (void* p : owned) rr::dev_free(p, stream);
    }
};

namespace rr {
namespace sur {

static unsigned g1(int64_t n, int t = 256) { return (unsigned)((n + t - 1) / t); }

struct TraceCfg {
    int early_rays, probe_rays, full_rays, per_launch;
    const float* air;
    double c;
    cudaStream_t s;
    rt_workspace* ws;
};

static rt_status trace_cfg(const rt_surrogate_trace_params* p, TraceCfg& t) {
    if (!p) {
        set_error("surrogate: null trace parameters");
        return RT_ERR_INVALID_ARG;
    }
    t.early_rays = p->early_rays > 0 ? p->early_rays : 65536;
    t.probe_rays = p->probe_rays > 0 ? p->probe_rays : 16384;
    t.full_rays = p->full_rays > 0 ? p->full_rays : 1000000;
    t.per_launch = p->rooms_per_launch > 0 ? p->rooms_per_launch : 16;
    t.air = p->air_beta;
    t.c = p->c > 0 ? p->c : 343.2;
    t.s = (cudaStream_t)p->stream;
    t.ws = p->workspace;
    return RT_OK;
}

static rt_status check_rooms(const rt_room* rooms, int32_t n, const double* volume) {
    if (!rooms || n < 1) {
        set_error("surrogate: need n >= 1 rooms");
        return RT_ERR_INVALID_ARG;
    }
    for (int k = 0; k < n; k++) {
        const rt_room& r = rooms[k];
        if (!r.tree || r.sources.n != 1 || r.receivers.n != 1 || !r.receivers.radius || !r.band_absorption) {
            set_error("surrogate: room %d needs a tree, one source and one receiver", k);
            return RT_ERR_INVALID_ARG;
        }
        if (volume && !(volume[k] > 0.0)) {
            set_error("surrogate: room %d has volume %g (need > 0)", k, volume ? volume[k] : 0.0);
            return RT_ERR_INVALID_ARG;
        }
    }
    return RT_OK;
}

// Histograms of rooms [k0, k1) traced in one batched launch: rays per source,
// n_bounces, path cut at max_distance, binned at fs over `duration`; rows
// [8][w] starting at bin `first` are copied to dst rows k0 .. k1-1.
static rt_status batch_hist(const rt_room* rooms, int k0, int k1, const TraceCfg& t, int64_t n_rays, int n_bounces,
                            double max_distance, double fs, double duration, int src_bins, int first, int w,
                            float* dst) {
    rt_trace_params tp{};
    tp.n_rays = n_rays;
    tp.n_bounces = n_bounces;
    tp.max_distance = max_distance;
    tp.air_beta = t.air;
    tp.c = t.c;
    // one launch in tail mode (lanes refilled as rays die), 128-thread blocks:
    // the fastest configuration measured for closed rooms, and no autotuner
    // trials inside timed surrogate calls
    tp.tail_rays = 0x7FFFFFFF;
    tp.block_size = 128;
    tp.stream = t.s;
    tp.workspace = t.ws;
    rt_image_sources* is = nullptr;
    RR_TRY(rt_trace_batch(rooms + k0, k1 - k0, &tp, &is));
    rt_response* resp = nullptr;
    const rt_status st = rt_rir(is, fs, duration, t.s, &resp);
    rt_image_sources_free(is);
    if (st != RT_OK) return st;
    const int m = k1 - k0;
    if (resp->v.n_rcv != m || resp->v.n_bins != src_bins) {
        rt_response_free(resp);
        set_error("surrogate: unexpected histogram shape");
        return RT_ERR_INTERNAL;
    }
    RR_LAUNCH(k_copy_bins, g1((int64_t)8 * m * w), 256, 0, t.s, resp->v.data, src_bins, first, m, w,
              dst + (int64_t)k0 * 8 * w);
    const cudaError_t e = cudaGetLastError();
    // the response's memory is freed stream-ordered after the copy
    rt_response_free(resp);
    return cuda_status(e, "k_copy_bins");
}

static rt_status inputs_impl(const rt_room* rooms, const double* volume, int32_t n, const TraceCfg& t, float* desc,
                             float* early, float* probe, float* prior_db, float* base_db, float* X) {
    cudaStream_t s = t.s;
    Arena tmp(s);
    if (!desc) RR_TRY(tmp.alloc(&desc, (size_t)n * N_DESC));
    if (!early) RR_TRY(tmp.alloc(&early, (size_t)n * 8 * N_EARLY));
    if (!probe) RR_TRY(tmp.alloc(&probe, (size_t)n * 8 * N_TAIL));
    if (!prior_db) RR_TRY(tmp.alloc(&prior_db, (size_t)n * 8 * N_TAIL));
    for (int k0 = 0; k0 < n; k0 += t.per_launch) {
        const int k1 = std::min(n, k0 + t.per_launch);
        RR_TRY(batch_hist(rooms, k0, k1, t, t.early_rays, EARLY_BOUNCES, EARLY_S * t.c, EARLY_FS, EARLY_S, N_EARLY,
                          0, N_EARLY, early));
        RR_TRY(batch_hist(rooms, k0, k1, t, t.probe_rays, FULL_BOUNCES, DURATION * t.c, TAIL_FS, DURATION, N_ENV,
                          FIRST_TAIL, N_TAIL, probe));
    }
    // descriptors from the trees' triangles and the absorption tables
    std::vector<DescRoom> h((size_t)n);
    std::vector<float> alpha;
    std::vector<size_t> a_off((size_t)n);
    for (int k = 0; k < n; k++) {
        a_off[k] = alpha.size();
        alpha.insert(alpha.end(), rooms[k].band_absorption,
                     rooms[k].band_absorption + (size_t)rooms[k].n_materials * RT_N_BANDS);
    }
    float* d_alpha;
    DescRoom* d_rooms;
    double* d_beta;
    RR_TRY(tmp.alloc(&d_alpha, std::max<size_t>(alpha.size(), 1)));
    RR_TRY(tmp.alloc(&d_rooms, (size_t)n));
    RR_TRY(tmp.alloc(&d_beta, 8));
    for (int k = 0; k < n; k++) {
        const rt_tree* tr = rooms[k].tree;
        h[k] = DescRoom{tr->tris, tr->mat_of_surf, d_alpha + a_off[k], tr->n_tris, volume[k],
                        rooms[k].receivers.radius[0]};
    }
    double hb[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    if (t.air)
        for (int f = 0; f < 8; f++) hb[f] = (double)t.air[f];
    RR_CUDA(cudaMemcpyAsync(d_alpha, alpha.data(), sizeof(float) * alpha.size(), cudaMemcpyHostToDevice, s));
    RR_CUDA(cudaMemcpyAsync(d_rooms, h.data(), sizeof(DescRoom) * h.size(), cudaMemcpyHostToDevice, s));
    RR_CUDA(cudaMemcpyAsync(d_beta, hb, sizeof hb, cudaMemcpyHostToDevice, s));
    RR_LAUNCH(k_descriptors, (unsigned)n, DESC_THREADS, 0, s, d_rooms, d_beta, t.c, desc);
    // the specular prior at the descriptors' rates and level
    float *rates, *air, *level, *prior_e;
    RR_TRY(tmp.alloc(&rates, (size_t)n * 24));
    RR_TRY(tmp.alloc(&air, (size_t)n * 8));
    RR_TRY(tmp.alloc(&level, (size_t)n));
    RR_TRY(tmp.alloc(&prior_e, (size_t)n * 8 * N_TAIL));
    RR_LAUNCH(k_prior_inputs, g1(n), 256, 0, s, desc, n, t.c, rates, air, level);
    RR_CUDA(cudaGetLastError());
    for (int k0 = 0; k0 < n; k0 += 65535) {
        const int m = std::min(n - k0, 65535);
        RR_TRY(rt_tail_prior(rates + (int64_t)24 * k0, air + (int64_t)8 * k0, level + k0, m, PRIOR_NODES,
                             (float)EARLY_S, (float)(1.0 / TAIL_FS), N_TAIL, prior_e + (int64_t)k0 * 8 * N_TAIL, s));
    }
    RR_LAUNCH(k_energy_to_db, g1((int64_t)8 * n), 256, 0, s, prior_e, n, prior_db);
    if (X || base_db) {
        float *Xw = X, *bw = base_db;
        if (!Xw) RR_TRY(tmp.alloc(&Xw, (size_t)n * N_FEAT));
        if (!bw) RR_TRY(tmp.alloc(&bw, (size_t)n * 8 * N_TAIL));
        RR_LAUNCH(k_features, g1((int64_t)8 * n, 128), 128, 0, s, desc, early, probe, prior_db, n, Xw, bw);
    }
    RR_CUDA(cudaGetLastError());
    // the temporaries are freed stream-ordered; the host copies above read
    // host vectors that must outlive the transfers
    RR_CUDA(cudaStreamSynchronize(s));
    return RT_OK;
}

static rt_status reference_impl(const rt_room* rooms, int32_t n, const TraceCfg& t, float* env, float* tail_db) {
    Arena tmp(t.s);
    float* e = env;
    if (!e) RR_TRY(tmp.alloc(&e, (size_t)n * 8 * N_ENV));
    for (int k0 = 0; k0 < n; k0 += t.per_launch) {
        const int k1 = std::min(n, k0 + t.per_launch);
        RR_TRY(batch_hist(rooms, k0, k1, t, t.full_rays, FULL_BOUNCES, DURATION * t.c, TAIL_FS, DURATION, N_ENV, 0,
                          N_ENV, e));
    }
    if (tail_db) RR_LAUNCH(k_hist_tail_db, g1((int64_t)8 * n), 256, 0, t.s, e, n, tail_db);
    RR_CUDA(cudaGetLastError());
    return RT_OK;
}

}  // namespace sur
}  // namespace rr

namespace rr {
namespace sur {

static rt_status predict_impl(const rt_surrogate* m, const float* X, const float* base_db, int32_t n, float* pred_db,
                              cudaStream_t s) {
    Arena tmp(s);
    float *xn, *Y;
    const int nn = (int)m->nets.size();
    RR_TRY(tmp.alloc(&xn, (size_t)n * N_IN));
    RR_TRY(tmp.alloc(&Y, (size_t)nn * n * N_OUT));
    RR_LAUNCH(k_norm_x, g1((int64_t)n * N_IN), 256, 0, s, X, (int64_t)n, m->stats + ST_XM, m->stats + ST_XS, xn);
    for (int k = 0; k < nn; k++) RR_TRY(rt_mlp_forward(m->nets[k], xn, n, Y + (int64_t)k * n * N_OUT, s));
    RR_LAUNCH(k_predict_db, g1((int64_t)8 * n, 128), 128, 0, s, Y, nn, (int64_t)n, m->stats + ST_YM,
              m->stats + ST_YS, base_db, m->residual, pred_db);
    RR_CUDA(cudaGetLastError());
    return RT_OK;
}

// gaps (device [n][2]) and the range verdicts (device [n])
static rt_status gaps_impl(const rt_surrogate* m, const float* desc, const float* X, const float* pred_db,
                           const float* prior_db, int32_t n, float* gaps, int32_t* in_range, cudaStream_t s) {
    RR_LAUNCH(k_gate, g1(n, 64), 64, 0, s, desc, X, pred_db, prior_db, n, m->stats + ST_LO, m->stats + ST_HI, gaps,
              in_range);
    RR_CUDA(cudaGetLastError());
    return RT_OK;
}

static rt_status gate_impl(const rt_surrogate* m, const float* desc, const float* X, const float* pred_db,
                           const float* prior_db, int32_t n, int32_t* pass, float* gaps_host, cudaStream_t s) {
    Arena tmp(s);
    float* gaps;
    int32_t* inr;
    RR_TRY(tmp.alloc(&gaps, (size_t)2 * n));
    RR_TRY(tmp.alloc(&inr, (size_t)n));
    RR_TRY(gaps_impl(m, desc, X, pred_db, prior_db, n, gaps, inr, s));
    std::vector<float> hg((size_t)2 * n);
    std::vector<int32_t> hr((size_t)n);
    RR_CUDA(cudaMemcpyAsync(hg.data(), gaps, sizeof(float) * 2 * n, cudaMemcpyDeviceToHost, s));
    RR_CUDA(cudaMemcpyAsync(hr.data(), inr, sizeof(int32_t) * n, cudaMemcpyDeviceToHost, s));
    RR_CUDA(cudaStreamSynchronize(s));
    for (int k = 0; k < n; k++) {
        if (pass) pass[k] = hr[k] && hg[2 * k] <= m->join_db && hg[2 * k + 1] <= m->probe_db;
        if (gaps_host) gaps_host[2 * k] = hg[2 * k], gaps_host[2 * k + 1] = hg[2 * k + 1];
    }
    return RT_OK;
}

// 99th percentile with linear interpolation between order statistics, over
// the finite values
static float percentile99(std::vector<float> v) {
    v.erase(std::remove_if(v.begin(), v.end(), [](float x) { return !std::isfinite(x); }), v.end());
    if (v.empty()) return INFINITY;
    std::sort(v.begin(), v.end());
    const double pos = 0.99 * (double)(v.size() - 1);
    const size_t i = (size_t)pos;
    const double f = pos - (double)i;
    return (float)(i + 1 < v.size() ? v[i] + f * (v[i + 1] - v[i]) : v[i]);
}

static rt_status train_impl(const float* X, const float* tail_db, const float* desc, const float* base_db,
                            const float* prior_db, int32_t n, const rt_surrogate_train_params* p, rt_surrogate** out) {
    const int n_nets = p->n_nets > 0 ? p->n_nets : 4;
    const int steps = p->steps > 0 ? p->steps : 6000;
    const int batch = p->batch > 0 ? p->batch : 1024;
    const float lr = p->lr > 0 ? p->lr : 1e-3f;
    const float wd = p->weight_decay < 0 ? 0.f : (p->weight_decay > 0 ? p->weight_decay : 1e-4f);
    const float noise = p->input_noise < 0 ? 0.f : (p->input_noise > 0 ? p->input_noise : 0.1f);
    const float val_frac = p->val_frac > 0 ? p->val_frac : 0.05f;
    const int log_every = p->log_every > 0 ? p->log_every : 250;
    cudaStream_t s = (cudaStream_t)p->stream;
    if (n_nets > 64 || batch > 65536 || !(val_frac < 0.5f)) {
        set_error("rt_surrogate_train: n_nets <= 64, batch <= 65536, val_frac < 0.5");
        return RT_ERR_INVALID_ARG;
    }
    // rooms held out for validation: a seeded permutation
    std::vector<int32_t> perm((size_t)n);
    std::iota(perm.begin(), perm.end(), 0);
    std::mt19937_64 rng(p->seed);
    std::shuffle(perm.begin(), perm.end(), rng);
    const int n_val = std::max(1, (int)(val_frac * (float)n));
    const int n_tr = n - n_val;
    std::vector<int32_t> val(perm.begin(), perm.begin() + n_val), tr(perm.begin() + n_val, perm.end());

    rt_surrogate* m = new rt_surrogate();
    struct Guard {
        rt_surrogate*& p;
        ~Guard() { delete p; }
    } guard{m};
    m->stream = s;
    Arena keep(s), tmp(s);
    RR_TRY(keep.alloc(&m->stats, (size_t)ST_N));
    float *Y, *xv, *yv, *yp, *xb, *yb;
    int32_t *d_tr, *d_val;
    double* part;
    const int64_t nv_out = (int64_t)n_val * N_OUT;
    RR_TRY(tmp.alloc(&Y, (size_t)n * N_OUT_RAW));
    RR_TRY(tmp.alloc(&xv, (size_t)n_val * N_IN));
    RR_TRY(tmp.alloc(&yv, (size_t)nv_out));
    RR_TRY(tmp.alloc(&yp, (size_t)nv_out));
    RR_TRY(tmp.alloc(&xb, (size_t)batch * N_IN));
    RR_TRY(tmp.alloc(&yb, (size_t)batch * N_OUT));
    RR_TRY(tmp.alloc(&d_tr, (size_t)n_tr));
    RR_TRY(tmp.alloc(&d_val, (size_t)n_val));
    RR_TRY(tmp.alloc(&part, (size_t)g1(nv_out)));
    RR_CUDA(cudaMemcpyAsync(d_tr, tr.data(), sizeof(int32_t) * n_tr, cudaMemcpyHostToDevice, s));
    RR_CUDA(cudaMemcpyAsync(d_val, val.data(), sizeof(int32_t) * n_val, cudaMemcpyHostToDevice, s));
    RR_LAUNCH(k_residual_targets, g1((int64_t)8 * n, 128), 128, 0, s, tail_db, base_db, (int64_t)n, 1, Y);
    float* st = m->stats;
    RR_LAUNCH(k_col_stats, g1(N_FEAT, 128), 128, 0, s, X, N_FEAT, d_tr, n_tr, 0, st + ST_XM, st + ST_XS);
    RR_LAUNCH(k_col_stats, g1(N_OUT_RAW, 128), 128, 0, s, Y, N_OUT_RAW, d_tr, n_tr, 1, st + ST_YM, st + ST_YS);
    RR_LAUNCH(k_desc_range, 1, 64, 0, s, desc, d_tr, n_tr, st + ST_LO, st + ST_HI);
    RR_LAUNCH(k_norm_rows, g1((int64_t)n_val * N_IN), 256, 0, s, X, N_FEAT, N_IN, d_val, n_val, st + ST_XM,
              st + ST_XS, xv);
    RR_LAUNCH(k_norm_rows, g1(nv_out), 256, 0, s, Y, N_OUT_RAW, N_OUT, d_val, n_val, st + ST_YM, st + ST_YS, yv);
    RR_CUDA(cudaGetLastError());
    std::vector<double> hpart(g1(nv_out));
    for (int k = 0; k < n_nets; k++) {
        rt_mlp* net = nullptr;
        RR_TRY(rt_mlp_create(N_IN, N_HIDDEN, N_OUT, p->seed + (uint64_t)k, s, &net));
        m->nets.push_back(net);
        RR_TRY(rt_mlp_set_weight_decay(net, wd));
        int64_t n_params = 0;
        RR_TRY(rt_mlp_info(net, nullptr, nullptr, nullptr, &n_params, nullptr));
        std::vector<float> best_w((size_t)n_params);
        double best = INFINITY;
        bool have_best = false;
        for (int step = 0; step < steps; step++) {
            const uint64_t key = mix64(p->seed * 0x100000001B3ULL + (uint64_t)k * 0x9E3779B9ULL + (uint64_t)step);
            RR_LAUNCH(k_batch, g1((int64_t)batch * (N_IN + N_OUT)), 256, 0, s, X, Y, d_tr, n_tr, st + ST_XM,
                      st + ST_XS, st + ST_YM, st + ST_YS, batch, key, noise, xb, yb);
            const double lr_t = lr * 0.5 * (1.0 + std::cos(3.14159265358979323846 * step / steps));
            RR_TRY(rt_mlp_train_step(net, xb, yb, batch, (float)std::max(lr_t, 1e-6), nullptr, s));
            if ((step + 1) % log_every == 0 || step == steps - 1) {
                RR_TRY(rt_mlp_forward(net, xv, n_val, yp, s));
                RR_LAUNCH(k_sq_err, g1(nv_out), 256, 0, s, yp, yv, (int64_t)n_val, part);
                RR_CUDA(cudaMemcpyAsync(hpart.data(), part, sizeof(double) * hpart.size(), cudaMemcpyDeviceToHost, s));
                RR_CUDA(cudaStreamSynchronize(s));
                double acc = 0.0;
                for (double x : hpart) acc += x;
                const double vloss = acc / ((double)n_val * N_OUT_RAW);
                m->history.insert(m->history.end(), {(float)k, (float)(step + 1), (float)vloss});
                if (vloss < best) {
                    best = vloss;
                    have_best = true;
                    RR_TRY(rt_mlp_copy(net, 0, best_w.data(), 0, s));
                }
            }
        }
        if (have_best) RR_TRY(rt_mlp_copy(net, 0, best_w.data(), 1, s));
    }
    // gate tolerances: 99th percentiles of the gaps on up to 4096 validation
    // rooms (never trained on, so their gaps are those of new rooms)
    m->join_db = m->probe_db = INFINITY;
    const int n_g = std::min(n_val, 4096);
    std::vector<int32_t> pick(val);
    std::shuffle(pick.begin(), pick.end(), rng);
    pick.resize((size_t)n_g);
    int32_t* d_pick;
    float *gX, *gd, *gb, *gp, *pred;
    RR_TRY(tmp.alloc(&d_pick, (size_t)n_g));
    RR_TRY(tmp.alloc(&gX, (size_t)n_g * N_FEAT));
    RR_TRY(tmp.alloc(&gd, (size_t)n_g * N_DESC));
    RR_TRY(tmp.alloc(&gb, (size_t)n_g * N_OUT_RAW));
    RR_TRY(tmp.alloc(&gp, (size_t)n_g * N_OUT_RAW));
    RR_TRY(tmp.alloc(&pred, (size_t)n_g * N_OUT_RAW));
    RR_CUDA(cudaMemcpyAsync(d_pick, pick.data(), sizeof(int32_t) * n_g, cudaMemcpyHostToDevice, s));
    RR_LAUNCH(k_gather_rows, g1((int64_t)n_g * N_FEAT), 256, 0, s, X, N_FEAT, d_pick, n_g, gX);
    RR_LAUNCH(k_gather_rows, g1((int64_t)n_g * N_DESC), 256, 0, s, desc, N_DESC, d_pick, n_g, gd);
    RR_LAUNCH(k_gather_rows, g1((int64_t)n_g * N_OUT_RAW), 256, 0, s, base_db, N_OUT_RAW, d_pick, n_g, gb);
    RR_LAUNCH(k_gather_rows, g1((int64_t)n_g * N_OUT_RAW), 256, 0, s, prior_db, N_OUT_RAW, d_pick, n_g, gp);
    RR_TRY(predict_impl(m, gX, gb, n_g, pred, s));
    std::vector<float> gaps((size_t)2 * n_g);
    RR_TRY(gate_impl(m, gd, gX, pred, gp, n_g, nullptr, gaps.data(), s));
    std::vector<float> jg((size_t)n_g), pg((size_t)n_g);
    for (int k = 0; k < n_g; k++) jg[k] = gaps[2 * k], pg[k] = gaps[2 * k + 1];
    m->join_db = std::max(3.0f, percentile99(jg));
    m->probe_db = std::max(3.0f, percentile99(pg));
    m->owned = keep.release();
    *out = m;
    m = nullptr;
    return RT_OK;
}

}  // namespace sur
}  // namespace rr

// ---------------------------------------------------------------------------
// serialisation: header, statistics, history, then per network its weight
// matrices in BF16 (what the GEMMs read) and its biases in FP32
// ---------------------------------------------------------------------------
namespace rr {
namespace sur {

struct SaveHeader {
    char magic[8];
    int32_t n_nets, n_in, n_hidden, n_out, residual, n_history;
    float join_db, probe_db;
    int64_t n_params;
    int64_t off[6];
};
static const char SAVE_MAGIC[8] = {'R', 'T', 'S', 'U', 'R', '0', '1', 0};

static inline uint16_t f32_to_bf16_rn(float x) {  // round to nearest even (finite inputs)
    uint32_t u;
    memcpy(&u, &x, 4);
    u += 0x7FFFu + ((u >> 16) & 1u);
    return (uint16_t)(u >> 16);
}
static inline float bf16_to_f32(uint16_t h) {
    const uint32_t u = (uint32_t)h << 16;
    float x;
    memcpy(&x, &u, 4);
    return x;
}

// element counts of the six parameter blocks (W1, b1, W2, b2, W3, b3)
static void block_sizes(int64_t* sz) {
    sz[0] = (int64_t)N_HIDDEN * N_IN, sz[1] = N_HIDDEN, sz[2] = (int64_t)N_HIDDEN * N_HIDDEN, sz[3] = N_HIDDEN;
    sz[4] = (int64_t)N_OUT * N_HIDDEN, sz[5] = N_OUT;
}

static size_t save_bytes(const rt_surrogate* m) {
    int64_t sz[6];
    block_sizes(sz);
    const size_t per_net = 2 * (size_t)(sz[0] + sz[2] + sz[4]) + 4 * (size_t)(sz[1] + sz[3] + sz[5]);
    return sizeof(SaveHeader) + 4 * (size_t)ST_N + 4 * m->history.size() + m->nets.size() * per_net;
}

static rt_status save_impl(const rt_surrogate* m, void* buf, size_t cap, size_t* bytes) {
    const size_t need = save_bytes(m);
    if (bytes) *bytes = need;
    if (!buf) return RT_OK;
    if (cap < need) {
        set_error("rt_surrogate_save: buffer of %zu bytes, need %zu", cap, need);
        return RT_ERR_INVALID_ARG;
    }
    unsigned char* o = (unsigned char*)buf;
    SaveHeader h{};
    memcpy(h.magic, SAVE_MAGIC, 8);
    h.n_nets = (int32_t)m->nets.size(), h.n_in = N_IN, h.n_hidden = N_HIDDEN, h.n_out = N_OUT;
    h.residual = m->residual, h.n_history = (int32_t)(m->history.size() / 3);
    h.join_db = m->join_db, h.probe_db = m->probe_db;
    RR_TRY(rt_mlp_info(m->nets[0], nullptr, nullptr, nullptr, &h.n_params, h.off));
    memcpy(o, &h, sizeof h);
    o += sizeof h;
    RR_CUDA(cudaMemcpy(o, m->stats, 4 * (size_t)ST_N, cudaMemcpyDeviceToHost));
    o += 4 * (size_t)ST_N;
    memcpy(o, m->history.data(), 4 * m->history.size());
    o += 4 * m->history.size();
    int64_t sz[6];
    block_sizes(sz);
    std::vector<float> w((size_t)h.n_params);
    for (rt_mlp* net : m->nets) {
        RR_TRY(rt_mlp_copy(net, 0, w.data(), 0, m->stream));
        for (int b = 0; b < 6; b++) {
            const float* src = w.data() + h.off[b];
            if (b % 2 == 0) {
                for (int64_t i = 0; i < sz[b]; i++) {
                    const uint16_t v = f32_to_bf16_rn(src[i]);
                    memcpy(o + 2 * i, &v, 2);
                }
                o += 2 * sz[b];
            } else {
                memcpy(o, src, 4 * (size_t)sz[b]);
                o += 4 * sz[b];
            }
        }
    }
    return RT_OK;
}

static rt_status load_impl(const void* buf, size_t bytes, cudaStream_t s, rt_surrogate** out) {
    SaveHeader h;
    if (!buf || bytes < sizeof h) {
        set_error("rt_surrogate_load: buffer too small");
        return RT_ERR_INVALID_ARG;
    }
    memcpy(&h, buf, sizeof h);
    if (memcmp(h.magic, SAVE_MAGIC, 8) != 0 || h.n_in != N_IN || h.n_hidden != N_HIDDEN || h.n_out != N_OUT ||
        h.n_nets < 1 || h.n_nets > 64 || h.n_history < 0) {
        set_error("rt_surrogate_load: not a surrogate model of this library's layout");
        return RT_ERR_INVALID_ARG;
    }
    rt_surrogate* m = new rt_surrogate();
    struct Guard {
        rt_surrogate*& p;
        ~Guard() { delete p; }
    } guard{m};
    m->stream = s;
    m->residual = h.residual, m->join_db = h.join_db, m->probe_db = h.probe_db;
    m->history.resize((size_t)3 * h.n_history);
    const size_t need = save_bytes(m);  // header, statistics and history (no network yet)
    int64_t sz[6];
    block_sizes(sz);
    const size_t per_net = 2 * (size_t)(sz[0] + sz[2] + sz[4]) + 4 * (size_t)(sz[1] + sz[3] + sz[5]);
    if (bytes != need + (size_t)h.n_nets * per_net) {
        set_error("rt_surrogate_load: %zu bytes, the header describes %zu", bytes, need + h.n_nets * per_net);
        return RT_ERR_INVALID_ARG;
    }
    const unsigned char* in = (const unsigned char*)buf + sizeof h;
    Arena keep(s);
    RR_TRY(keep.alloc(&m->stats, (size_t)ST_N));
    RR_CUDA(cudaMemcpy(m->stats, in, 4 * (size_t)ST_N, cudaMemcpyHostToDevice));
    in += 4 * (size_t)ST_N;
    memcpy(m->history.data(), in, 4 * m->history.size());
    in += 4 * m->history.size();
    for (int k = 0; k < h.n_nets; k++) {
        rt_mlp* net = nullptr;
        RR_TRY(rt_mlp_create(N_IN, N_HIDDEN, N_OUT, 0, s, &net));
        m->nets.push_back(net);
        int64_t n_params = 0, off[6];
        RR_TRY(rt_mlp_info(net, nullptr, nullptr, nullptr, &n_params, off));
        std::vector<float> w((size_t)n_params, 0.f);
        for (int b = 0; b < 6; b++) {
            float* dst = w.data() + off[b];
            if (b % 2 == 0) {
                for (int64_t i = 0; i < sz[b]; i++) {
                    uint16_t v;
                    memcpy(&v, in + 2 * i, 2);
                    dst[i] = bf16_to_f32(v);
                }
                in += 2 * sz[b];
            } else {
                memcpy(dst, in, 4 * (size_t)sz[b]);
                in += 4 * sz[b];
            }
        }
        RR_TRY(rt_mlp_copy(net, 0, w.data(), 1, s));
    }
    m->owned = keep.release();
    *out = m;
    m = nullptr;
    return RT_OK;
}

}  // namespace sur
}  // namespace rr

// ---------------------------------------------------------------------------
// the surrogate-tail response
// ---------------------------------------------------------------------------
namespace rr {
namespace sur {

static rt_status rir_surrogate_impl(const rt_room* rooms, const double* volume, int32_t n, const rt_surrogate* m,
                                    const TraceCfg& t, rt_response** out, int32_t* used_fallback) {
    cudaStream_t s = t.s;
    Arena tmp(s), keep(s);
    float *desc, *early, *probe, *prior_db, *base_db, *X, *pred, *env;
    RR_TRY(tmp.alloc(&desc, (size_t)n * N_DESC));
    RR_TRY(tmp.alloc(&early, (size_t)n * 8 * N_EARLY));
    RR_TRY(tmp.alloc(&probe, (size_t)n * 8 * N_TAIL));
    RR_TRY(tmp.alloc(&prior_db, (size_t)n * 8 * N_TAIL));
    RR_TRY(tmp.alloc(&base_db, (size_t)n * 8 * N_TAIL));
    RR_TRY(tmp.alloc(&X, (size_t)n * N_FEAT));
    RR_TRY(tmp.alloc(&pred, (size_t)n * 8 * N_TAIL));
    RR_TRY(keep.alloc(&env, (size_t)n * 8 * N_ENV));
    RR_TRY(inputs_impl(rooms, volume, n, t, desc, early, probe, prior_db, base_db, X));
    RR_TRY(predict_impl(m, X, base_db, n, pred, s));
    std::vector<int32_t> pass((size_t)n);
    RR_TRY(gate_impl(m, desc, X, pred, prior_db, n, pass.data(), nullptr, s));
    RR_LAUNCH(k_envelope, g1((int64_t)8 * n), 256, 0, s, early, pred, 1, n, env);
    RR_CUDA(cudaGetLastError());
    // rooms failing the gate: the method itself, traced in full
    std::vector<rt_room> fb;
    std::vector<int> fb_idx;
    for (int k = 0; k < n; k++)
        if (!pass[k]) fb.push_back(rooms[k]), fb_idx.push_back(k);
    if (!fb.empty()) {
        float* fenv;
        RR_TRY(tmp.alloc(&fenv, fb.size() * 8 * N_ENV));
        RR_TRY(reference_impl(fb.data(), (int32_t)fb.size(), t, fenv, nullptr));
        for (size_t j = 0; j < fb.size(); j++)
            RR_CUDA(cudaMemcpyAsync(env + (size_t)fb_idx[j] * 8 * N_ENV, fenv + j * 8 * N_ENV,
                                    sizeof(float) * 8 * N_ENV, cudaMemcpyDeviceToDevice, s));
    }
    RR_CUDA(cudaStreamSynchronize(s));
    if (used_fallback)
        for (int k = 0; k < n; k++) used_fallback[k] = pass[k] ? 0 : 1;
    rt_response* r = new rt_response();
    r->stream = s;
    r->v.n_rcv = n;
    r->v.n_bins = N_ENV;
    r->v.fs = TAIL_FS;
    r->v.data = env;
    r->owned = keep.release();
    *out = r;
    return RT_OK;
}

}  // namespace sur
}  // namespace rr

// ---------------------------------------------------------------------------
// C ABI
// ---------------------------------------------------------------------------
using namespace rr::sur;

extern "C" rt_status rt_surrogate_inputs(const rt_room* rooms, const double* volume, int32_t n,
                                         const rt_surrogate_trace_params* p, float* desc, float* early, float* probe,
                                         float* prior_db, float* base_db, float* X) {
    rr::NvtxRange nvtx_range("rt_surrogate_inputs");
    rr::clear_error();
    TraceCfg t;
    RR_TRY(trace_cfg(p, t));
    if (!volume) {
        rr::set_error("rt_surrogate_inputs: the room volumes are required");
        return RT_ERR_INVALID_ARG;
    }
    RR_TRY(check_rooms(rooms, n, volume));
    return inputs_impl(rooms, volume, n, t, desc, early, probe, prior_db, base_db, X);
}

extern "C" rt_status rt_surrogate_reference(const rt_room* rooms, int32_t n, const rt_surrogate_trace_params* p,
                                            float* env, float* tail_db) {
    rr::NvtxRange nvtx_range("rt_surrogate_reference");
    rr::clear_error();
    TraceCfg t;
    RR_TRY(trace_cfg(p, t));
    RR_TRY(check_rooms(rooms, n, nullptr));
    return reference_impl(rooms, n, t, env, tail_db);
}

extern "C" rt_status rt_surrogate_train(const float* X, const float* tail_db, const float* desc, const float* base_db,
                                        const float* prior_db, int32_t n, const rt_surrogate_train_params* p,
                                        rt_surrogate** out) {
    rr::NvtxRange nvtx_range("rt_surrogate_train");
    rr::clear_error();
    if (!X || !tail_db || !desc || !base_db || !prior_db || !p || !out || n < 64) {
        rr::set_error("rt_surrogate_train: need device X, tail_db, desc, base_db, prior_db, parameters, n >= 64");
        return RT_ERR_INVALID_ARG;
    }
    *out = nullptr;
    return train_impl(X, tail_db, desc, base_db, prior_db, n, p, out);
}

extern "C" void rt_surrogate_free(rt_surrogate* model) { delete model; }

extern "C" rt_status rt_surrogate_info(const rt_surrogate* m, int32_t* n_nets, float* join_db, float* probe_db,
                                       int32_t* n_history, float* history) {
    if (!m) {
        rr::set_error("rt_surrogate_info: null model");
        return RT_ERR_INVALID_ARG;
    }
    if (n_nets) *n_nets = (int32_t)m->nets.size();
    if (join_db) *join_db = m->join_db;
    if (probe_db) *probe_db = m->probe_db;
    if (n_history) *n_history = (int32_t)(m->history.size() / 3);
    if (history) memcpy(history, m->history.data(), sizeof(float) * m->history.size());
    return RT_OK;
}

extern "C" rt_status rt_surrogate_save(const rt_surrogate* m, void* buf, size_t cap, size_t* bytes) {
    rr::clear_error();
    if (!m || m->nets.empty()) {
        rr::set_error("rt_surrogate_save: null model");
        return RT_ERR_INVALID_ARG;
    }
    return save_impl(m, buf, cap, bytes);
}

extern "C" rt_status rt_surrogate_load(const void* buf, size_t bytes, void* stream, rt_surrogate** out) {
    rr::clear_error();
    if (!out) {
        rr::set_error("rt_surrogate_load: null output");
        return RT_ERR_INVALID_ARG;
    }
    *out = nullptr;
    return load_impl(buf, bytes, (cudaStream_t)stream, out);
}

extern "C" rt_status rt_surrogate_predict(const rt_surrogate* m, const float* X, const float* base_db, int32_t n,
                                          float* pred_db, void* stream) {
    rr::NvtxRange nvtx_range("rt_surrogate_predict");
    rr::clear_error();
    if (!m || !X || !base_db || !pred_db || n < 1) {
        rr::set_error("rt_surrogate_predict: need a model, device X, base_db, pred_db and n >= 1");
        return RT_ERR_INVALID_ARG;
    }
    return predict_impl(m, X, base_db, n, pred_db, (cudaStream_t)stream);
}

extern "C" rt_status rt_surrogate_gate(const rt_surrogate* m, const float* desc, const float* X, const float* pred_db,
                                       const float* prior_db, int32_t n, int32_t* pass, float* gaps, void* stream) {
    rr::NvtxRange nvtx_range("rt_surrogate_gate");
    rr::clear_error();
    if (!m || !desc || !X || !pred_db || !prior_db || n < 1) {
        rr::set_error("rt_surrogate_gate: need a model, device desc, X, pred_db, prior_db and n >= 1");
        return RT_ERR_INVALID_ARG;
    }
    return gate_impl(m, desc, X, pred_db, prior_db, n, pass, gaps, (cudaStream_t)stream);
}

extern "C" rt_status rt_surrogate_envelope(const float* early, const float* tail, int32_t tail_is_db, int32_t n,
                                           float* env, void* stream) {
    rr::NvtxRange nvtx_range("rt_surrogate_envelope");
    rr::clear_error();
    if (!early || !tail || !env || n < 1) {
        rr::set_error("rt_surrogate_envelope: need device early, tail, env and n >= 1");
        return RT_ERR_INVALID_ARG;
    }
    cudaStream_t s = (cudaStream_t)stream;
    RR_LAUNCH(k_envelope, g1((int64_t)8 * n), 256, 0, s, early, tail, tail_is_db ? 1 : 0, n, env);
    RR_CUDA(cudaGetLastError());
    return RT_OK;
}

extern "C" rt_status rt_rir_surrogate(const rt_room* rooms, const double* volume, int32_t n, const rt_surrogate* m,
                                      const rt_surrogate_trace_params* p, rt_response** out, int32_t* used_fallback) {
    rr::NvtxRange nvtx_range("rt_rir_surrogate");
    rr::clear_error();
    if (!m || !out || !volume) {
        rr::set_error("rt_rir_surrogate: need a model, the room volumes and an output");
        return RT_ERR_INVALID_ARG;
    }
    *out = nullptr;
    TraceCfg t;
    RR_TRY(trace_cfg(p, t));
    RR_TRY(check_rooms(rooms, n, volume));
    return rir_surrogate_impl(rooms, volume, n, m, t, out, used_fallback);
}
