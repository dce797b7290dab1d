// rt_prior.cu -- direction-integrated specular tail prior of the learned tail.
//
// A ray of direction d in a room whose walls are grouped by the axis of their
// normal loses energy at R(d) = sum_k |d_k| rate_k + air (1/s).  The energy
// histogram of a measurement sphere averages level * exp(-R t) over the ray
// directions (eq. 19: an image source found by n of N rays carries n / N of
// the source energy times the reflection product).  One block handles one
// (room, band): it stages R_j and the bin-averaging factor of each quadrature
// direction in shared memory, then each thread sums one bin over all
// directions in FP64.
#include "rt_internal.cuh"

namespace rr {

static constexpr int PRIOR_THREADS = 256;
static constexpr int PRIOR_CHUNK = 1024;   // directions staged per pass
static constexpr int PRIOR_MAX_NODES = 256;

// Gauss-Legendre node k of n on (-1, 1) and its weight: Newton's method on the
// three-term Legendre recurrence, started from Tricomi's estimate
// cos(pi (k + 3/4) / (n + 1/2)); at most 100 steps.
__device__ void gl_node(int k, int n, double& x, double& w) {
    double z = cos(3.14159265358979323846 * (k + 0.75) / (n + 0.5));
    double p1 = 1.0, p2 = 0.0, dp = 1.0;
    for (int it = 0; it < 100; it++) {
        p1 = 1.0;
        p2 = 0.0;
        for (int j = 1; j <= n; j++) {
            const double p3 = p2;
            p2 = p1;
            p1 = ((2.0 * j - 1.0) * z * p2 - (j - 1.0) * p3) / j;
        }
        dp = n * (z * p1 - p2) / (z * z - 1.0);
        const double step = p1 / dp;
        z -= step;
        if (fabs(step) < 1e-16) break;
    }
    p1 = 1.0;
    p2 = 0.0;
    for (int j = 1; j <= n; j++) {
        const double p3 = p2;
        p2 = p1;
        p1 = ((2.0 * j - 1.0) * z * p2 - (j - 1.0) * p3) / j;
    }
    dp = n * (z * p1 - p2) / (z * z - 1.0);
    x = z;
    w = 2.0 / ((1.0 - z * z) * dp * dp);
}

// One block per (bin block, band, room).  Directions: theta and phi on the n
// Gauss-Legendre nodes of (0, pi / 2), d = (sin theta cos phi,
// sin theta sin phi, cos theta), weight (pi / 4) w_theta sin theta * w_phi / 2
// with w the weights on (-1, 1): the octant's area element sin theta dtheta
// dphi over its area pi / 2.  Every component of d is smooth in (theta, phi),
// so the rule converges geometrically.
__global__ void __launch_bounds__(PRIOR_THREADS) k_tail_prior(const float* __restrict__ rates,
                                                               const float* __restrict__ air,
                                                               const float* __restrict__ level, int n_nodes,
                                                               float t0, float dt, int n_bins,
                                                               float* __restrict__ out) {
    __shared__ double s_st[PRIOR_MAX_NODES], s_ct[PRIOR_MAX_NODES], s_wt[PRIOR_MAX_NODES];
    __shared__ double s_c[PRIOR_MAX_NODES], s_s[PRIOR_MAX_NODES], s_wp[PRIOR_MAX_NODES];
    __shared__ float s_R[PRIOR_CHUNK];
    __shared__ float s_f[PRIOR_CHUNK];
    const int band = blockIdx.y, room = blockIdx.z;
    const int b = blockIdx.x * PRIOR_THREADS + threadIdx.x;
    for (int k = threadIdx.x; k < n_nodes; k += PRIOR_THREADS) {
        double x, w;
        gl_node(k, n_nodes, x, w);
        const double ang = 0.7853981633974483 * (x + 1.0);   // node of (0, pi / 2)
        s_st[k] = sin(ang);
        s_ct[k] = cos(ang);
        s_wt[k] = 0.7853981633974483 * w * sin(ang);
        s_c[k] = cos(ang);
        s_s[k] = sin(ang);
        s_wp[k] = 0.5 * w;
    }
    __syncthreads();
    const float r0 = rates[(room * 3 + 0) * 8 + band];
    const float r1 = rates[(room * 3 + 1) * 8 + band];
    const float r2 = rates[(room * 3 + 2) * 8 + band];
    const float ra = air[room * 8 + band];
    const float t = t0 + (float)b * dt;
    const int n_dirs = n_nodes * n_nodes;
    double acc = 0.0;
    for (int c0 = 0; c0 < n_dirs; c0 += PRIOR_CHUNK) {
        const int cn = min(PRIOR_CHUNK, n_dirs - c0);
        __syncthreads();
        for (int j = threadIdx.x; j < cn; j += PRIOR_THREADS) {
            const int it = (c0 + j) / n_nodes, ip = (c0 + j) % n_nodes;
            const double st = s_st[it];
            const float R = (float)(st * s_c[ip]) * r0 + (float)(st * s_s[ip]) * r1 + (float)s_ct[it] * r2 + ra;
            const float x = dt * R;
            // weight times the mean of exp(-R s) over s in [0, dt)
            const float avg = x < 1e-4f ? 1.0f - 0.5f * x : -expm1f(-x) / x;
            s_R[j] = R;
            s_f[j] = (float)(s_wt[it] * s_wp[ip]) * avg;
        }
        __syncthreads();
        if (b < n_bins)
            for (int j = 0; j < cn; j++) acc += (double)(s_f[j] * expf(-t * s_R[j]));
    }
    if (b < n_bins) out[((int64_t)room * 8 + band) * n_bins + b] = (float)(level[room] * acc);
}

}  // namespace rr

extern "C" rt_status rt_tail_prior(const float* rates, const float* air, const float* level, int32_t n,
                                   int32_t n_nodes, float t0, float dt, int32_t n_bins, float* out, void* stream) {
    rr::NvtxRange nvtx_range("rt_tail_prior");
    rr::clear_error();
    if (!rates || !air || !level || !out || n <= 0 || n_nodes <= 0 || n_nodes > rr::PRIOR_MAX_NODES ||
        n_bins <= 0 || !(dt > 0.0f) || !(t0 >= 0.0f) || n > 65535) {
        rr::set_error("rt_tail_prior: need device arrays, 0 < n <= 65535, 0 < n_nodes <= 256, n_bins > 0, "
                      "dt > 0, t0 >= 0");
        return RT_ERR_INVALID_ARG;
    }
    cudaStream_t s = (cudaStream_t)stream;
    dim3 grid((n_bins + rr::PRIOR_THREADS - 1) / rr::PRIOR_THREADS, 8, n);
    RR_LAUNCH(rr::k_tail_prior, grid, rr::PRIOR_THREADS, 0, s, rates, air, level, n_nodes, t0, dt, n_bins, out);
    RR_CUDA(cudaGetLastError());
    return RT_OK;
}
