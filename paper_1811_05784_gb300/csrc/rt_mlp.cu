// rt_mlp.cu -- the learned late-reverberation tail: a 3-layer MLP trained and
// run on the GPU with hand-written BF16 tensor-core kernels.
//
// Network: x[B][n_in] -> Linear(n_in, H) -> GELU -> Linear(H, H) -> GELU ->
// Linear(H, n_out).  Weights are kept as FP32 master copies (AdamW) and as
// BF16 copies (row-major [out][in] and transposed) that the GEMMs read;
// activations entering a GEMM are BF16, accumulation is FP32.
//
// Every product runs on the 5th-generation tensor cores (rt_tc_gemm.cuh:
// tcgen05.mma from swizzled shared-memory tiles into a TMEM accumulator):
// C[M][N] = A[M][K] . B[N][K]^T with both operands K-contiguous.  Backward
// products that need the other orientation read transposed BF16 copies made
// by k_transpose.
//   forward    Z = X W^T + b             (A = X, B = W)
//   dX         dX = dZ W                 (A = dZ, B = W^T)
//   dW         dW = dZ^T X               (A = dZ^T, B = X^T, K = batch)
// The paper has no learned component; the network is the learned tail of the
// surrogate mode (room descriptors and short traces in, late decay out).
#include "rt_internal.cuh"
#include "rt_tc_gemm.cuh"
#include "rt_tc_tma.cuh"

#include <cudaTypedefs.h>
#include <cuda_bf16.h>

#include <cmath>
#include <random>

namespace rr {

typedef __nv_bfloat16 bf16;

using tc::EPI_BIAS_F32;
using tc::EPI_BIAS_GELU;
using tc::EPI_F32;

__device__ __forceinline__ float gelu_grad(float x) {
    // d/dx [x Phi(x)] = Phi(x) + x phi(x)
    const float cdf = 0.5f * (1.0f + erff(x * 0.70710678118654752f));
    const float pdf = 0.3989422804014327f * expf(-0.5f * x * x);
    return cdf + x * pdf;
}

// out[C][R_pad] = in[R][C]^T, zero in columns R .. R_pad-1
__global__ void k_transpose(const bf16* __restrict__ in, int R, int C, int R_pad, bf16* __restrict__ out) {
    __shared__ bf16 tile[32][33];
    const int r0 = blockIdx.y * 32, c0 = blockIdx.x * 32;
    for (int k = threadIdx.y; k < 32; k += blockDim.y) {
        const int r = r0 + k, c = c0 + threadIdx.x;
        tile[k][threadIdx.x] = (r < R && c < C) ? in[(size_t)r * C + c] : __float2bfloat16_rn(0.f);
    }
    __syncthreads();
    for (int k = threadIdx.y; k < 32; k += blockDim.y) {
        const int c = c0 + k, r = r0 + threadIdx.x;
        if (c < C && r < R_pad) out[(size_t)c * R_pad + r] = tile[threadIdx.x][k];
    }
}

__global__ void k_f32_to_bf16(const float* __restrict__ in, int64_t n, bf16* __restrict__ out) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = __float2bfloat16_rn(in[i]);
}

// d = 2 (y - t) / (rows * cols) for rows < B (MSE gradient), loss partials per block
__global__ void k_mse(const float* __restrict__ y, const float* __restrict__ tg, int64_t n, float scale,
                      bf16* __restrict__ dy, float* __restrict__ loss_part) {
    __shared__ float red[256];
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    float e = 0.f;
    if (i < n) {
        const float d = y[i] - tg[i];
        e = d * d;
        dy[i] = __float2bfloat16_rn(2.0f * d * scale);
    }
    red[threadIdx.x] = e;
    __syncthreads();
    for (int s = 128; s > 0; s >>= 1) {
        if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) loss_part[blockIdx.x] = red[0];
}

// dZ = dH * gelu'(pre) -> bf16
__global__ void k_gelu_back(const float* __restrict__ dh, const float* __restrict__ pre, int64_t n,
                            bf16* __restrict__ dz) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) dz[i] = __float2bfloat16_rn(dh[i] * gelu_grad(pre[i]));
}

// db[c] = sum_r d[r][c]
__global__ void k_colsum(const bf16* __restrict__ d, int R, int C, float* __restrict__ db) {
    int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= C) return;
    float s = 0.f;
    for (int r = 0; r < R; r++) s += __bfloat162float(d[(size_t)r * C + c]);
    db[c] = s;
}

// Adam on FP32 masters (bias-corrected), then the BF16 copy
// Adam with decoupled weight decay (AdamW): w -= lr (m_hat / (sqrt(v_hat) + eps) + wd w)
__global__ void k_adam(float* __restrict__ w, const float* __restrict__ g, float* __restrict__ m, float* __restrict__ v,
                       int64_t n, float lr, float b1, float b2, float eps, float c1, float c2, float wd,
                       bf16* __restrict__ wb) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    const float wi = w[i] - lr * ((mi * c1) / (sqrtf(vi * c2) + eps) + wd * w[i]);
    w[i] = wi;
    if (wb) wb[i] = __float2bfloat16_rn(wi);
}

}  // namespace rr

// ---------------------------------------------------------------------------
// the network object
// ---------------------------------------------------------------------------
struct rt_mlp {
    int n_in = 0, n_h = 0, n_out = 0;
    // FP32 parameter block: W1 [H][n_in], b1 [H], W2 [H][H], b2 [H], W3 [n_out][H], b3 [n_out]
    int64_t off[6] = {};
    int64_t n_params = 0;
    float *w = nullptr, *g = nullptr, *m = nullptr, *v = nullptr;
    rr::bf16 *wb = nullptr;   // BF16 copies of the weight matrices (same offsets, biases unused)
    rr::bf16 *wt[3] = {};     // transposed BF16 weights: W1^T [n_in][H], W2^T [H][H], W3^T [H][n_out]
    int64_t step = 0;
    float weight_decay = 0.f;
    // activation scratch sized for cap_b rows
    int cap_b = 0;
    std::vector<void*> act;
    rr::bf16 *xb = nullptr, *h1 = nullptr, *h2 = nullptr;  // BF16 activations
    float *z1 = nullptr, *z2 = nullptr, *y = nullptr;        // pre-activations, output
    float *dh = nullptr;                                      // FP32 backward scratch
    rr::bf16 *dz = nullptr, *dzt = nullptr, *at = nullptr;   // backward BF16 scratch
    float* loss_part = nullptr;
    unsigned int* tc_status = nullptr;   // bit 0: a tensor-core GEMM gave up waiting for its MMAs
    float* splitk = nullptr;             // partial sums of the weight-gradient products cut along the batch
    size_t splitk_floats = 0;
    std::vector<void*> owned;
    cudaStream_t stream = nullptr;
};

namespace rr {

static unsigned gridn(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

static rt_status mlp_reserve(rt_mlp* net, int B, cudaStream_t s) {
    if (B <= net->cap_b) return RT_OK;
    for (void* p : net->act) dev_free(p, s);
    net->act.clear();
    Arena ar(s);
    const int Bp = (B + 31) / 32 * 32;
    const int W = std::max(std::max(net->n_in, net->n_h), net->n_out);
    RR_TRY(ar.alloc(&net->xb, (int64_t)Bp * net->n_in));
    RR_TRY(ar.alloc(&net->h1, (int64_t)Bp * net->n_h));
    RR_TRY(ar.alloc(&net->h2, (int64_t)Bp * net->n_h));
    RR_TRY(ar.alloc(&net->z1, (int64_t)Bp * net->n_h));
    RR_TRY(ar.alloc(&net->z2, (int64_t)Bp * net->n_h));
    RR_TRY(ar.alloc(&net->y, (int64_t)Bp * net->n_out));
    RR_TRY(ar.alloc(&net->dh, (int64_t)Bp * W));
    RR_TRY(ar.alloc(&net->dz, (int64_t)Bp * W));
    RR_TRY(ar.alloc(&net->dzt, (int64_t)Bp * W));
    RR_TRY(ar.alloc(&net->at, (int64_t)Bp * W));
    RR_TRY(ar.alloc(&net->loss_part, (int64_t)gridn((int64_t)Bp * net->n_out, 256)));
    // up to 8 partial sums of the largest weight gradient
    const int64_t wmax = std::max(std::max((int64_t)net->n_out * net->n_h, (int64_t)net->n_h * net->n_h),
                                  (int64_t)net->n_h * net->n_in);
    net->splitk_floats = (size_t)(8 * wmax);
    RR_TRY(ar.alloc(&net->splitk, net->splitk_floats));
    net->act = ar.release();
    net->cap_b = B;
    return RT_OK;
}

// TMA descriptor of a row-major BF16 matrix [rows][K] read in box_rows x
// 64-column boxes with the 128-byte swizzle (the layout the MMA descriptors
// expect); rows and columns past the matrix read as zero.  cuTensorMapEncodeTiled
// is taken from the driver through the runtime's entry-point query.
static rt_status tensor_map(CUtensorMap* map, const bf16* base, int rows, int K, int box_rows) {
    static PFN_cuTensorMapEncodeTiled_v12000 encode = nullptr;
    if (!encode) {
        void* fn = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) !=
                cudaSuccess ||
            q != cudaDriverEntryPointSuccess || !fn) {
            cudaGetLastError();
            set_error("rt_mlp: cuTensorMapEncodeTiled is not available from the driver");
            return RT_ERR_CUDA;
        }
        encode = (PFN_cuTensorMapEncodeTiled_v12000)fn;
    }
    if (((uintptr_t)base & 15u) || K % 8 || rows < 1 || K < 1) {
        set_error("rt_mlp: a GEMM operand needs 16-byte aligned rows (K %% 8 == 0)");
        return RT_ERR_INVALID_ARG;
    }
    const cuuint64_t dims[2] = {(cuuint64_t)K, (cuuint64_t)rows};
    const cuuint64_t strides[1] = {(cuuint64_t)K * sizeof(bf16)};
    const cuuint32_t box[2] = {(cuuint32_t)tma::BK, (cuuint32_t)box_rows};
    const cuuint32_t elem[2] = {1, 1};
    const CUresult r = encode(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, (void*)base, dims, strides, box, elem,
                              CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                              CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) {
        set_error("rt_mlp: cuTensorMapEncodeTiled failed (%d)", (int)r);
        return RT_ERR_CUDA;
    }
    return RT_OK;
}

static int sm_count() {
    static int cached[64] = {};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 148;
    if (!cached[dev] && cudaDeviceGetAttribute(&cached[dev], cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
        cudaGetLastError();
        return 148;
    }
    return cached[dev];
}

template <auto kernel>
static rt_status allow_smem(int bytes) {
    static bool done[64] = {};  // one per kernel and device
    int dev = 0;
    RR_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64 || !done[dev]) {
        RR_CUDA(cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes));
        if (dev >= 0 && dev < 64) done[dev] = true;
    }
    return RT_OK;
}

// C = A B^T through the persistent TMA-fed, warp-specialised tensor-core
// kernel (rt_tc_tma.cuh), one CTA per SM.  With a workspace (ws, ws_floats)
// a product with few output tiles is also cut along K and its partial sums
// added by k_splitk_reduce.  K % 8 == 0 for the TMA (16-byte rows).
template <int EPI>
static rt_status gemm(const bf16* A, const bf16* B, int M, int N, int K, const float* bias, float* Cf, float* Cpre,
                      bf16* Cb, unsigned int* status, cudaStream_t s, float* ws = nullptr, size_t ws_floats = 0) {
    const int sms = sm_count();
    const tma::Shape sh = tma::plan(M, N, K, sms, ws ? ws_floats : 0);
    CUtensorMap ma, mb;
    RR_TRY(tensor_map(&ma, A, M, K, tma::BM));
    RR_TRY(tensor_map(&mb, B, N, K, sh.bn));
    const int grid = std::min(sh.tiles * sh.splits, sms);
    if (sh.splits == 1) {
        RR_TRY(allow_smem<tma::k_gemm_tma<EPI>>(tma::SMEM_BYTES));
        RR_LAUNCH(tma::k_gemm_tma<EPI>, grid, tma::THREADS, tma::SMEM_BYTES, s, ma, mb, sh, bias, Cf, Cpre, Cb,
                  (int64_t)0, status);
    } else {
        const int64_t MN = (int64_t)M * N;
        RR_TRY(allow_smem<tma::k_gemm_tma<EPI_F32>>(tma::SMEM_BYTES));
        RR_LAUNCH(tma::k_gemm_tma<EPI_F32>, grid, tma::THREADS, tma::SMEM_BYTES, s, ma, mb, sh, nullptr, ws, nullptr,
                  nullptr, MN, status);
        RR_LAUNCH(tma::k_splitk_reduce<EPI>, (unsigned)std::min<int64_t>((MN / 4 + 255) / 256 + 1, 4 * sms), 256, 0,
                  s, ws, sh.splits, MN, N, bias, Cf, Cpre, Cb);
    }
    return RT_OK;
}

// the register-staged kernel (rt_tc_gemm.cuh), kept as the measured baseline
// of rt_gemm_bf16
template <int EPI>
static rt_status gemm_staged(const bf16* A, const bf16* B, int M, int N, int K, const float* bias, float* Cf,
                             float* Cpre, bf16* Cb, unsigned int* status, cudaStream_t s) {
    dim3 grid(gridn(N, tc::BN), gridn(M, tc::BM));
    RR_CUDA(cudaFuncSetAttribute(tc::k_gemm_tc<EPI>, cudaFuncAttributeMaxDynamicSharedMemorySize, tc::SMEM_BYTES));
    RR_LAUNCH(tc::k_gemm_tc<EPI>, grid, 128, tc::SMEM_BYTES, s, A, B, M, N, K, bias, Cf, Cpre, Cb, status);
    return RT_OK;
}

static void transpose(const bf16* in, int R, int C, int R_pad, bf16* out, cudaStream_t s) {
    dim3 grid(gridn(C, 32), gridn(R_pad, 32));
    RR_LAUNCH(k_transpose, grid, dim3(32, 8), 0, s, in, R, C, R_pad, out);
}

static void refresh_bf16(rt_mlp* net, cudaStream_t s) {
    const int L_in[3] = {net->n_in, net->n_h, net->n_h}, L_out[3] = {net->n_h, net->n_h, net->n_out};
    for (int l = 0; l < 3; l++) {
        const int64_t o = net->off[2 * l];
        const int64_t n = (int64_t)L_in[l] * L_out[l];
        RR_LAUNCH(k_f32_to_bf16, gridn(n, 256), 256, 0, s, net->w + o, n, net->wb + o);
        transpose(net->wb + o, L_out[l], L_in[l], L_out[l], net->wt[l], s);
    }
}

static rt_status mlp_forward_impl(rt_mlp* net, const float* x, int B, float* y_out, cudaStream_t s) {
    RR_TRY(mlp_reserve(net, B, s));
    RR_LAUNCH(k_f32_to_bf16, gridn((int64_t)B * net->n_in, 256), 256, 0, s, x, (int64_t)B * net->n_in, net->xb);
    RR_TRY(gemm<EPI_BIAS_GELU>(net->xb, net->wb + net->off[0], B, net->n_h, net->n_in, net->w + net->off[1], nullptr, net->z1,
                        net->h1, net->tc_status, s));
    RR_TRY(gemm<EPI_BIAS_GELU>(net->h1, net->wb + net->off[2], B, net->n_h, net->n_h, net->w + net->off[3], nullptr, net->z2,
                        net->h2, net->tc_status, s));
    RR_TRY(gemm<EPI_BIAS_F32>(net->h2, net->wb + net->off[4], B, net->n_out, net->n_h, net->w + net->off[5],
                       y_out ? y_out : net->y, nullptr, nullptr, net->tc_status, s));
    RR_CUDA(cudaGetLastError());
    return RT_OK;
}

// gradients of the mean squared error into net->g; loss partials into net->loss_part
static rt_status mlp_backward_impl(rt_mlp* net, const float* x, const float* target, int B, cudaStream_t s) {
    RR_TRY(mlp_forward_impl(net, x, B, nullptr, s));
    const int Bp = (B + 31) / 32 * 32;
    const int H = net->n_h, NI = net->n_in, NO = net->n_out;
    const int64_t ny = (int64_t)B * NO;
    RR_LAUNCH(k_mse, gridn(ny, 256), 256, 0, s, net->y, target, ny, 1.0f / (float)ny, net->dz, net->loss_part);
    // layer 3: dW3 = dY^T H2, db3 = colsum dY, dH2 = dY W3
    transpose(net->dz, B, NO, Bp, net->dzt, s);
    transpose(net->h2, B, H, Bp, net->at, s);
    RR_TRY(gemm<EPI_F32>(net->dzt, net->at, NO, H, Bp, nullptr, net->g + net->off[4], nullptr, nullptr, net->tc_status, s,
                         net->splitk, net->splitk_floats));
    RR_LAUNCH(k_colsum, gridn(NO, 128), 128, 0, s, net->dz, B, NO, net->g + net->off[5]);
    RR_TRY(gemm<EPI_F32>(net->dz, net->wt[2], B, H, NO, nullptr, net->dh, nullptr, nullptr, net->tc_status, s));
    RR_LAUNCH(k_gelu_back, gridn((int64_t)B * H, 256), 256, 0, s, net->dh, net->z2, (int64_t)B * H, net->dz);
    // layer 2
    transpose(net->dz, B, H, Bp, net->dzt, s);
    transpose(net->h1, B, H, Bp, net->at, s);
    RR_TRY(gemm<EPI_F32>(net->dzt, net->at, H, H, Bp, nullptr, net->g + net->off[2], nullptr, nullptr, net->tc_status, s,
                         net->splitk, net->splitk_floats));
    RR_LAUNCH(k_colsum, gridn(H, 128), 128, 0, s, net->dz, B, H, net->g + net->off[3]);
    RR_TRY(gemm<EPI_F32>(net->dz, net->wt[1], B, H, H, nullptr, net->dh, nullptr, nullptr, net->tc_status, s));
    RR_LAUNCH(k_gelu_back, gridn((int64_t)B * H, 256), 256, 0, s, net->dh, net->z1, (int64_t)B * H, net->dz);
    // layer 1 (no input gradient needed)
    transpose(net->dz, B, H, Bp, net->dzt, s);
    transpose(net->xb, B, NI, Bp, net->at, s);
    RR_TRY(gemm<EPI_F32>(net->dzt, net->at, H, NI, Bp, nullptr, net->g + net->off[0], nullptr, nullptr, net->tc_status, s,
                         net->splitk, net->splitk_floats));
    RR_LAUNCH(k_colsum, gridn(H, 128), 128, 0, s, net->dz, B, H, net->g + net->off[1]);
    RR_CUDA(cudaGetLastError());
    return RT_OK;
}

// after a synchronisation: did a tensor-core GEMM give up waiting?
static rt_status check_tc(rt_mlp* net, unsigned int st) {
    if (st) {
        set_error("rt_mlp: a tensor-core GEMM timed out waiting for its MMAs (results discarded)");
        return RT_ERR_CUDA;
    }
    (void)net;
    return RT_OK;
}

static rt_status read_loss(rt_mlp* net, int B, cudaStream_t s, float* loss) {
    const int64_t ny = (int64_t)B * net->n_out;
    const int nb = (int)gridn(ny, 256);
    std::vector<float> part((size_t)nb);
    unsigned int st = 0;
    RR_CUDA(cudaMemcpyAsync(part.data(), net->loss_part, sizeof(float) * nb, cudaMemcpyDeviceToHost, s));
    RR_CUDA(cudaMemcpyAsync(&st, net->tc_status, sizeof st, cudaMemcpyDeviceToHost, s));
    RR_CUDA(cudaStreamSynchronize(s));
    RR_TRY(check_tc(net, st));
    double acc = 0;
    for (float x : part) acc += x;
    *loss = (float)(acc / (double)ny);
    return RT_OK;
}

static bool dims_ok(int n_in, int n_h, int n_out) {
    return n_in > 0 && n_h > 0 && n_out > 0 && n_in % 32 == 0 && n_h % 32 == 0 && n_out % 32 == 0 &&
           n_in <= 16384 && n_h <= 16384 && n_out <= 16384;
}

}  // namespace rr

extern "C" rt_status rt_mlp_create(int32_t n_in, int32_t n_hidden, int32_t n_out, uint64_t seed, void* stream,
                                   rt_mlp** out) {
    rr::clear_error();
    if (!out || !rr::dims_ok(n_in, n_hidden, n_out)) {
        rr::set_error("rt_mlp_create: sizes must be positive multiples of 32 (<= 16384)");
        return RT_ERR_INVALID_ARG;
    }
    *out = nullptr;
    cudaStream_t s = (cudaStream_t)stream;
    rt_mlp* net = new rt_mlp();
    net->stream = s;
    net->n_in = n_in;
    net->n_h = n_hidden;
    net->n_out = n_out;
    const int64_t sizes[6] = {(int64_t)n_hidden * n_in, n_hidden, (int64_t)n_hidden * n_hidden, n_hidden,
                              (int64_t)n_out * n_hidden, n_out};
    int64_t o = 0;
    for (int k = 0; k < 6; k++) {
        net->off[k] = o;
        o += (sizes[k] + 63) / 64 * 64;  // keep every block 256-byte aligned
    }
    net->n_params = o;
    rr::Arena ar(s);
    rt_status st;
    if ((st = ar.alloc(&net->w, o)) || (st = ar.alloc(&net->g, o)) || (st = ar.alloc(&net->m, o)) ||
        (st = ar.alloc(&net->v, o)) || (st = ar.alloc(&net->wb, o)) ||
        (st = ar.alloc(&net->wt[0], sizes[0])) || (st = ar.alloc(&net->wt[1], sizes[2])) ||
        (st = ar.alloc(&net->wt[2], sizes[4])) || (st = ar.alloc(&net->tc_status, 1))) {
        delete net;
        return st;
    }
    // He-uniform weights from a seeded host generator, zero biases and moments
    std::vector<float> hw((size_t)o, 0.f);
    std::mt19937_64 rng(seed);
    const int fan_in[3] = {n_in, n_hidden, n_hidden};
    for (int l = 0; l < 3; l++) {
        const float a = std::sqrt(6.0f / (float)fan_in[l]);
        std::uniform_real_distribution<float> U(-a, a);
        for (int64_t i = 0; i < sizes[2 * l]; i++) hw[(size_t)(net->off[2 * l] + i)] = U(rng);
    }
    if (cudaMemcpyAsync(net->w, hw.data(), sizeof(float) * o, cudaMemcpyHostToDevice, s) != cudaSuccess ||
        cudaMemsetAsync(net->m, 0, sizeof(float) * o, s) != cudaSuccess ||
        cudaMemsetAsync(net->v, 0, sizeof(float) * o, s) != cudaSuccess ||
        cudaMemsetAsync(net->g, 0, sizeof(float) * o, s) != cudaSuccess ||
        cudaMemsetAsync(net->tc_status, 0, sizeof(unsigned int), s) != cudaSuccess) {
        rr::set_error("rt_mlp_create: initialisation copy failed");
        delete net;
        return RT_ERR_CUDA;
    }
    net->owned = ar.release();
    rr::refresh_bf16(net, s);
    if (cudaStreamSynchronize(s) != cudaSuccess) {
        rr::set_error("rt_mlp_create: %s", cudaGetErrorString(cudaGetLastError()));
        for (void* p : net->owned) rr::dev_free(p, s);
        delete net;
        return RT_ERR_CUDA;
    }
    *out = net;
    return RT_OK;
}

extern "C" void rt_mlp_free(rt_mlp* net) {
    if (!net) return;
    for (void* p : net->act) rr::dev_free(p, net->stream);
    for (void* p : net->owned) rr::dev_free(p, net->stream);
    delete net;
}

extern "C" rt_status rt_mlp_info(const rt_mlp* net, int32_t* n_in, int32_t* n_hidden, int32_t* n_out,
                                 int64_t* n_params, int64_t* offsets6) {
    if (!net) {
        rr::set_error("rt_mlp_info: null network");
        return RT_ERR_INVALID_ARG;
    }
    if (n_in) *n_in = net->n_in;
    if (n_hidden) *n_hidden = net->n_h;
    if (n_out) *n_out = net->n_out;
    if (n_params) *n_params = net->n_params;
    if (offsets6)
        for (int k = 0; k < 6; k++) offsets6[k] = net->off[k];
    return RT_OK;
}

extern "C" rt_status rt_mlp_forward(rt_mlp* net, const float* x, int32_t batch, float* y, void* stream) {
    rr::NvtxRange nvtx_range("rt_mlp_forward");
    rr::clear_error();
    if (!net || !x || !y || batch < 1) {
        rr::set_error("rt_mlp_forward: need a network, device x [batch][n_in], y [batch][n_out], batch >= 1");
        return RT_ERR_INVALID_ARG;
    }
    return rr::mlp_forward_impl(net, x, batch, y, (cudaStream_t)stream);
}

extern "C" rt_status rt_mlp_gradients(rt_mlp* net, const float* x, const float* target, int32_t batch,
                                      float* loss, void* stream) {
    rr::NvtxRange nvtx_range("rt_mlp_gradients");
    rr::clear_error();
    if (!net || !x || !target || batch < 1) {
        rr::set_error("rt_mlp_gradients: need a network, device x, target and batch >= 1");
        return RT_ERR_INVALID_ARG;
    }
    cudaStream_t s = (cudaStream_t)stream;
    RR_TRY(rr::mlp_backward_impl(net, x, target, batch, s));
    if (loss) RR_TRY(rr::read_loss(net, batch, s, loss));
    return RT_OK;
}

extern "C" rt_status rt_mlp_train_step(rt_mlp* net, const float* x, const float* target, int32_t batch, float lr,
                                       float* loss, void* stream) {
    rr::NvtxRange nvtx_range("rt_mlp_train_step");
    rr::clear_error();
    if (!net || !x || !target || batch < 1 || !(lr > 0)) {
        rr::set_error("rt_mlp_train_step: need a network, device x, target, batch >= 1 and lr > 0");
        return RT_ERR_INVALID_ARG;
    }
    cudaStream_t s = (cudaStream_t)stream;
    RR_TRY(rr::mlp_backward_impl(net, x, target, batch, s));
    net->step++;
    const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
    const float c1 = 1.0f / (1.0f - std::pow(b1, (float)net->step));
    const float c2 = 1.0f / (1.0f - std::pow(b2, (float)net->step));
    RR_LAUNCH(rr::k_adam, rr::gridn(net->n_params, 256), 256, 0, s, net->w, net->g, net->m, net->v, net->n_params, lr,
              b1, b2, eps, c1, c2, net->weight_decay, (rr::bf16*)nullptr);
    rr::refresh_bf16(net, s);
    RR_CUDA(cudaGetLastError());
    if (loss) RR_TRY(rr::read_loss(net, batch, s, loss));
    return RT_OK;
}

// parameter access (FP32 masters, gradients, or the Adam state) for checkpoints and checks
extern "C" rt_status rt_mlp_copy(rt_mlp* net, int32_t what, float* host, int32_t to_device, void* stream) {
    rr::clear_error();
    if (!net || !host || what < 0 || what > 3) {
        rr::set_error("rt_mlp_copy: what = 0 weights, 1 gradients, 2 first moments, 3 second moments");
        return RT_ERR_INVALID_ARG;
    }
    cudaStream_t s = (cudaStream_t)stream;
    float* dev = what == 0 ? net->w : (what == 1 ? net->g : (what == 2 ? net->m : net->v));
    const size_t bytes = sizeof(float) * (size_t)net->n_params;
    if (to_device) {
        RR_CUDA(cudaMemcpyAsync(dev, host, bytes, cudaMemcpyHostToDevice, s));
        if (what == 0) rr::refresh_bf16(net, s);
    } else {
        RR_CUDA(cudaMemcpyAsync(host, dev, bytes, cudaMemcpyDeviceToHost, s));
    }
    unsigned int st = 0;
    RR_CUDA(cudaMemcpyAsync(&st, net->tc_status, sizeof st, cudaMemcpyDeviceToHost, s));
    RR_CUDA(cudaStreamSynchronize(s));
    return rr::check_tc(net, st);
}

extern "C" rt_status rt_mlp_set_weight_decay(rt_mlp* net, float weight_decay) {
    if (!net || !(weight_decay >= 0.f)) {
        rr::set_error("rt_mlp_set_weight_decay: null network or negative decay");
        return RT_ERR_INVALID_ARG;
    }
    net->weight_decay = weight_decay;
    return RT_OK;
}

extern "C" rt_status rt_mlp_get_step(const rt_mlp* net, int64_t* step) {
    if (!net || !step) {
        rr::set_error("rt_mlp_get_step: null argument");
        return RT_ERR_INVALID_ARG;
    }
    *step = net->step;
    return RT_OK;
}

extern "C" rt_status rt_mlp_set_step(rt_mlp* net, int64_t step) {
    if (!net || step < 0) {
        rr::set_error("rt_mlp_set_step: null network or negative step");
        return RT_ERR_INVALID_ARG;
    }
    net->step = step;
    return RT_OK;
}

// Measurement and test entry point of the two GEMM kernels behind the network.
extern "C" rt_status rt_gemm_bf16(const void* A, const void* B, int32_t M, int32_t N, int32_t K, float* C,
                                  int32_t kernel, float* workspace, int64_t workspace_floats, float* ms,
                                  void* stream) {
    rr::NvtxRange nvtx_range("rt_gemm_bf16");
    rr::clear_error();
    if (!A || !B || !C || M < 1 || N < 1 || K < 1 || K % 8 || (kernel != RT_GEMM_TMA && kernel != RT_GEMM_STAGED) ||
        workspace_floats < 0 || (workspace_floats > 0 && !workspace)) {
        rr::set_error("rt_gemm_bf16: need device A [M][K], B [N][K], C [M][N], sizes >= 1, K %% 8 == 0, a kernel "
                      "and a workspace pointer with a positive size");
        return RT_ERR_INVALID_ARG;
    }
    if (((uintptr_t)A | (uintptr_t)B | (uintptr_t)C | (uintptr_t)workspace) & 15u) {
        rr::set_error("rt_gemm_bf16: A, B, C and the workspace must be 16-byte aligned");
        return RT_ERR_INVALID_ARG;
    }
    cudaStream_t s = (cudaStream_t)stream;
    rr::Arena tmp(s);
    unsigned int* status;
    RR_TRY(tmp.alloc(&status, 1));
    RR_CUDA(cudaMemsetAsync(status, 0, sizeof(unsigned int), s));
    cudaEvent_t ev[2] = {nullptr, nullptr};
    if (ms) {
        RR_CUDA(cudaEventCreate(&ev[0]));
        if (cudaEventCreate(&ev[1]) != cudaSuccess) {
            cudaEventDestroy(ev[0]);
            RR_CUDA(cudaGetLastError());
        }
        cudaEventRecord(ev[0], s);
    }
    const rr::bf16* a = (const rr::bf16*)A;
    const rr::bf16* b = (const rr::bf16*)B;
    rt_status st_launch = kernel == RT_GEMM_TMA
                              ? rr::gemm<rr::EPI_F32>(a, b, M, N, K, nullptr, C, nullptr, nullptr, status, s, workspace,
                                                      (size_t)workspace_floats)
                              : rr::gemm_staged<rr::EPI_F32>(a, b, M, N, K, nullptr, C, nullptr, nullptr, status, s);
    if (ms) cudaEventRecord(ev[1], s);
    unsigned int st = 0;
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpyAsync(&st, status, sizeof st, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (ms) {
        if (e == cudaSuccess && st_launch == RT_OK) e = cudaEventElapsedTime(ms, ev[0], ev[1]);
        cudaEventDestroy(ev[0]);
        cudaEventDestroy(ev[1]);
    }
    if (st_launch != RT_OK) return st_launch;
    if (e != cudaSuccess) {
        rr::set_error("rt_gemm_bf16: %s", cudaGetErrorString(e));
        return RT_ERR_CUDA;
    }
    if (st) {
        rr::set_error("rt_gemm_bf16: a tensor-core tile timed out waiting for its copies or MMAs");
        return RT_ERR_CUDA;
    }
    return RT_OK;
}
