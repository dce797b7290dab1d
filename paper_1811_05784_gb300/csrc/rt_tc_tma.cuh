// rt_tc_tma.cuh -- BF16 GEMM on the 5th-generation tensor cores with TMA tile
// loads, warp-specialised roles and a persistent tile loop.
//
// C[M][N] = A[M][K] . B[N][K]^T, both operands K-contiguous BF16, FP32
// accumulation in tensor memory.  The output is cut into 128 x bn tiles (bn a
// multiple of 16, at most 256, chosen by the host to fit N); a product with
// few tiles and a long K is also cut along K into `splits` ranges whose
// partial sums go to a workspace and are added in a fixed order afterwards
// (k_splitk_reduce), so results do not depend on timing.  One CTA of 192
// threads runs on each SM and walks the work units u = blockIdx.x,
// blockIdx.x + gridDim.x, ...:
//   warp 0 (one thread)  producer: for every 64-wide K step it waits until the
//                        ring stage is free, announces the stage's bytes on its
//                        "full" mbarrier and issues two TMA loads
//                        (cp.async.bulk.tensor.2d, 128-byte swizzle, this
//                        GPU's memory only, no multicast) of the A and B
//                        tiles; rows and columns past M, N, K read as zero;
//   warp 1 (one thread)  MMA issuer: alternates between two accumulators of
//                        256 TMEM columns; waits until the epilogue has
//                        drained the accumulator, then per stage waits for its
//                        bytes, issues four tcgen05.mma (kind::f16, M = 128,
//                        N = bn, K = 16) and commits them to the stage's
//                        "empty" mbarrier; after the unit's last step it
//                        commits to the accumulator's "full" mbarrier;
//   warps 2-5            epilogue: warp w reads TMEM lanes 32 (w % 4) ..
//                        + 31 (its 32 rows) 32 columns at a time with
//                        tcgen05.ld, passes them through a padded shared-memory
//                        block so that each store instruction writes four
//                        whole 128-byte row segments, applies bias / GELU and
//                        frees the accumulator for the MMA issuer.
// The epilogue of one unit thus overlaps the MMAs of the next.
// Every wait is bounded: a wait that gives up sets bit 0 of *status; all roles
// stop issuing work, every copy still in flight is waited for (bounded), the
// MMA issuer waits for its MMAs through one last commit, and the tensor memory
// is freed before the CTA exits; the unit's C is left unwritten.
#pragma once

#include <cuda.h>
#include <cuda_bf16.h>
#include <stdint.h>

#include "rt_tc_gemm.cuh"

namespace rr {
namespace tma {

static constexpr int BM = 128, BN_MAX = 256, BK = 64, STAGES = 4;
static constexpr int A_BYTES = BM * BK * 2;           // 16 KB
static constexpr int B_BYTES_MAX = BN_MAX * BK * 2;   // 32 KB
static constexpr int STAGE_BYTES = A_BYTES + B_BYTES_MAX;
static constexpr int EPI_WARPS = 4;
static constexpr int STG_LD = 36;   // floats per staged row: float4 writes by row and reads by column group
                                    // both hit 8 distinct 16-byte bank groups per quarter-warp (36 / 4 odd)
static constexpr int STG_FLOATS = 32 * STG_LD;
static constexpr int SMEM_BYTES = STAGES * STAGE_BYTES + EPI_WARPS * STG_FLOATS * 4 + 1024;  // + 1024-B alignment
static constexpr uint32_t TMEM_COLS = 512;            // two accumulators of up to 256 columns
static constexpr int THREADS = 64 + 32 * EPI_WARPS;
static constexpr int MAX_SPLITS = 16;

// the work decomposition of one product (computed on the host by plan())
struct Shape {
    int M, N, K;
    int bn;         // tile columns
    int tiles_n;    // tiles along N
    int tiles;      // tiles in all
    int splits;     // K ranges per tile (1: the kernel writes C itself)
    int steps_per;  // 64-wide K steps per range
    int n_steps;    // 64-wide K steps of the whole product
};

// bn: the largest multiple of 16 (<= 256) among those that cover N with the
// fewest columns; splits: when the tiles fill less than half of the SMs, as
// many K ranges (of at least 4 steps) as keep the SMs busy and the partial
// sums fit the workspace (ws_floats, 0 = no splitting)
static inline Shape plan(int M, int N, int K, int sms, size_t ws_floats) {
    Shape s{};
    s.M = M;
    s.N = N;
    s.K = K;
    int best_cols = 1 << 30;
    for (int bn = BN_MAX; bn >= 16; bn -= 16) {
        const int cols = (N + bn - 1) / bn * bn;
        if (cols < best_cols) {
            best_cols = cols;
            s.bn = bn;
        }
    }
    s.tiles_n = (N + s.bn - 1) / s.bn;
    s.tiles = (M + BM - 1) / BM * s.tiles_n;
    s.n_steps = (K + BK - 1) / BK;
    int splits = 1;
    if (ws_floats > 0 && 2 * s.tiles <= sms) {
        splits = sms / s.tiles;
        if (splits > s.n_steps / 4) splits = s.n_steps / 4;
        if (splits > MAX_SPLITS) splits = MAX_SPLITS;
        while (splits > 1 && (size_t)splits * M * N > ws_floats) splits--;
        if (splits < 1) splits = 1;
    }
    s.steps_per = (s.n_steps + splits - 1) / splits;
    s.splits = (s.n_steps + s.steps_per - 1) / s.steps_per;  // no empty range
    return s;
}

using tc::mbar_wait;
using tc::smem_desc;
using tc::smem_u32;

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(bar), "r"(bytes) : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];\n" ::"r"(bar) : "memory");
}

__device__ __forceinline__ void mma_commit(uint32_t bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(bar)
                 : "memory");
}

// 2D tile load into shared memory, completion counted on the mbarrier;
// x is the innermost (K) coordinate in elements, a multiple of 64 here
__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap* map, int x, int y, uint32_t bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];\n" ::
            "r"(dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(bar)
        : "memory");
}

struct Unit {
    int m0, n0, ks0, ks1, split;
};

__device__ __forceinline__ Unit unit_of(const Shape& sh, int u) {
    Unit w;
    const int t = u / sh.splits;
    w.split = u - t * sh.splits;
    w.m0 = (t / sh.tiles_n) * BM;
    w.n0 = (t % sh.tiles_n) * sh.bn;
    w.ks0 = w.split * sh.steps_per;
    w.ks1 = min(sh.n_steps, w.ks0 + sh.steps_per);
    return w;
}

// C (or the split's partial-sum block Cf + split * split_stride) of one unit
template <int EPI>
__device__ __forceinline__ void store4(const Shape& sh, int row, int col, int col_end, float4 x,
                                       const float* __restrict__ bias, float* __restrict__ Cf,
                                       float* __restrict__ Cpre, __nv_bfloat16* __restrict__ Cb) {
    float v[4] = {x.x, x.y, x.z, x.w};
    if (EPI != tc::EPI_F32) {
#pragma unroll
        for (int e = 0; e < 4; e++)
            if (col + e < col_end) v[e] += __ldg(bias + col + e);
    }
    const size_t o = (size_t)row * sh.N + col;
    if ((sh.N & 3) == 0 && col + 3 < col_end) {
        if (EPI == tc::EPI_BIAS_GELU) {
            *reinterpret_cast<float4*>(Cpre + o) = make_float4(v[0], v[1], v[2], v[3]);
            __nv_bfloat162 lo = __floats2bfloat162_rn(tc::gelu_exact(v[0]), tc::gelu_exact(v[1]));
            __nv_bfloat162 hi = __floats2bfloat162_rn(tc::gelu_exact(v[2]), tc::gelu_exact(v[3]));
            uint2 pk;
            pk.x = *reinterpret_cast<uint32_t*>(&lo);
            pk.y = *reinterpret_cast<uint32_t*>(&hi);
            *reinterpret_cast<uint2*>(Cb + o) = pk;
        } else {
            *reinterpret_cast<float4*>(Cf + o) = make_float4(v[0], v[1], v[2], v[3]);
        }
    } else {
#pragma unroll
        for (int e = 0; e < 4; e++) {
            if (col + e >= col_end) break;
            if (EPI == tc::EPI_BIAS_GELU) {
                Cpre[o + e] = v[e];
                Cb[o + e] = __float2bfloat16_rn(tc::gelu_exact(v[e]));
            } else {
                Cf[o + e] = v[e];
            }
        }
    }
}

template <int EPI>
__global__ void __launch_bounds__(THREADS, 1)
    k_gemm_tma(const __grid_constant__ CUtensorMap map_a, const __grid_constant__ CUtensorMap map_b, const Shape sh,
               const float* __restrict__ bias, float* __restrict__ Cf, float* __restrict__ Cpre,
               __nv_bfloat16* __restrict__ Cb, int64_t split_stride, unsigned int* __restrict__ status) {
    extern __shared__ uint8_t smem_raw[];
    __shared__ __align__(8) uint64_t full_bar[STAGES], empty_bar[STAGES], acc_full[2], acc_empty[2], drain_bar;
    __shared__ uint32_t tmem_base;
    __shared__ int failed, issued, consumed;
    uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
    float* stg_all = reinterpret_cast<float*>(smem + STAGES * STAGE_BYTES);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int units = sh.tiles * sh.splits;

    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_u32(&tmem_base)),
                     "r"(TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
    }
    if (tid == 0) {
        for (int s = 0; s < STAGES; s++) {
            mbar_init(smem_u32(&full_bar[s]), 1);
            mbar_init(smem_u32(&empty_bar[s]), 1);
        }
        for (int j = 0; j < 2; j++) {
            mbar_init(smem_u32(&acc_full[j]), 1);
            mbar_init(smem_u32(&acc_empty[j]), EPI_WARPS);
        }
        mbar_init(smem_u32(&drain_bar), 1);
        failed = 0;
        issued = 0;
        consumed = 0;
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    const uint32_t tmem = tmem_base;
    volatile int* vfailed = &failed;

    if (warp == 0) {
        if (lane == 0) {
            // producer
            asm volatile("prefetch.tensormap [%0];\n" ::"l"(reinterpret_cast<uint64_t>(&map_a)) : "memory");
            asm volatile("prefetch.tensormap [%0];\n" ::"l"(reinterpret_cast<uint64_t>(&map_b)) : "memory");
            const uint32_t bytes = (uint32_t)(A_BYTES + sh.bn * BK * 2);
            int it = 0;
            for (int u = blockIdx.x; u < units && !*vfailed; u += gridDim.x) {
                const Unit w = unit_of(sh, u);
                for (int ks = w.ks0; ks < w.ks1; ks++, it++) {
                    const int s = it % STAGES;
                    if (it >= STAGES && !mbar_wait(smem_u32(&empty_bar[s]), (uint32_t)(((it / STAGES) - 1) & 1))) {
                        atomicExch(&failed, 1);
                        break;
                    }
                    if (*vfailed) break;
                    uint8_t* sA = smem + s * STAGE_BYTES;
                    const uint32_t fb = smem_u32(&full_bar[s]);
                    mbar_expect_tx(fb, bytes);
                    tma_load_2d(smem_u32(sA), &map_a, ks * BK, w.m0, fb);
                    tma_load_2d(smem_u32(sA + A_BYTES), &map_b, ks * BK, w.n0, fb);
                    *(volatile int*)&issued = it + 1;
                }
            }
        }
    } else if (warp == 1) {
        if (lane == 0) {
            // MMA issuer
            const uint32_t idesc = tc::idesc_bf16(BM, sh.bn);
            int it = 0, i = 0;
            for (int u = blockIdx.x; u < units && !*vfailed; u += gridDim.x, i++) {
                const Unit w = unit_of(sh, u);
                const int j = i & 1;
                if (i >= 2 && !mbar_wait(smem_u32(&acc_empty[j]), (uint32_t)(((i >> 1) - 1) & 1))) {
                    atomicExch(&failed, 1);
                    break;
                }
                asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
                const uint32_t d = tmem + (uint32_t)(j * BN_MAX);
                bool ok = true;
                for (int ks = w.ks0; ks < w.ks1; ks++, it++) {
                    const int s = it % STAGES;
                    if (!mbar_wait(smem_u32(&full_bar[s]), (uint32_t)((it / STAGES) & 1))) {
                        atomicExch(&failed, 1);
                        ok = false;
                        break;
                    }
                    if (*vfailed) {
                        ok = false;
                        break;
                    }
                    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
                    const uint32_t a0 = smem_u32(smem + s * STAGE_BYTES), b0 = a0 + A_BYTES;
#pragma unroll
                    for (int kk = 0; kk < BK / 16; kk++) {
                        const uint64_t ad = smem_desc(a0 + kk * 32), bd = smem_desc(b0 + kk * 32);
                        const uint32_t acc = (ks > w.ks0 || kk > 0) ? 1u : 0u;
                        asm volatile(
                            "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                            " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d),
                            "l"(ad), "l"(bd), "r"(idesc), "r"(acc)
                            : "memory");
                    }
                    mma_commit(smem_u32(&empty_bar[s]));
                    *(volatile int*)&consumed = it + 1;
                }
                if (!ok) break;
                mma_commit(smem_u32(&acc_full[j]));  // complete once every MMA issued before it is
            }
        }
    } else {
        // epilogue
        const int quarter = warp & 3;  // TMEM lanes 32 quarter .. 32 quarter + 31
        float* stg = stg_all + (warp - 2) * STG_FLOATS;
        const int r_in = lane >> 3, cq = (lane & 7) * 4;
        float* out = Cf;
        int i = 0;
        for (int u = blockIdx.x; u < units; u += gridDim.x, i++) {
            const Unit w = unit_of(sh, u);
            const int j = i & 1;
            // the warp decides together: tcgen05.ld below is warp-wide
            const bool ok = __all_sync(0xffffffffu, mbar_wait(smem_u32(&acc_full[j]), (uint32_t)((i >> 1) & 1)));
            if (!ok) {
                if (lane == 0) atomicExch(&failed, 1);
                break;
            }
            if (__shfl_sync(0xffffffffu, *vfailed, 0)) break;
            asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
            if (sh.splits > 1) out = Cf + (size_t)w.split * (size_t)split_stride;
            const int col_end = min(sh.N, w.n0 + sh.bn);
            const uint32_t tbase = tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(j * BN_MAX);
#pragma unroll 1
            for (int c0 = 0; c0 < sh.bn && w.n0 + c0 < sh.N; c0 += 32) {
                uint32_t v[32];
                asm volatile(
                    "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
                    "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];\n"
                    : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
                      "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]),
                      "=r"(v[14]), "=r"(v[15]), "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]),
                      "=r"(v[21]), "=r"(v[22]), "=r"(v[23]), "=r"(v[24]), "=r"(v[25]), "=r"(v[26]), "=r"(v[27]),
                      "=r"(v[28]), "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
                    : "r"(tbase + (uint32_t)c0)
                    : "memory");
                asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
                // this lane's row into the staging block ...
#pragma unroll
                for (int q = 0; q < 8; q++)
                    *reinterpret_cast<float4*>(stg + lane * STG_LD + 4 * q) =
                        make_float4(__uint_as_float(v[4 * q]), __uint_as_float(v[4 * q + 1]),
                                    __uint_as_float(v[4 * q + 2]), __uint_as_float(v[4 * q + 3]));
                __syncwarp();
                // ... and out by rows: 8 lanes cover one row's 32 columns
#pragma unroll 2
                for (int rr = 0; rr < 8; rr++) {
                    const int r = rr * 4 + r_in;
                    const int row = w.m0 + quarter * 32 + r, col = w.n0 + c0 + cq;
                    const float4 x = *reinterpret_cast<const float4*>(stg + r * STG_LD + cq);
                    if (row < sh.M && col < col_end) store4<EPI>(sh, row, col, col_end, x, bias, out, Cpre, Cb);
                }
                __syncwarp();
            }
            asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
            __syncwarp();
            if (lane == 0) mbar_arrive(smem_u32(&acc_empty[j]));
        }
    }
    __syncwarp();
    __syncthreads();
    if (failed) {
        // let the copies and MMAs already issued land (bounded) before the
        // shared and tensor memory they write go away
        if (tid == 0) {
            atomicOr(status, 1u);
            const int c = *(volatile int*)&consumed, n = *(volatile int*)&issued;
            for (int k = c; k < n; k++) mbar_wait(smem_u32(&full_bar[k % STAGES]), (uint32_t)((k / STAGES) & 1));
        }
        if (tid == 32) {
            mma_commit(smem_u32(&drain_bar));
            mbar_wait(smem_u32(&drain_bar), 0u);
        }
        __syncthreads();
    }
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    if (warp == 1) {
        asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(TMEM_COLS) : "memory");
    }
}

// C = sum over the splits of the partial sums, in split order, then the
// epilogue; one thread per 4 consecutive elements of C (M N % 4 == 0) or per
// element
template <int EPI>
__global__ void k_splitk_reduce(const float* __restrict__ part, int splits, int64_t MN, int N,
                                const float* __restrict__ bias, float* __restrict__ Cf, float* __restrict__ Cpre,
                                __nv_bfloat16* __restrict__ Cb) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    if ((MN & 3) == 0 && (N & 3) == 0) {
        for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < MN / 4; q += stride) {
            float4 a = reinterpret_cast<const float4*>(part)[q];
            for (int s = 1; s < splits; s++) {
                const float4 b = reinterpret_cast<const float4*>(part + (size_t)s * MN)[q];
                a.x += b.x;
                a.y += b.y;
                a.z += b.z;
                a.w += b.w;
            }
            float v[4] = {a.x, a.y, a.z, a.w};
            const int col = (int)((4 * q) % N);
            if (EPI != tc::EPI_F32) {
#pragma unroll
                for (int e = 0; e < 4; e++) v[e] += bias[col + e];
            }
            if (EPI == tc::EPI_BIAS_GELU) {
                reinterpret_cast<float4*>(Cpre)[q] = make_float4(v[0], v[1], v[2], v[3]);
#pragma unroll
                for (int e = 0; e < 4; e++) Cb[4 * q + e] = __float2bfloat16_rn(tc::gelu_exact(v[e]));
            } else {
                reinterpret_cast<float4*>(Cf)[q] = make_float4(v[0], v[1], v[2], v[3]);
            }
        }
    } else {
        for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < MN; e += stride) {
            float a = part[e];
            for (int s = 1; s < splits; s++) a += part[(size_t)s * MN + e];
            if (EPI != tc::EPI_F32) a += bias[e % N];
            if (EPI == tc::EPI_BIAS_GELU) {
                Cpre[e] = a;
                Cb[e] = __float2bfloat16_rn(tc::gelu_exact(a));
            } else {
                Cf[e] = a;
            }
        }
    }
}

}  // namespace tma
}  // namespace rr
