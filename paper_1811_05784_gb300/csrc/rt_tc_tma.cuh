// rt_tc_tma.cuh -- BF16 GEMM on the 5th-generation tensor cores with TMA tile
// loads and warp-specialised roles.
//
// C[M][N] = A[M][K] . B[N][K]^T, both operands K-contiguous BF16, FP32
// accumulation in tensor memory.  One CTA of 192 threads computes a 128 x 128
// tile of C through a ring of STAGES shared-memory stages:
//   warp 0 (one thread)  producer: for every 64-wide K step it waits until the
//                        stage is free, announces the stage's bytes on the
//                        stage's "full" mbarrier and issues two TMA loads
//                        (cp.async.bulk.tensor.2d, 128-byte swizzle, this
//                        GPU's memory only, no multicast) of the A and B
//                        tiles; rows and columns past M, N, K read as zero;
//   warp 1 (one thread)  MMA issuer: waits for the stage's bytes, issues four
//                        tcgen05.mma (kind::f16, M = 128, N = 128, K = 16)
//                        from shared-memory descriptors and commits them to
//                        the stage's "empty" mbarrier, which frees the stage
//                        for the producer; after the last step it commits to
//                        the "accumulator" mbarrier;
//   warps 2-5            epilogue: wait for the accumulator, read their 32
//                        TMEM lanes (warp w may read lanes 32 (w % 4) ..) with
//                        tcgen05.ld and apply bias / GELU before storing.
// Every wait is bounded: a wait that gives up sets bit 0 of *status; the
// roles then stop issuing work, the MMA thread still commits so that the
// epilogue and the producer are released, every thread waits (bounded) for
// the copies and MMAs already issued, and the tensor memory is freed before
// the CTA exits; C is left unwritten for that tile.
#pragma once

#include <cuda.h>
#include <cuda_bf16.h>
#include <stdint.h>

#include "rt_tc_gemm.cuh"

namespace rr {
namespace tma {

static constexpr int BM = 128, BN = 128, BK = 64, STAGES = 4;
static constexpr int A_BYTES = BM * BK * 2;   // 16 KB
static constexpr int B_BYTES = BN * BK * 2;   // 16 KB
static constexpr int STAGE_BYTES = A_BYTES + B_BYTES;
static constexpr int SMEM_BYTES = STAGES * STAGE_BYTES + 1024;  // + alignment slack for the 1024-B swizzle atoms
static constexpr uint32_t TMEM_COLS = 128;
static constexpr int THREADS = 192;

using tc::smem_u32;
using tc::smem_desc;
using tc::mbar_wait;

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(bar), "r"(bytes) : "memory");
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

template <int EPI>
__global__ void __launch_bounds__(THREADS) k_gemm_tma(const __grid_constant__ CUtensorMap map_a,
                                                      const __grid_constant__ CUtensorMap map_b, int M, int N, int K,
                                                      const float* __restrict__ bias, float* __restrict__ Cf,
                                                      float* __restrict__ Cpre, __nv_bfloat16* __restrict__ Cb,
                                                      unsigned int* __restrict__ status) {
    extern __shared__ uint8_t smem_raw[];
    __shared__ __align__(8) uint64_t full_bar[STAGES], empty_bar[STAGES], acc_bar;
    __shared__ uint32_t tmem_base;
    __shared__ int failed;
    uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
    const int n_steps = (K + BK - 1) / BK;

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
        mbar_init(smem_u32(&acc_bar), 1);
        failed = 0;
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    const uint32_t tmem = tmem_base;

    if (warp == 0 && lane == 0) {
        // producer
        asm volatile("prefetch.tensormap [%0];\n" ::"l"(reinterpret_cast<uint64_t>(&map_a)) : "memory");
        asm volatile("prefetch.tensormap [%0];\n" ::"l"(reinterpret_cast<uint64_t>(&map_b)) : "memory");
        for (int ks = 0; ks < n_steps; ks++) {
            const int s = ks % STAGES;
            if (ks >= STAGES && !mbar_wait(smem_u32(&empty_bar[s]), (uint32_t)(((ks / STAGES) - 1) & 1))) {
                atomicExch(&failed, 1);
                break;
            }
            if (*(volatile int*)&failed) break;
            uint8_t* sA = smem + s * STAGE_BYTES;
            const uint32_t fb = smem_u32(&full_bar[s]);
            mbar_expect_tx(fb, STAGE_BYTES);
            tma_load_2d(smem_u32(sA), &map_a, ks * BK, m0, fb);
            tma_load_2d(smem_u32(sA + A_BYTES), &map_b, ks * BK, n0, fb);
        }
    } else if (warp == 1 && lane == 0) {
        // MMA issuer
        const uint32_t idesc = tc::idesc_bf16(BM, BN);
        for (int ks = 0; ks < n_steps; ks++) {
            const int s = ks % STAGES;
            if (!mbar_wait(smem_u32(&full_bar[s]), (uint32_t)((ks / STAGES) & 1))) {
                atomicExch(&failed, 1);
                break;
            }
            if (*(volatile int*)&failed) break;
            asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
            const uint32_t a0 = smem_u32(smem + s * STAGE_BYTES), b0 = a0 + A_BYTES;
#pragma unroll
            for (int kk = 0; kk < BK / 16; kk++) {
                const uint64_t ad = smem_desc(a0 + kk * 32), bd = smem_desc(b0 + kk * 32);
                const uint32_t acc = (ks > 0 || kk > 0) ? 1u : 0u;
                asm volatile(
                    "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                    " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
                    "l"(ad), "l"(bd), "r"(idesc), "r"(acc)
                    : "memory");
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(
                             smem_u32(&empty_bar[s]))
                         : "memory");
        }
        // the accumulator is complete once every MMA issued before this commit is
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(
                         smem_u32(&acc_bar))
                     : "memory");
    } else if (warp >= 2) {
        // epilogue
        const bool ok = mbar_wait(smem_u32(&acc_bar), 0u);
        if (!ok) atomicExch(&failed, 1);
        asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
        if (ok && !*(volatile int*)&failed) {
            const int quarter = warp & 3;  // TMEM lanes 32 quarter .. 32 quarter + 31
            const int row = m0 + quarter * 32 + lane;
#pragma unroll 1
            for (int c0 = 0; c0 < BN; c0 += 16) {
                uint32_t v[16];
                const uint32_t ta = tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)c0;
                asm volatile(
                    "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, "
                    "[%16];\n"
                    : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
                      "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]),
                      "=r"(v[14]), "=r"(v[15])
                    : "r"(ta)
                    : "memory");
                asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
                if (row < M) {
#pragma unroll
                    for (int j = 0; j < 16; j++) {
                        const int col = n0 + c0 + j;
                        if (col >= N) break;
                        float x = __uint_as_float(v[j]);
                        const size_t o = (size_t)row * N + col;
                        if (EPI == tc::EPI_F32) {
                            Cf[o] = x;
                        } else if (EPI == tc::EPI_BIAS_F32) {
                            Cf[o] = x + bias[col];
                        } else {
                            x += bias[col];
                            Cpre[o] = x;
                            Cb[o] = __float2bfloat16_rn(tc::gelu_exact(x));
                        }
                    }
                }
            }
        }
    }
    __syncwarp();
    __syncthreads();
    if (failed) {
        // let the copies and MMAs already issued land (bounded) before the
        // shared and tensor memory they write go away
        if (tid == 0) {
            atomicOr(status, 1u);
            for (int s = 0; s < STAGES; s++) {
                mbar_wait(smem_u32(&full_bar[s]), 0u);
                mbar_wait(smem_u32(&full_bar[s]), 1u);
            }
            mbar_wait(smem_u32(&acc_bar), 0u);
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

}  // namespace tma
}  // namespace rr
