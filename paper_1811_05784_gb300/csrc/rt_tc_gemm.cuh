// rt_tc_gemm.cuh -- BF16 GEMM on the 5th-generation tensor cores (tcgen05).
//
// C[M][N] = A[M][K] . B[N][K]^T, both operands K-contiguous (row-major with K
// innermost), FP32 accumulation in tensor memory (TMEM).  One CTA of 128
// threads computes a 128 x 64 tile of C:
//   * the four warps copy the 128 x 64 A tile and the 64 x 64 B tile of each
//     64-wide K step into shared memory in the 128-byte-swizzled K-major
//     layout (row r at r * 128 B, 16-byte chunk c stored at chunk c ^ (r % 8),
//     8-row groups 1024 B apart), zero-padding rows past M / N and columns
//     past K;
//   * one thread issues four tcgen05.mma (kind::f16, M = 128, N = 64,
//     K = 16 each) from shared-memory descriptors, the first of the whole
//     product overwriting the accumulator, and commits them to an mbarrier;
//   * every thread waits on that mbarrier (bounded) before the next K step
//     overwrites the tiles; two tile buffers alternate so that the copy of
//     step k + 1 overlaps the MMAs of step k;
//   * warp w reads TMEM lanes 32w .. 32w + 31 (rows) with tcgen05.ld and
//     applies the epilogue (bias, GELU) before storing.
// Requirements (checked by the launcher): K % 8 == 0, 16-byte aligned rows.
// A wait that runs out sets bit 0 of *status, waits once more (bounded) for
// the MMAs in flight, frees the tensor memory and leaves the tile unwritten.
#pragma once

#include <cuda_bf16.h>
#include <stdint.h>

namespace rr {
namespace tc {

static constexpr int BM = 128, BN = 64, BK = 64;
static constexpr int A_BYTES = BM * BK * 2;           // 16 KB
static constexpr int B_BYTES = BN * BK * 2;           // 8 KB
static constexpr int STAGE_BYTES = A_BYTES + B_BYTES;
static constexpr int SMEM_BYTES = 2 * STAGE_BYTES + 1024;   // two stages + alignment slack
static constexpr uint32_t TMEM_COLS = 64;             // FP32 accumulator: 128 lanes x 64 columns
static constexpr long long WAIT_LIMIT = 1ll << 22;    // mbarrier polls before giving up

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// byte offset of 16-byte chunk c of row r in a 128-byte-swizzled tile
__device__ __forceinline__ uint32_t sw128(int r, int c) { return (uint32_t)(r * 128 + ((c ^ (r & 7)) << 4)); }

// shared-memory matrix descriptor: start address, leading byte offset (unused
// for swizzled K-major, 16 B), stride byte offset 1024 B (8 rows x 128 B),
// descriptor version 1, 128-byte swizzle
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr) {
    uint64_t d = 0;
    d |= (uint64_t)((addr & 0x3FFFFu) >> 4);
    d |= (uint64_t)(16u >> 4) << 16;
    d |= (uint64_t)(1024u >> 4) << 32;
    d |= (uint64_t)1 << 46;
    d |= (uint64_t)2 << 61;
    return d;
}

// instruction descriptor, kind::f16: D F32, A and B BF16, both K-major,
// N >> 3 at bit 17, M >> 4 at bit 24
__host__ __device__ constexpr uint32_t idesc_bf16(int m, int n) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(m >> 4) << 24);
}

__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity) {
    for (long long it = 0; it < WAIT_LIMIT; it++) {
        uint32_t ok;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(ok)
            : "r"(bar), "r"(parity)
            : "memory");
        if (ok) return true;
    }
    return false;
}

enum { EPI_F32 = 0, EPI_BIAS_GELU = 1, EPI_BIAS_F32 = 2 };

__device__ __forceinline__ float gelu_exact(float x) { return 0.5f * x * (1.0f + erff(x * 0.70710678118654752f)); }

__device__ __forceinline__ void load_tile(const __nv_bfloat16* __restrict__ G, int rows_total, int K, int r0,
                                          int k0, int nrows, uint8_t* s) {
    for (int i = threadIdx.x; i < nrows * 8; i += 128) {
        const int r = i >> 3, c = i & 7;
        const int gr = r0 + r, gk = k0 + c * 8;
        uint4 v = make_uint4(0u, 0u, 0u, 0u);
        if (gr < rows_total && gk < K) v = *reinterpret_cast<const uint4*>(G + (size_t)gr * K + gk);
        *reinterpret_cast<uint4*>(s + sw128(r, c)) = v;
    }
}

template <int EPI>
__global__ void __launch_bounds__(128) k_gemm_tc(const __nv_bfloat16* __restrict__ A,
                                                 const __nv_bfloat16* __restrict__ B, int M, int N, int K,
                                                 const float* __restrict__ bias, float* __restrict__ Cf,
                                                 float* __restrict__ Cpre, __nv_bfloat16* __restrict__ Cb,
                                                 unsigned int* __restrict__ status) {
    extern __shared__ uint8_t smem_raw[];
    __shared__ __align__(8) uint64_t mbar[2];
    __shared__ uint32_t tmem_base;
    uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_u32(&tmem_base)),
                     "r"(TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
    }
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_u32(&mbar[0])) : "memory");
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_u32(&mbar[1])) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    const uint32_t tmem = tmem_base;
    const uint32_t idesc = idesc_bf16(BM, BN);

    const int n_steps = (K + BK - 1) / BK;
    uint32_t phase[2] = {0u, 0u};
    bool pending[2] = {false, false};
    bool ok = true;
    for (int step = 0; step < n_steps && ok; step++) {
        const int st = step & 1;
        uint8_t* sA = smem + st * STAGE_BYTES;
        uint8_t* sB = sA + A_BYTES;
        // the MMAs that last read this stage must have finished
        if (pending[st]) {
            ok = mbar_wait(smem_u32(&mbar[st]), phase[st]);
            phase[st] ^= 1u;
            pending[st] = false;
            if (!ok) break;
        }
        load_tile(A, M, K, m0, step * BK, BM, sA);
        load_tile(B, N, K, n0, step * BK, BN, sB);
        asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
        __syncthreads();
        if (tid == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
            const uint32_t a0 = smem_u32(sA), b0 = smem_u32(sB);
#pragma unroll
            for (int kk = 0; kk < BK / 16; kk++) {
                const uint64_t ad = smem_desc(a0 + kk * 32), bd = smem_desc(b0 + kk * 32);
                const uint32_t acc = (step > 0 || kk > 0) ? 1u : 0u;
                asm volatile(
                    "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                    " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
                    "l"(ad), "l"(bd), "r"(idesc), "r"(acc)
                    : "memory");
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(
                             smem_u32(&mbar[st]))
                         : "memory");
        }
        pending[st] = true;
    }
    // the last commit covers every MMA issued before it
    for (int st = 0; st < 2; st++) {
        if (!pending[st]) continue;
        const bool w = mbar_wait(smem_u32(&mbar[st]), phase[st]);
        if (!w && ok) {
            ok = false;
            mbar_wait(smem_u32(&mbar[st]), phase[st]);  // once more, for the MMAs still in flight
        }
    }
    if (!ok && tid == 0) atomicOr(status, 1u);
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    if (ok) {
        const int row = m0 + warp * 32 + lane;
#pragma unroll
        for (int c0 = 0; c0 < BN; c0 += 16) {
            uint32_t v[16];
            const uint32_t ta = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0;
            asm volatile(
                "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, "
                "[%16];\n"
                : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
                  "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]),
                  "=r"(v[15])
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
                    if (EPI == EPI_F32) {
                        Cf[o] = x;
                    } else if (EPI == EPI_BIAS_F32) {
                        Cf[o] = x + bias[col];
                    } else {
                        x += bias[col];
                        Cpre[o] = x;
                        Cb[o] = __float2bfloat16_rn(gelu_exact(x));
                    }
                }
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    if (warp == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(TMEM_COLS) : "memory");
    }
}

}  // namespace tc
}  // namespace rr
