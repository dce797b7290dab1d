// rt_levels.cu -- rt_nearest_hits: nearest-element queries of given rays, by
// the per-ray stack traversal of the bounce kernel, or by the paper's
// distribution of rays through the tree level by level (Sec. 2.2).
//
// The paper sorts rays into the tree from the mother box down: every ray of
// a box is tested against its two daughter boxes with the slab test and goes
// on into each daughter it meets, until the leaves, whose elements it then
// intersects; the nearest of them is the ray's hit.  On the GPU every level
// is one launch over the level's (ray, node) pairs: a pair tests the node's
// child boxes (the tree is stored 4-wide, so one launch covers two binary
// levels), appends a pair for every internal child its ray meets, and tests
// the triangles of every leaf child at once; the nearest hit of each ray is
// kept as one 64-bit word (distance bits above the triangle id) so that
// atomicMin picks the nearest distance and, on equal distances, the lowest
// triangle id -- the tie rule of the stack traversal.  Boxes farther than a
// ray's nearest hit so far are not entered (that hit is only known once some
// leaf was reached), so the result equals the stack traversal's.  Rays are
// processed in chunks whose pairs fit the pair buffers; a chunk whose pairs
// overflow is split and run again.
#include "rt_traverse.cuh"

#include <algorithm>
#include <vector>

namespace rr {

struct QueryTree {
    const float4* nodes;
    const float4* tris;
    int64_t n_nodes, n_tris;
};

// per-ray set-up shared by every level: origin, reciprocal direction, shear
struct RayRow {
    float4 a;  // o.x o.y o.z inv.x
    float4 b;  // inv.y inv.z Sx Sy
    float4 c;  // Sz, kx | ky << 2 | kz << 4 (bits), exclude surface (bits), unused
};

__device__ __forceinline__ RayPre row_pre(const RayRow& w) {
    RayPre r;
    r.o = make_float3(w.a.x, w.a.y, w.a.z);
    r.d = make_float3(0.f, 0.f, 0.f);
    r.inv = make_float3(w.a.w, w.b.x, w.b.y);
    r.Sx = w.b.z, r.Sy = w.b.w, r.Sz = w.c.x;
    const int k = __float_as_int(w.c.y);
    r.kx = k & 3, r.ky = (k >> 2) & 3, r.kz = (k >> 4) & 3;
    return r;
}

__device__ __forceinline__ unsigned long long pack_hit(float t, int id) {
    return ((unsigned long long)__float_as_uint(t) << 32) | (unsigned int)id;
}

__global__ void k_ray_rows(const float* __restrict__ org, const float* __restrict__ dir,
                           const int32_t* __restrict__ excl, int64_t n, RayRow* __restrict__ rows,
                           unsigned long long* __restrict__ best) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const RayPre r = ray_pre(make_float3(org[3 * i], org[3 * i + 1], org[3 * i + 2]),
                             make_float3(dir[3 * i], dir[3 * i + 1], dir[3 * i + 2]));
    RayRow w;
    w.a = make_float4(r.o.x, r.o.y, r.o.z, r.inv.x);
    w.b = make_float4(r.inv.y, r.inv.z, r.Sx, r.Sy);
    w.c = make_float4(r.Sz, __int_as_float(r.kx | (r.ky << 2) | (r.kz << 4)), __int_as_float(excl ? excl[i] : -1),
                      0.f);
    rows[i] = w;
    best[i] = ~0ull;
}

// one level: pairs (ray, node) -> child pairs and leaf tests.  The level's
// pair count is read from the device (n_in_p, written by the level before),
// so the host queues every level without reading it back; a count above the
// pair buffers' capacity means pairs were dropped, which the host finds in the
// counters afterwards and answers by running the chunk again in halves.
__global__ void k_level(QueryTree tr, const RayRow* __restrict__ rows, const int2* __restrict__ in,
                        const uint32_t* __restrict__ n_in_p, int2* __restrict__ out, uint32_t* __restrict__ n_out,
                        uint32_t cap, unsigned long long* __restrict__ best, unsigned long long* __restrict__ counts,
                        unsigned int* __restrict__ status) {
    const uint32_t n_in = min(*n_in_p, cap);
    const int lane = threadIdx.x & 31;
    for (uint32_t base = blockIdx.x * blockDim.x; base < n_in; base += gridDim.x * blockDim.x) {
        const uint32_t j = base + threadIdx.x;
        bool act = j < n_in;
        int ray = 0, node = 0;
        if (act) {
            const int2 p = in[j];
            ray = p.x, node = p.y;
            if ((int64_t)node >= tr.n_nodes || node < 0) {
                atomicOr(status, ST_BOUNDS);
                act = false;
            }
        }
        float t[4] = {INFINITY, INFINITY, INFINITY, INFINITY};
        int ref[4] = {0, 0, 0, 0};
        int tests = 0;
        if (act) {
            const RayRow w = rows[ray];
            const RayPre r = row_pre(w);
            const int exclude = __float_as_int(w.c.z);
            const unsigned long long b0 = best[ray];
            float tfar = b0 == ~0ull ? INFINITY : __uint_as_float((unsigned int)(b0 >> 32));
            const float4* np = tr.nodes + 8 * (int64_t)node;
            float4 lx, ly, lz, hx, hy, hz;
            ld_v8(np, lx, ly);
            ld_v8(np + 2, lz, hx);
            ld_v8(np + 4, hy, hz);
            const int4 rf = __ldg(reinterpret_cast<const int4*>(np + 6));
            t[0] = slab(r, lx.x, ly.x, lz.x, hx.x, hy.x, hz.x, tfar);
            t[1] = slab(r, lx.y, ly.y, lz.y, hx.y, hy.y, hz.y, tfar);
            t[2] = slab(r, lx.z, ly.z, lz.z, hx.z, hy.z, hz.z, tfar);
            t[3] = slab(r, lx.w, ly.w, lz.w, hx.w, hy.w, hz.w, tfar);
            ref[0] = rf.x, ref[1] = rf.y, ref[2] = rf.z, ref[3] = rf.w;
            // leaf children: their triangles now
            float bt = tfar;
            int bid = b0 == ~0ull ? 0x7FFFFFFF : (int)(unsigned int)(b0 & 0xFFFFFFFFu);
            for (int c = 0; c < 4; c++) {
                if (!(t[c] < INFINITY) || ref[c] >= 0) continue;
                const int code = ~ref[c];
                const int first = code >> 3, cnt = code & 7;
                if ((int64_t)first + cnt > tr.n_tris) {
                    atomicOr(status, ST_BOUNDS);
                    continue;
                }
                for (int k = 0; k < cnt; k++) tri_test(r, tr.tris + 3 * (int64_t)(first + k), exclude, bt, bid);
                tests += cnt;
            }
            if (bid != 0x7FFFFFFF && pack_hit(bt, bid) < b0) atomicMin(best + ray, pack_hit(bt, bid));
        }
        // internal children met: one pair each, one atomic per warp and child slot
        for (int c = 0; c < 4; c++) {
            const bool emit = act && t[c] < INFINITY && ref[c] >= 0;
            const unsigned int m = __ballot_sync(0xffffffffu, emit);
            if (!m) continue;
            const int leader = __ffs(m) - 1;
            uint32_t obase = 0;
            if (lane == leader) obase = atomicAdd(n_out, (uint32_t)__popc(m));
            obase = __shfl_sync(0xffffffffu, obase, leader);
            if (emit) {
                const uint32_t p = obase + __popc(m & ((1u << lane) - 1u));
                if (p < cap) out[p] = make_int2(ray, ref[c]);
            }
        }
        // node visits and triangle tests of this level
        const unsigned int nv = __popc(__ballot_sync(0xffffffffu, act));
        int tt = tests;
        for (int o = 16; o > 0; o >>= 1) tt += __shfl_down_sync(0xffffffffu, tt, o);
        if (lane == 0 && nv) {
            atomicAdd(counts, (unsigned long long)nv);
            atomicAdd(counts + 1, (unsigned long long)tt);
        }
    }
}

__global__ void k_level_seed(int64_t r0, uint32_t n, int2* __restrict__ out, uint32_t* __restrict__ n_level0) {
    const uint32_t j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j < n) out[j] = make_int2((int)(r0 + j), 0);
    if (j == 0) *n_level0 = n;
}

__global__ void k_level_finish(const unsigned long long* __restrict__ best, int64_t n, int32_t* __restrict__ hit,
                               float* __restrict__ t) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const unsigned long long b = best[i];
    hit[i] = b == ~0ull ? -1 : (int32_t)(unsigned int)(b & 0xFFFFFFFFu);
    t[i] = b == ~0ull ? INFINITY : __uint_as_float((unsigned int)(b >> 32));
}

// the stack traversal of the bounce kernel, one thread per query
template <int BT>
__global__ void __launch_bounds__(BT) k_query_stack(QueryTree tr, const float* __restrict__ org,
                                                    const float* __restrict__ dir, const int32_t* __restrict__ excl,
                                                    int64_t n, int step_cap, int32_t* __restrict__ hit,
                                                    float* __restrict__ tout, unsigned long long* __restrict__ counts,
                                                    unsigned int* __restrict__ status) {
    extern __shared__ int s_stack[];
    int* stack = s_stack + threadIdx.x;
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const bool act = i < n;
    float best_t = INFINITY;
    int best_id = -1, nn = 0, nt = 0;
    unsigned int err = 0;
    if (act) {
        const RayPre r = ray_pre(make_float3(org[3 * i], org[3 * i + 1], org[3 * i + 2]),
                                 make_float3(dir[3 * i], dir[3 * i + 1], dir[3 * i + 2]));
        nearest_hit<BT, STACK_SMEM>(step_cap, tr, r, excl ? excl[i] : -1, best_t, best_id, err, nn, nt, stack);
        hit[i] = best_id;
        tout[i] = best_id >= 0 ? best_t : INFINITY;
    }
    if (err) atomicOr(status, err);
    const int lane = threadIdx.x & 31;
    for (int o = 16; o > 0; o >>= 1) {
        nn += __shfl_down_sync(0xffffffffu, nn, o);
        nt += __shfl_down_sync(0xffffffffu, nt, o);
    }
    if (lane == 0) {
        atomicAdd(counts, (unsigned long long)nn);
        atomicAdd(counts + 1, (unsigned long long)nt);
    }
}

}  // namespace rr

namespace rr {

static rt_status nearest_impl(const rt_tree* tree, const float* org, const float* dir, const int32_t* excl, int64_t n,
                              int32_t method, int32_t* hit, float* t, int64_t* stats, cudaStream_t s) {
    if (!tree || !org || !dir || !hit || !t || n < 1 || n > INT32_MAX || (method != RT_NEAREST_STACK &&
                                                                         method != RT_NEAREST_LEVELS)) {
        set_error("rt_nearest_hits: need a tree, device origins, directions, outputs, 1 <= n < 2^31 and a method");
        return RT_ERR_INVALID_ARG;
    }
    const QueryTree tr{tree->nodes, tree->tris, tree->n_nodes, tree->n_tris};
    Arena tmp(s);
    unsigned long long* counts;
    unsigned int* status;
    RR_TRY(tmp.alloc(&counts, 2));
    RR_TRY(tmp.alloc(&status, 1));
    RR_CUDA(cudaMemsetAsync(counts, 0, 2 * sizeof(unsigned long long), s));
    RR_CUDA(cudaMemsetAsync(status, 0, sizeof(unsigned int), s));
    if (method == RT_NEAREST_STACK) {
        constexpr int BT = 128;
        const size_t smem = sizeof(int) * STACK_SMEM * BT;
        RR_CUDA(cudaFuncSetAttribute(k_query_stack<BT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        RR_LAUNCH(k_query_stack<BT>, (unsigned)((n + BT - 1) / BT), BT, smem, s, tr, org, dir, excl, n, 1 << 16, hit,
                  t, counts, status);
        RR_CUDA(cudaGetLastError());
    } else {
        RayRow* rows;
        unsigned long long* best;
        RR_TRY(tmp.alloc(&rows, (size_t)n));
        RR_TRY(tmp.alloc(&best, (size_t)n));
        RR_LAUNCH(k_ray_rows, (unsigned)((n + 255) / 256), 256, 0, s, org, dir, excl, n, rows, best);
        // pair buffers: 2^26 pairs (512 MiB) each, or fewer for small queries
        const uint32_t cap = (uint32_t)std::min<int64_t>((int64_t)1 << 26, std::max<int64_t>(1 << 20, 64 * n));
        int2 *pa, *pb;
        RR_TRY(tmp.alloc(&pa, cap));
        RR_TRY(tmp.alloc(&pb, cap));
        // the levels' pair counts stay on the device: a batch of L levels is
        // queued at once (a 4-wide tree of binary depth D has about D / 2 + 1
        // levels) and the counts are read once per batch
        const int L = (std::max(4, tree->depth / 2 + 3) + 1) & ~1;  // even: level L's pairs land in pa
        uint32_t* lvl;
        RR_TRY(tmp.alloc(&lvl, (size_t)L + 1));
        std::vector<uint32_t> hl((size_t)L + 1);
        const unsigned lgrid = (unsigned)(8 * device_sm_count());
        int64_t chunk = std::min<int64_t>(n, cap / 4);
        for (int64_t r0 = 0; r0 < n;) {
            const int64_t m = std::min(chunk, n - r0);
            bool overflow = false, done = false;
            RR_CUDA(cudaMemsetAsync(lvl, 0, sizeof(uint32_t) * ((size_t)L + 1), s));
            RR_LAUNCH(k_level_seed, (unsigned)((m + 255) / 256), 256, 0, s, r0, (uint32_t)m, pa, lvl);
            int2* buf[2] = {pa, pb};
            for (int batch = 0; batch < 64 && !done; batch++) {
                for (int l = 0; l < L; l++)
                    RR_LAUNCH(k_level, lgrid, 256, 0, s, tr, rows, buf[l & 1], lvl + l, buf[(l + 1) & 1], lvl + l + 1,
                              cap, best, counts, status);
                RR_CUDA(cudaGetLastError());
                RR_CUDA(cudaMemcpyAsync(hl.data(), lvl, sizeof(uint32_t) * ((size_t)L + 1), cudaMemcpyDeviceToHost, s));
                RR_CUDA(cudaStreamSynchronize(s));
                for (int l = 1; l <= L; l++)
                    if (hl[(size_t)l] > cap) overflow = true;
                if (overflow) break;
                if (hl[(size_t)L] == 0) {
                    done = true;
                    break;
                }
                // pairs left after L levels: they are in pa, go on from there
                hl[0] = hl[(size_t)L];
                RR_CUDA(cudaMemsetAsync(lvl, 0, sizeof(uint32_t) * ((size_t)L + 1), s));
                RR_CUDA(cudaMemcpyAsync(lvl, hl.data(), sizeof(uint32_t), cudaMemcpyHostToDevice, s));
                RR_CUDA(cudaStreamSynchronize(s));
            }
            if (!overflow && !done) {
                set_error("rt_nearest_hits: the level-by-level distribution did not finish in %d levels", 64 * L);
                return RT_ERR_INTERNAL;
            }
            if (overflow) {
                // the chunk's pairs did not fit: split it and start it again;
                // hits already found stay correct (each is a real hit of its ray)
                if (m == 1) {
                    set_error("rt_nearest_hits: one ray meets more than %u boxes of one level", cap);
                    return RT_ERR_CAPACITY;
                }
                chunk = std::max<int64_t>(1, m / 2);
                continue;
            }
            r0 += m;
        }
        RR_LAUNCH(k_level_finish, (unsigned)((n + 255) / 256), 256, 0, s, best, n, hit, t);
        RR_CUDA(cudaGetLastError());
    }
    unsigned long long hc[2] = {0, 0};
    unsigned int st = 0;
    RR_CUDA(cudaMemcpyAsync(hc, counts, sizeof hc, cudaMemcpyDeviceToHost, s));
    RR_CUDA(cudaMemcpyAsync(&st, status, sizeof st, cudaMemcpyDeviceToHost, s));
    RR_CUDA(cudaStreamSynchronize(s));
    if (st & (ST_STACK | ST_BOUNDS)) {
        set_error("rt_nearest_hits: a node or leaf reference lies outside the tree, or the stack overflowed");
        return st & ST_STACK ? RT_ERR_STACK : RT_ERR_INTERNAL;
    }
    if (st & ST_STEPS) {
        set_error("rt_nearest_hits: a traversal exceeded 65536 node visits");
        return RT_ERR_STEP_LIMIT;
    }
    if (stats) stats[0] = (int64_t)hc[0], stats[1] = (int64_t)hc[1];
    return RT_OK;
}

}  // namespace rr

extern "C" rt_status rt_nearest_hits(const rt_tree* tree, const float* origins, const float* directions,
                                     const int32_t* exclude_surface, int64_t n, int32_t method, int32_t* hit,
                                     float* t, int64_t* stats, void* stream) {
    rr::NvtxRange nvtx_range("rt_nearest_hits");
    rr::clear_error();
    return rr::nearest_impl(tree, origins, directions, exclude_surface, n, method, hit, t, stats,
                            (cudaStream_t)stream);
}
