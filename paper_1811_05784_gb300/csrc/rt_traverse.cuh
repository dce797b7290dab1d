// rt_traverse.cuh -- nearest-element search over the 4-wide tree: ray set-up,
// slab test, watertight triangle test and the per-ray stack traversal, shared
// by the bounce kernel and the standalone query kernels.
#pragma once

#include "rt_internal.cuh"

namespace rr {

// status bits set by device code, read once per call
enum : unsigned int { ST_STACK = 1u, ST_STEPS = 2u, ST_HISTORY = 4u, ST_BOUNDS = 8u };

// ---------------------------------------------------------------------------
// nearest hit
// ---------------------------------------------------------------------------
__device__ __forceinline__ float comp(const float3& v, int k) { return k == 0 ? v.x : (k == 1 ? v.y : v.z); }

struct RayPre {
    float3 o, d, inv;
    int kx, ky, kz;
    float Sx, Sy, Sz;
};

__device__ __forceinline__ RayPre ray_pre(float3 o, float3 d) {
    RayPre p;
    p.o = o;
    p.d = d;
    // zero components become tiny so that 1/d stays finite (no 0 * inf)
    float dx = fabsf(d.x) > 1e-30f ? d.x : copysignf(1e-30f, d.x);
    float dy = fabsf(d.y) > 1e-30f ? d.y : copysignf(1e-30f, d.y);
    float dz = fabsf(d.z) > 1e-30f ? d.z : copysignf(1e-30f, d.z);
    p.inv = make_float3(1.0f / dx, 1.0f / dy, 1.0f / dz);
    float ax = fabsf(d.x), ay = fabsf(d.y), az = fabsf(d.z);
    int kz = (ax > ay) ? ((ax > az) ? 0 : 2) : ((ay > az) ? 1 : 2);
    int kx = kz == 2 ? 0 : kz + 1;
    int ky = kx == 2 ? 0 : kx + 1;
    if (comp(d, kz) < 0.f) {
        int t = kx;
        kx = ky;
        ky = t;
    }
    p.kx = kx;
    p.ky = ky;
    p.kz = kz;
    float dkz = comp(d, kz);
    p.Sx = __fdiv_rn(comp(d, kx), dkz);
    p.Sy = __fdiv_rn(comp(d, ky), dkz);
    p.Sz = __fdiv_rn(1.0f, dkz);
    return p;
}

// 32-byte read-only load (one whole L1 sector per lane); p must be 32-byte
// aligned.  A divergent gather costs the L1 data pipe one pass per sector and
// load instruction, so a 128-byte node read as three 32-byte loads and one
// 16-byte load costs 4 passes instead of 7, and a 48-byte triangle 2 instead of 3.
__device__ __forceinline__ void ld_v8(const float4* p, float4& a, float4& b) {
    asm("ld.global.nc.v8.f32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
        : "=f"(a.x), "=f"(a.y), "=f"(a.z), "=f"(a.w), "=f"(b.x), "=f"(b.y), "=f"(b.z), "=f"(b.w)
        : "l"(p));
}

// slab test of one box; returns entry distance, or +inf on a miss.
// (lo - o) * (1/d) has a relative error of a few ulps of t itself, which the
// conservative margin on tmax covers (Ize 2013).
__device__ __forceinline__ float slab(const RayPre& r, float lx, float ly, float lz, float hx, float hy, float hz,
                                      float tfar) {
    float tx0 = __fmul_rn(__fsub_rn(lx, r.o.x), r.inv.x), tx1 = __fmul_rn(__fsub_rn(hx, r.o.x), r.inv.x);
    float ty0 = __fmul_rn(__fsub_rn(ly, r.o.y), r.inv.y), ty1 = __fmul_rn(__fsub_rn(hy, r.o.y), r.inv.y);
    float tz0 = __fmul_rn(__fsub_rn(lz, r.o.z), r.inv.z), tz1 = __fmul_rn(__fsub_rn(hz, r.o.z), r.inv.z);
    float tmin = fmaxf(fmaxf(fminf(tx0, tx1), fminf(ty0, ty1)), fmaxf(fminf(tz0, tz1), 0.0f));
    float tmax = fminf(fminf(fmaxf(tx0, tx1), fmaxf(ty0, ty1)), fminf(fmaxf(tz0, tz1), tfar));
    return (tmin <= tmax * 1.0000005f) ? tmin : INFINITY;
}

// watertight test; updates (best_t, best_id) on a nearer hit or an equal-
// distance hit of a lower triangle id
__device__ __forceinline__ void tri_test(const RayPre& r, const float4* __restrict__ tp, int exclude_surf,
                                         float& best_t, int& best_id) {
    // triangles are 48 bytes apart from a 32-byte aligned base: the aligned
    // pair of the three vectors comes in one 32-byte load
    float4 A4, B4, C4;
    if (((reinterpret_cast<uintptr_t>(tp) >> 4) & 1) == 0) {
        ld_v8(tp, A4, B4);
        C4 = __ldg(tp + 2);
    } else {
        A4 = __ldg(tp);
        ld_v8(tp + 1, B4, C4);
    }
    int id = __float_as_int(A4.w);
    // a ray leaving a planar surface cannot meet that plane again
    if (__float_as_int(B4.w) == exclude_surf) return;
    float3 A = make_float3(__fsub_rn(A4.x, r.o.x), __fsub_rn(A4.y, r.o.y), __fsub_rn(A4.z, r.o.z));
    float3 B = make_float3(__fsub_rn(B4.x, r.o.x), __fsub_rn(B4.y, r.o.y), __fsub_rn(B4.z, r.o.z));
    float3 C = make_float3(__fsub_rn(C4.x, r.o.x), __fsub_rn(C4.y, r.o.y), __fsub_rn(C4.z, r.o.z));
    float Akz = comp(A, r.kz), Bkz = comp(B, r.kz), Ckz = comp(C, r.kz);
    float Ax = __fsub_rn(comp(A, r.kx), __fmul_rn(r.Sx, Akz)), Ay = __fsub_rn(comp(A, r.ky), __fmul_rn(r.Sy, Akz));
    float Bx = __fsub_rn(comp(B, r.kx), __fmul_rn(r.Sx, Bkz)), By = __fsub_rn(comp(B, r.ky), __fmul_rn(r.Sy, Bkz));
    float Cx = __fsub_rn(comp(C, r.kx), __fmul_rn(r.Sx, Ckz)), Cy = __fsub_rn(comp(C, r.ky), __fmul_rn(r.Sy, Ckz));
    float U = __fsub_rn(__fmul_rn(Cx, By), __fmul_rn(Cy, Bx));
    float V = __fsub_rn(__fmul_rn(Ax, Cy), __fmul_rn(Ay, Cx));
    float W = __fsub_rn(__fmul_rn(Bx, Ay), __fmul_rn(By, Ax));
    if (U == 0.0f || V == 0.0f || W == 0.0f) {
        double u = __dsub_rn(__dmul_rn((double)Cx, (double)By), __dmul_rn((double)Cy, (double)Bx));
        double v = __dsub_rn(__dmul_rn((double)Ax, (double)Cy), __dmul_rn((double)Ay, (double)Cx));
        double w = __dsub_rn(__dmul_rn((double)Bx, (double)Ay), __dmul_rn((double)By, (double)Ax));
        U = (float)u;
        V = (float)v;
        W = (float)w;
        // keep the sign of tiny non-zero double values
        if (U == 0.0f && u != 0.0) U = u > 0 ? 1e-45f : -1e-45f;
        if (V == 0.0f && v != 0.0) V = v > 0 ? 1e-45f : -1e-45f;
        if (W == 0.0f && w != 0.0) W = w > 0 ? 1e-45f : -1e-45f;
    }
    if ((U < 0.0f || V < 0.0f || W < 0.0f) && (U > 0.0f || V > 0.0f || W > 0.0f)) return;
    float det = __fadd_rn(__fadd_rn(U, V), W);
    if (det == 0.0f) return;
    float Az = __fmul_rn(r.Sz, Akz), Bz = __fmul_rn(r.Sz, Bkz), Cz = __fmul_rn(r.Sz, Ckz);
    float T = __fadd_rn(__fadd_rn(__fmul_rn(U, Az), __fmul_rn(V, Bz)), __fmul_rn(W, Cz));
    if (det < 0.0f) {
        T = -T;
        det = -det;
    }
    if (!(T > 0.0f)) return;
    if (T > best_t * det * 1.000001f) return;  // cheap reject before the division
    float t = __fdiv_rn(T, det);
    if (t < best_t || (t == best_t && id < best_id)) {
        best_t = t;
        best_id = id;
    }
}

// traversal stack in shared memory: STACK_SMEM entries per thread, laid out
// [entry][thread] so that lanes at the same depth hit different banks.  A
// 4-wide node pushes at most 3 entries, so a tree of binary depth D needs at
// most 3 ceil(D / 2) <= 64 entries for D <= 42; deeper trees can overflow,
// which the kernel reports (ST_STACK) instead of writing past the stack.
// A 48-entry variant serves trees of binary depth <= 32 (3 * 16 = 48): it
// leaves more of the SM's unified shared memory / L1 to the cache.
static constexpr int STACK_SMEM = 64;
static constexpr int STACK_SHORT = 48;
static constexpr int STACK_SHORT_MAX_DEPTH = 32;

// compare-exchange of (t, ref) pairs, nearer first
__device__ __forceinline__ void cswap(float& ta, int& ra, float& tb, int& rb) {
    const bool sw = tb < ta;
    const float t = sw ? tb : ta;
    const int r = sw ? rb : ra;
    tb = sw ? ta : tb;
    rb = sw ? ra : rb;
    ta = t;
    ra = r;
}

// Nearest hit over the 4-wide tree, while-while traversal with postponed
// leaves (Aila & Laine 2009): a lane that meets a leaf keeps it aside and
// goes on descending until every lane of the warp holds a leaf, then all
// lanes test triangles together.  At a node the four child boxes are slab-
// tested, sorted by entry distance (a 5-exchange network; misses sort last),
// the nearest is visited next and the other hits are pushed far-to-near.
// Child references: >= 0 internal node, < 0 leaf ~(first_triangle << 3 | count).
template <int BT, int STACK, class Room>
__device__ __forceinline__ void nearest_hit(int step_cap, const Room& rm, const RayPre& r, int exclude,
                                            float& best_t, int& best_id, unsigned int& err, int& n_nodes,
                                            int& n_tests, int* __restrict__ stack) {
    const int SENTINEL = 0x7FFFFFFF;
    int sp = 0;
    int node = 0;
    int leaf = 0;
    int steps = 0;
    best_t = INFINITY;
    best_id = 0x7FFFFFFF;
    while (node != SENTINEL) {
        while ((unsigned)node < (unsigned)SENTINEL) {
            if (++steps > step_cap) {
                err |= ST_STEPS;
                node = SENTINEL;
                leaf = 0;
                break;
            }
            if ((int64_t)node >= rm.n_nodes) {  // never read outside the node array
                err |= ST_BOUNDS;
                node = SENTINEL;
                leaf = 0;
                break;
            }
            const float4* np = rm.nodes + 8 * (int64_t)node;
            float4 lx, ly, lz, hx, hy, hz;  // nodes are 128-byte aligned
            ld_v8(np, lx, ly);
            ld_v8(np + 2, lz, hx);
            ld_v8(np + 4, hy, hz);
            const int4 ref = __ldg(reinterpret_cast<const int4*>(np + 6));
            n_nodes++;
            float t0 = slab(r, lx.x, ly.x, lz.x, hx.x, hy.x, hz.x, best_t);
            float t1 = slab(r, lx.y, ly.y, lz.y, hx.y, hy.y, hz.y, best_t);
            float t2 = slab(r, lx.z, ly.z, lz.z, hx.z, hy.z, hz.z, best_t);
            float t3 = slab(r, lx.w, ly.w, lz.w, hx.w, hy.w, hz.w, best_t);
            int r0 = ref.x, r1 = ref.y, r2 = ref.z, r3 = ref.w;
            cswap(t0, r0, t1, r1);
            cswap(t2, r2, t3, r3);
            cswap(t0, r0, t2, r2);
            cswap(t1, r1, t3, r3);
            cswap(t1, r1, t2, r2);
            if (!(t0 < INFINITY)) {
                node = sp > 0 ? stack[--sp * BT] : SENTINEL;
            } else {
                node = r0;
                const int push = (t1 < INFINITY) + (t2 < INFINITY) + (t3 < INFINITY);
                if (sp + push > STACK) {
                    err |= ST_STACK;
                    node = SENTINEL;
                    leaf = 0;
                    break;
                }
                if (t3 < INFINITY) stack[sp++ * BT] = r3;
                if (t2 < INFINITY) stack[sp++ * BT] = r2;
                if (t1 < INFINITY) stack[sp++ * BT] = r1;
            }
            if (node < 0 && leaf == 0) {  // postpone the leaf, keep descending
                leaf = node;
                node = sp > 0 ? stack[--sp * BT] : SENTINEL;
            }
            if (__all_sync(__activemask(), leaf != 0)) break;
        }
        while (leaf != 0) {
            const int code = ~leaf;
            const int first = code >> 3, cnt = code & 7;
            if ((int64_t)first + cnt > rm.n_tris) {
                err |= ST_BOUNDS;
                node = SENTINEL;
                break;
            }
            for (int k = 0; k < cnt; k++) tri_test(r, rm.tris + 3 * (int64_t)(first + k), exclude, best_t, best_id);
            n_tests += cnt;
            leaf = 0;
            if (node < 0) {  // a leaf popped from the stack
                leaf = node;
                node = sp > 0 ? stack[--sp * BT] : SENTINEL;
            }
        }
    }
    if (best_id == 0x7FFFFFFF) best_id = -1;
}

}  // namespace rr
