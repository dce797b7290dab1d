// rt_trace.cu -- rt_trace: batched ray propagation and image sources.
//
// Wavefront design: all live rays of one bounce are processed by one fused
// kernel launch (k_bounce) that, per ray,
//   1. finds the nearest triangle through the LBVH (paper Sec. 2.1-2.2):
//      stack traversal, nearest child first, robust slab test (Williams et
//      al. 2005 with the conservative rounding margin of Ize 2013) and the
//      watertight ray/triangle test of Woop, Benthin & Wald (JCGT 2013) in
//      float32 (edge functions recomputed in double only when exactly 0);
//      exact distance ties go to the lowest triangle id;
//   2. tests the segment against the measurement spheres of its source
//      (eq. 22) and appends crossing records with one atomic per warp;
//   3. reflects specularly (eq. 15: u - 2 (u.n) n), multiplies the 8 band
//      energies by 1 - alpha(f) (eq. 16), adds the segment length to the path
//      length with a compensated (Kahan) sum, folds the surface id into the
//      ray's sequence hash, and starts the next segment a few ulps before
//      the hit point along the incoming ray (inside every wall that meets
//      the hit surface, so corner hits cannot leak), while candidates on
//      the surface just left are skipped (a ray leaving a plane cannot meet
//      it again), which makes an offset along the normal unnecessary;
//   4. compacts survivors into the next queue (warp ballot + popc, one
//      atomic per warp); rays that escape (open air, Sec. 2.1), reach the
//      bounce cap or exceed the eq. 13 range write their final state.
// Warps fetch 32 rays at a time from a per-bounce counter (persistent
// grid), and the live count of each bounce stays in device memory, so the
// B launches need no host round trip.
//
// Image sources (Sec. 1.4, eq. 19): records are radix-sorted by a 64-bit key
// of (receiver, order, sequence hash); equal keys are verified against the
// exact surface sequences read from the per-ray hit history; each segment
// of equal keys is one image source with n = segment length.  Its position
// is the source mirrored across the sequence's FP64 planes in hit order;
// distance, arrival time and E_s(f) = (n/N) prod(1 - alpha_j(f)) e^(-beta d)
// are computed in FP64.
#include "rt_internal.cuh"

#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <cctype>
#include <cstdio>
#include <unistd.h>

namespace rr {

static constexpr int DEFAULT_NODE_VISITS = 1 << 16;


struct Queue {
    float4* o;   // origin xyz, path length L
    float4* d;   // direction xyz, Kahan compensation of L
    float4* e0;  // band energies 0..3
    float4* e1;  // band energies 4..7
    uint4* m;    // traced ray index, last surface id, sequence hash lo, hi
};

// Per-room device tables: the tree of the room and where its materials start
// in the concatenated absorption table.  A single-room trace has one entry.
struct RoomDev {
    const float4* nodes;
    const float4* tris;
    const float4* tri_nrm;
    const int32_t* mat_of_surf;
    const int32_t* surf_of;
    const Plane* planes;
    const int32_t* pos_of;  // triangle id -> position in tree order
    int64_t n_nodes, n_tris;
    int32_t mat_base;
    int32_t pad;
};

struct BounceArgs {
    const RoomDev* __restrict__ rooms;
    const int32_t* __restrict__ room_of_src;  // [S] room of each source
    const float* __restrict__ refl;      // [sum of n_mat][8] 1 - alpha
    const float4* __restrict__ rcv;      // [R] centre, r^2 (sorted by source)
    const int32_t* __restrict__ rcv_id;  // [R] original receiver index
    const int32_t* __restrict__ rcv_beg; // [S+1] receiver range per source
    Queue in, out;
    int32_t* __restrict__ hist;          // [B][n_traced]
    float4* __restrict__ ray_e;          // [n_traced][2]
    float* __restrict__ ray_len;
    int32_t* __restrict__ ray_hits;
    int32_t* __restrict__ rec_rcv;
    int32_t* __restrict__ rec_ray;
    int32_t* __restrict__ rec_m;
    float* __restrict__ rec_len;
    uint64_t* __restrict__ rec_key;
    unsigned long long rec_cap;
    unsigned int* live;                  // [B+1]
    unsigned int* fetch;                 // [B]
    unsigned long long* n_rec;
    unsigned int* status;
    int64_t n_traced;
    int64_t per_src;                     // rays per source traced
    int b, B;                            // first bounce of this launch, bounces of the trace
    int launch, b_end;                   // counter index of this launch; its survivors are compacted at b_end
    unsigned int tail_threshold;         // live rays at or below which one launch finishes the trace
    unsigned long long* n_queries;
    int step_cap;                        // node visits per query
    float dmax;                          // <= 0: off
    float* debug_t;
    float* debug_state;
    int32_t* debug_cost;
    const int32_t* __restrict__ replay;  // [B][n_traced] hits of an earlier trace of the same rays, or null
};

// ---------------------------------------------------------------------------
// hashing of reflection sequences (MurmurHash3 64-bit finalizer, Appleby)
// ---------------------------------------------------------------------------
__host__ __device__ __forceinline__ uint64_t fmix64(uint64_t k) {
    k ^= k >> 33;
    k *= 0xff51afd7ed558ccdULL;
    k ^= k >> 33;
    k *= 0xc4ceb9fe1a85ec53ULL;
    k ^= k >> 33;
    return k;
}
static constexpr uint64_t HASH0 = 0x243F6A8885A308D3ULL;
__device__ __forceinline__ uint64_t hash_step(uint64_t h, int32_t surf) {
    return fmix64(h + (uint64_t)(uint32_t)(surf + 1) * 0x9E3779B97F4A7C15ULL);
}
__device__ __forceinline__ uint64_t record_key(uint64_t h, int32_t rcv, int32_t m) {
    return fmix64(h ^ ((((uint64_t)(uint32_t)rcv << 32) | (uint32_t)m) * 0xD6E8FEB86659FD93ULL + 1ULL));
}

// ---------------------------------------------------------------------------
// ray generation: Fibonacci rule (Sec. 1.2) in FP64, rounded to float32.
// z_i = 1 - (2i+1)/N, rho = sqrt(1 - z^2), phi = 2 pi frac(i g), g = (3-sqrt5)/2.
// Explicit _rn intrinsics keep every operation rounded as written.
// ---------------------------------------------------------------------------
__device__ __forceinline__ float3 fibonacci_dir(int64_t i, int64_t N, double g) {
    double z = __dsub_rn(1.0, __ddiv_rn((double)(2 * i + 1), (double)N));
    double rho = __dsqrt_rn(__dsub_rn(1.0, __dmul_rn(z, z)));
    double f = __dmul_rn((double)i, g);
    f = __dsub_rn(f, floor(f));
    double phi = __dmul_rn(6.283185307179586, f);
    double s, c;
    sincos(phi, &s, &c);
    return make_float3((float)__dmul_rn(rho, c), (float)__dmul_rn(rho, s), (float)z);
}

// Directional source (Sec. 1.2, footnote: a non-uniform spatial sampling):
// equal-energy rays with density (1 - a + a mu) / (2 (1 - a)) in mu = cos of
// the angle to the unit axis w, 0 <= a <= 1/2.  The uniform rule's z, as
// u = (1 + z) / 2, goes through the inverse cumulative: the root of
// (a/2) mu^2 + (1 - a) mu + (1 - a) - a/2 - 2 (1 - a) u = 0 in [-1, 1], taken
// as mu = -2 C / (B + sqrt(B^2 - 2 a C)) (no cancellation as a -> 0); a = 0
// keeps mu = z.  The direction is then turned from +z to w with the
// orthonormal basis of Duff et al. 2017.  One rounded FP64 operation per step,
// in the same order as the FP64 reference, so the float32 directions agree.
__device__ __forceinline__ float3 directional_dir(int64_t i, int64_t N, const double* w, double a, double g) {
    const double z = __dsub_rn(1.0, __ddiv_rn((double)(2 * i + 1), (double)N));
    double mu = z;
    if (a > 0.0) {
        const double uu = __ddiv_rn(__dadd_rn(1.0, z), 2.0);
        const double B = __dsub_rn(1.0, a);
        const double C = __dsub_rn(__dsub_rn(B, __ddiv_rn(a, 2.0)), __dmul_rn(__dmul_rn(2.0, B), uu));
        const double D = __dsub_rn(__dmul_rn(B, B), __dmul_rn(__dmul_rn(2.0, a), C));
        mu = __ddiv_rn(__dmul_rn(-2.0, C), __dadd_rn(B, __dsqrt_rn(D)));
    }
    const double rho = __dsqrt_rn(__dsub_rn(1.0, __dmul_rn(mu, mu)));
    double f = __dmul_rn((double)i, g);
    f = __dsub_rn(f, floor(f));
    const double phi = __dmul_rn(6.283185307179586, f);
    double sn, cs;
    sincos(phi, &sn, &cs);
    const double cx = __dmul_rn(rho, cs), cy = __dmul_rn(rho, sn);
    const double sg = w[2] >= 0.0 ? 1.0 : -1.0;
    const double A = __ddiv_rn(-1.0, __dadd_rn(sg, w[2]));
    const double Bq = __dmul_rn(__dmul_rn(w[0], w[1]), A);
    const double t1[3] = {__dadd_rn(1.0, __dmul_rn(__dmul_rn(__dmul_rn(sg, w[0]), w[0]), A)), __dmul_rn(sg, Bq),
                          -__dmul_rn(sg, w[0])};
    const double t2[3] = {Bq, __dadd_rn(sg, __dmul_rn(__dmul_rn(w[1], w[1]), A)), -w[1]};
    float u[3];
    for (int k = 0; k < 3; k++)
        u[k] = (float)__dadd_rn(__dadd_rn(__dmul_rn(cx, t1[k]), __dmul_rn(cy, t2[k])), __dmul_rn(mu, w[k]));
    return make_float3(u[0], u[1], u[2]);
}

// g = (3 - sqrt 5) / 2 of the Fibonacci rule, formed once on the host: IEEE
// square root, subtraction and division round the same way there as in the
// FP64 steps of the device code, so the value is the same double.
static const double GOLDEN_G = (3.0 - std::sqrt(5.0)) / 2.0;

// Queue order of the primary rays: Fibonacci indices j, j+F, j+2F, ... (F a
// Fibonacci number near sqrt(count)) lie along one spiral arm of the lattice,
// so consecutive queue slots (one warp) get neighbouring directions.  The
// map slot -> index is a bijection of [0, count); results do not depend on it.
__device__ __forceinline__ int64_t coherent_offset(int64_t r, int64_t count, int64_t F) {
    const int64_t q = count / F, rem = count % F;
    int64_t j, k;
    if (r < rem * (q + 1)) {
        j = r / (q + 1);
        k = r % (q + 1);
    } else {
        const int64_t r2 = r - rem * (q + 1);
        j = rem + r2 / q;
        k = r2 % q;
    }
    return j + k * F;
}

__global__ void k_gen_rays(Queue q, const float* __restrict__ src, const double* __restrict__ srcdir,
                           int64_t n_traced, int64_t per_src, int64_t ray_begin, int64_t N, int64_t F, double g) {
    int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n_traced) return;
    int64_t s = r / per_src;
    int64_t off = coherent_offset(r % per_src, per_src, F);
    int64_t i = ray_begin + off;
    float3 u;
    if (srcdir && srcdir[4 * s + 3] >= 0.0)
        u = directional_dir(i, N, srcdir + 4 * s, srcdir[4 * s + 3], g);
    else
        u = fibonacci_dir(i, N, g);
    float e = (float)(1.0 / (double)N);
    q.o[r] = make_float4(src[3 * s], src[3 * s + 1], src[3 * s + 2], 0.f);
    q.d[r] = make_float4(u.x, u.y, u.z, 0.f);
    q.e0[r] = make_float4(e, e, e, e);
    q.e1[r] = make_float4(e, e, e, e);
    q.m[r] = make_uint4((unsigned)(s * per_src + off), 0xFFFFFFFFu, (unsigned)(HASH0 & 0xFFFFFFFFu),
                        (unsigned)(HASH0 >> 32));
}

}  // namespace rr

#include "rt_traverse.cuh"

namespace rr {

// Replay of a recorded query: the triangle an earlier trace of this ray hit
// at this bounce is tested alone (the same watertight test, so the same
// distance); -1 (an escape) stays an escape.  Ids outside the mesh are
// reported (ST_BOUNDS) and read as escapes.
__device__ __forceinline__ void replay_hit(const BounceArgs& a, const RoomDev& rm, const RayPre& r, int exclude,
                                           int bb, int q, float& best_t, int& best_id, unsigned int& err,
                                           int& n_tests) {
    best_t = INFINITY;
    best_id = 0x7FFFFFFF;
    const int tri = a.replay[(int64_t)bb * a.n_traced + q];
    if (tri >= 0) {
        const int j = (int64_t)tri < rm.n_tris ? rm.pos_of[tri] : -1;
        if (j < 0 || (int64_t)j >= rm.n_tris) {
            err |= ST_BOUNDS;
        } else {
            tri_test(r, rm.tris + 3 * (int64_t)j, exclude, best_t, best_id);
            n_tests = 1;
        }
    }
    if (best_id == 0x7FFFFFFF) best_id = -1;
}

struct RayState {
    float4 o, d, e0, e1;
    uint4 m;
};

__device__ __forceinline__ void load_ray(const Queue& q, unsigned int slot, RayState& s) {
    s.o = q.o[slot];
    s.d = q.d[slot];
    s.e0 = q.e0[slot];
    s.e1 = q.e1[slot];
    s.m = q.m[slot];
}

// One bounce of the ray in s (bounce index bb).  Every lane of the warp calls
// it; lanes without a ray pass active = false.  Returns true if the ray goes on.
template <int BT, bool REPLAY, int STACK>
__device__ __forceinline__ bool step_ray(const BounceArgs& a, int lane, bool active, int bb, RayState& s,
                                         int* __restrict__ stack) {
    const int q = (int)s.m.x;
    const int src = active ? (int)(q / a.per_src) : 0;
    const RoomDev& rm = a.rooms[active ? a.room_of_src[src] : 0];
    float best_t = INFINITY;
    int hit = -1;
    unsigned int err = 0;
    float4 o4 = s.o, d4 = s.d;
    RayPre rp = ray_pre(make_float3(o4.x, o4.y, o4.z), make_float3(d4.x, d4.y, d4.z));
    int n_nodes = 0, n_tests = 0;
    if (active) {
        if (REPLAY)  // the query re-tests the triangle an earlier trace recorded
            replay_hit(a, rm, rp, (int)s.m.y, bb, q, best_t, hit, err, n_tests);
        else
            nearest_hit<BT, STACK>(a.step_cap, rm, rp, (int)s.m.y, best_t, hit, err, n_nodes, n_tests, stack);
    }
    if (err) atomicOr(a.status, err);
    const unsigned int amask = __ballot_sync(0xffffffffu, active);
    if (lane == 0 && amask) atomicAdd(a.n_queries, (unsigned long long)__popc(amask));
    const float seg = hit >= 0 ? best_t : INFINITY;
    // -- measurement spheres of this ray's source (eq. 22) -----------------
    // each sphere test is evaluated once; crossings of one receiver slot are
    // appended with one atomic per warp
    const int rb = active ? a.rcv_beg[src] : 0;
    const int nk = active ? a.rcv_beg[src + 1] - rb : 0;
    const int nk_max = __reduce_max_sync(0xffffffffu, (unsigned)nk);
    const uint64_t hseq = ((uint64_t)s.m.w << 32) | s.m.z;
    for (int j = 0; j < nk_max; j++) {
        bool x = false;
        float lc = 0.f;
        int rid = 0;
        if (j < nk) {
            float4 c = __ldg(a.rcv + rb + j);
            float wx = c.x - o4.x, wy = c.y - o4.y, wz = c.z - o4.z;
            float ts = fminf(fmaxf(wx * d4.x + wy * d4.y + wz * d4.z, 0.0f), seg);
            float qx = fmaf(ts, d4.x, o4.x) - c.x, qy = fmaf(ts, d4.y, o4.y) - c.y, qz = fmaf(ts, d4.z, o4.z) - c.z;
            lc = o4.w + ts;
            x = (qx * qx + qy * qy + qz * qz <= c.w) && (a.dmax <= 0.0f || lc <= a.dmax);
            rid = __ldg(a.rcv_id + rb + j);
        }
        const unsigned int msk = __ballot_sync(0xffffffffu, x);
        if (msk) {
            const int leader = __ffs(msk) - 1;
            unsigned long long rbase = 0;
            if (lane == leader) rbase = atomicAdd(a.n_rec, (unsigned long long)__popc(msk));
            rbase = __shfl_sync(0xffffffffu, rbase, leader);
            const unsigned long long pos = rbase + __popc(msk & ((1u << lane) - 1u));
            if (x && pos < a.rec_cap) {
                a.rec_rcv[pos] = rid;
                a.rec_ray[pos] = q;
                a.rec_m[pos] = bb;
                a.rec_len[pos] = lc;
                a.rec_key[pos] = record_key(hseq, rid, bb);
            }
        }
    }
    if (!active) return false;
    bool survive = false;
    const int64_t hb = (int64_t)bb * a.n_traced + q;
    a.hist[hb] = hit;
    if (a.debug_t) a.debug_t[hb] = seg;
    if (a.debug_cost) {
        a.debug_cost[2 * hb] = n_nodes;
        a.debug_cost[2 * hb + 1] = n_tests;
    }
    if (a.debug_state) {
        float* ds = a.debug_state + hb * 6;
        ds[0] = o4.x, ds[1] = o4.y, ds[2] = o4.z, ds[3] = d4.x, ds[4] = d4.y, ds[5] = d4.z;
    }
    if (hit >= 0) {
        // reflect (eq. 15), absorb (eq. 16), path length (Kahan), hash
        float4 nr = __ldg(rm.tri_nrm + hit);
        int surf = __float_as_int(nr.w);
        float dn = d4.x * nr.x + d4.y * nr.y + d4.z * nr.z;
        // next origin: the hit point pulled back along the incoming ray by
        // about four ulps of the largest coordinate
        float px = fmaf(best_t, d4.x, o4.x), py = fmaf(best_t, d4.y, o4.y), pz = fmaf(best_t, d4.z, o4.z);
        float scale = fmaxf(fmaxf(fabsf(px), fabsf(py)), fmaxf(fabsf(pz), 1e-3f));
        float tb = fmaxf(best_t - scale * 4.76837158e-7f, 0.0f);  // 2^-21
        o4.x = fmaf(tb, d4.x, o4.x);
        o4.y = fmaf(tb, d4.y, o4.y);
        o4.z = fmaf(tb, d4.z, o4.z);
        float rx = d4.x - 2.0f * dn * nr.x, ry = d4.y - 2.0f * dn * nr.y, rz = d4.z - 2.0f * dn * nr.z;
        float inv = rsqrtf(rx * rx + ry * ry + rz * rz);
        float y = best_t - d4.w;
        float t = o4.w + y;
        d4.w = (t - o4.w) - y;
        o4.w = t;
        d4.x = rx * inv;
        d4.y = ry * inv;
        d4.z = rz * inv;
        const float* rf = a.refl + 8 * (rm.mat_base + rm.mat_of_surf[surf]);
        s.e0.x *= __ldg(rf + 0);
        s.e0.y *= __ldg(rf + 1);
        s.e0.z *= __ldg(rf + 2);
        s.e0.w *= __ldg(rf + 3);
        s.e1.x *= __ldg(rf + 4);
        s.e1.y *= __ldg(rf + 5);
        s.e1.z *= __ldg(rf + 6);
        s.e1.w *= __ldg(rf + 7);
        uint64_t h = hash_step(hseq, surf);
        s.m.y = (unsigned int)surf;
        s.m.z = (unsigned int)(h & 0xFFFFFFFFu);
        s.m.w = (unsigned int)(h >> 32);
        s.o = o4;
        s.d = d4;
        survive = (bb + 1 < a.B) && !(a.dmax > 0.0f && o4.w > a.dmax) && !err;
    }
    if (!survive) {
        a.ray_e[2 * (int64_t)q] = s.e0;
        a.ray_e[2 * (int64_t)q + 1] = s.e1;
        a.ray_len[q] = s.o.w;
        a.ray_hits[q] = bb + (hit >= 0 ? 1 : 0);
    }
    return survive;
}

// ---------------------------------------------------------------------------
// the bounce kernel: launch k steps the rays of its input queue from bounce
// a.b (= k P for a compaction period P) and compacts the survivors at a.b_end
//   wavefront mode (P = 1, live rays > tail threshold): one bounce per ray,
//   survivors compacted into the next queue with one atomic per warp;
//   period mode (P > 1, live rays > tail threshold): each lane steps its ray
//   up to b_end and takes a new one as soon as its ray dies or is written
//   to the next queue (compaction every P bounces);
//   tail mode (few live rays): this launch finishes every remaining bounce,
//   lanes whose ray dies fetch the next one, so the last bounces do not each
//   wait for their slowest ray.  It writes no survivors, so the later
//   launches of the same trace find no live rays and return at once.
// ---------------------------------------------------------------------------
template <int BT, bool REPLAY, int STACK>
__global__ void __launch_bounds__(BT) k_bounce(BounceArgs a) {
    extern __shared__ int s_stack[];  // STACK * BT entries (stack_bytes)
    int* stack = s_stack + threadIdx.x;
    const int lane = threadIdx.x & 31;
    const int k = a.launch;
    const unsigned int n_live = a.live[k];
    const int b = a.b;
    if (n_live == 0) return;
    const bool tail = n_live <= a.tail_threshold;
    if (!tail && a.b_end == b + 1) {
        for (;;) {
            unsigned int base = 0;
            if (lane == 0) base = atomicAdd(&a.fetch[k], 32u);
            base = __shfl_sync(0xffffffffu, base, 0);
            if (base >= n_live) break;
            const unsigned int slot = base + lane;
            const bool active = slot < n_live;
            RayState s;
            s.o = make_float4(0, 0, 0, 0);
            s.d = make_float4(0, 0, 1, 0);
            s.e0 = s.e1 = s.o;
            s.m = make_uint4(0, 0xFFFFFFFFu, 0, 0);
            if (active) load_ray(a.in, slot, s);
            const bool survive = step_ray<BT, REPLAY, STACK>(a, lane, active, b, s, stack);
            const unsigned int mask = __ballot_sync(0xffffffffu, survive);
            if (mask) {
                unsigned int obase = 0;
                const int leader = __ffs(mask) - 1;
                if (lane == leader) obase = atomicAdd(&a.live[k + 1], (unsigned int)__popc(mask));
                obase = __shfl_sync(0xffffffffu, obase, leader);
                if (survive) {
                    unsigned int p = obase + __popc(mask & ((1u << lane) - 1u));
                    a.out.o[p] = s.o;
                    a.out.d[p] = s.d;
                    a.out.e0[p] = s.e0;
                    a.out.e1[p] = s.e1;
                    a.out.m[p] = s.m;
                }
            }
        }
        return;
    }
    // period mode and tail mode: per-lane refill
    const int end = tail ? a.B : a.b_end;
    RayState s;
    s.o = make_float4(0, 0, 0, 0);
    s.d = make_float4(0, 0, 1, 0);
    s.e0 = s.e1 = s.o;
    s.m = make_uint4(0, 0xFFFFFFFFu, 0, 0);
    bool has = false, exhausted = false;
    int bb = b;
    for (int iter = 0; iter < 1 << 30; iter++) {
        const unsigned int need = __ballot_sync(0xffffffffu, !has);
        if (need && !exhausted) {
            unsigned int base = 0;
            const int leader = __ffs(need) - 1;
            if (lane == leader) base = atomicAdd(&a.fetch[k], (unsigned int)__popc(need));
            base = __shfl_sync(0xffffffffu, base, leader);
            if (!has) {
                const unsigned int slot = base + __popc(need & ((1u << lane) - 1u));
                if (slot < n_live) {
                    load_ray(a.in, slot, s);
                    bb = b;
                    has = true;
                }
            }
            exhausted = base + __popc(need) >= n_live;
        }
        if (__ballot_sync(0xffffffffu, has) == 0) break;
        const bool survive = step_ray<BT, REPLAY, STACK>(a, lane, has, bb, s, stack);
        bool write = false;
        if (has) {
            if (survive) {
                bb++;
                write = bb == end;  // end < B here: a ray alive at B has no next bounce
            } else {
                has = false;
            }
        }
        const unsigned int wmask = __ballot_sync(0xffffffffu, write);
        if (wmask) {  // survivors of this launch's bounce range: compact into the next queue
            unsigned int obase = 0;
            const int leader = __ffs(wmask) - 1;
            if (lane == leader) obase = atomicAdd(&a.live[k + 1], (unsigned int)__popc(wmask));
            obase = __shfl_sync(0xffffffffu, obase, leader);
            if (write) {
                const unsigned int p = obase + __popc(wmask & ((1u << lane) - 1u));
                a.out.o[p] = s.o;
                a.out.d[p] = s.d;
                a.out.e0[p] = s.e0;
                a.out.e1[p] = s.e1;
                a.out.m[p] = s.m;
                has = false;
            }
        }
    }
}

// ---------------------------------------------------------------------------
// image sources
// ---------------------------------------------------------------------------
// Sort keys of the records: the reflection order (capped at 31) in the top 5
// bits above 59 bits of the record hash, so that the image sources come out
// grouped by order and the lanes of a reconstruction warp mirror the source
// about the same number of planes.  Equal keys of different beams (a 59-bit
// collision) are caught by the exact sequence comparison of k_seg_flags.
__global__ void k_dedup_init(const uint64_t* __restrict__ rec_key, const int32_t* __restrict__ rec_m, int64_t n,
                             uint64_t* __restrict__ keys, uint32_t* __restrict__ vals) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const uint64_t m = (uint64_t)min(max(rec_m[i], 0), 31);
    keys[i] = (m << 59) | (rec_key[i] >> 5);
    vals[i] = (uint32_t)i;
}

__device__ __forceinline__ bool same_beam(int64_t ra, int64_t rb, const int32_t* rec_rcv, const int32_t* rec_ray,
                                          const int32_t* rec_m, const int32_t* hist, const RoomDev* rooms,
                                          const int32_t* room_of_rcv, int64_t n_traced) {
    if (rec_rcv[ra] != rec_rcv[rb] || rec_m[ra] != rec_m[rb]) return false;
    const int32_t* surf_of = rooms[room_of_rcv[rec_rcv[ra]]].surf_of;
    int m = rec_m[ra];
    int64_t qa = rec_ray[ra], qb = rec_ray[rb];
    for (int k = 0; k < m; k++) {
        int ta = hist[(int64_t)k * n_traced + qa], tb = hist[(int64_t)k * n_traced + qb];
        if (ta < 0 || tb < 0 || surf_of[ta] != surf_of[tb]) return false;
    }
    return true;
}

__global__ void k_seg_flags(const uint64_t* __restrict__ keys, const uint32_t* __restrict__ vals, int64_t n,
                            const int32_t* __restrict__ rec_rcv, const int32_t* __restrict__ rec_ray,
                            const int32_t* __restrict__ rec_m, const int32_t* __restrict__ hist,
                            const RoomDev* __restrict__ rooms, const int32_t* __restrict__ room_of_rcv,
                            int64_t n_traced, uint32_t* __restrict__ flags, unsigned long long* collisions) {
    int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    uint32_t f = 1;
    if (j > 0 && keys[j] == keys[j - 1]) {
        f = 0;
        if (!same_beam(vals[j - 1], vals[j], rec_rcv, rec_ray, rec_m, hist, rooms, room_of_rcv, n_traced)) {
            f = 1;
            atomicAdd(collisions, 1ull);
        }
    }
    flags[j] = f;
}

// lowest ray index of every beam (atomicMin over the beam's records); the
// exclusive scan of the head flags gives a record's beam as segid + flag - 1
// lowest ray of each segment; the records of a segment are adjacent, so the
// lanes of a warp that share one reduce first and send one atomic
__global__ void k_seg_min(const uint32_t* __restrict__ vals, const uint32_t* __restrict__ flags,
                          const uint32_t* __restrict__ segid, int64_t n, const int32_t* __restrict__ rec_ray,
                          int32_t* __restrict__ rep) {
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int lane = threadIdx.x & 31;
    const uint32_t seg = j < n ? segid[j] + flags[j] - 1u : 0xFFFFFFFFu;
    const int32_t ray = j < n ? rec_ray[vals[j]] : INT_MAX;
    const unsigned int peers = __match_any_sync(0xffffffffu, seg);
    const int32_t lo = __reduce_min_sync(peers, ray);
    if (j < n && (peers & ((1u << lane) - 1u)) == 0) atomicMin(rep + seg, lo);
}

__global__ void k_seg_heads(const uint32_t* __restrict__ flags, const uint32_t* __restrict__ segid, int64_t n,
                            uint32_t* __restrict__ heads) {
    int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    if (flags[j]) heads[segid[j]] = (uint32_t)j;
    if (j == n - 1) heads[segid[j] + flags[j]] = (uint32_t)n;
}

struct ReconArgs {
    const uint32_t* heads;
    const uint32_t* vals;
    const unsigned int* n_unique_dev;
    unsigned int* status;
    const int32_t* rec_rcv;
    const int32_t* rec_ray;
    const int32_t* rec_m;
    const int32_t* hist;
    const RoomDev* rooms;
    const int32_t* room_of_rcv;
    const double* refl64;    // [sum of n_mat][8] 1 - alpha (FP64, formed on the host)
    const double* beta64;    // [8]
    const double* src64;     // [S][3]
    const double* rcv64;     // [R][3] by original receiver id
    int64_t n_traced, per_src;
    double N, c;
    int32_t *o_rcv, *o_order, *o_count, *o_rep;
    double *o_pos, *o_dist, *o_time, *o_energy;
};

// one thread per image source: beam size, representative ray, FP64 mirror chain
static constexpr int RECON_GROUP = 4;

__global__ void k_reconstruct(ReconArgs a) {
    const unsigned int u = blockIdx.x * blockDim.x + threadIdx.x;
    if (u >= *a.n_unique_dev) return;
    const uint32_t lo = a.heads[u], hi = a.heads[u + 1];
    const int32_t rep = a.o_rep[u];  // set by k_seg_min
    const uint32_t r0 = a.vals[lo];
    const int32_t rcv = a.rec_rcv[r0], m = a.rec_m[r0];
    const RoomDev& rm = a.rooms[a.room_of_rcv[rcv]];
    const int64_t s = rep / a.per_src;
    double x = a.src64[3 * s], y = a.src64[3 * s + 1], z = a.src64[3 * s + 2];
    double prod[RT_N_BANDS];
#pragma unroll
    for (int f = 0; f < RT_N_BANDS; f++) prod[f] = 1.0;
    // the sequence is read RECON_GROUP reflections at a time: the history,
    // surface and plane loads of a group are independent of one another, so
    // they are issued together instead of one dependent chain per reflection
    bool ok = true;
    for (int k0 = 0; k0 < m && ok; k0 += RECON_GROUP) {
        int tri[RECON_GROUP], sid[RECON_GROUP];
#pragma unroll
        for (int j = 0; j < RECON_GROUP; j++)
            tri[j] = k0 + j < m ? a.hist[(int64_t)(k0 + j) * a.n_traced + rep] : 0;
#pragma unroll
        for (int j = 0; j < RECON_GROUP; j++) sid[j] = tri[j] >= 0 ? rm.surf_of[tri[j]] : 0;
        Plane P[RECON_GROUP];
        int mt[RECON_GROUP];
#pragma unroll
        for (int j = 0; j < RECON_GROUP; j++) {
            P[j] = rm.planes[sid[j]];
            mt[j] = rm.mat_of_surf[sid[j]];
        }
#pragma unroll
        for (int j = 0; j < RECON_GROUP; j++) {
            if (k0 + j >= m) break;
            if (tri[j] < 0) {  // cannot happen for a consistent history; reported, never read
                atomicOr(a.status, ST_HISTORY);
                ok = false;
                break;
            }
            double dist = P[j].x * x + P[j].y * y + P[j].z * z - P[j].w;
            x -= 2.0 * dist * P[j].x;
            y -= 2.0 * dist * P[j].y;
            z -= 2.0 * dist * P[j].z;
            const double* rf = a.refl64 + 8 * (rm.mat_base + mt[j]);
#pragma unroll
            for (int f = 0; f < RT_N_BANDS; f++) prod[f] *= rf[f];
        }
    }
    const double* xm = a.rcv64 + 3 * rcv;
    double dx = x - xm[0], dy = y - xm[1], dz = z - xm[2];
    double d = sqrt(dx * dx + dy * dy + dz * dz);
    double n = (double)(hi - lo);
    a.o_rcv[u] = rcv;
    a.o_order[u] = m;
    a.o_count[u] = (int32_t)(hi - lo);
    a.o_pos[3 * (int64_t)u] = x;
    a.o_pos[3 * (int64_t)u + 1] = y;
    a.o_pos[3 * (int64_t)u + 2] = z;
    a.o_dist[u] = d;
    a.o_time[u] = d / a.c;
#pragma unroll
    for (int f = 0; f < RT_N_BANDS; f++) a.o_energy[8 * (int64_t)u + f] = (n / a.N) * prod[f] * exp(-a.beta64[f] * d);
}

static unsigned grid_of(int64_t n, int threads) { return (unsigned)((n + threads - 1) / threads); }

// ---------------------------------------------------------------------------
// host driver
// ---------------------------------------------------------------------------
static rt_status alloc_queue(Arena& ar, Queue& q, int64_t n) {
    RR_TRY(ar.alloc(&q.o, n));
    RR_TRY(ar.alloc(&q.d, n));
    RR_TRY(ar.alloc(&q.e0, n));
    RR_TRY(ar.alloc(&q.e1, n));
    RR_TRY(ar.alloc(&q.m, n));
    return RT_OK;
}

// -- bounce-kernel configurations and the online autotuner -------------------
// A configuration is a block size, a tail threshold (never / resident
// threads / every ray), a compaction period (bounces each launch runs before
// it compacts the survivors) and a traversal stack depth (64 entries, or 48
// for trees of binary depth <= 32; a deeper tree runs the 48-entry
// candidates with 64).  Every configuration gives identical results per ray,
// so the autotuner times the real calls: the first calls of a workload class
// each run the next candidate, every candidate twice (the faster time counts,
// which keeps one noisy call from deciding), and then the fastest is kept
// (optionally persisted in the file named by RT_AUTOTUNE_CACHE).
struct Config {
    int block;
    int tail_mode;  // 0 never, 1 resident threads, 2 every ray
    int period;     // compaction period: bounces per launch above the tail threshold
    int stack;      // traversal stack entries (STACK_SHORT only for trees it provably fits)
};
static const Config CANDIDATES[] = {{128, 2, 1, STACK_SMEM},  {256, 2, 1, STACK_SMEM}, {128, 2, 1, STACK_SHORT},
                                    {256, 2, 1, STACK_SHORT}, {128, 1, 1, STACK_SMEM}, {128, 1, 4, STACK_SMEM},
                                    {128, 0, 1, STACK_SMEM},  {128, 0, 4, STACK_SMEM}, {256, 0, 8, STACK_SHORT}};
static constexpr int N_CANDIDATES = sizeof(CANDIDATES) / sizeof(CANDIDATES[0]);
static constexpr int TUNE_ROUNDS = 2;

struct TuneState {
    float ms[N_CANDIDATES];
    int next = 0;
    int best = -1;
};
static std::mutex g_tune_mu;
static std::map<std::string, TuneState> g_tune;
static bool g_tune_loaded = false;

static void tune_load_locked() {
    if (g_tune_loaded) return;
    g_tune_loaded = true;
    const char* path = getenv("RT_AUTOTUNE_CACHE");
    if (!path) return;
    FILE* f = fopen(path, "r");
    if (!f) return;
    char key[256];
    int best;
    while (fscanf(f, "%255s %d", key, &best) == 2) {
        if (best >= 0 && best < N_CANDIDATES) {
            TuneState t;
            t.next = TUNE_ROUNDS * N_CANDIDATES;
            t.best = best;
            for (float& x : t.ms) x = 0.f;
            g_tune[key] = t;
        }
    }
    fclose(f);
}

// the whole table, written to a temporary file and renamed over the cache,
// so that another process never reads a half-written file
static void tune_save_locked() {
    const char* path = getenv("RT_AUTOTUNE_CACHE");
    if (!path) return;
    const std::string tmp = std::string(path) + ".tmp" + std::to_string((long long)getpid());
    FILE* f = fopen(tmp.c_str(), "w");
    if (!f) return;
    for (auto& kv : g_tune)
        if (kv.second.best >= 0) fprintf(f, "%s %d\n", kv.first.c_str(), kv.second.best);
    if (fclose(f) != 0 || rename(tmp.c_str(), path) != 0) remove(tmp.c_str());
}

// workload class: the device model (a cache written on another GPU does not
// apply), the candidate list's size (a changed list invalidates the stored
// indices), rooms, and the tree size, ray count and bounce count
static std::string tune_key(int64_t n_tris, int64_t n_traced, int B, int n_rooms) {
    int dev = 0;
    cudaGetDevice(&dev);
    static std::mutex name_mu;
    static std::string names[64];
    std::string name = "unknown";
    if (dev >= 0 && dev < 64) {
        std::lock_guard<std::mutex> lk(name_mu);
        if (names[dev].empty()) {
            cudaDeviceProp prop;
            std::string n = "unknown";
            if (cudaGetDeviceProperties(&prop, dev) == cudaSuccess) n = prop.name;
            cudaGetLastError();
            for (char& c : n)
                if (!isalnum((unsigned char)c)) c = '-';
            names[dev] = n;
        }
        name = names[dev];
    }
    auto lg = [](int64_t x) {
        int k = 0;
        while ((1ll << k) < x) k++;
        return k;
    };
    char buf[384];
    snprintf(buf, sizeof buf, "%s_c%d_rooms%d_tris2^%d_rays2^%d_b%d", name.c_str(), N_CANDIDATES, n_rooms,
             lg(n_tris), lg(n_traced), B);
    return buf;
}

static int tune_pick(const std::string& key) {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    tune_load_locked();
    TuneState& t = g_tune[key];
    if (t.best >= 0) return t.best;
    return t.next < TUNE_ROUNDS * N_CANDIDATES ? t.next % N_CANDIDATES : 0;
}

static void tune_report(const std::string& key, int cand, float ms) {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    TuneState& t = g_tune[key];
    if (t.best >= 0 || cand != t.next % N_CANDIDATES) return;
    t.ms[cand] = t.next < N_CANDIDATES ? ms : std::min(t.ms[cand], ms);
    t.next++;
    if (t.next == TUNE_ROUNDS * N_CANDIDATES) {
        int b = 0;
        for (int k = 1; k < N_CANDIDATES; k++)
            if (t.ms[k] < t.ms[b]) b = k;
        t.best = b;
        tune_save_locked();
    }
}

// dynamic shared memory of a bounce launch: the traversal stacks
static size_t stack_bytes(int block, int stack = STACK_SMEM) {
    return sizeof(int) * (size_t)stack * (size_t)block;
}

template <int BT>
static void* kernel_bt(bool replay, int stack) {
    if (stack == STACK_SHORT) return replay ? (void*)k_bounce<BT, true, STACK_SHORT> : (void*)k_bounce<BT, false, STACK_SHORT>;
    return replay ? (void*)k_bounce<BT, true, STACK_SMEM> : (void*)k_bounce<BT, false, STACK_SMEM>;
}

static void* kernel_of(int block, bool replay = false, int stack = STACK_SMEM) {
    switch (block) {
        case 64: return kernel_bt<64>(replay, stack);
        case 256: return kernel_bt<256>(replay, stack);
        default: return kernel_bt<128>(replay, stack);
    }
}

// allow the stacks above the 48 KB default (the 256-thread block needs 64 KB);
// a function attribute of the current device, set before any launch or capture
static rt_status allow_stack_smem(int block, bool replay = false, int stack = STACK_SMEM) {
    RR_CUDA(cudaFuncSetAttribute(kernel_of(block, replay, stack), cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)stack_bytes(block, stack)));
    return RT_OK;
}

// persistent grid: resident blocks per SM x SMs
static int grid_of_block(int block, int stack = STACK_SMEM) {
    int occ = 0;
    if (allow_stack_smem(block, false, stack) == RT_OK)
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kernel_of(block, false, stack), block,
                                                      stack_bytes(block, stack));
    cudaGetLastError();
    return device_sm_count() * (occ > 0 ? occ : 1);
}

}  // namespace rr

// -- workspace: reusable scratch and the graph of the bounce loop ------------
struct rt_workspace {
    cudaStream_t stream = nullptr;
    std::vector<void*> owned;
    int64_t cap_rays = 0;
    int cap_b = 0;
    rr::Queue q[2]{};
    unsigned int* counters = nullptr;
    unsigned long long* n2 = nullptr;
    cudaGraphExec_t exec = nullptr;
    cudaGraph_t graph = nullptr;
    std::vector<cudaGraphNode_t> nodes;
    int g_b = 0, g_grid = 0, g_block = 0, g_stack = 0;
    bool g_replay = false;
    long long graph_launches = 0;
    unsigned long long last_records = 0;  // capacity hint for the next trace

    void release_graph() {
        if (exec) cudaGraphExecDestroy(exec);
        if (graph) cudaGraphDestroy(graph);
        exec = nullptr;
        graph = nullptr;
        nodes.clear();
    }
    void release_buffers() {
        for (void* p : owned) rr::dev_free(p, stream);
        owned.clear();
        cap_rays = 0;
        cap_b = 0;
    }
};

namespace rr {

// Launch the bounce kernels: one per bounce, or only the first when the
// tail threshold covers every traced ray (that launch then finishes every
// bounce in tail mode and the others would find no live ray).  With a
// workspace on a capturable stream the loop is captured once into a CUDA
// graph and later replayed with updated kernel parameters (one graph launch
// per trace).
static rt_status run_bounces(BounceArgs a, const Queue q[2], int n_launch, int period, int stack, int block,
                             int grid, cudaStream_t s, rt_workspace* ws) {
    const bool replay = a.replay != nullptr;
    void* kern = kernel_of(block, replay, stack);
    const size_t smem = stack_bytes(block, stack);
    RR_TRY(allow_stack_smem(block, replay, stack));
    const int B = n_launch;
    std::vector<BounceArgs> args((size_t)B, a);
    for (int b = 0; b < B; b++) {
        args[b].launch = b;
        args[b].b = b * period;
        args[b].b_end = std::min(a.B, (b + 1) * period);
        args[b].in = q[b & 1];
        args[b].out = q[(b + 1) & 1];
    }
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    const bool can_graph = ws && s != nullptr && cudaStreamIsCapturing(s, &cs) == cudaSuccess &&
                           cs == cudaStreamCaptureStatusNone;
    cudaGetLastError();
    if (!can_graph) {
        for (int b = 0; b < B; b++) {
            void* params[] = {&args[b]};
            RR_CUDA(cudaLaunchKernel(kern, dim3(grid), dim3(block), params, smem, s));
            note_launch();
        }
        return RT_OK;
    }
    if (!ws->exec || ws->g_b != B || ws->g_grid != grid || ws->g_block != block || ws->g_replay != replay ||
        ws->g_stack != stack) {
        ws->release_graph();
        RR_CUDA(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
        for (int b = 0; b < B; b++) {
            void* params[] = {&args[b]};
            cudaLaunchKernel(kern, dim3(grid), dim3(block), params, smem, s);
        }
        cudaGraph_t g = nullptr;
        RR_CUDA(cudaStreamEndCapture(s, &g));
        ws->graph = g;
        RR_CUDA(cudaGraphInstantiate(&ws->exec, g, 0));
        // the captured launches form a chain: walk it from the root
        size_t n = 1;
        cudaGraphNode_t node;
        RR_CUDA(cudaGraphGetRootNodes(g, &node, &n));
        ws->nodes.clear();
        for (int b = 0; b < B; b++) {
            ws->nodes.push_back(node);
            size_t nd = 1;
            cudaGraphNode_t next = nullptr;
            if (b + 1 < B) {
                RR_CUDA(cudaGraphNodeGetDependentNodes(node, &next, nullptr, &nd));
                node = next;
            }
        }
        ws->g_b = B;
        ws->g_grid = grid;
        ws->g_block = block;
        ws->g_replay = replay;
        ws->g_stack = stack;
    } else {
        for (int b = 0; b < B; b++) {
            cudaKernelNodeParams kp{};
            void* params[] = {&args[b]};
            kp.func = kern;
            kp.gridDim = dim3(grid);
            kp.blockDim = dim3(block);
            kp.sharedMemBytes = (unsigned int)smem;
            kp.kernelParams = params;
            kp.extra = nullptr;
            RR_CUDA(cudaGraphExecKernelNodeSetParams(ws->exec, ws->nodes[b], &kp));
        }
    }
    RR_CUDA(cudaGraphLaunch(ws->exec, s));
    ws->graph_launches++;
    for (int b = 0; b < B; b++) note_launch();
    return RT_OK;
}

struct HostRoomTables {
    std::vector<RoomDev> rooms;
    std::vector<int32_t> room_of_src, room_of_rcv, rcv_id, rcv_beg;
    std::vector<float4> rcv;
    std::vector<float> src;
    std::vector<double> src64, rcv64, refl64;
    std::vector<double> srcdir;  // [S][4] unit axis, pattern a; a < 0: omnidirectional
    bool directional = false;
    std::vector<float> refl;
    int S = 0, R = 0;
    int64_t total_tris = 0;
};

static rt_status gather_rooms(const rt_room* rooms, int n_rooms, HostRoomTables& h) {
    if (!rooms || n_rooms < 1) {
        set_error("rt_trace: need at least one room");
        return RT_ERR_INVALID_ARG;
    }
    int mat_base = 0;
    // global source and receiver numbering: room after room
    std::vector<int> src_base((size_t)n_rooms + 1, 0), rcv_base((size_t)n_rooms + 1, 0);
    for (int r = 0; r < n_rooms; r++) {
        const rt_room& rm = rooms[r];
        if (!rm.tree || rm.sources.n < 1 || !rm.sources.pos || rm.receivers.n < 0 || !rm.band_absorption ||
            (rm.receivers.n > 0 && (!rm.receivers.center || !rm.receivers.radius || !rm.receivers.source_of))) {
            set_error("rt_trace: room %d needs a tree, >= 1 source, valid receivers and an absorption table", r);
            return RT_ERR_INVALID_ARG;
        }
        if (rm.n_materials < rm.tree->n_materials) {
            set_error("rt_trace: room %d: absorption table has %d materials, mesh uses %d", r, rm.n_materials,
                      rm.tree->n_materials);
            return RT_ERR_INVALID_ARG;
        }
        src_base[r + 1] = src_base[r] + rm.sources.n;
        rcv_base[r + 1] = rcv_base[r] + rm.receivers.n;
    }
    h.S = src_base[n_rooms];
    h.R = rcv_base[n_rooms];
    h.room_of_src.resize((size_t)h.S);
    h.src.resize((size_t)3 * h.S);
    h.src64.resize((size_t)3 * h.S);
    h.srcdir.assign((size_t)4 * h.S, 0.0);
    h.room_of_rcv.resize((size_t)std::max(h.R, 1), 0);
    h.rcv64.resize((size_t)3 * std::max(h.R, 1), 0.0);
    std::vector<int> gsrc((size_t)std::max(h.R, 1), 0);  // global source of each global receiver
    for (int r = 0; r < n_rooms; r++) {
        const rt_room& rm = rooms[r];
        for (int64_t k = 0; k < (int64_t)rm.n_materials * RT_N_BANDS; k++) {
            float al = rm.band_absorption[k];
            if (!(al >= 0.0f && al <= 1.0f)) {
                set_error("rt_trace: room %d: absorption coefficients must lie in [0, 1]", r);
                return RT_ERR_INVALID_ARG;
            }
            h.refl.push_back(1.0f - al);
            h.refl64.push_back(1.0 - (double)al);
        }
        for (int k = 0; k < rm.sources.n; k++) {
            const int g = src_base[r] + k;
            h.room_of_src[g] = r;
            for (int c = 0; c < 3; c++) {
                double x = rm.sources.pos[3 * k + c];
                if (!std::isfinite(x)) {
                    set_error("rt_trace: room %d: non-finite source position", r);
                    return RT_ERR_INVALID_ARG;
                }
                h.src64[3 * g + c] = x;
                h.src[3 * g + c] = (float)x;
            }
            h.srcdir[4 * g + 3] = -1.0;
            if (rm.sources.axis) {
                const double* w = rm.sources.axis + 3 * k;
                const double a = rm.sources.pattern ? rm.sources.pattern[k] : 0.0;
                const double n2 = w[0] * w[0] + w[1] * w[1] + w[2] * w[2];
                if (!(std::fabs(n2 - 1.0) <= 1e-9) || !(a >= 0.0 && a <= 0.5)) {
                    set_error("rt_trace: room %d: source axes must be unit vectors and patterns lie in [0, 1/2]",
                              r);
                    return RT_ERR_INVALID_ARG;
                }
                for (int c = 0; c < 3; c++) h.srcdir[4 * g + c] = w[c];
                h.srcdir[4 * g + 3] = a;
                h.directional = true;
            }
        }
        for (int k = 0; k < rm.receivers.n; k++) {
            const int g = rcv_base[r] + k;
            const int so = rm.receivers.source_of[k];
            if (so < 0 || so >= rm.sources.n || !(rm.receivers.radius[k] > 0)) {
                set_error("rt_trace: room %d receiver %d invalid (source index or radius)", r, k);
                return RT_ERR_INVALID_ARG;
            }
            for (int c = 0; c < 3; c++) {
                double x = rm.receivers.center[3 * k + c];
                if (!std::isfinite(x)) {
                    set_error("rt_trace: room %d receiver %d has a non-finite centre", r, k);
                    return RT_ERR_INVALID_ARG;
                }
                h.rcv64[3 * g + c] = x;
            }
            h.room_of_rcv[g] = r;
            gsrc[g] = src_base[r] + so;
        }
        RoomDev d{};
        d.nodes = rm.tree->nodes;
        d.tris = rm.tree->tris;
        d.tri_nrm = rm.tree->tri_nrm;
        d.mat_of_surf = rm.tree->mat_of_surf;
        d.surf_of = rm.tree->surf_of;
        d.planes = rm.tree->planes;
        d.pos_of = rm.tree->pos_of;
        d.n_nodes = rm.tree->n_nodes;
        d.n_tris = rm.tree->n_tris;
        d.mat_base = mat_base;
        mat_base += rm.n_materials;
        h.total_tris += rm.tree->n_tris;
        h.rooms.push_back(d);
    }
    // receivers grouped by global source
    std::vector<int> order((size_t)h.R);
    for (int k = 0; k < h.R; k++) order[k] = k;
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return gsrc[a] < gsrc[b]; });
    h.rcv.resize((size_t)std::max(h.R, 1));
    h.rcv_id.resize((size_t)std::max(h.R, 1), 0);
    h.rcv_beg.assign((size_t)h.S + 1, 0);
    for (int k = 0; k < h.R; k++) {
        const int o = order[k];
        const int r = h.room_of_rcv[o];
        const int local = o - rcv_base[r];
        const float rad = (float)rooms[r].receivers.radius[local];
        h.rcv[k] = make_float4((float)h.rcv64[3 * o], (float)h.rcv64[3 * o + 1], (float)h.rcv64[3 * o + 2], rad * rad);
        h.rcv_id[k] = o;
        h.rcv_beg[gsrc[o] + 1]++;
    }
    for (int k = 0; k < h.S; k++) h.rcv_beg[k + 1] += h.rcv_beg[k];
    return RT_OK;
}

// Host tables gathered into one buffer and copied with one call (16-byte
// aligned slices), so that the GPU does not wait for a chain of small copies.
struct Packer {
    std::vector<unsigned char> host;
    std::vector<std::pair<size_t, void**>> slots;
    template <class T>
    void add(const std::vector<T>& v, T** out) {
        const size_t off = (host.size() + 15) & ~(size_t)15;
        host.resize(off + std::max<size_t>(sizeof(T) * v.size(), 16), 0);
        if (!v.empty()) memcpy(host.data() + off, v.data(), sizeof(T) * v.size());
        slots.emplace_back(off, reinterpret_cast<void**>(out));
    }
    rt_status upload(Arena& ar, cudaStream_t s) {
        unsigned char* d;
        RR_TRY(ar.alloc(&d, host.size()));
        RR_CUDA(cudaMemcpyAsync(d, host.data(), host.size(), cudaMemcpyHostToDevice, s));
        for (auto& sl : slots) *sl.second = d + sl.first;
        return RT_OK;
    }
};

static rt_status trace_batch_impl(const rt_room* rooms, int n_rooms, const rt_trace_params* p,
                                  rt_image_sources** out) {
    if (!p || !out) {
        set_error("rt_trace: null argument");
        return RT_ERR_INVALID_ARG;
    }
    *out = nullptr;
    cudaStream_t s = (cudaStream_t)p->stream;
    rt_workspace* ws = p->workspace;
    const int64_t N = p->n_rays;
    const int B = p->n_bounces;
    if (N < 1 || B < 1 || B > RT_MAX_BOUNCES || !(p->c > 0)) {
        set_error("rt_trace: need n_rays >= 1, 1 <= n_bounces <= %d, c > 0", RT_MAX_BOUNCES);
        return RT_ERR_INVALID_ARG;
    }
    if (p->ray_begin < 0 || p->ray_begin >= N) {
        set_error("rt_trace: ray_begin out of range");
        return RT_ERR_INVALID_ARG;
    }
    const int64_t per_src = p->ray_count > 0 ? p->ray_count : N - p->ray_begin;
    if (p->ray_begin + per_src > N) {
        set_error("rt_trace: ray range exceeds n_rays");
        return RT_ERR_INVALID_ARG;
    }
    if (p->max_node_visits < 0) {
        set_error("rt_trace: max_node_visits must be >= 0");
        return RT_ERR_INVALID_ARG;
    }
    if (p->block_size != 0 && p->block_size != 64 && p->block_size != 128 && p->block_size != 256) {
        set_error("rt_trace: block_size must be 0, 64, 128 or 256");
        return RT_ERR_INVALID_ARG;
    }
    if (ws && ws->stream != s && !ws->owned.empty()) {
        set_error("rt_trace: a workspace serves one stream");
        return RT_ERR_INVALID_ARG;
    }
    HostRoomTables h;
    RR_TRY(gather_rooms(rooms, n_rooms, h));
    const int S = h.S, R = h.R;
    const int64_t n_traced = per_src * S;
    if (n_traced > (int64_t)INT32_MAX) {
        set_error("rt_trace: %lld rays exceed the 32-bit ray index", (long long)n_traced);
        return RT_ERR_INVALID_ARG;
    }
    std::vector<double> h_beta64(8, 0.0);
    if (p->air_beta)
        for (int f = 0; f < 8; f++) h_beta64[f] = (double)p->air_beta[f];

    Arena tmp(s), keep(s);
    RoomDev* d_rooms;
    int32_t *d_room_of_src, *d_room_of_rcv, *d_rcv_id, *d_beg;
    float4* d_rcv;
    float *d_src, *d_refl;
    double *d_refl64, *d_beta64, *d_src64, *d_rcv64, *d_srcdir = nullptr;
    {
        Packer pk;
        pk.add(h.rooms, &d_rooms);
        pk.add(h.room_of_src, &d_room_of_src);
        pk.add(h.room_of_rcv, &d_room_of_rcv);
        pk.add(h.rcv, &d_rcv);
        pk.add(h.rcv_id, &d_rcv_id);
        pk.add(h.rcv_beg, &d_beg);
        pk.add(h.src, &d_src);
        if (h.directional) pk.add(h.srcdir, &d_srcdir);
        pk.add(h.refl, &d_refl);
        pk.add(h.refl64, &d_refl64);
        pk.add(h_beta64, &d_beta64);
        pk.add(h.src64, &d_src64);
        pk.add(h.rcv64, &d_rcv64);
        RR_TRY(pk.upload(tmp, s));
    }

    // scratch: queues and counters (from the workspace when given)
    Queue q[2];
    unsigned int* counters;
    unsigned long long* n2d;
    const int n_counters = 2 * B + 4;
    if (ws) {
        if (ws->cap_rays < n_traced || ws->cap_b < B) {
            ws->release_graph();
            ws->release_buffers();
            ws->stream = s;
            Arena war(s);
            RR_TRY(alloc_queue(war, ws->q[0], n_traced));
            RR_TRY(alloc_queue(war, ws->q[1], n_traced));
            RR_TRY(war.alloc(&ws->counters, n_counters));
            RR_TRY(war.alloc(&ws->n2, 2));
            ws->owned = war.release();
            ws->cap_rays = n_traced;
            ws->cap_b = B;
        }
        q[0] = ws->q[0];
        q[1] = ws->q[1];
        counters = ws->counters;
        n2d = ws->n2;
    } else {
        RR_TRY(alloc_queue(tmp, q[0], n_traced));
        RR_TRY(alloc_queue(tmp, q[1], n_traced));
        RR_TRY(tmp.alloc(&counters, n_counters));
        RR_TRY(tmp.alloc(&n2d, 2));
    }
    // primary rays first, so that the GPU works while the host prepares the rest
    struct Events {
        cudaEvent_t e[4] = {nullptr, nullptr, nullptr, nullptr};
        ~Events() {
            for (auto x : e)
                if (x) cudaEventDestroy(x);
        }
    } ev;
    for (auto& x : ev.e) RR_CUDA(cudaEventCreate(&x));
    int64_t F = 1, F1 = 1;  // largest Fibonacci number <= sqrt(per_src)
    while (F1 * F1 <= per_src) {
        int64_t t = F + F1;
        F = F1;
        F1 = t;
    }
    auto gen_rays = [&]() -> rt_status {
        RR_CUDA(cudaEventRecord(ev.e[0], s));
        RR_LAUNCH(k_gen_rays, grid_of(n_traced, 256), 256, 0, s, q[0], d_src, d_srcdir, n_traced, per_src,
                  p->ray_begin, N, F, GOLDEN_G);
        RR_CUDA(cudaGetLastError());
        RR_CUDA(cudaEventRecord(ev.e[1], s));
        return RT_OK;
    };
    RR_TRY(gen_rays());
    int32_t* hist;
    float4* ray_e;
    float* ray_len;
    int32_t* ray_hits;
    {
        Carve cv;
        cv.add(&hist, (size_t)B * n_traced);
        cv.add(&ray_e, 2 * (size_t)n_traced);
        cv.add(&ray_len, (size_t)n_traced);
        cv.add(&ray_hits, (size_t)n_traced);
        RR_TRY(cv.alloc(keep));
    }

    // bounce-kernel configuration
    const int a_step_cap = p->max_node_visits > 0 ? p->max_node_visits : DEFAULT_NODE_VISITS;
    const bool autotune = p->tail_rays == RT_TAIL_AUTOTUNE;
    std::string key;
    int cand = -1;
    int block = p->block_size > 0 ? p->block_size : 128;
    int tail_mode = p->tail_rays < 0 ? 0 : 1;
    int period = 1, stack = STACK_SMEM;
    if (autotune) {
        key = tune_key(h.total_tris, n_traced, B, n_rooms) + (p->replay_hist ? "_replay" : "");
        cand = tune_pick(key);
        block = CANDIDATES[cand].block;
        tail_mode = CANDIDATES[cand].tail_mode;
        period = CANDIDATES[cand].period;
        stack = CANDIDATES[cand].stack;
    }
    if (p->compaction_period > 0) period = p->compaction_period;
    if (p->stack_entries > 0) stack = p->stack_entries <= STACK_SHORT ? STACK_SHORT : STACK_SMEM;
    int max_depth = 0;
    for (int r = 0; r < n_rooms; r++) max_depth = std::max(max_depth, (int)rooms[r].tree->depth);
    if (max_depth > STACK_SHORT_MAX_DEPTH) stack = STACK_SMEM;  // the short stack could overflow
    period = std::min(std::max(period, 1), B);
    const int grid = grid_of_block(block, stack);
    unsigned int tail = 0;
    if (autotune) {
        tail = tail_mode == 0 ? 0u : (tail_mode == 1 ? (unsigned int)grid * (unsigned int)block
                                                    : (unsigned int)std::min<int64_t>(n_traced, UINT32_MAX));
    } else if (p->tail_rays > 0) {
        tail = (unsigned int)p->tail_rays;
    } else if (p->tail_rays == 0) {
        tail = (unsigned int)grid * (unsigned int)block;
    }

    unsigned long long cap = (unsigned long long)std::min<int64_t>(
        std::max<int64_t>(1 << 20, 2 * n_traced), std::max<int64_t>(1, n_traced * (int64_t)B * std::max(R, 1)));
    if (ws && ws->last_records + ws->last_records / 4 > cap) cap = ws->last_records + ws->last_records / 4;
    unsigned long long n_rec = 0, n2[2] = {0, 0};
    std::vector<unsigned int> h_cnt((size_t)n_counters);
    Arena rec_arena(s);
    int32_t *rec_rcv = nullptr, *rec_ray = nullptr, *rec_m = nullptr;
    float* rec_len = nullptr;
    uint64_t* rec_key = nullptr;
    for (int attempt = 0; attempt < 2; attempt++) {
        {
            Carve cv;
            cv.add(&rec_rcv, (size_t)cap);
            cv.add(&rec_ray, (size_t)cap);
            cv.add(&rec_m, (size_t)cap);
            cv.add(&rec_len, (size_t)cap);
            cv.add(&rec_key, (size_t)cap);
            RR_TRY(cv.alloc(rec_arena));
        }
        RR_CUDA(cudaMemsetAsync(hist, 0xFF, sizeof(int32_t) * (size_t)B * n_traced, s));
        RR_CUDA(cudaMemsetAsync(counters, 0, sizeof(unsigned int) * n_counters, s));
        RR_CUDA(cudaMemsetAsync(n2d, 0, 2 * sizeof(unsigned long long), s));
        unsigned int n0 = (unsigned int)n_traced;
        RR_CUDA(cudaMemcpyAsync(counters, &n0, sizeof n0, cudaMemcpyHostToDevice, s));
        if (attempt > 0) RR_TRY(gen_rays());  // the first attempt consumed the queue
        BounceArgs a{};
        a.rooms = d_rooms;
        a.room_of_src = d_room_of_src;
        a.refl = d_refl;
        a.rcv = d_rcv;
        a.rcv_id = d_rcv_id;
        a.rcv_beg = d_beg;
        a.hist = hist;
        a.ray_e = ray_e;
        a.ray_len = ray_len;
        a.ray_hits = ray_hits;
        a.rec_rcv = rec_rcv;
        a.rec_ray = rec_ray;
        a.rec_m = rec_m;
        a.rec_len = rec_len;
        a.rec_key = rec_key;
        a.rec_cap = cap;
        a.live = counters;
        a.fetch = counters + (B + 1);
        a.status = counters + (2 * B + 1);
        a.n_rec = n2d;
        a.n_queries = n2d + 1;
        a.tail_threshold = tail;
        a.n_traced = n_traced;
        a.per_src = per_src;
        a.B = B;
        a.dmax = (float)(p->max_distance > 0 ? p->max_distance : 0.0);
        a.step_cap = a_step_cap;
        a.debug_t = p->debug_t;
        a.debug_state = p->debug_state;
        a.debug_cost = p->debug_cost;
        a.replay = p->replay_hist;
        const int n_launch = (uint64_t)tail >= (uint64_t)n_traced ? 1 : (B + period - 1) / period;
        RR_TRY(run_bounces(a, q, n_launch, period, stack, block, grid, s, ws));
        RR_CUDA(cudaGetLastError());
        RR_CUDA(cudaEventRecord(ev.e[2], s));
        RR_CUDA(cudaMemcpyAsync(h_cnt.data(), counters, sizeof(unsigned int) * n_counters, cudaMemcpyDeviceToHost, s));
        RR_CUDA(cudaMemcpyAsync(n2, n2d, sizeof n2, cudaMemcpyDeviceToHost, s));
        RR_CUDA(cudaStreamSynchronize(s));
        n_rec = n2[0];
        unsigned int st = h_cnt[2 * B + 1];
        if (st & ST_STACK) {
            set_error("rt_trace: traversal stack overflow (more than %d entries; a tree of binary depth <= 42 "
                      "always fits)", stack);
            return RT_ERR_STACK;
        }
        if (st & ST_BOUNDS) {
            set_error("rt_trace: a node, leaf or replayed triangle reference lies outside the tree");
            return RT_ERR_INTERNAL;
        }
        if (st & ST_STEPS) {
            set_error("rt_trace: a traversal exceeded %d node visits", a_step_cap);
            return RT_ERR_STEP_LIMIT;
        }
        if (n_rec <= cap) break;
        if (attempt == 1) {
            set_error("rt_trace: %llu records exceed the capacity %llu", n_rec, cap);
            return RT_ERR_CAPACITY;
        }
        // second attempt with the exact capacity
        for (void* ptr : rec_arena.release()) dev_free(ptr, s);
        cap = n_rec;
    }
    const int64_t queries = (int64_t)n2[1];
    if (ws) ws->last_records = n_rec;
    float ms_bounce = 0.f;
    cudaEventElapsedTime(&ms_bounce, ev.e[1], ev.e[2]);
    if (autotune) tune_report(key, cand, ms_bounce);

    // -- dedup + reconstruction ---------------------------------------------
    const int64_t nr = (int64_t)n_rec;
    rt_image_sources* is = new rt_image_sources();
    struct Guard {
        rt_image_sources*& p;
        ~Guard() {
            if (p) {
                for (void* q : p->owned) dev_free(q, p->stream);
                delete p;
            }
        }
    } guard{is};
    is->stream = s;
    is->n_rcv = R;
    is->c = p->c;
    int32_t *o_rcv, *o_order, *o_count, *o_rep;
    double *o_pos, *o_dist, *o_time, *o_energy;
    const int64_t ncap = std::max<int64_t>(nr, 1);
    {
        Carve cv;
        cv.add(&o_rcv, (size_t)ncap);
        cv.add(&o_order, (size_t)ncap);
        cv.add(&o_count, (size_t)ncap);
        cv.add(&o_rep, (size_t)ncap);
        cv.add(&o_pos, 3 * (size_t)ncap);
        cv.add(&o_dist, (size_t)ncap);
        cv.add(&o_time, (size_t)ncap);
        cv.add(&o_energy, 8 * (size_t)ncap);
        RR_TRY(cv.alloc(keep));
    }
    unsigned int n_unique = 0;
    unsigned long long collisions = 0;
    if (nr > 0) {
        uint64_t *keys, *keys_alt;
        uint32_t *vals, *vals_alt, *flags, *segid, *heads, *nuniq;
        unsigned long long* d_coll;
        Carve cv;
        cv.add(&keys, (size_t)nr);
        cv.add(&keys_alt, (size_t)nr);
        cv.add(&vals, (size_t)nr);
        cv.add(&vals_alt, (size_t)nr);
        cv.add(&flags, (size_t)nr);
        cv.add(&segid, (size_t)nr);
        cv.add(&heads, (size_t)nr + 1);
        cv.add(&nuniq, 1);
        cv.add(&d_coll, 1);
        unsigned char *sort_tmp, *scan_tmp;
        cv.add(&sort_tmp, sort_temp_bytes(nr));
        cv.add(&scan_tmp, scan_temp_bytes(nr));
        RR_TRY(cv.alloc(tmp));
        RR_CUDA(cudaMemsetAsync(d_coll, 0, sizeof(unsigned long long), s));
        RR_LAUNCH(k_dedup_init, grid_of(nr, 256), 256, 0, s, rec_key, rec_m, nr, keys, vals);
        RR_TRY(radix_sort_pairs(keys, vals, keys_alt, vals_alt, nr, 0, 64, sort_tmp, s));
        RR_LAUNCH(k_seg_flags, grid_of(nr, 256), 256, 0, s, keys, vals, nr, rec_rcv, rec_ray, rec_m, hist, d_rooms,
                  d_room_of_rcv, n_traced, flags, d_coll);
        RR_CUDA(cudaGetLastError());
        RR_TRY(exclusive_scan_u32(flags, segid, nr, nuniq, scan_tmp, s));
        RR_LAUNCH(k_seg_heads, grid_of(nr, 256), 256, 0, s, flags, segid, nr, heads);
        RR_CUDA(cudaMemsetAsync(o_rep, 0x7F, sizeof(int32_t) * nr, s));
        RR_LAUNCH(k_seg_min, grid_of(nr, 256), 256, 0, s, vals, flags, segid, nr, rec_ray, o_rep);
        ReconArgs ra;
        ra.heads = heads;
        ra.vals = vals;
        ra.n_unique_dev = nuniq;
        ra.status = counters + (2 * B + 1);
        ra.rec_rcv = rec_rcv;
        ra.rec_ray = rec_ray;
        ra.rec_m = rec_m;
        ra.hist = hist;
        ra.rooms = d_rooms;
        ra.room_of_rcv = d_room_of_rcv;
        ra.refl64 = d_refl64;
        ra.beta64 = d_beta64;
        ra.src64 = d_src64;
        ra.rcv64 = d_rcv64;
        ra.n_traced = n_traced;
        ra.per_src = per_src;
        ra.N = (double)N;
        ra.c = p->c;
        ra.o_rcv = o_rcv, ra.o_order = o_order, ra.o_count = o_count, ra.o_rep = o_rep;
        ra.o_pos = o_pos, ra.o_dist = o_dist, ra.o_time = o_time, ra.o_energy = o_energy;
        RR_LAUNCH(k_reconstruct, grid_of(nr, 128), 128, 0, s, ra);
        RR_CUDA(cudaGetLastError());
        RR_CUDA(cudaMemcpyAsync(&n_unique, nuniq, sizeof n_unique, cudaMemcpyDeviceToHost, s));
        RR_CUDA(cudaMemcpyAsync(&collisions, d_coll, sizeof collisions, cudaMemcpyDeviceToHost, s));
        RR_CUDA(cudaEventRecord(ev.e[3], s));
        unsigned int st = 0;
        RR_CUDA(cudaMemcpyAsync(&st, ra.status, sizeof st, cudaMemcpyDeviceToHost, s));
        RR_CUDA(cudaStreamSynchronize(s));
        if (st & ST_HISTORY) {
            set_error("rt_trace: an image source's ray has no hit history");
            return RT_ERR_INTERNAL;
        }
    }
    rt_is_view& v = is->v;
    v.n = n_unique;
    v.rcv = o_rcv;
    v.order = o_order;
    v.count = o_count;
    v.rep_ray = o_rep;
    v.pos = o_pos;
    v.dist = o_dist;
    v.time = o_time;
    v.energy = o_energy;
    v.n_traced = n_traced;
    v.n_bounces = B;
    v.hist = hist;
    v.ray_energy = (const float*)ray_e;
    v.ray_length = ray_len;
    v.ray_hits = ray_hits;
    v.n_records = nr;
    v.rec_rcv = rec_rcv;
    v.rec_ray = rec_ray;
    v.rec_order = rec_m;
    v.rec_length = rec_len;
    v.queries = queries;
    v.hash_collisions = (int64_t)collisions;
    v.block_size = block;
    v.tail_rays = (int64_t)tail;
    v.compaction_period = period;
    v.stack_entries = stack;
    cudaEventElapsedTime(&v.ms_rays, ev.e[0], ev.e[1]);
    v.ms_bounces = ms_bounce;
    if (nr > 0) cudaEventElapsedTime(&v.ms_image_sources, ev.e[2], ev.e[3]);
    v.n_rcv = is->n_rcv;
    cudaGetLastError();
    is->owned = keep.release();
    for (void* ptr : rec_arena.release()) is->owned.push_back(ptr);
    *out = is;
    is = nullptr;
    return RT_OK;
}

}  // namespace rr

extern "C" rt_status rt_trace(const rt_tree* tree, const rt_sources* src, const rt_receivers* rcv,
                              const float* band_absorption, int32_t n_materials, const rt_trace_params* params,
                              rt_image_sources** out) {
    rr::NvtxRange nvtx_range("rt_trace");
    rr::clear_error();
    if (!tree || !src || !rcv || !band_absorption) {
        rr::set_error("rt_trace: null argument");
        return RT_ERR_INVALID_ARG;
    }
    rt_room room;
    room.tree = tree;
    room.sources = *src;
    room.receivers = *rcv;
    room.band_absorption = band_absorption;
    room.n_materials = n_materials;
    return rr::trace_batch_impl(&room, 1, params, out);
}

extern "C" rt_status rt_trace_batch(const rt_room* rooms, int32_t n_rooms, const rt_trace_params* params,
                                    rt_image_sources** out) {
    rr::NvtxRange nvtx_range("rt_trace_batch");
    rr::clear_error();
    return rr::trace_batch_impl(rooms, n_rooms, params, out);
}

extern "C" rt_status rt_workspace_create(rt_workspace** out) {
    rr::clear_error();
    if (!out) {
        rr::set_error("rt_workspace_create: null output");
        return RT_ERR_INVALID_ARG;
    }
    *out = new rt_workspace();
    return RT_OK;
}

extern "C" int64_t rt_workspace_graph_launches(const rt_workspace* ws) { return ws ? ws->graph_launches : 0; }

extern "C" void rt_workspace_free(rt_workspace* ws) {
    if (!ws) return;
    ws->release_graph();
    ws->release_buffers();
    delete ws;
}

extern "C" rt_status rt_image_sources_view(const rt_image_sources* is, rt_is_view* out) {
    if (!is || !out) {
        rr::set_error("rt_image_sources_view: null argument");
        return RT_ERR_INVALID_ARG;
    }
    *out = is->v;
    return RT_OK;
}

extern "C" void rt_image_sources_free(rt_image_sources* is) {
    if (!is) return;
    for (void* p : is->owned) rr::dev_free(p, is->stream);
    delete is;
}
