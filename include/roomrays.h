/*
 * roomrays.h -- C ABI of the GB300 ray-propagation library.
 *
 * Hybrid ray-tracing / image-source room acoustics after Aussal & Gueguen
 * (2018), "Open-source platforms for fast room acoustic simulations in
 * complex structures" (arXiv:1811.05784).  Three calls make the path:
 *
 *   rt_build_tree  mesh of flat triangles with materials (Sec. 2.1) ->
 *                  bounding-volume tree (replaces the median-split tree of
 *                  Sec. 2.2 with a Morton-code LBVH built on the device)
 *   rt_trace       rays from each source (Sec. 1.2), nearest element per
 *                  bounce (Sec. 2.1, eq. 20-21), measurement spheres (eq. 22),
 *                  specular reflection (eq. 15), band absorption (eq. 16),
 *                  range cut (eq. 13), image sources by reflection sequence
 *                  with energies (Sec. 1.4, eq. 19)
 *   rt_rir         8-band energy impulse responses: arrival time d_s / c,
 *                  histogram at fs (Sec. 1.4)
 *
 * Conventions
 *   - Every call returns rt_status; nothing is thrown across the ABI.  On an
 *     error, rt_last_error() returns a message for the calling thread and no
 *     output handle is written.
 *   - Input pointers are borrowed for the duration of the call.  Host arrays
 *     are copied; device arrays must be readable on `stream`.
 *   - `stream` is a cudaStream_t (NULL = the legacy default stream).  Calls
 *     enqueue work on it; rt_trace and rt_rir synchronise it once or twice to
 *     size their outputs (record count, image-source count, bin count).
 *   - Output handles own device memory and are freed by their *_free call.
 *     Views hand out borrowed device pointers valid until that free.
 *   - Band index f = 0..7 is the octave 62.5 Hz * 2^f (paper Table 1).
 *   - Energies: each ray starts with 1/N per band (E_m = n/N, eq. 7).
 */
#ifndef ROOMRAYS_H
#define ROOMRAYS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define RT_N_BANDS 8
#define RT_MAX_BOUNCES 4096
#define RT_API_VERSION 1

typedef enum {
    RT_OK = 0,
    RT_ERR_INVALID_ARG = 1,     /* null / negative / out-of-range argument, NaN input */
    RT_ERR_DEGENERATE_MESH = 2, /* a triangle has zero area in float32 */
    RT_ERR_OOM = 3,             /* device allocation failed */
    RT_ERR_CUDA = 4,            /* a CUDA runtime call failed */
    RT_ERR_CAPACITY = 5,        /* record buffer still too small after one retry */
    RT_ERR_STEP_LIMIT = 6,      /* a traversal exceeded its node-visit cap */
    RT_ERR_STACK = 7,           /* traversal stack overflow */
    RT_ERR_INTERNAL = 8
} rt_status;

typedef enum { RT_MEM_HOST = 0, RT_MEM_DEVICE = 1 } rt_memory;

typedef struct rt_tree rt_tree;                   /* immutable after build */
typedef struct rt_image_sources rt_image_sources; /* device-resident results of rt_trace */
typedef struct rt_response rt_response;           /* device-resident histograms */
typedef struct rt_workspace rt_workspace;         /* reusable trace scratch + CUDA graph */

/* Mesh of flat triangles (Sec. 2.1).  `memory` says where the four arrays
 * live.  surface_id groups coplanar triangles of one material; image sources
 * are keyed by sequences of surface ids.  surface_id may be NULL only for
 * host memory: the library then groups triangles by (plane, material). */
typedef struct {
    const double* vertices;      /* [n_vertices][3] metres */
    int64_t n_vertices;
    const int32_t* tris;         /* [n_tris][3] vertex indices */
    int64_t n_tris;
    const int32_t* material_id;  /* [n_tris] index into the absorption table */
    const int32_t* surface_id;   /* [n_tris] or NULL (host memory only) */
    rt_memory memory;
} rt_mesh;

/* Point sources (host memory).  axis NULL: omnidirectional (the Fibonacci
 * rule, Sec. 1.2).  Otherwise every source is directional (Sec. 1.2 footnote:
 * a non-uniform spatial sampling): its N rays keep the energy 1/N and their
 * directions have density (1 - a + a cos theta) / (4 pi (1 - a)) about its
 * unit axis, a = pattern[k] in [0, 1/2] (NULL: 0) -- the uniform rule's z
 * mapped through the inverse cumulative of that density and turned to the
 * axis; the exact FP64 steps are those of directional_dir in csrc/rt_trace.cu.
 * Axes must be unit vectors within 1e-9 and patterns lie in [0, 1/2]
 * (RT_ERR_INVALID_ARG otherwise).  The arrays are read during the call. */
typedef struct {
    const double* pos;           /* [n][3] */
    int32_t n;
    const double* axis;          /* [n][3] unit axes, or NULL */
    const double* pattern;       /* [n] pattern coefficients a, or NULL */
} rt_sources;

/* Measurement spheres S(x_m, r) (Sec. 1.2, eq. 22), host memory.  Receiver k
 * listens to source source_of[k] only. */
typedef struct {
    const double* center;        /* [n][3] */
    const double* radius;        /* [n] */
    const int32_t* source_of;    /* [n] */
    int32_t n;
} rt_receivers;

typedef struct {
    int64_t n_rays;        /* N rays per source: Fibonacci directions i = 0..N-1, energy 1/N */
    int64_t ray_begin;     /* trace rays [ray_begin, ray_begin + ray_count) of every source */
    int64_t ray_count;     /* <= 0: all N (shards of one run add up exactly) */
    int32_t n_bounces;     /* nearest-element queries per ray, 1..RT_MAX_BOUNCES */
    double max_distance;   /* > 0: eq. 13 range; rays stop once their path exceeds it */
    const float* air_beta; /* [8] host, energy attenuation 1/m (eq. 19); NULL = none */
    double c;              /* sound speed m/s (> 0) */
    int32_t block_size;    /* bounce-kernel block size; 0 = library choice */
    int32_t max_node_visits; /* traversal cap per query (0 = 65536); exceeding it fails
                                the call with RT_ERR_STEP_LIMIT instead of looping on */
    int32_t tail_rays;     /* once a bounce starts with at most this many live rays, one
                              launch finishes all their remaining bounces (0 = the number
                              of resident threads, -1 = never: one launch per bounce,
                              RT_TAIL_AUTOTUNE = the library times each of its candidate
                              configurations (block size, threshold, compaction period,
                              stack depth) twice on the first calls of each workload class
                              and keeps the fastest; results do not depend on it.  If the
                              environment variable RT_AUTOTUNE_CACHE names a file, the
                              choices are read from it once per process and the file is
                              rewritten (atomically) whenever a class is tuned; a class is
                              the device model, the candidate list, the rooms, the tree and
                              ray counts (powers of two) and the bounces) */
    void* stream;          /* cudaStream_t */
    /* optional device outputs for parity checks (NULL = off) */
    float* debug_t;        /* [n_bounces][n_traced] hit distance, +inf on escape */
    float* debug_state;    /* [n_bounces][n_traced][6] origin and direction before each query */
    int32_t* debug_cost;   /* [n_bounces][n_traced][2] nodes visited, triangles tested per query */
    rt_workspace* workspace; /* NULL, or scratch reused across calls on one stream; on a
                                non-default stream the bounce loop then runs as one CUDA
                                graph launch (captured on the first call, parameters
                                updated on later ones) */
    const int32_t* replay_hist; /* NULL, or the hit history (rt_is_view.hist, device
                                [n_bounces][n_traced]) of an earlier trace of the same rays:
                                same trees, sources, n_rays, ray_begin / ray_count,
                                n_bounces, max_distance, air and c; the receivers may differ.
                                Each query then re-tests only the recorded triangle (no
                                traversal), so a moved or added listener costs a fraction of
                                a trace and gives exactly what a full trace with the new
                                receivers gives.  A recorded id outside the mesh is reported
                                (RT_ERR_INTERNAL); a history of other rays gives other
                                (meaningless) paths. */
    int32_t compaction_period; /* while more rays live than the tail threshold, each bounce
                                launch steps its rays this many bounces (refilling a lane as
                                soon as its ray dies) before it compacts the survivors into
                                the next queue (0 = 1: one bounce per launch) */
    int32_t stack_entries;   /* traversal stack per thread: 0 or 64, or 48 (used only when
                                every tree has binary depth <= 32, else 64) */
} rt_trace_params;

#define RT_TAIL_AUTOTUNE (-2)

/* One room of a batched trace: its tree, sources, receivers (source_of
 * indexes this room's sources) and absorption table. */
typedef struct {
    const rt_tree* tree;
    rt_sources sources;
    rt_receivers receivers;
    const float* band_absorption; /* [n_materials][8] */
    int32_t n_materials;
} rt_room;

/* Borrowed device views of rt_trace's results.  Traced ray q belongs to
 * source q / ray_count and has Fibonacci index ray_begin + q % ray_count. */
typedef struct {
    int64_t n;                 /* unique image sources */
    const int32_t* rcv;        /* [n] receiver */
    const int32_t* order;      /* [n] reflection order m */
    const int32_t* count;      /* [n] rays in the beam (eq. 7's n) */
    const int32_t* rep_ray;    /* [n] lowest traced-ray index in the beam */
    const double* pos;         /* [n][3] image-source position (FP64 mirror chain) */
    const double* dist;        /* [n] |x_is - x_m| */
    const double* time;        /* [n] dist / c */
    const double* energy;      /* [n][8] eq. 19 */
    int64_t n_traced;          /* rays traced */
    int32_t n_bounces;
    const int32_t* hist;       /* [n_bounces][n_traced] triangle hit per bounce, -1 = none */
    const float* ray_energy;   /* [n_traced][8] band energy after the last hit */
    const float* ray_length;   /* [n_traced] path length (compensated sum) */
    const int32_t* ray_hits;   /* [n_traced] surfaces hit */
    int64_t n_records;         /* sphere crossings */
    const int32_t* rec_rcv;    /* [n_records] */
    const int32_t* rec_ray;    /* [n_records] traced-ray index */
    const int32_t* rec_order;  /* [n_records] */
    const float* rec_length;   /* [n_records] path length at the closest point */
    int64_t queries;           /* nearest-element queries resolved (hits + escapes) */
    int64_t hash_collisions;   /* equal keys with different sequences (expected 0) */
    int32_t block_size;        /* bounce-kernel configuration used */
    int64_t tail_rays;
    float ms_rays;             /* device time of ray generation (CUDA events) */
    float ms_bounces;          /* device time of all bounce launches */
    float ms_image_sources;    /* device time of dedup + FP64 reconstruction */
    int32_t n_rcv;             /* receivers of the trace (all rooms of a batch) */
    int32_t compaction_period; /* bounce-kernel configuration used (with block_size, tail_rays) */
    int32_t stack_entries;
} rt_is_view;

typedef struct {
    int32_t n_rcv;
    int64_t n_bins;
    double fs;
    const float* data;         /* device [n_rcv][8][n_bins] energy per bin */
} rt_response_view;

/* Build the LBVH of a mesh (Sec. 2.2 replaced; see file header).
 * Errors: RT_ERR_INVALID_ARG (n_tris < 1, index out of range, NaN/Inf),
 * RT_ERR_DEGENERATE_MESH, RT_ERR_OOM, RT_ERR_CUDA. */
rt_status rt_build_tree(const rt_mesh* mesh, void* stream, rt_tree** out);
void rt_tree_free(rt_tree* tree);
/* The paper's own tree (Sec. 2.2), built on the device, for comparison with
 * the LBVH: the box of a node's triangles is split along its largest extent
 * at the median (the left child takes the first ceil(count / 2) triangles in
 * centroid order), recursively; nodes of at most two triangles are then
 * stored as leaves, and the tree is stored 4-wide like rt_build_tree's, so
 * every trace call takes it.  The build sorts once per level (ceil(log2 M)
 * segmented radix sorts), so it is slower than rt_build_tree; traces give
 * the same results on either tree.  Same arguments, errors and ownership as
 * rt_build_tree. */
rt_status rt_build_tree_median(const rt_mesh* mesh, void* stream, rt_tree** out);
/* The LBVH with its top levels rebuilt by the surface area heuristic (a tree
 * of the same kind as Sec. 2.2's, split by cost instead of at the median):
 * below "cells" (triangles whose 48-bit Morton codes share their top 24
 * bits) the tree is rt_build_tree's; above them a split minimises
 * area(left box) x triangles(left) + area(right box) x triangles(right),
 * over 16 bins of the cell centres per axis for large nodes and along the
 * Morton order for nodes of at most 32 cells.  No host synchronisation is
 * added; the build takes a few times as long as rt_build_tree's (1.7-2.6 ms
 * against 0.3-0.8 ms at 10^5-10^6 triangles), and a trace visits 15-35 %
 * fewer nodes, so it pays where traces are long or the tree is reused.
 * Traces give the same results on either tree.  Same arguments and
 * ownership as rt_build_tree; errors as rt_build_tree, plus RT_ERR_INTERNAL
 * if the top levels come out inconsistent (not expected for any mesh). */
rt_status rt_build_tree_sah(const rt_mesh* mesh, void* stream, rt_tree** out);

/* Nearest-element queries of n given rays (one ray-tracing iteration, Sec.
 * 2.1-2.2), for comparing the two ways through the tree:
 *   RT_NEAREST_STACK   each ray alone, front to back with a stack (the
 *                      traversal of rt_trace's bounce kernel);
 *   RT_NEAREST_LEVELS  the paper's distribution of rays through the tree
 *                      level by level (Sec. 2.2): every (ray, box) pair of a
 *                      level tests the box's daughters with the slab test and
 *                      the ray goes on into each daughter it meets; leaf
 *                      elements are intersected when reached; boxes beyond a
 *                      ray's nearest hit so far are not entered.
 * Both give the same hits: the nearest triangle with an inclusive watertight
 * test, ties to the lowest id, the surface exclude_surface[i] (NULL: none)
 * skipped.  origins, directions: device [n][3]; hit (device [n], -1 = none),
 * t (device [n], +inf = none).  stats (host [2], nullable): node visits
 * (4-wide nodes opened) and triangle tests.  Synchronises (the level method
 * once per level).  Errors: RT_ERR_INVALID_ARG, RT_ERR_CAPACITY (a single
 * ray meets more than 2^26 boxes of one level), RT_ERR_STEP_LIMIT,
 * RT_ERR_STACK, RT_ERR_INTERNAL. */
#define RT_NEAREST_STACK 0
#define RT_NEAREST_LEVELS 1
rt_status rt_nearest_hits(const rt_tree* tree, const float* origins, const float* directions,
                          const int32_t* exclude_surface, int64_t n, int32_t method, int32_t* hit, float* t,
                          int64_t* stats, void* stream);

/* Tree statistics: nodes, leaves, depth, triangles, surfaces. */
rt_status rt_tree_info(const rt_tree* tree, int64_t* n_nodes, int64_t* n_tris, int32_t* depth,
                       int32_t* n_surfaces);

/* Propagate rays and build image sources.  band_absorption: host
 * [n_materials][8] alpha(f) in [0,1] (eq. 16).
 * Errors: RT_ERR_INVALID_ARG, RT_ERR_OOM, RT_ERR_CUDA, RT_ERR_CAPACITY (the
 * record buffer is resized and the trace re-run once before this is
 * returned), RT_ERR_STACK, RT_ERR_STEP_LIMIT. */
rt_status rt_trace(const rt_tree* tree, const rt_sources* src, const rt_receivers* rcv,
                   const float* band_absorption, int32_t n_materials, const rt_trace_params* params,
                   rt_image_sources** out);
/* Many rooms of uneven size in one persistent launch (config: batched rooms).
 * Every source of every room sends params->n_rays rays; sources and receivers
 * are numbered room after room (receiver k of room r has global index
 * sum_{r'<r} n_receivers(r') + k), and so are traced rays (ray q belongs to
 * global source q / ray_count).  Each ray meets only its own room's tree.
 * Errors as rt_trace. */
rt_status rt_trace_batch(const rt_room* rooms, int32_t n_rooms, const rt_trace_params* params,
                         rt_image_sources** out);
rt_status rt_image_sources_view(const rt_image_sources* is, rt_is_view* out);
void rt_image_sources_free(rt_image_sources* is);

/* Energy impulse responses: H[k][f][floor(t_s fs)] += E_s(f) summed in FP64
 * in a fixed order (deterministic), stored as float.  duration <= 0: up to
 * the latest arrival.  Image sources later than duration are dropped. */
rt_status rt_rir(const rt_image_sources* is, double fs, double duration, void* stream, rt_response** out);
rt_status rt_response_get(const rt_response* rir, rt_response_view* out);
/* Copy the histograms to host memory dst [n_rcv][8][n_bins] (synchronous). */
rt_status rt_response_download(const rt_response* rir, float* dst, void* stream);
void rt_response_free(rt_response* rir);

/* rt_rir_static -- the histogram step of rt_rir without any device
 * allocation, for callers that cannot allocate while they run (a real-time
 * auralisation loop re-binning image sources for a moving listener under an
 * audio deadline; an application that reserves its GPU memory up front).
 * The paper has no counterpart: this is a deployment variant of rt_rir.
 *   time, rcv, energy: device arrays of n image sources (e.g. the time /
 *     rcv / energy fields of an rt_is_view): arrival time (s), receiver
 *     index, [n][8] band energy;
 *   hist: device output [n_rcv][8][n_bins], zero-filled and then summed by
 *     this call exactly as rt_rir does (same bins, same FP64 order);
 *   image sources with a receiver outside [0, n_rcv) or a bin outside
 *     [0, n_bins) are dropped.
 * Its sort scratch is one static device array of RT_RIR_STATIC_SCRATCH_BYTES
 * that every GPU loading the library holds until exit; all calls share it,
 * so calls whose GPU work overlaps race (serialise them).  The first call on
 * a device looks up the array's address, which loads the library's device
 * code on that device if nothing has loaded it yet: that first call may make
 * the driver allocate and may block, so a real-time caller makes one warm-up
 * call (any n, e.g. 0) before its deadline loop and before any stream
 * capture.  The address is kept for the life of the process: after
 * cudaDeviceReset (or a release of the device's primary context) later calls
 * are invalid.
 * Errors: RT_ERR_INVALID_ARG (n > RT_RIR_STATIC_MAX_SOURCES, bad sizes or
 * null arrays), RT_ERR_CUDA. */
#define RT_RIR_STATIC_MAX_SOURCES 524288
#define RT_RIR_STATIC_SCRATCH_BYTES 12910592
rt_status rt_rir_static(const double* time, const int32_t* rcv, const double* energy, int64_t n, int32_t n_rcv,
                        double fs, int64_t n_bins, float* hist, void* stream);

/* Message of the last error on this thread ("" if none). */
const char* rt_last_error(void);
int32_t rt_api_version(void);
/* Kernel launches made by this library in this process so far (for
 * accounting; monotonic, thread-safe). */
int64_t rt_launch_count(void);

/* Measurement utility (no counterpart in the paper): L2 read bandwidth of
 * the current device in GB/s, from streaming a 32 MiB L2-resident buffer 64
 * times per launch with L1-bypassing 128-bit loads: launches for at least
 * 200 ms first (a cold GPU raises its clocks), then the best of 10.  Used as
 * the roofline denominator of the traversal kernel.  Synchronises. */
rt_status rt_measure_l2_bandwidth(double* read_gbs, void* stream);

/* ---------------------------------------------------------------------------
 * Learned late-reverberation tail (no counterpart in the paper: the network
 * of the surrogate-tail mode, which predicts the traced tail).  A 3-layer
 * MLP: Linear(n_in, H) - GELU - Linear(H, H) - GELU - Linear(H, n_out), FP32
 * master weights with Adam, BF16 copies read by hand-written tensor-core
 * GEMMs (tcgen05.mma from swizzled shared-memory tiles into an FP32
 * accumulator in tensor memory).  Sizes must be multiples of 32.  x, target,
 * y are device float arrays [batch][n_in] / [batch][n_out].  The loss is the
 * mean squared error over batch x n_out.  Calls that synchronise (a loss
 * requested, rt_mlp_copy) return RT_ERR_CUDA if a GEMM timed out waiting for
 * its tensor-core operations.  Parameter block layout (rt_mlp_info offsets):
 * W1 [H][n_in], b1 [H], W2 [H][H], b2 [H], W3 [n_out][H], b3 [n_out].
 * ------------------------------------------------------------------------- */
typedef struct rt_mlp rt_mlp;
rt_status rt_mlp_create(int32_t n_in, int32_t n_hidden, int32_t n_out, uint64_t seed, void* stream, rt_mlp** out);
void rt_mlp_free(rt_mlp* net);
rt_status rt_mlp_info(const rt_mlp* net, int32_t* n_in, int32_t* n_hidden, int32_t* n_out, int64_t* n_params,
                      int64_t* offsets6);
rt_status rt_mlp_forward(rt_mlp* net, const float* x, int32_t batch, float* y, void* stream);
/* gradients of the loss into the network's gradient block; loss to *loss (host, nullable; synchronises) */
rt_status rt_mlp_gradients(rt_mlp* net, const float* x, const float* target, int32_t batch, float* loss,
                           void* stream);
/* gradients + one Adam step (beta 0.9 / 0.999, eps 1e-8, decoupled weight
 * decay as set by rt_mlp_set_weight_decay, default 0) */
rt_status rt_mlp_train_step(rt_mlp* net, const float* x, const float* target, int32_t batch, float lr,
                            float* loss, void* stream);
/* copy a parameter-sized FP32 block to or from host memory (synchronous):
 * what = 0 weights, 1 gradients, 2 first moments, 3 second moments */
rt_status rt_mlp_copy(rt_mlp* net, int32_t what, float* host, int32_t to_device, void* stream);
rt_status rt_mlp_set_weight_decay(rt_mlp* net, float weight_decay);
rt_status rt_mlp_get_step(const rt_mlp* net, int64_t* step);
rt_status rt_mlp_set_step(rt_mlp* net, int64_t step);

/* The BF16 GEMM of the network (measurement and test entry point, no
 * counterpart in the paper): C[M][N] = A[M][K] . B[N][K]^T with FP32
 * accumulation; A, B device BF16 row-major (K innermost, K % 8 == 0, rows
 * 16-byte aligned), C device float [M][N]; A, B, C and the workspace start on
 * 16-byte boundaries (RT_ERR_INVALID_ARG otherwise).
 * kernel RT_GEMM_TMA (the network's kernel): one persistent CTA per SM walks
 * 128 x bn output tiles (bn <= 256, a multiple of 16 chosen to cover N with
 * the fewest columns); tile loads by TMA into a 4-stage ring, one producer
 * warp, one MMA-issuing thread, two tensor-memory accumulators so that four
 * epilogue warps store one tile while the next is computed.  With a device
 * workspace (workspace_floats > 0) a product whose tiles fill less than half
 * of the SMs is also cut along K (at most 16 ranges, at least 4 K steps of 64
 * each, splits x M x N <= workspace_floats); the partial sums are added in
 * range order, so results do not depend on timing.  workspace may be NULL
 * with workspace_floats 0 (no cutting); the caller owns it.
 * kernel RT_GEMM_STAGED: tiles copied through registers by all warps,
 * 128 x 64 tiles (the earlier kernel; workspace unused).
 * ms (host, nullable): device time of the product's kernels, from CUDA events
 * recorded on the stream around them.
 * Synchronises; RT_ERR_CUDA if a tile timed out. */
#define RT_GEMM_TMA 0
#define RT_GEMM_STAGED 1
rt_status rt_gemm_bf16(const void* A, const void* B, int32_t M, int32_t N, int32_t K, float* C, int32_t kernel,
                       float* workspace, int64_t workspace_floats, float* ms, void* stream);

/* Specular tail prior of the learned tail (no counterpart in the paper).  In a
 * room whose walls are grouped by the axis their normal is closest to, a ray
 * of direction d loses energy at R(d) = sum_k |d_k| rate[k][f] + air[f] (1/s);
 * the energy histogram of a measurement sphere (Sec. 1.4, eq. 19 with beams of
 * n / N rays) then averages level * exp(-R t) over directions.  For every room
 * i, band f and bin b this writes
 *   out[i][f][b] = level[i] * sum_j w_j (1/dt) int_{t0 + b dt}^{t0 + (b+1) dt} exp(-R(d_j) t) dt
 * with the product Gauss-Legendre rule of n_nodes x n_nodes directions of the
 * first octant: theta and phi on the nodes of (0, pi / 2), d = (sin theta
 * cos phi, sin theta sin phi, cos theta), w_j = (pi / 4) w_theta sin theta *
 * w_phi / 2 for weights w on (-1, 1) (the area element over the octant's area
 * pi / 2).  R depends on |d_k| only, so this is the mean over the sphere.
 * rates [n][3][8], air [n][8], level [n], out [n][8][n_bins]: device float
 * arrays owned by the caller; rates and air must be >= 0 (not checked: a
 * negative rate gives a growing curve).  0 < n <= 65535, 0 < n_nodes <= 256,
 * n_bins > 0, dt > 0, t0 >= 0 are checked (RT_ERR_INVALID_ARG). */
rt_status rt_tail_prior(const float* rates, const float* air, const float* level, int32_t n, int32_t n_nodes,
                        float t0, float dt, int32_t n_bins, float* out, void* stream);

/* ---------------------------------------------------------------------------
 * Surrogate-tail mode (no counterpart in the paper: the learned late
 * reverberation of a room, with the method as fallback and judge).  A room is
 * traced twice with few rays -- 0-50 ms in 1 ms bins ("early") and a 2 s tail
 * probe in 10 ms bins, each a batched trace in one tail-mode launch of
 * 128-thread blocks -- and an ensemble of rt_mlp networks predicts its
 * 8-band tail (50 ms - 2 s in 10 ms bins) from those traces, the room's
 * descriptors and the specular tail prior (rt_tail_prior).  A gate sends the
 * room to full tracing when its descriptors leave the training range or the
 * prediction disagrees with its traces.  Every room of these calls is an
 * rt_room with one source and one receiver (receiver 0 listens to source 0);
 * volume[k] is room k's volume in m^3 (given, not derived: the mesh may be open
 * or inconsistently oriented).  All arrays are device float, row-major, owned
 * by the caller unless stated:
 *   desc  [n][RT_SUR_N_DESC]   log10 V, log10 S, area-weighted mean alpha [8],
 *         log10 (share of S whose normal is closest to x, y, z + 1e-6) [3],
 *         log10 (c A_k a_kf / (2 V) + 1e-6) [3][8] (A_k the area of axis group
 *         k, a_kf its area-weighted -ln(1 - alpha_f)), c beta [8], log10 r,
 *         log10 (V / bounding-box volume)
 *   early [n][8][RT_SUR_N_EARLY]  energy per 1 ms bin, 0-50 ms
 *   probe [n][8][RT_SUR_N_TAIL]   energy per 10 ms bin, 50 ms - 2 s, of the probe
 *   *_db  [n][8][RT_SUR_N_TAIL]   tail decay curve: 10 log10 (energy arriving
 *         from each 10 ms bin start to 2 s + 1e-30)
 *   X     [n][RT_SUR_N_FEAT]      network features: desc, 10 log10 (early +
 *         1e-10), and the probe's minus the prior's decay at 63 bins per band
 *         (each curve as its first value, then its decay relative to it
 *         clamped at -50 dB)
 *   env   [n][8][RT_SUR_N_ENV]    energy per 10 ms bin, 0-2 s
 * ------------------------------------------------------------------------- */
#define RT_SUR_N_DESC 47
#define RT_SUR_N_EARLY 50
#define RT_SUR_N_TAIL 195
#define RT_SUR_N_ENV 200
#define RT_SUR_N_FEAT 951

typedef struct rt_surrogate rt_surrogate;

typedef struct {
    int32_t early_rays;       /* rays of the 0-50 ms trace (0 = 65,536) */
    int32_t probe_rays;       /* rays of the 2 s tail probe (0 = 16,384) */
    int32_t full_rays;        /* rays of a full 2 s trace: fallback and reference (0 = 1,000,000) */
    int32_t rooms_per_launch; /* rooms traced together in one batched trace (0 = 16) */
    const float* air_beta;    /* [8] host, 1/m energy (eq. 19); NULL = none */
    double c;                 /* sound speed, 0 = 343.2 m/s */
    void* stream;
    rt_workspace* workspace;  /* NULL or a workspace for the batched traces */
} rt_surrogate_trace_params;

/* What the surrogate reads of n rooms: descriptors, the early trace, the
 * probe, the prior's decay curve, the base curve the networks correct (the
 * probe's level and decay over the first 200 ms of the tail, then the prior's
 * decay joined without a step) and the features.  Any output may be NULL.
 * Errors: RT_ERR_INVALID_ARG (n < 1, a room without exactly one receiver, a
 * volume <= 0), and those of rt_trace_batch. */
rt_status rt_surrogate_inputs(const rt_room* rooms, const double* volume, int32_t n,
                              const rt_surrogate_trace_params* p, float* desc, float* early, float* probe,
                              float* prior_db, float* base_db, float* X);
/* Full traces of n rooms (p->full_rays rays, 2 s of path, 10 ms bins): the
 * envelope env and its tail decay curve tail_db (either may be NULL). */
rt_status rt_surrogate_reference(const rt_room* rooms, int32_t n, const rt_surrogate_trace_params* p, float* env,
                                 float* tail_db);

typedef struct {
    int32_t n_nets;           /* ensemble members (0 = 4) */
    int32_t steps;            /* AdamW steps per member (0 = 6000), cosine learning-rate schedule */
    int32_t batch;            /* rooms per step (0 = 1024) */
    float lr;                 /* peak learning rate (0 = 1e-3) */
    float weight_decay;       /* decoupled weight decay (< 0: none; 0 = 1e-4) */
    float input_noise;        /* Gaussian noise on the normalised features, in standard deviations (< 0: none; 0 = 0.1) */
    float val_frac;           /* share of the rooms held out for validation (0 = 0.05) */
    int32_t log_every;        /* validation every this many steps; each member keeps its best weights (0 = 250) */
    uint64_t seed;
    void* stream;
} rt_surrogate_train_params;

/* Train the networks on n rooms: features X, target tail decay curves
 * tail_db (from rt_surrogate_reference), desc, base_db and prior_db (from
 * rt_surrogate_inputs).  The networks learn the difference between the
 * target and the base curve in the target form, normalised per column
 * (output columns scaled so that the level at 50 ms weighs 9 and the first
 * 300 ms 4 in the squared error).  The training range is the descriptors'
 * span over the training rooms; the gate's tolerances are the 99th
 * percentiles (at least 3 dB) of the join and probe gaps (rt_surrogate_gate)
 * on up to 4096 of the validation rooms.  Synchronises; n >= 64. */
rt_status rt_surrogate_train(const float* X, const float* tail_db, const float* desc, const float* base_db,
                             const float* prior_db, int32_t n, const rt_surrogate_train_params* p,
                             rt_surrogate** out);
void rt_surrogate_free(rt_surrogate* model);
/* Ensemble size, gate tolerances (dB) and validation history
 * (n_history x (member, step, loss), copied when history is not NULL). */
rt_status rt_surrogate_info(const rt_surrogate* model, int32_t* n_nets, float* join_db, float* probe_db,
                            int32_t* n_history, float* history);
/* Serialise a model into host memory: with buf NULL only *bytes is set. */
rt_status rt_surrogate_save(const rt_surrogate* model, void* buf, size_t cap, size_t* bytes);
rt_status rt_surrogate_load(const void* buf, size_t bytes, void* stream, rt_surrogate** out);

/* Predicted tail decay curves pred_db of n rooms from their features and
 * base curves (ensemble mean in the target form, plus the base curve). */
rt_status rt_surrogate_predict(const rt_surrogate* model, const float* X, const float* base_db, int32_t n,
                               float* pred_db, void* stream);
/* Gate of n rooms: pass (host [n]) = descriptors within the training range
 * widened by 2 % of its span, join gap <= join_db and probe gap <= probe_db.
 * Join gap: the largest over the bands with traced energy in 40-50 ms of
 * |predicted 50-60 ms energy - traced 40-50 ms energy| in dB (0 when no band
 * has any: sparse early traces of large rooms say nothing about the join, and
 * the probe gap checks the level); probe gap: the largest over bands of the RMS difference (dB)
 * between the predicted and the probe's decay, both relative to the prior, at
 * the features' probe bins.  gaps (host [n][2], nullable) receives both.
 * Synchronises. */
rt_status rt_surrogate_gate(const rt_surrogate* model, const float* desc, const float* X, const float* pred_db,
                            const float* prior_db, int32_t n, int32_t* pass, float* gaps, void* stream);
/* Envelope env of n rooms: the early trace summed into 10 ms bins, then the
 * tail: per-bin energies (tail_is_db = 0) or a decay curve turned into
 * per-bin energies (made non-increasing first). */
rt_status rt_surrogate_envelope(const float* early, const float* tail, int32_t tail_is_db, int32_t n, float* env,
                                void* stream);

/* The surrogate-tail response of n rooms: rt_surrogate_inputs, prediction,
 * gate, and a full trace (p->full_rays) for every room that fails the gate.
 * *out: [n][8][RT_SUR_N_ENV] energies at fs = 100 Hz (rt_response_get; its
 * n_rcv is n); used_fallback (host [n], nullable): 1 where the room was traced
 * in full.  Synchronises. */
rt_status rt_rir_surrogate(const rt_room* rooms, const double* volume, int32_t n, const rt_surrogate* model,
                           const rt_surrogate_trace_params* p, rt_response** out, int32_t* used_fallback);

/* ---------------------------------------------------------------------------
 * What the impulse responses feed (Sec. 1.4 and the perceptive factors of
 * Sec. 4).  The paper names the metrics and the octave-band FIR synthesis
 * without formulas; these are the usual definitions, on a histogram of
 * energies e[b] per bin [b / fs, (b + 1) / fs):
 *   E = sum e;  S[b] = sum_{b' >= b} e[b'];  L[b] = 10 log10 (S[b] / E) at t = b / fs
 *   b0 = first bin with e > 0 (the direct sound); n80 = ceil(0.08 fs), n50 = ceil(0.05 fs)
 *   EDT, T20, T30: -60 / slope of the least-squares line through the (t, L)
 *     of the bins b >= b0 with L in [0, -10], [-5, -25], [-5, -35] dB
 *     (seconds; NaN when no finite L reaches the lower limit, fewer than 2
 *     points qualify, or the slope is not negative)
 *   C80 = 10 log10 (sum_{b - b0 < n80} e / sum_{b - b0 >= n80} e) dB (+inf without late energy)
 *   D50 = sum_{b - b0 < n50} e / E;  Ts = sum ((b - b0 + 1/2) / fs) e / E seconds
 *   SPL = 10 log10 E, dB re the source energy (E_0 = 1)
 * ------------------------------------------------------------------------- */
#define RT_N_ROOM_PARAMS 7   /* EDT, T20, T30, C80, D50, Ts, SPL */

/* Parameters of device histograms H [n_rcv][8][n_bins] (float, e.g. an
 * rt_response's data) into host out [n_rcv][8][RT_N_ROOM_PARAMS] (FP64 sums,
 * fixed order: the same result on every run).  A band without energy gets
 * NaN throughout.  Synchronises `stream`.  0 < n_rcv <= 65535, n_bins > 0,
 * fs > 0 (RT_ERR_INVALID_ARG otherwise). */
rt_status rt_room_parameters(const float* H, int32_t n_rcv, int64_t n_bins, double fs, double* out,
                             void* stream);

/* Pressure impulse responses of image sources (p = sqrt(E) per image source,
 * Sec. 1.4), synthesised over the 8 octave bands:
 *   p[k][t] = sum_{s of receiver k} sum_f sqrt(E_s(f)) g_f[t - floor(t_s fs) + D]
 * for t in [0, n_out), with g_f the linear-phase octave band-pass filter of
 * band f (centre 62.5 Hz * 2^f, edges f_c / sqrt 2 and f_c sqrt 2): the
 * difference of two ideal low-pass sincs 2 F / fs sinc(2 F (n - D) / fs) for
 * the two edges, times the Hann window 1/2 (1 - cos(2 pi n / (n_taps - 1))),
 * n = 0 .. n_taps - 1, D = (n_taps - 1) / 2 (zero-phase alignment on the
 * arrival bin).  out: device float [n_rcv][n_out], every sample written; sums
 * in FP64 over the sources in (arrival bin, index) order.  Synchronises
 * `stream`.  fs > 0, 0 < n_out < 2^31, odd 3 <= n_taps <= 2^20. */
rt_status rt_pressure_rir(const rt_image_sources* is, double fs, int64_t n_out, int32_t n_taps, float* out,
                          void* stream);

/* Workspace: queues and counters kept between traces on one stream, and the
 * CUDA graph of the bounce loop.  Free it after its last trace finished. */
rt_status rt_workspace_create(rt_workspace** out);
void rt_workspace_free(rt_workspace* ws);
/* Number of graph launches the workspace has made (0 if graphs were not used). */
int64_t rt_workspace_graph_launches(const rt_workspace* ws);

/* Optional device allocator (e.g. a framework's caching allocator).  Both
 * NULL restores cudaMallocAsync / cudaFreeAsync on the call's stream.  An
 * allocator that returns NULL makes the call fail with RT_ERR_OOM.  Blocks
 * must be 256-byte aligned, as cudaMalloc's are (the kernels use 16- and
 * 32-byte vector accesses): a block that is not goes straight back to
 * free_fn and the call fails with RT_ERR_OOM, before any kernel uses it. */
typedef void* (*rt_alloc_fn)(size_t bytes, void* stream, void* ctx);
typedef void (*rt_free_fn)(void* ptr, void* stream, void* ctx);
rt_status rt_set_allocator(rt_alloc_fn alloc, rt_free_fn free_fn, void* ctx);

#ifdef __cplusplus
}
#endif
#endif /* ROOMRAYS_H */
