/*
 * rt_oracle.c -- plain FP64 CPU oracle of the ray-propagation path.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the CPU
 * baseline leg of the benchmark load this file's library.  It shares no code,
 * header, table or constant generator with the CUDA library: both read the
 * same seeded input arrays and nothing else from each other.
 *
 * What it follows (paper: Aussal & Gueguen 2018, "Open-source platforms for
 * fast room acoustic simulations in complex structures"):
 *   - rays from an omnidirectional source: origin x_s, directions from a
 *     uniform sphere sampling (Fibonacci rule), equal energies      Sec. 1.2
 *   - nearest element: parametric line a + delta u against the plane
 *     b + lambda v + mu w of each triangle, 0<=lambda, 0<=mu,
 *     lambda+mu<=1, delta>0, delta minimal; solved with the
 *     Moller-Trumbore algorithm                                     Sec. 2.1, eq. 20-21
 *   - measurement sphere (x - x_m)^2 - r^2 = 0                       Sec. 2.1, eq. 22
 *   - specular reflection u_r = (u.T)T - (u.n)n                      Sec. 1.3, eq. 15
 *   - band absorption E_r(f) = E_i(f)(1 - alpha(f))                  Sec. 1.3, eq. 16
 *   - propagate while the distance travelled obeys eq. 13; rays that
 *     meet no surface (open air) are eliminated                      Sec. 2.1
 *   - binary tree: mother box, split along the largest dimension at
 *     the median until one element per leaf                          Sec. 2.2
 *
 * Readings where the paper is silent:
 *   - Fibonacci rule: z_i = 1-(2i+1)/N, rho = sqrt(1-z^2),
 *     phi_i = 2 pi frac(i g), g = (3 - sqrt 5)/2; each direction
 *     component is rounded to float32 and promoted back.
 *   - exact delta ties go to the lowest triangle index; the triangle hit on
 *     the previous bounce is excluded and delta must exceed eps_self.
 *   - receiver crossing of segment [o, o + delta u]: closest point
 *     t* = clamp((x_m - o).u, 0, delta), crossing iff |o + t* u - x_m| <= r.
 *   - energy per ray starts at 1/N per band (E_m = n/N, eq. 7).
 *   - bounce b (0-based) is the b-th nearest-element query; its segment has
 *     reflection order m = b.
 *
 * Ambiguity report (not part of the method; tells the tests which decisions
 * a float32 implementation may legitimately take the other way):
 *   - near tie: the second-nearest admissible hit is within 1e-6 relative of
 *     the nearest;
 *   - near edge: some triangle whose plane is met no farther than the
 *     nearest hit (times 1+1e-6) is missed, or hit, within eps_edge of its
 *     boundary (eps_edge = eps_rel * (|o|_inf + delta + 1)).
 *
 * Compile with -ffp-contract=off so every product and sum rounds as written.
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define NB 8

typedef struct {
    int64_t M;
    double *v0, *e1, *e2;      /* [M][3] */
    double *nrm;               /* [M][3] unit normal */
    double *h;                 /* [M][3] heights opposite vertex 0,1,2 */
    int32_t *mat, *surf;
    double *alpha;             /* [n_mat][NB] */
    int32_t n_mat;
    double diam;
    /* median-split tree: nodes with box and either two children or one leaf */
    int64_t n_nodes;
    double *lo, *hi;           /* [n_nodes][3] */
    int64_t *left, *right;     /* child node ids, -1 for leaf */
    int64_t *leaf_tri;         /* triangle id for a leaf, -1 otherwise */
    int64_t root;
} orc_scene;

/* ------------------------------------------------------------------------ */
/* median-split binary tree (Sec. 2.2): split the box's largest dimension at
 * the median of the element centroids, recursively, one element per leaf.   */
/* ------------------------------------------------------------------------ */
typedef struct { orc_scene* s; double* cen; int64_t* idx; int axis; } sort_ctx;
static sort_ctx g_sort; /* qsort has no context argument; build is single-threaded */

static int cmp_centroid(const void* a, const void* b) {
    int64_t i = *(const int64_t*)a, j = *(const int64_t*)b;
    double ci = g_sort.cen[3 * i + g_sort.axis], cj = g_sort.cen[3 * j + g_sort.axis];
    if (ci < cj) return -1;
    if (ci > cj) return 1;
    return (i < j) ? -1 : (i > j);
}

static void tri_box(const orc_scene* s, int64_t t, double* lo, double* hi) {
    for (int k = 0; k < 3; k++) {
        double a = s->v0[3 * t + k], b = a + s->e1[3 * t + k], c = a + s->e2[3 * t + k];
        double mn = a < b ? a : b, mx = a > b ? a : b;
        mn = mn < c ? mn : c;
        mx = mx > c ? mx : c;
        lo[k] = mn;
        hi[k] = mx;
    }
}

static int64_t build_rec(orc_scene* s, int64_t* idx, int64_t n, double* cen) {
    int64_t id = s->n_nodes++;
    double lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
    for (int64_t i = 0; i < n; i++) {
        double a[3], b[3];
        tri_box(s, idx[i], a, b);
        for (int k = 0; k < 3; k++) {
            if (a[k] < lo[k]) lo[k] = a[k];
            if (b[k] > hi[k]) hi[k] = b[k];
        }
    }
    memcpy(s->lo + 3 * id, lo, sizeof lo);
    memcpy(s->hi + 3 * id, hi, sizeof hi);
    if (n == 1) {
        s->left[id] = s->right[id] = -1;
        s->leaf_tri[id] = idx[0];
        return id;
    }
    int axis = 0;
    double ext[3] = {hi[0] - lo[0], hi[1] - lo[1], hi[2] - lo[2]};
    if (ext[1] > ext[axis]) axis = 1;
    if (ext[2] > ext[axis]) axis = 2;
    g_sort.s = s;
    g_sort.cen = cen;
    g_sort.axis = axis;
    qsort(idx, (size_t)n, sizeof(int64_t), cmp_centroid);
    int64_t half = n / 2;
    s->leaf_tri[id] = -1;
    int64_t l = build_rec(s, idx, half, cen);
    int64_t r = build_rec(s, idx + half, n - half, cen);
    s->left[id] = l;
    s->right[id] = r;
    return id;
}

void orc_scene_free(void* p) {
    orc_scene* s = (orc_scene*)p;
    if (!s) return;
    free(s->v0); free(s->e1); free(s->e2); free(s->nrm); free(s->h);
    free(s->mat); free(s->surf); free(s->alpha);
    free(s->lo); free(s->hi); free(s->left); free(s->right); free(s->leaf_tri);
    free(s);
}

static void cross3(const double* a, const double* b, double* c) {
    c[0] = a[1] * b[2] - a[2] * b[1];
    c[1] = a[2] * b[0] - a[0] * b[2];
    c[2] = a[0] * b[1] - a[1] * b[0];
}
static double dot3(const double* a, const double* b) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }

void* orc_scene_new(const double* V, int64_t nV, const int32_t* T, int64_t M, const int32_t* mat,
                    const int32_t* surf, const double* alpha, int32_t n_mat, int32_t build_tree) {
    (void)nV;
    orc_scene* s = (orc_scene*)calloc(1, sizeof(orc_scene));
    s->M = M;
    s->v0 = malloc(sizeof(double) * 3 * (M + 1));
    s->e1 = malloc(sizeof(double) * 3 * (M + 1));
    s->e2 = malloc(sizeof(double) * 3 * (M + 1));
    s->nrm = malloc(sizeof(double) * 3 * (M + 1));
    s->h = malloc(sizeof(double) * 3 * (M + 1));
    s->mat = malloc(sizeof(int32_t) * (M + 1));
    s->surf = malloc(sizeof(int32_t) * (M + 1));
    s->alpha = malloc(sizeof(double) * NB * (n_mat + 1));
    s->n_mat = n_mat;
    memcpy(s->alpha, alpha, sizeof(double) * NB * n_mat);
    double lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
    for (int64_t t = 0; t < M; t++) {
        const double *a = V + 3 * T[3 * t], *b = V + 3 * T[3 * t + 1], *c = V + 3 * T[3 * t + 2];
        for (int k = 0; k < 3; k++) {
            s->v0[3 * t + k] = a[k];
            s->e1[3 * t + k] = b[k] - a[k];
            s->e2[3 * t + k] = c[k] - a[k];
            double m3[3] = {a[k], b[k], c[k]};
            for (int q = 0; q < 3; q++) {
                if (m3[q] < lo[k]) lo[k] = m3[q];
                if (m3[q] > hi[k]) hi[k] = m3[q];
            }
        }
        double n[3];
        cross3(s->e1 + 3 * t, s->e2 + 3 * t, n);
        double len = sqrt(dot3(n, n));
        for (int k = 0; k < 3; k++) s->nrm[3 * t + k] = n[k] / len;
        /* heights: twice the area over the opposite edge length */
        double ea[3] = {c[0] - b[0], c[1] - b[1], c[2] - b[2]};
        double la = sqrt(dot3(ea, ea)), lb = sqrt(dot3(s->e2 + 3 * t, s->e2 + 3 * t)),
               lc = sqrt(dot3(s->e1 + 3 * t, s->e1 + 3 * t));
        s->h[3 * t + 0] = len / la;  /* opposite vertex 0: edge b-c */
        s->h[3 * t + 1] = len / lb;  /* opposite vertex 1: edge c-a */
        s->h[3 * t + 2] = len / lc;  /* opposite vertex 2: edge a-b */
        s->mat[t] = mat[t];
        s->surf[t] = surf[t];
    }
    double ext[3] = {hi[0] - lo[0], hi[1] - lo[1], hi[2] - lo[2]};
    s->diam = M ? sqrt(dot3(ext, ext)) : 1.0;
    if (build_tree && M > 0) {
        int64_t cap = 2 * M;
        s->lo = malloc(sizeof(double) * 3 * cap);
        s->hi = malloc(sizeof(double) * 3 * cap);
        s->left = malloc(sizeof(int64_t) * cap);
        s->right = malloc(sizeof(int64_t) * cap);
        s->leaf_tri = malloc(sizeof(int64_t) * cap);
        int64_t* idx = malloc(sizeof(int64_t) * M);
        double* cen = malloc(sizeof(double) * 3 * M);
        for (int64_t t = 0; t < M; t++) {
            idx[t] = t;
            for (int k = 0; k < 3; k++)
                cen[3 * t + k] = s->v0[3 * t + k] + (s->e1[3 * t + k] + s->e2[3 * t + k]) / 3.0;
        }
        s->n_nodes = 0;
        s->root = build_rec(s, idx, M, cen);
        free(idx);
        free(cen);
    } else {
        s->root = -1;
    }
    return s;
}

int64_t orc_tree_nodes(void* p) { return ((orc_scene*)p)->n_nodes; }
double orc_scene_diameter(void* p) { return ((orc_scene*)p)->diam; }

/* ------------------------------------------------------------------------ */
/* Fibonacci sphere directions (Sec. 1.2), rounded to float32.               */
/* ------------------------------------------------------------------------ */
static void fib_dir(int64_t i, int64_t N, double* u) {
    double g = (3.0 - sqrt(5.0)) / 2.0;
    double z = 1.0 - (double)(2 * i + 1) / (double)N;
    double zz = z * z;
    double rho = sqrt(1.0 - zz);
    double f = (double)i * g;
    f = f - floor(f);
    double phi = 2.0 * M_PI * f;
    double x = rho * cos(phi), y = rho * sin(phi);
    u[0] = (double)(float)x;
    u[1] = (double)(float)y;
    u[2] = (double)(float)z;
}

void orc_fibonacci(int64_t N, int64_t n, const int64_t* ids, double* out) {
    for (int64_t k = 0; k < n; k++) fib_dir(ids[k], N, out + 3 * k);
}

/* Directional source (Sec. 1.2, footnote: a non-uniform spatial sampling).
 * Rays keep the energy 1/N; their directions follow the power pattern
 * p(mu) = (1 - a + a mu) / (2 (1 - a)) of mu = cos(angle to the axis w),
 * 0 <= a <= 1/2: the uniform rule's z, as u = (1 + z) / 2, is mapped through
 * the inverse of the cumulative F(mu) = u, the root of
 *   (a/2) mu^2 + (1 - a) mu + (1 - a) - a/2 - 2 (1 - a) u = 0
 * in [-1, 1], taken as mu = -2 C / (B + sqrt(B^2 - 2 a C)) (no cancellation
 * as a -> 0); a = 0 keeps mu = z.  The direction (rho cos phi, rho sin phi,
 * mu) is then turned from +z to the unit axis w with the orthonormal basis of
 * Duff et al. 2017 ("Building an orthonormal basis, revisited").  Every step
 * is one rounded FP64 operation in a fixed order. */
static void dir_dir(int64_t i, int64_t N, const double* w, double a, double* u) {
    double g = (3.0 - sqrt(5.0)) / 2.0;
    double z = 1.0 - (double)(2 * i + 1) / (double)N;
    double mu = z;
    if (a > 0.0) {
        double uu = (1.0 + z) / 2.0;
        double B = 1.0 - a;
        double C = (B - a / 2.0) - (2.0 * B) * uu;
        double D = B * B - (2.0 * a) * C;
        mu = (-2.0 * C) / (B + sqrt(D));
    }
    double rho = sqrt(1.0 - mu * mu);
    double f = (double)i * g;
    f = f - floor(f);
    double phi = 2.0 * M_PI * f;
    double cx = rho * cos(phi), cy = rho * sin(phi);
    double sg = w[2] >= 0.0 ? 1.0 : -1.0;
    double A = -1.0 / (sg + w[2]);
    double Bq = (w[0] * w[1]) * A;
    double t1[3] = {1.0 + ((sg * w[0]) * w[0]) * A, sg * Bq, -(sg * w[0])};
    double t2[3] = {Bq, sg + (w[1] * w[1]) * A, -w[1]};
    for (int k = 0; k < 3; k++) u[k] = (double)(float)((cx * t1[k] + cy * t2[k]) + mu * w[k]);
}

void orc_directions(int64_t N, int64_t n, const int64_t* ids, const double* axis, double a, double* out) {
    for (int64_t k = 0; k < n; k++) dir_dir(ids[k], N, axis, a, out + 3 * k);
}

/* ------------------------------------------------------------------------ */
/* Nearest element along a ray (Sec. 2.1, eq. 20-21; Moller-Trumbore).       */
/* ------------------------------------------------------------------------ */
typedef struct {
    int64_t best;     /* triangle, -1 = none */
    double d1, d2;    /* nearest and second-nearest admissible distance */
    double near_edge; /* smallest plane distance of a triangle met within eps_edge of its border */
} hit_acc;

/* Moller-Trumbore: returns 1 if the line meets the triangle's plane at a
 * finite parameter; fills delta and the signed distance of the plane point
 * from the triangle's border (>= 0 inside, inclusive). */
static int mt_plane(const orc_scene* s, int64_t t, const double* o, const double* u, double* delta,
                    double* border) {
    const double *v0 = s->v0 + 3 * t, *e1 = s->e1 + 3 * t, *e2 = s->e2 + 3 * t;
    double p[3], q[3], w[3];
    cross3(u, e2, p);
    double det = dot3(e1, p);
    if (det == 0.0) return 0;
    double inv = 1.0 / det;
    w[0] = o[0] - v0[0];
    w[1] = o[1] - v0[1];
    w[2] = o[2] - v0[2];
    double lam = dot3(w, p) * inv;
    cross3(w, e1, q);
    double mu = dot3(u, q) * inv;
    *delta = dot3(e2, q) * inv;
    double b0 = 1.0 - lam - mu;
    double d0 = b0 * s->h[3 * t + 0], d1 = lam * s->h[3 * t + 1], d2 = mu * s->h[3 * t + 2];
    double m = d0 < d1 ? d0 : d1;
    *border = m < d2 ? m : d2;
    return 1;
}

typedef struct {
    const double *o, *u;
    int64_t exclude;
    double eps_self, eps_edge_rel, oscale;
} query;

static void visit_tri(const orc_scene* s, const query* qy, int64_t t, hit_acc* acc) {
    if (t == qy->exclude) return;
    double delta, border;
    if (!mt_plane(s, t, qy->o, qy->u, &delta, &border)) return;
    if (!(delta > qy->eps_self)) return;
    double eps_edge = qy->eps_edge_rel * (qy->oscale + delta + 1.0);
    if (border >= 0.0) {
        if (delta < acc->d1 || (delta == acc->d1 && t < acc->best)) {
            if (acc->best >= 0) acc->d2 = acc->d1 < acc->d2 ? acc->d1 : acc->d2;
            acc->d1 = delta;
            acc->best = t;
        } else if (delta < acc->d2) {
            acc->d2 = delta;
        }
    }
    if (border > -eps_edge && border < eps_edge) {
        if (delta < acc->near_edge) acc->near_edge = delta;
    }
}

/* slab test (Williams et al.) against a box grown by pad; returns the entry distance */
static int box_hit(const double* lo, const double* hi, const double* o, const double* u, double pad,
                   double tmax, double* tenter) {
    double t0 = 0.0, t1 = tmax;
    for (int k = 0; k < 3; k++) {
        double a = lo[k] - pad, b = hi[k] + pad;
        if (u[k] == 0.0) {
            if (o[k] < a || o[k] > b) return 0;
            continue;
        }
        double ta = (a - o[k]) / u[k], tb = (b - o[k]) / u[k];
        if (ta > tb) { double x = ta; ta = tb; tb = x; }
        if (ta > t0) t0 = ta;
        if (tb < t1) t1 = tb;
        if (t0 > t1) return 0;
    }
    *tenter = t0;
    return 1;
}

static double cull_limit(const hit_acc* acc) {
    /* anything met beyond the nearest hit (with the tie band) cannot matter */
    if (acc->best < 0) return INFINITY;
    return acc->d1 * (1.0 + 2e-6) + 1e-12;
}

static void tree_rec(const orc_scene* s, const query* qy, int64_t node, hit_acc* acc, double pad) {
    double te;
    if (!box_hit(s->lo + 3 * node, s->hi + 3 * node, qy->o, qy->u, pad, cull_limit(acc), &te)) return;
    if (s->leaf_tri[node] >= 0) {
        visit_tri(s, qy, s->leaf_tri[node], acc);
        return;
    }
    /* front-to-back: visit the child whose box is entered first */
    int64_t a = s->left[node], b = s->right[node];
    double ta, tb;
    int ha = box_hit(s->lo + 3 * a, s->hi + 3 * a, qy->o, qy->u, pad, INFINITY, &ta);
    int hb = box_hit(s->lo + 3 * b, s->hi + 3 * b, qy->o, qy->u, pad, INFINITY, &tb);
    if (ha && hb && tb < ta) { int64_t x = a; a = b; b = x; }
    if (ha || hb) {
        tree_rec(s, qy, a, acc, pad);
        tree_rec(s, qy, b, acc, pad);
    }
}

/* Nearest admissible triangle for one ray.  Returns the ambiguity flag. */
static int nearest(const orc_scene* s, const double* o, const double* u, int64_t exclude, int brute,
                   double eps_self, double eps_edge_rel, int64_t* tri, double* d1, double* d2) {
    query qy = {o, u, exclude, eps_self, eps_edge_rel, 0.0};
    double om = fabs(o[0]);
    if (fabs(o[1]) > om) om = fabs(o[1]);
    if (fabs(o[2]) > om) om = fabs(o[2]);
    qy.oscale = om;
    hit_acc acc = {-1, INFINITY, INFINITY, INFINITY};
    if (brute || s->root < 0) {
        for (int64_t t = 0; t < s->M; t++) visit_tri(s, &qy, t, &acc);
    } else {
        double pad = eps_edge_rel * (om + s->diam + 1.0) * 4.0;
        tree_rec(s, &qy, s->root, &acc, pad);
    }
    *tri = acc.best;
    *d1 = acc.d1;
    *d2 = acc.d2;
    int amb = 0;
    if (acc.best >= 0 && acc.d2 <= acc.d1 * (1.0 + 1e-6)) amb = 1;
    if (acc.near_edge < INFINITY && (acc.best < 0 || acc.near_edge <= acc.d1 * (1.0 + 1e-6))) amb = 1;
    return amb;
}

/* ------------------------------------------------------------------------ */
/* threading helper                                                         */
/* ------------------------------------------------------------------------ */
typedef void (*range_fn)(void* ctx, int64_t begin, int64_t end, int tid);
typedef struct { range_fn fn; void* ctx; int64_t b, e; int tid; } th_arg;
static void* th_main(void* p) {
    th_arg* a = (th_arg*)p;
    a->fn(a->ctx, a->b, a->e, a->tid);
    return NULL;
}
static void parallel_for(int64_t n, int nthreads, range_fn fn, void* ctx) {
    if (nthreads < 1) nthreads = 1;
    if (nthreads > 256) nthreads = 256;
    if (n < nthreads) nthreads = n > 0 ? (int)n : 1;
    pthread_t th[256];
    th_arg args[256];
    for (int k = 0; k < nthreads; k++) {
        args[k].fn = fn;
        args[k].ctx = ctx;
        args[k].b = n * k / nthreads;
        args[k].e = n * (k + 1) / nthreads;
        args[k].tid = k;
    }
    for (int k = 1; k < nthreads; k++) pthread_create(&th[k], NULL, th_main, &args[k]);
    th_main(&args[0]);
    for (int k = 1; k < nthreads; k++) pthread_join(th[k], NULL);
}

/* ------------------------------------------------------------------------ */
/* lockstep queries: nearest triangle from given (origin, direction)         */
/* ------------------------------------------------------------------------ */
typedef struct {
    const orc_scene* s;
    const double *o, *u;
    const int32_t* excl;
    int brute;
    double eps_edge_rel;
    int32_t* tri;
    double *d1, *d2;
    int32_t* amb;
} nq_ctx;

static void nq_range(void* p, int64_t b, int64_t e, int tid) {
    (void)tid;
    nq_ctx* c = (nq_ctx*)p;
    double eps_self = 1e-9 * c->s->diam;
    for (int64_t i = b; i < e; i++) {
        int64_t t;
        c->amb[i] = nearest(c->s, c->o + 3 * i, c->u + 3 * i, c->excl ? c->excl[i] : -1, c->brute, eps_self,
                            c->eps_edge_rel, &t, c->d1 + i, c->d2 + i);
        c->tri[i] = (int32_t)t;
    }
}

void orc_nearest(void* scene, int64_t n, const double* o, const double* u, const int32_t* exclude,
                 int32_t brute, double eps_edge_rel, int32_t nthreads, int32_t* tri, double* d1, double* d2,
                 int32_t* amb) {
    nq_ctx c = {(orc_scene*)scene, o, u, exclude, brute, eps_edge_rel, tri, d1, d2, amb};
    parallel_for(n, nthreads, nq_range, &c);
}

/* ------------------------------------------------------------------------ */
/* Full propagation (free running) for a list of rays.                       */
/* ------------------------------------------------------------------------ */
typedef struct {
    int32_t rcv;
    int32_t m;
    int64_t ray;          /* index into the ray list */
    double L;             /* path length at the closest point */
    double margin;        /* (r - distance) / r */
    double pos[3], dir[3];
} rec_t;

/* Closest point of the segment [o, o + seg u] to the sphere centre x_m:
 * t* = clamp((x_m - o).u, 0, seg); crossing iff |o + t* u - x_m| <= r
 * (eq. 22), and, with the eq. 13 range on, L + t* <= dmax. */
static int sphere_crossing(const double* o, const double* u, double seg, const double* xm, double rad, double L,
                           double dmax, rec_t* out) {
    double w[3] = {xm[0] - o[0], xm[1] - o[1], xm[2] - o[2]};
    double ts = dot3(w, u);
    if (ts < 0.0) ts = 0.0;
    if (ts > seg) ts = seg;
    double q[3] = {o[0] + ts * u[0] - xm[0], o[1] + ts * u[1] - xm[1], o[2] + ts * u[2] - xm[2]};
    double dist = sqrt(dot3(q, q));
    if (!(dist <= rad && (dmax <= 0.0 || L + ts <= dmax))) return 0;
    out->L = L + ts;
    out->margin = (rad - dist) / rad;
    for (int k = 0; k < 3; k++) {
        out->pos[k] = o[k] + ts * u[k];
        out->dir[k] = u[k];
    }
    return 1;
}

/* Lockstep crossings: segment k starts at o[k] along u[k] for seg[k] (inf =
 * escaped) from a ray of source ray_src[k].  Writes up to cap (segment,
 * receiver, margin) triples and returns how many exist. */
int64_t orc_crossings(int64_t n, const double* o, const double* u, const double* seg, const int32_t* ray_src,
                      int64_t n_rcv, const double* rcv_c, const double* rcv_r, const int32_t* rcv_src, int64_t cap,
                      int64_t* out_seg, int32_t* out_rcv, double* out_margin) {
    int64_t k = 0;
    for (int64_t i = 0; i < n; i++) {
        for (int64_t r = 0; r < n_rcv; r++) {
            if (rcv_src[r] != ray_src[i]) continue;
            rec_t rc;
            if (sphere_crossing(o + 3 * i, u + 3 * i, seg[i], rcv_c + 3 * r, rcv_r[r], 0.0, 0.0, &rc)) {
                if (k < cap) {
                    out_seg[k] = i;
                    out_rcv[k] = (int32_t)r;
                    out_margin[k] = rc.margin;
                }
                k++;
            }
        }
    }
    return k;
}

typedef struct {
    const orc_scene* s;
    const double* src;
    const double* axis;     /* [S][3] unit source axes, or NULL: omnidirectional */
    const double* pattern;  /* [S] pattern coefficient a of each source */
    int64_t n_rcv;
    const double *rc, *rr;
    const int32_t* rsrc;
    int64_t N;
    const int32_t* lsrc;
    const int64_t* lray;
    int32_t B;
    double dmax;
    int brute;
    double eps_edge_rel;
    int32_t *hist, *first_amb, *n_hits;
    double *hist_t, *E, *L;
    rec_t** recs;         /* per thread */
    int64_t *nrec, *caprec;
} tr_ctx;

static void push_rec(tr_ctx* c, int tid, const rec_t* r) {
    if (c->nrec[tid] == c->caprec[tid]) {
        c->caprec[tid] = c->caprec[tid] ? 2 * c->caprec[tid] : 1024;
        c->recs[tid] = realloc(c->recs[tid], sizeof(rec_t) * c->caprec[tid]);
    }
    c->recs[tid][c->nrec[tid]++] = *r;
}

static void tr_range(void* p, int64_t b, int64_t e, int tid) {
    tr_ctx* c = (tr_ctx*)p;
    const orc_scene* s = c->s;
    double eps_self = 1e-9 * s->diam;
    for (int64_t i = b; i < e; i++) {
        int32_t si = c->lsrc[i];
        double o[3] = {c->src[3 * si], c->src[3 * si + 1], c->src[3 * si + 2]};
        double u[3];
        if (c->axis)
            dir_dir(c->lray[i], c->N, c->axis + 3 * c->lsrc[i], c->pattern[c->lsrc[i]], u);
        else
            fib_dir(c->lray[i], c->N, u);
        double E[NB];
        for (int f = 0; f < NB; f++) E[f] = 1.0 / (double)c->N;
        double L = 0.0;
        int64_t last = -1;
        int32_t famb = c->B, nh = 0;
        for (int32_t k = 0; k < c->B; k++) {
            c->hist[i * c->B + k] = -1;
            c->hist_t[i * c->B + k] = INFINITY;
        }
        for (int32_t bnc = 0; bnc < c->B; bnc++) {
            int64_t t;
            double d1, d2;
            int amb = nearest(s, o, u, last, c->brute, eps_self, c->eps_edge_rel, &t, &d1, &d2);
            if (amb && famb == c->B) famb = bnc;
            double seg = (t >= 0) ? d1 : INFINITY;
            /* measurement spheres of this ray's source (eq. 22) */
            for (int64_t r = 0; r < c->n_rcv; r++) {
                if (c->rsrc[r] != si) continue;
                rec_t rc;
                if (sphere_crossing(o, u, seg, c->rc + 3 * r, c->rr[r], L, c->dmax, &rc)) {
                    rc.rcv = (int32_t)r;
                    rc.m = bnc;
                    rc.ray = i;
                    push_rec(c, tid, &rc);
                }
            }
            if (t < 0) break; /* open air: the ray is eliminated */
            c->hist[i * c->B + bnc] = (int32_t)t;
            c->hist_t[i * c->B + bnc] = d1;
            nh++;
            /* move to the hit point, reflect (eq. 15), absorb (eq. 16) */
            for (int k = 0; k < 3; k++) o[k] = o[k] + d1 * u[k];
            const double* n = s->nrm + 3 * t;
            double un = dot3(u, n);
            for (int k = 0; k < 3; k++) u[k] = u[k] - 2.0 * un * n[k];
            const double* al = s->alpha + NB * s->mat[t];
            for (int f = 0; f < NB; f++) E[f] = E[f] * (1.0 - al[f]);
            L = L + d1;
            last = t;
            if (c->dmax > 0.0 && L > c->dmax) break; /* eq. 13 range */
        }
        for (int f = 0; f < NB; f++) c->E[i * NB + f] = E[f];
        c->L[i] = L;
        c->first_amb[i] = famb;
        c->n_hits[i] = nh;
    }
}

/* Returns the number of records found; writes at most rec_cap of them (in
 * ray-list order, then bounce, then receiver).  Call again with a larger
 * capacity if the return value exceeds rec_cap. */
int64_t orc_trace(void* scene, const double* src, const double* src_axis, const double* src_pattern,
                  int64_t n_rcv, const double* rcv_c, const double* rcv_r,
                  const int32_t* rcv_src, int64_t N, int64_t n_list, const int32_t* list_src,
                  const int64_t* list_ray, int32_t B, double max_distance, int32_t brute, double eps_edge_rel,
                  int32_t nthreads, int32_t* hist, double* hist_t, double* E_final, double* L_final,
                  int32_t* first_amb, int32_t* n_hits, int64_t rec_cap, int32_t* rec_rcv, int64_t* rec_ray,
                  int32_t* rec_m, double* rec_L, double* rec_margin, double* rec_pos, double* rec_dir) {
    if (nthreads < 1) nthreads = 1;
    if (nthreads > 256) nthreads = 256;
    tr_ctx c;
    memset(&c, 0, sizeof c);
    c.s = (orc_scene*)scene;
    c.src = src;
    c.axis = src_axis;
    c.pattern = src_pattern;
    c.n_rcv = n_rcv;
    c.rc = rcv_c;
    c.rr = rcv_r;
    c.rsrc = rcv_src;
    c.N = N;
    c.lsrc = list_src;
    c.lray = list_ray;
    c.B = B;
    c.dmax = max_distance;
    c.brute = brute;
    c.eps_edge_rel = eps_edge_rel;
    c.hist = hist;
    c.hist_t = hist_t;
    c.E = E_final;
    c.L = L_final;
    c.first_amb = first_amb;
    c.n_hits = n_hits;
    c.recs = calloc(256, sizeof(rec_t*));
    c.nrec = calloc(256, sizeof(int64_t));
    c.caprec = calloc(256, sizeof(int64_t));
    int nt = nthreads;
    if (n_list < nt) nt = n_list > 0 ? (int)n_list : 1;
    parallel_for(n_list, nt, tr_range, &c);
    int64_t total = 0;
    for (int k = 0; k < nt; k++) {
        for (int64_t j = 0; j < c.nrec[k]; j++) {
            if (total < rec_cap) {
                rec_t* r = &c.recs[k][j];
                rec_rcv[total] = r->rcv;
                rec_ray[total] = r->ray;
                rec_m[total] = r->m;
                rec_L[total] = r->L;
                rec_margin[total] = r->margin;
                for (int q = 0; q < 3; q++) {
                    rec_pos[3 * total + q] = r->pos[q];
                    rec_dir[3 * total + q] = r->dir[q];
                }
            }
            total++;
        }
        free(c.recs[k]);
    }
    free(c.recs);
    free(c.nrec);
    free(c.caprec);
    return total;
}
