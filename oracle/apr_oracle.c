/*
 * FP64 CPU oracle for adaptive particle refinement (APR) in compressible SPH.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test-suite, the smoke check and the CPU
 * baseline leg of the benchmark may load this library.  It shares no code,
 * header, table or constant generator with the CUDA library, and the CUDA
 * library never calls it.
 *
 * What it computes, and where each piece comes from (Nealon & Price,
 * "Adaptive particle refinement for compressible SPH", arXiv 2409.11470):
 *
 *   refinement level from position ............ Sec. 2.1 rules 1-3, Table 1 caption
 *   mass per level m(l) = m0 / 2^l ............. Sec. 2.1 rule 5, Eq. 1
 *   split: 1 parent -> 2 children, h scaled by (1/2)^(1/3), children at
 *          +-r_sep along a direction tangential to the zone boundary, rotated
 *          by a random angle, r_sep = min(0.2 h, 0.35 d_nn) ..... Sec. 2.2, Eq. 2
 *   merge: pairing by a k-d tree cut through the centre of mass with an even
 *          count on each side, leaves of exactly two; merge if the leaf's
 *          centre of mass lies at a lower level; survivor at the pair's centre
 *          of mass and velocity, h scaled by 2^(1/3); an odd particle is left
 *          for the next step ........................... Sec. 2.3, Eq. 3, Eq. 4
 *   per-step order: split levels ascending, then merge levels descending,
 *          one level change per particle per step ............... Sec. 2.6
 *   density / smoothing length: the paper cites the iterative h-rho solve of
 *          the Phantom code (Sec. 2.2) without printing it; this oracle takes
 *          the standard grad-h SPH definition: h is the unique root of
 *          sum_b m_b W(r_ab, h) = m_a (h_fact/h)^3 (self included), found by
 *          bisection to machine precision; M4 kernel, h_fact = 1.2 (Table 2)
 *   forces: standard grad-h SPH momentum/energy equations with the
 *          signal-velocity artificial viscosity and (optionally) artificial
 *          conductivity (the paper cites them, Sec. 3 and Sec. 4) -- a proposed
 *          reading, pinned by conservation laws, a lattice, a linear pressure
 *          gradient and the Sod shock tube closed form.
 *   density error of one split pass and its gradient with respect to the
 *          children's offsets and smoothing lengths (h held fixed): not in the
 *          paper, which motivates it (Sec. 2.2 r_sep choice, Sec. 2.5 relaxing
 *          to the original density); pinned by a hand-worked isolated split,
 *          exact reproduction when children sit on their parent, periodic
 *          translation invariance and central finite differences.
 *
 * Decisions (neighbour membership, nearest-neighbour distance, the pairing
 * tree's cuts) are taken on a quantised integer lattice x_int = floor((x-lo)/D)
 * so that they are exact and independent of summation order; all physical
 * values use the plain float64 coordinates.
 *
 * Build: gcc -O2 -std=c11 -fopenmp -ffp-contract=off -fPIC -shared.
 * -ffp-contract=off keeps every float64 operation a separately rounded IEEE
 * operation (no fused multiply-add), which the bit-exact split/merge
 * geometry relies on.
 */
#define _GNU_SOURCE
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_FLAG_CHANGED 1u
#define ORC_FLAG_FIXED 2u
#define ORC_FLAG_DEAD 4u
#define ORC_FLAG_NEW 8u /* introduced by a split or merge, until relaxed (Sec. 2.4) */
#define ORC_FLAG_INACTIVE 16u /* individual time steps: not at the end of its step */

#define ORC_MAXLEV 8
#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif
#define ORC_COORD_BITS 30
#define ORC_COORD_MAX ((1LL << ORC_COORD_BITS) - 1)

/* (1/2)^(1/3) and 2^(1/3) as float64 literals (Eq. 2 and Eq. 3) */
#define ORC_SPLIT_HFAC 0.7937005259840998
#define ORC_MERGE_HFAC 1.2599210498948732

typedef struct {
    double lo[3], hi[3];
    int periodic[3];
    double delta;
    double hfact, gamma;
    int eos; /* 0 adiabatic, 1 locally isothermal */
    double cs0, qcs;
    double alpha_av, beta_av, alpha_u;
    double rsep_fac, dnn_cap;
    double m0;
    int lmax;
    unsigned long long seed;
    double ccour, cforce, G;
    int nthreads;
    int enumerate; /* 0 brute force, 1 uniform cell list (same sets, sorted) */
    int kernel;        /* 0 M4 cubic spline, 1 Wendland C2 (both support 2h) */
    int level_default; /* 0: zones refine; L >= 1: zones derefine from level L */
} orc_cfg;

typedef struct {
    int shape; /* 0 sphere, 1 slab, 2 cylinder along axis */
    int axis;
    int track_sink; /* -1 fixed */
    int nlev;
    double centre[3];
    double R[ORC_MAXLEV];
} orc_region;

typedef struct {
    double x[3], v[3], a[3];
    double m, racc;
} orc_sink;

typedef struct {
    long long n, cap, next_id;
    double *x, *y, *z, *vx, *vy, *vz, *u, *h;
    double *rho, *omega, *ax, *ay, *az, *dudt, *vsig, *dnn, *pres, *cs;
    unsigned char *level, *flags;
    unsigned long long *id;
    unsigned char* bin; /* time-step bin (individual time steps); may be NULL otherwise */
} orc_state;

typedef struct {
    long long n_split[ORC_MAXLEV], n_merge[ORC_MAXLEV], n_spare[ORC_MAXLEV];
    long long n_accreted, n_dead;
} orc_counts;

typedef struct {
    double mass, mom[3], ang[3], ekin, etherm;
} orc_stats;

/* ------------------------------------------------------------------ basics */

int orc_threads(const orc_cfg* c)
{
#ifdef _OPENMP
    if (c && c->nthreads > 0) return c->nthreads;
    return omp_get_max_threads();
#else
    (void)c;
    return 1;
#endif
}

static void set_threads(const orc_cfg* c)
{
#ifdef _OPENMP
    if (c->nthreads > 0) omp_set_num_threads(c->nthreads);
#else
    (void)c;
#endif
}

/* particle mass from its refinement level: m(l) = m0 / 2^l (Eq. 1) */
static double mass_of(const orc_cfg* c, int level) { return ldexp(c->m0, -level); }

static double box_len(const orc_cfg* c, int k) { return c->hi[k] - c->lo[k]; }

long long orc_lattice_len(const orc_cfg* c, int k)
{
    return (long long)llround(box_len(c, k) / c->delta);
}

/* integer lattice coordinate of one component */
static long long quant1(const orc_cfg* c, int k, double x)
{
    long long q = (long long)floor((x - c->lo[k]) / c->delta);
    if (c->periodic[k]) {
        long long L = orc_lattice_len(c, k);
        q %= L;
        if (q < 0) q += L;
    } else {
        if (q < 0) q = 0;
        if (q > ORC_COORD_MAX) q = ORC_COORD_MAX;
    }
    return q;
}

void orc_quantise(const orc_cfg* c, long long n, const double* x, const double* y,
                  const double* z, long long* xi)
{
    for (long long i = 0; i < n; ++i) {
        xi[3 * i + 0] = quant1(c, 0, x[i]);
        xi[3 * i + 1] = quant1(c, 1, y[i]);
        xi[3 * i + 2] = quant1(c, 2, z[i]);
    }
}

/* squared lattice separation with the minimum image on periodic axes (exact) */
static unsigned long long r2_lattice(const orc_cfg* c, const long long* a, const long long* b)
{
    unsigned long long r2 = 0;
    for (int k = 0; k < 3; ++k) {
        long long d = a[k] - b[k];
        if (c->periodic[k]) {
            long long L = orc_lattice_len(c, k);
            if (2 * d > L) d -= L;
            else if (2 * d < -L) d += L;
        }
        r2 += (unsigned long long)(d * d);
    }
    return r2;
}

/* neighbour threshold: b is within the kernel radius 2h of a iff r2_lattice < thr(h) */
unsigned long long orc_threshold(const orc_cfg* c, double h)
{
    double t = (2.0 * h) / c->delta;
    double t2 = t * t;
    if (!(t2 < 4.6e18)) return 4611686018427387904ULL;
    return (unsigned long long)ceil(t2);
}

/* float64 minimum-image separation a - b */
static void sep64(const orc_cfg* c, const orc_state* s, long long a, long long b, double d[3])
{
    d[0] = s->x[a] - s->x[b];
    d[1] = s->y[a] - s->y[b];
    d[2] = s->z[a] - s->z[b];
    for (int k = 0; k < 3; ++k) {
        if (c->periodic[k]) {
            double L = box_len(c, k);
            if (d[k] > 0.5 * L) d[k] -= L;
            else if (d[k] < -0.5 * L) d[k] += L;
        }
    }
}

static int is_live(const orc_state* s, long long i) { return !(s->flags[i] & ORC_FLAG_DEAD); }

/* --------------------------------------------------------- M4 cubic spline */

/* f(q) and f'(q) of the M4 kernel, W = f(q)/(pi h^3), q = r/h, support 2h */
static void m4(double q, double* f, double* df)
{
    if (q < 1.0) {
        *f = 1.0 - 1.5 * q * q + 0.75 * q * q * q;
        *df = -3.0 * q + 2.25 * q * q;
    } else if (q < 2.0) {
        double t = 2.0 - q;
        *f = 0.25 * t * t * t;
        *df = -0.75 * t * t;
    } else {
        *f = 0.0;
        *df = 0.0;
    }
}

void orc_kernel_m4(double q, double* out2) { m4(q, &out2[0], &out2[1]); }

/* Wendland C2 with support 2h: f(q) = (1 - q/2)^4 (2q + 1); W = 21 f / (16 pi h^3) */
static void wendland_c2(double q, double* f, double* df)
{
    if (q < 2.0) {
        double t = 1.0 - 0.5 * q;
        *f = t * t * t * t * (2.0 * q + 1.0);
        *df = -5.0 * q * t * t * t;
    } else {
        *f = 0.0;
        *df = 0.0;
    }
}

/* the configured kernel shape f(q), f'(q) */
static void kern(const orc_cfg* c, double q, double* f, double* df)
{
    if (c->kernel == 1)
        wendland_c2(q, f, df);
    else
        m4(q, f, df);
}

/* W = f(q) / (kinv h^3): the inverse of the kernel's normalisation constant */
static double kinv(const orc_cfg* c) { return c->kernel == 1 ? 16.0 * M_PI / 21.0 : M_PI; }

void orc_kernel(int kernel, double q, double* out2)
{
    if (kernel == 1)
        wendland_c2(q, &out2[0], &out2[1]);
    else
        m4(q, &out2[0], &out2[1]);
}

/* ------------------------------------------------ candidate enumeration */

typedef struct {
    int nc[3];
    double cw[3];
    long long* head; /* first particle of each cell (CSR over cells) */
    long long* items;
    long long ncell;
} cellgrid;

static long long cell_coord(const orc_cfg* c, const cellgrid* g, int k, double x)
{
    long long i = (long long)floor((x - c->lo[k]) / g->cw[k]);
    if (c->periodic[k]) {
        i %= g->nc[k];
        if (i < 0) i += g->nc[k];
    } else {
        if (i < 0) i = 0;
        if (i >= g->nc[k]) i = g->nc[k] - 1;
    }
    return i;
}

static void grid_build(const orc_cfg* c, const orc_state* s, double width, cellgrid* g)
{
    long long n = s->n;
    for (int k = 0; k < 3; ++k) {
        double L = box_len(c, k);
        int m = (int)floor(L / width);
        if (m < 1) m = 1;
        if (m > 256) m = 256;
        g->nc[k] = m;
        g->cw[k] = L / m;
    }
    g->ncell = (long long)g->nc[0] * g->nc[1] * g->nc[2];
    g->head = (long long*)calloc((size_t)g->ncell + 1, sizeof(long long));
    g->items = (long long*)malloc(sizeof(long long) * (size_t)(n > 0 ? n : 1));
    long long* cid = (long long*)malloc(sizeof(long long) * (size_t)(n > 0 ? n : 1));
    for (long long i = 0; i < n; ++i) {
        long long cx = cell_coord(c, g, 0, s->x[i]);
        long long cy = cell_coord(c, g, 1, s->y[i]);
        long long cz = cell_coord(c, g, 2, s->z[i]);
        cid[i] = (cx * g->nc[1] + cy) * g->nc[2] + cz;
        g->head[cid[i] + 1]++;
    }
    for (long long k = 0; k < g->ncell; ++k) g->head[k + 1] += g->head[k];
    long long* fill = (long long*)malloc(sizeof(long long) * (size_t)g->ncell);
    for (long long k = 0; k < g->ncell; ++k) fill[k] = g->head[k];
    for (long long i = 0; i < n; ++i) g->items[fill[cid[i]]++] = i;
    free(fill);
    free(cid);
}

static void grid_free(cellgrid* g)
{
    free(g->head);
    free(g->items);
}

typedef struct {
    long long* idx;
    double* r2;
    long long n, cap;
} blist;

static void bl_push(blist* L, long long b, double r2)
{
    if (L->n == L->cap) {
        L->cap = L->cap ? 2 * L->cap : 256;
        L->idx = (long long*)realloc(L->idx, sizeof(long long) * (size_t)L->cap);
        L->r2 = (double*)realloc(L->r2, sizeof(double) * (size_t)L->cap);
    }
    L->idx[L->n] = b;
    L->r2[L->n] = r2;
    L->n++;
}

/*
 * k-d tree over the particles for range queries (enumeration only: a query
 * returns exactly the particles a scan over all of them would, and every
 * caller sorts them by index, so the tree's shape never enters a result).
 * Each node holds the bounding box and the largest h of its live particles;
 * internal nodes split at the median of their widest axis; leaves hold at
 * most KD_LEAF particles.  Unlike a uniform grid it stays efficient where the
 * particle density spans orders of magnitude (a disc's midplane and tails).
 */
#define KD_LEAF 16

typedef struct {
    double lo[3], hi[3];
    double hmax;
    long long first, count;
    long long left, right; /* -1 for a leaf */
} kdnode;

typedef struct {
    kdnode* node;
    long long nnode, cap;
    long long* items;
} kdtree;

static double coord_of(const orc_state* s, int k, long long i)
{
    return k == 0 ? s->x[i] : (k == 1 ? s->y[i] : s->z[i]);
}

/* rearrange it[0..n) so that it[m] holds the element of rank m along axis k,
 * smaller-or-equal ones before it and larger-or-equal ones after (quickselect) */
static void kd_select(const orc_state* s, int k, long long* it, long long n, long long m)
{
    long long lo = 0, hi = n - 1;
    while (lo < hi) {
        const double pivot = coord_of(s, k, it[lo + (hi - lo) / 2]);
        long long i = lo, j = hi;
        while (i <= j) {
            while (coord_of(s, k, it[i]) < pivot) ++i;
            while (coord_of(s, k, it[j]) > pivot) --j;
            if (i <= j) {
                long long tmp = it[i];
                it[i] = it[j];
                it[j] = tmp;
                ++i;
                --j;
            }
        }
        if (m <= j) hi = j;
        else if (m >= i) lo = i;
        else break;
    }
}

static long long kd_build_node(kdtree* t, const orc_state* s, long long first, long long count)
{
    long long id;
#pragma omp atomic capture
    id = t->nnode++;
    kdnode* nd = &t->node[id];
    nd->first = first;
    nd->count = count;
    nd->left = nd->right = -1;
    nd->hmax = 0.0;
    for (int k = 0; k < 3; ++k) {
        nd->lo[k] = INFINITY;
        nd->hi[k] = -INFINITY;
    }
    for (long long q = first; q < first + count; ++q) {
        long long i = t->items[q];
        for (int k = 0; k < 3; ++k) {
            double v = coord_of(s, k, i);
            if (v < nd->lo[k]) nd->lo[k] = v;
            if (v > nd->hi[k]) nd->hi[k] = v;
        }
        if (s->h[i] > nd->hmax) nd->hmax = s->h[i];
    }
    if (count <= KD_LEAF) return id;
    int axis = 0;
    for (int k = 1; k < 3; ++k)
        if (nd->hi[k] - nd->lo[k] > nd->hi[axis] - nd->lo[axis]) axis = k;
    const long long m = count / 2;
    kd_select(s, axis, t->items + first, count, m);
    long long l, r;
    if (count > 65536) {
#pragma omp task shared(l)
        l = kd_build_node(t, s, first, m);
#pragma omp task shared(r)
        r = kd_build_node(t, s, first + m, count - m);
#pragma omp taskwait
    } else {
        l = kd_build_node(t, s, first, m);
        r = kd_build_node(t, s, first + m, count - m);
    }
    t->node[id].left = l;
    t->node[id].right = r;
    return id;
}

/* a tree over the live particles of s */
static void kd_build(const orc_state* s, kdtree* t)
{
    long long n = 0;
    for (long long i = 0; i < s->n; ++i)
        if (is_live(s, i)) ++n;
    t->items = (long long*)malloc(sizeof(long long) * (size_t)(n ? n : 1));
    n = 0;
    for (long long i = 0; i < s->n; ++i)
        if (is_live(s, i)) t->items[n++] = i;
    /* leaves hold at least KD_LEAF / 2 particles: fewer than 4 n / KD_LEAF + 1 nodes */
    t->cap = 4 * n / KD_LEAF + 2;
    t->node = (kdnode*)malloc(sizeof(kdnode) * (size_t)t->cap);
    t->nnode = 0;
    if (n == 0) return;
#pragma omp parallel
#pragma omp single
    kd_build_node(t, s, 0, n);
}

static void kd_free(kdtree* t)
{
    free(t->node);
    free(t->items);
}

/* squared distance from p to the node's box, the smallest over periodic images
 * (never more than the computed separation of p from a particle inside it) */
static double kd_gap2(const orc_cfg* c, const double p[3], const kdnode* nd)
{
    double s2 = 0.0;
    for (int k = 0; k < 3; ++k) {
        double g = 0.0;
        if (p[k] < nd->lo[k]) g = nd->lo[k] - p[k];
        else if (p[k] > nd->hi[k]) g = p[k] - nd->hi[k];
        if (c->periodic[k] && g > 0.0) {
            const double L = box_len(c, k);
            for (int img = -1; img <= 1; img += 2) {
                const double v = p[k] + img * L;
                double gi = 0.0;
                if (v < nd->lo[k]) gi = nd->lo[k] - v;
                else if (v > nd->hi[k]) gi = v - nd->hi[k];
                if (gi < g) g = gi;
            }
        }
        s2 += g * g;
    }
    return s2;
}

/*
 * Every live b with |x_a - x_b| < R (sym = 0), or a superset of the b with
 * |x_a - x_b| < 2 max(h_a, h_b) (sym = 1: nodes whose box is farther than
 * 2 max(h_a, largest h inside) are skipped), appended to out unsorted with
 * their squared separations.  A node is skipped only when its box gap exceeds
 * the radius by a relative 1e-9, far above the rounding of either distance.
 */
static void kd_query(const orc_cfg* c, const orc_state* s, const kdtree* t, long long a, double R,
                     int sym, blist* out)
{
    if (t->nnode == 0) return;
    const double p[3] = {s->x[a], s->y[a], s->z[a]};
    long long stack[128];
    int sp = 0;
    stack[sp++] = 0;
    while (sp > 0) {
        const kdnode* nd = &t->node[stack[--sp]];
        double Rn = R;
        if (sym) Rn = 2.0 * (s->h[a] > nd->hmax ? s->h[a] : nd->hmax);
        if (kd_gap2(c, p, nd) > Rn * Rn * (1.0 + 1e-9)) continue;
        if (nd->left < 0) {
            const double R2 = Rn * Rn;
            for (long long q = nd->first; q < nd->first + nd->count; ++q) {
                long long b = t->items[q];
                double d[3];
                sep64(c, s, a, b, d);
                double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
                if (r2 < R2) bl_push(out, b, r2);
            }
        } else {
            stack[sp++] = nd->right;
            stack[sp++] = nd->left;
        }
    }
}


static int cmp_ll(const void* a, const void* b)
{
    long long x = *(const long long*)a, y = *(const long long*)b;
    return (x > y) - (x < y);
}

/* sort a gathered list by particle index, so that sums do not depend on the
 * enumeration */
static void sort_gathered(const orc_cfg* c, const orc_state* s, long long a, blist* out);

/* all live b (b may equal a) with |x_a - x_b| < R, sorted by index (g == NULL:
 * a scan over every particle; else the k-d tree) */
static void gather_within(const orc_cfg* c, const orc_state* s, const kdtree* g, long long a,
                          double R, blist* out)
{
    out->n = 0;
    double R2 = R * R;
    if (!g) {
        for (long long b = 0; b < s->n; ++b) {
            if (!is_live(s, b)) continue;
            double d[3];
            sep64(c, s, a, b, d);
            double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
            if (r2 < R2) bl_push(out, b, r2);
        }
        return;
    }
    kd_query(c, s, g, a, R, 0, out);
    sort_gathered(c, s, a, out);
}

/* a superset, sorted by index, of the live b with |x_a - x_b| < 2 max(h_a, h_b) */
static void gather_symmetric(const orc_cfg* c, const orc_state* s, const kdtree* g, long long a,
                             double hmax, blist* out)
{
    if (!g) {
        gather_within(c, s, NULL, a, 2.0 * (s->h[a] > hmax ? s->h[a] : hmax), out);
        return;
    }
    out->n = 0;
    kd_query(c, s, g, a, 0.0, 1, out);
    sort_gathered(c, s, a, out);
}

static void sort_gathered(const orc_cfg* c, const orc_state* s, long long a, blist* out)
{
    /* sort by particle index so that sums do not depend on the enumeration */
    long long* key = (long long*)malloc(sizeof(long long) * (size_t)(out->n ? out->n : 1));
    for (long long t = 0; t < out->n; ++t) key[t] = out->idx[t];
    qsort(key, (size_t)out->n, sizeof(long long), cmp_ll);
    for (long long t = 0; t < out->n; ++t) {
        long long b = key[t];
        double d[3];
        sep64(c, s, a, b, d);
        out->idx[t] = b;
        out->r2[t] = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
    }
    free(key);
}

static double max_live_h(const orc_state* s)
{
    double m = 0.0;
    for (long long i = 0; i < s->n; ++i)
        if (is_live(s, i) && s->h[i] > m) m = s->h[i];
    return m;
}

/* ------------------------------------------------------ neighbour lists */

/*
 * Neighbour lists on the quantised lattice.  mode 0 (gather): b != a with
 * r2 < thr(h_a).  mode 1 (symmetric): r2 < max(thr(h_a), thr(h_b)).  Lists are
 * in ascending index order.  Returns the total number of entries, or -1 if it
 * exceeds cap (offsets are still complete).
 */
long long orc_neighbours(const orc_cfg* c, const orc_state* s, int mode, long long* offsets,
                         int* idx, long long cap)
{
    long long n = s->n;
    long long* xi = (long long*)malloc(sizeof(long long) * 3 * (size_t)(n ? n : 1));
    orc_quantise(c, n, s->x, s->y, s->z, xi);
    unsigned long long* thr =
        (unsigned long long*)malloc(sizeof(unsigned long long) * (size_t)(n ? n : 1));
    for (long long i = 0; i < n; ++i) thr[i] = orc_threshold(c, s->h[i]);
    long long* cnt = (long long*)calloc((size_t)n + 1, sizeof(long long));
    set_threads(c);
#pragma omp parallel for schedule(dynamic, 64)
    for (long long a = 0; a < n; ++a) {
        if (!is_live(s, a)) continue;
        long long k = 0;
        for (long long b = 0; b < n; ++b) {
            if (b == a || !is_live(s, b)) continue;
            unsigned long long r2 = r2_lattice(c, &xi[3 * a], &xi[3 * b]);
            unsigned long long t = thr[a];
            if (mode == 1 && thr[b] > t) t = thr[b];
            if (r2 < t) ++k;
        }
        cnt[a] = k;
    }
    offsets[0] = 0;
    for (long long a = 0; a < n; ++a) offsets[a + 1] = offsets[a] + cnt[a];
    long long total = offsets[n];
    if (total > cap) {
        free(xi);
        free(thr);
        free(cnt);
        return -1;
    }
#pragma omp parallel for schedule(dynamic, 64)
    for (long long a = 0; a < n; ++a) {
        if (!is_live(s, a)) continue;
        long long k = offsets[a];
        for (long long b = 0; b < n; ++b) {
            if (b == a || !is_live(s, b)) continue;
            unsigned long long r2 = r2_lattice(c, &xi[3 * a], &xi[3 * b]);
            unsigned long long t = thr[a];
            if (mode == 1 && thr[b] > t) t = thr[b];
            if (r2 < t) idx[k++] = (int)b;
        }
    }
    free(xi);
    free(thr);
    free(cnt);
    return total;
}

/* -------------------------------------------------------------- density */

/*
 * pi h^3 (rho_sum(h) - rho_h(h)) and its h-derivative over a candidate list of
 * (r, m_b); non-decreasing in h with a single sign change.
 */
static double g_of_h(const orc_cfg* c, const double* r, const double* mb, long long n, double ma,
                     double h, double* dg)
{
    double sum = 0.0, d = 0.0;
    for (long long t = 0; t < n; ++t) {
        double q = r[t] / h, f, df;
        kern(c, q, &f, &df);
        sum += mb[t] * f;
        d += mb[t] * df * (-q / h);
    }
    if (dg) *dg = d;
    return sum - kinv(c) * ma * c->hfact * c->hfact * c->hfact;
}

static void eos(const orc_cfg* c, const orc_state* s, long long a, double rho, double* P,
                double* cs)
{
    if (c->eos == 0) {
        *P = (c->gamma - 1.0) * rho * s->u[a];
        *cs = sqrt(c->gamma * (*P) / rho);
    } else {
        double R = sqrt(s->x[a] * s->x[a] + s->y[a] * s->y[a]);
        *cs = c->cs0 * pow(R, -c->qcs);
        *P = (*cs) * (*cs) * rho;
    }
}

/* density, h, Omega, nearest-neighbour distance, pressure and sound speed of particle a */
static int density_one(const orc_cfg* c, orc_state* s, const kdtree* g, const long long* xi,
                       long long a, blist* L, double** rbuf, double** mbuf, long long* bufcap)
{
    double ma = mass_of(c, s->level[a]);
    double hi = s->h[a] > 0.0 ? s->h[a] : c->delta * 1024.0;
    /* find an upper bracket: enough mass within 2*hi */
    long long n = 0;
    double *r = NULL, *mb = NULL;
    for (int it = 0;; ++it) {
        gather_within(c, s, g, a, 2.0 * hi, L);
        n = L->n;
        if (n > *bufcap) {
            *bufcap = 2 * n;
            *rbuf = (double*)realloc(*rbuf, sizeof(double) * (size_t)*bufcap);
            *mbuf = (double*)realloc(*mbuf, sizeof(double) * (size_t)*bufcap);
        }
        r = *rbuf;
        mb = *mbuf;
        for (long long t = 0; t < n; ++t) {
            r[t] = sqrt(L->r2[t]);
            mb[t] = mass_of(c, s->level[L->idx[t]]);
        }
        if (g_of_h(c, r, mb, n, ma, hi, NULL) > 0.0) break;
        hi *= 1.5;
        if (it > 200) return -1;
    }
    double lo = hi;
    for (int it = 0; g_of_h(c, r, mb, n, ma, lo, NULL) >= 0.0; ++it) {
        lo /= 1.5;
        if (it > 400) return -1;
    }
    /* the root of g in (lo, hi): Newton steps kept inside the bracket, else bisection */
    double h = 0.5 * (lo + hi);
    for (int it = 0; it < 400; ++it) {
        double dg;
        double gv = g_of_h(c, r, mb, n, ma, h, &dg);
        if (gv > 0.0) hi = h;
        else lo = h;
        double hn = (dg > 0.0) ? h - gv / dg : 0.5 * (lo + hi);
        if (!(hn > lo && hn < hi)) hn = 0.5 * (lo + hi);
        if (!(hn > lo && hn < hi) || hn == h) break;
        if (fabs(hn - h) <= 4.0 * 2.220446049250313e-16 * h) {
            h = hn;
            break;
        }
        h = hn;
    }
    double hr = c->hfact / h;
    double rho = ma * hr * hr * hr;
    double dwdh = 0.0;
    for (long long t = 0; t < n; ++t) {
        double q = r[t] / h, f, df;
        kern(c, q, &f, &df);
        dwdh += mb[t] * (-(3.0 * f + q * df) / (kinv(c) * h * h * h * h));
    }
    s->h[a] = h;
    s->rho[a] = rho;
    s->omega[a] = 1.0 + h / (3.0 * rho) * dwdh;
    /* nearest neighbour on the lattice among b != a with r2 < thr(h) */
    unsigned long long thr = orc_threshold(c, h);
    unsigned long long best = ~0ULL;
    gather_within(c, s, g, a, 2.0 * h + 4.0 * c->delta, L);
    for (long long t = 0; t < L->n; ++t) {
        long long b = L->idx[t];
        if (b == a) continue;
        unsigned long long r2 = r2_lattice(c, &xi[3 * a], &xi[3 * b]);
        if (r2 < thr && r2 < best) best = r2;
    }
    s->dnn[a] = best == ~0ULL ? INFINITY : sqrt((double)best) * c->delta;
    double P, cs;
    eos(c, s, a, rho, &P, &cs);
    s->pres[a] = P;
    s->cs[a] = cs;
    return 0;
}

/*
 * Solve for h, rho, Omega (and d_nn, P, c_s) of every live particle, or of the
 * listed sample only (the others are read, not written).  Returns the number
 * of particles whose bracket could not be found.
 */
long long orc_density(const orc_cfg* c, orc_state* s, const long long* sample, long long nsample)
{
    long long n = s->n;
    long long* xi = (long long*)malloc(sizeof(long long) * 3 * (size_t)(n ? n : 1));
    orc_quantise(c, n, s->x, s->y, s->z, xi);
    kdtree tree, *g = NULL;
    if (c->enumerate == 1 && n > 0) {
        kd_build(s, &tree);
        g = &tree;
    }
    long long m = sample ? nsample : n;
    long long bad = 0;
    set_threads(c);
#pragma omp parallel reduction(+ : bad)
    {
        blist L = {0};
        double *rbuf = NULL, *mbuf = NULL;
        long long bufcap = 0;
#pragma omp for schedule(dynamic, 16)
        for (long long t = 0; t < m; ++t) {
            long long a = sample ? sample[t] : t;
            if (!is_live(s, a)) continue;
            if (density_one(c, s, g, xi, a, &L, &rbuf, &mbuf, &bufcap) != 0) ++bad;
        }
        free(rbuf);
        free(mbuf);
        free(L.idx);
        free(L.r2);
    }
    if (g) kd_free(g);
    free(xi);
    return bad;
}

/* rho_sum(h) and sum_b m_b dW/dh(h) of particle a at a given h (self included) */
void orc_rho_sum(const orc_cfg* c, const orc_state* s, long long a, double h, double* out2)
{
    blist L = {0};
    gather_within(c, s, NULL, a, 2.0 * h, &L);
    double rho = 0.0, dwdh = 0.0;
    for (long long t = 0; t < L.n; ++t) {
        double q = sqrt(L.r2[t]) / h, f, df;
        kern(c, q, &f, &df);
        double mb = mass_of(c, s->level[L.idx[t]]);
        rho += mb * f / (kinv(c) * h * h * h);
        dwdh += mb * (-(3.0 * f + q * df) / (kinv(c) * h * h * h * h));
    }
    out2[0] = rho;
    out2[1] = dwdh;
    free(L.idx);
    free(L.r2);
}

/* ---------------------------------------------------------------- force */

/* sum over the symmetric neighbour set nb[0..nn) (ascending index) of particle a */
static void force_sum(const orc_cfg* c, orc_state* s, long long a, const long long* nb,
                      long long nn)
{
    double axa = 0.0, aya = 0.0, aza = 0.0, du = 0.0, vsig = 0.0;
    double ha = s->h[a], rhoa = s->rho[a], Oa = s->omega[a], Pa = s->pres[a], ca = s->cs[a];
    for (long long t = 0; t < nn; ++t) {
        long long b = nb[t];
        if (b == a) continue;
        double d[3];
        sep64(c, s, a, b, d);
        double r = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
        double hb = s->h[b];
        double qa = r / ha, qb = r / hb;
        if (!(qa < 2.0 || qb < 2.0)) continue;
        double rx = d[0] / r, ry = d[1] / r, rz = d[2] / r;
        double fa, dfa, fb, dfb;
        kern(c, qa, &fa, &dfa);
        kern(c, qb, &fb, &dfb);
        double Fa = dfa / (kinv(c) * ha * ha * ha * ha);
        double Fb = dfb / (kinv(c) * hb * hb * hb * hb);
        double vx = s->vx[a] - s->vx[b], vy = s->vy[a] - s->vy[b], vz = s->vz[a] - s->vz[b];
        double vr = vx * rx + vy * ry + vz * rz;
        double mb = mass_of(c, s->level[b]);
        double rhob = s->rho[b], Ob = s->omega[b], Pb = s->pres[b], cb = s->cs[b];
        /* artificial viscosity: approaching pairs only, signal speed alpha c_s + beta |v.r| */
        double qava = 0.0, qavb = 0.0;
        if (vr < 0.0) {
            double vsa = c->alpha_av * ca + c->beta_av * (-vr);
            double vsb = c->alpha_av * cb + c->beta_av * (-vr);
            qava = -0.5 * rhoa * vsa * vr;
            qavb = -0.5 * rhob * vsb * vr;
        }
        double ta = (Pa + qava) / (Oa * rhoa * rhoa) * Fa;
        double tb = (Pb + qavb) / (Ob * rhob * rhob) * Fb;
        double fac = -mb * (ta + tb);
        axa += fac * rx;
        aya += fac * ry;
        aza += fac * rz;
        if (c->eos == 0) {
            du += mb * (Pa + qava) / (Oa * rhoa * rhoa) * vr * Fa;
            if (c->alpha_u > 0.0) {
                double vsu = sqrt(fabs(Pa - Pb) / (0.5 * (rhoa + rhob)));
                du += mb * c->alpha_u * vsu * (s->u[a] - s->u[b]) * 0.5 *
                      (Fa / (Oa * rhoa) + Fb / (Ob * rhob));
            }
        }
        double vs = ca + c->beta_av * (vr < 0.0 ? -vr : 0.0);
        if (vs > vsig) vsig = vs;
    }
    s->ax[a] = axa;
    s->ay[a] = aya;
    s->az[a] = aza;
    s->dudt[a] = du;
    s->vsig[a] = vsig > ca ? vsig : ca;
}

/*
 * Hydrodynamic acceleration, du/dt and signal speed of every live particle
 * (or of the sample).  Requires h, rho, omega, pres, cs of all neighbours.
 * The symmetric set of a is {b : |r_ab| < 2 h_a} U {b : |r_ab| < 2 h_b}: built
 * as the union of a's own gather list and the lists that contain a.
 */
void orc_force(const orc_cfg* c, orc_state* s, const long long* sample, long long nsample)
{
    long long n = s->n;
    double hmax = max_live_h(s);
    kdtree tree, *g = NULL;
    if (c->enumerate == 1 && n > 0) {
        kd_build(s, &tree);
        g = &tree;
    }
    set_threads(c);
    if (sample) {
#pragma omp parallel
        {
            blist L = {0};
#pragma omp for schedule(dynamic, 16)
            for (long long t = 0; t < nsample; ++t) {
                long long a = sample[t];
                if (!is_live(s, a)) continue;
                gather_symmetric(c, s, g, a, hmax, &L);
                force_sum(c, s, a, L.idx, L.n);
            }
            free(L.idx);
            free(L.r2);
        }
        if (g) kd_free(g);
        return;
    }
    /* gather lists G_a (ascending), then reverse lists R_b = {a : b in G_a} (ascending) */
    long long* gcnt = (long long*)calloc((size_t)n + 1, sizeof(long long));
    long long** glist = (long long**)calloc((size_t)(n ? n : 1), sizeof(long long*));
#pragma omp parallel
    {
        blist L = {0};
#pragma omp for schedule(dynamic, 16)
        for (long long a = 0; a < n; ++a) {
            if (!is_live(s, a)) continue;
            gather_within(c, s, g, a, 2.0 * s->h[a], &L);
            glist[a] = (long long*)malloc(sizeof(long long) * (size_t)(L.n ? L.n : 1));
            memcpy(glist[a], L.idx, sizeof(long long) * (size_t)L.n);
            gcnt[a] = L.n;
        }
        free(L.idx);
        free(L.r2);
    }
    long long* roff = (long long*)calloc((size_t)n + 1, sizeof(long long));
    for (long long a = 0; a < n; ++a)
        for (long long t = 0; t < gcnt[a]; ++t) roff[glist[a][t] + 1]++;
    for (long long b = 0; b < n; ++b) roff[b + 1] += roff[b];
    long long* rlist = (long long*)malloc(sizeof(long long) * (size_t)(roff[n] ? roff[n] : 1));
    long long* fill = (long long*)malloc(sizeof(long long) * (size_t)(n ? n : 1));
    for (long long b = 0; b < n; ++b) fill[b] = roff[b];
    for (long long a = 0; a < n; ++a)
        for (long long t = 0; t < gcnt[a]; ++t) rlist[fill[glist[a][t]]++] = a;
#pragma omp parallel
    {
        long long* u = NULL;
        long long ucap = 0;
#pragma omp for schedule(dynamic, 16)
        for (long long a = 0; a < n; ++a) {
            if (!is_live(s, a)) continue;
            long long na = gcnt[a], nr = roff[a + 1] - roff[a];
            if (na + nr > ucap) {
                ucap = 2 * (na + nr);
                u = (long long*)realloc(u, sizeof(long long) * (size_t)ucap);
            }
            const long long* A = glist[a];
            const long long* B = rlist + roff[a];
            long long i = 0, j = 0, k = 0;
            while (i < na || j < nr) {
                long long v;
                if (j >= nr || (i < na && A[i] < B[j])) v = A[i++];
                else if (i >= na || B[j] < A[i]) v = B[j++];
                else {
                    v = A[i++];
                    ++j;
                }
                u[k++] = v;
            }
            force_sum(c, s, a, u, k);
        }
        free(u);
    }
    for (long long a = 0; a < n; ++a) free(glist[a]);
    free(glist);
    free(gcnt);
    free(roff);
    free(rlist);
    free(fill);
    if (g) kd_free(g);
}

/* point-mass gravity: sinks on gas (added to a), gas and sinks on sinks */
/* gets == NULL: every live gas particle takes the point masses' pull; else only
 * those with gets[i] != 0.  The point masses feel every live gas particle. */
static void sink_gravity_some(const orc_cfg* c, orc_state* s, orc_sink* k, int nk,
                              const unsigned char* gets)
{
    for (int j = 0; j < nk; ++j) k[j].a[0] = k[j].a[1] = k[j].a[2] = 0.0;
    for (long long i = 0; i < s->n; ++i) {
        if (!is_live(s, i)) continue;
        double mi = mass_of(c, s->level[i]);
        const int pulled = gets == NULL || gets[i];
        for (int j = 0; j < nk; ++j) {
            double dx = s->x[i] - k[j].x[0], dy = s->y[i] - k[j].x[1], dz = s->z[i] - k[j].x[2];
            double r2 = dx * dx + dy * dy + dz * dz;
            double r = sqrt(r2);
            double f = c->G / (r2 * r);
            if (pulled) {
                s->ax[i] -= f * k[j].m * dx;
                s->ay[i] -= f * k[j].m * dy;
                s->az[i] -= f * k[j].m * dz;
            }
            k[j].a[0] += f * mi * dx;
            k[j].a[1] += f * mi * dy;
            k[j].a[2] += f * mi * dz;
        }
    }
    for (int j = 0; j < nk; ++j)
        for (int l = 0; l < nk; ++l) {
            if (l == j) continue;
            double dx = k[j].x[0] - k[l].x[0], dy = k[j].x[1] - k[l].x[1],
                   dz = k[j].x[2] - k[l].x[2];
            double r2 = dx * dx + dy * dy + dz * dz;
            double r = sqrt(r2);
            double f = c->G * k[l].m / (r2 * r);
            k[j].a[0] -= f * dx;
            k[j].a[1] -= f * dy;
            k[j].a[2] -= f * dz;
        }
}

void orc_sink_gravity(const orc_cfg* c, orc_state* s, orc_sink* k, int nk)
{
    sink_gravity_some(c, s, k, nk, NULL);
}

/* ----------------------------------------------------- refinement levels */

/* level a region asks for at point p (Sec. 2.1 rule 1; nested boundaries, Table 1) */
static int region_level(const orc_region* r, const double p[3])
{
    int lev = 0;
    for (int k = 0; k < r->nlev; ++k) {
        int inside;
        if (r->shape == 0) {
            double dx = p[0] - r->centre[0], dy = p[1] - r->centre[1], dz = p[2] - r->centre[2];
            double d2 = dx * dx + dy * dy + dz * dz;
            inside = d2 < r->R[k] * r->R[k];
        } else if (r->shape == 2) { /* cylinder: distance from the axis line */
            double d[3] = {p[0] - r->centre[0], p[1] - r->centre[1], p[2] - r->centre[2]};
            int a1 = r->axis == 0 ? 1 : 0, a2 = r->axis == 2 ? 1 : 2;
            double d2 = d[a1] * d[a1] + d[a2] * d[a2];
            inside = d2 < r->R[k] * r->R[k];
        } else {
            double d = p[r->axis] - r->centre[r->axis];
            inside = fabs(d) < r->R[k];
        }
        if (inside) lev = k + 1;
    }
    return lev;
}

/*
 * Target level (Sec. 2.1).  Refinement (level_default 0): the deepest zone's
 * level, default 0, capped at lmax.  Derefinement (level_default L >= 1, the
 * lower-resolution zones of Sec. 2.1 and Sec. 4): L minus the deepest zone's
 * depth, floored at 0.  *which = the deciding zone (the deepest, lowest index
 * on a tie; in derefinement a point outside every zone is decided by zone 0),
 * -1 if there is none.
 */
static int target_level(const orc_cfg* c, const orc_region* rg, int nr, const double p[3],
                        int* which)
{
    int best = 0, w = -1;
    for (int j = 0; j < nr; ++j) {
        int l = region_level(&rg[j], p);
        if (l > best) {
            best = l;
            w = j;
        }
    }
    int t;
    if (c->level_default > 0) {
        t = c->level_default - best;
        if (t < 0) t = 0;
        if (w < 0 && nr > 0) w = 0;
    } else {
        t = best > c->lmax ? c->lmax : best;
    }
    if (which) *which = w;
    return t;
}

void orc_target_levels(const orc_cfg* c, const orc_region* rg, int nr, long long n,
                       const double* x, const double* y, const double* z, unsigned char* out)
{
    for (long long i = 0; i < n; ++i) {
        double p[3] = {x[i], y[i], z[i]};
        out[i] = (unsigned char)target_level(c, rg, nr, p, NULL);
    }
}

void orc_track_regions(orc_region* rg, int nr, const orc_sink* k, int nk)
{
    for (int j = 0; j < nr; ++j) {
        int t = rg[j].track_sink;
        if (t >= 0 && t < nk)
            for (int d = 0; d < 3; ++d) rg[j].centre[d] = k[t].x[d];
    }
}

/* --------------------------------------------------------------- split */

/* SplitMix64 output function (Steele, Lea & Flood 2014) */
static unsigned long long splitmix64(unsigned long long z)
{
    z += 0x9E3779B97F4A7C15ULL;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

unsigned long long orc_splitmix64(unsigned long long z) { return splitmix64(z); }

/* the split's random number in [-1, 1) from (seed, particle id, step) */
double orc_split_uniform(unsigned long long seed, unsigned long long id, unsigned long long step)
{
    unsigned long long z = splitmix64(splitmix64(splitmix64(seed) ^ id) ^ step);
    return (double)(z >> 11) * 2.220446049250313e-16 - 1.0;
}

static double wrap1(const orc_cfg* c, int k, double x)
{
    if (c->periodic[k]) {
        double L = box_len(c, k);
        if (x >= c->hi[k]) x -= L;
        else if (x < c->lo[k]) x += L;
    }
    return x;
}

/*
 * Unit direction w along which the two children are placed: perpendicular to
 * the vector v from the zone centre to the parent (so tangential to a sphere;
 * in the plane of a slab), rotated about v by a random angle (Sec. 2.2).
 * The angle enters through t in [-1,1): cos = (1-t^2)/(1+t^2), sin = 2t/(1+t^2).
 */
void orc_split_direction(const orc_region* r, const double p[3], double t, double w[3])
{
    double v[3];
    if (r->shape == 0) {
        v[0] = p[0] - r->centre[0];
        v[1] = p[1] - r->centre[1];
        v[2] = p[2] - r->centre[2];
        double vn = sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
        if (vn > 0.0) {
            v[0] = v[0] / vn;
            v[1] = v[1] / vn;
            v[2] = v[2] / vn;
        } else {
            v[0] = 1.0;
            v[1] = 0.0;
            v[2] = 0.0;
        }
    } else if (r->shape == 2) { /* cylinder: radial from the axis line */
        v[0] = p[0] - r->centre[0];
        v[1] = p[1] - r->centre[1];
        v[2] = p[2] - r->centre[2];
        v[r->axis] = 0.0;
        double vn = sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
        if (vn > 0.0) {
            v[0] = v[0] / vn;
            v[1] = v[1] / vn;
            v[2] = v[2] / vn;
        } else {
            v[0] = v[1] = v[2] = 0.0;
            v[r->axis == 0 ? 1 : 0] = 1.0;
        }
    } else {
        v[0] = v[1] = v[2] = 0.0;
        v[r->axis] = p[r->axis] - r->centre[r->axis] >= 0.0 ? 1.0 : -1.0;
    }
    /* axis least aligned with v (lowest index on a tie) */
    int k = 0;
    for (int j = 1; j < 3; ++j)
        if (fabs(v[j]) < fabs(v[k])) k = j;
    double e[3] = {0.0, 0.0, 0.0};
    e[k] = 1.0;
    double w1[3] = {v[1] * e[2] - v[2] * e[1], v[2] * e[0] - v[0] * e[2], v[0] * e[1] - v[1] * e[0]};
    double n1 = sqrt(w1[0] * w1[0] + w1[1] * w1[1] + w1[2] * w1[2]);
    w1[0] = w1[0] / n1;
    w1[1] = w1[1] / n1;
    w1[2] = w1[2] / n1;
    double w2[3] = {v[1] * w1[2] - v[2] * w1[1], v[2] * w1[0] - v[0] * w1[2],
                    v[0] * w1[1] - v[1] * w1[0]};
    double den = 1.0 + t * t;
    double cs = (1.0 - t * t) / den;
    double sn = (2.0 * t) / den;
    for (int j = 0; j < 3; ++j) w[j] = cs * w1[j] + sn * w2[j];
}

static void copy_particle(orc_state* s, long long dst, long long src)
{
#define CP(f) s->f[dst] = s->f[src]
    CP(x); CP(y); CP(z); CP(vx); CP(vy); CP(vz); CP(u); CP(h);
    CP(rho); CP(omega); CP(ax); CP(ay); CP(az); CP(dudt); CP(vsig); CP(dnn); CP(pres); CP(cs);
    CP(level); CP(flags); CP(id);
    if (s->bin) CP(bin);
#undef CP
}

/*
 * One split pass over level l (Sec. 2.2, Sec. 2.6): every live, unchanged,
 * non-fixed particle at level l whose target level exceeds l is split.  In
 * ascending index order the k-th split parent keeps its slot (child at +r_sep w)
 * and the new child goes to slot n + k (at -r_sep w) with id next_id + k.
 * Returns the number of splits, or -1 (state untouched) if capacity is short.
 */
long long orc_split_pass(const orc_cfg* c, orc_state* s, const orc_region* rg, int nr, int l,
                         unsigned long long step)
{
    long long n = s->n, ns = 0;
    for (long long i = 0; i < n; ++i) {
        if (s->level[i] != l || (s->flags[i] & (ORC_FLAG_CHANGED | ORC_FLAG_FIXED | ORC_FLAG_DEAD | ORC_FLAG_INACTIVE)))
            continue;
        double p[3] = {s->x[i], s->y[i], s->z[i]};
        if (target_level(c, rg, nr, p, NULL) > l) ++ns;
    }
    if (n + ns > s->cap) return -1;
    long long k = 0;
    for (long long i = 0; i < n; ++i) {
        if (s->level[i] != l || (s->flags[i] & (ORC_FLAG_CHANGED | ORC_FLAG_FIXED | ORC_FLAG_DEAD | ORC_FLAG_INACTIVE)))
            continue;
        double p[3] = {s->x[i], s->y[i], s->z[i]};
        int which;
        if (target_level(c, rg, nr, p, &which) <= l) continue;
        double t = orc_split_uniform(c->seed, s->id[i], step);
        double w[3];
        if (which >= 0) {
            orc_split_direction(&rg[which], p, t, w);
        } else {
            /* no zone decides (derefinement without zones): a sphere centred on
               the parent, whose direction falls back to the x axis */
            orc_region self;
            memset(&self, 0, sizeof(self));
            self.shape = 0;
            self.centre[0] = p[0];
            self.centre[1] = p[1];
            self.centre[2] = p[2];
            orc_split_direction(&self, p, t, w);
        }
        double rsep = c->rsep_fac * s->h[i];
        double cap = c->dnn_cap * s->dnn[i];
        if (cap < rsep) rsep = cap;
        long long j = n + k;
        copy_particle(s, j, i);
        s->x[i] = wrap1(c, 0, p[0] + rsep * w[0]);
        s->y[i] = wrap1(c, 1, p[1] + rsep * w[1]);
        s->z[i] = wrap1(c, 2, p[2] + rsep * w[2]);
        s->x[j] = wrap1(c, 0, p[0] - rsep * w[0]);
        s->y[j] = wrap1(c, 1, p[1] - rsep * w[1]);
        s->z[j] = wrap1(c, 2, p[2] - rsep * w[2]);
        double hn = s->h[i] * ORC_SPLIT_HFAC;
        s->h[i] = s->h[j] = hn;
        s->level[i] = s->level[j] = (unsigned char)(l + 1);
        s->flags[i] |= ORC_FLAG_CHANGED | ORC_FLAG_NEW;
        s->flags[j] |= ORC_FLAG_CHANGED | ORC_FLAG_NEW;
        s->id[j] = (unsigned long long)(s->next_id + k);
        ++k;
    }
    s->n = n + ns;
    s->next_id += ns;
    return ns;
}

/* --------------------------------------------------------------- merge */

static int cmp_u64(const void* a, const void* b)
{
    unsigned long long x = *(const unsigned long long*)a, y = *(const unsigned long long*)b;
    return (x > y) - (x < y);
}

/*
 * Pairing tree (Sec. 2.3).  set[0..m) holds particle indices (m even); xi are
 * their lattice coordinates indexed by particle.  A node with more than two
 * particles is cut through its centre of mass (all masses equal within a
 * level, so the mean lattice coordinate, floored) along the axis of largest
 * extent; the cut count is kept even by moving the cut across one particle
 * towards the more balanced side.  On return set is reordered so that
 * (set[2j], set[2j+1]) are the leaves.  Returns 0, or -1 on bad input.
 */
int orc_pair_tree(const long long* xi, long long* set, long long m)
{
    if (m % 2) return -1;
    if (m == 0) return 0;
    unsigned long long* key = (unsigned long long*)malloc(sizeof(unsigned long long) * (size_t)m);
    long long* stk = (long long*)malloc(sizeof(long long) * 2 * (size_t)(m + 2));
    long long sp = 0;
    stk[sp++] = 0;
    stk[sp++] = m;
    while (sp > 0) {
        long long n = stk[--sp];
        long long off = stk[--sp];
        if (n <= 2) continue;
        long long* S = set + off;
        long long lo[3], hi[3];
        for (int k = 0; k < 3; ++k) lo[k] = hi[k] = xi[3 * S[0] + k];
        for (long long t = 1; t < n; ++t)
            for (int k = 0; k < 3; ++k) {
                long long v = xi[3 * S[t] + k];
                if (v < lo[k]) lo[k] = v;
                if (v > hi[k]) hi[k] = v;
            }
        int ax = 0;
        for (int k = 1; k < 3; ++k)
            if (hi[k] - lo[k] > hi[ax] - lo[ax]) ax = k;
        unsigned long long sum = 0;
        for (long long t = 0; t < n; ++t) sum += (unsigned long long)xi[3 * S[t] + ax];
        long long com = (long long)(sum / (unsigned long long)n);
        for (long long t = 0; t < n; ++t)
            key[t] = ((unsigned long long)xi[3 * S[t] + ax] << 32) | (unsigned long long)S[t];
        qsort(key, (size_t)n, sizeof(unsigned long long), cmp_u64);
        for (long long t = 0; t < n; ++t) S[t] = (long long)(key[t] & 0xffffffffULL);
        long long k = 0;
        while (k < n && xi[3 * S[k] + ax] < com) ++k;
        if (k == 0)
            while (k < n && xi[3 * S[k] + ax] <= com) ++k;
        if (k == n) {
            k = 2 * (n / 4);
        } else if (k % 2) {
            long long a = k - 1, b = k + 1;
            long long da = 2 * a - n, db = 2 * b - n;
            if (da < 0) da = -da;
            if (db < 0) db = -db;
            k = (da <= db) ? a : b;
        }
        stk[sp++] = off;
        stk[sp++] = k;
        stk[sp++] = off + k;
        stk[sp++] = n - k;
    }
    free(key);
    free(stk);
    return 0;
}

/*
 * One merge pass over level l >= 1 (Sec. 2.3).  Candidates: live, unchanged,
 * non-fixed particles at level l in ascending index order; with an odd count
 * the last one is left out (*spare = its index, else -1).  For each leaf pair
 * whose centre of mass lies at a target level below l, the lower index
 * survives at the centre of mass with the mean velocity and thermal energy,
 * h * 2^(1/3), level l-1; the other is marked dead.  Returns merges done.
 */
long long orc_merge_pass(const orc_cfg* c, orc_state* s, const orc_region* rg, int nr, int l,
                         long long* spare)
{
    long long n = s->n, m = 0;
    *spare = -1;
    long long* set = (long long*)malloc(sizeof(long long) * (size_t)(n ? n : 1));
    for (long long i = 0; i < n; ++i)
        if (s->level[i] == l &&
            !(s->flags[i] & (ORC_FLAG_CHANGED | ORC_FLAG_FIXED | ORC_FLAG_DEAD | ORC_FLAG_INACTIVE)))
            set[m++] = i;
    if (m % 2) {
        *spare = set[m - 1];
        --m;
    }
    long long nm = 0;
    if (m >= 2) {
        long long* xi = (long long*)malloc(sizeof(long long) * 3 * (size_t)n);
        orc_quantise(c, n, s->x, s->y, s->z, xi);
        orc_pair_tree(xi, set, m);
        for (long long j = 0; j < m; j += 2) {
            long long a = set[j], b = set[j + 1];
            if (b < a) {
                long long t = a;
                a = b;
                b = t;
            }
            double pa[3] = {s->x[a], s->y[a], s->z[a]}, pb[3] = {s->x[b], s->y[b], s->z[b]};
            double com[3];
            for (int k = 0; k < 3; ++k) {
                double d = pb[k] - pa[k];
                if (c->periodic[k]) {
                    double L = box_len(c, k);
                    if (d > 0.5 * L) d -= L;
                    else if (d < -0.5 * L) d += L;
                }
                com[k] = wrap1(c, k, pa[k] + 0.5 * d);
            }
            if (target_level(c, rg, nr, com, NULL) >= l) continue;
            s->x[a] = com[0];
            s->y[a] = com[1];
            s->z[a] = com[2];
            s->vx[a] = 0.5 * (s->vx[a] + s->vx[b]);
            s->vy[a] = 0.5 * (s->vy[a] + s->vy[b]);
            s->vz[a] = 0.5 * (s->vz[a] + s->vz[b]);
            s->u[a] = 0.5 * (s->u[a] + s->u[b]);
            s->h[a] = s->h[a] * ORC_MERGE_HFAC;
            s->level[a] = (unsigned char)(l - 1);
            s->flags[a] |= ORC_FLAG_CHANGED | ORC_FLAG_NEW;
            s->flags[b] |= ORC_FLAG_DEAD;
            ++nm;
        }
        free(xi);
    }
    free(set);
    return nm;
}

/* stable removal of dead particles; returns the number removed */
long long orc_compact(orc_state* s)
{
    long long k = 0, n = s->n;
    for (long long i = 0; i < n; ++i) {
        if (s->flags[i] & ORC_FLAG_DEAD) continue;
        if (k != i) copy_particle(s, k, i);
        ++k;
    }
    s->n = k;
    return n - k;
}

/*
 * Full split/merge pass of one step (Sec. 2.6): clear the changed marks, split
 * level by level from 0 up, merge level by level from lmax down, then compact.
 * Returns 0, or -1 if capacity ran out (splits done so far are kept).
 */
int orc_split_merge(const orc_cfg* c, orc_state* s, const orc_region* rg, int nr,
                    unsigned long long step, orc_counts* cnt)
{
    memset(cnt, 0, sizeof(*cnt));
    for (long long i = 0; i < s->n; ++i) s->flags[i] &= (unsigned char)~ORC_FLAG_CHANGED;
    for (int l = 0; l < c->lmax; ++l) {
        long long ns = orc_split_pass(c, s, rg, nr, l, step);
        if (ns < 0) return -1;
        cnt->n_split[l] = ns;
    }
    for (int l = c->lmax; l >= 1; --l) {
        long long spare;
        cnt->n_merge[l] = orc_merge_pass(c, s, rg, nr, l, &spare);
        cnt->n_spare[l] = spare >= 0 ? 1 : 0;
    }
    cnt->n_dead = orc_compact(s);
    return 0;
}

/* ------------------------------------------------------ sinks / stepping */

/* accretion: a live gas particle inside a sink's radius is absorbed (first sink wins) */
long long orc_accrete(const orc_cfg* c, orc_state* s, orc_sink* k, int nk)
{
    long long na = 0;
    for (int j = 0; j < nk; ++j) {
        double M = 0.0, P[3] = {0, 0, 0}, X[3] = {0, 0, 0};
        for (long long i = 0; i < s->n; ++i) {
            if (s->flags[i] & (ORC_FLAG_DEAD | ORC_FLAG_FIXED)) continue;
            double dx = s->x[i] - k[j].x[0], dy = s->y[i] - k[j].x[1], dz = s->z[i] - k[j].x[2];
            double r2 = dx * dx + dy * dy + dz * dz;
            if (!(r2 < k[j].racc * k[j].racc)) continue;
            double mi = mass_of(c, s->level[i]);
            M += mi;
            P[0] += mi * s->vx[i];
            P[1] += mi * s->vy[i];
            P[2] += mi * s->vz[i];
            X[0] += mi * s->x[i];
            X[1] += mi * s->y[i];
            X[2] += mi * s->z[i];
            s->flags[i] |= ORC_FLAG_DEAD;
            ++na;
        }
        if (M > 0.0) {
            double mt = k[j].m + M;
            for (int d = 0; d < 3; ++d) {
                k[j].v[d] = (k[j].m * k[j].v[d] + P[d]) / mt;
                k[j].x[d] = (k[j].m * k[j].x[d] + X[d]) / mt;
            }
            k[j].m = mt;
        }
    }
    return na;
}

void orc_stats_compute(const orc_cfg* c, const orc_state* s, const orc_sink* k, int nk,
                       orc_stats* st)
{
    memset(st, 0, sizeof(*st));
    for (long long i = 0; i < s->n; ++i) {
        if (!is_live(s, i)) continue;
        double m = mass_of(c, s->level[i]);
        st->mass += m;
        st->mom[0] += m * s->vx[i];
        st->mom[1] += m * s->vy[i];
        st->mom[2] += m * s->vz[i];
        st->ang[0] += m * (s->y[i] * s->vz[i] - s->z[i] * s->vy[i]);
        st->ang[1] += m * (s->z[i] * s->vx[i] - s->x[i] * s->vz[i]);
        st->ang[2] += m * (s->x[i] * s->vy[i] - s->y[i] * s->vx[i]);
        st->ekin += 0.5 * m * (s->vx[i] * s->vx[i] + s->vy[i] * s->vy[i] + s->vz[i] * s->vz[i]);
        if (c->eos == 0) st->etherm += m * s->u[i];
    }
    for (int j = 0; j < nk; ++j) {
        double m = k[j].m;
        st->mass += m;
        for (int d = 0; d < 3; ++d) st->mom[d] += m * k[j].v[d];
        st->ang[0] += m * (k[j].x[1] * k[j].v[2] - k[j].x[2] * k[j].v[1]);
        st->ang[1] += m * (k[j].x[2] * k[j].v[0] - k[j].x[0] * k[j].v[2]);
        st->ang[2] += m * (k[j].x[0] * k[j].v[1] - k[j].x[1] * k[j].v[0]);
        st->ekin += 0.5 * m * (k[j].v[0] * k[j].v[0] + k[j].v[1] * k[j].v[1] + k[j].v[2] * k[j].v[2]);
    }
}

/* next time step: min over moving particles of C_cour h / v_sig and C_force sqrt(h/|a|) */
double orc_timestep(const orc_cfg* c, const orc_state* s)
{
    double dt = INFINITY;
    for (long long i = 0; i < s->n; ++i) {
        if (s->flags[i] & (ORC_FLAG_DEAD | ORC_FLAG_FIXED)) continue;
        if (s->vsig[i] > 0.0) {
            double t = c->ccour * s->h[i] / s->vsig[i];
            if (t < dt) dt = t;
        }
        double a = sqrt(s->ax[i] * s->ax[i] + s->ay[i] * s->ay[i] + s->az[i] * s->az[i]);
        if (a > 0.0) {
            double t = c->cforce * sqrt(s->h[i] / a);
            if (t < dt) dt = t;
        }
    }
    return dt;
}

/* density, then hydro forces, then point-mass gravity */
long long orc_density_force(const orc_cfg* c, orc_state* s, orc_sink* k, int nk)
{
    long long bad = orc_density(c, s, NULL, 0);
    orc_force(c, s, NULL, 0);
    if (nk > 0) orc_sink_gravity(c, s, k, nk);
    return bad;
}

/*
 * Initial refinement: repeat (density; one split/merge pass) until no particle
 * changes level, so that particles reach the full depth of nested zones; then
 * density and forces.  Returns passes used, or -1 on capacity shortage.
 */
int orc_init(const orc_cfg* c, orc_state* s, orc_region* rg, int nr, orc_sink* k, int nk,
             unsigned long long* step)
{
    orc_track_regions(rg, nr, k, nk);
    int passes = 0;
    for (;;) {
        orc_density(c, s, NULL, 0);
        orc_counts cnt;
        if (orc_split_merge(c, s, rg, nr, *step, &cnt) != 0) return -1;
        (*step)++;
        ++passes;
        long long changed = 0;
        for (int l = 0; l < ORC_MAXLEV; ++l) changed += cnt.n_split[l] + cnt.n_merge[l];
        if (changed == 0 || passes > 4 * ORC_MAXLEV) break;
    }
    for (long long i = 0; i < s->n; ++i) s->flags[i] &= (unsigned char)~ORC_FLAG_CHANGED;
    orc_density_force(c, s, k, nk);
    return passes;
}

/*
 * One kick-drift-kick step: half kick (gas and sinks), drift, accretion,
 * regions follow their sinks, split/merge + compaction, density, forces,
 * half kick.  Fixed particles are not moved.
 */
int orc_step(const orc_cfg* c, orc_state* s, orc_region* rg, int nr, orc_sink* k, int nk,
             double dt, unsigned long long step, orc_counts* cnt, orc_stats* st)
{
    double hdt = 0.5 * dt;
    for (long long i = 0; i < s->n; ++i) {
        if (s->flags[i] & (ORC_FLAG_FIXED | ORC_FLAG_DEAD)) continue;
        s->vx[i] += hdt * s->ax[i];
        s->vy[i] += hdt * s->ay[i];
        s->vz[i] += hdt * s->az[i];
        if (c->eos == 0) s->u[i] += hdt * s->dudt[i];
    }
    for (int j = 0; j < nk; ++j)
        for (int d = 0; d < 3; ++d) k[j].v[d] += hdt * k[j].a[d];
    for (long long i = 0; i < s->n; ++i) {
        if (s->flags[i] & (ORC_FLAG_FIXED | ORC_FLAG_DEAD)) continue;
        s->x[i] = wrap1(c, 0, s->x[i] + dt * s->vx[i]);
        s->y[i] = wrap1(c, 1, s->y[i] + dt * s->vy[i]);
        s->z[i] = wrap1(c, 2, s->z[i] + dt * s->vz[i]);
    }
    for (int j = 0; j < nk; ++j)
        for (int d = 0; d < 3; ++d) k[j].x[d] += dt * k[j].v[d];
    long long na = nk > 0 ? orc_accrete(c, s, k, nk) : 0;
    orc_track_regions(rg, nr, k, nk);
    if (orc_split_merge(c, s, rg, nr, step, cnt) != 0) return -1;
    cnt->n_accreted = na;
    orc_density_force(c, s, k, nk);
    for (long long i = 0; i < s->n; ++i) {
        if (s->flags[i] & (ORC_FLAG_FIXED | ORC_FLAG_DEAD)) continue;
        s->vx[i] += hdt * s->ax[i];
        s->vy[i] += hdt * s->ay[i];
        s->vz[i] += hdt * s->az[i];
        if (c->eos == 0) s->u[i] += hdt * s->dudt[i];
    }
    for (int j = 0; j < nk; ++j)
        for (int d = 0; d < 3; ++d) k[j].v[d] += hdt * k[j].a[d];
    orc_stats_compute(c, s, k, nk, st);
    return 0;
}

/* ------------------------------------------- density error of a split, adjoint */

/*
 * The density error that one split pass creates, and its gradient with respect
 * to the children's offsets and smoothing lengths.  The paper has no such
 * function: Sec. 2.2 picks r_sep and Sec. 2.5 relaxes children so that the new
 * distribution reproduces the density of the original one; this is a
 * differentiable statement of that error.
 *
 * Reference set: the live particles of s, at their own h.  Split k replaces
 * parent[k] by two children at x_p + d_k (child 2k) and x_p - d_k (child 2k+1),
 * one level finer (Eq. 1 mass), with smoothing lengths hc[2k], hc[2k+1].  The
 * new set is the reference set without the parents, plus the children.
 *
 *   rho_new(a)  = sum_{b in new set} m_b W(|x_a - x_b|, h_a)    (self included)
 *   rho_ref(x)  = sum_{b in reference set} m_b W(|x - x_b|, h_b)
 *   J           = sum_{children a} (rho_new(a) - rho_ref(x_a))^2
 *
 * With W' = dW/dr = f'(q) / (pi h^4), u_ab = (x_a - x_b)/|x_a - x_b| and
 * e_a = rho_new(a) - rho_ref(x_a):
 *   dJ/dx_a = 2 e_a [ sum_{b new, b != a} m_b W'(r_ab, h_a) u_ab
 *                     - sum_{b ref} m_b W'(r_ab, h_b) u_ab ]
 *             + sum_{children c != a} 2 e_c m_a W'(r_ac, h_c) u_ac
 *   dJ/dh_a = 2 e_a sum_{b new} m_b dW/dh(r_ab, h_a),
 *             dW/dh = -(3 f(q) + q f'(q)) / (pi h^4)
 *   dJ/dd_k = dJ/dx_(child 2k) - dJ/dx_(child 2k+1)
 *
 * Gradients are computed for the splits with want[k] != 0 (all if want is
 * NULL; the rest are set to 0); J always covers every child.  Returns 0, or -1
 * if a parent index is out of range, dead or repeated.
 */
#define ORC_ROLE_NEW 1u
#define ORC_ROLE_REF 2u
#define ORC_ROLE_CHILD 4u

static void free_state_arrays(orc_state* t)
{
    free(t->x);
    free(t->y);
    free(t->z);
    free(t->h);
    free(t->level);
    free(t->flags);
}

int orc_split_loss_grad(const orc_cfg* c, const orc_state* s, long long npar,
                        const long long* parent, const double* d, const double* hc,
                        const unsigned char* want, double* J, double* grad_d, double* grad_hc)
{
    const long long n = s->n, nt = n + 2 * npar;
    orc_state T;
    memset(&T, 0, sizeof(T));
    T.n = nt;
    T.cap = nt;
    size_t sz = (size_t)(nt > 0 ? nt : 1);
    T.x = (double*)malloc(sizeof(double) * sz);
    T.y = (double*)malloc(sizeof(double) * sz);
    T.z = (double*)malloc(sizeof(double) * sz);
    T.h = (double*)malloc(sizeof(double) * sz);
    T.level = (unsigned char*)malloc(sz);
    T.flags = (unsigned char*)malloc(sz);
    unsigned char* role = (unsigned char*)malloc(sz);
    for (long long i = 0; i < n; ++i) {
        T.x[i] = s->x[i];
        T.y[i] = s->y[i];
        T.z[i] = s->z[i];
        T.h[i] = s->h[i];
        T.level[i] = s->level[i];
        T.flags[i] = is_live(s, i) ? 0 : ORC_FLAG_DEAD;
        role[i] = is_live(s, i) ? (ORC_ROLE_NEW | ORC_ROLE_REF) : 0;
    }
    for (long long k = 0; k < npar; ++k) {
        long long p = parent[k];
        if (p < 0 || p >= n || role[p] != (ORC_ROLE_NEW | ORC_ROLE_REF)) {
            free_state_arrays(&T);
            free(role);
            return -1;
        }
        role[p] = ORC_ROLE_REF; /* the parent leaves the new set */
        double xp[3] = {s->x[p], s->y[p], s->z[p]};
        for (int side = 0; side < 2; ++side) {
            long long j = n + 2 * k + side;
            double sg = side == 0 ? 1.0 : -1.0, q[3];
            for (int m = 0; m < 3; ++m) q[m] = wrap1(c, m, xp[m] + sg * d[3 * k + m]);
            T.x[j] = q[0];
            T.y[j] = q[1];
            T.z[j] = q[2];
            T.h[j] = hc[2 * k + side];
            T.level[j] = (unsigned char)(s->level[p] + 1);
            T.flags[j] = 0;
            role[j] = ORC_ROLE_NEW | ORC_ROLE_CHILD;
        }
    }
    double hmax = 0.0;
    for (long long i = 0; i < nt; ++i)
        if (role[i] && T.h[i] > hmax) hmax = T.h[i];
    kdtree tree, *g = NULL;
    if (c->enumerate && nt > 0) {
        kd_build(&T, &tree);
        g = &tree;
    }
    double* e = (double*)calloc(sz, sizeof(double));
    set_threads(c);
    /* forward: the density error of every child */
#pragma omp parallel
    {
        blist L = {0};
#pragma omp for schedule(dynamic, 64)
        for (long long a = n; a < nt; ++a) {
            gather_within(c, &T, g, a, 2.0 * hmax, &L);
            const double ha = T.h[a];
            double rho_new = 0.0, rho_ref = 0.0;
            for (long long t = 0; t < L.n; ++t) {
                long long b = L.idx[t];
                double r = sqrt(L.r2[t]), mb = mass_of(c, T.level[b]), f, df;
                if (role[b] & ORC_ROLE_NEW) {
                    kern(c, r / ha, &f, &df);
                    rho_new += mb * f / (kinv(c) * ha * ha * ha);
                }
                if (role[b] & ORC_ROLE_REF) {
                    double hb = T.h[b];
                    kern(c, r / hb, &f, &df);
                    rho_ref += mb * f / (kinv(c) * hb * hb * hb);
                }
            }
            e[a] = rho_new - rho_ref;
        }
        free(L.idx);
        free(L.r2);
    }
    double sum = 0.0;
    for (long long a = n; a < nt; ++a) sum += e[a] * e[a];
    *J = sum;
    /* reverse: gradients of the wanted splits */
#pragma omp parallel
    {
        blist L = {0};
#pragma omp for schedule(dynamic, 16)
        for (long long k = 0; k < npar; ++k) {
            if (want && !want[k]) {
                for (int m = 0; m < 3; ++m) grad_d[3 * k + m] = 0.0;
                grad_hc[2 * k] = grad_hc[2 * k + 1] = 0.0;
                continue;
            }
            double gx[2][3];
            for (int side = 0; side < 2; ++side) {
                long long a = n + 2 * k + side;
                gather_within(c, &T, g, a, 2.0 * hmax, &L);
                const double ha = T.h[a], ma = mass_of(c, T.level[a]);
                double own[3] = {0.0, 0.0, 0.0}, rev[3] = {0.0, 0.0, 0.0}, dh = 0.0;
                for (long long t = 0; t < L.n; ++t) {
                    long long b = L.idx[t];
                    double r = sqrt(L.r2[t]), mb = mass_of(c, T.level[b]), f, df;
                    double sep[3] = {0.0, 0.0, 0.0};
                    if (b != a && r > 0.0) { /* coincident pairs: f'(0) = 0, no direction */
                        sep64(c, &T, a, b, sep);
                        for (int m = 0; m < 3; ++m) sep[m] /= r; /* u_ab */
                    }
                    if (role[b] & ORC_ROLE_NEW) {
                        double q = r / ha;
                        kern(c, q, &f, &df);
                        dh += mb * (-(3.0 * f + q * df) / (kinv(c) * ha * ha * ha * ha));
                        if (b != a)
                            for (int m = 0; m < 3; ++m)
                                own[m] += mb * (df / (kinv(c) * ha * ha * ha * ha)) * sep[m];
                    }
                    if (role[b] & ORC_ROLE_REF) {
                        double hb = T.h[b];
                        kern(c, r / hb, &f, &df);
                        for (int m = 0; m < 3; ++m)
                            own[m] -= mb * (df / (kinv(c) * hb * hb * hb * hb)) * sep[m];
                    }
                    if ((role[b] & ORC_ROLE_CHILD) && b != a) {
                        double hb = T.h[b];
                        kern(c, r / hb, &f, &df);
                        for (int m = 0; m < 3; ++m)
                            rev[m] += 2.0 * e[b] * ma * (df / (kinv(c) * hb * hb * hb * hb)) * sep[m];
                    }
                }
                for (int m = 0; m < 3; ++m) gx[side][m] = 2.0 * e[a] * own[m] + rev[m];
                grad_hc[2 * k + side] = 2.0 * e[a] * dh;
            }
            for (int m = 0; m < 3; ++m) grad_d[3 * k + m] = gx[0][m] - gx[1][m];
        }
        free(L.idx);
        free(L.r2);
    }
    if (g) kd_free(g);
    free(e);
    free(role);
    free_state_arrays(&T);
    return 0;
}

/* ------------------------------------------------------------- relaxing */

/* live particles b of s with |p - x_b| < 2 h_b (each at its own h), sorted by index */
static void gather_point_scatter(const orc_cfg* c, const orc_state* s, const cellgrid* g,
                                 const double p[3], double hmax, blist* out)
{
    out->n = 0;
    const double R = 2.0 * hmax;
    long long lo[3], hi[3], cnt[3];
    for (int k = 0; k < 3; ++k) {
        if (!g) break;
        long long ck = cell_coord(c, g, k, p[k]);
        long long m = (long long)ceil(R / g->cw[k]);
        if (c->periodic[k] && 2 * m + 1 >= g->nc[k]) {
            lo[k] = 0;
            hi[k] = g->nc[k] - 1;
        } else if (c->periodic[k]) {
            lo[k] = ck - m;
            hi[k] = ck + m;
        } else {
            lo[k] = ck - m < 0 ? 0 : ck - m;
            hi[k] = ck + m >= g->nc[k] ? g->nc[k] - 1 : ck + m;
        }
        cnt[k] = g->nc[k];
    }
    long long nb = 0;
    long long* cand = NULL;
    if (!g) {
        cand = (long long*)malloc(sizeof(long long) * (size_t)(s->n ? s->n : 1));
        for (long long b = 0; b < s->n; ++b) cand[nb++] = b;
    } else {
        long long capc = 64;
        cand = (long long*)malloc(sizeof(long long) * (size_t)capc);
        for (long long i = lo[0]; i <= hi[0]; ++i)
            for (long long j = lo[1]; j <= hi[1]; ++j)
                for (long long k = lo[2]; k <= hi[2]; ++k) {
                    long long ii = (i % cnt[0] + cnt[0]) % cnt[0];
                    long long jj = (j % cnt[1] + cnt[1]) % cnt[1];
                    long long kk = (k % cnt[2] + cnt[2]) % cnt[2];
                    long long cell = (ii * cnt[1] + jj) * cnt[2] + kk;
                    for (long long t = g->head[cell]; t < g->head[cell + 1]; ++t) {
                        if (nb == capc) {
                            capc *= 2;
                            cand = (long long*)realloc(cand, sizeof(long long) * (size_t)capc);
                        }
                        cand[nb++] = g->items[t];
                    }
                }
        qsort(cand, (size_t)nb, sizeof(long long), cmp_ll);
    }
    for (long long t = 0; t < nb; ++t) {
        long long b = cand[t];
        if (!is_live(s, b)) continue;
        double d[3] = {p[0] - s->x[b], p[1] - s->y[b], p[2] - s->z[b]};
        for (int k = 0; k < 3; ++k)
            if (c->periodic[k]) {
                double L = box_len(c, k);
                if (d[k] > 0.5 * L) d[k] -= L;
                else if (d[k] < -0.5 * L) d[k] += L;
            }
        double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
        if (r2 < 4.0 * s->h[b] * s->h[b]) bl_push(out, b, r2);
    }
    free(cand);
}

/* sum over the reference set of (m_b / rho_b) a_b W(|p - x_b|, h_b) at point p */
static void interp_ref(const orc_cfg* c, const orc_state* ref, const cellgrid* g, double hmax,
                       const double p[3], blist* L, double out[3])
{
    gather_point_scatter(c, ref, g, p, hmax, L);
    out[0] = out[1] = out[2] = 0.0;
    for (long long t = 0; t < L->n; ++t) {
        long long b = L->idx[t];
        double hb = ref->h[b], f, df;
        kern(c, sqrt(L->r2[t]) / hb, &f, &df);
        double wgt = mass_of(c, ref->level[b]) / ref->rho[b] * f / (kinv(c) * hb * hb * hb);
        out[0] += wgt * ref->ax[b];
        out[1] += wgt * ref->ay[b];
        out[2] += wgt * ref->az[b];
    }
}

/* the reference accelerations interpolated to npts points (xyz interleaved) */
void orc_interp_ref(const orc_cfg* c, const orc_state* ref, long long npts, const double* pts,
                    double* out)
{
    double hmax = 0.0;
    for (long long b = 0; b < ref->n; ++b)
        if (is_live(ref, b) && ref->h[b] > hmax) hmax = ref->h[b];
    blist L = {0};
    for (long long i = 0; i < npts; ++i) interp_ref(c, ref, NULL, hmax, &pts[3 * i], &L, &out[3 * i]);
    free(L.idx);
    free(L.r2);
}

/*
 * Relaxing (Sec. 2.4).  The particles of s flagged NEW (introduced by splits
 * and merges) are shuffled towards the reference set ref (the particles before
 * the split/merge, with their density and accelerations):
 *   a_new: the accelerations of s at the current positions (density, forces,
 *          point masses);
 *   a_ref: the reference accelerations interpolated to the same position,
 *          sum over ref of (m_b / rho_b) a_b W(|x - x_b|, h_b);
 *   dx = 0.5 dt^2 (a_new - a_ref), dt = 0.3 h / c_s of the moved particle, |dx|
 *   capped at h; the shuffle's "kinetic energy" is sum |dx| / dt^2.
 * Shuffles repeat until that energy is at most tol times the first shuffle's, or
 * max_iter shuffles are done; then density and forces are recomputed and the NEW
 * flags cleared.  Returns the shuffles done; *ke_ratio = last energy / first.
 */
int orc_relax(const orc_cfg* c, orc_state* s, const orc_state* ref, orc_sink* k, int nk,
              int max_iter, double tol, double* ke_ratio)
{
    double hmax = 0.0;
    for (long long b = 0; b < ref->n; ++b)
        if (is_live(ref, b) && ref->h[b] > hmax) hmax = ref->h[b];
    cellgrid grid, *g = NULL;
    if (c->enumerate && ref->n > 0) {
        grid_build(c, ref, 2.0 * hmax, &grid);
        g = &grid;
    }
    double ke0 = 0.0, ke = 0.0;
    int it = 0;
    *ke_ratio = 0.0;
    const long long n = s->n;
    double* dx = (double*)calloc((size_t)(3 * (n ? n : 1)), sizeof(double));
    double* kt = (double*)calloc((size_t)(n ? n : 1), sizeof(double));
    for (it = 0; it < max_iter; ++it) {
        orc_density_force(c, s, k, nk);
        set_threads(c);
#pragma omp parallel
        {
            blist L = {0};
#pragma omp for schedule(dynamic, 64)
            for (long long a = 0; a < n; ++a) {
                kt[a] = 0.0;
                dx[3 * a] = dx[3 * a + 1] = dx[3 * a + 2] = 0.0;
                if (!is_live(s, a) || !(s->flags[a] & ORC_FLAG_NEW)) continue;
                double p[3] = {s->x[a], s->y[a], s->z[a]};
                double aref[3];
                interp_ref(c, ref, g, hmax, p, &L, aref);
                double dt = 0.3 * s->h[a] / s->cs[a];
                double d[3] = {0.5 * dt * dt * (s->ax[a] - aref[0]), 0.5 * dt * dt * (s->ay[a] - aref[1]),
                               0.5 * dt * dt * (s->az[a] - aref[2])};
                double len = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
                if (len > s->h[a]) {
                    double sc = s->h[a] / len;
                    d[0] *= sc;
                    d[1] *= sc;
                    d[2] *= sc;
                    len = s->h[a];
                }
                dx[3 * a] = d[0];
                dx[3 * a + 1] = d[1];
                dx[3 * a + 2] = d[2];
                kt[a] = len / (dt * dt);
            }
            free(L.idx);
            free(L.r2);
        }
        ke = 0.0;
        for (long long a = 0; a < n; ++a) {
            ke += kt[a];
            if (kt[a] > 0.0 || dx[3 * a] != 0.0 || dx[3 * a + 1] != 0.0 || dx[3 * a + 2] != 0.0) {
                s->x[a] = wrap1(c, 0, s->x[a] + dx[3 * a]);
                s->y[a] = wrap1(c, 1, s->y[a] + dx[3 * a + 1]);
                s->z[a] = wrap1(c, 2, s->z[a] + dx[3 * a + 2]);
            }
        }
        if (it == 0) ke0 = ke;
        if (ke0 <= 0.0 || ke <= tol * ke0) {
            ++it;
            break;
        }
    }
    *ke_ratio = ke0 > 0.0 ? ke / ke0 : 0.0;
    orc_density_force(c, s, k, nk);
    for (long long a = 0; a < n; ++a) s->flags[a] &= (unsigned char)~ORC_FLAG_NEW;
    if (g) grid_free(g);
    free(dx);
    free(kt);
    return it;
}

/* ------------------------------------------------- individual time steps */

/* the time-step limit of particle i: min(ccour h / v_sig, cforce sqrt(h / |a|)) */
static double particle_dt(const orc_cfg* c, const orc_state* s, long long i)
{
    double dt = INFINITY;
    if (s->vsig[i] > 0.0) {
        double t = c->ccour * s->h[i] / s->vsig[i];
        if (t < dt) dt = t;
    }
    double a = sqrt(s->ax[i] * s->ax[i] + s->ay[i] * s->ay[i] + s->az[i] * s->az[i]);
    if (a > 0.0) {
        double t = c->cforce * sqrt(s->h[i] / a);
        if (t < dt) dt = t;
    }
    return dt;
}

/* the smallest bin b <= B with dt_max / 2^b <= dt (B if none) */
static int wanted_bin(double dt, double dt_max, int B)
{
    int b = 0;
    double d = dt_max;
    while (b < B && d > dt) {
        d *= 0.5;
        ++b;
    }
    return b;
}

static void kick_one(const orc_cfg* c, orc_state* s, long long i, double hdt)
{
    s->vx[i] += hdt * s->ax[i];
    s->vy[i] += hdt * s->ay[i];
    s->vz[i] += hdt * s->az[i];
    if (c->eos == 0) s->u[i] += hdt * s->dudt[i];
}

/*
 * One step of length dt_max with individual time steps (Sec. 2.5): particle i
 * in bin b_i (0 <= b_i <= B) takes steps of dt_max / 2^b_i on the grid of the
 * 2^B substeps of dt_min = dt_max / 2^B.  Per substep k:
 *   half kick of the particles whose step starts at k (old accelerations);
 *   drift of every particle by dt_min;
 *   for the particles whose step ends at k + 1 (the active ones), in the order
 *   of the global step: split/merge restricted to them (Sec. 2.5: APR over
 *   active particles only; children keep the parent's bin for this kick),
 *   density and forces of the active particles (the others keep their last
 *   values), their second half kick, and their new bins: a split or merged
 *   particle goes to bin B (Sec. 2.5), the others to the bin of their time-step
 *   limit, moving to a longer step only where its grid meets the current time.
 * Point masses take every substep (bin B): half kick, drift, accretion of the
 * live gas inside their radii and zones moved onto them after the drift, and
 * after the active particles' forces their pull on the active gas and their
 * accelerations from every live gas particle at its current position, then the
 * closing half kick.
 * init_bins != 0 first assigns every particle's bin from its limit.  With B = 0
 * this is the global step.  Returns 0, or -1 if capacity ran out.  *updates:
 * particle force updates done; *saturated: updates whose limit was below
 * dt_min (kept in bin B).
 */
int orc_step_bins(const orc_cfg* c, orc_state* s, orc_region* rg, int nr, orc_sink* kk, int nk,
                  double dt_max, int B, int init_bins, unsigned long long* step, orc_counts* cnt,
                  long long* updates, long long* saturated)
{
    const long long nsub = 1LL << B;
    const double dtmin = dt_max / (double)nsub;
    memset(cnt, 0, sizeof(*cnt));
    *updates = 0;
    *saturated = 0;
    if (init_bins)
        for (long long i = 0; i < s->n; ++i) s->bin[i] = (unsigned char)wanted_bin(particle_dt(c, s, i), dt_max, B);
    long long* act = (long long*)malloc(sizeof(long long) * (size_t)(s->cap ? s->cap : 1));
    unsigned char* pulled = (unsigned char*)malloc((size_t)(s->cap ? s->cap : 1));
    for (long long k = 0; k < nsub; ++k) {
        for (long long i = 0; i < s->n; ++i) {
            if (s->flags[i] & (ORC_FLAG_FIXED | ORC_FLAG_DEAD)) continue;
            long long period = nsub >> s->bin[i];
            if (k % period == 0) kick_one(c, s, i, 0.5 * dt_max / (double)(1LL << s->bin[i]));
        }
        for (int j = 0; j < nk; ++j)
            for (int d = 0; d < 3; ++d) kk[j].v[d] += 0.5 * dtmin * kk[j].a[d];
        for (long long i = 0; i < s->n; ++i) {
            if (s->flags[i] & (ORC_FLAG_FIXED | ORC_FLAG_DEAD)) continue;
            s->x[i] = wrap1(c, 0, s->x[i] + dtmin * s->vx[i]);
            s->y[i] = wrap1(c, 1, s->y[i] + dtmin * s->vy[i]);
            s->z[i] = wrap1(c, 2, s->z[i] + dtmin * s->vz[i]);
        }
        for (int j = 0; j < nk; ++j)
            for (int d = 0; d < 3; ++d) kk[j].x[d] += dtmin * kk[j].v[d];
        if (nk > 0) cnt->n_accreted += orc_accrete(c, s, kk, nk);
        orc_track_regions(rg, nr, kk, nk);
        /* APR over the particles whose step ends now */
        for (long long i = 0; i < s->n; ++i)
            if ((k + 1) % (nsub >> s->bin[i]) != 0) s->flags[i] |= ORC_FLAG_INACTIVE;
        orc_counts cs;
        int rc = orc_split_merge(c, s, rg, nr, *step, &cs);
        (*step)++;
        for (long long i = 0; i < s->n; ++i) s->flags[i] &= (unsigned char)~ORC_FLAG_INACTIVE;
        if (rc != 0) {
            free(act);
            free(pulled);
            return -1;
        }
        for (int l = 0; l < ORC_MAXLEV; ++l) {
            cnt->n_split[l] += cs.n_split[l];
            cnt->n_merge[l] += cs.n_merge[l];
            cnt->n_spare[l] = cs.n_spare[l];
        }
        cnt->n_dead += cs.n_dead;
        long long na = 0;
        for (long long i = 0; i < s->n; ++i)
            if (!(s->flags[i] & ORC_FLAG_DEAD) && (k + 1) % (nsub >> s->bin[i]) == 0) act[na++] = i;
        orc_density(c, s, act, na);
        orc_force(c, s, act, na);
        if (nk > 0) {
            memset(pulled, 0, (size_t)s->n);
            for (long long t = 0; t < na; ++t) pulled[act[t]] = 1;
            sink_gravity_some(c, s, kk, nk, pulled);
        }
        for (long long t = 0; t < na; ++t) {
            long long i = act[t];
            if (s->flags[i] & ORC_FLAG_FIXED) continue;
            kick_one(c, s, i, 0.5 * dt_max / (double)(1LL << s->bin[i]));
        }
        for (int j = 0; j < nk; ++j)
            for (int d = 0; d < 3; ++d) kk[j].v[d] += 0.5 * dtmin * kk[j].a[d];
        *updates += na;
        /* new bins, on the grid point k + 1 */
        int aligned = B; /* the longest step whose grid contains k + 1 */
        while (aligned > 0 && (k + 1) % (nsub >> (aligned - 1)) == 0) --aligned;
        for (long long t = 0; t < na; ++t) {
            long long i = act[t];
            double dti = particle_dt(c, s, i);
            int b;
            if (s->flags[i] & ORC_FLAG_CHANGED) {
                b = B;
            } else {
                b = wanted_bin(dti, dt_max, B);
                if (b < aligned) b = aligned;
            }
            if (dti < dtmin) ++(*saturated);
            s->bin[i] = (unsigned char)b;
        }
    }
    free(act);
    free(pulled);
    return 0;
}
