/*
 * FP64 CPU oracle for the list-driven 4th-order Hermite force evaluation of
 * Fukushige & Kawai (arXiv:1602.02832).  TEST INFRASTRUCTURE ONLY: the tests,
 * the package smoke check and the benchmark's CPU-baseline leg call it; the
 * product library never does, and the two share no code.
 *
 * The paper describes its loop (Section 2, the numbered steps of the original
 * GRAPE-6 Hermite loop and of the tree loop) but prints none of the formulas it
 * relies on.  This file writes out the textbook forms of the methods it cites:
 *   - Hermite scheme with block individual timesteps: Makino & Aarseth 1992,
 *     McMillan 1986 (Section 1);
 *   - Aarseth 1999 timestep criterion with eta (Section 3);
 *   - Barnes-Hut tree with centre-of-mass virtual particles (Section 1) and
 *     Barnes 1990 grouping with n_crit (Section 2);
 *   - tree nodes as pseudo-particles with position, velocity, acceleration and
 *     jerk that are predicted like particles (Section 2, step 1).
 * Every point where the paper is silent is a documented reading.  The tree is
 * Morton-ordered by default; Peano-Hilbert order (the paper's, Section 2) is an
 * option: it orders the same octree's children along the curve.
 *
 * Plain by intent: sums run in index order, no blocking or reordering; OpenMP
 * only splits independent i-particles (or groups) across threads.
 */
#include "hermite_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define MORTON_BITS 21
#define MORTON_MAX ((1u << MORTON_BITS) - 1u)

int hho_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* ------------------------------------------------------------------------ */
/* Pairwise Plummer-softened interaction (Makino & Aarseth 1992).           */
/*   r = x_j - x_i, w = v_j - v_i, s = |r|^2 + eps^2                        */
/*   a   += m_j r / s^{3/2}                                                 */
/*   jerk += m_j [ w / s^{3/2} - 3 (r.w) r / s^{5/2} ]                     */
/*   pot -= m_j / s^{1/2}                                                   */
/* ------------------------------------------------------------------------ */
static void add_pair(const double xi[3], const double vi[3],
                     const double xj[3], const double vj[3], double mj, double eps2,
                     double acc[3], double jerk[3], double *pot)
{
    double r[3], w[3];
    for (int k = 0; k < 3; k++) {
        r[k] = xj[k] - xi[k];
        w[k] = vj[k] - vi[k];
    }
    double s = r[0] * r[0] + r[1] * r[1] + r[2] * r[2] + eps2;
    double rw = r[0] * w[0] + r[1] * w[1] + r[2] * w[2];
    double inv_s12 = 1.0 / sqrt(s);
    double inv_s32 = inv_s12 / s;
    double inv_s52 = inv_s32 / s;
    for (int k = 0; k < 3; k++) {
        acc[k] += mj * r[k] * inv_s32;
        jerk[k] += mj * (w[k] * inv_s32 - 3.0 * rw * r[k] * inv_s52);
    }
    *pot -= mj * inv_s12;
}

static void force_on(int i, int n, const double *x, const double *v, const double *m,
                     double eps2, double *acc, double *jerk, double *pot)
{
    double a[3] = {0, 0, 0}, jk[3] = {0, 0, 0}, p = 0.0;
    for (int j = 0; j < n; j++) {
        if (j == i) continue;
        add_pair(&x[3 * i], &v[3 * i], &x[3 * j], &v[3 * j], m[j], eps2, a, jk, &p);
    }
    for (int k = 0; k < 3; k++) {
        acc[k] = a[k];
        jerk[k] = jk[k];
    }
    *pot = p;
}

/* Section 2, the original (GRAPE-6) Hermite loop, step 5: force from all
 * other particles. */
void hho_direct_force(int n, const double *x, const double *v, const double *m,
                      double eps2, double *acc, double *jerk, double *pot)
{
#pragma omp parallel for schedule(dynamic, 16)
    for (int i = 0; i < n; i++)
        force_on(i, n, x, v, m, eps2, &acc[3 * i], &jerk[3 * i], &pot[i]);
}

void hho_direct_force_subset(int n, const double *x, const double *v, const double *m,
                             double eps2, int n_i, const int32_t *i_idx,
                             double *acc, double *jerk, double *pot)
{
#pragma omp parallel for schedule(dynamic, 4)
    for (int k = 0; k < n_i; k++)
        force_on(i_idx[k], n, x, v, m, eps2, &acc[3 * k], &jerk[3 * k], &pot[k]);
}

/* Section 2, tree loop steps 4a and 5: the force on i from its group's list
 * only (nodes enter as particles at their predicted centre of mass). */
void hho_list_force(int n_j, const double *xj, const double *vj, const double *mj,
                    int n_act, const int32_t *i_idx, const int32_t *gid,
                    const int64_t *list_off, const int32_t *list_idx, double eps2,
                    double *acc, double *jerk, double *pot)
{
    (void)n_j;
#pragma omp parallel for schedule(dynamic, 4)
    for (int k = 0; k < n_act; k++) {
        int i = i_idx[k];
        int g = gid[k];
        double a[3] = {0, 0, 0}, jk[3] = {0, 0, 0}, p = 0.0;
        for (int64_t e = list_off[g]; e < list_off[g + 1]; e++) {
            int j = list_idx[e];
            if (j == i) continue;
            add_pair(&xj[3 * i], &vj[3 * i], &xj[3 * j], &vj[3 * j], mj[j], eps2, a, jk, &p);
        }
        for (int c = 0; c < 3; c++) {
            acc[3 * k + c] = a[c];
            jerk[3 * k + c] = jk[c];
        }
        pot[k] = p;
    }
}

/* ------------------------------------------------------------------------ */
/* Hermite predictor / corrector / timesteps                                 */
/* ------------------------------------------------------------------------ */

/* Predictor (Makino & Aarseth 1992; for tree nodes, Section 2 step 1):
 *   x_p = x + v D + a D^2/2 + jk D^3/6,   v_p = v + a D + jk D^2/2,  D = t - t0. */
void hho_predict(int n, const double *x, const double *v, const double *a, const double *jk,
                 const double *t0, double t, double *xp, double *vp)
{
    for (int i = 0; i < n; i++) {
        double d = t - t0[i];
        for (int k = 0; k < 3; k++) {
            int q = 3 * i + k;
            xp[q] = x[q] + v[q] * d + a[q] * d * d / 2.0 + jk[q] * d * d * d / 6.0;
            vp[q] = v[q] + a[q] * d + jk[q] * d * d / 2.0;
        }
    }
}

/* 4th-order Hermite corrector (Makino & Aarseth 1992).  With a0, j0 at the
 * start and a1, j1 at the end of a step of length D, the interpolating cubic
 * for a(t) has, at the start,
 *   a^(2) = (-6 (a0 - a1) - D (4 j0 + 2 j1)) / D^2
 *   a^(3) = (12 (a0 - a1) + 6 D (j0 + j1)) / D^3
 * and the corrected state is
 *   x1 = x_p + a^(2) D^4/24 + a^(3) D^5/120,  v1 = v_p + a^(2) D^3/6 + a^(3) D^4/24.
 * a^(2) at the end of the step is a^(2) + a^(3) D. */
void hho_correct_one(double dt, const double xp[3], const double vp[3],
                     const double a0[3], const double j0[3],
                     const double a1[3], const double j1[3],
                     double x1[3], double v1[3], double a2_end[3], double a3[3])
{
    double d = dt, d2 = dt * dt, d3 = d2 * dt;
    for (int k = 0; k < 3; k++) {
        double a2s = (-6.0 * (a0[k] - a1[k]) - d * (4.0 * j0[k] + 2.0 * j1[k])) / d2;
        double a3s = (12.0 * (a0[k] - a1[k]) + 6.0 * d * (j0[k] + j1[k])) / d3;
        x1[k] = xp[k] + a2s * d2 * d2 / 24.0 + a3s * d2 * d3 / 120.0;
        v1[k] = vp[k] + a2s * d3 / 6.0 + a3s * d2 * d2 / 24.0;
        a2_end[k] = a2s + a3s * d;
        a3[k] = a3s;
    }
}

static double norm3(const double u[3]) { return sqrt(u[0] * u[0] + u[1] * u[1] + u[2] * u[2]); }

/* Aarseth (1999) criterion:
 *   dt = sqrt( eta (|a| |a^(2)| + |jk|^2) / (|jk| |a^(3)| + |a^(2)|^2) ). */
double hho_aarseth_dt(double eta, const double a[3], const double j[3],
                      const double a2[3], const double a3[3])
{
    double na = norm3(a), nj = norm3(j), n2 = norm3(a2), n3 = norm3(a3);
    return sqrt(eta * (na * n2 + nj * nj) / (nj * n3 + n2 * n2));
}

/* Largest power of two that is <= x (x > 0, finite). */
static double pow2_floor(double x)
{
    int e;
    double f = frexp(x, &e); /* x = f 2^e, f in [0.5, 1) */
    (void)f;
    return ldexp(1.0, e - 1);
}

/* Block timestep quantisation (McMillan 1986), reading used throughout:
 *   q = largest power of two <= dt_want;
 *   at most doubling per step: q <= 2 dt_old;
 *   a larger step only where t_new is a multiple of it, else keep dt_old;
 *   clamp to [dt_min, dt_max].
 * A NaN request keeps dt_old; an infinite one asks for doubling. */
double hho_block_dt(double dt_want, double dt_old, double t_new, double dt_min, double dt_max)
{
    double q;
    if (isnan(dt_want))
        q = dt_old;
    else if (isinf(dt_want))
        q = 2.0 * dt_old;
    else
        q = pow2_floor(dt_want);
    if (q > 2.0 * dt_old) q = 2.0 * dt_old;
    if (q > dt_old && fmod(t_new, q) != 0.0) q = dt_old;
    if (q > dt_max) q = dt_max;
    if (q < dt_min) q = dt_min;
    return q;
}

/* Initial step: eta_s |a| / |jk| (reading), quantised and clamped. */
double hho_initial_dt(double eta_s, const double a[3], const double j[3],
                      double dt_min, double dt_max)
{
    double nj = norm3(j);
    double q;
    if (nj == 0.0)
        q = dt_max;
    else {
        double want = eta_s * norm3(a) / nj;
        q = (want > 0.0 && isfinite(want)) ? pow2_floor(want) : dt_max;
    }
    if (q > dt_max) q = dt_max;
    if (q < dt_min) q = dt_min;
    return q;
}

/* ------------------------------------------------------------------------ */
/* Section 2, tree loop step 1: the octree.  Morton order by default        */
/* (reading: the paper orders particles along a Peano-Hilbert curve, which  */
/* hho_tree_build_ordered offers; 21 bits per axis either way).              */
/*   root cube: lo_c = min_k x_kc, S = max_c (max_k x_kc - lo_c) (1 if 0);   */
/*   key digit at level l (0 = coarsest) is (bx<<2)|(by<<1)|bz of bit 20-l;  */
/*   u_c = floor((x_c - lo_c) * (2^21 / S)), clamped to [0, 2^21 - 1];      */
/*   particles sorted by (key, input index);                                 */
/*   a cell is split while it holds more than `leaf` particles and its depth */
/*   is below 21; children in octant order; cells numbered in pre-order.     */
/* ------------------------------------------------------------------------ */

struct hho_tree {
    int n, n_cells, cap_cells, n_groups;
    int leaf, n_crit;
    double theta;
    int32_t *perm;
    uint64_t *key;
    int32_t *c_begin, *c_end, *c_depth, *c_nchild;
    int32_t *c_child; /* [cap][8] */
    double *c_side;
    double *c_m, *c_x, *c_v, *c_a, *c_j;
    int32_t *g_cell, *g_begin, *g_end;
    int32_t *group_of;
    int64_t *list_off;
    int32_t *list_idx;
};

typedef struct {
    uint64_t key;
    int32_t idx;
} key_idx;

static int cmp_key_idx(const void *pa, const void *pb)
{
    const key_idx *a = (const key_idx *)pa, *b = (const key_idx *)pb;
    if (a->key < b->key) return -1;
    if (a->key > b->key) return 1;
    return (a->idx > b->idx) - (a->idx < b->idx);
}

static uint64_t spread3(uint32_t u)
{
    uint64_t out = 0;
    for (int b = 0; b < MORTON_BITS; b++)
        out |= (uint64_t)((u >> b) & 1u) << (3 * b);
    return out;
}

uint64_t hho_morton_key(uint32_t ix, uint32_t iy, uint32_t iz)
{
    return (spread3(ix) << 2) | (spread3(iy) << 1) | spread3(iz);
}

/* Peano-Hilbert index of cell (ix, iy, iz) of a 2^bits grid, after Skilling
 * (2004, "Programming the Hilbert curve").  Working from the top bit down,
 * each lower bit field of the three coordinates is brought into the frame of
 * the sub-cube the higher bits selected: where a coordinate's current bit is
 * set, the low bits of the first coordinate are complemented, otherwise the
 * low bits of the first coordinate and that coordinate are swapped.  The
 * coordinates are then Gray-coded against each other, a common correction
 * from the last coordinate's bits is applied, and the bits are read out
 * level by level, first coordinate first, giving 3 bits per level. */
uint64_t hho_hilbert_key(uint32_t ix, uint32_t iy, uint32_t iz, int bits)
{
    uint32_t c[3] = {ix, iy, iz};
    for (int lev = bits - 1; lev >= 1; lev--) {
        const uint32_t bit = 1u << lev, low = bit - 1u;
        for (int k = 0; k < 3; k++) {
            if (c[k] & bit) {
                c[0] ^= low;
            } else {
                const uint32_t diff = (c[0] ^ c[k]) & low;
                c[0] ^= diff;
                c[k] ^= diff;
            }
        }
    }
    c[1] ^= c[0];
    c[2] ^= c[1];
    uint32_t fix = 0;
    for (int lev = bits - 1; lev >= 1; lev--)
        if (c[2] & (1u << lev)) fix ^= (1u << lev) - 1u;
    for (int k = 0; k < 3; k++) c[k] ^= fix;
    uint64_t key = 0;
    for (int lev = bits - 1; lev >= 0; lev--)
        for (int k = 0; k < 3; k++) key = (key << 1) | ((c[k] >> lev) & 1u);
    return key;
}

static int new_cell(hho_tree *t)
{
    if (t->n_cells == t->cap_cells) {
        int cap = t->cap_cells ? 2 * t->cap_cells : 1024;
        t->c_begin = realloc(t->c_begin, sizeof(int32_t) * cap);
        t->c_end = realloc(t->c_end, sizeof(int32_t) * cap);
        t->c_depth = realloc(t->c_depth, sizeof(int32_t) * cap);
        t->c_nchild = realloc(t->c_nchild, sizeof(int32_t) * cap);
        t->c_child = realloc(t->c_child, sizeof(int32_t) * 8 * cap);
        t->c_side = realloc(t->c_side, sizeof(double) * cap);
        t->cap_cells = cap;
    }
    return t->n_cells++;
}

static int octant(uint64_t key, int depth)
{
    return (int)((key >> (3 * (MORTON_BITS - 1 - depth))) & 7u);
}

static int build_cell(hho_tree *t, int begin, int end, int depth, double side)
{
    int c = new_cell(t);
    t->c_begin[c] = begin;
    t->c_end[c] = end;
    t->c_depth[c] = depth;
    t->c_side[c] = side;
    t->c_nchild[c] = 0;
    if (end - begin <= t->leaf || depth >= MORTON_BITS) return c;
    int b = begin;
    for (int o = 0; o < 8; o++) {
        int e = b;
        while (e < end && octant(t->key[e], depth) == o) e++;
        if (e > b) {
            int ch = build_cell(t, b, e, depth + 1, side * 0.5);
            t->c_child[8 * c + t->c_nchild[c]] = ch;
            t->c_nchild[c]++;
        }
        b = e;
    }
    return c;
}

/* Groups (Barnes 1990): the maximal cells holding at most n_crit particles. */
static void find_groups(hho_tree *t, int c, int *cap)
{
    if (t->c_end[c] - t->c_begin[c] <= t->n_crit || t->c_nchild[c] == 0) {
        if (t->n_groups == *cap) {
            *cap = *cap ? 2 * *cap : 256;
            t->g_cell = realloc(t->g_cell, sizeof(int32_t) * *cap);
            t->g_begin = realloc(t->g_begin, sizeof(int32_t) * *cap);
            t->g_end = realloc(t->g_end, sizeof(int32_t) * *cap);
        }
        t->g_cell[t->n_groups] = c;
        t->g_begin[t->n_groups] = t->c_begin[c];
        t->g_end[t->n_groups] = t->c_end[c];
        t->n_groups++;
        return;
    }
    for (int k = 0; k < t->c_nchild[c]; k++) find_groups(t, t->c_child[8 * c + k], cap);
}

typedef struct {
    int32_t *v;
    int64_t n, cap;
} ivec;

static void ivec_push(ivec *a, int32_t x)
{
    if (a->n == a->cap) {
        a->cap = a->cap ? 2 * a->cap : 1024;
        a->v = realloc(a->v, sizeof(int32_t) * a->cap);
    }
    a->v[a->n++] = x;
}

static int cmp_i32(const void *pa, const void *pb)
{
    int32_t a = *(const int32_t *)pa, b = *(const int32_t *)pb;
    return (a > b) - (a < b);
}

/* Interaction list of group g (reading of Barnes 1990; the paper gives no
 * opening criterion).  Walk from the root:
 *   - g itself: its particles enter directly (in-group interactions are
 *     computed directly, Section 2);
 *   - an ancestor of g: always opened;
 *   - any other cell C with one particle: that particle enters;
 *   - otherwise C enters as a node iff side_C < theta * d, d = distance from
 *     C's centre of mass to the bounding box of g's member positions;
 *   - else a leaf C contributes its particles and an internal C is opened.
 * The list is sorted ascending. */
static void walk(const hho_tree *t, int c, int g, const double blo[3], const double bhi[3], ivec *out)
{
    int gb = t->g_begin[g], ge = t->g_end[g];
    int cb = t->c_begin[c], ce = t->c_end[c];
    if (c == t->g_cell[g]) {
        for (int p = cb; p < ce; p++) ivec_push(out, p);
        return;
    }
    if (cb <= gb && ge <= ce) {
        for (int k = 0; k < t->c_nchild[c]; k++) walk(t, t->c_child[8 * c + k], g, blo, bhi, out);
        return;
    }
    if (ce - cb == 1) {
        ivec_push(out, cb);
        return;
    }
    double d2 = 0.0;
    for (int k = 0; k < 3; k++) {
        double cm = t->c_x[3 * c + k];
        double gap = 0.0;
        if (cm < blo[k]) gap = blo[k] - cm;
        else if (cm > bhi[k]) gap = cm - bhi[k];
        d2 += gap * gap;
    }
    double d = sqrt(d2);
    if (t->c_side[c] < t->theta * d) {
        ivec_push(out, t->n + c);
        return;
    }
    if (t->c_nchild[c] == 0) {
        for (int p = cb; p < ce; p++) ivec_push(out, p);
        return;
    }
    for (int k = 0; k < t->c_nchild[c]; k++) walk(t, t->c_child[8 * c + k], g, blo, bhi, out);
}

hho_tree *hho_tree_build(int n, const double *x, const double *v, const double *a,
                         const double *jk, const double *m,
                         int leaf, int n_crit, double theta)
{
    return hho_tree_build_ordered(n, x, v, a, jk, m, leaf, n_crit, theta, 0);
}

hho_tree *hho_tree_build_ordered(int n, const double *x, const double *v, const double *a,
                                 const double *jk, const double *m,
                                 int leaf, int n_crit, double theta, int order)
{
    if (n < 1 || leaf < 1 || n_crit < 1) return NULL;
    hho_tree *t = calloc(1, sizeof(hho_tree));
    t->n = n;
    t->leaf = leaf;
    t->n_crit = n_crit;
    t->theta = theta;

    /* root cube and keys */
    double lo[3], hi[3];
    for (int k = 0; k < 3; k++) lo[k] = hi[k] = x[k];
    for (int i = 1; i < n; i++)
        for (int k = 0; k < 3; k++) {
            if (x[3 * i + k] < lo[k]) lo[k] = x[3 * i + k];
            if (x[3 * i + k] > hi[k]) hi[k] = x[3 * i + k];
        }
    double side = 0.0;
    for (int k = 0; k < 3; k++)
        if (hi[k] - lo[k] > side) side = hi[k] - lo[k];
    if (side == 0.0) side = 1.0;
    double scale = (double)(1u << MORTON_BITS) / side;
    key_idx *ki = malloc(sizeof(key_idx) * n);
    for (int i = 0; i < n; i++) {
        uint32_t u[3];
        for (int k = 0; k < 3; k++) {
            double f = floor((x[3 * i + k] - lo[k]) * scale);
            if (f < 0.0) f = 0.0;
            if (f > (double)MORTON_MAX) f = (double)MORTON_MAX;
            u[k] = (uint32_t)f;
        }
        ki[i].key = order == 1 ? hho_hilbert_key(u[0], u[1], u[2], MORTON_BITS) : hho_morton_key(u[0], u[1], u[2]);
        ki[i].idx = i;
    }
    qsort(ki, n, sizeof(key_idx), cmp_key_idx);
    t->perm = malloc(sizeof(int32_t) * n);
    t->key = malloc(sizeof(uint64_t) * n);
    for (int i = 0; i < n; i++) {
        t->perm[i] = ki[i].idx;
        t->key[i] = ki[i].key;
    }
    free(ki);

    build_cell(t, 0, n, 0, side);

    /* node records: mass-weighted moments summed in Morton index order */
    int nc = t->n_cells;
    t->c_m = malloc(sizeof(double) * nc);
    t->c_x = malloc(sizeof(double) * 3 * nc);
    t->c_v = malloc(sizeof(double) * 3 * nc);
    t->c_a = malloc(sizeof(double) * 3 * nc);
    t->c_j = malloc(sizeof(double) * 3 * nc);
#pragma omp parallel for schedule(dynamic, 64)
    for (int c = 0; c < nc; c++) {
        double M = 0.0, sx[3] = {0, 0, 0}, sv[3] = {0, 0, 0}, sa[3] = {0, 0, 0}, sj[3] = {0, 0, 0};
        for (int p = t->c_begin[c]; p < t->c_end[c]; p++) {
            int i = t->perm[p];
            double mi = m[i];
            M += mi;
            for (int k = 0; k < 3; k++) {
                sx[k] += mi * x[3 * i + k];
                sv[k] += mi * v[3 * i + k];
                sa[k] += mi * a[3 * i + k];
                sj[k] += mi * jk[3 * i + k];
            }
        }
        t->c_m[c] = M;
        for (int k = 0; k < 3; k++) {
            t->c_x[3 * c + k] = sx[k] / M;
            t->c_v[3 * c + k] = sv[k] / M;
            t->c_a[3 * c + k] = sa[k] / M;
            t->c_j[3 * c + k] = sj[k] / M;
        }
    }

    int gcap = 0;
    find_groups(t, 0, &gcap);
    t->group_of = malloc(sizeof(int32_t) * n);
    for (int g = 0; g < t->n_groups; g++)
        for (int p = t->g_begin[g]; p < t->g_end[g]; p++) t->group_of[p] = g;

    /* lists, one independent walk per group */
    ivec *lists = calloc(t->n_groups, sizeof(ivec));
#pragma omp parallel for schedule(dynamic, 1)
    for (int g = 0; g < t->n_groups; g++) {
        double blo[3], bhi[3];
        int i0 = t->perm[t->g_begin[g]];
        for (int k = 0; k < 3; k++) blo[k] = bhi[k] = x[3 * i0 + k];
        for (int p = t->g_begin[g]; p < t->g_end[g]; p++) {
            int i = t->perm[p];
            for (int k = 0; k < 3; k++) {
                if (x[3 * i + k] < blo[k]) blo[k] = x[3 * i + k];
                if (x[3 * i + k] > bhi[k]) bhi[k] = x[3 * i + k];
            }
        }
        walk(t, 0, g, blo, bhi, &lists[g]);
        qsort(lists[g].v, lists[g].n, sizeof(int32_t), cmp_i32);
    }
    t->list_off = malloc(sizeof(int64_t) * (t->n_groups + 1));
    t->list_off[0] = 0;
    for (int g = 0; g < t->n_groups; g++) t->list_off[g + 1] = t->list_off[g] + lists[g].n;
    t->list_idx = malloc(sizeof(int32_t) * (t->list_off[t->n_groups] > 0 ? t->list_off[t->n_groups] : 1));
    for (int g = 0; g < t->n_groups; g++) {
        if (lists[g].n) memcpy(&t->list_idx[t->list_off[g]], lists[g].v, sizeof(int32_t) * lists[g].n);
        free(lists[g].v);
    }
    free(lists);
    return t;
}

void hho_tree_free(hho_tree *t)
{
    if (!t) return;
    free(t->perm); free(t->key);
    free(t->c_begin); free(t->c_end); free(t->c_depth); free(t->c_nchild); free(t->c_child);
    free(t->c_side); free(t->c_m); free(t->c_x); free(t->c_v); free(t->c_a); free(t->c_j);
    free(t->g_cell); free(t->g_begin); free(t->g_end); free(t->group_of);
    free(t->list_off); free(t->list_idx);
    free(t);
}

int hho_tree_n_cells(const hho_tree *t) { return t->n_cells; }
int hho_tree_n_groups(const hho_tree *t) { return t->n_groups; }
int64_t hho_tree_list_len(const hho_tree *t) { return t->list_off[t->n_groups]; }
void hho_tree_perm(const hho_tree *t, int32_t *perm) { memcpy(perm, t->perm, sizeof(int32_t) * t->n); }
void hho_tree_keys(const hho_tree *t, uint64_t *keys) { memcpy(keys, t->key, sizeof(uint64_t) * t->n); }

void hho_tree_nodes(const hho_tree *t, double *x, double *v, double *a, double *jk, double *m)
{
    int nc = t->n_cells;
    memcpy(x, t->c_x, sizeof(double) * 3 * nc);
    memcpy(v, t->c_v, sizeof(double) * 3 * nc);
    memcpy(a, t->c_a, sizeof(double) * 3 * nc);
    memcpy(jk, t->c_j, sizeof(double) * 3 * nc);
    memcpy(m, t->c_m, sizeof(double) * nc);
}

void hho_tree_cells(const hho_tree *t, int32_t *begin, int32_t *end, int32_t *depth, double *side)
{
    int nc = t->n_cells;
    memcpy(begin, t->c_begin, sizeof(int32_t) * nc);
    memcpy(end, t->c_end, sizeof(int32_t) * nc);
    memcpy(depth, t->c_depth, sizeof(int32_t) * nc);
    memcpy(side, t->c_side, sizeof(double) * nc);
}

void hho_tree_groups(const hho_tree *t, int32_t *g_cell, int32_t *g_begin, int32_t *g_end,
                     int32_t *group_of)
{
    memcpy(g_cell, t->g_cell, sizeof(int32_t) * t->n_groups);
    memcpy(g_begin, t->g_begin, sizeof(int32_t) * t->n_groups);
    memcpy(g_end, t->g_end, sizeof(int32_t) * t->n_groups);
    memcpy(group_of, t->group_of, sizeof(int32_t) * t->n);
}

void hho_tree_lists(const hho_tree *t, int64_t *off, int32_t *idx)
{
    memcpy(off, t->list_off, sizeof(int64_t) * (t->n_groups + 1));
    if (t->list_off[t->n_groups])
        memcpy(idx, t->list_idx, sizeof(int32_t) * t->list_off[t->n_groups]);
}

/* ------------------------------------------------------------------------ */
/* The block-step loop (Section 2, tree loop steps 1-7; with use_tree = 0    */
/* the original Hermite loop with direct forces).                            */
/*   1. at t = 0 and every dt_tree: build tree, groups, lists, node records; */
/*   2. t_next = min_i (t_i + dt_i), active set {i : t_i + dt_i = t_next};   */
/*   4. predict every j entry (particles from t_i, nodes from t_tree);       */
/*   4a/5. force on each active i from its group's list;                     */
/*   6. correct, new Aarseth step, block-quantised;                          */
/*   7. advance, and rebuild when t_next reaches t_tree + dt_tree.           */
/* Readings: the block ending at t_tree + dt_tree is evaluated with the old  */
/* lists and the rebuild follows from the synchronised state; at t = 0 the   */
/* nodes are first built with zero a and jk (unused at zero prediction       */
/* interval), forces are evaluated, and the tree is rebuilt with them.       */
/* ------------------------------------------------------------------------ */

typedef struct {
    hho_tree *t;
    int n_j;
    double *xj, *vj, *aj, *jj, *mj, *tj; /* Morton-ordered particles, then nodes */
    int32_t *inv; /* input index -> Morton position */
} tree_view;

static void view_build(tree_view *tv, int n, const double *x, const double *v, const double *a,
                       const double *jk, const double *m, const double *ti, double t_tree,
                       const hho_params *p)
{
    tv->t = hho_tree_build(n, x, v, a, jk, m, p->leaf, p->n_crit, p->theta);
    int nc = tv->t->n_cells;
    tv->n_j = n + nc;
    tv->xj = malloc(sizeof(double) * 3 * tv->n_j);
    tv->vj = malloc(sizeof(double) * 3 * tv->n_j);
    tv->aj = malloc(sizeof(double) * 3 * tv->n_j);
    tv->jj = malloc(sizeof(double) * 3 * tv->n_j);
    tv->mj = malloc(sizeof(double) * tv->n_j);
    tv->tj = malloc(sizeof(double) * tv->n_j);
    tv->inv = malloc(sizeof(int32_t) * n);
    for (int k = 0; k < n; k++) {
        int i = tv->t->perm[k];
        tv->inv[i] = k;
        tv->mj[k] = m[i];
        tv->tj[k] = ti[i];
    }
    for (int c = 0; c < nc; c++) {
        tv->mj[n + c] = tv->t->c_m[c];
        tv->tj[n + c] = t_tree;
        for (int k = 0; k < 3; k++) {
            tv->xj[3 * (n + c) + k] = tv->t->c_x[3 * c + k];
            tv->vj[3 * (n + c) + k] = tv->t->c_v[3 * c + k];
            tv->aj[3 * (n + c) + k] = tv->t->c_a[3 * c + k];
            tv->jj[3 * (n + c) + k] = tv->t->c_j[3 * c + k];
        }
    }
}

static void view_free(tree_view *tv)
{
    hho_tree_free(tv->t);
    free(tv->xj); free(tv->vj); free(tv->aj); free(tv->jj); free(tv->mj); free(tv->tj); free(tv->inv);
    memset(tv, 0, sizeof(*tv));
}

/* Copy the particle part of the state (input order) into the Morton-ordered view. */
static void view_load_particles(tree_view *tv, int n, const double *x, const double *v,
                                const double *a, const double *jk, const double *ti)
{
    for (int k = 0; k < n; k++) {
        int i = tv->t->perm[k];
        tv->tj[k] = ti[i];
        for (int c = 0; c < 3; c++) {
            tv->xj[3 * k + c] = x[3 * i + c];
            tv->vj[3 * k + c] = v[3 * i + c];
            tv->aj[3 * k + c] = a[3 * i + c];
            tv->jj[3 * k + c] = jk[3 * i + c];
        }
    }
}

/* Forces on the active input-index set at time t. */
static void eval_forces(int n, const double *x, const double *v, const double *a, const double *jk,
                        const double *m, const double *ti, double t, int n_act, const int32_t *act,
                        tree_view *tv, const hho_params *p, double *acc, double *jerk, double *pot,
                        int64_t *n_int)
{
    if (!p->use_tree) {
        double *xp = malloc(sizeof(double) * 3 * n), *vp = malloc(sizeof(double) * 3 * n);
        hho_predict(n, x, v, a, jk, ti, t, xp, vp);
        hho_direct_force_subset(n, xp, vp, m, p->eps2, n_act, act, acc, jerk, pot);
        free(xp); free(vp);
        *n_int += (int64_t)n_act * (n - 1);
        return;
    }
    view_load_particles(tv, n, x, v, a, jk, ti);
    double *xp = malloc(sizeof(double) * 3 * tv->n_j), *vp = malloc(sizeof(double) * 3 * tv->n_j);
    hho_predict(tv->n_j, tv->xj, tv->vj, tv->aj, tv->jj, tv->tj, t, xp, vp);
    int32_t *ia = malloc(sizeof(int32_t) * (n_act > 0 ? n_act : 1));
    int32_t *gd = malloc(sizeof(int32_t) * (n_act > 0 ? n_act : 1));
    for (int k = 0; k < n_act; k++) {
        ia[k] = tv->inv[act[k]];
        gd[k] = tv->t->group_of[ia[k]];
        *n_int += tv->t->list_off[gd[k] + 1] - tv->t->list_off[gd[k]] - 1;
    }
    hho_list_force(tv->n_j, xp, vp, tv->mj, n_act, ia, gd, tv->t->list_off, tv->t->list_idx,
                   p->eps2, acc, jerk, pot);
    free(ia); free(gd); free(xp); free(vp);
}

/* Block steps from a synchronised state at t_tree (every t_i = t_tree) with
 * forces a, jk at t_tree, steps dti and the tree view tv built at t_tree,
 * until the next block time passes t_end.  Updates x, v, a, jk, ti, dti in
 * place and adds to *st. */
static int run_loop(int n, double *x, double *v, double *a, double *jk, double *ti, double *dti,
                    const double *m, double t_tree, double t_end, const hho_params *p, tree_view *tv,
                    hho_stats *st)
{
    double *acc = malloc(sizeof(double) * 3 * n), *jerk = malloc(sizeof(double) * 3 * n);
    double *pot = malloc(sizeof(double) * n);
    int32_t *act = malloc(sizeof(int32_t) * n);
    int rc = 0;
    for (;;) {
        double t_next = ti[0] + dti[0];
        for (int i = 1; i < n; i++)
            if (ti[i] + dti[i] < t_next) t_next = ti[i] + dti[i];
        if (t_next > t_end) break;
        int n_act = 0;
        for (int i = 0; i < n; i++)
            if (ti[i] + dti[i] == t_next) act[n_act++] = i;
        eval_forces(n, x, v, a, jk, m, ti, t_next, n_act, act, tv, p, acc, jerk, pot, &st->interactions);
        for (int k = 0; k < n_act; k++) {
            int i = act[k];
            double d = t_next - ti[i];
            double xp[3], vp[3], x1[3], v1[3], a2e[3], a3[3];
            for (int c = 0; c < 3; c++) {
                int q = 3 * i + c;
                xp[c] = x[q] + v[q] * d + a[q] * d * d / 2.0 + jk[q] * d * d * d / 6.0;
                vp[c] = v[q] + a[q] * d + jk[q] * d * d / 2.0;
            }
            hho_correct_one(d, xp, vp, &a[3 * i], &jk[3 * i], &acc[3 * k], &jerk[3 * k], x1, v1, a2e, a3);
            double want = hho_aarseth_dt(p->eta, &acc[3 * k], &jerk[3 * k], a2e, a3);
            double nd = hho_block_dt(want, dti[i], t_next, p->dt_min, p->dt_max);
            for (int c = 0; c < 3; c++) {
                x[3 * i + c] = x1[c];
                v[3 * i + c] = v1[c];
                a[3 * i + c] = acc[3 * k + c];
                jk[3 * i + c] = jerk[3 * k + c];
            }
            ti[i] = t_next;
            dti[i] = nd;
        }
        st->block_steps++;
        st->particle_steps += n_act;
        if (p->use_tree && t_next == t_tree + p->dt_tree) {
            for (int i = 0; i < n; i++)
                if (ti[i] != t_next) rc = -2;
            if (rc) break;
            view_free(tv);
            t_tree = t_next;
            view_build(tv, n, x, v, a, jk, m, ti, t_tree, p);
            st->rebuilds++;
        }
    }
    free(acc); free(jerk); free(pot); free(act);
    return rc;
}

static void copy_out(int n, const double *a, const double *jk, const double *ti, const double *dti,
                     double *a_out, double *jk_out, double *t_out, double *dt_out)
{
    if (a_out) memcpy(a_out, a, sizeof(double) * 3 * n);
    if (jk_out) memcpy(jk_out, jk, sizeof(double) * 3 * n);
    if (t_out) memcpy(t_out, ti, sizeof(double) * n);
    if (dt_out) memcpy(dt_out, dti, sizeof(double) * n);
}

int hho_run(int n, double *x, double *v, const double *m, double t_end,
            const hho_params *p, double *a_out, double *jk_out, double *t_out, double *dt_out,
            hho_stats *stats)
{
    if (n < 2 || p->dt_min <= 0.0 || p->dt_max < p->dt_min) return -1;
    if (p->use_tree && (p->dt_max > p->dt_tree)) return -1;
    hho_stats st = {0, 0, 0, 0};
    double *a = calloc(3 * n, sizeof(double)), *jk = calloc(3 * n, sizeof(double));
    double *ti = calloc(n, sizeof(double)), *dti = calloc(n, sizeof(double));
    double *acc = malloc(sizeof(double) * 3 * n), *jerk = malloc(sizeof(double) * 3 * n);
    double *pot = malloc(sizeof(double) * n);
    int32_t *act = malloc(sizeof(int32_t) * n);
    tree_view tv;
    memset(&tv, 0, sizeof(tv));

    /* initial forces at t = 0, all particles */
    for (int i = 0; i < n; i++) act[i] = i;
    int64_t dummy = 0;
    if (p->use_tree) view_build(&tv, n, x, v, a, jk, m, ti, 0.0, p);
    eval_forces(n, x, v, a, jk, m, ti, 0.0, n, act, &tv, p, acc, jerk, pot, &dummy);
    memcpy(a, acc, sizeof(double) * 3 * n);
    memcpy(jk, jerk, sizeof(double) * 3 * n);
    if (p->use_tree) {
        view_free(&tv);
        view_build(&tv, n, x, v, a, jk, m, ti, 0.0, p);
        st.rebuilds++;
    }
    for (int i = 0; i < n; i++) dti[i] = hho_initial_dt(p->eta_s, &a[3 * i], &jk[3 * i], p->dt_min, p->dt_max);

    int rc = run_loop(n, x, v, a, jk, ti, dti, m, 0.0, t_end, p, &tv, &st);
    if (p->use_tree && tv.t) view_free(&tv);
    copy_out(n, a, jk, ti, dti, a_out, jk_out, t_out, dt_out);
    if (stats) *stats = st;
    free(a); free(jk); free(ti); free(dti); free(acc); free(jerk); free(pot); free(act);
    return rc;
}

/* The same loop continued from a synchronised state at t0 = k dt_tree (every
 * particle at t0 with its forces a, jk there and its block step dt): step 1
 * rebuilds the tree from that state (Section 2), then block steps follow as
 * in hho_run until t_end.  x, v, a, jk, dt are updated in place. */
int hho_resume(int n, double *x, double *v, double *a, double *jk, double *dt, const double *m, double t0,
               double t_end, const hho_params *p, hho_stats *stats)
{
    if (n < 2 || p->dt_min <= 0.0 || p->dt_max < p->dt_min || !(t_end >= t0)) return -1;
    if (p->use_tree && (p->dt_max > p->dt_tree || floor(t0 / p->dt_tree) != t0 / p->dt_tree)) return -1;
    hho_stats st = {0, 0, 0, 0};
    double *ti = malloc(sizeof(double) * n);
    for (int i = 0; i < n; i++) ti[i] = t0;
    tree_view tv;
    memset(&tv, 0, sizeof(tv));
    if (p->use_tree) view_build(&tv, n, x, v, a, jk, m, ti, t0, p);
    int rc = run_loop(n, x, v, a, jk, ti, dt, m, t0, t_end, p, &tv, &st);
    if (p->use_tree && tv.t) view_free(&tv);
    if (stats) *stats = st;
    free(ti);
    return rc;
}

/* Total energy, E = sum m v^2 / 2 + (1/2) sum_i m_i phi_i with phi from the
 * direct softened sum (Section 3: the potential energy is obtained by direct
 * summation, not with the tree). */
double hho_energy(int n, const double *x, const double *v, const double *m, double eps2)
{
    double *acc = malloc(sizeof(double) * 3 * n), *jerk = malloc(sizeof(double) * 3 * n);
    double *pot = malloc(sizeof(double) * n);
    hho_direct_force(n, x, v, m, eps2, acc, jerk, pot);
    double ek = 0.0, ep = 0.0;
    for (int i = 0; i < n; i++) {
        ek += 0.5 * m[i] * (v[3 * i] * v[3 * i] + v[3 * i + 1] * v[3 * i + 1] + v[3 * i + 2] * v[3 * i + 2]);
        ep += 0.5 * m[i] * pot[i];
    }
    free(acc); free(jerk); free(pot);
    return ek + ep;
}
