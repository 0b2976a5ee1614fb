/*
 * oracle.c -- FP64 CPU oracle (test infrastructure only; see oracle.h).
 *
 * Written to be read against the paper, not to be fast:
 *   Eq. 1 ............ oracle_direct, kernel_term
 *   Sect. 1 (tree) ... oracle_tree_build (recursive subdivision), node moments
 *   Eq. 2 (MAC) ...... mac_accept
 *   Sect. 1 (list) ... walk_group / walk_particle (one shared list per group)
 * Readings where the paper is silent are marked READING and repeated in the
 * design notes.
 */
#include "oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

int oracle_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* Threads of the following parallel loops (k < 1: all cores). */
void oracle_set_threads(int k)
{
#ifdef _OPENMP
    omp_set_num_threads(k >= 1 ? k : omp_get_num_procs());
#else
    (void)k;
#endif
}

/* ------------------------------------------------------------------------ */
/* Eq. 1: one softened pair term, accumulated into s[0..2] (acceleration) and
 * s[3] (potential).  (dx,dy,dz) = r_j - r_i. */
static inline void kernel_term(double dx, double dy, double dz, double mj, double e2, double *s)
{
    double r2 = dx * dx + dy * dy + dz * dz + e2;
    double rinv = 1.0 / sqrt(r2);
    double w = mj * rinv * rinv * rinv; /* m_j / (|r|^2 + eps^2)^{3/2} */
    s[0] += w * dx;
    s[1] += w * dy;
    s[2] += w * dz;
    s[3] -= mj * rinv;
}

/* A node's pseudo particle with its quadrupole (an extension beyond the
 * paper's monopoles): the potential of mass M and traceless quadrupole Q at
 * offset s = r_i - com is -M/|s| - s.Q.s / (2 |s|^5); its negative gradient,
 * written with d = com - r_i = -s, is
 *     M d / r^3 - Q d / r^5 + (5/2) (d.Q.d) d / r^7,
 * and, as for the monopole, |d|^2 is softened to |d|^2 + eps^2 in every
 * power of r.  Q = {xx, yy, zz, xy, xz, yz}. */
static inline void quad_term(double dx, double dy, double dz, double M, const double *Q,
                             double e2, double *s)
{
    double r2 = dx * dx + dy * dy + dz * dz + e2;
    double rinv = 1.0 / sqrt(r2), rinv2 = rinv * rinv;
    double rinv3 = rinv * rinv2, rinv5 = rinv3 * rinv2, rinv7 = rinv5 * rinv2;
    double qx = Q[0] * dx + Q[3] * dy + Q[4] * dz;
    double qy = Q[3] * dx + Q[1] * dy + Q[5] * dz;
    double qz = Q[4] * dx + Q[5] * dy + Q[2] * dz;
    double dqd = dx * qx + dy * qy + dz * qz;
    double c = M * rinv3 + 2.5 * dqd * rinv7;
    s[0] += c * dx - qx * rinv5;
    s[1] += c * dy - qy * rinv5;
    s[2] += c * dz - qz * rinv5;
    s[3] -= M * rinv + 0.5 * dqd * rinv5;
}

static void direct_one(int64_t n, const double *x, const double *y, const double *z,
                       const double *m, int64_t i, double G, double e2, double *out)
{
    double s[4] = {0, 0, 0, 0};
    for (int64_t j = 0; j < n; j++) {
        if (j == i) continue; /* j != i in Eq. 1 */
        kernel_term(x[j] - x[i], y[j] - y[i], z[j] - z[i], m[j], e2, s);
    }
    for (int k = 0; k < 4; k++) out[k] = G * s[k];
}

void oracle_direct(int64_t n, const double *x, const double *y, const double *z,
                   const double *m, double G, double eps,
                   double *ax, double *ay, double *az, double *phi)
{
    double e2 = eps * eps;
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t i = 0; i < n; i++) {
        double o[4];
        direct_one(n, x, y, z, m, i, G, e2, o);
        ax[i] = o[0]; ay[i] = o[1]; az[i] = o[2];
        if (phi) phi[i] = o[3];
    }
}

void oracle_direct_targets(int64_t n, const double *x, const double *y, const double *z,
                           const double *m, int64_t nt, const int64_t *tgt,
                           double G, double eps,
                           double *ax, double *ay, double *az, double *phi)
{
    double e2 = eps * eps;
#pragma omp parallel for schedule(dynamic, 4)
    for (int64_t k = 0; k < nt; k++) {
        double o[4];
        direct_one(n, x, y, z, m, tgt[k], G, e2, o);
        ax[k] = o[0]; ay[k] = o[1]; az[k] = o[2];
        if (phi) phi[k] = o[3];
    }
}

/* ------------------------------------------------------------------------ */
/* Bounding cube and FP32 cell quantisation.  READING: the paper sorts
 * space-filling-curve keys (Sect. 4.1) but gives no formula; the cube is the
 * axis-aligned box of the particles, widened by 2^-20 so the maximum maps
 * inside, and cell indices are taken in FP32 so that both implementations
 * quantise identically. */
void oracle_cube(int64_t n, const float *x, const float *y, const float *z, float cube[4])
{
    float lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
    const float *p[3] = {x, y, z};
    for (int64_t i = 0; i < n; i++)
        for (int a = 0; a < 3; a++) {
            float v = p[a][i];
            if (v < lo[a]) lo[a] = v;
            if (v > hi[a]) hi[a] = v;
        }
    if (n <= 0) {
        lo[0] = lo[1] = lo[2] = 0.0f;
        hi[0] = hi[1] = hi[2] = 0.0f;
    }
    float ext = hi[0] - lo[0];
    float ey = hi[1] - lo[1], ez = hi[2] - lo[2];
    if (ey > ext) ext = ey;
    if (ez > ext) ext = ez;
    volatile float L = ext * (1.0f + 0x1p-20f);
    cube[0] = lo[0];
    cube[1] = lo[1];
    cube[2] = lo[2];
    cube[3] = (L > 0.0f) ? L : 1.0f;
}

void oracle_cells(int64_t n, const float *x, const float *y, const float *z,
                  const float cube[4], int levels,
                  uint32_t *qx, uint32_t *qy, uint32_t *qz)
{
    const float *p[3] = {x, y, z};
    uint32_t *q[3] = {qx, qy, qz};
    uint32_t top = (1u << levels) - 1u;
    volatile float scale = (float)(1u << levels) / cube[3];
    for (int64_t i = 0; i < n; i++)
        for (int a = 0; a < 3; a++) {
            volatile float d = p[a][i] - cube[a];
            volatile float t = d * scale;
            float f = floorf(t);
            uint32_t c = (f <= 0.0f) ? 0u : (uint32_t)f;
            q[a][i] = c > top ? top : c;
        }
}

uint64_t oracle_interleave(uint32_t qx, uint32_t qy, uint32_t qz, int levels)
{
    uint64_t key = 0;
    for (int l = levels - 1; l >= 0; l--) {
        key = (key << 3) | ((uint64_t)((qx >> l) & 1u) << 2)
                         | ((uint64_t)((qy >> l) & 1u) << 1)
                         | (uint64_t)((qz >> l) & 1u);
    }
    return key;
}

static const uint64_t *g_sort_keys;
static int cmp_key_index(const void *a, const void *b)
{
    int64_t i = *(const int64_t *)a, j = *(const int64_t *)b;
    uint64_t ki = g_sort_keys[i], kj = g_sort_keys[j];
    if (ki < kj) return -1;
    if (ki > kj) return 1;
    return (i > j) - (i < j);
}

void oracle_sort(int64_t n, const uint64_t *keys, int64_t *order)
{
    for (int64_t i = 0; i < n; i++) order[i] = i;
    g_sort_keys = keys;
    qsort(order, (size_t)n, sizeof(int64_t), cmp_key_index);
    g_sort_keys = NULL;
}

/* ------------------------------------------------------------------------ */
/* Octree (Sect. 1, Barnes & Hut), built by recursive subdivision. */
struct oracle_tree {
    int64_t n;
    int levels, leaf_cap;
    float cube[4];
    double *x, *y, *z, *m;
    uint32_t *q[3];
    uint64_t *key;
    int64_t *order; /* particle ids in tree order */
    /* nodes */
    int64_t nn, capn;
    int32_t *lev, *nchild;
    int64_t *first, *count, *child;
    uint64_t *prefix;
    double *cx, *cy, *cz, *M, *b;
    double *Q; /* traceless quadrupole about com: 6 per node (xx, yy, zz, xy, xz, yz) */
};

static int grow_nodes(oracle_tree *t)
{
    int64_t nc = t->capn ? 2 * t->capn : 1024;
#define GROW(f, T) do { void *p_ = realloc(t->f, (size_t)nc * sizeof(T)); if (!p_) return 0; t->f = (T *)p_; } while (0)
    GROW(lev, int32_t); GROW(nchild, int32_t);
    GROW(first, int64_t); GROW(count, int64_t); GROW(child, int64_t);
    GROW(prefix, uint64_t);
    GROW(cx, double); GROW(cy, double); GROW(cz, double); GROW(M, double); GROW(b, double);
    {
        void *p_ = realloc(t->Q, (size_t)nc * 6 * sizeof(double));
        if (!p_) return 0;
        t->Q = (double *)p_;
    }
#undef GROW
    t->capn = nc;
    return 1;
}

static int64_t new_node(oracle_tree *t)
{
    if (t->nn == t->capn && !grow_nodes(t)) return -1;
    return t->nn++;
}

static const oracle_tree *g_leaf_tree;
static int cmp_leaf(const void *a, const void *b)
{
    int64_t i = *(const int64_t *)a, j = *(const int64_t *)b;
    uint64_t ki = g_leaf_tree->key[i], kj = g_leaf_tree->key[j];
    if (ki < kj) return -1;
    if (ki > kj) return 1;
    return (i > j) - (i < j);
}

/* Node `id` holds order[lo..hi).  Split into the 8 octants of its cell while
 * it holds more than leaf_cap particles and is above the finest level. */
static int build_rec(oracle_tree *t, int64_t id, int level, uint64_t prefix,
                     int64_t lo, int64_t hi, int64_t *tmp)
{
    t->lev[id] = level;
    t->prefix[id] = prefix;
    t->first[id] = lo;
    t->count[id] = hi - lo;
    t->nchild[id] = 0;
    t->child[id] = -1;
    if (hi - lo <= t->leaf_cap || level == t->levels) {
        g_leaf_tree = t;
        qsort(t->order + lo, (size_t)(hi - lo), sizeof(int64_t), cmp_leaf);
        return 1;
    }
    int shift = t->levels - 1 - level;
    int64_t cnt[8] = {0}, pos[8];
    for (int64_t k = lo; k < hi; k++) {
        int64_t p = t->order[k];
        int o = (int)((((t->q[0][p] >> shift) & 1u) << 2) | (((t->q[1][p] >> shift) & 1u) << 1) |
                      ((t->q[2][p] >> shift) & 1u));
        cnt[o]++;
    }
    pos[0] = lo;
    for (int o = 1; o < 8; o++) pos[o] = pos[o - 1] + cnt[o - 1];
    int64_t start[8];
    memcpy(start, pos, sizeof start);
    for (int64_t k = lo; k < hi; k++) {
        int64_t p = t->order[k];
        int o = (int)((((t->q[0][p] >> shift) & 1u) << 2) | (((t->q[1][p] >> shift) & 1u) << 1) |
                      ((t->q[2][p] >> shift) & 1u));
        tmp[pos[o]++] = p;
    }
    memcpy(t->order + lo, tmp + lo, (size_t)(hi - lo) * sizeof(int64_t));
    /* allocate the non-empty children contiguously, then recurse */
    int64_t ids[8];
    int nc = 0;
    for (int o = 0; o < 8; o++) {
        if (!cnt[o]) continue;
        int64_t c = new_node(t);
        if (c < 0) return 0;
        ids[o] = c;
        if (!nc) t->child[id] = c;
        nc++;
    }
    t->nchild[id] = nc;
    for (int o = 0; o < 8; o++) {
        if (!cnt[o]) continue;
        if (!build_rec(t, ids[o], level + 1, (prefix << 3) | (uint64_t)o, start[o],
                       start[o] + cnt[o], tmp))
            return 0;
    }
    return 1;
}

/* Integer cell coordinates of node id at its level (from its prefix). */
static void node_cell(const oracle_tree *t, int64_t id, uint32_t c[3])
{
    c[0] = c[1] = c[2] = 0;
    uint64_t p = t->prefix[id];
    for (int l = 0; l < t->lev[id]; l++) {
        uint32_t o = (uint32_t)((p >> (3 * l)) & 7u);
        c[0] |= ((o >> 2) & 1u) << l;
        c[1] |= ((o >> 1) & 1u) << l;
        c[2] |= (o & 1u) << l;
    }
}

/* Monopole (Sect. 2.2: centre of mass and total mass of each node) and size
 * b_J for the MAC (Eq. 2).  READING for b_J: an upper bound on the distance
 * from the centre of mass to any member particle -- exact (the maximum) for
 * leaves, for internal nodes the smaller of max_c(|com_c - com| + b_c) and
 * the distance from com to the farthest corner of the node's cell, the cell
 * being widened by one finest-level cell width on every side to cover the
 * FP32 quantisation. */
static void node_moments(oracle_tree *t, int refit)
{
    for (int64_t id = t->nn - 1; id >= 0; id--) {
        double M = 0, sx = 0, sy = 0, sz = 0;
        for (int64_t k = t->first[id]; k < t->first[id] + t->count[id]; k++) {
            int64_t p = t->order[k];
            M += t->m[p];
            sx += t->m[p] * t->x[p];
            sy += t->m[p] * t->y[p];
            sz += t->m[p] * t->z[p];
        }
        uint32_t c[3];
        node_cell(t, id, c);
        double side = (double)t->cube[3] / (double)(1u << t->lev[id]);
        double pad = (double)t->cube[3] / (double)(1u << t->levels);
        double lo[3], hi[3];
        for (int a = 0; a < 3; a++) {
            lo[a] = (double)t->cube[a] + (double)c[a] * side - pad;
            hi[a] = (double)t->cube[a] + (double)(c[a] + 1) * side + pad;
        }
        double com[3];
        if (M > 0) {
            com[0] = sx / M; com[1] = sy / M; com[2] = sz / M;
        } else { /* massless node: use the cell centre */
            for (int a = 0; a < 3; a++) com[a] = 0.5 * (lo[a] + hi[a]);
        }
        t->M[id] = M;
        t->cx[id] = com[0]; t->cy[id] = com[1]; t->cz[id] = com[2];
        /* quadrupole (an extension beyond the paper's monopoles): the
         * traceless tensor Q_ab = sum_k m_k (3 s_a s_b - |s|^2 delta_ab) of the
         * members' offsets s from the centre of mass */
        double q6[6] = {0, 0, 0, 0, 0, 0};
        for (int64_t k = t->first[id]; k < t->first[id] + t->count[id]; k++) {
            int64_t p = t->order[k];
            double sx_ = t->x[p] - com[0], sy_ = t->y[p] - com[1], sz_ = t->z[p] - com[2];
            double r2_ = sx_ * sx_ + sy_ * sy_ + sz_ * sz_, mk = t->m[p];
            q6[0] += mk * (3 * sx_ * sx_ - r2_);
            q6[1] += mk * (3 * sy_ * sy_ - r2_);
            q6[2] += mk * (3 * sz_ * sz_ - r2_);
            q6[3] += mk * 3 * sx_ * sy_;
            q6[4] += mk * 3 * sx_ * sz_;
            q6[5] += mk * 3 * sy_ * sz_;
        }
        memcpy(t->Q + 6 * id, q6, sizeof q6);
        double bb;
        if (t->nchild[id] == 0) {
            bb = 0;
            for (int64_t k = t->first[id]; k < t->first[id] + t->count[id]; k++) {
                int64_t p = t->order[k];
                double dx = t->x[p] - com[0], dy = t->y[p] - com[1], dz = t->z[p] - com[2];
                double d = sqrt(dx * dx + dy * dy + dz * dz);
                if (d > bb) bb = d;
            }
        } else {
            double rec = 0;
            for (int64_t ch = t->child[id]; ch < t->child[id] + t->nchild[id]; ch++) {
                double dx = t->cx[ch] - com[0], dy = t->cy[ch] - com[1], dz = t->cz[ch] - com[2];
                double d = sqrt(dx * dx + dy * dy + dz * dz) + t->b[ch];
                if (d > rec) rec = d;
            }
            double c2 = 0;
            for (int a = 0; a < 3; a++) {
                double e = fmax(com[a] - lo[a], hi[a] - com[a]);
                c2 += e * e;
            }
            double corner = sqrt(c2);
            /* after a refit members may have left the cell: the recurrence
             * alone still bounds every member's distance */
            bb = (refit || rec < corner) ? rec : corner;
        }
        t->b[id] = bb;
    }
}

oracle_tree *oracle_tree_build(int64_t n, const double *x, const double *y, const double *z,
                               const double *m, int levels, int leaf_cap)
{
    if (n <= 0 || levels < 1 || levels > 21 || leaf_cap < 1) return NULL;
    oracle_tree *t = (oracle_tree *)calloc(1, sizeof *t);
    if (!t) return NULL;
    t->n = n;
    t->levels = levels;
    t->leaf_cap = leaf_cap;
    size_t nd = (size_t)n * sizeof(double);
    t->x = malloc(nd); t->y = malloc(nd); t->z = malloc(nd); t->m = malloc(nd);
    float *fx = malloc((size_t)n * sizeof(float)), *fy = malloc((size_t)n * sizeof(float)),
          *fz = malloc((size_t)n * sizeof(float));
    for (int a = 0; a < 3; a++) t->q[a] = malloc((size_t)n * sizeof(uint32_t));
    t->key = malloc((size_t)n * sizeof(uint64_t));
    t->order = malloc((size_t)n * sizeof(int64_t));
    int64_t *tmp = malloc((size_t)n * sizeof(int64_t));
    int ok = t->x && t->y && t->z && t->m && fx && fy && fz && t->q[0] && t->q[1] && t->q[2] &&
             t->key && t->order && tmp;
    if (ok) {
        memcpy(t->x, x, nd); memcpy(t->y, y, nd); memcpy(t->z, z, nd); memcpy(t->m, m, nd);
        for (int64_t i = 0; i < n; i++) {
            fx[i] = (float)x[i]; fy[i] = (float)y[i]; fz[i] = (float)z[i];
            t->order[i] = i;
        }
        oracle_cube(n, fx, fy, fz, t->cube);
        oracle_cells(n, fx, fy, fz, t->cube, levels, t->q[0], t->q[1], t->q[2]);
        for (int64_t i = 0; i < n; i++)
            t->key[i] = oracle_interleave(t->q[0][i], t->q[1][i], t->q[2][i], levels);
        int64_t root = new_node(t);
        ok = root == 0 && build_rec(t, root, 0, 0, 0, n, tmp);
        if (ok) node_moments(t, 0);
    }
    free(fx); free(fy); free(fz); free(tmp);
    if (!ok) {
        oracle_tree_free(t);
        return NULL;
    }
    return t;
}

/* Refit: the tree kept between rebuilds (the paper's code rebuilds its tree
 * only every few steps while the node moments, "calcNode", are recomputed
 * every step; Sect. 1 and Sect. 4.1).  Node membership, tree order and
 * groups stay as built; the positions are replaced and the moments
 * recomputed.  READING for b_J after a refit: members may have left their
 * node's cell, so the cell-corner bound is dropped -- leaves take the exact
 * largest member distance, internal nodes max_c(|com_c - com| + b_c). */
void oracle_tree_refit(oracle_tree *t, const double *x, const double *y, const double *z)
{
    size_t nd = (size_t)t->n * sizeof(double);
    memcpy(t->x, x, nd);
    memcpy(t->y, y, nd);
    memcpy(t->z, z, nd);
    node_moments(t, 1);
}

void oracle_tree_free(oracle_tree *t)
{
    if (!t) return;
    free(t->x); free(t->y); free(t->z); free(t->m);
    free(t->q[0]); free(t->q[1]); free(t->q[2]);
    free(t->key); free(t->order);
    free(t->lev); free(t->nchild); free(t->first); free(t->count); free(t->child);
    free(t->prefix); free(t->cx); free(t->cy); free(t->cz); free(t->M); free(t->b);
    free(t->Q);
    free(t);
}

int64_t oracle_tree_nnodes(const oracle_tree *t) { return t->nn; }

void oracle_tree_cube(const oracle_tree *t, float cube[4]) { memcpy(cube, t->cube, sizeof t->cube); }

void oracle_tree_nodes(const oracle_tree *t, int32_t *level, uint64_t *prefix,
                       int64_t *first, int64_t *count, int32_t *nchild, int64_t *child,
                       double *cx, double *cy, double *cz, double *M, double *b)
{
    for (int64_t i = 0; i < t->nn; i++) {
        if (level) level[i] = t->lev[i];
        if (prefix) prefix[i] = t->prefix[i];
        if (first) first[i] = t->first[i];
        if (count) count[i] = t->count[i];
        if (nchild) nchild[i] = t->nchild[i];
        if (child) child[i] = t->child[i];
        if (cx) cx[i] = t->cx[i];
        if (cy) cy[i] = t->cy[i];
        if (cz) cz[i] = t->cz[i];
        if (M) M[i] = t->M[i];
        if (b) b[i] = t->b[i];
    }
}

void oracle_tree_quadrupoles(const oracle_tree *t, double *q6)
{
    memcpy(q6, t->Q, (size_t)t->nn * 6 * sizeof(double));
}

void oracle_tree_order(const oracle_tree *t, int64_t *order)
{
    memcpy(order, t->order, (size_t)t->n * sizeof(int64_t));
}

/* ------------------------------------------------------------------------ */
/* Groups of particles sharing one interaction list (Sect. 1: 32 threads of a
 * warp share a list).  READING: under a node holding more than group_size
 * particles, consecutive children (octant order) that each hold at most
 * group_size are packed into runs of at most group_size particles, one group
 * per run; children holding more are grouped recursively.  A root holding at
 * most group_size is one group; a finest-level leaf holding more is cut into
 * chunks. */
static int64_t add_group(int64_t ng, int64_t f, int64_t c, int64_t *first, int64_t *count)
{
    if (first) { first[ng] = f; count[ng] = c; }
    return ng + 1;
}

static int64_t groups_rec(const oracle_tree *t, int64_t id, int G, int64_t ng,
                          int64_t *first, int64_t *count)
{
    if (t->count[id] <= G) return add_group(ng, t->first[id], t->count[id], first, count);
    if (t->nchild[id] == 0) {
        for (int64_t s = 0; s < t->count[id]; s += G)
            ng = add_group(ng, t->first[id] + s, (t->count[id] - s < G) ? t->count[id] - s : G,
                           first, count);
        return ng;
    }
    int64_t run_first = -1, run_count = 0;
    for (int64_t c = t->child[id]; c < t->child[id] + t->nchild[id]; c++) {
        if (t->count[c] > G) {
            if (run_count) ng = add_group(ng, run_first, run_count, first, count);
            run_count = 0;
            ng = groups_rec(t, c, G, ng, first, count);
        } else if (run_count && run_count + t->count[c] <= G) {
            run_count += t->count[c];
        } else {
            if (run_count) ng = add_group(ng, run_first, run_count, first, count);
            run_first = t->first[c];
            run_count = t->count[c];
        }
    }
    if (run_count) ng = add_group(ng, run_first, run_count, first, count);
    return ng;
}

int64_t oracle_tree_groups(const oracle_tree *t, int group_size, int64_t *first, int64_t *count)
{
    return groups_rec(t, 0, group_size, 0, first, count);
}

/* ------------------------------------------------------------------------ */
/* Eq. 2, the acceleration MAC:  G M_J / d^2 (b_J / d)^2 <= dacc |a_old|,
 * evaluated as G M_J b_J^2 <= dacc |a_old| d^4 (accept on equality), plus the
 * READING that a node is accepted only if d > b_J (it cannot contain the
 * target).  Geometric variant: b_J <= theta d, also with d > b_J. */
static inline int mac_accept(int geometric, double d, double bJ, double MJ, double G,
                             double dacc, double amin, double theta)
{
    if (!(d > bJ)) return 0;
    if (geometric) return bJ <= theta * d;
    double d2 = d * d;
    return G * MJ * bJ * bJ <= dacc * amin * d2 * d2;
}

typedef struct {
    const oracle_tree *t;
    int geometric, quad;
    double G, e2, dacc, theta;
} walk_ctx;

/* Walk for the particles tree-order[k0 .. k0+cnt) sharing one list.  The MAC
 * uses the group sphere (c, r) and amin; for particle mode cnt = 1, r = 0. */
static void walk_list(const walk_ctx *w, int64_t k0, int64_t cnt, const double c[3], double r,
                      double amin, double *acc /* 4*cnt */, int64_t *nint /* cnt */,
                      int64_t *stack)
{
    const oracle_tree *t = w->t;
    int64_t sp = 0;
    stack[sp++] = 0;
    while (sp) {
        int64_t J = stack[--sp];
        double dx = t->cx[J] - c[0], dy = t->cy[J] - c[1], dz = t->cz[J] - c[2];
        double d = sqrt(dx * dx + dy * dy + dz * dz) - r;
        if (mac_accept(w->geometric, d, t->b[J], t->M[J], w->G, w->dacc, amin, w->theta)) {
            /* the node's pseudo particle enters every member's list */
            for (int64_t k = 0; k < cnt; k++) {
                int64_t i = t->order[k0 + k];
                if (w->quad)
                    quad_term(t->cx[J] - t->x[i], t->cy[J] - t->y[i], t->cz[J] - t->z[i], t->M[J],
                              t->Q + 6 * J, w->e2, acc + 4 * k);
                else
                    kernel_term(t->cx[J] - t->x[i], t->cy[J] - t->y[i], t->cz[J] - t->z[i],
                                t->M[J], w->e2, acc + 4 * k);
                nint[k]++;
            }
        } else if (t->nchild[J] == 0) {
            for (int64_t k = 0; k < cnt; k++) {
                int64_t i = t->order[k0 + k];
                for (int64_t q = t->first[J]; q < t->first[J] + t->count[J]; q++) {
                    int64_t j = t->order[q];
                    nint[k]++;
                    if (j == i) continue; /* j != i in Eq. 1 */
                    kernel_term(t->x[j] - t->x[i], t->y[j] - t->y[i], t->z[j] - t->z[i], t->m[j],
                                w->e2, acc + 4 * k);
                }
            }
        } else {
            /* push children in reverse so they are visited in octant order */
            for (int64_t ch = t->child[J] + t->nchild[J] - 1; ch >= t->child[J]; ch--)
                stack[sp++] = ch;
        }
    }
}

static void tree_walk_impl(const oracle_tree *t, int mode, double G, double eps,
                           double delta_acc, double theta, int group_size, const double *a_old,
                           int64_t nsel, const int64_t *sel,
                           double *ax, double *ay, double *az, double *phi, int64_t *ninter)
{
    const int quad = (mode & ORACLE_QUADRUPOLE) != 0;
    mode &= ~ORACLE_QUADRUPOLE;
    walk_ctx w = {t, mode == ORACLE_MAC_PARTICLE_GEO || mode == ORACLE_MAC_GROUP_GEO, quad, G,
                  eps * eps, delta_acc, theta};
    int group_mode = (mode == ORACLE_MAC_GROUP_ACC || mode == ORACLE_MAC_GROUP_GEO);
    int64_t ng;
    int64_t *gf = NULL, *gc = NULL;
    if (group_mode) {
        gf = malloc((size_t)t->n * sizeof(int64_t));
        gc = malloc((size_t)t->n * sizeof(int64_t));
        ng = oracle_tree_groups(t, group_size, gf, gc);
    } else {
        ng = t->n;
    }
    int64_t stack_cap = 8 * (int64_t)(t->levels + 2) + 8;
    int64_t nwork = sel ? nsel : ng;
#pragma omp parallel
    {
        int64_t cmax = group_mode ? group_size : 1;
        double *acc = malloc((size_t)(4 * cmax) * sizeof(double));
        int64_t *nint = malloc((size_t)cmax * sizeof(int64_t));
        int64_t *stack = malloc((size_t)stack_cap * sizeof(int64_t));
#pragma omp for schedule(dynamic, 16)
        for (int64_t w_ = 0; w_ < nwork; w_++) {
            int64_t g = sel ? sel[w_] : w_;
            if (g < 0 || g >= ng) continue;
            int64_t k0 = group_mode ? gf[g] : g, cnt = group_mode ? gc[g] : 1;
            double c[3], r = 0, amin = INFINITY;
            if (group_mode) {
                double lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
                for (int64_t k = 0; k < cnt; k++) {
                    int64_t i = t->order[k0 + k];
                    double p[3] = {t->x[i], t->y[i], t->z[i]};
                    for (int a = 0; a < 3; a++) {
                        if (p[a] < lo[a]) lo[a] = p[a];
                        if (p[a] > hi[a]) hi[a] = p[a];
                    }
                }
                for (int a = 0; a < 3; a++) c[a] = 0.5 * (lo[a] + hi[a]);
                for (int64_t k = 0; k < cnt; k++) {
                    int64_t i = t->order[k0 + k];
                    double dx = t->x[i] - c[0], dy = t->y[i] - c[1], dz = t->z[i] - c[2];
                    double d = sqrt(dx * dx + dy * dy + dz * dz);
                    if (d > r) r = d;
                    if (a_old && a_old[i] < amin) amin = a_old[i];
                }
            } else {
                int64_t i = t->order[g];
                c[0] = t->x[i]; c[1] = t->y[i]; c[2] = t->z[i];
                amin = a_old ? a_old[i] : 0.0;
            }
            if (!a_old) amin = 0.0;
            memset(acc, 0, (size_t)(4 * cnt) * sizeof(double));
            memset(nint, 0, (size_t)cnt * sizeof(int64_t));
            walk_list(&w, k0, cnt, c, r, amin, acc, nint, stack);
            for (int64_t k = 0; k < cnt; k++) {
                int64_t i = t->order[k0 + k];
                ax[i] = G * acc[4 * k + 0];
                ay[i] = G * acc[4 * k + 1];
                az[i] = G * acc[4 * k + 2];
                if (phi) phi[i] = G * acc[4 * k + 3];
                if (ninter) ninter[i] = nint[k];
            }
        }
        free(acc); free(nint); free(stack);
    }
    free(gf);
    free(gc);
}

void oracle_tree_walk(const oracle_tree *t, int mode, double G, double eps,
                      double delta_acc, double theta, int group_size, const double *a_old,
                      double *ax, double *ay, double *az, double *phi, int64_t *ninter)
{
    tree_walk_impl(t, mode, G, eps, delta_acc, theta, group_size, a_old, 0, NULL,
                   ax, ay, az, phi, ninter);
}

void oracle_tree_walk_groups(const oracle_tree *t, int mode, double G, double eps,
                             double delta_acc, double theta, int group_size, const double *a_old,
                             int64_t nsel, const int64_t *sel,
                             double *ax, double *ay, double *az, double *phi, int64_t *ninter)
{
    tree_walk_impl(t, mode, G, eps, delta_acc, theta, group_size, a_old, nsel, sel,
                   ax, ay, az, phi, ninter);
}

/* ------------------------------------------------------------------------ */
void oracle_kick(int64_t n, double *vx, double *vy, double *vz,
                 const double *ax, const double *ay, const double *az, double h)
{
    for (int64_t i = 0; i < n; i++) {
        vx[i] += ax[i] * h;
        vy[i] += ay[i] * h;
        vz[i] += az[i] * h;
    }
}

void oracle_drift(int64_t n, double *x, double *y, double *z,
                  const double *vx, const double *vy, const double *vz, double h)
{
    for (int64_t i = 0; i < n; i++) {
        x[i] += vx[i] * h;
        y[i] += vy[i] * h;
        z[i] += vz[i] * h;
    }
}

void oracle_diagnostics(int64_t n, const double *x, const double *y, const double *z,
                        const double *vx, const double *vy, const double *vz,
                        const double *m, const double *phi, double out[8])
{
    double s[8] = {0};
    for (int64_t i = 0; i < n; i++) {
        s[0] += 0.5 * m[i] * (vx[i] * vx[i] + vy[i] * vy[i] + vz[i] * vz[i]);
        if (phi) s[1] += 0.5 * m[i] * phi[i];
        s[2] += m[i] * vx[i];
        s[3] += m[i] * vy[i];
        s[4] += m[i] * vz[i];
        s[5] += m[i] * (y[i] * vz[i] - z[i] * vy[i]);
        s[6] += m[i] * (z[i] * vx[i] - x[i] * vz[i]);
        s[7] += m[i] * (x[i] * vy[i] - y[i] * vx[i]);
    }
    memcpy(out, s, sizeof s);
}

/* ------------------------------------------------------------------------ */
/* Cost-model MLP, 8 -> 32 -> 32 -> 1 with ReLU, mean-squared error.  Plain
 * FP64 forward pass and backpropagation (chain rule written out), for the
 * gradient checks of the GPU kernels.  Parameter vector: W1[8][32], b1[32],
 * W2[32][32], b2[32], W3[32], b3. */
#define MLP_IN 8
#define MLP_H 32
#define MLP_P (MLP_IN * MLP_H + MLP_H + MLP_H * MLP_H + MLP_H + MLP_H + 1)

int oracle_mlp_params(void) { return MLP_P; }

void oracle_mlp_eval(int64_t n, const double *feat, const double *target, const double *w,
                     const double *norm, double *pred, double *grad, double *loss)
{
    const double *W1 = w, *b1 = W1 + MLP_IN * MLP_H, *W2 = b1 + MLP_H, *b2 = W2 + MLP_H * MLP_H;
    const double *W3 = b2 + MLP_H, *b3 = W3 + MLP_H;
    double *gW1 = grad, *gb1 = gW1 ? gW1 + MLP_IN * MLP_H : NULL, *gW2 = gb1 ? gb1 + MLP_H : NULL;
    double *gb2 = gW2 ? gW2 + MLP_H * MLP_H : NULL, *gW3 = gb2 ? gb2 + MLP_H : NULL;
    double *gb3 = gW3 ? gW3 + MLP_H : NULL;
    if (grad) memset(grad, 0, MLP_P * sizeof(double));
    double L = 0;
    for (int64_t s = 0; s < n; s++) {
        double x[MLP_IN], h1[MLP_H], h2[MLP_H];
        for (int i = 0; i < MLP_IN; i++)
            x[i] = norm ? (feat[s * MLP_IN + i] - norm[i]) / norm[MLP_IN + i] : feat[s * MLP_IN + i];
        for (int j = 0; j < MLP_H; j++) {
            double a = b1[j];
            for (int i = 0; i < MLP_IN; i++) a += x[i] * W1[i * MLP_H + j];
            h1[j] = a > 0 ? a : 0;
        }
        for (int k = 0; k < MLP_H; k++) {
            double a = b2[k];
            for (int j = 0; j < MLP_H; j++) a += h1[j] * W2[j * MLP_H + k];
            h2[k] = a > 0 ? a : 0;
        }
        double y = b3[0];
        for (int k = 0; k < MLP_H; k++) y += h2[k] * W3[k];
        if (pred) pred[s] = y;
        double e = y - target[s];
        L += e * e / (double)n;
        if (!grad) continue;
        double dy = 2.0 * e / (double)n, d2[MLP_H], d1[MLP_H];
        gb3[0] += dy;
        for (int k = 0; k < MLP_H; k++) {
            gW3[k] += dy * h2[k];
            d2[k] = h2[k] > 0 ? dy * W3[k] : 0;
            gb2[k] += d2[k];
        }
        for (int j = 0; j < MLP_H; j++) {
            double a = 0;
            for (int k = 0; k < MLP_H; k++) {
                gW2[j * MLP_H + k] += h1[j] * d2[k];
                a += d2[k] * W2[j * MLP_H + k];
            }
            d1[j] = h1[j] > 0 ? a : 0;
            gb1[j] += d1[j];
        }
        for (int i = 0; i < MLP_IN; i++)
            for (int j = 0; j < MLP_H; j++) gW1[i * MLP_H + j] += x[i] * d1[j];
    }
    if (loss) *loss = L;
}
