/*
 * oracle.h -- plain, slow, FP64 CPU oracle for the gravitational octree method.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the package smoke check and
 * the benchmark's CPU-baseline leg call this code.  The CUDA library never
 * links it, includes it or calls it, and it shares no source with it.
 *
 * What it computes (paper: Y. Miki, "Gravitational octree code performance
 * evaluation on Volta GPU"):
 *   - Eq. 1, softened Newtonian acceleration, by direct summation;
 *   - the Barnes-Hut octree (Sect. 1) built by recursive subdivision of the
 *     bounding cube, with monopole moments (centre of mass, total mass) and the
 *     node size b_J used by the acceleration MAC;
 *   - the tree walk under the acceleration MAC of Eq. 2, per particle or per
 *     group of particles sharing one interaction list (Sect. 1);
 *   - leapfrog kick / drift and FP64 energy / momentum diagnostics.
 *
 * Conventions: positions and masses are passed as FP64 (exact copies of the
 * FP32 inputs); every sum is FP64; particle index i runs 0..n-1 in caller
 * order.  No function keeps a pointer to its arguments after returning,
 * except oracle_tree_build, which copies what it needs.
 */
#ifndef NBODY_ORACLE_H
#define NBODY_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Eq. 1 for every i (j != i skipped explicitly).  phi (nullable) receives
 * phi_i = -G sum_{j != i} m_j / sqrt(r_ij^2 + eps^2). */
void oracle_direct(int64_t n, const double *x, const double *y, const double *z,
                   const double *m, double G, double eps,
                   double *ax, double *ay, double *az, double *phi);

/* Eq. 1 for the nt targets tgt[k] against all n sources. */
void oracle_direct_targets(int64_t n, const double *x, const double *y, const double *z,
                           const double *m, int64_t nt, const int64_t *tgt,
                           double G, double eps,
                           double *ax, double *ay, double *az, double *phi);

/* Bounding cube: cube = {x0, y0, z0, L}, all FP32 arithmetic:
 * (x0,y0,z0) = per-axis minimum, L = max extent * (1 + 2^-20), L = 1 if 0. */
void oracle_cube(int64_t n, const float *x, const float *y, const float *z, float cube[4]);

/* Integer cell coordinates at resolution 2^levels, decided in FP32:
 * q = min(floor((x - x0) * (2^levels / L)), 2^levels - 1). */
void oracle_cells(int64_t n, const float *x, const float *y, const float *z,
                  const float cube[4], int levels,
                  uint32_t *qx, uint32_t *qy, uint32_t *qz);

/* Morton key: bits of (qx, qy, qz) interleaved, x in the top bit of each
 * 3-bit group, most significant level first. */
uint64_t oracle_interleave(uint32_t qx, uint32_t qy, uint32_t qz, int levels);

/* Stable sort of keys: order[k] = index of the k-th smallest (key, index). */
void oracle_sort(int64_t n, const uint64_t *keys, int64_t *order);

/* ------------------------------------------------------------------------ */
typedef struct oracle_tree oracle_tree;

/* Octree by recursive subdivision of the cube of the particles (FP32 cube and
 * cells as above).  A cell is split while it holds more than leaf_cap
 * particles and its level is below `levels`.  Children of a node are stored
 * contiguously in octant order.  Returns NULL on allocation failure. */
oracle_tree *oracle_tree_build(int64_t n, const double *x, const double *y, const double *z,
                               const double *m, int levels, int leaf_cap);
/* Replace the positions of a built tree (same particles, caller order) and
 * recompute its moments without rebuilding: membership, order and groups
 * stay; b_J of internal nodes uses only the child recurrence. */
void oracle_tree_refit(oracle_tree *t, const double *x, const double *y, const double *z);
/* Traceless quadrupole of every node about its centre of mass, 6 doubles per
 * node (xx, yy, zz, xy, xz, yz), Q_ab = sum m (3 s_a s_b - |s|^2 delta_ab). */
void oracle_tree_quadrupoles(const oracle_tree *t, double *q6);
void oracle_tree_free(oracle_tree *t);
int64_t oracle_tree_nnodes(const oracle_tree *t);
void oracle_tree_cube(const oracle_tree *t, float cube[4]);

/* Node arrays (length nnodes).  prefix = the node's cell as a 3*level-bit
 * Morton prefix; child = index of first child (-1 for leaves). */
void oracle_tree_nodes(const oracle_tree *t, int32_t *level, uint64_t *prefix,
                       int64_t *first, int64_t *count, int32_t *nchild, int64_t *child,
                       double *cx, double *cy, double *cz, double *M, double *b);

/* Particle order of the tree (depth-first, octant order, leaves sorted by
 * (key, index)): order[k] = caller index of the k-th particle. */
void oracle_tree_order(const oracle_tree *t, int64_t *order);

/* Groups: largest nodes holding at most group_size particles; a leaf at the
 * finest level with more is cut into consecutive chunks of group_size.
 * Returns the number of groups; if first/count are non-NULL they receive each
 * group's range in tree order (capacity n). */
int64_t oracle_tree_groups(const oracle_tree *t, int group_size, int64_t *first, int64_t *count);

/* Walk modes */
#define ORACLE_MAC_PARTICLE_ACC 0 /* Eq. 2 per particle: d = |com_J - r_i|            */
#define ORACLE_MAC_GROUP_ACC    1 /* Eq. 2 per group:    d = |com_J - c_g| - r_g      */
#define ORACLE_MAC_PARTICLE_GEO 2 /* opening angle b_J <= theta d, per particle       */
#define ORACLE_MAC_GROUP_GEO    3 /* opening angle b_J <= theta d, per group          */
/* Or-ed into a mode: accepted nodes contribute their monopole plus their
 * traceless quadrupole (an extension beyond the paper's monopoles). */
#define ORACLE_QUADRUPOLE      16

/* Tree force for every particle.  a_old (caller order, may be NULL for the
 * geometric modes) holds |a_i^old|.  Outputs in caller order; ninter
 * (nullable) receives the number of kernel evaluations of particle i
 * (accepted nodes + particles of opened leaves, the zero self term included). */
void oracle_tree_walk(const oracle_tree *t, int mode, double G, double eps,
                      double delta_acc, double theta, int group_size, const double *a_old,
                      double *ax, double *ay, double *az, double *phi, int64_t *ninter);

/* As oracle_tree_walk, but only for the groups (group mode) or tree-order
 * particles (particle mode) listed in sel[0..nsel); outputs of other
 * particles are left untouched. */
void oracle_tree_walk_groups(const oracle_tree *t, int mode, double G, double eps,
                             double delta_acc, double theta, int group_size, const double *a_old,
                             int64_t nsel, const int64_t *sel,
                             double *ax, double *ay, double *az, double *phi, int64_t *ninter);

/* ------------------------------------------------------------------------ */
/* Leapfrog pieces: v += a * h ; x += v * h. */
void oracle_kick(int64_t n, double *vx, double *vy, double *vz,
                 const double *ax, const double *ay, const double *az, double h);
void oracle_drift(int64_t n, double *x, double *y, double *z,
                  const double *vx, const double *vy, const double *vz, double h);

/* FP64 diagnostics: out = {E_kin, E_pot, Px, Py, Pz, Lx, Ly, Lz};
 * E_pot = 1/2 sum m_i phi_i (phi may be NULL: E_pot = 0). */
void oracle_diagnostics(int64_t n, const double *x, const double *y, const double *z,
                        const double *vx, const double *vy, const double *vz,
                        const double *m, const double *phi, double out[8]);

/* Cost-model MLP (8 -> 32 -> 32 -> 1, ReLU), FP64: predictions, mean squared
 * error and its gradient for n samples.  feat [n][8], target [n], w
 * [oracle_mlp_params()] = W1[8][32], b1[32], W2[32][32], b2[32], W3[32], b3;
 * norm [16] (means then standard deviations) or NULL.  pred, grad, loss
 * nullable. */
int oracle_mlp_params(void);
void oracle_mlp_eval(int64_t n, const double *feat, const double *target, const double *w,
                     const double *norm, double *pred, double *grad, double *loss);

/* Number of threads OpenMP uses (1 without OpenMP). */
int oracle_threads(void);
/* Threads of the following parallel loops (k < 1: all cores). */
void oracle_set_threads(int k);

#ifdef __cplusplus
}
#endif
#endif
