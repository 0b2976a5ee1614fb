/*
 * nbody.h -- C ABI of libnbody.so, a GB300 (sm_103a) implementation of the
 * gravitational octree force calculation of Y. Miki, "Gravitational octree
 * code performance evaluation on Volta GPU" (arXiv:1811.02761).
 *
 * The library computes, per step:
 *   - the softened Newtonian acceleration of Eq. 1
 *       a_i = sum_{j != i} G m_j (r_j - r_i) / (|r_j - r_i|^2 + eps^2)^{3/2}
 *     either by direct summation or by the Barnes-Hut tree method (Sect. 1);
 *   - the tree from radix-sorted space-filling-curve (Morton) keys (Sect. 4.1,
 *     "makeTree"), node centres of mass and masses ("calcNode", Sect. 2.2),
 *   - a tree walk in which groups of particles share one interaction list
 *     (Sect. 1) and distant nodes are accepted by the acceleration MAC of Eq. 2
 *       G m_J / d^2 (b_J / d)^2 <= delta_acc |a_i^old|,
 *   - leapfrog kick-drift-kick orbit integration (the paper's code uses a
 *     second-order Runge-Kutta scheme; this library integrates with leapfrog),
 *     with one shared step or block (hierarchical) steps (Sect. 1), the tree
 *     rebuilt every step or refitted between rebuilds at an interval that can
 *     be tuned by timing (Sect. 1 and 4.1);
 *   - optionally, quadrupole moments for the nodes (an extension beyond the
 *     paper's monopoles), many independent systems in one forest and one
 *     walk, and a learned cost model that orders the walk's queue.
 *
 * Conventions for every entry point
 *   - Pointers may be device pointers or host pointers (pageable or pinned);
 *     the library inspects each with cudaPointerGetAttributes and stages host
 *     data through its own device buffers.  Device pointers are used in place,
 *     and so are page-locked host arrays of nbody_step(_batched), whose state
 *     is read once by one kernel and written back once by another.
 *   - Arrays are structure-of-arrays, length n, in the caller's particle
 *     order; the library's internal Morton order never leaks out.
 *   - Every call returns an nbody_status; no C++ exception crosses the ABI.
 *     Argument errors are detected before any launch.  Device-side errors
 *     (traversal stack overflow, an index that failed a bounds check, a
 *     bounded device wait that ran out) are reported through a device status
 *     word that the call reads after synchronising its stream.
 *   - All work of a context is enqueued on the stream given at creation
 *     (NULL = the legacy default stream).  A context is not thread-safe.
 *   - Calls that return results synchronise the context's stream before
 *     returning, so outputs are complete when the call returns.
 *   - Ownership: the caller owns every array it passes.  The context owns all
 *     scratch (keys, tree, groups, interaction lists); it grows on demand with
 *     cudaMalloc and is released by nbody_destroy.
 */
#ifndef NBODY_H
#define NBODY_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define NBODY_ABI_VERSION 2

typedef enum {
    NBODY_OK = 0,
    NBODY_EINVAL = 1,    /* bad argument (n < 0, NULL, eps < 0, bad config)  */
    NBODY_ENOMEM = 2,    /* device or host allocation failed                 */
    NBODY_EOVERFLOW = 3, /* a traversal stack overflowed; results invalid    */
    NBODY_ETIMEOUT = 4,  /* a bounded device wait ran out; results invalid  */
    NBODY_ECUDA = 5,     /* a CUDA runtime call failed (see nbody_last_error)*/
    NBODY_ENOTBUILT = 6  /* nbody_walk before nbody_build                    */
} nbody_status;

/* Scheduling of the persistent walk's group queue. */
typedef enum {
    NBODY_SCHED_MORTON = 0,   /* groups in Morton order                       */
    NBODY_SCHED_MLP = 1,      /* descending cost predicted by the MLP         */
    NBODY_SCHED_LASTCOST = 2  /* descending cost measured in the previous walk*/
} nbody_schedule;

/* Parameters.  Fill with nbody_config_default() and then override. */
typedef struct {
    float G;             /* gravitational constant of Eq. 1 (default 1)             */
    float eps;           /* Plummer softening eps of Eq. 1, >= 0 (default 1/64)       */
    float delta_acc;     /* delta_acc of Eq. 2, >= 0 (default 2^-9)                  */
    float theta;         /* opening angle of the bootstrap geometric MAC used when
                            no |a_old| is given, 0 < theta < 1 (default 0.5)        */
    int32_t leaf_cap;    /* max particles in a leaf, 1..32 (default 16)             */
    int32_t group_size;  /* max particles sharing one list, leaf_cap..32*ipl (64)   */
    int32_t ipl;         /* most i-particles a lane of a walking warp holds, 1..4;
                            slot j of a lane covers 2^k members of a group and
                            cuts the list 32 / 2^k ways, the 2^k the fewest powers
                            of two covering the group (3)                         */
    int32_t list_depth;  /* interaction-list entries per warp, 64..1024, multiple
                            of 32 (default 256)                                    */
    int32_t stack_depth; /* traversal stack entries per warp, 64..4096 (256)        */
    int32_t warps_per_block; /* walk warps per CTA, 1..16 (default 4)             */
    int32_t compensated; /* 1: per-flush partial sums added with Neumaier
                            compensation; 0: plain FP32 sums; 2 (default): automatic,
                            compensated where the MAC is tight (delta_acc <= 2^-18,
                            where plain FP32 sums start to add measurably to the
                            force error)                                           */
    int32_t want_potential; /* 1: also accumulate phi (default 0)                 */
    int32_t schedule;    /* nbody_schedule (default NBODY_SCHED_MORTON)             */
    int32_t use_graph;   /* 1: nbody_step(_batched) replays a CUDA graph of two
                            steps (captured on first use, on an internal stream
                            ordered after cuda_stream; only with
                            rebuild_interval = 1); 0: eager launches (0)     */
    int32_t rebuild_interval; /* tree rebuilds in nbody_step(_batched): 1 = every
                            step (default); k >= 2 = every k-th step of a call,
                            the steps between refit the tree (nbody_refit:
                            moments and group spheres at the new positions,
                            structure kept); 0 = automatic: rebuild when the
                            last step cost more than the mean step of the cycle
                            since the last rebuild (nbody_rebuild_due; the
                            paper's code tunes its rebuild interval by timing,
                            Sect. 1 and 4.1), at most every 32 steps; this
                            synchronises the stream after every step.  The
                            first step of every call rebuilds.  0..1024.     */
    int32_t quadrupole;  /* 1: nodes also carry their traceless quadrupole
                            Q_ab = sum m (3 s_a s_b - |s|^2 delta_ab) about the
                            centre of mass, and an accepted node contributes
                            M d/r^3 - Q d/r^5 + 5/2 (d.Q.d) d/r^7 (r^2 = |d|^2 +
                            eps^2; an extension beyond the paper's monopoles,
                            same MAC); 0: monopoles (default)                */
    int32_t block_levels; /* block (hierarchical) time steps in nbody_step(_batched):
                            0 = one shared step dt (default); K = 1..20: each
                            particle steps by dt / 2^k on level k <= K, chosen
                            from dt_i = sqrt(2 block_eta eps / |a_i|) (the paper's
                            code uses block steps, Sect. 1; this criterion is
                            a reading); only groups with a particle whose step
                            ends at a tick are walked.  nsteps counts steps of
                            dt; the state returned is synchronised.  Not with
                            use_graph; the stream is synchronised after every
                            processed tick.                                 */
    float block_eta;     /* accuracy parameter of the block step criterion
                            (default 0.025), > 0                             */
    int32_t walk_pipeline; /* 1: the walk runs in warp pairs, one warp
                            traversing the tree and handing interaction lists
                            through shared memory to one warp evaluating Eq. 1
                            (monopole walks without the potential; identical
                            results); needs an even warps_per_block.  0: each
                            warp traverses and evaluates (default)          */
} nbody_config;

typedef struct {
    int64_t n_nodes;       /* nodes of the last build                        */
    int64_t n_groups;      /* i-groups of the last walk                      */
    int64_t interactions;  /* kernel evaluations of the last walk (the zero
                              self term of each particle included)            */
    int64_t list_entries;  /* interaction-list entries flushed (sum over groups) */
    int32_t max_stack;     /* deepest traversal stack seen                   */
    int32_t levels;        /* tree levels below the root                     */
    int64_t kernels;       /* kernels this library launched in the last call  */
    float ms_build;        /* device time of the build phase(s) (CUDA events)  */
    float ms_walk;         /* device time of the walk phase(s) (CUDA events)   */
    float ms_walk_kernel;  /* device time of the walk kernel launches alone: the
                              eager steps' launches and, when nbody_step
                              replayed a CUDA graph, the last replay's two
                              (event nodes in the graph)                      */
    int32_t walk_launches; /* walk kernel launches behind ms_walk_kernel       */
    int32_t rebuilds;      /* steps of the last nbody_step call that rebuilt the
                              tree (the others refitted it)                    */
    int64_t quad_interactions; /* of `interactions`, those with quadrupole
                              nodes (quadrupole = 1)                          */
    int32_t walk_warps;    /* resident walk warps (queue consumers) of the last
                              walk launch                                      */
} nbody_stats;

typedef struct nbody_ctx nbody_ctx;

/* Version of this ABI (NBODY_ABI_VERSION). */
int32_t nbody_abi_version(void);

/* Default parameters (values listed in nbody_config). */
void nbody_config_default(nbody_config *cfg);

/* Create a context on the current device.  cuda_stream is a cudaStream_t
 * (NULL for the default stream); the caller keeps it alive until destroy.
 * Errors: EINVAL (cfg invalid or out NULL), ECUDA. */
nbody_status nbody_create(nbody_ctx **out, const nbody_config *cfg, void *cuda_stream);

/* Release every buffer of the context.  NULL is accepted. */
nbody_status nbody_destroy(nbody_ctx *ctx);

/* Replace the parameters (e.g. after autotuning); the next build or walk
 * uses them.  Errors: EINVAL. */
nbody_status nbody_set_config(nbody_ctx *ctx, const nbody_config *cfg);
nbody_status nbody_get_config(const nbody_ctx *ctx, nbody_config *cfg);

/* Build the octree of one system (Sect. 4.1 "makeTree" + Sect. 2.2
 * "calcNode"): bounding cube, 63-bit Morton keys (21 bits per axis, FP32
 * quantisation), stable LSD radix sort, level-ordered octree with leaves of
 * at most leaf_cap particles, bottom-up monopoles and node sizes b_J.
 * x, y, z, m: FP32 [n], n >= 1.  The context keeps its own sorted copy.
 * Errors: EINVAL, ENOMEM, ECUDA. */
nbody_status nbody_build(nbody_ctx *ctx, int64_t n, const float *x, const float *y,
                         const float *z, const float *m);

/* Build a forest of nsys independent systems in one pass: system s holds
 * particles offsets[s] .. offsets[s+1]-1 (offsets: HOST int64 [nsys+1],
 * offsets[0] = 0, non-decreasing).  eps_sys: HOST float [nsys], the
 * softening of each system (NULL: cfg.eps for all).  Keys carry the system id
 * above the Morton bits, so one sort orders all systems; each system has its
 * own cube and root.  1 <= nsys <= 2^20.  Errors: EINVAL, ENOMEM, ECUDA. */
nbody_status nbody_build_batched(nbody_ctx *ctx, int32_t nsys, const int64_t *offsets,
                                 const float *eps_sys, const float *x, const float *y,
                                 const float *z, const float *m);

/* Refit the tree of the last build to new positions of the same particles
 * (caller order, FP32 [n], host or device): the node structure, tree order
 * and groups are kept; node monopoles, sizes b_J (from the child recurrence
 * only, as members may have left their cells) and group spheres are
 * recomputed -- the paper's calcNode without makeTree (its code rebuilds the
 * tree only every few steps, Sect. 1 and 4.1).  m must be the masses of the
 * build.  Errors: ENOTBUILT, EINVAL, ECUDA. */
nbody_status nbody_refit(nbody_ctx *ctx, const float *x, const float *y, const float *z,
                         const float *m);

/* Policy of rebuild_interval = 0: cost_ms[0] is the step that rebuilt the
 * tree, cost_ms[1..m-1] the refitted steps since (tree phase + walk, device
 * time).  Returns 1 when the last step cost more than the mean of the m steps
 * (continuing to refit would raise the mean cost per step), else 0; m < 2
 * returns 0.  Host-only, needs no device. */
int32_t nbody_rebuild_due(const float *cost_ms, int32_t m);

/* Tree accelerations for every particle of the last build (Eq. 1 evaluated
 * over the interaction lists of Sect. 1, nodes accepted by Eq. 2).
 * a_old: FP32 [n], |a_i^old| in caller order, or NULL: then one walk with the
 * geometric criterion b_J <= theta d provides |a| for the acceleration-MAC
 * walk.  Outputs ax, ay, az: FP32 [n]; phi: FP32 [n] or NULL (requires
 * want_potential = 1 in the config).  stats: nullable.
 * Errors: ENOTBUILT, EINVAL, EOVERFLOW (stack_depth too small), ECUDA. */
nbody_status nbody_walk(nbody_ctx *ctx, const float *a_old, float *ax, float *ay, float *az,
                        float *phi, nbody_stats *stats);

/* Eq. 1 by direct O(n^2) summation on the GPU (FP32, rsqrt; compensated = 1
 * adds per-tile partial sums with Neumaier compensation).  Stateless: uses
 * cuda_stream (NULL = default stream) and synchronises it.  phi nullable.
 * Errors: EINVAL, ENOMEM, ECUDA. */
nbody_status nbody_direct(int64_t n, const float *x, const float *y, const float *z,
                          const float *m, float G, float eps, int32_t compensated,
                          float *ax, float *ay, float *az, float *phi, void *cuda_stream);

/* nsteps leapfrog kick-drift-kick steps of length dt with the tree force,
 * the tree rebuilt every step:
 *   v += a dt/2;  x += v dt (FP64 positions);  rebuild;  walk with |a|;
 *   v += a dt/2.
 * x, y, z: FP64 [n]; vx, vy, vz: FP32 [n]; m: FP32 [n];
 * ax, ay, az: FP32 [n], on entry the acceleration at the entry positions (from
 * nbody_walk), on return the acceleration at the final positions.  All arrays
 * are updated in place, in caller order.  Sorting is the stable sort of the
 * Morton keys in caller order (Sect. 4.1); inside a call each rebuild starts
 * from the previous build's order, and a call's first rebuild from the order
 * the context's last call of the same n ended in -- which makes it faster,
 * never different.  Errors: EINVAL, ENOMEM, EOVERFLOW, ECUDA. */
nbody_status nbody_step(nbody_ctx *ctx, int64_t n, double *x, double *y, double *z,
                        float *vx, float *vy, float *vz, const float *m,
                        float *ax, float *ay, float *az, float dt, int32_t nsteps,
                        nbody_stats *stats);

/* nbody_step for nsys independent systems (offsets, eps_sys as in
 * nbody_build_batched): one sort, one forest, one persistent walk over all
 * groups of all systems per step. */
nbody_status nbody_step_batched(nbody_ctx *ctx, int32_t nsys, const int64_t *offsets,
                                const float *eps_sys, double *x, double *y, double *z,
                                float *vx, float *vy, float *vz, const float *m,
                                float *ax, float *ay, float *az, float dt, int32_t nsteps,
                                nbody_stats *stats);

/* FP64 diagnostics over n particles: out (HOST double [8]) = {E_kin, E_pot,
 * Px, Py, Pz, Lx, Ly, Lz} with E_kin = 1/2 sum m v^2, E_pot = 1/2 sum m phi
 * (phi NULL: 0), P = sum m v, L = sum m r x v; FP64 reductions on the device.
 * Errors: EINVAL, ENOMEM, ECUDA. */
nbody_status nbody_diagnostics(nbody_ctx *ctx, int64_t n, const double *x, const double *y,
                               const double *z, const float *vx, const float *vy,
                               const float *vz, const float *m, const float *phi,
                               double *out);

/* nbody_diagnostics without any device allocation (no counterpart in the
 * paper: this serves callers that cannot call cudaMalloc -- for instance
 * when a framework's caching allocator or a fixed arena already reserves the
 * device memory, or when an allocation's implicit device-wide synchronisation
 * is not acceptable inside a time-step loop).
 * Same sums and result as nbody_diagnostics.  x, y, z (FP64), vx, vy, vz, m
 * and phi (FP32, phi nullable) must be DEVICE pointers of n elements; out is
 * 8 doubles, device or host.  Runs on cuda_stream (NULL = default stream)
 * and synchronises it.  Its scratch is a fixed file-scope device array
 * (1024 x 8 + 8 doubles, 65.6 KB per GPU, held until the process exits) that
 * every call shares: calls that overlap on the GPU race on it.  The first
 * call on a device looks up the array's device address; make that first call
 * before any stream capture.  That address is cached for the life of the
 * device's CUDA context: do not use the library across a cudaDeviceReset.
 * n must be in 1..2^31-1 (larger n: EINVAL).  Inputs must be device (or
 * managed) memory of the current device; out may be host memory or device
 * memory of the current device.
 * Errors: EINVAL (bad n, NULL input, host input, or an array on another
 * GPU), ECUDA. */
nbody_status nbody_diagnostics_noalloc(int64_t n, const double *x, const double *y,
                                       const double *z, const float *vx, const float *vy,
                                       const float *vz, const float *m, const float *phi,
                                       double *out, void *cuda_stream);

/* Per-group cost log of the last walk: counts[g] = interaction-list entries
 * group g processed, groups in Morton order.  counts: int32 [cap] (host or
 * device); *n_groups receives the number of groups (may exceed cap: then
 * only cap entries are written).  Errors: ENOTBUILT, EINVAL, ECUDA. */
nbody_status nbody_get_group_costs(nbody_ctx *ctx, int32_t *counts, int64_t cap,
                                   int64_t *n_groups);

/* Autotuner search space (the analogue of the paper's micro-benchmarked
 * thread-block configuration, Sect. 2.2 Table 2).  Each list holds n_*
 * candidates; combinations violating the config rules (leaf_cap <=
 * group_size <= 32 ipl) are skipped, and so are those with group_size <=
 * 8 ipl, whose extra i-slots no lane tiling would use. */
typedef struct {
    int32_t n_leaf_cap, leaf_cap[4];
    int32_t n_group_size, group_size[6];
    int32_t n_ipl, ipl[3];
    int32_t n_list_depth, list_depth[4];
    int32_t n_warps_per_block, warps_per_block[4];
    int32_t repeats;            /* timed walks per candidate (the minimum counts) */
} nbody_tune_space;

/* Default space: leaf_cap {8, 16}, group_size {32, 64, 128}, ipl {2, 3, 4},
 * list_depth {128, 256}, warps_per_block {2, 4, 8}, repeats 2. */
void nbody_tune_space_default(nbody_tune_space *space);

/* Grid search over `space` for the fastest build + walk of the given systems
 * (nsys = 1 and offsets = NULL for one system; arrays as in
 * nbody_build_batched, a_old as in nbody_walk).  Every candidate is timed
 * with CUDA events on the context's stream: build once per (leaf_cap,
 * group_size), walk `repeats` times per (ipl, list_depth, warps_per_block).
 * The context keeps the best configuration; *best receives it, *best_ms its
 * build + walk time and *n_tried the number of timed candidates (all three
 * nullable).  The context's other parameters (G, eps, delta_acc, ...) are
 * kept.  Errors: EINVAL, ENOMEM, EOVERFLOW, ECUDA. */
nbody_status nbody_autotune(nbody_ctx *ctx, int32_t nsys, const int64_t *offsets,
                            const float *eps_sys, const float *x, const float *y,
                            const float *z, const float *m, const float *a_old,
                            const nbody_tune_space *space, nbody_config *best, float *best_ms,
                            int32_t *n_tried);

/* ---------------------------------------------------------------------------
 * Learned cost model ordering the persistent walk's queue (no counterpart in
 * the paper; the scheduling layer around its walk).  An MLP 8 -> 32 -> 32 -> 1
 * (ReLU) predicts log2 of each group's walk cost from 8 group features (log2
 * count, log2 r_g, log2 min|a_old|, log2 distance to the system's centre of
 * mass, cell level, log2 count per cell volume, log2 mean|a_old|, log2 N_sys),
 * standardised with statistics frozen at the first training call.  Forward
 * and backward passes use BF16 weights with FP32 accumulation; Adam keeps FP32
 * master weights.  With schedule = NBODY_SCHED_MLP the walk pops groups in
 * descending predicted cost (times the i-slots a group occupies); the
 * accelerations are identical for every schedule.
 * Parameter vector (NBODY_MLP_PARAMS floats): W1[8][32], b1[32], W2[32][32],
 * b2[32], W3[32], b3 (W[i][j] connects input i to unit j). */
#define NBODY_MLP_PARAMS 1377
#define NBODY_MLP_FEATURES 8

/* Set the parameters (host or device FP32 [NBODY_MLP_PARAMS], e.g. a seeded
 * initialisation); resets the Adam moments and the feature statistics. */
nbody_status nbody_mlp_set_params(nbody_ctx *ctx, const float *params);
/* Current FP32 master parameters (host or device [NBODY_MLP_PARAMS]). */
nbody_status nbody_mlp_get_params(nbody_ctx *ctx, float *params);

/* Train on the groups and costs the last walk logged: `epochs` passes of Adam
 * (learning rate lr) over minibatches of at most `batch` groups (strided
 * through the Morton order), MSE on log2(cost).  *loss (nullable) receives
 * the mean minibatch loss of the last epoch.  Errors: EINVAL (no params, no
 * walk since the last build), ECUDA. */
nbody_status nbody_mlp_train(nbody_ctx *ctx, int32_t epochs, float lr, int32_t batch,
                             float *loss);

/* Predicted log2 cost of every group of the last build (host or device FP32,
 * cap entries); *n_groups receives the group count.  Also copies the groups'
 * features (FP32 [groups][8], nullable).  Errors: EINVAL, ECUDA. */
nbody_status nbody_mlp_predict(nbody_ctx *ctx, float *pred, float *features, int64_t cap,
                               int64_t *n_groups);

/* Stateless forward + MSE loss + gradient for n samples (n <= 2^20):
 * features [n][8] and targets [n] (FP32, host or device), params
 * [NBODY_MLP_PARAMS] (FP32, rounded to BF16 inside, as the training kernels
 * use them), norm [16] (feature means then standard deviations; NULL = none).
 * Outputs (host or device, nullable): pred [n], grad [NBODY_MLP_PARAMS] of the
 * mean loss, loss (one float).  Errors: EINVAL, ENOMEM, ECUDA. */
nbody_status nbody_mlp_eval(int64_t n, const float *features, const float *targets,
                            const float *params, const float *norm, float *pred, float *grad,
                            float *loss, void *cuda_stream);

/* Internal arrays of the last build, for inspection and testing. */
typedef enum {
    NBODY_EXPORT_PERM = 0,         /* int32 [n]: caller index of sorted particle k  */
    NBODY_EXPORT_KEYS = 1,         /* uint64 [n]: sorted Morton keys (system id on
                                      top of 3*levels Morton bits)                  */
    NBODY_EXPORT_NODE_LEVEL = 2,   /* int8 [nodes]                                  */
    NBODY_EXPORT_NODE_START = 3,   /* int32 [nodes]: first sorted particle          */
    NBODY_EXPORT_NODE_COUNT = 4,   /* int32 [nodes]: particles in the node          */
    NBODY_EXPORT_NODE_PARENT = 5,  /* int32 [nodes]: parent, -1 for roots           */
    NBODY_EXPORT_NODE_A = 6,       /* float4 [nodes]: com.x, com.y, com.z, M        */
    NBODY_EXPORT_NODE_B = 7,       /* float4 [nodes]: b_J, G M b_J^2, link, meta    */
    NBODY_EXPORT_GROUP_FIRST = 8,  /* int32 [groups]: first sorted particle         */
    NBODY_EXPORT_GROUP_COUNT = 9,  /* int32 [groups]                                */
    NBODY_EXPORT_GROUP_SPHERE = 10,/* float4 [groups]: centre, radius               */
    NBODY_EXPORT_SYS_BOX = 11,     /* float4 [nsys]: x0, y0, z0, L of each cube     */
    NBODY_EXPORT_NODE_Q = 12       /* float [nodes][8]: quadrupole xx, yy, zz, xy,
                                      xz, yz, 0, 0 (quadrupole = 1 only)         */
} nbody_export_what;

/* Copy internal array `what` of the last build into dst (host or device),
 * at most cap elements; *count receives the array's length.  Nodes are in
 * level-major order (children of a node contiguous).  Errors: ENOTBUILT,
 * EINVAL, ECUDA. */
nbody_status nbody_export(nbody_ctx *ctx, int32_t what, void *dst, int64_t cap, int64_t *count);

/* Stable sort of 64-bit keys: the ordering step of the tree build (Sect.
 * 4.1, particles sorted along the Morton curve), callable on its own so that
 * both of the build's sort paths can be checked on any key set.
 * keys: DEVICE uint64 [n], read only.  keys_out: DEVICE uint64 [n], the keys
 * in ascending order.  perm_out: DEVICE int32 [n], perm_out[k] = the input
 * index of keys_out[k]; equal keys keep their input order.
 * method: NBODY_SORT_RADIX, the one-sweep LSD radix sort over all 64 bits
 * (a build from the caller's order), or NBODY_SORT_NEAR_ORDER, the bucket
 * sort of the builds inside a step (splitters from one key per 1984, a
 * scatter into buckets, a shared-memory merge sort per bucket): fastest on
 * nearly sorted keys, the same result for any input, and the radix sort for
 * n > 16384 * 1984.  Runs on the context's stream with its sort buffers
 * (grown as needed) and synchronises it; the tree of the last build is
 * invalidated.  1 <= n < 2^31.  Errors: EINVAL (n, method, a pointer that is
 * NULL or not memory of the context's device), ENOMEM, ECUDA, ETIMEOUT. */
#define NBODY_SORT_RADIX 0
#define NBODY_SORT_NEAR_ORDER 1
nbody_status nbody_sort_keys(nbody_ctx *ctx, int32_t method, const uint64_t *keys, int64_t n,
                             uint64_t *keys_out, int32_t *perm_out);

/* Self-tests of the library's failure paths (no counterpart in the paper).
 * NBODY_SELFTEST_SORT_WAIT: runs one radix-sort pass kernel on a two-tile
 * input whose first tile is never processed, so the second tile's look-back
 * (the decoupled look-back of the one-sweep sort, the default path's only
 * device wait; the opt-in warp-pair walk's hand-offs are the other, bounded
 * the same way) finds nothing to wait for; the wait is bounded (2^20 polls) and the
 * kernel records a timeout and finishes.  Returns the status the device
 * reported: NBODY_ETIMEOUT when the bound works.  Allocates and frees its own
 * buffers (about 200 KB) and synchronises cuda_stream (NULL = default
 * stream).  The device stays usable afterwards.  Errors: EINVAL (unknown
 * test), ECUDA. */
#define NBODY_SELFTEST_SORT_WAIT 1
nbody_status nbody_selftest(int32_t which, void *cuda_stream);

/* Message of the last error of this context (or of the last stateless call
 * on this thread if ctx is NULL), NUL-terminated, truncated to len. */
nbody_status nbody_last_error(const nbody_ctx *ctx, char *buf, size_t len);

#ifdef __cplusplus
}
#endif
#endif /* NBODY_H */
