// internal.cuh -- shared declarations of libnbody (not part of the public ABI).
//
// Data layout in device memory (sorted = Morton order of the last build):
//   particles  pos4[n]   float4 (x, y, z, m), sorted
//              perm[n]   int32, sorted index -> caller index
//              keys[n]   uint64 Morton keys (system id above the Morton bits)
//   boundaries delta[n+1] int8: deepest shared level of particles i-1 and i
//              (-1 at 0, n and where the system changes); leaflev[n] int8
//   nodes      level-major order (all level-0 nodes, then level 1, ...);
//              the children of a node are contiguous.
//              nodeA[k] float4 (com.x, com.y, com.z, M)          -- walk data
//              nodeB[k] float4 (b_J, G M b_J^2, link, meta)      -- walk data
//                link = first child (internal) or first particle (leaf)
//                meta = (nchild << 1) | 0 (internal), (count << 1) | 1 (leaf)
//              mass2[k] float2 (hi, lo): M as an unevaluated sum of two
//                floats (about 48 bits), for the bottom-up mass sums
//   groups     Morton order: first, count, sphere (centre, radius), alpha =
//              delta_acc * min |a_old|, system id, cost log
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

#include "nbody.h"

#define NB_FULL 0xffffffffu

namespace nb {

constexpr int kMaxLevels = 21;              // 21 bits per axis -> 63-bit keys
constexpr int kMaxNL = kMaxLevels + 1;      // levels 0..21
constexpr int kMlpParams = 8 * 32 + 32 + 32 * 32 + 32 + 32 + 1;  // 8 -> 32 -> 32 -> 1
constexpr int kStatusStackOverflow = 1;
constexpr int kStatusBadTree = 2;  // an index failed a bounds check (skipped)
constexpr int kStatusTimeout = 4;  // a bounded device wait ran out (results invalid)

// Device-resident counters and small per-build values.
struct DevState {
    int32_t nnodes;
    int32_t ngroups;
    int32_t queue_head;
    int32_t status;
    int32_t max_stack;
    int32_t pad0;
    unsigned long long list_entries;
    unsigned long long interactions;
    unsigned long long quad_entries;  // list entries that were quadrupole nodes
    int32_t lvl_off[kMaxNL + 1];
    int32_t block_maxlvl;   // block time steps: deepest occupied level
    int32_t block_nactive;  // block time steps: groups with an active particle
};

// Error-free transformations in FP32 (Knuth's TwoSum, Dekker's Fast2Sum)
// and the "double-float" sum built from them: a value hi + lo with |lo| <=
// ulp(hi) / 2 carries about 48 significant bits with FP32 arithmetic only.
// (GB300 runs FP64 at a small fraction of its FP32 rate.)
__device__ __forceinline__ float2 two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    return make_float2(s, e);
}
__device__ __forceinline__ float2 fast_two_sum(float a, float b) {  // |a| >= |b|
    const float s = __fadd_rn(a, b);
    return make_float2(s, __fsub_rn(b, __fsub_rn(s, a)));
}
__device__ __forceinline__ float2 df_add(float2 a, float2 b) {
    const float2 s = two_sum(a.x, b.x);
    return fast_two_sum(s.x, __fadd_rn(s.y, __fadd_rn(a.y, b.y)));
}

// Geometry of one system: cube corner, side and the FP32 quantisation scale.
struct SysBox {
    float x0, y0, z0, L;
    float scale;  // 2^levels / L (FP32, correctly rounded)
    float pad[3];
};

// Problem layout shared by the build kernels.
struct Layout {
    int64_t n;
    int32_t nsys;
    int32_t sysbits;
    int32_t levels;   // Morton levels below the root (21 for one system)
    int32_t keybits;  // sysbits + 3 * levels
};

// ---------------------------------------------------------------- warp helpers
__device__ __forceinline__ unsigned lane_id() { return threadIdx.x & 31u; }
__device__ __forceinline__ unsigned lanemask_lt() { return (1u << lane_id()) - 1u; }

__device__ __forceinline__ int warp_incl_scan(int v) {
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int t = __shfl_up_sync(NB_FULL, v, o);
        if ((int)lane_id() >= o) v += t;
    }
    return v;
}

// Hardware reciprocal square root and square root (one MUFU instruction each,
// relative error below 2^-22), with denormal inputs flushed to zero.  The
// softened r^2 + eps^2 of Eq. 1 is never denormal, so this changes no result
// of the force loops; it only drops the denormal handling around the MUFU.
__device__ __forceinline__ float rsqrt_fast(float x) {
    float y;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float sqrt_fast(float x) {
    float y;
    asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// Order-preserving map of a float onto uint32 (for atomic min/max).
__device__ __forceinline__ uint32_t f2ord(float f) {
    uint32_t u = __float_as_uint(f);
    return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}
__device__ __forceinline__ float ord2f(uint32_t u) {
    return __uint_as_float((u & 0x80000000u) ? (u & 0x7fffffffu) : ~u);
}

// System of sorted/caller particle i from the CSR offsets (nsys small).
__device__ __forceinline__ int sys_of(const int64_t *off, int nsys, int64_t i) {
    if (nsys <= 1) return 0;
    int lo = 0, hi = nsys;  // invariant: off[lo] <= i < off[hi]
    while (hi - lo > 1) {
        int mid = (lo + hi) >> 1;
        if (off[mid] <= i) lo = mid; else hi = mid;
    }
    return lo;
}

// ---------------------------------------------------------------- launchers
// sort.cu
void launch_bbox(cudaStream_t s, const Layout &L, const void *x, const void *y, const void *z,
                 bool dbl, const int64_t *d_off, uint32_t *d_boxord, SysBox *d_box, int nsm);
// Morton keys (vals = 0..n-1).  With sort_temp (cleared by radix_prepare),
// the kernel also accumulates the radix sort's digit histograms, and the
// sort is then called with hist_done = true.
void launch_keys(cudaStream_t s, const Layout &L, const void *x, const void *y, const void *z,
                 bool dbl, const int64_t *d_off, const SysBox *d_box, uint64_t *keys,
                 uint32_t *vals, void *sort_temp, int nsm);
size_t radix_temp_bytes(int64_t n);
// Clears the sort's counters, histograms and look-back words (one memset).
void radix_prepare(cudaStream_t s, int64_t n, void *temp);
// Sorts (keys, vals) by the low `bits` bits of keys, stably (ties keep their
// input order); vals must hold 0..n-1 on entry.  hist_done: the histograms in
// temp are already complete (launch_keys with sort_temp); else the sort
// clears temp and computes them.  Device-side failures (a look-back wait
// that ran out, a destination out of range) are or-ed into *status.  dn
// (nullable): the key count on the device, n then being an upper bound (no
// host read, so the sort can be captured in a graph).
// Returns 1 if the result ended in the alt buffers, else 0.
int radix_sort(cudaStream_t s, uint64_t *keys, uint32_t *vals, uint64_t *keys_alt,
               uint32_t *vals_alt, int64_t n, int bits, void *temp, bool hist_done,
               int32_t *status, int nsm, const int32_t *dn = nullptr);
int radix_passes(int bits);
// Sort of keys that are nearly in order already (the previous build's order
// with new keys, as inside a time step): splitters from one key per tile,
// buckets, a scatter and a shared-memory sort per bucket (nosort.cu).
// keys (overwritten: scratch) -> kout (sorted keys), vout (the value of each
// sorted key: its index in the input, or vin[index] when vin is given);
// vscr: uint32 [n] scratch (may be vin: read before vscr is written).  The
// result is the sort by (key, value): with the indices as values, the stable
// sort of the keys for any input order; with vin a permutation, the stable
// sort of the keys in the order vin names.  Device-side failures are or-ed
// into *status.
bool nosort_fits(int64_t n);
size_t nosort_temp_bytes(int64_t n);
void nosort(cudaStream_t s, uint64_t *keys, uint64_t *kout, uint32_t *vscr, uint32_t *vout,
            int64_t n, void *temp, int32_t *status, const uint32_t *vin = nullptr);
// kout[k] = keys[hint[k]], vout[k] = hint[k]: keys put in a hinted order
// (a permutation of 0..n-1) before the near-order sort.
void nosort_hint_gather(cudaStream_t s, int64_t n, const uint64_t *keys, const uint32_t *hint,
                        uint64_t *kout, uint32_t *vout);
int nosort_kernels();
// True for memory the current device dev can read in place (its own device
// memory, or managed memory); diag_noalloc.cu.
bool on_device(const void *p, int dev);
// Runs the radix pass kernel on an input whose look-back can never complete
// and waits for it; the bounded wait records kStatusTimeout in *status.
cudaError_t radix_selftest_wait(cudaStream_t s, int32_t *status);
// Single-block exclusive scan of sums[0..nb) in place (total to *total_out).
void launch_scan_sums(cudaStream_t s, uint32_t *sums, int nb, int32_t *total_out);
void launch_gather_pos4(cudaStream_t s, int64_t n, const uint32_t *perm, const void *x,
                        const void *y, const void *z, bool dbl, const float *m, float4 *pos4);

// tree.cu
size_t tree_temp_bytes(int64_t n, int levels);
void build_tree(cudaStream_t s, const Layout &L, const uint64_t *keys, const float4 *pos4,
                const SysBox *d_box, const int64_t *d_off, int leaf_cap, float G,
                int64_t cap_nodes, int8_t *delta, int8_t *leaflev, void *temp, DevState *ds,
                int32_t *node_start, int8_t *node_level, int32_t *node_parent,
                int32_t *node_link, int32_t *node_count, int32_t *node_nchild,
                int32_t *node_arrive, float4 *nodeA, float4 *nodeB, float2 *mass2, float4 *nodeQ,
                int32_t *sys_root, int nsm);
// Node moments of the current tree from pos4 (refit: positions moved since
// the build; b_J of internal nodes from the child recurrence only).
// nodeQ (nullable): also the traceless quadrupoles, 2 float4 per node.
void tree_moments(cudaStream_t s, const Layout &L, const uint64_t *keys, const float4 *pos4,
                  const SysBox *d_box, int leaf_cap, float G, DevState *ds,
                  const int32_t *node_start, const int8_t *node_level, const int32_t *node_parent,
                  const int32_t *node_link, int32_t *node_count, const int32_t *node_nchild,
                  int32_t *node_arrive, float4 *nodeA, float4 *nodeB, float2 *mass2,
                  float4 *nodeQ, int nsm, bool refit);
void refit_groups(cudaStream_t s, const Layout &L, int group_size, const float4 *pos4,
                  const int64_t *d_off, DevState *ds, const int32_t *grp_first,
                  int32_t *grp_count, float4 *grp_sphere, int32_t *grp_sys, int nsm);
void build_groups(cudaStream_t s, const Layout &L, int group_size, const float4 *pos4,
                  const int64_t *d_off, const int32_t *node_start, const int32_t *node_parent,
                  const int32_t *node_count, const int32_t *node_nchild, const int32_t *node_link,
                  DevState *ds, uint8_t *gflag, void *temp, int32_t *grp_first,
                  int32_t *grp_count, float4 *grp_sphere, int32_t *grp_sys, int nsm);
void launch_group_alpha(cudaStream_t s, int64_t n, const DevState *ds, const int32_t *grp_first,
                        const int32_t *grp_count, const float *aold_sorted, float delta_acc,
                        float *grp_alpha, int nsm);

// walk.cu
// Shared memory of one walk warp: the list (16 B per entry), the traversal
// stack (4 B per entry) and kWalkScratch words for compacting opened leaves,
// rounded up to 16 B so that every warp's list stays float4-aligned.
constexpr int kWalkScratch = 32;
// With quadrupoles, accepted nodes go to a second list of walk_quad_depth
// entries of 40 B (centre of mass and mass, then the six quadrupole terms).
__host__ __device__ inline int walk_quad_depth(int list_depth) {
    return list_depth / 4 > 32 ? list_depth / 4 : 32;
}
__host__ __device__ inline size_t walk_smem_per_warp(int list_depth, int stack_depth,
                                                     bool quad = false) {
    const size_t b = (size_t)list_depth * 16 + (quad ? (size_t)walk_quad_depth(list_depth) * 40 : 0) +
                     (size_t)stack_depth * 4 + (size_t)kWalkScratch * 4;
    return (b + 15) & ~(size_t)15;
}
struct WalkArgs {
    const float4 *pos4;
    const float4 *nodeA;
    const float4 *nodeB;
    const float4 *nodeQ;       // 2 per node: (xx, yy, zz, xy), (xz, yz, 0, 0); quadrupole walk only
    const int32_t *grp_first;
    const int32_t *grp_count;
    const float4 *grp_sphere;
    const float *grp_alpha;
    const int32_t *grp_sys;
    const int32_t *order;      // schedule permutation (NULL: Morton order)
    const float *sys_eps2;
    const int32_t *sys_root;
    DevState *ds;
    const int32_t *nactive;    // non-NULL: walk only order[0 .. *nactive) (block time steps)
    int32_t *grp_cost;         // list entries per group (NULL: not logged)
    int64_t n;                 // particles (bounds of pos4)
    float G;
    float theta;
    int list_depth;
    int stack_depth;
    // outputs: scatter mode (perm != NULL) or sorted mode
    const int32_t *perm;
    float *ax, *ay, *az, *phi;
    float4 *acc_sorted;        // (ax, ay, az, phi)
};
struct WalkShape {
    int ipl;
    bool geometric;
    bool potential;
    bool compensated;
    bool safe;                  // some eps == 0: guard the self term
    bool quad;                  // accepted nodes add their quadrupole
    bool pipeline;              // warp pairs: traversal and evaluation (monopole, no potential)
    int warps_per_block;
    int *warps_launched;        // host, nullable: receives the resident walk warps
};
cudaError_t launch_walk(cudaStream_t s, const WalkArgs &a, const WalkShape &sh, int nsm);
cudaError_t launch_direct(cudaStream_t s, int64_t n, const float *x, const float *y,
                          const float *z, const float *m, float G, float eps, bool compensated,
                          float *ax, float *ay, float *az, float *phi);
void launch_acc_mag(cudaStream_t s, int64_t n, const float4 *acc_sorted, float *aold_sorted);
void launch_gather_f32(cudaStream_t s, int64_t n, const uint32_t *perm, const float *src,
                       float *dst);

// mlp.cu
void launch_mlp_features(cudaStream_t s, const Layout &L, const DevState *ds,
                         const int32_t *grp_first, const int32_t *grp_count,
                         const float4 *grp_sphere, const int32_t *grp_sys, const float *aold,
                         const uint64_t *keys, const float4 *nodeA, const int32_t *sys_root,
                         const SysBox *box, const int64_t *off, float *feat, int nsm);
void launch_mlp_forward(cudaStream_t s, const int32_t *pn, int64_t n, const float *feat,
                        const __nv_bfloat16 *wb, const float *norm, const float *tnorm,
                        float *pred, int nsm);
size_t mlp_grad_smem();
cudaError_t launch_mlp_train_step(cudaStream_t s, const float *feat, const float *target,
                                  int64_t base, int64_t stride, int count,
                                  const __nv_bfloat16 *wb, const float *norm, float *gpart,
                                  float *lpart, float *grad, float *loss, float *w, float *m1,
                                  float *m2, __nv_bfloat16 *wb_out, float lr, int t, bool update);
void launch_mlp_round(cudaStream_t s, const float *w, __nv_bfloat16 *wb);
void launch_mlp_norm(cudaStream_t s, const int32_t *pn, const float *feat, const float *target,
                     float *norm);
void launch_mlp_target(cudaStream_t s, const int32_t *pn, const int32_t *cost, const float *tnorm,
                       float *target,
                       int nsm);
void launch_order_keys(cudaStream_t s, const int32_t *pn, const float *score,
                       const int32_t *grp_count, uint64_t *key, uint32_t *val, int nsm);
void launch_lastcost_score(cudaStream_t s, const int32_t *pn, const int32_t *grp_first,
                           const float *pcost, float *score, int nsm);
void launch_spread_cost(cudaStream_t s, const int32_t *pn, const int32_t *grp_first,
                        const int32_t *grp_count, const int32_t *cost, float *pcost, int nsm);

// integrate.cu
struct StepState {
    double *x, *y, *z;
    float *vx, *vy, *vz, *m;
    float *aold;
    uint32_t *id;    // caller index of each sorted particle
    float *pcost;    // cost of each particle's group in the last walk (may be NULL)
    uint8_t *lvl;    // block time-step level of each particle (may be NULL)
};
// Block time steps (levels 0..K, step dt / 2^k).  block_start: every
// particle's level from |a| and the opening half kick of its step;
// block_kick at clock tick T (of total): closing half kick, new level and
// (T < total) the opening half kick for the particles active at T.  Both
// record the deepest occupied level in *maxlvl (cleared by the caller).
void launch_block_start(cudaStream_t s, int64_t n, StepState st, const float4 *acc, float dt,
                        int K, float eta, const int64_t *off, int nsys, const float *sys_eps,
                        int32_t *maxlvl);
void launch_block_kick(cudaStream_t s, int64_t n, StepState st, const float4 *acc, int64_t T,
                       int64_t total, float dt, int K, float eta, const int64_t *off, int nsys,
                       const float *sys_eps, int32_t *maxlvl);
// The groups holding a particle active at tick T, in *count entries of order.
void launch_block_active_groups(cudaStream_t s, const DevState *ds, const int32_t *grp_first,
                                const int32_t *grp_count, const uint8_t *lvl, int64_t T, int K,
                                int32_t *order, int32_t *count, int nsm);
// pos4 (nullable): also refresh the FP32 walk copy (x, y, z, m) in place.
// hclose != 0: apply the previous step's closing half kick (v += a hclose,
// a_old = |a|) first, as the kick kernel would.
void launch_kick_drift(cudaStream_t s, int64_t n, StepState st, const float4 *acc, float hdt,
                       float dt, float4 *pos4, float hclose = 0.0f);
void launch_kick(cudaStream_t s, int64_t n, StepState st, const float4 *acc, float hdt);
void launch_permute_state(cudaStream_t s, int64_t n, const uint32_t *perm, StepState src,
                          StepState dst, float4 *pos4);
// kick_drift: also the first step's opening half kick (v += a hdt) and drift
// (x += v dt), with the kick-drift pass's arithmetic.
void launch_load_state(cudaStream_t s, int64_t n, const double *x, const double *y,
                       const double *z, const float *vx, const float *vy, const float *vz,
                       const float *m, const float *ax, const float *ay, const float *az,
                       StepState st, float4 *acc, bool kick_drift = false, float hdt = 0.0f,
                       float dt = 0.0f, void *rec = nullptr);
// (rec != nullptr: only x, y, z, acc go to the SoA state; the rest of each
// particle, with x, y, z, is written as its 64-byte record into rec, ready
// for launch_permute_state_recs(..., packed = true).)
// The same permutation through 64-byte particle records (rec: 64 n bytes of
// scratch): for a far-from-identity perm (the first sort of a call).
// packed: rec already holds src's records (written by the state load).
void launch_permute_state_recs(cudaStream_t s, int64_t n, const uint32_t *perm, StepState src,
                               StepState dst, float4 *pos4, void *rec, bool packed = false);
// The state back in caller order (x, y, z, v, a), through 64-byte records
// scattered to the caller indices (rec: 64 n bytes of scratch); hkick != 0:
// the velocities get the last step's closing half kick on the way out (the
// device state itself is left without it).
void launch_store_state(cudaStream_t s, int64_t n, StepState st, const float4 *acc, double *x,
                        double *y, double *z, float *vx, float *vy, float *vz, float *ax,
                        float *ay, float *az, void *rec, float hkick = 0.0f);
size_t diag_temp_bytes();
// Message returned by nbody_last_error(NULL, ...) on this thread.
void set_stateless_error(const std::string &msg);
void launch_diagnostics(cudaStream_t s, int64_t n, const double *x, const double *y,
                        const double *z, const float *vx, const float *vy, const float *vz,
                        const float *m, const float *phi, void *temp, double *d_out);

}  // namespace nb
