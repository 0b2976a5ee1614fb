// tree.cu -- octree from sorted Morton keys ("makeTree"), bottom-up monopoles
// and node sizes ("calcNode", Sect. 2.2), and the i-groups that share one
// interaction list in the walk (Sect. 1).
//
// Octree definition.  A node at level l is a maximal run of sorted particles
// sharing the top 3l Morton bits (plus the system id).  A node is split into
// its non-empty octants while it holds more than leaf_cap particles and
// l < levels.  Writing delta_i for the deepest level shared by particles i-1
// and i (-1 at 0, n and at system changes), and L_i for the level of the leaf
// that holds particle i, the nodes that start at particle i are exactly the
// levels delta_i < l <= L_i, and
//     L_i = min(levels, 1 + min over boundary pairs (left <= i < right,
//               right - left <= leaf_cap) of max(delta_left, delta_right)),
// because a run bounded by two boundaries whose shared levels are both below
// l+1 is cut at level l+1.  So the whole tree structure comes from
// per-particle work in a window of 2*leaf_cap boundaries plus one scan per
// level -- no level-by-level launches.
//
// Monopoles are accumulated bottom-up in one launch: the leaves from their
// particles, then each internal node by the thread that finishes its last
// child (an atomic count per node), so neither a launch per level nor the
// grid-wide barriers of the paper's calcNode (App. A) are needed.
#include <cuda_runtime.h>

#include "internal.cuh"

namespace nb {

constexpr int TB = 256;  // particles per block in the per-particle tree kernels

__device__ __forceinline__ int delta_of(uint64_t a, uint64_t b, int mbits, int levels) {
    uint64_t x = a ^ b;
    if (x >> mbits) return -1;  // different systems
    if (x == 0) return levels;
    int h = 63 - __clzll((long long)x);
    return (mbits - 1 - h) / 3;
}

__device__ __forceinline__ uint32_t level_mask(int d, int L) {
    if (L <= d) return 0u;
    uint32_t hi = (2u << L) - 1u;
    uint32_t lo = d < 0 ? 0u : ((2u << d) - 1u);
    return hi & ~lo;
}

// delta, leaf level and per-level node counts of each block of TB particles.
// A CTA takes VB consecutive blocks (VB * TB particles, one per thread and
// block): the keys of all of them and of the window around them are loaded
// together, so one load latency covers VB blocks.
constexpr int kMaxCap = 32;
constexpr int VB = 4;
// CAPT: a power of two >= cap, the unrolled length of the window loops.
template <int CAPT>
__global__ void __launch_bounds__(TB) leaflevel_kernel(Layout L, int cap,
                                                       const uint64_t *__restrict__ keys,
                                                       int8_t *__restrict__ delta,
                                                       int8_t *__restrict__ leaflev,
                                                       uint32_t *__restrict__ blockcnt, int nblk) {
    __shared__ uint64_t sk[VB * TB + 2 * kMaxCap + 1];
    __shared__ int sd[VB * TB + 2 * kMaxCap];
    __shared__ uint32_t wc[VB][kMaxNL][TB / 32];
    const int64_t n = L.n;
    const int64_t blk0 = (int64_t)blockIdx.x * VB;
    const int64_t lo = blk0 * TB - cap;  // global boundary index of sd[0]
    for (int t = threadIdx.x; t < VB * TB + 2 * cap + 1; t += TB) {
        int64_t g = lo - 1 + t;
        sk[t] = (g >= 0 && g < n) ? keys[g] : 0ull;
    }
    __syncthreads();
    // boundaries outside (0, n) read as -1 ("no shared level"), so the window
    // loops need no range checks: a pair with an end beyond the range
    // repeats one that ends at 0 or n
    for (int t = threadIdx.x; t < VB * TB + 2 * cap; t += TB) {
        int64_t g = lo + t;
        sd[t] = (g <= 0 || g >= n) ? -1 : delta_of(sk[t], sk[t + 1], 3 * L.levels, L.levels);
    }
    __syncthreads();
    const int NL = L.levels + 1;
    const unsigned w = threadIdx.x >> 5;
    for (int v = 0; v < VB; v++) {
        const int64_t i = (blk0 + v) * TB + threadIdx.x;
        uint32_t mask = 0;
        if (i < n) {
            const int ti = v * TB + threadIdx.x + cap;
            int R = 127, best = 127;
            // R = min delta over boundaries i+1..i+k; a run [i-cap+k, right)
            // with right <= i-cap+k+cap is cut at level max(delta_left, R) + 1.
#pragma unroll
            for (int k = 1; k <= CAPT; k++) {
                if (k <= cap) {
                    R = min(R, sd[ti + k]);
                    best = min(best, max(sd[ti - cap + k], R));
                }
            }
            int Li = min(L.levels, best + 1);
            int di = sd[ti];
            delta[i] = (int8_t)di;
            leaflev[i] = (int8_t)Li;
            if (i == n - 1) delta[n] = -1;
            mask = level_mask(di, Li);
        }
        // per-warp node counts, visiting only the levels some lane starts a node at
        if (lane_id() < (unsigned)NL) wc[v][lane_id()][w] = 0u;
        __syncwarp();
        const unsigned any = __reduce_or_sync(NB_FULL, mask);
        for (unsigned m = any; m; m &= m - 1) {
            const int l = __ffs(m) - 1;
            const unsigned b = __ballot_sync(NB_FULL, (mask >> l) & 1u);
            if (lane_id() == 0) wc[v][l][w] = (uint32_t)__popc(b);
        }
    }
    __syncthreads();
    for (int t = threadIdx.x; t < VB * NL; t += TB) {
        const int v = t / NL, l = t % NL;
        if (blk0 + v >= nblk) continue;
        uint32_t c = 0;
        for (int q = 0; q < TB / 32; q++) c += wc[v][l][q];
        blockcnt[(int64_t)l * nblk + blk0 + v] = c;
    }
}

// One block per level: exclusive scan of that level's block counts; the
// level's node count goes to lvl_off[l + 1] (turned into offsets below).
// Each thread scans LS_IPT consecutive counts, so a level of 32768 blocks
// takes four block-wide scans.
constexpr int LS_T = 1024, LS_IPT = 8;
__global__ void __launch_bounds__(LS_T) level_scan_kernel(uint32_t *blockcnt, int nblk,
                                                          DevState *ds) {
    __shared__ uint32_t sh[32];
    const int l = blockIdx.x;
    const int w = threadIdx.x >> 5;
    uint32_t carry = 0;
    uint32_t *row = blockcnt + (int64_t)l * nblk;
    for (int base = 0; base < nblk; base += LS_T * LS_IPT) {
        const int i0 = base + threadIdx.x * LS_IPT;
        uint32_t v[LS_IPT], t = 0;
#pragma unroll
        for (int k = 0; k < LS_IPT; k++) {
            v[k] = i0 + k < nblk ? row[i0 + k] : 0u;
            t += v[k];
        }
        const uint32_t incl = (uint32_t)warp_incl_scan((int)t);
        if (lane_id() == 31) sh[w] = incl;
        __syncthreads();
        if (threadIdx.x < 32) sh[threadIdx.x] = (uint32_t)warp_incl_scan((int)sh[threadIdx.x]);
        __syncthreads();
        uint32_t ex = carry + incl - t + (w ? sh[w - 1] : 0u);
#pragma unroll
        for (int k = 0; k < LS_IPT; k++) {
            if (i0 + k < nblk) row[i0 + k] = ex;
            ex += v[k];
        }
        carry += sh[31];
        __syncthreads();
    }
    if (threadIdx.x == 0) ds->lvl_off[l + 1] = (int32_t)carry;
}

__global__ void level_offsets_kernel(int NL, DevState *ds, int64_t cap_nodes) {
    if (threadIdx.x != 0) return;
    int32_t off = 0;
    ds->lvl_off[0] = 0;
    for (int l = 0; l < NL; l++) {
        off += ds->lvl_off[l + 1];
        ds->lvl_off[l + 1] = off;
    }
    ds->nnodes = off;
    if (off > cap_nodes) atomicOr(&ds->status, kStatusStackOverflow);
}

// Zeroes the child counts and the moments pass's arrival counters of the
// nodes about to be made (the node count is on the device).
__global__ void node_zero_kernel(const DevState *__restrict__ ds, int64_t cap_nodes,
                                 int32_t *node_nchild, int32_t *node_arrive) {
    const int64_t nn = min((int64_t)ds->nnodes, cap_nodes);
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nn;
         i += (int64_t)gridDim.x * blockDim.x) {
        node_nchild[i] = 0;
        node_arrive[i] = 0;
    }
}

// Writes every node: start, level, parent, first child / first particle and,
// for leaves, the particle count.  Children bump their parent's child count.
// The node at level l starting at particle i gets the id
//   lvl_off[l] + (nodes of level l in earlier blocks) + (in earlier warps of
//   this block) + (in earlier lanes of this warp),
// and only the levels at which some lane of the warp starts a node are
// visited.  A particle's nodes sit on the consecutive levels delta_i + 1 ..
// L_i, so each one's parent is the particle's previous node, and the first
// one's parent is the last node of level delta_i starting before particle i.
__global__ void __launch_bounds__(TB) nodes_kernel(Layout L, const int8_t *__restrict__ delta,
                                                   const int8_t *__restrict__ leaflev,
                                                   const uint32_t *__restrict__ blockcnt, int nblk,
                                                   const DevState *__restrict__ ds,
                                                   int64_t cap_nodes, int32_t *node_start,
                                                   int8_t *node_level, int32_t *node_parent,
                                                   int32_t *node_link, int32_t *node_count,
                                                   int32_t *node_nchild) {
    __shared__ uint32_t wc[kMaxNL][TB / 32];
    __shared__ int32_t sbase[kMaxNL];
    const int64_t n = L.n;
    const int NL = L.levels + 1;
    const int64_t i = (int64_t)blockIdx.x * TB + threadIdx.x;
    const unsigned w = threadIdx.x >> 5;
    int di = -1, Li = -1;
    uint32_t mask = 0;
    if (i < n) {
        di = delta[i];
        Li = leaflev[i];
        mask = level_mask(di, Li);
    }
    for (int t = threadIdx.x; t < kMaxNL * (TB / 32); t += TB) (&wc[0][0])[t] = 0u;
    if (threadIdx.x < NL)
        sbase[threadIdx.x] = ds->lvl_off[threadIdx.x] +
                             (int32_t)blockcnt[(int64_t)threadIdx.x * nblk + blockIdx.x];
    __syncthreads();
    const unsigned any = __reduce_or_sync(NB_FULL, mask);
    for (unsigned m = any; m; m &= m - 1) {
        const int l = __ffs(m) - 1;
        const unsigned b = __ballot_sync(NB_FULL, (mask >> l) & 1u);
        if (lane_id() == 0) wc[l][w] = (uint32_t)__popc(b);
    }
    __syncthreads();
    if (threadIdx.x < NL) {
        uint32_t run = 0;
        for (int q = 0; q < TB / 32; q++) {
            uint32_t c = wc[threadIdx.x][q];
            wc[threadIdx.x][q] = run;
            run += c;
        }
    }
    __syncthreads();
    const unsigned lt = lanemask_lt();
    // id of the last node of level di starting before i (no lane of this warp
    // starts one there unless the loop below finds that level in `any`)
    int pex = di >= 0 ? sbase[di] + (int)wc[di][w] : 0;
    int prev_id = -1;
    // warp-uniform level set: the levels with nodes plus every lane's di
    const unsigned visit = any | __reduce_or_sync(NB_FULL, di >= 0 ? (1u << di) : 0u);
    for (unsigned m = visit; m; m &= m - 1) {
        const int l = __ffs(m) - 1;
        const int bit = (mask >> l) & 1u;
        const unsigned b = __ballot_sync(NB_FULL, bit);
        const int ex = sbase[l] + (int)wc[l][w] + __popc(b & lt);
        if (l == di) pex = ex;
        if (!bit) continue;
        const int id = ex;
        if (prev_id >= 0 && prev_id < cap_nodes) node_link[prev_id] = id;  // first child
        if (id < cap_nodes) {
            node_start[id] = (int32_t)i;
            node_level[id] = (int8_t)l;
            const int par = prev_id >= 0 ? prev_id : (di >= 0 ? pex - 1 : -1);
            node_parent[id] = par;
            if (par >= 0) atomicAdd(&node_nchild[par], 1);
            if (l == Li) {  // leaf: particles until the next boundary above level l
                int64_t j = i + 1;
                while (j < n && delta[j] >= l) j++;
                node_link[id] = (int32_t)i;
                node_count[id] = (int32_t)(j - i);
            }
        }
        prev_id = id;
    }
}

__global__ void sys_root_kernel(const DevState *ds, const int32_t *node_start, const int64_t *off,
                                int nsys, int32_t *sys_root) {
    int nroot = ds->lvl_off[1];
    for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < nroot; r += gridDim.x * blockDim.x)
        sys_root[sys_of(off, nsys, node_start[r])] = r;
}

__global__ void sys_root_init_kernel(int nsys, int32_t *sys_root) {
    for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < nsys; s += gridDim.x * blockDim.x)
        sys_root[s] = -1;
}

// ---------------------------------------------------------------- moments
__device__ __forceinline__ int &ds_status(DevState *ds) { return ds->status; }



__device__ __forceinline__ uint32_t compact3(uint64_t x) {
    x &= 0x1249249249249249ull;
    x = (x ^ (x >> 2)) & 0x10c30c30c30c30c3ull;
    x = (x ^ (x >> 4)) & 0x100f00f00f00f00full;
    x = (x ^ (x >> 8)) & 0x001f0000ff0000ffull;
    x = (x ^ (x >> 16)) & 0x001f00000000ffffull;
    x = (x ^ (x >> 32)) & 0x00000000001fffffull;
    return (uint32_t)x;
}

// Centre and half-size of a node's cell, the half-size widened by one finest
// cell (covers the FP32 quantisation of member positions).  FP32: the cell
// side is the cube side scaled by an exact power of two.
struct CellF {
    float c[3];
    float h;
};

__device__ __forceinline__ float pow2f(int e) { return __int_as_float((127 + e) << 23); }

__device__ __forceinline__ CellF node_cell(const Layout &L, uint64_t key, int level,
                                           const SysBox *box) {
    const int mbits = 3 * L.levels;
    int s = L.sysbits ? (int)(key >> mbits) : 0;
    SysBox b = box[s];
    uint64_t morton = mbits >= 64 ? key : (key & ((1ull << mbits) - 1ull));
    uint64_t prefix = morton >> (3 * (L.levels - level));
    uint32_t q[3] = {compact3(prefix >> 2), compact3(prefix >> 1), compact3(prefix)};
    float side = b.L * pow2f(-level);
    float o[3] = {b.x0, b.y0, b.z0};
    CellF cell;
#pragma unroll
    for (int a = 0; a < 3; a++) cell.c[a] = o[a] + ((float)q[a] + 0.5f) * side;
    cell.h = 0.5f * side + b.L * pow2f(-L.levels);
    return cell;
}

// Round-up factor for FP32 upper bounds (a few ulps of slack).
constexpr float kUp = 1.0f + 0x1p-20f;

// Node record: centre of mass, mass (hi + lo), size b and the MAC numerator
// G M b^2, rounded up from the FP32 values.
__device__ __forceinline__ void write_node(int id, float cx, float cy, float cz, float2 M,
                                           float b, float G, int link, int meta, float4 *nodeA,
                                           float4 *nodeB, float2 *mass2) {
    const float Mup = M.y > 0.0f ? __int_as_float(__float_as_int(M.x) + 1) : M.x;  // M.x >= 0
    const float q = __fmul_ru(__fmul_ru(__fmul_ru(G, Mup), b), b);
    nodeA[id] = make_float4(cx, cy, cz, M.x);
    nodeB[id] = make_float4(b, q, __int_as_float(link), __int_as_float(meta));
    mass2[id] = M;
}

// Quadrupole (an extension beyond the paper's monopoles): the traceless
// Q_ab = sum m (3 s_a s_b - |s|^2 delta_ab) over offsets s from the centre of
// mass; q = {xx, yy, zz, xy, xz, yz}.  A child of mass m at offset s with its
// own quadrupole Qc contributes Qc plus the point-mass term (parallel axes).
__device__ __forceinline__ void quad_add(float q[6], float m, float dx, float dy, float dz,
                                         float r2) {
    const float m3 = 3.0f * m;
    q[0] = fmaf(m3 * dx, dx, fmaf(-m, r2, q[0]));
    q[1] = fmaf(m3 * dy, dy, fmaf(-m, r2, q[1]));
    q[2] = fmaf(m3 * dz, dz, fmaf(-m, r2, q[2]));
    q[3] = fmaf(m3 * dx, dy, q[3]);
    q[4] = fmaf(m3 * dx, dz, q[4]);
    q[5] = fmaf(m3 * dy, dz, q[5]);
}

__device__ __forceinline__ void write_quad(int id, const float q[6], float4 *nodeQ) {
    nodeQ[2 * id] = make_float4(q[0], q[1], q[2], q[3]);
    nodeQ[2 * id + 1] = make_float4(q[4], q[5], 0.0f, 0.0f);
}

// Monopoles (centre of mass, mass) and node sizes b_J, bottom-up.  FP32 sums
// relative to a reference point inside the node (first particle for leaves,
// the cell centre for internal nodes) keep the error a few ulps of the node
// size; masses are summed as double-float pairs (about 48 bits, FP32
// arithmetic only).  b_J is rounded up so it bounds the distance from the
// FP32 centre of mass to every member.
//
// One launch for the whole tree, no pass per level.  Leaves: a team of T
// lanes takes one leaf (T = 1 up to leaf capacity 16: a lane per leaf, its
// member loads issued in batches), lane j loading members j, j + T, ...; the
// sums and the largest member distance are team reductions.  Internal nodes:
// every finished node counts itself in at its parent (an atomic counter), and
// the thread whose count completes the parent computes it from the children's
// records and climbs on.  No thread waits for another.  The counters are
// zeroed when the nodes are made, and each is reset by the thread that
// completes its node, so a later pass over the same tree (a refit) starts
// from zero too; a node that fails its bounds check is still counted in at
// its parent, which keeps every counter consistent.

// One internal node from its children's records (contiguous, at most 8), by
// one thread.  Sums run over the children in octant order, relative to the
// cell centre; the size is
//   b = min(max_c (|com_c - com| + b_c), distance from com to the farthest
//           corner of the cell widened by one finest cell),
// rounded up.  After a refit (positions moved since the build, members may
// have left the cell) only the child recurrence bounds b.  Children finished
// by other SMs in this launch are read past L1 (ld.global.cg): a sibling's
// cache line may already sit in this SM's L1 from before it was written.
__device__ __forceinline__ bool internal_node(const Layout &L, int p, int c0, int nc, int level,
                                              uint64_t key, int refit, int nn,
                                              const SysBox *__restrict__ box, float G,
                                              int32_t *node_count, float4 *nodeA, float4 *nodeB,
                                              float2 *mass2, float4 *nodeQ) {
    if (c0 <= p || nc < 1 || nc > 8 || c0 + nc > nn) return false;
    const CellF cell = node_cell(L, key, level, box);
    // every field of every child in one round trip; the positions and sizes
    // stay in registers for the size bound
    float CX[8], CY[8], CZ[8], CB[8];
    float2 M = make_float2(0.0f, 0.0f);
    float px = 0.0f, py = 0.0f, pz = 0.0f;
    int count = 0;
#pragma unroll
    for (int k = 0; k < 8; k++) {
        const int j = k < nc ? c0 + k : c0;
        const float4 A = __ldcg(nodeA + j);
        const float2 mk = __ldcg(mass2 + j);
        const int ck = __ldcg(node_count + j);
        CB[k] = __ldcg(&nodeB[j].x);
        CX[k] = A.x; CY[k] = A.y; CZ[k] = A.z;
        if (k < nc) {
            M = df_add(M, mk);
            count += ck;
            px = fmaf(A.w, A.x - cell.c[0], px);
            py = fmaf(A.w, A.y - cell.c[1], py);
            pz = fmaf(A.w, A.z - cell.c[2], pz);
        }
    }
    float cp[3] = {cell.c[0], cell.c[1], cell.c[2]};
    if (M.x > 0.0f) {
        const float inv = 1.0f / M.x;
        cp[0] = fmaf(px, inv, cp[0]); cp[1] = fmaf(py, inv, cp[1]); cp[2] = fmaf(pz, inv, cp[2]);
    }
    float rec = 0.0f;
    float q[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
#pragma unroll
    for (int k = 0; k < 8; k++) {
        if (k < nc) {
            const float dx = CX[k] - cp[0], dy = CY[k] - cp[1], dz = CZ[k] - cp[2];
            const float r2 = fmaf(dz, dz, fmaf(dy, dy, dx * dx));
            rec = fmaxf(rec, __fadd_ru(__fsqrt_ru(r2), CB[k]));
        }
    }
    if (nodeQ) {
#pragma unroll
        for (int k = 0; k < 8; k++) {
            if (k >= nc) break;
            const int j = c0 + k;
            const float4 A = __ldcg(nodeA + j);
            const float dx = A.x - cp[0], dy = A.y - cp[1], dz = A.z - cp[2];
            const float r2 = fmaf(dz, dz, fmaf(dy, dy, dx * dx));
            const float4 q0 = __ldcg(nodeQ + 2 * j), q1 = __ldcg(nodeQ + 2 * j + 1);
            q[0] += q0.x; q[1] += q0.y; q[2] += q0.z; q[3] += q0.w; q[4] += q1.x; q[5] += q1.y;
            quad_add(q, A.w, dx, dy, dz, r2);
        }
    }
    float c2 = 0.0f;
#pragma unroll
    for (int a = 0; a < 3; a++) {
        const float e = fabsf(cp[a] - cell.c[a]) + cell.h;
        c2 = fmaf(e, e, c2);
    }
    const float bp = (refit ? rec : fminf(rec, __fsqrt_ru(c2))) * kUp;
    node_count[p] = count;
    write_node(p, cp[0], cp[1], cp[2], M, bp, G, c0, nc << 1, nodeA, nodeB, mass2);
    if (nodeQ) write_quad(p, q, nodeQ);
    return true;
}

// Count a finished node in at its parent `par` (one atomic add with release
// and acquire semantics: this thread's writes of the node are published by
// it, and the thread that completes the parent sees every child's records).
// Returns how many of the parent's children have now arrived.
__device__ __forceinline__ int count_in(int par, int32_t *node_arrive) {
    int old;
    asm volatile("atom.acq_rel.gpu.global.add.s32 %0, [%1], 1;"
                 : "=r"(old)
                 : "l"(node_arrive + par)
                 : "memory");
    return old + 1;
}

#ifndef NB_MOMENTS_MIN_CTAS
#define NB_MOMENTS_MIN_CTAS 4  // resident 256-thread CTAs per SM the moments pass is compiled for
#endif

// Members loaded per batch by each lane of a leaf team (independent loads in
// flight together).
constexpr int kLeafUnroll = 4;
template <int T>
__global__ void __launch_bounds__(256, NB_MOMENTS_MIN_CTAS) moments_kernel(
    Layout L, int refit, const uint64_t *__restrict__ keys, const float4 *__restrict__ pos4,
    const SysBox *__restrict__ box, float G, DevState *ds,
    const int32_t *__restrict__ node_start, const int8_t *__restrict__ node_level,
    const int32_t *__restrict__ node_parent, const int32_t *__restrict__ node_link,
    int32_t *node_count, const int32_t *__restrict__ node_nchild, int32_t *node_arrive,
    float4 *nodeA, float4 *nodeB, float2 *mass2, float4 *nodeQ) {
    constexpr int TEAMS = 32 / T;
    const int nn = ds->nnodes;
    const int lane = (int)lane_id(), team = lane / T, tl = lane % T;
    const int64_t wid = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    bool bad = false;
    // deepest chunks first (ids are level-major): the long climbs from deep
    // leaves start early, and the last leaves to finish sit near the roots
    const int64_t nchunk = ((int64_t)nn + 31) / 32;
    for (int64_t ch = wid; ch < nchunk; ch += nw) {
        const int64_t base = (nchunk - 1 - ch) * 32;
        const int id0 = (int)base + lane;
        // every field this lane's node needs, in one round trip
        const bool inb = id0 < nn;
        const int nch0 = inb ? node_nchild[id0] : -1;
        const int link0 = inb ? node_link[id0] : 0;
        const int cnt0 = inb ? node_count[id0] : 0;
        const int par0 = inb ? node_parent[id0] : -1;
        const int lev0 = inb ? (int)node_level[id0] : 0;
        const int st0 = inb ? node_start[id0] : 0;
        const bool leaf = nch0 == 0;
        // the climb needs a member key: load it now, beside the members
        const uint64_t key0 = leaf ? keys[st0] : 0ull;
        unsigned lm = __ballot_sync(NB_FULL, leaf);
        while (lm) {
            // one lane per leaf: each lane takes its own node (its fields are
            // loaded); teams: team t takes the t-th remaining leaf
            int mine = -1;
            if constexpr (T == 1) {
                mine = leaf ? lane : -1;
                lm = 0;
            } else {
#pragma unroll
                for (int t = 0; t < TEAMS; t++) {
                    const int b = lm ? __ffs(lm) - 1 : -1;
                    if (b >= 0) lm &= lm - 1;
                    if (t == team) mine = b;
                }
            }
            const int id = mine >= 0 ? (int)base + mine : -1;
            int first = 0, cnt = 0;
            if (id >= 0) {
                first = T == 1 ? link0 : node_link[id];
                cnt = T == 1 ? cnt0 : node_count[id];
                if (first < 0 || cnt < 1 || (int64_t)first + cnt > L.n) {
                    bad = true;
                    cnt = 0;
                }
            }
            // a leaf may hold more than T members (leaf_cap > T, or a
            // finest-level leaf): chunks of T, as many as the warp's largest
            const int nch = __reduce_max_sync(NB_FULL, (cnt + T - 1) / T);
            const float4 r0 = cnt > 0 ? pos4[first] : make_float4(0.f, 0.f, 0.f, 0.f);
            float2 M = make_float2(0.0f, 0.0f);
            float sx = 0.0f, sy = 0.0f, sz = 0.0f;
#pragma unroll kLeafUnroll
            for (int ch = 0; ch < nch; ch++) {
                const int k = ch * T + tl;
                if (k < cnt) {
                    const float4 p = pos4[first + k];
                    M = df_add(M, make_float2(p.w, 0.0f));
                    sx = fmaf(p.w, p.x - r0.x, sx);
                    sy = fmaf(p.w, p.y - r0.y, sy);
                    sz = fmaf(p.w, p.z - r0.z, sz);
                }
            }
#pragma unroll
            for (int o = T / 2; o > 0; o >>= 1) {
                const float2 Mo = make_float2(__shfl_xor_sync(NB_FULL, M.x, o),
                                              __shfl_xor_sync(NB_FULL, M.y, o));
                M = df_add(M, Mo);
                sx += __shfl_xor_sync(NB_FULL, sx, o);
                sy += __shfl_xor_sync(NB_FULL, sy, o);
                sz += __shfl_xor_sync(NB_FULL, sz, o);
            }
            float c[3] = {r0.x, r0.y, r0.z};
            if (M.x > 0.0f) {
                const float inv = 1.0f / M.x;
                c[0] = fmaf(sx, inv, c[0]); c[1] = fmaf(sy, inv, c[1]); c[2] = fmaf(sz, inv, c[2]);
            } else if (cnt > 0) {
                const CellF cell = node_cell(L, keys[node_start[id]], node_level[id], box);
#pragma unroll
                for (int a = 0; a < 3; a++) c[a] = cell.c[a];
            }
            float b2 = 0.0f;
            float q[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
#pragma unroll kLeafUnroll
            for (int ch = 0; ch < nch; ch++) {
                const int k = ch * T + tl;
                if (k < cnt) {
                    const float4 p = pos4[first + k];
                    const float dx = p.x - c[0], dy = p.y - c[1], dz = p.z - c[2];
                    const float r2 = fmaf(dz, dz, fmaf(dy, dy, dx * dx));
                    b2 = fmaxf(b2, r2);
                    if (nodeQ) quad_add(q, p.w, dx, dy, dz, r2);
                }
            }
#pragma unroll
            for (int o = T / 2; o > 0; o >>= 1) b2 = fmaxf(b2, __shfl_xor_sync(NB_FULL, b2, o));
            if (nodeQ) {
#pragma unroll
                for (int o = T / 2; o > 0; o >>= 1)
#pragma unroll
                    for (int j = 0; j < 6; j++) q[j] += __shfl_xor_sync(NB_FULL, q[j], o);
            }
            if (tl == 0 && cnt > 0) {
                write_node(id, c[0], c[1], c[2], M, __fsqrt_ru(b2) * kUp, G, first,
                           (cnt << 1) | 1, nodeA, nodeB, mass2);
                if (nodeQ) write_quad(id, q, nodeQ);
            }
        }
        // internal nodes: the chunk's leaf records are device-visible before
        // any lane counts a leaf in (the writers' fence, then the warp
        // barrier).  A climbing thread carries a member key (its leaf's first
        // particle): every ancestor's cell follows from it and the ancestor's
        // level, one up per step.
        __threadfence();
        __syncwarp();
        int node = id0, par = -1, level = 0;
        uint64_t key = 0;
        if (leaf) {
            par = par0;
            level = lev0;
            key = key0;
        }
        while (par >= 0) {       // a root has none
            if (par >= node) {   // parents precede their children
                bad = true;
                break;
            }
            // the parent's fields load beside the count-in atomic; the thread
            // that brings the last child computes the parent
            const int c0 = node_link[par], nc = node_nchild[par];
            const int up = node_parent[par];
            if (count_in(par, node_arrive) != nc) break;
            level--;
            if (!internal_node(L, par, c0, nc, level, key, refit, nn, box, G, node_count, nodeA,
                               nodeB, mass2, nodeQ))
                bad = true;  // still counted in above, so the counters stay consistent
            node_arrive[par] = 0;
            node = par;
            par = up;
        }
    }
    if (bad) atomicOr(&ds_status(ds), kStatusBadTree);
}

size_t tree_temp_bytes(int64_t n, int levels) {
    int64_t nblk = (n + TB - 1) / TB;
    return (size_t)(levels + 1) * (size_t)nblk * sizeof(uint32_t) + 256;
}

void build_tree(cudaStream_t s, const Layout &L, const uint64_t *keys, const float4 *pos4,
                const SysBox *d_box, const int64_t *d_off, int leaf_cap, float G,
                int64_t cap_nodes, int8_t *delta, int8_t *leaflev, void *temp, DevState *ds,
                int32_t *node_start, int8_t *node_level, int32_t *node_parent,
                int32_t *node_link, int32_t *node_count, int32_t *node_nchild,
                int32_t *node_arrive, float4 *nodeA, float4 *nodeB, float2 *mass2, float4 *nodeQ,
                int32_t *sys_root, int nsm) {
    const int nblk = (int)((L.n + TB - 1) / TB);
    uint32_t *blockcnt = (uint32_t *)temp;
    if (leaf_cap <= 8)
        leaflevel_kernel<8><<<(nblk + VB - 1) / VB, TB, 0, s>>>(L, leaf_cap, keys, delta, leaflev, blockcnt, nblk);
    else if (leaf_cap <= 16)
        leaflevel_kernel<16><<<(nblk + VB - 1) / VB, TB, 0, s>>>(L, leaf_cap, keys, delta, leaflev, blockcnt, nblk);
    else
        leaflevel_kernel<32><<<(nblk + VB - 1) / VB, TB, 0, s>>>(L, leaf_cap, keys, delta, leaflev, blockcnt, nblk);
    level_scan_kernel<<<L.levels + 1, LS_T, 0, s>>>(blockcnt, nblk, ds);
    level_offsets_kernel<<<1, 32, 0, s>>>(L.levels + 1, ds, cap_nodes);
    node_zero_kernel<<<nsm * 8, 256, 0, s>>>(ds, cap_nodes, node_nchild, node_arrive);
    nodes_kernel<<<nblk, TB, 0, s>>>(L, delta, leaflev, blockcnt, nblk, ds, cap_nodes, node_start,
                                     node_level, node_parent, node_link, node_count, node_nchild);
    sys_root_init_kernel<<<(L.nsys + 255) / 256, 256, 0, s>>>(L.nsys, sys_root);
    sys_root_kernel<<<(L.nsys + 255) / 256, 256, 0, s>>>(ds, node_start, d_off, L.nsys, sys_root);
    tree_moments(s, L, keys, pos4, d_box, leaf_cap, G, ds, node_start, node_level, node_parent,
                 node_link, node_count, node_nchild, node_arrive, nodeA, nodeB, mass2, nodeQ, nsm,
                 false);
}

// CTAs per SM of the warp-per-group passes (sphere, alpha), build-time tunable.
#ifndef NB_GROUP_CTAS_PER_SM
#define NB_GROUP_CTAS_PER_SM 8
#endif
// CTAs per SM of the moments pass (build-time tunable).
#ifndef NB_LEAF_CTAS_PER_SM
#define NB_LEAF_CTAS_PER_SM 64
#endif

// Moments of every node of the current tree from pos4 in one launch (one warp
// per 32 consecutive nodes for the leaves; internal nodes climb from the
// leaves).  The arrival counters must be zero: the build zeroes them and a
// completed pass leaves them zero.
void tree_moments(cudaStream_t s, const Layout &L, const uint64_t *keys, const float4 *pos4,
                  const SysBox *d_box, int leaf_cap, float G, DevState *ds,
                  const int32_t *node_start, const int8_t *node_level, const int32_t *node_parent,
                  const int32_t *node_link, int32_t *node_count, const int32_t *node_nchild,
                  int32_t *node_arrive, float4 *nodeA, float4 *nodeB, float2 *mass2,
                  float4 *nodeQ, int nsm, bool refit) {
    int64_t mb = (L.n / 4 + 255) / 256;
    if (mb > (int64_t)nsm * NB_LEAF_CTAS_PER_SM) mb = (int64_t)nsm * NB_LEAF_CTAS_PER_SM;
    if (mb < 1) mb = 1;
    const int rf = refit ? 1 : 0;
    // one lane per leaf up to leaf capacity 16 (each lane's member loads in
    // batches; measured fastest), teams of 8 lanes for larger leaves
    if (leaf_cap <= 16)
        moments_kernel<1><<<(int)mb, 256, 0, s>>>(L, rf, keys, pos4, d_box, G, ds, node_start,
                                                  node_level, node_parent, node_link, node_count,
                                                  node_nchild, node_arrive, nodeA, nodeB, mass2,
                                                  nodeQ);
    else
        moments_kernel<8><<<(int)mb, 256, 0, s>>>(L, rf, keys, pos4, d_box, G, ds, node_start,
                                                  node_level, node_parent, node_link, node_count,
                                                  node_nchild, node_arrive, nodeA, nodeB, mass2,
                                                  nodeQ);
}

// ---------------------------------------------------------------- groups
constexpr int FL_T = 1024, FL_IPT = 4, FL_CH = FL_T * FL_IPT;

// Groups (the particles that share one interaction list).  Under a node
// holding more than G particles, consecutive children that each hold at most
// G are packed greedily, in octant order, into runs of at most G particles;
// each run is one group.  A root holding at most G is one group, and a
// finest-level leaf holding more than G is cut into chunks of G.  Packing
// siblings keeps a group inside its parent's cell while filling the warp.
// Mark each group's first particle.
__global__ void group_mark_kernel(const DevState *__restrict__ ds, int G,
                                  const int32_t *__restrict__ node_start,
                                  const int32_t *__restrict__ node_parent,
                                  const int32_t *__restrict__ node_link,
                                  const int32_t *__restrict__ node_count,
                                  const int32_t *__restrict__ node_nchild, uint8_t *gflag) {
    const int nn = ds->nnodes;
    for (int id = blockIdx.x * blockDim.x + threadIdx.x; id < nn; id += gridDim.x * blockDim.x) {
        const int cnt = node_count[id], nc = node_nchild[id];
        if (cnt <= G) {
            if (node_parent[id] < 0) gflag[node_start[id]] = 1;
        } else if (nc == 0) {
            for (int k = 0; k < cnt; k += G) gflag[node_start[id] + k] = 1;
        } else {
            const int c0 = node_link[id];
            int run = 0;
            for (int c = c0; c < c0 + nc; c++) {
                const int cc = node_count[c];
                if (cc > G) {
                    run = 0;  // grouped below that child
                } else if (run == 0 || run + cc > G) {
                    gflag[node_start[c]] = 1;
                    run = cc;
                } else {
                    run += cc;
                }
            }
        }
    }
}

__device__ __forceinline__ uint32_t block_excl_scan_1024(uint32_t v, uint32_t *sh) {
    uint32_t incl = (uint32_t)warp_incl_scan((int)v);
    if (lane_id() == 31) sh[threadIdx.x >> 5] = incl;
    __syncthreads();
    if (threadIdx.x < 32) sh[threadIdx.x] = (uint32_t)warp_incl_scan((int)sh[threadIdx.x]);
    __syncthreads();
    uint32_t r = incl - v + ((threadIdx.x >> 5) ? sh[(threadIdx.x >> 5) - 1] : 0u);
    __syncthreads();
    return r;
}

__global__ void __launch_bounds__(FL_T) flag_count_kernel(const uint8_t *__restrict__ f, int64_t n,
                                                          uint32_t *bsum) {
    __shared__ uint32_t sh[32];
    int64_t base = (int64_t)blockIdx.x * FL_CH + threadIdx.x * FL_IPT;
    uint32_t t = 0;
    for (int k = 0; k < FL_IPT; k++)
        if (base + k < n) t += f[base + k];
    uint32_t incl = (uint32_t)warp_incl_scan((int)t);
    if (lane_id() == 31) sh[threadIdx.x >> 5] = incl;
    __syncthreads();
    if (threadIdx.x == 0) {
        uint32_t s = 0;
        for (int q = 0; q < 32; q++) s += sh[q];
        bsum[blockIdx.x] = s;
    }
}

__global__ void __launch_bounds__(FL_T) flag_write_kernel(const uint8_t *__restrict__ f, int64_t n,
                                                          const uint32_t *__restrict__ bsum,
                                                          int32_t *__restrict__ out) {
    __shared__ uint32_t sh[32];
    int64_t base = (int64_t)blockIdx.x * FL_CH + threadIdx.x * FL_IPT;
    uint32_t v[FL_IPT], t = 0;
    for (int k = 0; k < FL_IPT; k++) {
        v[k] = (base + k < n) ? f[base + k] : 0u;
        t += v[k];
    }
    uint32_t ex = block_excl_scan_1024(t, sh) + bsum[blockIdx.x];
    for (int k = 0; k < FL_IPT; k++) {
        if (v[k]) out[ex] = (int32_t)(base + k);
        ex += v[k];
    }
}

// Warp per group: count, bounding-box centre and enclosing radius, system.
__global__ void __launch_bounds__(256) group_info_kernel(Layout L, int G,
                                                         const float4 *__restrict__ pos4,
                                                         const int64_t *__restrict__ off,
                                                         const DevState *__restrict__ ds,
                                                         const int32_t *__restrict__ grp_first,
                                                         int32_t *grp_count, float4 *grp_sphere,
                                                         int32_t *grp_sys) {
    // a half-warp per group, two groups per warp at a time: both groups'
    // member loads are in flight together (min, max and the largest distance
    // do not depend on the order of the reduction)
    const int ng = ds->ngroups;
    const unsigned lane = lane_id(), sl = lane & 15u;
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nw = (gridDim.x * blockDim.x) >> 5;
    for (int g0 = 2 * warp; g0 < ng; g0 += 2 * nw) {
        const int g = g0 + (int)(lane >> 4);
        int first = 0, cnt = 0;
        if (g < ng) {
            first = grp_first[g];
            const int end = (g + 1 < ng) ? grp_first[g + 1] : (int)L.n;
            cnt = end - first;
        }
        float lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
#pragma unroll 4
        for (int k = (int)sl; k < cnt; k += 16) {
            float4 p = pos4[first + k];
            lo[0] = fminf(lo[0], p.x); hi[0] = fmaxf(hi[0], p.x);
            lo[1] = fminf(lo[1], p.y); hi[1] = fmaxf(hi[1], p.y);
            lo[2] = fminf(lo[2], p.z); hi[2] = fmaxf(hi[2], p.z);
        }
        for (int a = 0; a < 3; a++)
            for (int o = 8; o; o >>= 1) {
                lo[a] = fminf(lo[a], __shfl_xor_sync(NB_FULL, lo[a], o));
                hi[a] = fmaxf(hi[a], __shfl_xor_sync(NB_FULL, hi[a], o));
            }
        float c[3];
        for (int a = 0; a < 3; a++) c[a] = 0.5f * (lo[a] + hi[a]);
        float r2 = 0.0f;
#pragma unroll 4
        for (int k = (int)sl; k < cnt; k += 16) {
            float4 p = pos4[first + k];
            float dx = p.x - c[0], dy = p.y - c[1], dz = p.z - c[2];
            r2 = fmaxf(r2, dx * dx + dy * dy + dz * dz);
        }
        for (int o = 8; o; o >>= 1) r2 = fmaxf(r2, __shfl_xor_sync(NB_FULL, r2, o));
        if (sl == 0 && g < ng) {
            // rounded up so the sphere encloses every member despite FP32 error
            float r = __fsqrt_ru(r2) * (1.0f + 0x1p-20f);
            grp_count[g] = cnt;
            grp_sphere[g] = make_float4(c[0], c[1], c[2], r);
            grp_sys[g] = sys_of(off, L.nsys, first);
        }
    }
}

void build_groups(cudaStream_t s, const Layout &L, int group_size, const float4 *pos4,
                  const int64_t *d_off, const int32_t *node_start, const int32_t *node_parent,
                  const int32_t *node_count, const int32_t *node_nchild, const int32_t *node_link,
                  DevState *ds, uint8_t *gflag, void *temp, int32_t *grp_first,
                  int32_t *grp_count, float4 *grp_sphere, int32_t *grp_sys, int nsm) {

    cudaMemsetAsync(gflag, 0, (size_t)L.n, s);
    int mb = (int)((L.n + 255) / 256);
    if (mb > nsm * 16) mb = nsm * 16;
    group_mark_kernel<<<mb, 256, 0, s>>>(ds, group_size, node_start, node_parent, node_link, node_count,
                                         node_nchild, gflag);
    int nb = (int)((L.n + FL_CH - 1) / FL_CH);
    uint32_t *bsum = (uint32_t *)temp;
    flag_count_kernel<<<nb, FL_T, 0, s>>>(gflag, L.n, bsum);
    launch_scan_sums(s, bsum, nb, &ds->ngroups);
    flag_write_kernel<<<nb, FL_T, 0, s>>>(gflag, L.n, bsum, grp_first);
    int gb = nsm * NB_GROUP_CTAS_PER_SM;
    group_info_kernel<<<gb, 256, 0, s>>>(L, group_size, pos4, d_off, ds, grp_first, grp_count,
                                         grp_sphere, grp_sys);
}

// Spheres (and counts, systems) of the existing groups from pos4: after a
// refit the membership stays and only the geometry is recomputed.
void refit_groups(cudaStream_t s, const Layout &L, int group_size, const float4 *pos4,
                  const int64_t *d_off, DevState *ds, const int32_t *grp_first,
                  int32_t *grp_count, float4 *grp_sphere, int32_t *grp_sys, int nsm) {
    group_info_kernel<<<nsm * NB_GROUP_CTAS_PER_SM, 256, 0, s>>>(L, group_size, pos4, d_off, ds, grp_first, grp_count,
                                              grp_sphere, grp_sys);
}

// alpha_g = delta_acc * min over members of |a_old| (Eq. 2 per group).
__global__ void group_alpha_kernel(const DevState *__restrict__ ds,
                                   const int32_t *__restrict__ grp_first,
                                   const int32_t *__restrict__ grp_count,
                                   const float *__restrict__ aold, float dacc, float *grp_alpha) {
    // a half-warp per group, two groups per warp at a time (as group_info)
    const int ng = ds->ngroups;
    const unsigned lane = lane_id(), sl = lane & 15u;
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nw = (gridDim.x * blockDim.x) >> 5;
    for (int g0 = 2 * warp; g0 < ng; g0 += 2 * nw) {
        const int g = g0 + (int)(lane >> 4);
        int first = 0, cnt = 0;
        if (g < ng) {
            first = grp_first[g];
            cnt = grp_count[g];
        }
        float m = INFINITY;
#pragma unroll 4
        for (int k = (int)sl; k < cnt; k += 16) m = fminf(m, aold[first + k]);
        for (int o = 8; o; o >>= 1) m = fminf(m, __shfl_xor_sync(NB_FULL, m, o));
        if (sl == 0 && g < ng) grp_alpha[g] = dacc * m;
    }
}

void launch_group_alpha(cudaStream_t s, int64_t n, const DevState *ds, const int32_t *grp_first,
                        const int32_t *grp_count, const float *aold_sorted, float delta_acc,
                        float *grp_alpha, int nsm) {
    (void)n;
    group_alpha_kernel<<<nsm * NB_GROUP_CTAS_PER_SM, 256, 0, s>>>(ds, grp_first, grp_count, aold_sorted, delta_acc,
                                                grp_alpha);
}

}  // namespace nb
