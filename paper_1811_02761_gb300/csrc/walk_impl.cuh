// walk_impl.cuh -- the tree walk ("walkTree", the dominant kernel of the
// paper, Sect. 3 and Table 2).
//
// Design (GB300 re-think of Sect. 1's shared interaction list):
//   * persistent grid, one warp per i-group, groups popped from a device queue
//     (one atomicAdd per group); the queue order is Morton order or a cost
//     order chosen by the scheduler;
//   * each lane holds up to IPL i-particles (group <= 32*IPL particles) in
//     slots; the slots form runs, each a number of rows of the group times
//     a number of list splits, chosen per group size from a table so that
//     the flush issues the fewest instructions (lane_tiling below);
//   * traversal: a per-warp stack in shared memory whose entries are child
//     ranges (first node, count <= 8).  Each round the warp pops the top four
//     ranges (up to 32 nodes, one per lane), evaluates the MAC of Eq. 2
//     against the group's bounding sphere, and compacts the outcomes with
//     ballot/popc:
//       accepted node       -> its pseudo particle (com, M) joins the list,
//       opened internal node -> its child range is pushed,
//       opened leaf          -> its particles join the list;
//   * the list (float4 x, y, z, m in shared memory) is flushed whenever the
//     next append would overflow it: every lane evaluates Eq. 1 for its q
//     particles against its split of the entries, read as pairs (two LDS.128)
//     laid out for the packed FP32 instructions -- 12 FP32-pipe operations +
//     1 MUFU.RSQ per interaction;
//   * optional Neumaier compensation of the per-flush partial sums.
// No warp ever waits on another warp or CTA.
#pragma once

#include <cuda_runtime.h>

#include "internal.cuh"
#include "walk_tiling.cuh"

namespace nb {

__device__ __forceinline__ void neumaier_add(float &s, float &c, float x) {
    float t = s + x;
    if (fabsf(s) >= fabsf(x))
        c += (s - t) + x;
    else
        c += (x - t) + s;
    s = t;
}

// The interaction list of a warp holds entries in pairs, structure-of-arrays
// within the pair, the two halves of a pair side by side: L[2k] = (x_2k,
// x_2k+1, y_2k, y_2k+1) and L[2k+1] = (z_2k, z_2k+1, m_2k, m_2k+1).  Two
// LDS.128 broadcasts from one address register then give every lane two
// entries laid out for Blackwell's packed FP32 instructions (FFMA2/FADD2/
// FMUL2), which evaluate Eq. 1 for both entries against one i-particle in one
// instruction each -- half the issue slots of scalar code, which is what
// bounds this loop.
__device__ __forceinline__ void list_put(float4 *L, int e, float4 v) {
    float *p = reinterpret_cast<float *>(L + 2 * (e >> 1)) + (e & 1);
    p[0] = v.x;
    p[2] = v.y;
    p[4] = v.z;
    p[6] = v.w;
}

// Unroll depth of the flush loop over entry pairs (build-time tunable).
#ifndef NB_FLUSH_UNROLL
#define NB_FLUSH_UNROLL 1
#endif
constexpr int kFlushUnroll = NB_FLUSH_UNROLL;

// Per-lane i-slot state: negated position, broadcast to both halves of a
// packed pair, and the running sums of (ax, ay, az, phi): packed pairs that
// every flush accumulates into (plain), or scalars with Neumaier compensation
// that take each flush's packed partial sums (compensated).  Only the members
// a variant uses occupy registers.
template <int IPL>
struct ISlots {
    float2 nx[IPL], ny[IPL], nz[IPL];
    float mi[IPL];
    float2 run[IPL][4];
    float acc[IPL][4], cmp[IPL][4];
};

// Eq. 1 for the first NQ i-slots of a lane against its share of the nl list
// entries: the entry pairs k0, k0 + ks, k0 + 2 ks, ... (see the lane tiling
// below).  Plain sums accumulate straight into the packed running sums; with
// COMP each flush forms packed partial sums that are folded into the running
// sums at its end with Neumaier compensation.
template <int J0, int NQ, int IPL, bool PHI, bool COMP, bool SAFE>
__device__ __forceinline__ void flush_list(float4 *L, int nl, float eps2, int k0, int ks,
                                           ISlots<IPL> &I) {
    if (nl & 1) {  // pad to a whole pair with a massless, distant entry
        if (lane_id() == 0) list_put(L, nl, make_float4(1e18f, 1e18f, 1e18f, 0.0f));
        __syncwarp();
    }
    const int np = (nl + 1) >> 1;
    const float2 e2 = make_float2(eps2, eps2);
    const float2 neg1 = make_float2(-1.0f, -1.0f);
    float2 sx[NQ], sy[NQ], sz[NQ], sp[NQ];
#pragma unroll
    for (int q = 0; q < NQ; q++) {
        if constexpr (COMP) {
            sx[q] = sy[q] = sz[q] = sp[q] = make_float2(0.0f, 0.0f);
        } else {
            sx[q] = I.run[J0 + q][0];
            sy[q] = I.run[J0 + q][1];
            sz[q] = I.run[J0 + q][2];
            sp[q] = I.run[J0 + q][3];
        }
    }
    // this lane's pairs k0, k0 + ks, ... < np (idle lanes: k0 >= np)
    const float4 *pe = L + 2 * np;
    const int step = 2 * ks;
#pragma unroll kFlushUnroll
    for (const float4 *pk = L + 2 * min(k0, np); pk < pe; pk += step) {
        const float4 A = pk[0], B = pk[1];
        const float2 px = make_float2(A.x, A.y), py = make_float2(A.z, A.w);
        const float2 pz = make_float2(B.x, B.y), pm = make_float2(B.z, B.w);
#pragma unroll
        for (int q = 0; q < NQ; q++) {
            const float2 dx = __fadd2_rn(px, I.nx[J0 + q]);
            const float2 dy = __fadd2_rn(py, I.ny[J0 + q]);
            const float2 dz = __fadd2_rn(pz, I.nz[J0 + q]);
            float2 r2 = __ffma2_rn(dx, dx, e2);
            r2 = __ffma2_rn(dy, dy, r2);
            r2 = __ffma2_rn(dz, dz, r2);
            float2 ri = make_float2(rsqrt_fast(r2.x), rsqrt_fast(r2.y));
            if constexpr (SAFE) {
                ri.x = r2.x >= 1.17549435e-38f ? ri.x : 0.0f;
                ri.y = r2.y >= 1.17549435e-38f ? ri.y : 0.0f;
            }
            const float2 mr = __fmul2_rn(pm, ri);
            const float2 w3 = __fmul2_rn(__fmul2_rn(mr, ri), ri);
            sx[q] = __ffma2_rn(w3, dx, sx[q]);
            sy[q] = __ffma2_rn(w3, dy, sy[q]);
            sz[q] = __ffma2_rn(w3, dz, sz[q]);
            if constexpr (PHI) sp[q] = __ffma2_rn(mr, neg1, sp[q]);
        }
    }
#pragma unroll
    for (int q = 0; q < NQ; q++) {
        if constexpr (COMP) {
            const float part[4] = {sx[q].x + sx[q].y, sy[q].x + sy[q].y, sz[q].x + sz[q].y,
                                   sp[q].x + sp[q].y};
#pragma unroll
            for (int c = 0; c < 4; c++) neumaier_add(I.acc[J0 + q][c], I.cmp[J0 + q][c], part[c]);
        } else {
            I.run[J0 + q][0] = sx[q];
            I.run[J0 + q][1] = sy[q];
            I.run[J0 + q][2] = sz[q];
            I.run[J0 + q][3] = sp[q];
        }
    }
}

// Quadrupole nodes (an extension beyond the paper's monopoles).  The node
// list holds entries in pairs, five float4 per pair, each component of the
// two entries side by side: (x, y), (z, M), (Qxx, Qyy), (Qzz, Qxy),
// (Qxz, Qyz) -- the layout of the packed FP32 instructions, as for the
// particle list.
__device__ __forceinline__ void quad_put(float4 *LQ, int e, float4 A, float4 Q0, float4 Q1) {
    float *p = reinterpret_cast<float *>(LQ + 5 * (e >> 1));
    const int h = e & 1;
    p[0 + h] = A.x;
    p[2 + h] = A.y;
    p[4 + h] = A.z;
    p[6 + h] = A.w;
    p[8 + h] = Q0.x;
    p[10 + h] = Q0.y;
    p[12 + h] = Q0.z;
    p[14 + h] = Q0.w;
    p[16 + h] = Q1.x;
    p[18 + h] = Q1.y;
}

// For each node entry (com, M, Q) and each of the lane's first NQ i-slots,
// with d = com - r_i softened as r^2 = |d|^2 + eps^2,
//     a += M d / r^3 - Q d / r^5 + (5/2) (d.Q.d) d / r^7,
//     phi -= M / r + (d.Q.d) / (2 r^5),
// the negative gradient of the node's monopole + quadrupole potential,
// evaluated for two entries per packed instruction.  The lane takes the
// entry pairs k0, k0 + ks, ... like the particle flush.
template <int J0, int NQ, int IPL, bool PHI, bool COMP, bool SAFE>
__device__ __forceinline__ void flush_quad_list(float4 *LQ, int nq, float eps2, int k0, int ks,
                                                ISlots<IPL> &I) {
    if (nq & 1) {  // pad to a whole pair with a massless, distant entry
        if (lane_id() == 0)
            quad_put(LQ, nq, make_float4(1e18f, 1e18f, 1e18f, 0.0f), make_float4(0.f, 0.f, 0.f, 0.f),
                     make_float4(0.f, 0.f, 0.f, 0.f));
        __syncwarp();
    }
    const int np = (nq + 1) >> 1;
    const float2 e2 = make_float2(eps2, eps2);
    const float2 c25 = make_float2(2.5f, 2.5f), neg1 = make_float2(-1.0f, -1.0f);
    const float2 half = make_float2(0.5f, 0.5f);
    float2 sx[NQ], sy[NQ], sz[NQ], sp[NQ];
#pragma unroll
    for (int q = 0; q < NQ; q++) {
        if constexpr (COMP) {
            sx[q] = sy[q] = sz[q] = sp[q] = make_float2(0.0f, 0.0f);
        } else {
            sx[q] = I.run[J0 + q][0];
            sy[q] = I.run[J0 + q][1];
            sz[q] = I.run[J0 + q][2];
            sp[q] = I.run[J0 + q][3];
        }
    }
    for (int k = k0; k < np; k += ks) {
        const float4 F0 = LQ[5 * k], F1 = LQ[5 * k + 1], F2 = LQ[5 * k + 2], F3 = LQ[5 * k + 3],
                     F4 = LQ[5 * k + 4];
        const float2 px = make_float2(F0.x, F0.y), py = make_float2(F0.z, F0.w);
        const float2 pz = make_float2(F1.x, F1.y), pm = make_float2(F1.z, F1.w);
        const float2 qxx = make_float2(F2.x, F2.y), qyy = make_float2(F2.z, F2.w);
        const float2 qzz = make_float2(F3.x, F3.y), qxy = make_float2(F3.z, F3.w);
        const float2 qxz = make_float2(F4.x, F4.y), qyz = make_float2(F4.z, F4.w);
#pragma unroll
        for (int q = 0; q < NQ; q++) {
            const float2 dx = __fadd2_rn(px, I.nx[J0 + q]);
            const float2 dy = __fadd2_rn(py, I.ny[J0 + q]);
            const float2 dz = __fadd2_rn(pz, I.nz[J0 + q]);
            float2 r2 = __ffma2_rn(dx, dx, e2);
            r2 = __ffma2_rn(dy, dy, r2);
            r2 = __ffma2_rn(dz, dz, r2);
            float2 ri = make_float2(rsqrt_fast(r2.x), rsqrt_fast(r2.y));
            if constexpr (SAFE) {
                ri.x = r2.x >= 1.17549435e-38f ? ri.x : 0.0f;
                ri.y = r2.y >= 1.17549435e-38f ? ri.y : 0.0f;
            }
            const float2 ri2 = __fmul2_rn(ri, ri);
            const float2 ri3 = __fmul2_rn(ri, ri2);
            const float2 ri5 = __fmul2_rn(ri3, ri2);
            const float2 gx = __ffma2_rn(qxx, dx, __ffma2_rn(qxy, dy, __fmul2_rn(qxz, dz)));
            const float2 gy = __ffma2_rn(qxy, dx, __ffma2_rn(qyy, dy, __fmul2_rn(qyz, dz)));
            const float2 gz = __ffma2_rn(qxz, dx, __ffma2_rn(qyz, dy, __fmul2_rn(qzz, dz)));
            const float2 dqd = __ffma2_rn(dx, gx, __ffma2_rn(dy, gy, __fmul2_rn(dz, gz)));
            const float2 c = __ffma2_rn(__fmul2_rn(c25, dqd), __fmul2_rn(ri5, ri2), __fmul2_rn(pm, ri3));
            const float2 nri5 = __fmul2_rn(ri5, neg1);
            sx[q] = __ffma2_rn(c, dx, __ffma2_rn(gx, nri5, sx[q]));
            sy[q] = __ffma2_rn(c, dy, __ffma2_rn(gy, nri5, sy[q]));
            sz[q] = __ffma2_rn(c, dz, __ffma2_rn(gz, nri5, sz[q]));
            if constexpr (PHI)
                sp[q] = __ffma2_rn(__fmul2_rn(half, dqd), nri5, __ffma2_rn(pm, __fmul2_rn(ri, neg1), sp[q]));
        }
    }
#pragma unroll
    for (int q = 0; q < NQ; q++) {
        if constexpr (COMP) {
            const float part[4] = {sx[q].x + sx[q].y, sy[q].x + sy[q].y, sz[q].x + sz[q].y,
                                   sp[q].x + sp[q].y};
#pragma unroll
            for (int c = 0; c < 4; c++) neumaier_add(I.acc[J0 + q][c], I.cmp[J0 + q][c], part[c]);
        } else {
            I.run[J0 + q][0] = sx[q];
            I.run[J0 + q][1] = sy[q];
            I.run[J0 + q][2] = sz[q];
            I.run[J0 + q][3] = sp[q];
        }
    }
}

// Lane tiling of a group of cnt particles (walk_tiling.cuh, written by
// gen_tiling.py): the slots of a lane form runs; run k has r_k slots, P_k
// rows and s_k = floor(32 / P_k) splits.  Lane L is row L % P_k of split
// L / P_k (idle in run k when L / P_k >= s_k), its t-th slot of the run holds
// particle base_k + row + P_k t, and it takes every s_k-th entry pair of the
// list from pair L / P_k on.  One flush loop serves a run.  The table picks,
// for every cnt, the runs with the fewest issued instructions per list entry
// (the loop's loads and control once per pair, the arithmetic once per slot).
struct Tiling {
    uint64_t code;  // the table entry: number of runs, then (r, P, s) per run
    int k0[3];      // this lane's first entry pair in each run (idle: 1 << 30)
};
__device__ __forceinline__ int run_field(uint64_t code, int k, int shift, int bits) {
    return (int)((code >> (2 + 16 * k + shift)) & ((1u << bits) - 1u));
}
__device__ __forceinline__ int run_r(uint64_t code, int k) { return run_field(code, k, 0, 4); }
__device__ __forceinline__ int run_P(uint64_t code, int k) { return run_field(code, k, 4, 6); }
__device__ __forceinline__ int run_s(uint64_t code, int k) { return run_field(code, k, 10, 6); }

template <int IPL>
__device__ __forceinline__ Tiling lane_tiling(int cnt) {
    // a group larger than the slots allow (flagged by the caller) still gets
    // a well-formed layout: the largest one
    const int c = cnt < 1 ? 1 : (cnt > 32 * IPL ? 32 * IPL : cnt);
    Tiling t;
    t.code = __ldg(&kTiling[IPL - 1][c]);
    const int nr = (int)(t.code & 3u), lane = (int)lane_id();
#pragma unroll
    for (int k = 0; k < 3; k++) {
        const int P = k < nr ? run_P(t.code, k) : 32, s = k < nr ? run_s(t.code, k) : 1;
        const int split = lane / P;
        t.k0[k] = (k < nr && split < s) ? split : (1 << 30);
    }
    return t;
}

// The flush loops of the runs from slot J on (run K).
template <int J, int K, int IPL, bool PHI, bool COMP, bool SAFE, bool QUADL>
__device__ __forceinline__ void flush_runs(const Tiling &t, float4 *L, int nl, float eps2,
                                           ISlots<IPL> &I) {
    if constexpr (J < IPL && K < 3) {
        if (K >= (int)(t.code & 3u)) return;
        const int r = run_r(t.code, K), ks = run_s(t.code, K), k0 = t.k0[K];
#define NB_FLUSH(R)                                                                            \
    do {                                                                                       \
        if constexpr (QUADL) flush_quad_list<J, R, IPL, PHI, COMP, SAFE>(L, nl, eps2, k0, ks, I); \
        else flush_list<J, R, IPL, PHI, COMP, SAFE>(L, nl, eps2, k0, ks, I);                  \
    } while (0)
        if constexpr (J + 4 <= IPL) {
            if (r == 4) { NB_FLUSH(4); return; }
        }
        if constexpr (J + 3 <= IPL) {
            if (r == 3) { NB_FLUSH(3); flush_runs<J + 3, K + 1, IPL, PHI, COMP, SAFE, QUADL>(t, L, nl, eps2, I); return; }
        }
        if constexpr (J + 2 <= IPL) {
            if (r == 2) { NB_FLUSH(2); flush_runs<J + 2, K + 1, IPL, PHI, COMP, SAFE, QUADL>(t, L, nl, eps2, I); return; }
        }
        NB_FLUSH(1);
        flush_runs<J + 1, K + 1, IPL, PHI, COMP, SAFE, QUADL>(t, L, nl, eps2, I);
#undef NB_FLUSH
    }
}

// Run k, slot t within it, of the lane's slot j (j < the slots in use).
__device__ __forceinline__ void slot_run(uint64_t code, int j, int &k, int &t) {
    const int r0 = run_r(code, 0), r1 = run_r(code, 1);
    k = j < r0 ? 0 : (j < r0 + r1 ? 1 : 2);
    t = j - (k == 0 ? 0 : (k == 1 ? r0 : r0 + r1));
}
__device__ __forceinline__ int slots_used(uint64_t code) {
    const int nr = (int)(code & 3u);
    return (nr > 0 ? run_r(code, 0) : 0) + (nr > 1 ? run_r(code, 1) : 0) + (nr > 2 ? run_r(code, 2) : 0);
}

// A group's i-particles into the lanes' slots (past the group's end, or on an
// idle row: massless copies of the sphere centre) and zeroed sums.
template <int IPL>
__device__ __forceinline__ void load_slots(const Tiling &tile, const float4 *__restrict__ pos4,
                                           int first, int cnt, float4 sph, ISlots<IPL> &I) {
    const int lane = (int)lane_id(), used = slots_used(tile.code);
#pragma unroll
    for (int q = 0; q < IPL; q++) {
        int k = 0, t = 0;
        slot_run(tile.code, q, k, t);
        const int P = run_P(tile.code, k);
        const int base = k == 0 ? 0 : run_r(tile.code, 0) * run_P(tile.code, 0) +
                                          (k == 2 ? run_r(tile.code, 1) * run_P(tile.code, 1) : 0);
        const int idx = base + lane % P + P * t;
        const float4 p = (q < used && idx < cnt) ? pos4[first + idx]
                                                 : make_float4(sph.x, sph.y, sph.z, 0.0f);
        I.nx[q] = make_float2(-p.x, -p.x);
        I.ny[q] = make_float2(-p.y, -p.y);
        I.nz[q] = make_float2(-p.z, -p.z);
        I.mi[q] = p.w;
#pragma unroll
        for (int c = 0; c < 4; c++) {
            I.acc[q][c] = I.cmp[q][c] = 0.0f;
            I.run[q][c] = make_float2(0.0f, 0.0f);
        }
    }
}

// End of a group: the s_k splits of every row are summed onto split 0 in
// split order (with compensation: Neumaier), then the results are written (G
// applied once; the potential's self term removed).
template <int IPL, bool PHI, bool COMP, bool SAFE>
__device__ __forceinline__ void finish_group(const Tiling &tile, int first, int cnt, float eps2,
                                             const WalkArgs &a, ISlots<IPL> &I) {
    const int lane = (int)lane_id(), used = slots_used(tile.code);
    const float G = a.G;
    const float self = SAFE ? 0.0f : rsqrt_fast(eps2);
#pragma unroll
    for (int q = 0; q < IPL; q++) {
        if (q < used) {  // warp-uniform
            int k = 0, t = 0;
            slot_run(tile.code, q, k, t);
            const int P = run_P(tile.code, k), s = run_s(tile.code, k);
            const int base = k == 0 ? 0 : run_r(tile.code, 0) * run_P(tile.code, 0) +
                                              (k == 2 ? run_r(tile.code, 1) * run_P(tile.code, 1) : 0);
            const int row = lane % P, split = lane / P;
            float r[4];
#pragma unroll
            for (int c = 0; c < 4; c++) {
                if (c == 3 && !PHI) {
                    r[c] = 0.0f;
                    continue;
                }
                if constexpr (COMP) {
                    for (int u = 1; u < s; u++) {
                        const float v = __shfl_sync(NB_FULL, I.acc[q][c] + I.cmp[q][c], row + P * u);
                        if (split == 0) neumaier_add(I.acc[q][c], I.cmp[q][c], v);
                    }
                    r[c] = I.acc[q][c] + I.cmp[q][c];
                } else {
                    float v = I.run[q][c].x + I.run[q][c].y;
                    float sum = v;
                    for (int u = 1; u < s; u++) sum += __shfl_sync(NB_FULL, v, row + P * u);
                    r[c] = sum;
                }
            }
            const int idx = base + row + P * t;
            if (split == 0 && idx < cnt) {
                const float ph = PHI ? G * (r[3] + I.mi[q] * self) : 0.0f;
                const int i = first + idx;
                if (a.perm) {
                    const int o = a.perm[i];
                    a.ax[o] = G * r[0];
                    a.ay[o] = G * r[1];
                    a.az[o] = G * r[2];
                    if (PHI && a.phi) a.phi[o] = ph;
                } else {
                    a.acc_sorted[i] = make_float4(G * r[0], G * r[1], G * r[2], ph);
                }
            }
        }
    }
}

// Register budget of the walk kernel per thread: 64 (32 resident warps per
// SM) while a lane holds at most two i-particles; more slots need more
// registers for the positions and sums they keep (build-time tunable).
#ifndef NB_WALK_REGS_2
#define NB_WALK_REGS_2 64
#endif
#ifndef NB_WALK_REGS_3
#define NB_WALK_REGS_3 80
#endif
#ifndef NB_WALK_REGS_4
#define NB_WALK_REGS_4 96
#endif
template <int IPL>
constexpr int walk_regs() {
    return IPL <= 2 ? NB_WALK_REGS_2 : (IPL == 3 ? NB_WALK_REGS_3 : NB_WALK_REGS_4);
}

template <int IPL, bool PHI, bool COMP, bool SAFE, bool QUAD>
__global__ void __maxnreg__(walk_regs<IPL>()) walk_kernel(WalkArgs a, int geometric) {
    extern __shared__ __align__(16) unsigned char walk_smem[];
    const int D = a.list_depth, S = a.stack_depth;
    const int DQ = QUAD ? walk_quad_depth(D) : 0;
    const unsigned lane = lane_id(), w = threadIdx.x >> 5;
    // per warp: the paired list (D entries = D/2 pairs in LA), with
    // quadrupoles the paired node list (DQ entries, 40 B each), the stack and
    // kWalkScratch words for the leaf compaction
    const size_t per_warp = walk_smem_per_warp(D, S, QUAD);
    float4 *LA = reinterpret_cast<float4 *>(walk_smem + w * per_warp);
    float4 *LQ = LA + D;
    uint32_t *stk = reinterpret_cast<uint32_t *>(walk_smem + w * per_warp + (size_t)D * sizeof(float4) +
                                                 (size_t)DQ * 40);
    int *scr = reinterpret_cast<int *>(stk + S);
    DevState *ds = a.ds;
    const int ng = a.nactive ? *a.nactive : ds->ngroups;
    const int nnodes = ds->nnodes;
    const int npart = (int)a.n;
    const unsigned lt = lanemask_lt();
    int max_sp = 0;
    unsigned long long warp_entries = 0, warp_inter = 0, warp_quad = 0;
    bool overflow = false, bad = false;

    for (;;) {
        int qi = 0;
        if (lane == 0) qi = atomicAdd(&ds->queue_head, 1);
        qi = __shfl_sync(NB_FULL, qi, 0);
        if (qi >= ng) break;
        const int g = a.order ? a.order[qi] : qi;
        const int first = a.grp_first[g], cnt = a.grp_count[g];
        const float4 sph = a.grp_sphere[g];
        const float alpha = geometric ? 0.0f : a.grp_alpha[g];
        const int sys = a.grp_sys[g];
        const float eps2 = a.sys_eps2[sys];
        const int root = a.sys_root[sys];

        if (cnt > 32 * IPL) bad = true;  // larger than the group size allows
        const Tiling tile = lane_tiling<IPL>(cnt);

        ISlots<IPL> I;
        load_slots<IPL>(tile, a.pos4, first, cnt, sph, I);

        if (lane == 0) stk[0] = (uint32_t)root << 3;  // one node: the system's root
        int sp = 1, nl = 0, nq = 0;
        long long entries = 0, qentries = 0;
        __syncwarp();
        while (sp > 0) {
            // ---- pop the top four child ranges (<= 8 nodes each): lane L takes
            // node L % 8 of range L / 8.  Opened internal nodes have close to 8
            // children, so the lanes stay nearly full without a scan of the
            // range sizes (a scan costs a chain of dependent shuffles per round).
            const int take = sp < 4 ? sp : 4;
            const int rr = (int)(lane >> 3), jj = (int)(lane & 7);
            uint32_t e = 0;
            if (rr < take) e = stk[sp - 1 - rr];
            const int node = (int)(e >> 3) + jj;
            const bool slot = rr < take && jj <= (int)(e & 7u);
            const bool in_range = node >= 0 && node < nnodes;
            if (slot && !in_range) bad = true;
            const bool has = slot && in_range;
            sp -= take;
            __syncwarp();

            // ---- MAC (Eq. 2) against the group's bounding sphere
            // every lane loads (a lane without a node reads node 0): no branch
            const int nd = has ? node : 0;
            const float4 A = __ldg(&a.nodeA[nd]), B = __ldg(&a.nodeB[nd]);
            const float dx = A.x - sph.x, dy = A.y - sph.y, dz = A.z - sph.z;
            const float d = sqrt_fast(fmaf(dz, dz, fmaf(dy, dy, dx * dx))) - sph.w;
            bool accept;
            if (geometric) {
                accept = has && d > B.x && B.x <= a.theta * d;
            } else {
                const float d2 = d * d;
                accept = has && d > B.x && B.y <= alpha * (d2 * d2);
            }
            const int link = __float_as_int(B.z), meta = __float_as_int(B.w);
            const bool leaf = (meta & 1) != 0;
            const int mcount = meta >> 1;
            const bool open_leaf = has && !accept && leaf;
            // children sit on the next level, so their ids exceed the parent's:
            // a descent that does not increase the id would be a corrupt tree
            const bool bad_link = has && !accept && !leaf &&
                                  (link <= node || mcount < 1 || mcount > 8 || link + mcount > nnodes);
            if (bad_link) bad = true;
            const bool open_node = has && !accept && !leaf && !bad_link;

            // ---- push the child ranges of opened internal nodes
            const unsigned om = __ballot_sync(NB_FULL, open_node);
            const int npush = __popc(om);
            if (open_node) {
                const int pos = sp + __popc(om & lt);
                if (pos < S) stk[pos] = ((uint32_t)link << 3) | (uint32_t)(mcount - 1);
            }
            sp += npush;
            if (sp > S) {
                overflow = true;
                sp = S;
            }
            if (sp > max_sp) max_sp = sp;

            // ---- accepted nodes join the list (with quadrupoles: the node list)
            const unsigned am = __ballot_sync(NB_FULL, accept);
            const int na = __popc(am);
            if constexpr (QUAD) {
                if (nq + na > DQ) {
                    __syncwarp();
                    flush_runs<0, 0, IPL, PHI, COMP, SAFE, true>(tile, LQ, nq, eps2, I);
                    qentries += nq;
                    nq = 0;
                    __syncwarp();
                }
                if (accept)
                    quad_put(LQ, nq + __popc(am & lt), A, __ldg(&a.nodeQ[2 * node]),
                             __ldg(&a.nodeQ[2 * node + 1]));
                nq += na;
            } else {
                if (nl + na > D) {
                    __syncwarp();
                    flush_runs<0, 0, IPL, PHI, COMP, SAFE, false>(tile, LA, nl, eps2, I);
                    entries += nl;
                    nl = 0;
                    __syncwarp();
                }
                if (accept) list_put(LA, nl + __popc(am & lt), A);
                nl += na;
            }

            // ---- particles of opened leaves join the list, 32 per chunk: the
            // opened leaves are compacted to lanes 0..nlf-1 (through the warp's
            // scratch words), their counts scanned, and each chunk's slots are
            // mapped to their leaf with a bit map of the leaf starts, as in the
            // pop above -- one load latency per 32 particles, not per leaf
            const bool leaf_ok = open_leaf && link >= 0 && mcount >= 1 && link + mcount <= npart;
            if (open_leaf && !leaf_ok) bad = true;
            const unsigned lm = __ballot_sync(NB_FULL, leaf_ok);
            if (lm) {
                const int nlf = __popc(lm);
                if (leaf_ok) scr[__popc(lm & lt)] = (int)lane;
                __syncwarp();
                const int src = (int)lane < nlf ? scr[lane] : 0;
                const int lf = __shfl_sync(NB_FULL, link, src);
                const int lcs = __shfl_sync(NB_FULL, mcount, src);
                const int lc = (int)lane < nlf ? lcs : 0;
                const int lincl = warp_incl_scan(lc);
                const int lexcl = lincl - lc;
                const int total = __shfl_sync(NB_FULL, lincl, 31);
                for (int base = 0; base < total; base += 32) {
                    const int c = (total - base) < 32 ? (total - base) : 32;
                    if (nl + c > D) {
                        __syncwarp();
                        flush_runs<0, 0, IPL, PHI, COMP, SAFE, false>(tile, LA, nl, eps2, I);
                        entries += nl;
                        nl = 0;
                        __syncwarp();
                    }
                    // leaves are in increasing start order with counts >= 1, so
                    // the owner of slot base+lane is the last leaf starting at
                    // or before it: those before the chunk plus the starts
                    // inside it up to this lane
                    const bool starts = lc > 0 && lexcl >= base && lexcl < base + 32;
                    const unsigned smap = __reduce_or_sync(NB_FULL, starts ? 1u << (lexcl - base) : 0u);
                    const int before = __popc(__ballot_sync(NB_FULL, lc > 0 && lexcl < base));
                    const int k = before + __popc(smap & (0xffffffffu >> (31 - lane))) - 1;
                    const int of = __shfl_sync(NB_FULL, lf, k & 31);
                    const int oex = __shfl_sync(NB_FULL, lexcl, k & 31);
                    if ((int)lane < c) list_put(LA, nl + lane, __ldg(&a.pos4[of + base + (int)lane - oex]));
                    nl += c;
                }
            }
            __syncwarp();
        }
        if (nl > 0) {
            __syncwarp();
            flush_runs<0, 0, IPL, PHI, COMP, SAFE, false>(tile, LA, nl, eps2, I);
            entries += nl;
            nl = 0;
        }
        if constexpr (QUAD) {
            if (nq > 0) {
                __syncwarp();
                flush_runs<0, 0, IPL, PHI, COMP, SAFE, true>(tile, LQ, nq, eps2, I);
                qentries += nq;
                nq = 0;
            }
        }
        __syncwarp();

        finish_group<IPL, PHI, COMP, SAFE>(tile, first, cnt, eps2, a, I);
        entries += qentries;
        if (lane == 0 && a.grp_cost) a.grp_cost[g] = (int32_t)entries;
        warp_entries += (unsigned long long)entries;
        warp_inter += (unsigned long long)entries * (unsigned long long)cnt;
        warp_quad += (unsigned long long)qentries * (unsigned long long)cnt;
    }
    if (lane == 0) {
        atomicMax(&ds->max_stack, max_sp);
        if (warp_entries) {
            atomicAdd(&ds->list_entries, warp_entries);
            atomicAdd(&ds->interactions, warp_inter);
        }
        if (QUAD && warp_quad) atomicAdd(&ds->quad_entries, warp_quad);
        if (overflow) atomicOr(&ds->status, kStatusStackOverflow);
    }
    if (bad) atomicOr(&ds->status, kStatusBadTree);
}

template <int IPL, bool QUAD>
cudaError_t launch_walk_ipl(cudaStream_t s, const WalkArgs &a, const WalkShape &sh, int nsm) {
    const int threads = 32 * sh.warps_per_block;
    const size_t smem =
        (size_t)sh.warps_per_block * walk_smem_per_warp(a.list_depth, a.stack_depth, QUAD);
    void (*k)(WalkArgs, int);
    if (sh.potential) {
        if (sh.compensated) k = sh.safe ? walk_kernel<IPL, true, true, true, QUAD> : walk_kernel<IPL, true, true, false, QUAD>;
        else k = sh.safe ? walk_kernel<IPL, true, false, true, QUAD> : walk_kernel<IPL, true, false, false, QUAD>;
    } else {
        if (sh.compensated) k = sh.safe ? walk_kernel<IPL, false, true, true, QUAD> : walk_kernel<IPL, false, true, false, QUAD>;
        else k = sh.safe ? walk_kernel<IPL, false, false, true, QUAD> : walk_kernel<IPL, false, false, false, QUAD>;
    }
    cudaError_t err = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (err != cudaSuccess) return err;
    int per_sm = 0;
    err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, threads, smem);
    if (err != cudaSuccess) return err;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    if (sh.warps_launched) *sh.warps_launched = nsm * per_sm * sh.warps_per_block;
    k<<<nsm * per_sm, threads, smem, s>>>(a, sh.geometric ? 1 : 0);
    return cudaGetLastError();
}

}  // namespace nb
