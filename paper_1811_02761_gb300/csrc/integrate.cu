// integrate.cu -- leapfrog kick-drift-kick on the sorted particle state, state
// permutation after each re-sort, and FP64 energy/momentum diagnostics.
//
// The paper's code integrates with a second-order Runge-Kutta predictor /
// corrector under block time steps (Sect. 1, Table 2 "predict"/"correct");
// this library uses the (also second-order) leapfrog with a shared step.
// Positions are FP64 so that x += v dt keeps its low bits at large N;
// velocities and accelerations are FP32.
#include <cuda_runtime.h>

#include "internal.cuh"

namespace nb {

static inline int grid_for(int64_t n, int threads = 256) {
    int64_t b = (n + threads - 1) / threads;
    return (int)(b > 65535 * 8 ? 65535 * 8 : (b < 1 ? 1 : b));
}

#define NB_GRID_LOOP(i, n) \
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < (n); i += (int64_t)gridDim.x * blockDim.x)

// |a| as the next step's a_old (one expression for every kernel that sets it).
__device__ __forceinline__ float acc_mag(float4 a) {
    return sqrtf(fmaf(a.z, a.z, fmaf(a.y, a.y, a.x * a.x)));
}

// hclose != 0: first the closing half kick of the previous step (and its
// a_old), fused into this pass; the same two roundings as two kernels.
__global__ void kick_drift_kernel(int64_t n, StepState st, const float4 *__restrict__ acc,
                                  float hclose, float hdt, double dt, float4 *pos4) {
    NB_GRID_LOOP(i, n) {
        const float4 a = acc[i];
        float vx = st.vx[i], vy = st.vy[i], vz = st.vz[i];
        const double x0 = st.x[i], y0 = st.y[i], z0 = st.z[i];
        const float m = pos4 ? st.m[i] : 0.0f;
        if (hclose != 0.0f) {
            vx = fmaf(a.x, hclose, vx);
            vy = fmaf(a.y, hclose, vy);
            vz = fmaf(a.z, hclose, vz);
            st.aold[i] = acc_mag(a);
        }
        vx = fmaf(a.x, hdt, vx);
        vy = fmaf(a.y, hdt, vy);
        vz = fmaf(a.z, hdt, vz);
        st.vx[i] = vx;
        st.vy[i] = vy;
        st.vz[i] = vz;
        const double x = x0 + (double)vx * dt;
        const double y = y0 + (double)vy * dt;
        const double z = z0 + (double)vz * dt;
        st.x[i] = x;
        st.y[i] = y;
        st.z[i] = z;
        if (pos4) pos4[i] = make_float4((float)x, (float)y, (float)z, m);
    }
}

__global__ void kick_kernel(int64_t n, StepState st, const float4 *__restrict__ acc, float hdt) {
    NB_GRID_LOOP(i, n) {
        const float4 a = acc[i];
        const float vx = st.vx[i], vy = st.vy[i], vz = st.vz[i];
        st.vx[i] = fmaf(a.x, hdt, vx);
        st.vy[i] = fmaf(a.y, hdt, vy);
        st.vz[i] = fmaf(a.z, hdt, vz);
        st.aold[i] = acc_mag(a);
    }
}

void launch_kick_drift(cudaStream_t s, int64_t n, StepState st, const float4 *acc, float hdt,
                       float dt, float4 *pos4, float hclose) {
    kick_drift_kernel<<<grid_for(n), 256, 0, s>>>(n, st, acc, hclose, hdt, (double)dt, pos4);
}

void launch_kick(cudaStream_t s, int64_t n, StepState st, const float4 *acc, float hdt) {
    kick_kernel<<<grid_for(n), 256, 0, s>>>(n, st, acc, hdt);
}

// Gather the state into the new Morton order and refresh the FP32 walk copy.
// In these per-particle kernels every load is issued before the first store:
// the compiler may not move a load above a store to memory it cannot prove
// distinct, so interleaving them would serialise the thread's round trips.
__global__ void __launch_bounds__(256) permute_state_kernel(int64_t n,
                                                            const uint32_t *__restrict__ perm,
                                                            StepState src, StepState dst,
                                                            float4 *__restrict__ pos4) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const uint32_t j = perm[i];
    const double px = src.x[j], py = src.y[j], pz = src.z[j];
    const float vx = src.vx[j], vy = src.vy[j], vz = src.vz[j];
    const float m = src.m[j], ao = src.aold[j];
    const uint32_t id = src.id[j];
    const float pc = src.pcost ? src.pcost[j] : 0.0f;
    const uint8_t lv = src.lvl ? src.lvl[j] : (uint8_t)0;
    dst.x[i] = px;
    dst.y[i] = py;
    dst.z[i] = pz;
    pos4[i] = make_float4((float)px, (float)py, (float)pz, m);
    dst.vx[i] = vx;
    dst.vy[i] = vy;
    dst.vz[i] = vz;
    dst.m[i] = m;
    dst.aold[i] = ao;
    dst.id[i] = id;
    if (src.pcost) dst.pcost[i] = pc;
    if (src.lvl) dst.lvl[i] = lv;
}

void launch_permute_state(cudaStream_t s, int64_t n, const uint32_t *perm, StepState src,
                          StepState dst, float4 *pos4) {
    const int64_t b = (n + 255) / 256;
    permute_state_kernel<<<(int)(b < 1 ? 1 : b), 256, 0, s>>>(n, perm, src, dst, pos4);
}

// 64-byte particle records for the two full permutations of a call (the
// first sort, from the caller's order, and the return to it).  Gathering
// field by field reads one sector for every 4- or 8-byte value; a record
// moves a particle's whole state in one aligned 64-byte line.
union StateRec {
    struct {
        double x, y, z;
        float vx, vy, vz, m, aold;
        uint32_t id;
        float pcost;
        uint32_t lvl;
    } f;
    uint4 q[4];
};
static_assert(sizeof(StateRec) == 64, "one 64-byte line per particle");

__device__ __forceinline__ void rec_store(uint4 *rec, int64_t i, const StateRec &r) {
#pragma unroll
    for (int k = 0; k < 4; k++) rec[4 * i + k] = r.q[k];
}
__device__ __forceinline__ StateRec rec_load(const uint4 *__restrict__ rec, int64_t i) {
    StateRec r;
#pragma unroll
    for (int k = 0; k < 4; k++) r.q[k] = rec[4 * i + k];
    return r;
}

__global__ void __launch_bounds__(256) pack_state_kernel(int64_t n, StepState st, uint4 *rec) {
    NB_GRID_LOOP(i, n) {
        StateRec r;
        r.f.x = st.x[i];
        r.f.y = st.y[i];
        r.f.z = st.z[i];
        r.f.vx = st.vx[i];
        r.f.vy = st.vy[i];
        r.f.vz = st.vz[i];
        r.f.m = st.m[i];
        r.f.aold = st.aold[i];
        r.f.id = st.id[i];
        r.f.pcost = st.pcost ? st.pcost[i] : 0.0f;
        r.f.lvl = st.lvl ? st.lvl[i] : 0u;
        r.q[3].z = r.q[3].w = 0u;
        rec_store(rec, i, r);
    }
}

// Each load instruction of a warp fetches eight whole records (four lanes
// per 64-byte line); the records reach their threads through shared memory.
__global__ void __launch_bounds__(256) permute_recs_kernel(int64_t n,
                                                           const uint32_t *__restrict__ perm,
                                                           const uint4 *__restrict__ rec,
                                                           StepState dst, float4 *__restrict__ pos4) {
    __shared__ uint4 srec[256 * 4];
    const int64_t i = (int64_t)blockIdx.x * 256 + threadIdx.x;
    const int64_t src = i < n ? (int64_t)perm[i] : -1;
    const int lane = (int)(threadIdx.x & 31), w0 = (int)(threadIdx.x & ~31u);
#pragma unroll
    for (int k = 0; k < 4; k++) {
        const int c = 32 * k + lane, j = c >> 2, part = c & 3;  // record j of the warp, piece part
        const int64_t sj = __shfl_sync(NB_FULL, src, j);
        if (sj >= 0) srec[4 * (w0 + j) + part] = rec[4 * sj + part];
    }
    __syncwarp();
    if (i >= n) return;
    StateRec r;
#pragma unroll
    for (int k = 0; k < 4; k++) r.q[k] = srec[4 * threadIdx.x + k];
    dst.x[i] = r.f.x;
    dst.y[i] = r.f.y;
    dst.z[i] = r.f.z;
    pos4[i] = make_float4((float)r.f.x, (float)r.f.y, (float)r.f.z, r.f.m);
    dst.vx[i] = r.f.vx;
    dst.vy[i] = r.f.vy;
    dst.vz[i] = r.f.vz;
    dst.m[i] = r.f.m;
    dst.aold[i] = r.f.aold;
    dst.id[i] = r.f.id;
    if (dst.pcost) dst.pcost[i] = r.f.pcost;
    if (dst.lvl) dst.lvl[i] = (uint8_t)r.f.lvl;
}

void launch_permute_state_recs(cudaStream_t s, int64_t n, const uint32_t *perm, StepState src,
                               StepState dst, float4 *pos4, void *rec, bool packed) {
    if (!packed) pack_state_kernel<<<grid_for(n), 256, 0, s>>>(n, src, (uint4 *)rec);
    permute_recs_kernel<<<(int)((n + 255) / 256), 256, 0, s>>>(n, perm, (const uint4 *)rec, dst, pos4);
}

// kd != 0: the first step's opening half kick (hdt) and drift (dt) applied
// on the way in, with the kick-drift pass's arithmetic.
__global__ void load_state_kernel(int64_t n, const double *x, const double *y, const double *z,
                                  const float *vx, const float *vy, const float *vz,
                                  const float *m, const float *ax, const float *ay,
                                  const float *az, StepState st, float4 *acc, int kd, float hdt,
                                  double dt, uint4 *rec) {
    NB_GRID_LOOP(i, n) {
        double px = x[i], py = y[i], pz = z[i];
        float qx = vx[i], qy = vy[i], qz = vz[i];
        const float mi = m[i];
        const float a0 = ax[i], a1 = ay[i], a2 = az[i];
        if (kd) {
            qx = fmaf(a0, hdt, qx);
            qy = fmaf(a1, hdt, qy);
            qz = fmaf(a2, hdt, qz);
            px = px + (double)qx * dt;
            py = py + (double)qy * dt;
            pz = pz + (double)qz * dt;
        }
        st.x[i] = px;
        st.y[i] = py;
        st.z[i] = pz;
        acc[i] = make_float4(a0, a1, a2, 0.0f);
        const float ao = sqrtf(a0 * a0 + a1 * a1 + a2 * a2);
        if (rec) {  // the rest of the state only as the record the first sort gathers
            StateRec r;
            r.f.x = px;
            r.f.y = py;
            r.f.z = pz;
            r.f.vx = qx;
            r.f.vy = qy;
            r.f.vz = qz;
            r.f.m = mi;
            r.f.aold = ao;
            r.f.id = (uint32_t)i;
            r.f.pcost = 1.0f;
            r.f.lvl = 0u;
            r.q[3].z = r.q[3].w = 0u;
            rec_store(rec, i, r);
        } else {
            st.vx[i] = qx;
            st.vy[i] = qy;
            st.vz[i] = qz;
            st.m[i] = mi;
            st.aold[i] = ao;
            st.id[i] = (uint32_t)i;
            if (st.pcost) st.pcost[i] = 1.0f;
        }
    }
}

void launch_load_state(cudaStream_t s, int64_t n, const double *x, const double *y,
                       const double *z, const float *vx, const float *vy, const float *vz,
                       const float *m, const float *ax, const float *ay, const float *az,
                       StepState st, float4 *acc, bool kick_drift, float hdt, float dt,
                       void *rec) {
    load_state_kernel<<<grid_for(n), 256, 0, s>>>(n, x, y, z, vx, vy, vz, m, ax, ay, az, st, acc,
                                                  kick_drift ? 1 : 0, hdt, (double)dt,
                                                  (uint4 *)rec);
}

// The state back in the caller's order: every sorted particle's output
// record (x, y, z, v, a) goes to its caller index as one whole 64-byte line
// (a random write of full sectors, no read-modify-write), then the records
// are unpacked into the caller's arrays with coalesced writes.
union OutRec {
    struct {
        double x, y, z;
        float vx, vy, vz, ax, ay, az;
    } f;
    uint4 q[4];
};
static_assert(sizeof(OutRec) == 64, "one 64-byte line per particle");

// One thread per sorted particle builds its record in shared memory; then
// each store instruction of a warp writes eight whole records (four lanes
// per 64-byte line) instead of one 16-byte piece of 32 different lines.
__global__ void __launch_bounds__(256) scatter_out_kernel(int64_t n, StepState st,
                                                          const float4 *__restrict__ acc,
                                                          uint4 *rec, float hkick) {
    __shared__ uint4 srec[256 * 4];
    const int64_t i = (int64_t)blockIdx.x * 256 + threadIdx.x;
    OutRec r;
    r.q[0] = r.q[1] = r.q[2] = r.q[3] = make_uint4(0u, 0u, 0u, 0u);
    int64_t o = -1;
    if (i < n) {
        const float4 a = acc[i];
        r.f.x = st.x[i];
        r.f.y = st.y[i];
        r.f.z = st.z[i];
        r.f.vx = hkick != 0.0f ? fmaf(a.x, hkick, st.vx[i]) : st.vx[i];
        r.f.vy = hkick != 0.0f ? fmaf(a.y, hkick, st.vy[i]) : st.vy[i];
        r.f.vz = hkick != 0.0f ? fmaf(a.z, hkick, st.vz[i]) : st.vz[i];
        r.f.ax = a.x;
        r.f.ay = a.y;
        r.f.az = a.z;
        o = st.id[i];
    }
#pragma unroll
    for (int k = 0; k < 4; k++) srec[4 * threadIdx.x + k] = r.q[k];
    __syncwarp();
    const int lane = (int)(threadIdx.x & 31), w0 = (int)(threadIdx.x & ~31u);
#pragma unroll
    for (int k = 0; k < 4; k++) {
        const int c = 32 * k + lane, j = c >> 2, part = c & 3;  // record j of the warp, piece part
        const int64_t oj = __shfl_sync(NB_FULL, o, j);
        if (oj >= 0) rec[4 * oj + part] = srec[4 * (w0 + j) + part];
    }
}

__global__ void __launch_bounds__(256) unpack_out_kernel(int64_t n, const uint4 *__restrict__ rec,
                                                         double *x, double *y, double *z,
                                                         float *vx, float *vy, float *vz,
                                                         float *ax, float *ay, float *az) {
    NB_GRID_LOOP(o, n) {
        OutRec r;
#pragma unroll
        for (int k = 0; k < 4; k++) r.q[k] = rec[4 * o + k];
        x[o] = r.f.x;
        y[o] = r.f.y;
        z[o] = r.f.z;
        vx[o] = r.f.vx;
        vy[o] = r.f.vy;
        vz[o] = r.f.vz;
        ax[o] = r.f.ax;
        ay[o] = r.f.ay;
        az[o] = r.f.az;
    }
}

void launch_store_state(cudaStream_t s, int64_t n, StepState st, const float4 *acc, double *x,
                        double *y, double *z, float *vx, float *vy, float *vz, float *ax,
                        float *ay, float *az, void *rec, float hkick) {
    scatter_out_kernel<<<(int)((n + 255) / 256), 256, 0, s>>>(n, st, acc, (uint4 *)rec, hkick);
    unpack_out_kernel<<<grid_for(n), 256, 0, s>>>(n, (const uint4 *)rec, x, y, z, vx, vy, vz, ax,
                                                  ay, az);
}

// ---------------------------------------------------------------- block time steps
// The paper's code integrates with block (hierarchical) time steps (Sect. 1);
// its step criterion is not given.  Reading: dt_i = sqrt(2 eta eps / |a_i|),
// level = the smallest k in 0..K with dt / 2^k <= dt_i (|a| = 0: level 0),
// decided in FP32 in this operation order.
__device__ __forceinline__ int block_level(float amag, float eps, float eta, float dt, int K) {
    if (!(amag > 0.0f)) return 0;
    const float dti = sqrtf(2.0f * eta * eps / amag);
    int k = 0;
    float h = dt;
    while (k < K && h > dti) {
        h *= 0.5f;
        k++;
    }
    return k;
}

__device__ __forceinline__ void warp_max_to(int32_t *dst, int v) {
    v = __reduce_max_sync(NB_FULL, v);
    if (lane_id() == 0) atomicMax(dst, v);
}

__global__ void block_start_kernel(int64_t n, StepState st, const float4 *__restrict__ acc, float dt,
                                   int K, float eta, const int64_t *__restrict__ off, int nsys,
                                   const float *__restrict__ sys_eps, int32_t *maxlvl) {
    for (int64_t b = (int64_t)blockIdx.x * blockDim.x; b < n; b += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = b + threadIdx.x;
        int k = 0;
        if (i < n) {
            const float4 a = acc[i];
            const float am = acc_mag(a);
            k = block_level(am, sys_eps[sys_of(off, nsys, i)], eta, dt, K);
            const float h = ldexpf(dt, -k) * 0.5f;
            st.vx[i] = fmaf(a.x, h, st.vx[i]);
            st.vy[i] = fmaf(a.y, h, st.vy[i]);
            st.vz[i] = fmaf(a.z, h, st.vz[i]);
            st.lvl[i] = (uint8_t)k;
        }
        warp_max_to(maxlvl, k);
    }
}

__global__ void block_kick_kernel(int64_t n, StepState st, const float4 *__restrict__ acc, int64_t T,
                                  int64_t total, float dt, int K, float eta,
                                  const int64_t *__restrict__ off, int nsys,
                                  const float *__restrict__ sys_eps, int32_t *maxlvl) {
    for (int64_t b = (int64_t)blockIdx.x * blockDim.x; b < n; b += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = b + threadIdx.x;
        int k = 0;
        if (i < n) {
            k = st.lvl[i];
            if ((T & ((int64_t(1) << (K - k)) - 1)) == 0) {  // active at T
                const float4 a = acc[i];
                const float am = acc_mag(a);
                const float h = ldexpf(dt, -k) * 0.5f;  // closing half kick of the old step
                float vx = fmaf(a.x, h, st.vx[i]), vy = fmaf(a.y, h, st.vy[i]),
                      vz = fmaf(a.z, h, st.vz[i]);
                st.aold[i] = am;
                if (T < total) {
                    int kn = block_level(am, sys_eps[sys_of(off, nsys, i)], eta, dt, K);
                    // a coarser level only where T is a multiple of its step
                    while (kn < k && (T & ((int64_t(1) << (K - kn)) - 1)) != 0) kn++;
                    const float hn = ldexpf(dt, -kn) * 0.5f;
                    vx = fmaf(a.x, hn, vx);
                    vy = fmaf(a.y, hn, vy);
                    vz = fmaf(a.z, hn, vz);
                    k = kn;
                    st.lvl[i] = (uint8_t)kn;
                }
                st.vx[i] = vx;
                st.vy[i] = vy;
                st.vz[i] = vz;
            }
        }
        warp_max_to(maxlvl, k);
    }
}

void launch_block_start(cudaStream_t s, int64_t n, StepState st, const float4 *acc, float dt,
                        int K, float eta, const int64_t *off, int nsys, const float *sys_eps,
                        int32_t *maxlvl) {
    block_start_kernel<<<grid_for(n), 256, 0, s>>>(n, st, acc, dt, K, eta, off, nsys, sys_eps, maxlvl);
}

void launch_block_kick(cudaStream_t s, int64_t n, StepState st, const float4 *acc, int64_t T,
                       int64_t total, float dt, int K, float eta, const int64_t *off, int nsys,
                       const float *sys_eps, int32_t *maxlvl) {
    block_kick_kernel<<<grid_for(n), 256, 0, s>>>(n, st, acc, T, total, dt, K, eta, off, nsys,
                                                  sys_eps, maxlvl);
}

// Warp per group: the group is listed when one of its members is active.
__global__ void block_active_groups_kernel(const DevState *__restrict__ ds,
                                           const int32_t *__restrict__ grp_first,
                                           const int32_t *__restrict__ grp_count,
                                           const uint8_t *__restrict__ lvl, int64_t T, int K,
                                           int32_t *order, int32_t *count) {
    const int ng = ds->ngroups;
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nw = (gridDim.x * blockDim.x) >> 5;
    for (int g = warp; g < ng; g += nw) {
        const int first = grp_first[g], cnt = grp_count[g];
        bool act = false;
        for (int k = (int)lane_id(); k < cnt; k += 32)
            act |= (T & ((int64_t(1) << (K - lvl[first + k])) - 1)) == 0;
        if (__any_sync(NB_FULL, act) && lane_id() == 0) order[atomicAdd(count, 1)] = g;
    }
}

void launch_block_active_groups(cudaStream_t s, const DevState *ds, const int32_t *grp_first,
                                const int32_t *grp_count, const uint8_t *lvl, int64_t T, int K,
                                int32_t *order, int32_t *count, int nsm) {
    block_active_groups_kernel<<<nsm * 8, 256, 0, s>>>(ds, grp_first, grp_count, lvl, T, K, order,
                                                       count);
}

// ---------------------------------------------------------------- diagnostics
constexpr int DG_T = 256;
constexpr int DG_BLOCKS = 1024;

// Per block: FP64 partial sums of {E_kin, E_pot, P, L}; then one block adds
// the partials in a fixed order, so the result is deterministic.
__global__ void __launch_bounds__(DG_T) diag_partial_kernel(int64_t n, const double *x,
                                                            const double *y, const double *z,
                                                            const float *vx, const float *vy,
                                                            const float *vz, const float *m,
                                                            const float *phi, double *part) {
    __shared__ double sh[8][DG_T];
    double s[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    NB_GRID_LOOP(i, n) {
        double mi = m[i], u = vx[i], v = vy[i], w = vz[i];
        double px = x[i], py = y[i], pz = z[i];
        s[0] += 0.5 * mi * (u * u + v * v + w * w);
        if (phi) s[1] += 0.5 * mi * (double)phi[i];
        s[2] += mi * u;
        s[3] += mi * v;
        s[4] += mi * w;
        s[5] += mi * (py * w - pz * v);
        s[6] += mi * (pz * u - px * w);
        s[7] += mi * (px * v - py * u);
    }
    for (int k = 0; k < 8; k++) sh[k][threadIdx.x] = s[k];
    __syncthreads();
    for (int h = DG_T / 2; h > 0; h >>= 1) {
        if ((int)threadIdx.x < h)
            for (int k = 0; k < 8; k++) sh[k][threadIdx.x] += sh[k][threadIdx.x + h];
        __syncthreads();
    }
    if (threadIdx.x < 8) part[blockIdx.x * 8 + threadIdx.x] = sh[threadIdx.x][0];
}

__global__ void diag_final_kernel(int nb, const double *part, double *out) {
    if (threadIdx.x < 8) {
        double t = 0;
        for (int b = 0; b < nb; b++) t += part[b * 8 + threadIdx.x];
        out[threadIdx.x] = t;
    }
}

size_t diag_temp_bytes() { return (size_t)DG_BLOCKS * 8 * sizeof(double); }

void launch_diagnostics(cudaStream_t s, int64_t n, const double *x, const double *y,
                        const double *z, const float *vx, const float *vy, const float *vz,
                        const float *m, const float *phi, void *temp, double *d_out) {
    int nb = grid_for(n, DG_T);
    if (nb > DG_BLOCKS) nb = DG_BLOCKS;
    double *part = (double *)temp;
    diag_partial_kernel<<<nb, DG_T, 0, s>>>(n, x, y, z, vx, vy, vz, m, phi, part);
    diag_final_kernel<<<1, 32, 0, s>>>(nb, part, d_out);
}

}  // namespace nb
