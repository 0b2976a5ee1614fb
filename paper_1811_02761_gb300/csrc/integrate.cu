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

__global__ void load_state_kernel(int64_t n, const double *x, const double *y, const double *z,
                                  const float *vx, const float *vy, const float *vz,
                                  const float *m, const float *ax, const float *ay,
                                  const float *az, StepState st, float4 *acc) {
    NB_GRID_LOOP(i, n) {
        const double px = x[i], py = y[i], pz = z[i];
        const float qx = vx[i], qy = vy[i], qz = vz[i], mi = m[i];
        const float a0 = ax[i], a1 = ay[i], a2 = az[i];
        st.x[i] = px;
        st.y[i] = py;
        st.z[i] = pz;
        st.vx[i] = qx;
        st.vy[i] = qy;
        st.vz[i] = qz;
        st.m[i] = mi;
        acc[i] = make_float4(a0, a1, a2, 0.0f);
        st.aold[i] = sqrtf(a0 * a0 + a1 * a1 + a2 * a2);
        st.id[i] = (uint32_t)i;
        if (st.pcost) st.pcost[i] = 1.0f;
    }
}

void launch_load_state(cudaStream_t s, int64_t n, const double *x, const double *y,
                       const double *z, const float *vx, const float *vy, const float *vz,
                       const float *m, const float *ax, const float *ay, const float *az,
                       StepState st, float4 *acc) {
    load_state_kernel<<<grid_for(n), 256, 0, s>>>(n, x, y, z, vx, vy, vz, m, ax, ay, az, st, acc);
}

// The state back in the caller's order, as a gather: inv[o] = the sorted index
// of caller index o, then every output array is written in caller order
// (coalesced writes; the reads are random but fetch whole sectors, where a
// scatter's random writes of 4- and 8-byte values would each cost a
// partial-sector write).
__global__ void inverse_perm_kernel(int64_t n, const uint32_t *__restrict__ id, uint32_t *inv) {
    NB_GRID_LOOP(i, n) inv[id[i]] = (uint32_t)i;
}

__global__ void gather_state_kernel(int64_t n, StepState st, const float4 *__restrict__ acc,
                                    const uint32_t *__restrict__ inv, double *x, double *y,
                                    double *z, float *vx, float *vy, float *vz, float *ax,
                                    float *ay, float *az) {
    NB_GRID_LOOP(o, n) {
        const uint32_t i = inv[o];
        const double px = st.x[i], py = st.y[i], pz = st.z[i];
        const float qx = st.vx[i], qy = st.vy[i], qz = st.vz[i];
        const float4 a = acc[i];
        x[o] = px;
        y[o] = py;
        z[o] = pz;
        vx[o] = qx;
        vy[o] = qy;
        vz[o] = qz;
        ax[o] = a.x;
        ay[o] = a.y;
        az[o] = a.z;
    }
}

void launch_store_state(cudaStream_t s, int64_t n, StepState st, const float4 *acc, double *x,
                        double *y, double *z, float *vx, float *vy, float *vz, float *ax,
                        float *ay, float *az, uint32_t *inv) {
    inverse_perm_kernel<<<grid_for(n), 256, 0, s>>>(n, st.id, inv);
    gather_state_kernel<<<grid_for(n), 256, 0, s>>>(n, st, acc, inv, x, y, z, vx, vy, vz, ax, ay, az);
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
