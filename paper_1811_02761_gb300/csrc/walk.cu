// walk.cu -- walk dispatch, the direct O(N^2) sum of Eq. 1, small helpers.
#include <cuda_runtime.h>

#include "internal.cuh"

namespace nb {

template <int IPL, bool QUAD>
cudaError_t launch_walk_ipl(cudaStream_t s, const WalkArgs &a, const WalkShape &sh, int nsm);
#define NB_WALK_EXTERN(I, Q) \
    extern template cudaError_t launch_walk_ipl<I, Q>(cudaStream_t, const WalkArgs &, const WalkShape &, int);
NB_WALK_EXTERN(1, false) NB_WALK_EXTERN(2, false) NB_WALK_EXTERN(3, false) NB_WALK_EXTERN(4, false)
NB_WALK_EXTERN(1, true) NB_WALK_EXTERN(2, true) NB_WALK_EXTERN(3, true) NB_WALK_EXTERN(4, true)
#undef NB_WALK_EXTERN

template <int IPL>
cudaError_t launch_walk_pipe_ipl(cudaStream_t s, const WalkArgs &a, const WalkShape &sh, int nsm);
#define NB_PIPE_EXTERN(I) \
    extern template cudaError_t launch_walk_pipe_ipl<I>(cudaStream_t, const WalkArgs &, const WalkShape &, int);
NB_PIPE_EXTERN(1) NB_PIPE_EXTERN(2) NB_PIPE_EXTERN(3) NB_PIPE_EXTERN(4)
#undef NB_PIPE_EXTERN

cudaError_t launch_walk(cudaStream_t s, const WalkArgs &a, const WalkShape &sh, int nsm) {
    if (sh.pipeline && !sh.quad && !sh.potential) {
        if (sh.warps_per_block % 2) return cudaErrorInvalidConfiguration;
        switch (sh.ipl) {
            case 1: return launch_walk_pipe_ipl<1>(s, a, sh, nsm);
            case 2: return launch_walk_pipe_ipl<2>(s, a, sh, nsm);
            case 3: return launch_walk_pipe_ipl<3>(s, a, sh, nsm);
            case 4: return launch_walk_pipe_ipl<4>(s, a, sh, nsm);
            default: return cudaErrorInvalidValue;
        }
    }
    if (sh.quad) {
        switch (sh.ipl) {
            case 1: return launch_walk_ipl<1, true>(s, a, sh, nsm);
            case 2: return launch_walk_ipl<2, true>(s, a, sh, nsm);
            case 3: return launch_walk_ipl<3, true>(s, a, sh, nsm);
            case 4: return launch_walk_ipl<4, true>(s, a, sh, nsm);
            default: return cudaErrorInvalidValue;
        }
    }
    switch (sh.ipl) {
        case 1: return launch_walk_ipl<1, false>(s, a, sh, nsm);
        case 2: return launch_walk_ipl<2, false>(s, a, sh, nsm);
        case 3: return launch_walk_ipl<3, false>(s, a, sh, nsm);
        case 4: return launch_walk_ipl<4, false>(s, a, sh, nsm);
        default: return cudaErrorInvalidValue;
    }
}

// ---------------------------------------------------------------- direct sum
constexpr int DT = 128;

__device__ __forceinline__ void neumaier(float &s, float &c, float x) {
    float t = s + x;
    if (fabsf(s) >= fabsf(x))
        c += (s - t) + x;
    else
        c += (x - t) + s;
    s = t;
}

// One thread per target i, sources staged through shared memory in tiles of
// DT.  COMP: the reciprocal square root gets one Newton-Raphson step,
// y <- y (3 - r2 y^2) / 2, and each tile's partial sum is added to the total
// with Neumaier compensation.
template <bool PHI, bool COMP, bool SAFE>
__global__ void __launch_bounds__(DT) direct_kernel(int64_t n, const float *__restrict__ x,
                                                    const float *__restrict__ y,
                                                    const float *__restrict__ z,
                                                    const float *__restrict__ m, float eps2,
                                                    float G, float *ax, float *ay, float *az,
                                                    float *phi) {
    __shared__ float4 tile[DT];
    const int64_t i = (int64_t)blockIdx.x * DT + threadIdx.x;
    const float xi = i < n ? x[i] : 0.0f, yi = i < n ? y[i] : 0.0f, zi = i < n ? z[i] : 0.0f;
    float s[4] = {0, 0, 0, 0}, c[4] = {0, 0, 0, 0};
    for (int64_t base = 0; base < n; base += DT) {
        const int64_t j = base + threadIdx.x;
        tile[threadIdx.x] = j < n ? make_float4(x[j], y[j], z[j], m[j])
                                  : make_float4(1e18f, 1e18f, 1e18f, 0.0f);
        __syncthreads();
        float p[4] = {0, 0, 0, 0};
        float(&T)[4] = COMP ? p : s;
#pragma unroll 8
        for (int k = 0; k < DT; k++) {
            const float4 q = tile[k];
            const float dx = q.x - xi, dy = q.y - yi, dz = q.z - zi;
            const float r2 = fmaf(dz, dz, fmaf(dy, dy, fmaf(dx, dx, eps2)));
            float rinv = rsqrt_fast(r2);
            if constexpr (COMP) rinv = rinv * (1.5f - 0.5f * r2 * rinv * rinv);
            if constexpr (SAFE) rinv = r2 >= 1.17549435e-38f ? rinv : 0.0f;
            const float mr = q.w * rinv;
            const float w3 = mr * rinv * rinv;
            T[0] = fmaf(w3, dx, T[0]);
            T[1] = fmaf(w3, dy, T[1]);
            T[2] = fmaf(w3, dz, T[2]);
            if constexpr (PHI) T[3] -= mr;
        }
        if constexpr (COMP) {
#pragma unroll
            for (int a = 0; a < 4; a++) neumaier(s[a], c[a], p[a]);
        }
        __syncthreads();
    }
    if (i < n) {
        float r[4];
        for (int a = 0; a < 4; a++) r[a] = COMP ? s[a] + c[a] : s[a];
        ax[i] = G * r[0];
        ay[i] = G * r[1];
        az[i] = G * r[2];
        if (PHI) {
            float self = 0.0f;
            if (!SAFE) {
                float rs = rsqrt_fast(eps2);
                if (COMP) rs = rs * (1.5f - 0.5f * eps2 * rs * rs);
                self = m[i] * rs;  // the j = i term, excluded by Eq. 1
            }
            phi[i] = G * (r[3] + self);
        }
    }
}

cudaError_t launch_direct(cudaStream_t s, int64_t n, const float *x, const float *y,
                          const float *z, const float *m, float G, float eps, bool compensated,
                          float *ax, float *ay, float *az, float *phi) {
    const float eps2 = eps * eps;
    const bool safe = !(eps2 > 0.0f);
    const int64_t blocks = (n + DT - 1) / DT;
#define NB_DIRECT(P, C, S) \
    direct_kernel<P, C, S><<<(unsigned)blocks, DT, 0, s>>>(n, x, y, z, m, eps2, G, ax, ay, az, phi)
    if (phi) {
        if (compensated) { if (safe) NB_DIRECT(true, true, true); else NB_DIRECT(true, true, false); }
        else { if (safe) NB_DIRECT(true, false, true); else NB_DIRECT(true, false, false); }
    } else {
        if (compensated) { if (safe) NB_DIRECT(false, true, true); else NB_DIRECT(false, true, false); }
        else { if (safe) NB_DIRECT(false, false, true); else NB_DIRECT(false, false, false); }
    }
#undef NB_DIRECT
    return cudaGetLastError();
}

// ---------------------------------------------------------------- helpers
__global__ void acc_mag_kernel(int64_t n, const float4 *__restrict__ acc, float *__restrict__ out) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        float4 a = acc[i];
        out[i] = sqrtf(a.x * a.x + a.y * a.y + a.z * a.z);
    }
}

void launch_acc_mag(cudaStream_t s, int64_t n, const float4 *acc_sorted, float *aold_sorted) {
    int blocks = (int)((n + 255) / 256);
    if (blocks > 65535 * 8) blocks = 65535 * 8;
    acc_mag_kernel<<<blocks, 256, 0, s>>>(n, acc_sorted, aold_sorted);
}

__global__ void gather_f32_kernel(int64_t n, const uint32_t *__restrict__ perm,
                                  const float *__restrict__ src, float *__restrict__ dst) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        dst[i] = src[perm[i]];
}

void launch_gather_f32(cudaStream_t s, int64_t n, const uint32_t *perm, const float *src,
                       float *dst) {
    int blocks = (int)((n + 255) / 256);
    if (blocks > 65535 * 8) blocks = 65535 * 8;
    gather_f32_kernel<<<blocks, 256, 0, s>>>(n, perm, src, dst);
}

}  // namespace nb
