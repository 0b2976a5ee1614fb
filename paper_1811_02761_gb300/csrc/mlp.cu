// mlp.cu -- learned cost model that orders the persistent walk's queue.
//
// A small MLP (8 group features -> 32 -> 32 -> 1, ReLU) predicts log2 of the
// walk cost of each i-group (interaction-list entries it processes).  It is
// trained online on the costs the walk itself logs, with hand-written
// forward / backward / Adam kernels: BF16 weights in the forward and backward
// passes, FP32 accumulation, FP32 master weights and Adam moments.  The
// persistent walk then pops groups in descending predicted cost (longest
// first), which shortens the tail of the walk; accelerations do not depend on
// the order (each group's walk is independent of which warp runs it, when).
//
// Parameter layout (kMlpParams floats): W1[8][32], b1[32], W2[32][32],
// b2[32], W3[32], b3 -- W1[i][j] connects input i to hidden unit j.
//
// Features of a group (computed here from the walk's own data):
//   0 log2 count            1 log2 r_g              2 log2 min |a_old|
//   3 log2 |c_g - com_root| 4 level of the group's cell
//   5 log2 (count / cell volume of that level)      6 log2 mean |a_old|
//   7 log2 N of the group's system
// The model input is the standardised feature (x - mean) / std with the
// statistics frozen from the first training batch.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "internal.cuh"

namespace nb {

constexpr int kIn = 8, kH = 32;
constexpr int oW1 = 0, oB1 = oW1 + kIn * kH, oW2 = oB1 + kH, oB2 = oW2 + kH * kH, oW3 = oB2 + kH,
              oB3 = oW3 + kH;
static_assert(oB3 + 1 == kMlpParams, "parameter layout");

__device__ __forceinline__ float safe_log2(float x) { return __log2f(fmaxf(x, 1e-30f)); }

// ---------------------------------------------------------------- features
__global__ void mlp_features_kernel(Layout L, const DevState *__restrict__ ds,
                                    const int32_t *__restrict__ grp_first,
                                    const int32_t *__restrict__ grp_count,
                                    const float4 *__restrict__ grp_sphere,
                                    const int32_t *__restrict__ grp_sys,
                                    const float *__restrict__ aold, const uint64_t *__restrict__ keys,
                                    const float4 *__restrict__ nodeA,
                                    const int32_t *__restrict__ sys_root,
                                    const SysBox *__restrict__ box, const int64_t *__restrict__ off,
                                    float *__restrict__ feat) {
    const int ng = ds->ngroups;
    const unsigned lane = lane_id();
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nw = (gridDim.x * blockDim.x) >> 5;
    const int mbits = 3 * L.levels;
    for (int g = warp; g < ng; g += nw) {
        const int first = grp_first[g], cnt = grp_count[g];
        float amin = INFINITY, asum = 0.0f;
        for (int k = lane; k < cnt; k += 32) {
            float a = aold[first + k];
            amin = fminf(amin, a);
            asum += a;
        }
        for (int o = 16; o; o >>= 1) {
            amin = fminf(amin, __shfl_xor_sync(NB_FULL, amin, o));
            asum += __shfl_xor_sync(NB_FULL, asum, o);
        }
        if (lane == 0) {
            const int s = grp_sys[g];
            const float4 sph = grp_sphere[g];
            const int root = sys_root[s];
            const float4 rc = root >= 0 ? nodeA[root] : make_float4(sph.x, sph.y, sph.z, 0.f);
            const float dx = sph.x - rc.x, dy = sph.y - rc.y, dz = sph.z - rc.z;
            // level of the smallest cell holding the whole group
            uint64_t x = keys[first] ^ keys[first + cnt - 1];
            x &= mbits >= 64 ? ~0ull : ((1ull << mbits) - 1ull);
            const int level = x == 0 ? L.levels : (mbits - 1 - (63 - __clzll((long long)x))) / 3;
            const float Lbox = box[s].L;
            const float nsys = (float)(off[s + 1] - off[s]);
            float *f = feat + (int64_t)g * kIn;
            f[0] = safe_log2((float)cnt);
            f[1] = safe_log2(sph.w);
            f[2] = safe_log2(amin);
            f[3] = safe_log2(sqrtf(dx * dx + dy * dy + dz * dz));
            f[4] = (float)level;
            f[5] = safe_log2((float)cnt) - 3.0f * (safe_log2(Lbox) - (float)level);
            f[6] = safe_log2(asum / (float)cnt);
            f[7] = safe_log2(nsys);
        }
    }
}

// ---------------------------------------------------------------- forward
struct MlpSmem {
    float w[kMlpParams];
    float mu[kIn], isd[kIn];
};

__device__ __forceinline__ void load_weights(MlpSmem &S, const __nv_bfloat16 *wb,
                                             const float *norm) {
    for (int p = threadIdx.x; p < kMlpParams; p += blockDim.x) S.w[p] = __bfloat162float(wb[p]);
    if (threadIdx.x < kIn) {
        S.mu[threadIdx.x] = norm ? norm[threadIdx.x] : 0.0f;
        S.isd[threadIdx.x] = norm ? 1.0f / norm[kIn + threadIdx.x] : 1.0f;
    }
    __syncthreads();
}

// Forward pass of one sample; keeps the activations for the backward pass.
__device__ __forceinline__ float mlp_fwd(const MlpSmem &S, const float *x, float (&xn)[kIn],
                                         float (&h1)[kH], float (&h2)[kH]) {
#pragma unroll
    for (int i = 0; i < kIn; i++) xn[i] = (x[i] - S.mu[i]) * S.isd[i];
#pragma unroll 4
    for (int j = 0; j < kH; j++) {
        float a = S.w[oB1 + j];
#pragma unroll
        for (int i = 0; i < kIn; i++) a = fmaf(xn[i], S.w[oW1 + i * kH + j], a);
        h1[j] = fmaxf(a, 0.0f);
    }
#pragma unroll 4
    for (int k = 0; k < kH; k++) {
        float a = S.w[oB2 + k];
#pragma unroll
        for (int j = 0; j < kH; j++) a = fmaf(h1[j], S.w[oW2 + j * kH + k], a);
        h2[k] = fmaxf(a, 0.0f);
    }
    float y = S.w[oB3];
#pragma unroll
    for (int k = 0; k < kH; k++) y = fmaf(h2[k], S.w[oW3 + k], y);
    return y;
}

// tnorm (nullable): target mean and standard deviation; the network output
// is de-standardised with them.
__global__ void __launch_bounds__(128) mlp_forward_kernel(const int32_t *__restrict__ pn, int64_t n_host,
                                                          const float *__restrict__ feat,
                                                          const __nv_bfloat16 *__restrict__ wb,
                                                          const float *__restrict__ norm,
                                                          const float *__restrict__ tnorm,
                                                          float *__restrict__ pred) {
    __shared__ MlpSmem S;
    load_weights(S, wb, norm);
    const float tm = tnorm ? tnorm[0] : 0.0f, ts = tnorm ? tnorm[1] : 1.0f;
    const int64_t n = pn ? (int64_t)*pn : n_host;
    for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < n;
         g += (int64_t)gridDim.x * blockDim.x) {
        float xn[kIn], h1[kH], h2[kH];
        pred[g] = fmaf(mlp_fwd(S, feat + g * kIn, xn, h1, h2), ts, tm);
    }
}

// ---------------------------------------------------------------- backward
constexpr int kGB = 128;  // samples per block in the gradient kernel

struct GradSmem {
    MlpSmem m;
    float xn[kGB][kIn];
    float h1[kGB][kH + 1];
    float d1[kGB][kH + 1];
    float h2[kGB][kH + 1];
    float d2[kGB][kH + 1];
    float dy[kGB];
    float loss[kGB];
};

// Mean-squared-error gradient of one minibatch: samples idx = base + s *
// stride (s = 0 .. count-1); each block handles kGB of them and writes its
// partial gradient (kMlpParams floats) and partial loss -- reduced in a fixed
// order afterwards, so training is deterministic.
__global__ void __launch_bounds__(kGB) mlp_grad_kernel(const float *__restrict__ feat,
                                                       const float *__restrict__ target,
                                                       int64_t base, int64_t stride, int count,
                                                       float inv_count,
                                                       const __nv_bfloat16 *__restrict__ wb,
                                                       const float *__restrict__ norm,
                                                       float *__restrict__ gpart,
                                                       float *__restrict__ lpart) {
    extern __shared__ __align__(16) unsigned char mlp_smem[];
    GradSmem &S = *reinterpret_cast<GradSmem *>(mlp_smem);
    load_weights(S.m, wb, norm);
    const int t = threadIdx.x;
    const int s = blockIdx.x * kGB + t;
    if (s < count) {
        const int64_t g = base + (int64_t)s * stride;
        float xn[kIn], h1[kH], h2[kH];
        const float y = mlp_fwd(S.m, feat + g * kIn, xn, h1, h2);
        const float e = y - target[g];
        const float dy = 2.0f * e * inv_count;
        S.dy[t] = dy;
        S.loss[t] = e * e * inv_count;
        float d2[kH];
#pragma unroll
        for (int k = 0; k < kH; k++) d2[k] = h2[k] > 0.0f ? dy * S.m.w[oW3 + k] : 0.0f;
#pragma unroll 4
        for (int j = 0; j < kH; j++) {
            float a = 0.0f;
#pragma unroll
            for (int k = 0; k < kH; k++) a = fmaf(d2[k], S.m.w[oW2 + j * kH + k], a);
            S.d1[t][j] = h1[j] > 0.0f ? a : 0.0f;
        }
#pragma unroll
        for (int i = 0; i < kIn; i++) S.xn[t][i] = xn[i];
#pragma unroll
        for (int j = 0; j < kH; j++) {
            S.h1[t][j] = h1[j];
            S.h2[t][j] = h2[j];
            S.d2[t][j] = d2[j];
        }
    } else {
        S.dy[t] = 0.0f;
        S.loss[t] = 0.0f;
#pragma unroll
        for (int i = 0; i < kIn; i++) S.xn[t][i] = 0.0f;
#pragma unroll
        for (int j = 0; j < kH; j++) S.h1[t][j] = S.h2[t][j] = S.d1[t][j] = S.d2[t][j] = 0.0f;
    }
    __syncthreads();
    float *gp = gpart + (int64_t)blockIdx.x * kMlpParams;
    // every parameter's gradient is a sum over the block's samples
    for (int p = t; p < kMlpParams; p += kGB) {
        float acc = 0.0f;
        if (p < oB1) {  // W1[i][j] = sum xn_i d1_j
            const int i = p / kH, j = p % kH;
            for (int q = 0; q < kGB; q++) acc = fmaf(S.xn[q][i], S.d1[q][j], acc);
        } else if (p < oW2) {
            const int j = p - oB1;
            for (int q = 0; q < kGB; q++) acc += S.d1[q][j];
        } else if (p < oB2) {  // W2[j][k] = sum h1_j d2_k
            const int j = (p - oW2) / kH, k = (p - oW2) % kH;
            for (int q = 0; q < kGB; q++) acc = fmaf(S.h1[q][j], S.d2[q][k], acc);
        } else if (p < oW3) {
            const int k = p - oB2;
            for (int q = 0; q < kGB; q++) acc += S.d2[q][k];
        } else if (p < oB3) {  // W3[k] = sum h2_k dy
            const int k = p - oW3;
            for (int q = 0; q < kGB; q++) acc = fmaf(S.h2[q][k], S.dy[q], acc);
        } else {
            for (int q = 0; q < kGB; q++) acc += S.dy[q];
        }
        gp[p] = acc;
    }
    if (t == 0) {
        float l = 0.0f;
        for (int q = 0; q < kGB; q++) l += S.loss[q];
        lpart[blockIdx.x] = l;
    }
}

// Fixed-order reduction of the block partials; then one Adam step (Kingma &
// Ba 2015) on the FP32 master weights and the BF16 working copy.
__global__ void mlp_reduce_adam_kernel(int nblocks, const float *__restrict__ gpart,
                                       const float *__restrict__ lpart, float *__restrict__ grad,
                                       float *__restrict__ loss, float *__restrict__ w,
                                       float *__restrict__ m1, float *__restrict__ m2,
                                       __nv_bfloat16 *__restrict__ wb, float lr, float b1,
                                       float b2, float epsa, float c1, float c2, int do_update) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p == 0 && loss) {
        float l = 0.0f;
        for (int b = 0; b < nblocks; b++) l += lpart[b];
        *loss = l;
    }
    if (p >= kMlpParams) return;
    float g = 0.0f;
    for (int b = 0; b < nblocks; b++) g += gpart[(int64_t)b * kMlpParams + p];
    if (grad) grad[p] = g;
    if (!do_update) return;
    const float mm = b1 * m1[p] + (1.0f - b1) * g;
    const float vv = b2 * m2[p] + (1.0f - b2) * g * g;
    m1[p] = mm;
    m2[p] = vv;
    const float wn = w[p] - lr * (mm * c1) / (sqrtf(vv * c2) + epsa);
    w[p] = wn;
    wb[p] = __float2bfloat16_rn(wn);
}

__global__ void mlp_round_kernel(const float *__restrict__ w, __nv_bfloat16 *__restrict__ wb) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p < kMlpParams) wb[p] = __float2bfloat16_rn(w[p]);
}

// Mean and standard deviation of each feature and of the raw target over n
// samples (one block): norm = {mean[8], std[8], target mean, target std}.
__global__ void mlp_norm_kernel(const int32_t *__restrict__ pn, const float *__restrict__ feat,
                                const float *__restrict__ target, float *__restrict__ norm) {
    constexpr int C = kIn + 1;
    __shared__ double s1[256][C], s2[256][C];
    const int64_t n = *pn;
    double a[C] = {0}, b[C] = {0};
    for (int64_t g = threadIdx.x; g < n; g += blockDim.x)
        for (int i = 0; i < C; i++) {
            const double v = i < kIn ? feat[g * kIn + i] : target[g];
            a[i] += v;
            b[i] += v * v;
        }
    for (int i = 0; i < C; i++) {
        s1[threadIdx.x][i] = a[i];
        s2[threadIdx.x][i] = b[i];
    }
    __syncthreads();
    if (threadIdx.x < C) {
        double t1 = 0, t2 = 0;
        for (int q = 0; q < 256; q++) {
            t1 += s1[q][threadIdx.x];
            t2 += s2[q][threadIdx.x];
        }
        const double mean = n ? t1 / (double)n : 0.0;
        const double var = n ? t2 / (double)n - mean * mean : 1.0;
        const float sd = (float)sqrt(var > 1e-12 ? var : 1.0);
        if (threadIdx.x < kIn) {
            norm[threadIdx.x] = (float)mean;
            norm[kIn + threadIdx.x] = sd;
        } else {
            norm[2 * kIn] = (float)mean;
            norm[2 * kIn + 1] = sd;
        }
    }
}

// log2 of the logged cost of each group (list entries, at least 1), then
// standardised with the frozen target statistics once they exist.
__global__ void mlp_target_kernel(const int32_t *__restrict__ pn, const int32_t *__restrict__ cost,
                                  const float *__restrict__ tnorm, float *__restrict__ target) {
    const int n = *pn;
    const float tm = tnorm ? tnorm[0] : 0.0f, its = tnorm ? 1.0f / tnorm[1] : 1.0f;
    for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < n; g += gridDim.x * blockDim.x)
        target[g] = (__log2f((float)max(cost[g], 1)) - tm) * its;
}

// Queue keys: descending score -> ascending key; value = group id.  The score
// of a group is its predicted log2 cost plus log2 of the i-slots it occupies.
__global__ void order_keys_kernel(const int32_t *__restrict__ pn, const float *__restrict__ score,
                                  const int32_t *__restrict__ grp_count, uint64_t *__restrict__ key,
                                  uint32_t *__restrict__ val) {
    const int n = *pn;
    for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < n; g += gridDim.x * blockDim.x) {
        const float slots = (float)((grp_count[g] + 31) >> 5);
        const float sc = score[g] + __log2f(slots);
        key[g] = (uint64_t)(~f2ord(sc));
        val[g] = (uint32_t)g;
    }
}

// Last-cost heuristic: score of a group = log2 of the cost its first particle's
// group had in the previous walk.
__global__ void lastcost_score_kernel(const int32_t *__restrict__ pn,
                                      const int32_t *__restrict__ grp_first,
                                      const float *__restrict__ pcost, float *__restrict__ score) {
    const int n = *pn;
    for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < n; g += gridDim.x * blockDim.x)
        score[g] = __log2f(fmaxf(pcost[grp_first[g]], 1.0f));
}

// Spread each group's logged cost to its particles (sorted order).
__global__ void spread_cost_kernel(const int32_t *__restrict__ pn,
                                   const int32_t *__restrict__ grp_first,
                                   const int32_t *__restrict__ grp_count,
                                   const int32_t *__restrict__ cost, float *__restrict__ pcost) {
    const int n = *pn;
    for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < n; g += gridDim.x * blockDim.x) {
        const float c = (float)cost[g];
        for (int k = 0; k < grp_count[g]; k++) pcost[grp_first[g] + k] = c;
    }
}

// ---------------------------------------------------------------- launchers
void launch_mlp_features(cudaStream_t s, const Layout &L, const DevState *ds,
                         const int32_t *grp_first, const int32_t *grp_count,
                         const float4 *grp_sphere, const int32_t *grp_sys, const float *aold,
                         const uint64_t *keys, const float4 *nodeA, const int32_t *sys_root,
                         const SysBox *box, const int64_t *off, float *feat, int nsm) {
    mlp_features_kernel<<<nsm * 8, 256, 0, s>>>(L, ds, grp_first, grp_count, grp_sphere, grp_sys,
                                                aold, keys, nodeA, sys_root, box, off, feat);
}

void launch_mlp_forward(cudaStream_t s, const int32_t *pn, int64_t n, const float *feat,
                        const __nv_bfloat16 *wb, const float *norm, const float *tnorm,
                        float *pred, int nsm) {
    mlp_forward_kernel<<<nsm * 4, 128, 0, s>>>(pn, n, feat, wb, norm, tnorm, pred);
}

size_t mlp_grad_smem() { return sizeof(GradSmem); }

cudaError_t launch_mlp_train_step(cudaStream_t s, const float *feat, const float *target,
                                  int64_t base, int64_t stride, int count,
                                  const __nv_bfloat16 *wb, const float *norm, float *gpart,
                                  float *lpart, float *grad, float *loss, float *w, float *m1,
                                  float *m2, __nv_bfloat16 *wb_out, float lr, int t, bool update) {
    // per call: the attribute belongs to the current device's context
    cudaError_t e = cudaFuncSetAttribute(mlp_grad_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)sizeof(GradSmem));
    if (e != cudaSuccess) return e;
    const int nb = (count + kGB - 1) / kGB;
    mlp_grad_kernel<<<nb, kGB, sizeof(GradSmem), s>>>(feat, target, base, stride, count,
                                                      1.0f / (float)count, wb, norm, gpart, lpart);
    const float b1 = 0.9f, b2 = 0.999f;
    const float c1 = 1.0f / (1.0f - powf(b1, (float)t)), c2 = 1.0f / (1.0f - powf(b2, (float)t));
    mlp_reduce_adam_kernel<<<(kMlpParams + 255) / 256, 256, 0, s>>>(
        nb, gpart, lpart, grad, loss, w, m1, m2, wb_out, lr, b1, b2, 1e-8f, c1, c2, update ? 1 : 0);
    return cudaGetLastError();
}

void launch_mlp_round(cudaStream_t s, const float *w, __nv_bfloat16 *wb) {
    mlp_round_kernel<<<(kMlpParams + 255) / 256, 256, 0, s>>>(w, wb);
}

void launch_mlp_norm(cudaStream_t s, const int32_t *pn, const float *feat, const float *target,
                     float *norm) {
    mlp_norm_kernel<<<1, 256, 0, s>>>(pn, feat, target, norm);
}

void launch_mlp_target(cudaStream_t s, const int32_t *pn, const int32_t *cost, const float *tnorm,
                       float *target, int nsm) {
    mlp_target_kernel<<<nsm * 4, 256, 0, s>>>(pn, cost, tnorm, target);
}

void launch_order_keys(cudaStream_t s, const int32_t *pn, const float *score,
                       const int32_t *grp_count, uint64_t *key, uint32_t *val, int nsm) {
    order_keys_kernel<<<nsm * 4, 256, 0, s>>>(pn, score, grp_count, key, val);
}

void launch_lastcost_score(cudaStream_t s, const int32_t *pn, const int32_t *grp_first,
                           const float *pcost, float *score, int nsm) {
    lastcost_score_kernel<<<nsm * 4, 256, 0, s>>>(pn, grp_first, pcost, score);
}

void launch_spread_cost(cudaStream_t s, const int32_t *pn, const int32_t *grp_first,
                        const int32_t *grp_count, const int32_t *cost, float *pcost, int nsm) {
    spread_cost_kernel<<<nsm * 8, 256, 0, s>>>(pn, grp_first, grp_count, cost, pcost);
}

}  // namespace nb
