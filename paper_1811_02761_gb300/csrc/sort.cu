// sort.cu -- bounding cube, Morton keys and the LSD radix sort of the tree
// build ("makeTree", Sect. 2.2; its time is dominated by the radix sort of
// the space-filling-curve keys, Sect. 4.1).
//
// All passes are HBM-bound.  The radix sort is a one-sweep LSD sort: the
// digit histograms of every pass come from the key kernel's single read of
// the positions, and each pass is one kernel that ranks a tile's keys with
// warp match/popc, finds the tile's global offsets by a bounded decoupled
// look-back, and stages the tile in shared memory so global writes are runs
// of one digit.
#include <cuda_runtime.h>

#include "internal.cuh"

namespace nb {

// CTAs per SM of the grid-strided passes over the particles (cube, keys),
// build-time tunable.
#ifndef NB_SCAN_CTAS_PER_SM
#define NB_SCAN_CTAS_PER_SM 8
#endif

// ---------------------------------------------------------------- bounding cube
// Per-system bounding box: each warp keeps running min/max while its chunks
// stay in one system, the block merges its warps, and one set of atomics per
// (block, system) publishes the result.
template <typename T>
__global__ void __launch_bounds__(256) bbox_kernel(int64_t n, const T *__restrict__ x,
                                                   const T *__restrict__ y, const T *__restrict__ z,
                                                   const int64_t *__restrict__ off, int nsys,
                                                   uint32_t *boxord) {
    __shared__ float sh_lo[8][3], sh_hi[8][3];
    __shared__ int sh_s[8];
    const unsigned lane = lane_id(), w = threadIdx.x >> 5;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const T *p[3] = {x, y, z};
    float lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
    int cur = -1;
    auto flush = [&](int s_) {
        for (int a = 0; a < 3; a++)
            for (int o = 16; o; o >>= 1) {
                lo[a] = fminf(lo[a], __shfl_xor_sync(NB_FULL, lo[a], o));
                hi[a] = fmaxf(hi[a], __shfl_xor_sync(NB_FULL, hi[a], o));
            }
        if (lane == 0 && s_ >= 0)
            for (int a = 0; a < 3; a++) {
                atomicMin(&boxord[s_ * 6 + a], f2ord(lo[a]));
                atomicMax(&boxord[s_ * 6 + 3 + a], f2ord(hi[a]));
            }
        for (int a = 0; a < 3; a++) {
            lo[a] = INFINITY;
            hi[a] = -INFINITY;
        }
    };
    for (int64_t base = warp * 256; base < n; base += nwarps * 256) {
        int64_t last = (base + 256 < n ? base + 256 : n) - 1;
        int s0 = sys_of(off, nsys, base), s1 = sys_of(off, nsys, last);
        if (s0 == s1) {
            if (s0 != cur) {
                if (cur >= 0) flush(cur);
                cur = s0;
            }
#pragma unroll
            for (int k = 0; k < 8; k++) {
                int64_t i = base + k * 32 + lane;
                if (i < n) {
#pragma unroll
                    for (int a = 0; a < 3; a++) {
                        float v = (float)p[a][i];
                        lo[a] = fminf(lo[a], v);
                        hi[a] = fmaxf(hi[a], v);
                    }
                }
            }
        } else {
            for (int k = 0; k < 8; k++) {
                int64_t i = base + k * 32 + lane;
                if (i < n) {
                    int s = sys_of(off, nsys, i);
                    for (int a = 0; a < 3; a++) {
                        uint32_t v = f2ord((float)p[a][i]);
                        atomicMin(&boxord[s * 6 + a], v);
                        atomicMax(&boxord[s * 6 + 3 + a], v);
                    }
                }
            }
        }
    }
    // merge the warps of this block that ended in the same system
    for (int a = 0; a < 3; a++)
        for (int o = 16; o; o >>= 1) {
            lo[a] = fminf(lo[a], __shfl_xor_sync(NB_FULL, lo[a], o));
            hi[a] = fmaxf(hi[a], __shfl_xor_sync(NB_FULL, hi[a], o));
        }
    if (lane == 0) {
        sh_s[w] = cur;
        for (int a = 0; a < 3; a++) {
            sh_lo[w][a] = lo[a];
            sh_hi[w][a] = hi[a];
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        const int nw = blockDim.x >> 5;
        for (int q = 0; q < nw; q++) {
            int s = sh_s[q];
            if (s < 0) continue;
            float l3[3], h3[3];
            for (int a = 0; a < 3; a++) {
                l3[a] = sh_lo[q][a];
                h3[a] = sh_hi[q][a];
            }
            for (int r = q + 1; r < nw; r++)
                if (sh_s[r] == s) {
                    for (int a = 0; a < 3; a++) {
                        l3[a] = fminf(l3[a], sh_lo[r][a]);
                        h3[a] = fmaxf(h3[a], sh_hi[r][a]);
                    }
                    sh_s[r] = -1;
                }
            for (int a = 0; a < 3; a++) {
                atomicMin(&boxord[s * 6 + a], f2ord(l3[a]));
                atomicMax(&boxord[s * 6 + 3 + a], f2ord(h3[a]));
            }
        }
    }
}

__global__ void bbox_init_kernel(int nsys, uint32_t *boxord) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nsys * 6; i += gridDim.x * blockDim.x)
        boxord[i] = (i % 6) < 3 ? 0xffffffffu : 0u;
}

// Cube of each system, in FP32 with the stated operation order:
// corner = per-axis minimum; L = (max extent) * (1 + 2^-20); L = 1 if 0;
// scale = 2^levels / L.
__global__ void bbox_finalize_kernel(int nsys, int levels, const uint32_t *boxord, SysBox *box) {
    for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < nsys; s += gridDim.x * blockDim.x) {
        SysBox b;
        if (boxord[s * 6] == 0xffffffffu) {  // empty system
            b.x0 = b.y0 = b.z0 = 0.0f;
            b.L = 1.0f;
        } else {
            float lo[3], hi[3];
            for (int a = 0; a < 3; a++) {
                lo[a] = ord2f(boxord[s * 6 + a]);
                hi[a] = ord2f(boxord[s * 6 + 3 + a]);
            }
            float ext = __fsub_rn(hi[0], lo[0]);
            float ey = __fsub_rn(hi[1], lo[1]), ez = __fsub_rn(hi[2], lo[2]);
            if (ey > ext) ext = ey;
            if (ez > ext) ext = ez;
            float L = __fmul_rn(ext, 1.0f + 0x1p-20f);
            b.x0 = lo[0];
            b.y0 = lo[1];
            b.z0 = lo[2];
            b.L = (L > 0.0f) ? L : 1.0f;
        }
        b.scale = __fdiv_rn((float)(1u << levels), b.L);
        b.pad[0] = b.pad[1] = b.pad[2] = 0.0f;
        box[s] = b;
    }
}

void launch_bbox(cudaStream_t s, const Layout &L, const void *x, const void *y, const void *z,
                 bool dbl, const int64_t *d_off, uint32_t *d_boxord, SysBox *d_box, int nsm) {
    bbox_init_kernel<<<(L.nsys * 6 + 255) / 256, 256, 0, s>>>(L.nsys, d_boxord);
    int64_t warps = (L.n + 255) / 256;
    int blocks = (int)((warps + 7) / 8);
    int maxb = nsm * NB_SCAN_CTAS_PER_SM;
    if (blocks > maxb) blocks = maxb;
    if (blocks < 1) blocks = 1;
    if (dbl)
        bbox_kernel<double><<<blocks, 256, 0, s>>>(L.n, (const double *)x, (const double *)y,
                                                   (const double *)z, d_off, L.nsys, d_boxord);
    else
        bbox_kernel<float><<<blocks, 256, 0, s>>>(L.n, (const float *)x, (const float *)y,
                                                  (const float *)z, d_off, L.nsys, d_boxord);
    bbox_finalize_kernel<<<(L.nsys + 127) / 128, 128, 0, s>>>(L.nsys, L.levels, d_boxord, d_box);
}

// ---------------------------------------------------------------- Morton keys
// Spread the low 21 bits of v so that bit k lands on bit 3k.
__device__ __forceinline__ uint64_t spread3(uint32_t v) {
    uint64_t x = v & 0x1fffffu;
    x = (x | (x << 32)) & 0x001f00000000ffffull;
    x = (x | (x << 16)) & 0x001f0000ff0000ffull;
    x = (x | (x << 8)) & 0x100f00f00f00f00full;
    x = (x | (x << 4)) & 0x10c30c30c30c30c3ull;
    x = (x | (x << 2)) & 0x1249249249249249ull;
    return x;
}

// Cell index along one axis: floor((v - v0) * scale) in FP32, clamped.
__device__ __forceinline__ uint32_t quantise(float v, float v0, float scale, uint32_t top) {
    float d = __fsub_rn(v, v0);
    float t = __fmul_rn(d, scale);
    float f = floorf(t);
    uint32_t c = (f <= 0.0f) ? 0u : (uint32_t)f;
    return c > top ? top : c;
}

// ---------------------------------------------------------------- radix sort
// One-sweep LSD radix sort: 9-bit digits; the digit histograms of all passes
// come from one read of the keys (fused into the key kernel, or a separate
// histogram kernel), then one kernel per pass.  In a pass, each CTA takes the
// next tile (4096 keys) from an atomic counter, ranks its keys by digit with
// warp match/popc, and finds how many keys of each digit precede the tile by
// a decoupled look-back over the per-(tile, digit) words of the tiles before
// it: a tile first publishes its own digit counts (an "aggregate"), then,
// walking back, adds aggregates until it meets a tile that has published its
// inclusive prefix, and publishes its own.  Tiles take their numbers in the
// order the CTAs start, so a tile only ever waits for tiles that are already
// running, and those publish their aggregates without waiting for anyone.
// Every wait is bounded (RS_SPIN_LIMIT polls); on expiry the kernel records
// kStatusTimeout and carries on, and a destination outside [0, n) is skipped
// and recorded, so a failure is reported, never a hang or a wild write.
constexpr int RS_BITS = 9;
constexpr int RS_BINS = 1 << RS_BITS;
constexpr int RS_MAXPASS = 8;
constexpr int RS_THREADS = 512;
constexpr int RS_WARPS = RS_THREADS / 32;
#ifndef NB_RS_IPT
#define NB_RS_IPT 8  // keys per thread of a radix pass (build-time tunable)
#endif
#ifndef NB_RS_MIN_CTAS
#define NB_RS_MIN_CTAS 2  // resident CTAs per SM the pass kernel is compiled for
#endif
constexpr int RS_IPT = NB_RS_IPT;
constexpr int RS_TILE = RS_THREADS * RS_IPT;
constexpr int RS_SPIN_LIMIT = 1 << 20;
#ifndef NB_RS_LB
#define NB_RS_LB 4  // look-back words loaded per round trip (build-time tunable)
#endif
constexpr int RS_LB = NB_RS_LB;
constexpr int SCAN_T = 1024;
static_assert(RS_BINS == RS_THREADS, "one digit per thread");

// Look-back word of one (tile, digit): bits 63..60 = pass + 1 (a word left by
// another pass or sort reads as "not yet published"), bit 59 = inclusive
// prefix (else aggregate), bits 58..0 = the count.
constexpr unsigned long long RS_INCL = 1ull << 59;
constexpr unsigned long long RS_CNT = RS_INCL - 1;

// Temporary layout: tile counters, digit histograms, their exclusive
// prefixes (where each digit's keys start in the output, per pass), look-back
// words.
constexpr size_t RS_OFF_HIST = 256;
constexpr size_t RS_OFF_GSTART = RS_OFF_HIST + (size_t)RS_MAXPASS * RS_BINS * sizeof(uint32_t);
constexpr size_t RS_OFF_STATUS = RS_OFF_GSTART + (size_t)RS_MAXPASS * RS_BINS * sizeof(uint32_t);

__device__ __forceinline__ void st_relaxed_u64(unsigned long long *p, unsigned long long v) {
    asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
__device__ __forceinline__ unsigned long long ld_relaxed_u64(const unsigned long long *p) {
    unsigned long long v;
    asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

// Exclusive scan of one value per thread over a block of NT threads.
template <int NT>
__device__ __forceinline__ uint32_t block_excl_scan(uint32_t v, uint32_t *sh /* NT/32 */,
                                                    uint32_t *total) {
    const unsigned lane = lane_id(), w = threadIdx.x >> 5;
    uint32_t incl = (uint32_t)warp_incl_scan((int)v);
    if (lane == 31) sh[w] = incl;
    __syncthreads();
    if (w == 0) {
        uint32_t t = lane < NT / 32 ? sh[lane] : 0u;
        t = (uint32_t)warp_incl_scan((int)t);
        if (lane < NT / 32) sh[lane] = t;
    }
    __syncthreads();
    uint32_t r = incl - v + (w ? sh[w - 1] : 0u);
    if (total) *total = sh[NT / 32 - 1];
    __syncthreads();
    return r;
}

// Adds one key (if `valid`) to the shared digit histograms of `passes`
// passes.  A digit shared by every valid lane of the warp (the common case
// for the high digits of keys in near-sorted order) costs one atomic.
__device__ __forceinline__ void hist_add(uint32_t (*h)[RS_BINS], uint64_t key, bool valid,
                                         int passes) {
    const unsigned vm = __ballot_sync(NB_FULL, valid);
    if (!vm) return;
    const int leader = __ffs(vm) - 1;
    for (int p = 0; p < passes; p++) {
        const uint32_t d = (uint32_t)(key >> (p * RS_BITS)) & (RS_BINS - 1);
        const uint32_t d0 = __shfl_sync(NB_FULL, d, leader);
        if (__all_sync(NB_FULL, !valid || d == d0)) {
            if ((int)lane_id() == leader) atomicAdd(&h[p][d0], (uint32_t)__popc(vm));
        } else if (valid) {
            atomicAdd(&h[p][d], 1u);
        }
    }
}

// Publishes a block's shared histograms (non-zero bins only).
__device__ __forceinline__ void hist_flush(uint32_t (*h)[RS_BINS], int passes, uint32_t *g) {
    __syncthreads();
    for (int i = threadIdx.x; i < passes * RS_BINS; i += blockDim.x) {
        const uint32_t c = (&h[0][0])[i];
        if (c) atomicAdd(&g[i], c);
    }
}

__device__ __forceinline__ void hist_zero(uint32_t (*h)[RS_BINS], int passes) {
    for (int i = threadIdx.x; i < passes * RS_BINS; i += blockDim.x) (&h[0][0])[i] = 0;
    __syncthreads();
}

__global__ void __launch_bounds__(256) rs_hist_kernel(const uint64_t *__restrict__ keys, int64_t n,
                                                      const int32_t *dn, int passes, uint32_t *hist) {
    __shared__ uint32_t h[RS_MAXPASS][RS_BINS];
    if (dn) n = min(n, (int64_t)max(*dn, 0));
    hist_zero(h, passes);
    for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < n;
         base += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = base + threadIdx.x;
        const bool ok = i < n;
        hist_add(h, ok ? keys[i] : 0ull, ok, passes);
    }
    hist_flush(h, passes, hist);
}

// Morton key of every particle; with `hist`, also the digit histograms of
// all radix-sort passes (the sort then needs no histogram pass of its own).
template <typename T>
__global__ void __launch_bounds__(256) keys_kernel(Layout L, const T *__restrict__ x,
                                                   const T *__restrict__ y,
                                                   const T *__restrict__ z,
                                                   const int64_t *__restrict__ off,
                                                   const SysBox *__restrict__ box,
                                                   uint64_t *__restrict__ keys,
                                                   uint32_t *__restrict__ vals, uint32_t *hist,
                                                   int passes) {
    __shared__ uint32_t h[RS_MAXPASS][RS_BINS];
    if (hist) hist_zero(h, passes);
    const uint32_t top = (1u << L.levels) - 1u;
    const int mbits = 3 * L.levels;
    for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < L.n;
         base += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = base + threadIdx.x;
        uint64_t k = 0;
        if (i < L.n) {
            int s = sys_of(off, L.nsys, i);
            SysBox b = box[s];
            uint32_t qx = quantise((float)x[i], b.x0, b.scale, top);
            uint32_t qy = quantise((float)y[i], b.y0, b.scale, top);
            uint32_t qz = quantise((float)z[i], b.z0, b.scale, top);
            k = (spread3(qx) << 2) | (spread3(qy) << 1) | spread3(qz);
            if (L.sysbits) k |= (uint64_t)s << mbits;
            keys[i] = k;
            vals[i] = (uint32_t)i;
        }
        if (hist) hist_add(h, k, i < L.n, passes);
    }
    if (hist) hist_flush(h, passes, hist);
}

void launch_keys(cudaStream_t s, const Layout &L, const void *x, const void *y, const void *z,
                 bool dbl, const int64_t *d_off, const SysBox *d_box, uint64_t *keys,
                 uint32_t *vals, void *sort_temp, int nsm) {
    int64_t b = (L.n + 255) / 256;
    int blocks = (int)(b < (int64_t)nsm * NB_SCAN_CTAS_PER_SM ? b : (int64_t)nsm * NB_SCAN_CTAS_PER_SM);
    if (blocks < 1) blocks = 1;
    const int passes = (L.keybits + RS_BITS - 1) / RS_BITS;
    uint32_t *hist = sort_temp ? (uint32_t *)((char *)sort_temp + RS_OFF_HIST) : nullptr;
    if (dbl)
        keys_kernel<double><<<blocks, 256, 0, s>>>(L, (const double *)x, (const double *)y,
                                                   (const double *)z, d_off, d_box, keys, vals,
                                                   hist, passes);
    else
        keys_kernel<float><<<blocks, 256, 0, s>>>(L, (const float *)x, (const float *)y,
                                                  (const float *)z, d_off, d_box, keys, vals,
                                                  hist, passes);
}

// Single-block exclusive scan of sums[0..nb) in place; the grand total goes
// to *total_out when given.
__global__ void __launch_bounds__(SCAN_T) scan_sums_kernel(uint32_t *sums, int nb,
                                                           int32_t *total_out) {
    __shared__ uint32_t sh[SCAN_T / 32];
    uint32_t carry = 0;
    for (int base = 0; base < nb; base += SCAN_T) {
        int i = base + threadIdx.x;
        uint32_t v = i < nb ? sums[i] : 0u;
        uint32_t total;
        uint32_t ex = block_excl_scan<SCAN_T>(v, sh, &total);
        if (i < nb) sums[i] = carry + ex;
        carry += total;
    }
    if (total_out && threadIdx.x == 0) *total_out = (int32_t)carry;
}

void launch_scan_sums(cudaStream_t s, uint32_t *sums, int nb, int32_t *total_out) {
    scan_sums_kernel<<<1, SCAN_T, 0, s>>>(sums, nb, total_out);
}

// Where each digit's keys start in a pass's output: the exclusive prefix of
// that pass's histogram (one block per pass; the same for every tile).
__global__ void __launch_bounds__(RS_BINS) rs_gstart_kernel(const uint32_t *__restrict__ hist,
                                                          uint32_t *__restrict__ gstart) {
    __shared__ uint32_t sh[RS_BINS / 32];
    const int p = blockIdx.x, d = threadIdx.x;
    gstart[p * RS_BINS + d] = block_excl_scan<RS_BINS>(hist[p * RS_BINS + d], sh, nullptr);
}

struct RsShared {
    union {
        uint32_t whist[RS_WARPS][RS_BINS];  // per-warp digit counts, then offsets
        struct {
            uint64_t k[RS_TILE];
            uint32_t v[RS_TILE];
        } st;                                // the tile in digit order
    } u;
    uint32_t loff[RS_BINS];  // first tile slot of each digit
    uint32_t goff[RS_BINS];  // destination of tile slot p with digit d: goff[d] + p
    uint32_t wsum[RS_WARPS];
    int tile;
    int flags;
};

// One pass over the digit at `shift`.  vin is ignored on the first pass
// (values = input positions).
template <bool FIRST>
__global__ void __launch_bounds__(RS_THREADS, NB_RS_MIN_CTAS) rs_onesweep_kernel(
    const uint64_t *__restrict__ kin, const uint32_t *__restrict__ vin, uint64_t *__restrict__ kout,
    uint32_t *__restrict__ vout, int64_t n, int shift, int pass, int ntiles, void *temp,
    int32_t *status, const int32_t *dn) {
    extern __shared__ __align__(16) unsigned char rs_smem[];
    RsShared &S = *reinterpret_cast<RsShared *>(rs_smem);
    uint32_t *counter = (uint32_t *)temp;
    const uint32_t *gstart_p = (const uint32_t *)((char *)temp + RS_OFF_GSTART) + pass * RS_BINS;
    unsigned long long *look = (unsigned long long *)((char *)temp + RS_OFF_STATUS);
    const unsigned lane = lane_id(), w = threadIdx.x >> 5;
    const int d = threadIdx.x;  // the digit this thread scans and looks back for

    if (dn) {  // the key count lives on the device; n and the grid are bounds
        n = min(n, (int64_t)max(*dn, 0));
        ntiles = (int)((n + RS_TILE - 1) / RS_TILE);
    }
    if (threadIdx.x == 0) {
        S.tile = (int)atomicAdd(&counter[pass], 1u);
        S.flags = 0;
    }
    __syncthreads();
    const int tile = S.tile;
    if (tile >= ntiles) return;  // block-uniform; the grid has at least ntiles CTAs
    for (int i = threadIdx.x; i < RS_WARPS * RS_BINS; i += RS_THREADS) (&S.u.whist[0][0])[i] = 0;
    __syncthreads();
    const uint32_t gstart = gstart_p[d];
    const int64_t base = (int64_t)tile * RS_TILE;
    const int valid = (int)((n - base) < RS_TILE ? (n - base) : RS_TILE);

    uint64_t key[RS_IPT];
    uint32_t val[RS_IPT], dg[RS_IPT], rk[RS_IPT];
    // warp-striped: warp w owns the contiguous run [w*32*IPT, (w+1)*32*IPT);
    // keys past n get digit RS_BINS-1 and rank last in the tile
#pragma unroll
    for (int k = 0; k < RS_IPT; k++) {
        int64_t i = base + (int64_t)w * 32 * RS_IPT + k * 32 + lane;
        if (i < n) {
            key[k] = kin[i];
            val[k] = FIRST ? (uint32_t)i : vin[i];
        } else {
            key[k] = ~0ull;
            val[k] = 0;
        }
        dg[k] = (uint32_t)(key[k] >> shift) & (RS_BINS - 1);
    }
    const unsigned lt = lanemask_lt();
#pragma unroll
    for (int k = 0; k < RS_IPT; k++) {
        unsigned peers = __match_any_sync(NB_FULL, dg[k]);
        uint32_t b = S.u.whist[w][dg[k]];
        __syncwarp();
        if ((peers & lt) == 0) S.u.whist[w][dg[k]] = b + (uint32_t)__popc(peers);
        __syncwarp();
        rk[k] = b + (uint32_t)__popc(peers & lt);
    }
    __syncthreads();
    // digit d: exclusive prefix over the warps, and the tile's count
    uint32_t tot = 0;
#pragma unroll
    for (int q = 0; q < RS_WARPS; q++) {
        uint32_t c = S.u.whist[q][d];
        S.u.whist[q][d] = tot;
        tot += c;
    }
    const uint32_t lex = block_excl_scan<RS_THREADS>(tot, S.wsum, nullptr);
    S.loff[d] = lex;

    // publish this tile's digit counts (an aggregate; tile 0's are already
    // its inclusive prefix) before staging, so the tiles after it can walk
    // past it while this one stages its keys
    const unsigned long long tag = (unsigned long long)(pass + 1) << 60;
    const unsigned long long mine =
        tot - (d == RS_BINS - 1 ? (uint32_t)(RS_TILE - valid) : 0u);  // keys past n excluded
    unsigned long long *slot = look + (size_t)tile * RS_BINS + d;
    st_relaxed_u64(slot, tile == 0 ? (tag | RS_INCL | mine) : (tag | mine));
    __syncthreads();

    // stage the tile in digit order (needs only this tile's offsets)
    uint32_t pos[RS_IPT];
#pragma unroll
    for (int k = 0; k < RS_IPT; k++) pos[k] = S.loff[dg[k]] + S.u.whist[w][dg[k]] + rk[k];
    __syncthreads();  // the staging area overlays the per-warp counts
#pragma unroll
    for (int k = 0; k < RS_IPT; k++) {
        S.u.st.k[pos[k]] = key[k];
        S.u.st.v[pos[k]] = val[k];
    }

    // decoupled look-back for digit d: how many keys of digit d the tiles
    // before this one hold
    unsigned long long excl = 0;
    if (tile > 0) {
        // walk back RS_LB words per round trip: the words of tiles j, j-1,
        // ... are loaded together and consumed in order until an inclusive
        // prefix; a word not yet published is polled again (bounded)
        int j = tile - 1, spins = 0;
        bool done = false;
        while (!done) {
            unsigned long long v[RS_LB];
#pragma unroll
            for (int u = 0; u < RS_LB; u++)
                v[u] = (j - u >= 0) ? ld_relaxed_u64(look + (size_t)(j - u) * RS_BINS + d)
                                    : (tag | RS_INCL);  // before tile 0: prefix 0
            int used = 0;
            bool stalled = false;
#pragma unroll
            for (int u = 0; u < RS_LB; u++) {
                if (done || stalled) continue;
                if ((v[u] >> 60) != (unsigned long long)(pass + 1)) {
                    stalled = true;
                    continue;
                }
                excl += v[u] & RS_CNT;
                used++;
                if (v[u] & RS_INCL) done = true;
            }
            j -= used;
            if (stalled && !done) {
                if (++spins > RS_SPIN_LIMIT) {
                    atomicOr(&S.flags, kStatusTimeout);
                    break;
                }
                __nanosleep(32);
            }
        }
        st_relaxed_u64(slot, tag | RS_INCL | (excl + mine));
    }
    S.goff[d] = (uint32_t)((unsigned long long)gstart + excl) - lex;
    __syncthreads();
    bool bad = false;
    for (int p = threadIdx.x; p < valid; p += RS_THREADS) {
        const uint64_t kk = S.u.st.k[p];
        const uint32_t dd = (uint32_t)(kk >> shift) & (RS_BINS - 1);
        const uint32_t dst = S.goff[dd] + (uint32_t)p;
        if (dst < (uint64_t)n) {
            kout[dst] = kk;
            vout[dst] = S.u.st.v[p];
        } else {
            bad = true;
        }
    }
    if (bad) atomicOr(&S.flags, kStatusBadTree);
    __syncthreads();
    if (threadIdx.x == 0 && S.flags) atomicOr(status, S.flags);
}

size_t radix_temp_bytes(int64_t n) {
    int64_t ntiles = (n + RS_TILE - 1) / RS_TILE;
    return RS_OFF_STATUS + (size_t)ntiles * RS_BINS * sizeof(unsigned long long);
}

void radix_prepare(cudaStream_t s, int64_t n, void *temp) {
    cudaMemsetAsync(temp, 0, radix_temp_bytes(n), s);
}

int radix_sort(cudaStream_t s, uint64_t *keys, uint32_t *vals, uint64_t *keys_alt,
               uint32_t *vals_alt, int64_t n, int bits, void *temp, bool hist_done,
               int32_t *status, int nsm, const int32_t *dn) {
    // per call: the attribute belongs to the current device's context
    cudaFuncSetAttribute(rs_onesweep_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)sizeof(RsShared));
    cudaFuncSetAttribute(rs_onesweep_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)sizeof(RsShared));
    const int passes = (bits + RS_BITS - 1) / RS_BITS;
    if (!hist_done) {
        radix_prepare(s, n, temp);
        int64_t b = (n + 255) / 256;
        int blocks = (int)(b < (int64_t)nsm * 8 ? b : (int64_t)nsm * 8);
        if (blocks < 1) blocks = 1;
        rs_hist_kernel<<<blocks, 256, 0, s>>>(keys, n, dn, passes,
                                              (uint32_t *)((char *)temp + RS_OFF_HIST));
    }
    rs_gstart_kernel<<<passes, RS_BINS, 0, s>>>((const uint32_t *)((char *)temp + RS_OFF_HIST),
                                                (uint32_t *)((char *)temp + RS_OFF_GSTART));
    const int ntiles = (int)((n + RS_TILE - 1) / RS_TILE);
    uint64_t *kin = keys, *kout = keys_alt;
    uint32_t *vin = vals, *vout = vals_alt;
    for (int p = 0; p < passes; p++) {
        const int shift = p * RS_BITS;
        if (p == 0)
            rs_onesweep_kernel<true><<<ntiles, RS_THREADS, sizeof(RsShared), s>>>(
                kin, vin, kout, vout, n, shift, p, ntiles, temp, status, dn);
        else
            rs_onesweep_kernel<false><<<ntiles, RS_THREADS, sizeof(RsShared), s>>>(
                kin, vin, kout, vout, n, shift, p, ntiles, temp, status, dn);
        uint64_t *tk = kin; kin = kout; kout = tk;
        uint32_t *tv = vin; vin = vout; vout = tv;
    }
    return kin != keys;  // 1: the sorted result is in the alt buffers
}

int radix_passes(int bits) { return (bits + RS_BITS - 1) / RS_BITS; }

// Self-test of the bounded look-back wait: one pass over two tiles in which
// tile 0 is never taken (the tile counter starts at 1), so the only CTA takes
// tile 1 and its look-back finds no word for tile 0.  The wait must run out,
// record kStatusTimeout in *status and let the kernel finish.
cudaError_t radix_selftest_wait(cudaStream_t s, int32_t *status) {
    const int64_t n = 2 * RS_TILE;
    void *buf = nullptr;
    const size_t kb = (size_t)n * sizeof(uint64_t), vb = (size_t)n * sizeof(uint32_t);
    const size_t tb = radix_temp_bytes(n);
    cudaError_t e = cudaMalloc(&buf, 2 * kb + 2 * vb + tb);
    if (e != cudaSuccess) return e;
    char *p = (char *)buf;
    uint64_t *kin = (uint64_t *)p, *kout = (uint64_t *)(p + kb);
    uint32_t *vin = (uint32_t *)(p + 2 * kb), *vout = (uint32_t *)(p + 2 * kb + vb);
    void *temp = p + 2 * kb + 2 * vb;
    const uint32_t one = 1;
    e = cudaFuncSetAttribute(rs_onesweep_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)sizeof(RsShared));
    if (e == cudaSuccess) e = cudaMemsetAsync(buf, 0, 2 * kb + 2 * vb + tb, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(temp, &one, sizeof one, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) {
        rs_onesweep_kernel<true><<<1, RS_THREADS, sizeof(RsShared), s>>>(kin, vin, kout, vout, n, 0, 0,
                                                                         2, temp, status, nullptr);
        e = cudaGetLastError();
    }
    cudaError_t e2 = cudaStreamSynchronize(s);
    if (e == cudaSuccess) e = e2;
    cudaFree(buf);
    return e;
}

// ---------------------------------------------------------------- gather
template <typename T>
__global__ void gather_pos4_kernel(int64_t n, const uint32_t *__restrict__ perm,
                                   const T *__restrict__ x, const T *__restrict__ y,
                                   const T *__restrict__ z, const float *__restrict__ m,
                                   float4 *__restrict__ pos4) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        uint32_t j = perm[i];
        pos4[i] = make_float4((float)x[j], (float)y[j], (float)z[j], m[j]);
    }
}

void launch_gather_pos4(cudaStream_t s, int64_t n, const uint32_t *perm, const void *x,
                        const void *y, const void *z, bool dbl, const float *m, float4 *pos4) {
    int blocks = (int)((n + 255) / 256);
    if (blocks > 65535 * 8) blocks = 65535 * 8;
    if (dbl)
        gather_pos4_kernel<double><<<blocks, 256, 0, s>>>(n, perm, (const double *)x,
                                                          (const double *)y, (const double *)z,
                                                          m, pos4);
    else
        gather_pos4_kernel<float><<<blocks, 256, 0, s>>>(n, perm, (const float *)x,
                                                         (const float *)y, (const float *)z, m,
                                                         pos4);
}

}  // namespace nb
