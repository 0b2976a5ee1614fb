// nosort.cu -- sort of Morton keys that are already nearly in order.
//
// Inside a time step the particles are in the Morton order of the previous
// build and move a little: their new keys are almost sorted (on the N = 2^23
// galaxy 99.9 % of them end within 731 places of where they start, and only
// 1.1 % of neighbours are out of order).  A global LSD radix sort ignores
// that and moves every key through seven passes.  This sort moves every key
// twice:
//   1. splitters: the element (key, value) at the start of every tile of
//      NS_T keys, ranked among all of them and placed at their rank; bucket
//      b holds the elements from splitter b up to (not including) splitter
//      b + 1 in the order by (key, value), so equal keys spread over buckets;
//   2. count: each tile finds the bucket of each of its keys -- almost always
//      its own or a neighbour's, checked first; a binary search otherwise --
//      and counts them;
//   3. the buckets' starts (a scan of the counts);
//   4. scatter: every key and its value go to a slot of their bucket;
//   5. each bucket is sorted in shared memory (a block merge sort), or, when
//      it holds more than NS_CAP keys, sorted in chunks that are then merged
//      pairwise in global memory.
// The value of an element is its index, or the caller's value for it (vin, a
// permutation).  The result is the sort by (key, value), which is unique with
// distinct values: with indices, the stable sort of the keys, whatever order
// the scatter's atomics fill a bucket in.  A chunk is first sorted by key
// alone (half the shared-memory reads); if two of its keys are equal it is
// sorted again by (key, value).  Any input order gives the right result; a
// far-from-sorted one only makes the buckets uneven and the count and
// scatter slower.
#include <cuda_runtime.h>

#include "internal.cuh"

namespace nb {

// Tiles a little shorter than a power of two: a bucket gains or loses a few
// keys to its neighbours, and one of at most NS_CAP = 2048 keys sorts in one
// shared-memory pass.
constexpr int NS_T = 1984;           // keys per tile = nominal bucket size
constexpr int NS_THREADS = 512;      // threads of the count and scatter kernels
constexpr int NSS_THREADS = 256;     // threads of the bucket sort
constexpr int NSS_ITEMS = 8;         // keys per thread of the bucket sort
constexpr int NS_CAP = NSS_THREADS * NSS_ITEMS;  // largest range sorted in one pass
constexpr int NS_KPAD = NS_CAP + NS_CAP / 16;    // padded shared key slots
constexpr int NS_VPAD = NS_CAP + NS_CAP / 32;    // padded shared index slots
constexpr int NS_MAX_BUCKETS = 16384;
constexpr int NS_RANK_X = 256, NS_RANK_Y = 256;  // samples per rank block: own, compared

// Temporary layout: splitter keys u64 [nb] and values u32 [nb], sample ranks
// u32 [nb], counts u32 [nb], fill u32 [nb], starts u32 [nb + 1] (ranks,
// counts and fill are cleared with one memset).
static size_t ns_nb(int64_t n) { return (size_t)((n + NS_T - 1) / NS_T); }

bool nosort_fits(int64_t n) { return n >= 1 && ns_nb(n) <= NS_MAX_BUCKETS; }

size_t nosort_temp_bytes(int64_t n) {
    const size_t nb = ns_nb(n);
    return nb * 8 + nb * 16 + (nb + 1) * 4 + 64;
}

struct NsTemp {
    uint64_t *spl;
    uint32_t *splv, *rank, *cnt, *fill, *start;
};
static NsTemp ns_temp(void *temp, int64_t n) {
    const size_t nb = ns_nb(n);
    NsTemp t;
    t.spl = (uint64_t *)temp;
    t.splv = (uint32_t *)(t.spl + nb);
    t.rank = t.splv + nb;
    t.cnt = t.rank + nb;
    t.fill = t.cnt + nb;
    t.start = t.fill + nb;
    return t;
}

__device__ __forceinline__ bool pair_less(uint64_t ka, uint32_t va, uint64_t kb, uint32_t vb) {
    return ka < kb || (ka == kb && va < vb);
}

// The order of the bucket sort: by key alone (PAIR false), or by (key, value).
template <bool PAIR>
__device__ __forceinline__ bool ns_less(uint64_t ka, uint32_t va, uint64_t kb, uint32_t vb) {
    if constexpr (PAIR) return pair_less(ka, va, kb, vb);
    else return ka < kb;
}

template <bool PAIR>
__device__ __forceinline__ void cswap(uint64_t &ka, uint32_t &va, uint64_t &kb, uint32_t &vb) {
    if (ns_less<PAIR>(kb, vb, ka, va)) {
        const uint64_t tk = ka; ka = kb; kb = tk;
        const uint32_t tv = va; va = vb; vb = tv;
    }
}

// Padded shared-memory slots: one spare slot per 16 keys (per 32 indices)
// puts the eight consecutive entries of each thread of a warp in distinct
// banks.
__device__ __forceinline__ int pk(int L) { return L + (L >> 4); }
__device__ __forceinline__ int pv(int L) { return L + (L >> 5); }

// Sorts the m <= NS_CAP pairs (k[i], v[i]) in place, through the padded
// shared arrays sk [NS_KPAD] and sv [NS_VPAD]; all NSS_THREADS threads take
// part.  Each thread sorts its NSS_ITEMS pairs with a 19-comparator network,
// then runs of 8, 16, ... pairs are merged two at a time: each thread finds
// by binary search where its NSS_ITEMS outputs start on the merge path of its
// two runs and merges them from there, keeping the heads of both runs in
// registers.  The merge takes the A run first on equal keys, in the search
// and in the merge alike, so the result is always a permutation in order.
// With PAIR false the order is by key alone and the function returns false
// (k, v untouched) if two of the m keys are equal; otherwise it writes the
// sorted pairs back and returns true.
template <bool PAIR>
__device__ bool sort_chunk_impl(uint64_t *k, uint32_t *v, int m, uint64_t *sk, uint32_t *sv) {
    static_assert(NSS_ITEMS == 8, "the in-register network sorts eight");
    constexpr int I = NSS_ITEMS;
    const int t = threadIdx.x;
    __syncthreads();
    for (int i = t; i < NS_CAP; i += NSS_THREADS) {  // padding keys sort last
        sk[pk(i)] = i < m ? k[i] : ~0ull;
        sv[pv(i)] = i < m ? v[i] : ~0u;
    }
    __syncthreads();
    uint64_t rk[I];
    uint32_t rv[I];
#pragma unroll
    for (int j = 0; j < I; j++) {
        rk[j] = sk[pk(I * t + j)];
        rv[j] = sv[pv(I * t + j)];
    }
#define NS_CS(a, b) cswap<PAIR>(rk[a], rv[a], rk[b], rv[b])
    NS_CS(0, 2); NS_CS(1, 3); NS_CS(4, 6); NS_CS(5, 7);
    NS_CS(0, 4); NS_CS(1, 5); NS_CS(2, 6); NS_CS(3, 7);
    NS_CS(0, 1); NS_CS(2, 3); NS_CS(4, 5); NS_CS(6, 7);
    NS_CS(2, 4); NS_CS(3, 5);
    NS_CS(1, 4); NS_CS(3, 6);
    NS_CS(1, 2); NS_CS(3, 4); NS_CS(5, 6);
#undef NS_CS
    for (int w = I; w < NS_CAP; w <<= 1) {  // runs of w pairs -> runs of 2 w
        __syncthreads();
#pragma unroll
        for (int j = 0; j < I; j++) {
            sk[pk(I * t + j)] = rk[j];
            sv[pv(I * t + j)] = rv[j];
        }
        __syncthreads();
        const int o0 = I * t;
        const int A0 = o0 & ~(2 * w - 1), B0 = A0 + w;  // the two runs
        const int o = o0 - A0;                          // first output within the merge
        int lo = o > w ? o - w : 0, hi = o < w ? o : w;  // how many of A precede output o
        while (lo < hi) {
            const int mid = (lo + hi) >> 1;
            const int jb = B0 + o - mid - 1;
            bool a_first;
            if constexpr (PAIR)
                a_first = !pair_less(sk[pk(jb)], sv[pv(jb)], sk[pk(A0 + mid)], sv[pv(A0 + mid)]);
            else
                a_first = !(sk[pk(jb)] < sk[pk(A0 + mid)]);
            if (a_first) lo = mid + 1;
            else hi = mid;
        }
        int ia = lo, ib = o - lo;
        uint64_t ka = ia < w ? sk[pk(A0 + ia)] : ~0ull, kb = ib < w ? sk[pk(B0 + ib)] : ~0ull;
        uint32_t va = 0, vb = 0;
        if constexpr (PAIR) {
            va = ia < w ? sv[pv(A0 + ia)] : ~0u;
            vb = ib < w ? sv[pv(B0 + ib)] : ~0u;
        }
#pragma unroll
        for (int j = 0; j < I; j++) {
            const bool takeA = ib >= w || (ia < w && !ns_less<PAIR>(kb, vb, ka, va));
            const int src = takeA ? A0 + ia : B0 + ib;
            rk[j] = takeA ? ka : kb;
            if constexpr (PAIR) rv[j] = takeA ? va : vb;
            else rv[j] = sv[pv(src)];
            ia += takeA ? 1 : 0;
            ib += takeA ? 0 : 1;
            if (j + 1 < I) {  // the next head of the run just taken from
                const int nx = takeA ? ia : ib;
                const uint64_t kn = nx < w ? sk[pk(src + 1)] : ~0ull;
                if (takeA) ka = kn; else kb = kn;
                if constexpr (PAIR) {
                    const uint32_t vn = nx < w ? sv[pv(src + 1)] : ~0u;
                    if (takeA) va = vn; else vb = vn;
                }
            }
        }
    }
    __syncthreads();
#pragma unroll
    for (int j = 0; j < I; j++) {
        sk[pk(I * t + j)] = rk[j];
        sv[pv(I * t + j)] = rv[j];
    }
    __syncthreads();
    if constexpr (!PAIR) {
        bool tie = false;
        // (a key equal to the padding key ~0 counts as a tie too)
        const int mt = m < NS_CAP ? m + 1 : m;
        for (int i = t + 1; i < mt; i += NSS_THREADS) tie |= sk[pk(i)] == sk[pk(i - 1)];
        if (__syncthreads_or(tie)) return false;
    }
    for (int i = t; i < m; i += NSS_THREADS) {
        k[i] = sk[pk(i)];
        v[i] = sv[pv(i)];
    }
    __syncthreads();
    return true;
}

// Sorts m <= NS_CAP pairs in place by (key, value): by key alone when the
// keys are distinct, by both otherwise.
__device__ void block_sort_chunk(uint64_t *k, uint32_t *v, int m, uint64_t *sk, uint32_t *sv) {
    if (!sort_chunk_impl<false>(k, v, m, sk, sv)) sort_chunk_impl<true>(k, v, m, sk, sv);
}

// Bucket of an element (key, value): the largest b whose splitter (spl[b],
// splv[b]) is not above it in the order by (key, value).  Splitting by pairs
// spreads equal keys over buckets by value, so no bucket grows with the
// number of equal keys.  Tile t's elements almost always belong to bucket t
// or a neighbour, which are checked first.
__device__ __forceinline__ bool ns_le(const uint64_t *__restrict__ spl,
                                      const uint32_t *__restrict__ splv, int b, uint64_t key,
                                      uint32_t val) {
    const uint64_t k = spl[b];
    return k < key || (k == key && splv[b] <= val);
}
__device__ __forceinline__ int ns_bucket(const uint64_t *__restrict__ spl,
                                         const uint32_t *__restrict__ splv, int nb, int t,
                                         uint64_t key, uint32_t val) {
    // in bucket b: splitter b at or below, splitter b + 1 (if any) above
    auto in = [&](int b) { return ns_le(spl, splv, b, key, val) && (b + 1 == nb || !ns_le(spl, splv, b + 1, key, val)); };
    if (in(t)) return t;
    if (t > 0 && in(t - 1)) return t - 1;
    if (t + 1 < nb && in(t + 1)) return t + 1;
    int lo = 0, hi = nb;  // splitter lo at or below (splitter 0 = (0, 0)), hi above (nb: none)
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (ns_le(spl, splv, mid, key, val)) lo = mid; else hi = mid;
    }
    return lo;
}

constexpr int NS_IPT = (NS_T + NS_THREADS - 1) / NS_THREADS;

// Per-warp aggregation of the band counts: the lanes whose key goes to the
// bucket d - 1 after the tile's own (d = 0, 1, 2) are counted with one
// ballot each; returns this lane's rank among them and the warp's counts.
__device__ __forceinline__ void band_ballots(int d, bool valid, unsigned (&m)[3]) {
#pragma unroll
    for (int q = 0; q < 3; q++) m[q] = __ballot_sync(NB_FULL, valid && d == q - 1);
}

// 2. Counts per bucket: the three buckets around the tile's own in shared
// memory, the rest with global atomics.
__global__ void __launch_bounds__(NS_THREADS) ns_count_kernel(const uint64_t *__restrict__ keys,
                                                              int64_t n, int nb,
                                                              const uint64_t *__restrict__ spl,
                                                              const uint32_t *__restrict__ splv,
                                                              const uint32_t *__restrict__ vin,
                                                              uint32_t *cnt) {
    __shared__ uint32_t band[3];
    const int t = blockIdx.x;
    if (threadIdx.x < 3) band[threadIdx.x] = 0;
    __syncthreads();
    const int64_t end = (int64_t)t * NS_T + NS_T < n ? (int64_t)t * NS_T + NS_T : n;
#pragma unroll
    for (int u = 0; u < NS_IPT; u++) {
        const int64_t i = (int64_t)t * NS_T + u * NS_THREADS + threadIdx.x;
        const bool valid = i < end;
        const int b = valid ? ns_bucket(spl, splv, nb, t, keys[i], vin ? vin[i] : (uint32_t)i) : t;
        const int d = b - t;
        if (valid && (d < -1 || d > 1)) atomicAdd(&cnt[b], 1u);
        unsigned m[3];
        band_ballots(d, valid, m);
        if (lane_id() < 3 && m[lane_id()]) atomicAdd(&band[lane_id()], (uint32_t)__popc(m[lane_id()]));
    }
    __syncthreads();
    if (threadIdx.x < 3) {
        const int b = t + (int)threadIdx.x - 1;
        if (b >= 0 && b < nb && band[threadIdx.x]) atomicAdd(&cnt[b], band[threadIdx.x]);
    }
}

// 4. Scatter of every key and its value to a slot of its bucket: the tile
// reserves one run of slots per neighbouring bucket, far keys take single
// slots.  A slot outside the bucket (impossible unless the counts were
// wrong) is skipped and recorded.
__global__ void __launch_bounds__(NS_THREADS, 3) ns_scatter_kernel(const uint64_t *__restrict__ keys,
                                                                int64_t n, int nb,
                                                                const uint64_t *__restrict__ spl,
                                                                const uint32_t *__restrict__ splv,
                                                                const uint32_t *__restrict__ start,
                                                                uint32_t *fill, uint64_t *kout,
                                                                uint32_t *vout,
                                                                const uint32_t *__restrict__ vin,
                                                                int32_t *status) {
    __shared__ uint32_t band[3], base[3];
    const int t = blockIdx.x;
    if (threadIdx.x < 3) band[threadIdx.x] = 0;
    __syncthreads();
    uint64_t key[NS_IPT];
    int bk[NS_IPT];
    uint32_t rk[NS_IPT];  // rank among the warp's keys of the same band bucket, + warp base
    const int64_t end = (int64_t)t * NS_T + NS_T < n ? (int64_t)t * NS_T + NS_T : n;
#pragma unroll
    for (int u = 0; u < NS_IPT; u++) {
        const int64_t i = (int64_t)t * NS_T + u * NS_THREADS + threadIdx.x;
        key[u] = i < end ? keys[i] : 0ull;
    }
    const unsigned lt = lanemask_lt();
#pragma unroll
    for (int u = 0; u < NS_IPT; u++) {
        const int64_t i = (int64_t)t * NS_T + u * NS_THREADS + threadIdx.x;
        const bool valid = i < end;
        bk[u] = valid ? ns_bucket(spl, splv, nb, t, key[u], vin ? vin[i] : (uint32_t)i) : -1;
        const int d = valid ? bk[u] - t : -5;
        unsigned m[3];
        band_ballots(d, valid, m);
        uint32_t wb = 0;
        if (lane_id() < 3 && m[lane_id()]) wb = atomicAdd(&band[lane_id()], (uint32_t)__popc(m[lane_id()]));
        const int q = d + 1;
        const uint32_t wbase = __shfl_sync(NB_FULL, wb, q >= 0 && q <= 2 ? q : 0);
        rk[u] = (q >= 0 && q <= 2) ? wbase + (uint32_t)__popc(m[q >= 0 && q <= 2 ? q : 0] & lt) : 0u;
    }
    __syncthreads();
    if (threadIdx.x < 3) {
        const int b = t + (int)threadIdx.x - 1;
        base[threadIdx.x] = (b >= 0 && b < nb && band[threadIdx.x]) ? atomicAdd(&fill[b], band[threadIdx.x]) : 0u;
    }
    __syncthreads();
    bool bad = false;
#pragma unroll
    for (int u = 0; u < NS_IPT; u++) {
        const int64_t i = (int64_t)t * NS_T + u * NS_THREADS + threadIdx.x;
        if (i >= end) break;
        const int b = bk[u], d = b - t;
        uint32_t slot;
        if (d >= -1 && d <= 1) slot = base[d + 1] + rk[u];
        else slot = atomicAdd(&fill[b], 1u);
        const uint32_t s0 = start[b], s1 = start[b + 1];
        if (slot < s1 - s0) {
            kout[s0 + slot] = key[u];
            vout[s0 + slot] = vin ? vin[i] : (uint32_t)i;
        } else {
            bad = true;
        }
    }
    if (bad) atomicOr(status, kStatusBadTree);
}

// Merge of the sorted runs src[a, a + la) and src[a + la, a + la + lb) into
// dst[a, ...) by the whole block: each thread finds where its share of the
// output starts on the merge path, then merges its share.
__device__ void block_merge(const uint64_t *sk, const uint32_t *sv, uint64_t *dk, uint32_t *dv,
                            int64_t a, int64_t la, int64_t lb) {
    const int64_t total = la + lb;
    const int64_t seg = (total + blockDim.x - 1) / blockDim.x;
    const int64_t d0 = (int64_t)threadIdx.x * seg;
    if (d0 >= total) return;
    const int64_t d1 = d0 + seg < total ? d0 + seg : total;
    const uint64_t *ak = sk + a, *bk = sk + a + la;
    const uint32_t *av = sv + a, *bv = sv + a + la;
    // i = how many of A precede output position d0
    int64_t lo = d0 > lb ? d0 - lb : 0, hi = d0 < la ? d0 : la;
    while (lo < hi) {
        const int64_t mid = (lo + hi) >> 1;
        // take A[mid] before B[d0 - mid - 1]?
        if (pair_less(ak[mid], av[mid], bk[d0 - mid - 1], bv[d0 - mid - 1])) lo = mid + 1;
        else hi = mid;
    }
    int64_t i = lo, j = d0 - lo;
    for (int64_t d = d0; d < d1; d++) {
        const bool takeA = j >= lb || (i < la && pair_less(ak[i], av[i], bk[j], bv[j]));
        if (takeA) {
            dk[a + d] = ak[i];
            dv[a + d] = av[i];
            i++;
        } else {
            dk[a + d] = bk[j];
            dv[a + d] = bv[j];
            j++;
        }
    }
}

// Sorts the m pairs (k[i], v[i]) in place by (key, value) with the whole
// block: chunks of NS_CAP in shared memory, then (m > NS_CAP) pairwise merges
// of the sorted chunks through global memory, ping-ponging with the scratch
// ranges (kscr, vscr) of the same length.
__device__ void sort_range(uint64_t *k, uint32_t *v, int64_t m, uint64_t *kscr, uint32_t *vscr,
                           uint64_t *sk, uint32_t *sv) {
    for (int64_t c0 = 0; c0 < m; c0 += NS_CAP)
        block_sort_chunk(k + c0, v + c0, (int)(m - c0 < NS_CAP ? m - c0 : NS_CAP), sk, sv);
    if (m <= NS_CAP) return;
    uint64_t *srck = k, *dstk = kscr;
    uint32_t *srcv = v, *dstv = vscr;
    for (int64_t r = NS_CAP; r < m; r <<= 1) {
        __syncthreads();
        for (int64_t a = 0; a < m; a += 2 * r) {
            const int64_t la = m - a < r ? m - a : r;
            const int64_t lb = m - a - la < r ? m - a - la : r;
            block_merge(srck, srcv, dstk, dstv, a, la, lb);
            __syncthreads();
        }
        uint64_t *tk = srck; srck = dstk; dstk = tk;
        uint32_t *tv = srcv; srcv = dstv; dstv = tv;
    }
    if (srck != k) {  // an odd number of merge levels: copy the result back
        __syncthreads();
        for (int64_t t = threadIdx.x; t < m; t += blockDim.x) {
            k[t] = srck[t];
            v[t] = srcv[t];
        }
        __syncthreads();
    }
}

// 1a. Splitter ranks: sample i is the first element (key, value) of tile i;
// its rank is the number of samples below it in the order by (key, value)
// (values are distinct).  Block (x, y) counts, for its NS_RANK_X samples,
// the smaller ones among samples [NS_RANK_Y y, NS_RANK_Y (y + 1)).
__global__ void __launch_bounds__(NS_RANK_X) ns_rank_kernel(const uint64_t *__restrict__ keys,
                                                            const uint32_t *__restrict__ vin,
                                                            int nb, uint32_t *rank) {
    __shared__ uint64_t sk_s[NS_RANK_Y];
    __shared__ uint32_t sv_s[NS_RANK_Y];
    const int j0 = blockIdx.y * NS_RANK_Y;
    const int cnt = nb - j0 < NS_RANK_Y ? nb - j0 : NS_RANK_Y;
    for (int j = threadIdx.x; j < cnt; j += blockDim.x) {
        const int64_t e = (int64_t)(j0 + j) * NS_T;
        sk_s[j] = keys[e];
        sv_s[j] = vin ? vin[e] : (uint32_t)e;
    }
    __syncthreads();
    const int i = blockIdx.x * NS_RANK_X + threadIdx.x;
    if (i >= nb) return;
    const int64_t ei = (int64_t)i * NS_T;
    const uint64_t ki = keys[ei];
    const uint32_t vi = vin ? vin[ei] : (uint32_t)ei;
    uint32_t c = 0;
    for (int j = 0; j < cnt; j++) {
        const uint64_t kj = sk_s[j];
        c += (kj < ki || (kj == ki && sv_s[j] < vi)) ? 1u : 0u;
    }
    if (c) atomicAdd(&rank[i], c);
}

// 1b. Each sample goes to its rank; the smallest becomes (0, 0), so that
// every element has a bucket.
__global__ void ns_place_kernel(const uint64_t *__restrict__ keys,
                                const uint32_t *__restrict__ vin, int nb,
                                const uint32_t *__restrict__ rank, uint64_t *spl, uint32_t *splv) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nb) return;
    const uint32_t r = rank[i];
    const int64_t e = (int64_t)i * NS_T;
    spl[r] = r == 0 ? 0ull : keys[e];
    splv[r] = r == 0 ? 0u : (vin ? vin[e] : (uint32_t)e);
}

// 5. Sort of each bucket by (key, value), in place in (kout, vout); (kscr,
// vscr), the input keys and a free index array, give the merges of a bucket
// of more than NS_CAP keys their scratch over the same index range.
__global__ void __launch_bounds__(NSS_THREADS, 4) ns_bucket_kernel(const uint32_t *__restrict__ start,
                                                                uint64_t *kout, uint32_t *vout,
                                                                uint64_t *kscr, uint32_t *vscr) {
    __shared__ __align__(16) uint64_t sk_s[NS_KPAD];
    __shared__ uint32_t sv_s[NS_VPAD];
    const int b = blockIdx.x;
    const int64_t s0 = start[b];
    const int64_t m = (int64_t)start[b + 1] - s0;
    if (m <= 1) return;
    sort_range(kout + s0, vout + s0, m, kscr + s0, vscr + s0, sk_s, sv_s);
}

void nosort(cudaStream_t s, uint64_t *keys, uint64_t *kout, uint32_t *vscr, uint32_t *vout,
            int64_t n, void *temp, int32_t *status, const uint32_t *vin) {
    const int nb = (int)ns_nb(n);
    NsTemp T = ns_temp(temp, n);
    cudaMemsetAsync(T.rank, 0, (size_t)nb * 12, s);  // ranks, counts, fill
    ns_rank_kernel<<<dim3((nb + NS_RANK_X - 1) / NS_RANK_X, (nb + NS_RANK_Y - 1) / NS_RANK_Y),
                     NS_RANK_X, 0, s>>>(keys, vin, nb, T.rank);
    ns_place_kernel<<<(nb + 255) / 256, 256, 0, s>>>(keys, vin, nb, T.rank, T.spl, T.splv);
    ns_count_kernel<<<nb, NS_THREADS, 0, s>>>(keys, n, nb, T.spl, T.splv, vin, T.cnt);
    cudaMemcpyAsync(T.start, T.cnt, (size_t)nb * 4, cudaMemcpyDeviceToDevice, s);
    launch_scan_sums(s, T.start, nb, reinterpret_cast<int32_t *>(T.start + nb));
    ns_scatter_kernel<<<nb, NS_THREADS, 0, s>>>(keys, n, nb, T.spl, T.splv, T.start, T.fill, kout,
                                                vout, vin, status);
    ns_bucket_kernel<<<nb, NSS_THREADS, 0, s>>>(T.start, kout, vout, keys, vscr);
}

// Keys in a hinted order: kout[k] = keys[hint[k]], vout[k] = hint[k] (hint: a
// permutation of 0..n-1, e.g. the Morton order of the previous build).
__global__ void __launch_bounds__(256) ns_hint_gather_kernel(int64_t n, const uint64_t *__restrict__ keys,
                                                             const uint32_t *__restrict__ hint,
                                                             uint64_t *kout, uint32_t *vout) {
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n;
         k += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t j = hint[k];
        kout[k] = j < n ? keys[j] : ~0ull;
        vout[k] = j;
    }
}

void nosort_hint_gather(cudaStream_t s, int64_t n, const uint64_t *keys, const uint32_t *hint,
                        uint64_t *kout, uint32_t *vout) {
    int64_t b = (n + 255) / 256;
    if (b > 65535 * 8) b = 65535 * 8;
    ns_hint_gather_kernel<<<(int)(b < 1 ? 1 : b), 256, 0, s>>>(n, keys, hint, kout, vout);
}

int nosort_kernels() { return 6; }  // rank, place, count, scan, scatter, bucket sort

}  // namespace nb
