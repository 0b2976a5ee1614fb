// walk_pipe.cuh -- the tree walk with warp specialisation: each i-group is
// handled by a pair of warps, a traversal warp and an evaluation warp, that
// pass interaction lists through two shared-memory buffers.
//
// The traversal warp runs the same traversal as walk_kernel (pop four child
// ranges of up to 8 nodes, MAC of Eq. 2 against the group's sphere,
// ballot/popc compaction of accepted nodes, opened nodes and opened leaves)
// and publishes a buffer whenever walk_kernel would flush its list; the
// evaluation warp holds the group's i-particles and evaluates Eq. 1 over each
// published buffer with the same packed-FP32 flush.  Lists, flush boundaries and the order of every sum
// are those of walk_kernel, so the results are identical bit for bit; what
// changes is that the traversal (integer, shared-memory and load work) and
// the evaluation (FP32 FMA work) of different groups run in different warps
// at the same time instead of alternating inside one warp.
//
// Hand-off: per buffer an mbarrier "full" (the traversal warp arrives after
// writing the buffer and its header) and an mbarrier "empty" (the evaluation
// warp arrives when it has read the buffer).  Every wait polls at most
// kPipeSpinLimit times; a wait that runs out records kStatusTimeout and both
// warps leave the kernel (each of their waits is bounded too).
#pragma once

#include "walk_impl.cuh"

namespace nb {

constexpr int kPipeSpinLimit = 1 << 22;
constexpr int kPipeFirst = 1, kPipeLast = 2, kPipeStop = 4;

struct PipeHdr {
    int g, first, cnt, nl, flags;
    float eps2;
    int pad[2];
};

// Shared memory of one warp pair: two mbarriers per buffer, two headers, two
// paired lists of D entries, the traversal stack and the leaf-compaction
// scratch.
__host__ __device__ inline size_t walk_pipe_smem_per_pair(int list_depth, int stack_depth) {
    const size_t b = 32 + 2 * sizeof(PipeHdr) + 2 * (size_t)list_depth * 16 +
                     (size_t)stack_depth * 4 + (size_t)kWalkScratch * 4;
    return (b + 15) & ~(size_t)15;
}

__device__ __forceinline__ uint32_t smem_addr(const void *p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
    asm volatile("{\n\t.reg .b64 st;\n\tmbarrier.arrive.shared::cta.b64 st, [%0];\n\t}" ::"r"(smem_addr(bar))
                 : "memory");
}
__device__ __forceinline__ bool mbar_test(uint64_t *bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
// Wait (all lanes) until the phase with this parity has completed; false if
// the bounded number of polls ran out.  test_wait never blocks, so the bound
// is kPipeSpinLimit polls of about 0.1 us each.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity) {
    bool done = false;
    if (lane_id() == 0) {
        for (int i = 0; i < kPipeSpinLimit; i++) {
            if (mbar_test(bar, parity)) {
                done = true;
                break;
            }
            __nanosleep(20);
        }
    }
    const bool ok = __shfl_sync(NB_FULL, done ? 1 : 0, 0) != 0;
    __syncwarp();  // lane 0's acquire orders the other lanes' accesses too
    return ok;
}

template <int IPL, bool COMP, bool SAFE>
__global__ void __maxnreg__(walk_regs<IPL>()) walk_pipe_kernel(WalkArgs a, int geometric) {
    extern __shared__ __align__(16) unsigned char walk_smem[];
    const int D = a.list_depth, S = a.stack_depth;
    const unsigned lane = lane_id(), w = threadIdx.x >> 5;
    const int pair = (int)(w >> 1);
    const bool traverse = (w & 1) == 0;
    unsigned char *base = walk_smem + (size_t)pair * walk_pipe_smem_per_pair(D, S);
    uint64_t *full = reinterpret_cast<uint64_t *>(base);  // full[0], full[1]
    uint64_t *empty = full + 2;                           // empty[0], empty[1]
    PipeHdr *hdr = reinterpret_cast<PipeHdr *>(base + 32);
    float4 *buf = reinterpret_cast<float4 *>(base + 32 + 2 * sizeof(PipeHdr));  // 2 x D entries
    uint32_t *stk = reinterpret_cast<uint32_t *>(buf + 2 * (size_t)D);
    int *scr = reinterpret_cast<int *>(stk + S);
    if (traverse && lane == 0) {
        mbar_init(&full[0], 1);
        mbar_init(&full[1], 1);
        mbar_init(&empty[0], 1);
        mbar_init(&empty[1], 1);
    }
    __syncthreads();

    DevState *ds = a.ds;
    const int ng = a.nactive ? *a.nactive : ds->ngroups;
    bool timeout = false, bad = false;

    if (traverse) {
        const int nnodes = ds->nnodes;
        const int npart = (int)a.n;
        const unsigned lt = lanemask_lt();
        int max_sp = 0;
        unsigned long long warp_entries = 0, warp_inter = 0;
        bool overflow = false;
        int b = 0;
        uint32_t used[2] = {0u, 0u};
        // take buffer b for writing: after its first use, wait until the
        // evaluation warp has released it
        auto acquire = [&](int bb) -> bool {
            if (used[bb] == 0) return true;
            if (mbar_wait(&empty[bb], (used[bb] - 1) & 1u)) return true;
            timeout = true;
            return false;
        };
        auto publish = [&](int bb, const PipeHdr &h) {
            __syncwarp();
            if (lane == 0) {
                hdr[bb] = h;
                mbar_arrive(&full[bb]);
            }
            used[bb]++;
        };
        for (;;) {
            int qi = 0;
            if (lane == 0) qi = atomicAdd(&ds->queue_head, 1);
            qi = __shfl_sync(NB_FULL, qi, 0);
            if (qi >= ng) {
                if (acquire(b)) publish(b, PipeHdr{0, 0, 0, 0, kPipeStop, 0.0f, {0, 0}});
                break;
            }
            const int g = a.order ? a.order[qi] : qi;
            const int first = a.grp_first[g], cnt = a.grp_count[g];
            const float4 sph = a.grp_sphere[g];
            const float alpha = geometric ? 0.0f : a.grp_alpha[g];
            const int sys = a.grp_sys[g];
            const float eps2 = a.sys_eps2[sys];
            const int root = a.sys_root[sys];
            if (cnt > 32 * IPL) bad = true;
            if (!acquire(b)) break;
            float4 *LA = buf + (size_t)b * D;
            int flags = kPipeFirst;
            auto hand_over = [&](int nl) -> bool {
                publish(b, PipeHdr{g, first, cnt, nl, flags, eps2, {0, 0}});
                flags = 0;
                b ^= 1;
                if (!acquire(b)) return false;
                LA = buf + (size_t)b * D;
                return true;
            };

            if (lane == 0) stk[0] = (uint32_t)root << 3;
            int sp = 1, nl = 0;
            long long entries = 0;
            bool alive = true;
            __syncwarp();
            while (sp > 0 && alive) {
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
                float4 A = make_float4(0.f, 0.f, 0.f, 0.f), B = make_float4(0.f, 0.f, 0.f, 0.f);
                if (has) {
                    A = __ldg(&a.nodeA[node]);
                    B = __ldg(&a.nodeB[node]);
                }
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

                // ---- accepted nodes join the list
                const unsigned am = __ballot_sync(NB_FULL, accept);
                const int na = __popc(am);
                if (nl + na > D) {
                    entries += nl;
                    if (!hand_over(nl)) {
                        alive = false;
                        break;
                    }
                    nl = 0;
                }
                if (accept) list_put(LA, nl + __popc(am & lt), A);
                nl += na;

                // ---- particles of opened leaves join the list, 32 per chunk
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
                    for (int base_ = 0; base_ < total; base_ += 32) {
                        const int c = (total - base_) < 32 ? (total - base_) : 32;
                        if (nl + c > D) {
                            entries += nl;
                            if (!hand_over(nl)) {
                                alive = false;
                                break;
                            }
                            nl = 0;
                        }
                        const bool starts = lc > 0 && lexcl >= base_ && lexcl < base_ + 32;
                        const unsigned sm2 = __reduce_or_sync(NB_FULL, starts ? 1u << (lexcl - base_) : 0u);
                        const int before = __popc(__ballot_sync(NB_FULL, lc > 0 && lexcl < base_));
                        const int k = before + __popc(sm2 & (0xffffffffu >> (31 - lane))) - 1;
                        const int of = __shfl_sync(NB_FULL, lf, k & 31);
                        const int oex2 = __shfl_sync(NB_FULL, lexcl, k & 31);
                        if ((int)lane < c)
                            list_put(LA, nl + lane, __ldg(&a.pos4[of + base_ + (int)lane - oex2]));
                        nl += c;
                    }
                }
                __syncwarp();
            }
            if (!alive) break;
            entries += nl;
            publish(b, PipeHdr{g, first, cnt, nl, flags | kPipeLast, eps2, {0, 0}});
            b ^= 1;
            if (lane == 0 && a.grp_cost) a.grp_cost[g] = (int32_t)entries;
            warp_entries += (unsigned long long)entries;
            warp_inter += (unsigned long long)entries * (unsigned long long)cnt;
        }
        if (lane == 0) {
            atomicMax(&ds->max_stack, max_sp);
            if (warp_entries) {
                atomicAdd(&ds->list_entries, warp_entries);
                atomicAdd(&ds->interactions, warp_inter);
            }
            if (overflow) atomicOr(&ds->status, kStatusStackOverflow);
        }
    } else {
        // ---- evaluation warp
        int b = 0;
        uint32_t seen[2] = {0u, 0u};
        ISlots<IPL> I;
        Tiling tile = lane_tiling<IPL>(1);
        int first = 0, cnt = 0;
        float eps2 = 0.0f;
        for (;;) {
            if (!mbar_wait(&full[b], seen[b] & 1u)) {
                timeout = true;
                break;
            }
            const PipeHdr h = hdr[b];
            if (h.flags & kPipeStop) break;
            if (h.flags & kPipeFirst) {
                first = h.first;
                cnt = h.cnt;
                eps2 = h.eps2;
                tile = lane_tiling<IPL>(cnt);
                load_slots<IPL>(tile, a.pos4, first, cnt, a.grp_sphere[h.g], I);
            }
            float4 *LA = buf + (size_t)b * D;
            if (h.nl > 0) flush_runs<0, 0, IPL, false, COMP, SAFE, false>(tile, LA, h.nl, eps2, I);
            __syncwarp();
            if (lane == 0) mbar_arrive(&empty[b]);
            seen[b]++;
            b ^= 1;
            if (h.flags & kPipeLast) finish_group<IPL, false, COMP, SAFE>(tile, first, cnt, eps2, a, I);
        }
    }
    if (lane == 0 && timeout) atomicOr(&ds->status, kStatusTimeout);
    if (bad) atomicOr(&ds->status, kStatusBadTree);
}

template <int IPL>
cudaError_t launch_walk_pipe_ipl(cudaStream_t s, const WalkArgs &a, const WalkShape &sh, int nsm) {
    const int threads = 32 * sh.warps_per_block;
    const size_t smem = (size_t)(sh.warps_per_block / 2) * walk_pipe_smem_per_pair(a.list_depth, a.stack_depth);
    void (*k)(WalkArgs, int);
    if (sh.compensated) k = sh.safe ? walk_pipe_kernel<IPL, true, true> : walk_pipe_kernel<IPL, true, false>;
    else k = sh.safe ? walk_pipe_kernel<IPL, false, true> : walk_pipe_kernel<IPL, false, false>;
    cudaError_t err = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (err != cudaSuccess) return err;
    int per_sm = 0;
    err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, threads, smem);
    if (err != cudaSuccess) return err;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    if (sh.warps_launched) *sh.warps_launched = nsm * per_sm * sh.warps_per_block / 2;
    k<<<nsm * per_sm, threads, smem, s>>>(a, sh.geometric ? 1 : 0);
    return cudaGetLastError();
}

}  // namespace nb
