// api.cu -- the C ABI of libnbody (declared in include/nbody.h): argument
// checks, the context and its device buffers, host/device staging, and the
// order of kernel launches for build, walk, direct, step and diagnostics.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "internal.cuh"

using namespace nb;

namespace {

thread_local std::string g_last_error;

}  // namespace

void nb::set_stateless_error(const std::string &msg) { g_last_error = msg; }

namespace {

struct DevBuf {
    void *p = nullptr;
    size_t bytes = 0;
};

// What a captured step graph depends on: sizes, parameters and the buffers
// its kernels were captured with.
struct GraphKey {
    int64_t n;
    int32_t nsys;
    float dt;
    bool safe;
    bool mlp_norm;  // the cost model's input statistics were set at capture
    nbody_config cfg;
    const void *bufs[8];
};

}  // namespace

struct nbody_ctx {
    nbody_config cfg;
    cudaStream_t stream = nullptr;
    int device = 0, nsm = 0;
    std::string err;

    // capacities
    int64_t cap_n = 0, cap_nodes = 0;
    int cap_sys = 0;
    std::vector<DevBuf *> owned;

    DevState *ds = nullptr;
    DevState *h_ds = nullptr;  // pinned
    // particles (sorted)
    DevBuf keys, keys_alt, vals, vals_alt, pos4, delta, leaflev;
    DevBuf rs_temp, tree_temp, grp_temp, diag_temp, diag_out;
    // nodes
    DevBuf node_start, node_level, node_parent, node_link, node_count, node_nchild, node_arrive;
    DevBuf nodeA, nodeB, mass2, nodeQ;
    // groups
    DevBuf gflag, grp_first, grp_count, grp_sphere, grp_sys, grp_alpha, grp_cost, grp_order;
    // systems
    DevBuf sys_off, sys_box, sys_boxord, sys_eps2, sys_eps, sys_root;
    // walk / step
    DevBuf acc_s, aold_s;
    DevBuf st_buf[2][11];
    DevBuf recs;  // 64-byte particle records of a call's full permutations
    // the Morton order (caller indices) at the end of the last step call: the
    // next call's first sort starts from it (hint_n: its particle count, 0 =
    // none)
    DevBuf last_ids;
    int64_t hint_n = 0;
    int32_t hint_nsys = 0;
    // learned scheduling
    DevBuf mlp_w, mlp_m1, mlp_m2, mlp_wb, mlp_norm, mlp_gpart, mlp_lpart, mlp_loss;
    DevBuf feat, target, score, okey, okey_alt, oval, oval_alt, pcost_walk;
    int mlp_t = 0;
    bool mlp_ready = false, mlp_norm_set = false;
    bool costs_valid = false;  // grp_cost holds the costs of the current groups
    // staging of host arrays
    DevBuf stage[12];
    double *h_diag = nullptr;  // pinned

    cudaEvent_t ev[4] = {nullptr, nullptr, nullptr, nullptr};
    std::vector<cudaEvent_t> wev;  // (start, end) pairs around walk-kernel launches
    // (start, end) pairs around the two walks of the step graph, recorded by
    // event nodes at every replay: the last replay's walk times
    cudaEvent_t gwev[4] = {nullptr, nullptr, nullptr, nullptr};
    int gwev_used = 0, gwev_pairs = 0;  // pairs recorded while capturing / in the graph
    int wev_used = 0;
    std::vector<cudaEvent_t> evpool;  // phase boundaries of asynchronous multi-step calls
    int evused = 0;
    // CUDA graph of two leapfrog steps (nbody_config.use_graph)
    cudaStream_t gstream = nullptr;
    cudaGraphExec_t gexec = nullptr;
    GraphKey gkey{};
    int64_t gkernels = 0;
    bool capturing = false;  // enqueueing into a graph: no timing events
    int walk_warps = 0;      // resident warps of the last walk launch
    int64_t kernels = 0;           // kernels launched by the current call
    bool built = false;
    bool eps_zero = false;  // some system of the last build has eps == 0
    Layout L{};
    float last_ms_build = 0.0f;
    nbody_stats last{};

    nbody_ctx() {
        DevBuf *all[] = {&keys, &keys_alt, &vals, &vals_alt, &pos4, &delta, &leaflev, &rs_temp,
                         &tree_temp, &grp_temp, &diag_temp, &diag_out, &node_start, &node_level,
                         &node_parent, &node_link, &node_count, &node_nchild, &node_arrive,
                         &nodeA, &nodeB, &mass2, &nodeQ, &gflag, &grp_first, &grp_count, &grp_sphere,
                         &grp_sys, &grp_alpha, &grp_cost, &grp_order, &sys_off, &sys_box,
                         &sys_boxord, &sys_eps2, &sys_eps, &sys_root, &acc_s, &aold_s, &mlp_w, &mlp_m1,
                         &mlp_m2, &mlp_wb, &mlp_norm, &mlp_gpart, &mlp_lpart, &mlp_loss, &feat,
                         &target, &score, &okey, &okey_alt, &oval, &oval_alt, &pcost_walk, &recs, &last_ids};
        for (DevBuf *b : all) owned.push_back(b);
        for (auto &a : st_buf)
            for (auto &b : a) owned.push_back(&b);
        for (auto &b : stage) owned.push_back(&b);
    }
};

namespace {

nbody_status fail(nbody_ctx *ctx, nbody_status st, const std::string &msg) {
    if (ctx) ctx->err = msg;
    g_last_error = msg;
    return st;
}

nbody_status cuda_fail(nbody_ctx *ctx, cudaError_t e, const char *where) {
    std::string msg = std::string(where) + ": " + cudaGetErrorString(e);
    return fail(ctx, NBODY_ECUDA, msg);
}

#define NB_CUDA(ctx, call)                                             \
    do {                                                               \
        cudaError_t e_ = (call);                                       \
        if (e_ != cudaSuccess) return cuda_fail((ctx), e_, #call);     \
    } while (0)

bool is_device_ptr(const void *p) {
    if (!p) return false;
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

cudaError_t ensure(DevBuf &b, size_t bytes) {
    if (b.bytes >= bytes && b.p) return cudaSuccess;
    if (b.p) {
        cudaError_t e = cudaFree(b.p);
        b.p = nullptr;
        b.bytes = 0;
        if (e != cudaSuccess) return e;
    }
    size_t want = bytes ? bytes : 16;
    cudaError_t e = cudaMalloc(&b.p, want);
    if (e != cudaSuccess) {
        b.p = nullptr;
        return e;
    }
    b.bytes = want;
    return cudaSuccess;
}

template <typename T>
T *P(DevBuf &b) {
    return reinterpret_cast<T *>(b.p);
}

bool config_ok(const nbody_config *c, std::string &why) {
    char buf[160];
    auto bad = [&](const char *m) {
        why = m;
        return false;
    };
    if (!(c->eps >= 0.0f) || !std::isfinite(c->eps)) return bad("eps must be finite and >= 0");
    if (!(c->delta_acc >= 0.0f) || !std::isfinite(c->delta_acc)) return bad("delta_acc must be finite and >= 0");
    if (!(c->theta > 0.0f && c->theta < 1.0f)) return bad("theta must be in (0, 1)");
    if (!std::isfinite(c->G)) return bad("G must be finite");
    if (c->ipl < 1 || c->ipl > 4) return bad("ipl must be in 1..4");
    if (c->leaf_cap < 1 || c->leaf_cap > 32) return bad("leaf_cap must be in 1..32");
    if (c->group_size < c->leaf_cap || c->group_size > 32 * c->ipl) {
        snprintf(buf, sizeof buf, "group_size must be in leaf_cap..32*ipl (%d..%d)", c->leaf_cap,
                 32 * c->ipl);
        why = buf;
        return false;
    }
    if (c->list_depth < 64 || c->list_depth > 1024 || c->list_depth % 32)
        return bad("list_depth must be a multiple of 32 in 64..1024");
    if (c->stack_depth < 64 || c->stack_depth > 4096) return bad("stack_depth must be in 64..4096");
    if (c->warps_per_block < 1 || c->warps_per_block > 16) return bad("warps_per_block must be in 1..16");
    if (c->schedule < 0 || c->schedule > 2) return bad("schedule must be 0, 1 or 2");
    if (c->compensated < 0 || c->compensated > 2) return bad("compensated must be 0, 1 or 2");
    if (c->rebuild_interval < 0 || c->rebuild_interval > 1024)
        return bad("rebuild_interval must be in 0..1024");
    if (c->quadrupole != 0 && c->quadrupole != 1) return bad("quadrupole must be 0 or 1");
    if (c->block_levels < 0 || c->block_levels > 20) return bad("block_levels must be in 0..20");
    if (c->walk_pipeline != 0 && c->walk_pipeline != 1) return bad("walk_pipeline must be 0 or 1");
    if (c->walk_pipeline && c->warps_per_block % 2)
        return bad("walk_pipeline needs an even warps_per_block (warp pairs)");
    if (!(c->block_eta > 0.0f) || !std::isfinite(c->block_eta)) return bad("block_eta must be finite and > 0");
    size_t smem = (size_t)c->warps_per_block *
                  nb::walk_smem_per_warp(c->list_depth, c->stack_depth, c->quadrupole != 0);
    if (smem > 227 * 1024)
        return bad("warps_per_block * (16 list_depth + 4 stack_depth + 128, + 12 list_depth with "
                   "quadrupoles) exceeds 227 KB");
    return true;
}

// Stage a caller array: device pointers pass through, host arrays are copied
// into staging slot `slot`.
cudaError_t stage_in(nbody_ctx *c, int slot, const void *p, size_t bytes, const void **out) {
    if (!p) {
        *out = nullptr;
        return cudaSuccess;
    }
    if (is_device_ptr(p)) {
        *out = p;
        return cudaSuccess;
    }
    cudaError_t e = ensure(c->stage[slot], bytes);
    if (e != cudaSuccess) return e;
    e = cudaMemcpyAsync(c->stage[slot].p, p, bytes, cudaMemcpyHostToDevice, c->stream);
    *out = c->stage[slot].p;
    return e;
}

// Output array: device pointers pass through; host arrays get a staging slot
// and are copied back by stage_out_finish.
cudaError_t stage_out(nbody_ctx *c, int slot, void *p, size_t bytes, void **out) {
    if (!p) {
        *out = nullptr;
        return cudaSuccess;
    }
    if (is_device_ptr(p)) {
        *out = p;
        return cudaSuccess;
    }
    cudaError_t e = ensure(c->stage[slot], bytes);
    *out = c->stage[slot].p;
    return e;
}

// An array the step's kernels touch exactly once (read in, or written back):
// device pointers pass through, page-locked host memory is passed as its
// device mapping (the kernel reads or writes it across the host link in one
// coalesced pass, with no staging copy), and other host memory is staged as
// in stage_in.  *direct tells whether no copy-back is needed.
cudaError_t stage_once(nbody_ctx *c, int slot, const void *p, size_t bytes, const void **out,
                       bool *direct) {
    *direct = true;
    if (!p) {
        *out = nullptr;
        return cudaSuccess;
    }
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        at.type = cudaMemoryTypeUnregistered;
    }
    if (at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged) {
        *out = p;
        return cudaSuccess;
    }
    if (at.type == cudaMemoryTypeHost && at.devicePointer) {
        *out = at.devicePointer;
        return cudaSuccess;
    }
    *direct = false;
    return stage_in(c, slot, p, bytes, out);
}

cudaError_t stage_out_finish(nbody_ctx *c, void *host, const void *dev, size_t bytes) {
    if (!host || host == dev) return cudaSuccess;
    return cudaMemcpyAsync(host, dev, bytes, cudaMemcpyDeviceToHost, c->stream);
}

int64_t node_capacity(int64_t n, int levels, int leaf_cap, int nsys) {
    // internal nodes of one level are disjoint and hold > leaf_cap particles;
    // leaves are disjoint and non-empty.
    return n + (int64_t)levels * (n / (leaf_cap + 1)) + nsys + 8;
}

cudaError_t ensure_capacity(nbody_ctx *c, int64_t n, int nsys, int levels) {
    cudaError_t e;
#define NB_E(x) do { e = (x); if (e != cudaSuccess) return e; } while (0)
    if (n > c->cap_n) {
        NB_E(ensure(c->keys, n * 8)); NB_E(ensure(c->keys_alt, n * 8));
        NB_E(ensure(c->vals, n * 4)); NB_E(ensure(c->vals_alt, n * 4));
        NB_E(ensure(c->pos4, n * 16)); NB_E(ensure(c->delta, n + 1)); NB_E(ensure(c->leaflev, n));
        NB_E(ensure(c->rs_temp, std::max(radix_temp_bytes(n), nosort_temp_bytes(n))));
        NB_E(ensure(c->tree_temp, tree_temp_bytes(n, kMaxLevels)));
        NB_E(ensure(c->grp_temp, (size_t)((n + 4095) / 4096 + 64) * 4));
        NB_E(ensure(c->gflag, n));
        NB_E(ensure(c->grp_first, n * 4)); NB_E(ensure(c->grp_count, n * 4));
        NB_E(ensure(c->grp_sphere, n * 16)); NB_E(ensure(c->grp_sys, n * 4));
        NB_E(ensure(c->grp_alpha, n * 4)); NB_E(ensure(c->grp_cost, n * 4));
        NB_E(ensure(c->grp_order, n * 4));
        NB_E(ensure(c->acc_s, n * 16)); NB_E(ensure(c->aold_s, n * 4));
        c->cap_n = n;
    }
    int64_t cn = node_capacity(n, levels, c->cfg.leaf_cap, nsys);
    if (cn > c->cap_nodes) {
        NB_E(ensure(c->node_start, cn * 4)); NB_E(ensure(c->node_level, cn));
        NB_E(ensure(c->node_parent, cn * 4)); NB_E(ensure(c->node_link, cn * 4));
        NB_E(ensure(c->node_count, cn * 4)); NB_E(ensure(c->node_nchild, cn * 4));
        NB_E(ensure(c->node_arrive, cn * 4));
        NB_E(ensure(c->nodeA, cn * 16)); NB_E(ensure(c->nodeB, cn * 16));
        NB_E(ensure(c->mass2, cn * 8)); NB_E(ensure(c->nodeQ, cn * 32));
        c->cap_nodes = cn;
    }
    if (nsys > c->cap_sys) {
        NB_E(ensure(c->sys_off, (size_t)(nsys + 1) * 8)); NB_E(ensure(c->sys_box, (size_t)nsys * sizeof(SysBox)));
        NB_E(ensure(c->sys_boxord, (size_t)nsys * 24)); NB_E(ensure(c->sys_eps2, (size_t)nsys * 4));
        NB_E(ensure(c->sys_eps, (size_t)nsys * 4));
        NB_E(ensure(c->sys_root, (size_t)nsys * 4));
        c->cap_sys = nsys;
    }
#undef NB_E
    return cudaSuccess;
}

Layout make_layout(int64_t n, int nsys) {
    Layout L;
    L.n = n;
    L.nsys = nsys;
    int sb = 0;
    while ((1 << sb) < nsys) sb++;
    L.sysbits = nsys > 1 ? sb : 0;
    L.levels = std::min(kMaxLevels, (63 - L.sysbits) / 3);
    L.keybits = L.sysbits + 3 * L.levels;
    return L;
}

// Keys, sort and tree of n particles whose positions are x, y, z (FP32, or
// FP64 when dbl); pos4 must be filled by the caller-specific gather given
// the permutation in vals (fill_pos4 == true: gather from x, y, z, m here).
// near_order: the positions are in the order of the previous build (the
// particles have moved since), so their keys are nearly sorted: the near-order
// sort moves every key twice where the radix sort moves it seven times.
// hint (nullable, not near_order): a permutation of 0..n-1 that nearly sorts
// the keys (the Morton order of this context's last step call, as caller
// indices): the keys are gathered into that order and sorted by the
// near-order sort by (key, caller index), the same result as the radix sort
// of the caller's order.
nbody_status build_core(nbody_ctx *c, const Layout &L, const void *x, const void *y,
                        const void *z, bool dbl, const float *m, bool fill_pos4,
                        bool near_order = false, const uint32_t *hint = nullptr) {
    cudaStream_t s = c->stream;
    launch_bbox(s, L, x, y, z, dbl, P<int64_t>(c->sys_off), P<uint32_t>(c->sys_boxord),
                P<SysBox>(c->sys_box), c->nsm);
    c->kernels += 3;
    if (near_order && nosort_fits(L.n)) {
        launch_keys(s, L, x, y, z, dbl, P<int64_t>(c->sys_off), P<SysBox>(c->sys_box),
                    P<uint64_t>(c->keys), P<uint32_t>(c->vals), nullptr, c->nsm);
        nosort(s, P<uint64_t>(c->keys), P<uint64_t>(c->keys_alt), P<uint32_t>(c->vals),
               P<uint32_t>(c->vals_alt), L.n, c->rs_temp.p, &c->ds->status);
        c->kernels += 1 + nosort_kernels();
        std::swap(c->keys, c->keys_alt);
        std::swap(c->vals, c->vals_alt);
    } else if (hint && nosort_fits(L.n)) {
        launch_keys(s, L, x, y, z, dbl, P<int64_t>(c->sys_off), P<SysBox>(c->sys_box),
                    P<uint64_t>(c->keys), P<uint32_t>(c->vals), nullptr, c->nsm);
        nosort_hint_gather(s, L.n, P<uint64_t>(c->keys), hint, P<uint64_t>(c->keys_alt),
                           P<uint32_t>(c->vals_alt));
        // values: the caller indices; vals_alt is read by the scatter before
        // the bucket pass uses it as scratch
        nosort(s, P<uint64_t>(c->keys_alt), P<uint64_t>(c->keys), P<uint32_t>(c->vals_alt),
               P<uint32_t>(c->vals), L.n, c->rs_temp.p, &c->ds->status, P<uint32_t>(c->vals_alt));
        c->kernels += 2 + nosort_kernels();
    } else {
        radix_prepare(s, L.n, c->rs_temp.p);
        launch_keys(s, L, x, y, z, dbl, P<int64_t>(c->sys_off), P<SysBox>(c->sys_box),
                    P<uint64_t>(c->keys), P<uint32_t>(c->vals), c->rs_temp.p, c->nsm);
        c->kernels += 2 + radix_passes(L.keybits);  // keys, digit starts, passes
        if (radix_sort(s, P<uint64_t>(c->keys), P<uint32_t>(c->vals), P<uint64_t>(c->keys_alt),
                       P<uint32_t>(c->vals_alt), L.n, L.keybits, c->rs_temp.p, true,
                       &c->ds->status, c->nsm)) {
            std::swap(c->keys, c->keys_alt);
            std::swap(c->vals, c->vals_alt);
        }
    }
    if (fill_pos4) {
        launch_gather_pos4(s, L.n, P<uint32_t>(c->vals), x, y, z, dbl, m, P<float4>(c->pos4));
        c->kernels += 1;
    }
    NB_CUDA(c, cudaGetLastError());
    return NBODY_OK;
}

// The hint for a call's first sort: the Morton order (as caller indices) that
// the context's last step call ended in, when it had the same particle count
// and systems.
const uint32_t *first_sort_hint(const nbody_ctx *c, const Layout &L) {
    return (c->hint_n == L.n && c->hint_nsys == L.nsys && c->last_ids.p)
               ? static_cast<const uint32_t *>(c->last_ids.p)
               : nullptr;
}

nbody_status build_tree_groups(nbody_ctx *c, const Layout &L) {
    cudaStream_t s = c->stream;
    c->costs_valid = false;
    build_tree(s, L, P<uint64_t>(c->keys), P<float4>(c->pos4), P<SysBox>(c->sys_box),
               P<int64_t>(c->sys_off), c->cfg.leaf_cap, c->cfg.G, c->cap_nodes, P<int8_t>(c->delta),
               P<int8_t>(c->leaflev), c->tree_temp.p, c->ds, P<int32_t>(c->node_start),
               P<int8_t>(c->node_level), P<int32_t>(c->node_parent), P<int32_t>(c->node_link),
               P<int32_t>(c->node_count), P<int32_t>(c->node_nchild), P<int32_t>(c->node_arrive),
               P<float4>(c->nodeA), P<float4>(c->nodeB), P<float2>(c->mass2),
               c->cfg.quadrupole ? P<float4>(c->nodeQ) : nullptr, P<int32_t>(c->sys_root), c->nsm);
    build_groups(s, L, c->cfg.group_size, P<float4>(c->pos4), P<int64_t>(c->sys_off),
                 P<int32_t>(c->node_start), P<int32_t>(c->node_parent), P<int32_t>(c->node_count),
                 P<int32_t>(c->node_nchild), P<int32_t>(c->node_link), c->ds,
                 P<uint8_t>(c->gflag), c->grp_temp.p, P<int32_t>(c->grp_first),
                 P<int32_t>(c->grp_count), P<float4>(c->grp_sphere), P<int32_t>(c->grp_sys),
                 c->nsm);
    // tree: leaflevel, level scan, level offsets, node zeroing, nodes, two
    // system-root kernels, moments; groups: 5
    c->kernels += 8 + 5;
    NB_CUDA(c, cudaGetLastError());
    return NBODY_OK;
}

// Refit of the current tree to the positions now in pos4 (sorted order):
// moments with the child-recurrence b_J, then the group spheres.
nbody_status refit_tree_groups(nbody_ctx *c, const Layout &L) {
    cudaStream_t s = c->stream;
    c->costs_valid = false;
    tree_moments(s, L, P<uint64_t>(c->keys), P<float4>(c->pos4), P<SysBox>(c->sys_box),
                 c->cfg.leaf_cap, c->cfg.G, c->ds, P<int32_t>(c->node_start),
                 P<int8_t>(c->node_level), P<int32_t>(c->node_parent), P<int32_t>(c->node_link),
                 P<int32_t>(c->node_count), P<int32_t>(c->node_nchild), P<int32_t>(c->node_arrive),
                 P<float4>(c->nodeA), P<float4>(c->nodeB),
                 P<float2>(c->mass2), c->cfg.quadrupole ? P<float4>(c->nodeQ) : nullptr, c->nsm,
                 true);
    refit_groups(s, L, c->cfg.group_size, P<float4>(c->pos4), P<int64_t>(c->sys_off), c->ds,
                 P<int32_t>(c->grp_first), P<int32_t>(c->grp_count), P<float4>(c->grp_sphere),
                 P<int32_t>(c->grp_sys), c->nsm);
    c->kernels += 1 + 1;
    NB_CUDA(c, cudaGetLastError());
    return NBODY_OK;
}

// Upload the CSR offsets and per-system eps^2.
nbody_status upload_systems(nbody_ctx *c, int nsys, const int64_t *offsets, const float *eps_sys) {
    std::vector<int64_t> off(nsys + 1);
    std::vector<float> e2(nsys), e1(nsys);
    if (offsets) {
        std::memcpy(off.data(), offsets, sizeof(int64_t) * (nsys + 1));
    } else {
        off[0] = 0;
    }
    for (int s = 0; s < nsys; s++) {
        float e = eps_sys ? eps_sys[s] : c->cfg.eps;
        e1[s] = e;
        e2[s] = e * e;
    }
    NB_CUDA(c, cudaMemcpyAsync(c->sys_off.p, off.data(), sizeof(int64_t) * (nsys + 1),
                               cudaMemcpyHostToDevice, c->stream));
    NB_CUDA(c, cudaMemcpyAsync(c->sys_eps2.p, e2.data(), sizeof(float) * nsys,
                               cudaMemcpyHostToDevice, c->stream));
    NB_CUDA(c, cudaMemcpyAsync(c->sys_eps.p, e1.data(), sizeof(float) * nsys,
                               cudaMemcpyHostToDevice, c->stream));
    // the copies read pageable host vectors: make sure they have completed
    NB_CUDA(c, cudaStreamSynchronize(c->stream));
    return NBODY_OK;
}

bool any_zero_eps(nbody_ctx *c, int nsys, const float *eps_sys) {
    if (!eps_sys) return !(c->cfg.eps > 0.0f);
    for (int s = 0; s < nsys; s++)
        if (!(eps_sys[s] > 0.0f)) return true;
    return false;
}

nbody_status check_systems(nbody_ctx *c, int32_t nsys, const int64_t *offsets,
                           const float *eps_sys) {
    if (nsys < 1 || nsys > (1 << 20)) return fail(c, NBODY_EINVAL, "nsys must be in 1..2^20");
    if (!offsets) return fail(c, NBODY_EINVAL, "offsets is NULL");
    if (offsets[0] != 0) return fail(c, NBODY_EINVAL, "offsets[0] must be 0");
    for (int s = 0; s < nsys; s++)
        if (offsets[s + 1] < offsets[s]) return fail(c, NBODY_EINVAL, "offsets must be non-decreasing");
    if (offsets[nsys] < 1) return fail(c, NBODY_EINVAL, "no particles");
    if (offsets[nsys] >= (int64_t)1 << 31) return fail(c, NBODY_EINVAL, "n must be < 2^31");
    if (eps_sys)
        for (int s = 0; s < nsys; s++)
            if (!(eps_sys[s] >= 0.0f) || !std::isfinite(eps_sys[s]))
                return fail(c, NBODY_EINVAL, "eps_sys must be finite and >= 0");
    return NBODY_OK;
}

nbody_status read_status(nbody_ctx *c) {
    NB_CUDA(c, cudaMemcpyAsync(c->h_ds, c->ds, sizeof(DevState), cudaMemcpyDeviceToHost, c->stream));
    NB_CUDA(c, cudaStreamSynchronize(c->stream));
    if (c->h_ds->status & kStatusTimeout)
        return fail(c, NBODY_ETIMEOUT, "a bounded device wait (radix-sort look-back) ran out");
    if (c->h_ds->status & kStatusBadTree)
        return fail(c, NBODY_ECUDA, "internal error: a tree index failed its bounds check");
    if (c->h_ds->status & kStatusStackOverflow)
        return fail(c, NBODY_EOVERFLOW,
                    "traversal stack or node capacity overflowed; increase stack_depth");
    return NBODY_OK;
}

nbody_status do_build(nbody_ctx *c, int64_t n, int nsys, const int64_t *offsets,
                      const float *eps_sys, const float *x, const float *y, const float *z,
                      const float *m) {
    Layout L = make_layout(n, nsys);
    cudaError_t e = ensure_capacity(c, n, nsys, L.levels);
    if (e != cudaSuccess) return fail(c, NBODY_ENOMEM, std::string("allocation: ") + cudaGetErrorString(e));
    std::vector<int64_t> off1 = {0, n};
    nbody_status st = upload_systems(c, nsys, offsets ? offsets : off1.data(), eps_sys);
    if (st != NBODY_OK) return st;
    c->kernels = 0;
    c->wev_used = 0;
    NB_CUDA(c, cudaMemsetAsync(c->ds, 0, sizeof(DevState), c->stream));
    const void *dx, *dy, *dz, *dm;
    size_t fb = (size_t)n * 4;
    NB_CUDA(c, stage_in(c, 0, x, fb, &dx));
    NB_CUDA(c, stage_in(c, 1, y, fb, &dy));
    NB_CUDA(c, stage_in(c, 2, z, fb, &dz));
    NB_CUDA(c, stage_in(c, 3, m, fb, &dm));
    NB_CUDA(c, cudaEventRecord(c->ev[0], c->stream));
    st = build_core(c, L, dx, dy, dz, false, (const float *)dm, true);
    if (st != NBODY_OK) return st;
    st = build_tree_groups(c, L);
    if (st != NBODY_OK) return st;
    NB_CUDA(c, cudaEventRecord(c->ev[1], c->stream));
    st = read_status(c);
    if (st != NBODY_OK) return st;
    NB_CUDA(c, cudaEventElapsedTime(&c->last_ms_build, c->ev[0], c->ev[1]));
    c->L = L;
    c->built = true;
    c->eps_zero = any_zero_eps(c, nsys, eps_sys);
    c->last.n_nodes = c->h_ds->nnodes;
    c->last.n_groups = c->h_ds->ngroups;
    c->last.levels = L.levels;
    c->last.ms_build = c->last_ms_build;
    c->last.kernels = c->kernels;
    return NBODY_OK;
}

// Compensated accumulation: on request, or (automatic) where the MAC is so
// tight that the FP32 rounding of plain sums adds measurably to the force
// error: the precision sweep on the N = 2^23 galaxy saw plain and
// compensated p50 errors part from Delta_acc = 2^-18 down.
constexpr float kAutoCompensateDacc = 0x1p-18f;
bool use_compensation(const nbody_config &c) {
    return c.compensated == 1 || (c.compensated == 2 && c.delta_acc <= kAutoCompensateDacc);
}

WalkShape walk_shape(nbody_ctx *c, bool geometric, bool phi, bool safe) {
    WalkShape sh;
    sh.ipl = c->cfg.ipl;
    sh.geometric = geometric;
    sh.potential = phi;
    sh.compensated = use_compensation(c->cfg);
    sh.safe = safe;
    sh.quad = c->cfg.quadrupole != 0;
    sh.pipeline = c->cfg.walk_pipeline != 0;
    sh.warps_per_block = c->cfg.warps_per_block;
    sh.warps_launched = &c->walk_warps;
    return sh;
}

WalkArgs walk_args(nbody_ctx *c) {
    WalkArgs a{};
    a.pos4 = P<float4>(c->pos4);
    a.nodeA = P<float4>(c->nodeA);
    a.nodeB = P<float4>(c->nodeB);
    a.nodeQ = P<float4>(c->nodeQ);
    a.grp_first = P<int32_t>(c->grp_first);
    a.grp_count = P<int32_t>(c->grp_count);
    a.grp_sphere = P<float4>(c->grp_sphere);
    a.grp_alpha = P<float>(c->grp_alpha);
    a.grp_sys = P<int32_t>(c->grp_sys);
    a.order = nullptr;
    a.sys_eps2 = P<float>(c->sys_eps2);
    a.sys_root = P<int32_t>(c->sys_root);
    a.ds = c->ds;
    a.grp_cost = P<int32_t>(c->grp_cost);
    a.n = c->L.n;
    a.G = c->cfg.G;
    a.theta = c->cfg.theta;
    a.list_depth = c->cfg.list_depth;
    a.stack_depth = c->cfg.stack_depth;
    return a;
}

// Reset the walk's queue head and counters (status is kept).
nbody_status reset_walk_counters(nbody_ctx *c, bool accumulators) {
    char *base = reinterpret_cast<char *>(c->ds);
    NB_CUDA(c, cudaMemsetAsync(base + offsetof(DevState, queue_head), 0, sizeof(int32_t), c->stream));
    if (accumulators) {
        NB_CUDA(c, cudaMemsetAsync(base + offsetof(DevState, max_stack), 0, sizeof(int32_t), c->stream));
        NB_CUDA(c, cudaMemsetAsync(base + offsetof(DevState, list_entries), 0,
                                   3 * sizeof(unsigned long long), c->stream));
    }
    return NBODY_OK;
}

// Events from a pool that grows on demand (timing of asynchronous phases).
cudaError_t pool_event(nbody_ctx *c, cudaEvent_t *out);

cudaError_t pool_event(nbody_ctx *c, cudaEvent_t *out) {
    if ((int)c->evpool.size() <= c->evused) {
        cudaEvent_t ev;
        cudaError_t e = cudaEventCreate(&ev);
        if (e != cudaSuccess) return e;
        c->evpool.push_back(ev);
    }
    *out = c->evpool[c->evused++];
    return cudaSuccess;
}

// Number of groups of the current build, read back to the host (a sync).
nbody_status host_ngroups(nbody_ctx *c, int64_t *ng) {
    NB_CUDA(c, cudaMemcpyAsync(&c->h_ds->ngroups, &c->ds->ngroups, sizeof(int32_t),
                               cudaMemcpyDeviceToHost, c->stream));
    NB_CUDA(c, cudaStreamSynchronize(c->stream));
    *ng = c->h_ds->ngroups;
    return NBODY_OK;
}

cudaError_t ensure_mlp_buffers(nbody_ctx *c) {
    const int64_t n = std::max<int64_t>(c->cap_n, 1);
    cudaError_t e = ensure(c->feat, (size_t)n * 8 * sizeof(float));
    if (e == cudaSuccess) e = ensure(c->target, (size_t)n * 4);
    if (e == cudaSuccess) e = ensure(c->score, (size_t)n * 4);
    if (e == cudaSuccess) e = ensure(c->okey, (size_t)n * 8);
    if (e == cudaSuccess) e = ensure(c->okey_alt, (size_t)n * 8);
    if (e == cudaSuccess) e = ensure(c->oval, (size_t)n * 4);
    if (e == cudaSuccess) e = ensure(c->oval_alt, (size_t)n * 4);
    return e;
}

void launch_features(nbody_ctx *c) {
    launch_mlp_features(c->stream, c->L, c->ds, P<int32_t>(c->grp_first), P<int32_t>(c->grp_count),
                        P<float4>(c->grp_sphere), P<int32_t>(c->grp_sys), P<float>(c->aold_s),
                        P<uint64_t>(c->keys), P<float4>(c->nodeA), P<int32_t>(c->sys_root),
                        P<SysBox>(c->sys_box), P<int64_t>(c->sys_off), P<float>(c->feat), c->nsm);
    c->kernels += 1;
}

// Queue order of the walk for the configured schedule (NULL: Morton order).
// pcost: per-particle cost of the previous walk (sorted order), for LASTCOST.
nbody_status compute_order(nbody_ctx *c, const float *pcost, const int32_t **order) {
    *order = nullptr;
    const int sched = c->cfg.schedule;
    if (sched == NBODY_SCHED_MORTON) return NBODY_OK;
    if (sched == NBODY_SCHED_MLP && !c->mlp_ready)
        return fail(c, NBODY_EINVAL, "schedule MLP needs parameters (nbody_mlp_set_params)");
    if (sched == NBODY_SCHED_LASTCOST && !pcost)
        return fail(c, NBODY_EINVAL, "schedule LASTCOST needs a previous walk");
    // The group count stays on the device: every kernel below reads it there
    // and the sort takes it as its key count, so nothing here waits for the
    // build and the ordering can be captured in a graph.
    cudaError_t e = ensure_mlp_buffers(c);
    if (e != cudaSuccess) return fail(c, NBODY_ENOMEM, "allocation");
    const int32_t *png = &c->ds->ngroups;
    if (sched == NBODY_SCHED_MLP) {
        launch_features(c);
        const float *nrm = c->mlp_norm_set ? P<float>(c->mlp_norm) : nullptr;
        launch_mlp_forward(c->stream, png, 0, P<float>(c->feat),
                           reinterpret_cast<const __nv_bfloat16 *>(c->mlp_wb.p), nrm,
                           nrm ? nrm + 16 : nullptr, P<float>(c->score), c->nsm);
    } else {
        launch_lastcost_score(c->stream, png, P<int32_t>(c->grp_first), pcost, P<float>(c->score),
                              c->nsm);
    }
    launch_order_keys(c->stream, png, P<float>(c->score), P<int32_t>(c->grp_count),
                      P<uint64_t>(c->okey), P<uint32_t>(c->oval), c->nsm);
    // score (MLP: features + forward) and order keys; histogram, digit starts, passes
    c->kernels += (sched == NBODY_SCHED_MLP ? 3 : 2) + 2 + radix_passes(32);
    if (radix_sort(c->stream, P<uint64_t>(c->okey), P<uint32_t>(c->oval), P<uint64_t>(c->okey_alt),
                   P<uint32_t>(c->oval_alt), std::max<int64_t>(c->cap_n, 1), 32, c->rs_temp.p,
                   false, &c->ds->status, c->nsm, png)) {
        std::swap(c->okey, c->okey_alt);
        std::swap(c->oval, c->oval_alt);
    }
    NB_CUDA(c, cudaGetLastError());
    *order = P<int32_t>(c->oval);
    return NBODY_OK;
}

// Walk over the current groups; aold_s (sorted) must hold |a_old|.
nbody_status run_walk(nbody_ctx *c, bool geometric, bool phi, bool safe, const int32_t *perm,
                      float *ax, float *ay, float *az, float *ph, float4 *acc_sorted,
                      bool reset_accumulators = true, const float *pcost = nullptr,
                      const int32_t *active_order = nullptr, const int32_t *nactive = nullptr) {
    const int32_t *order = active_order;
    if (!geometric && !active_order) {
        nbody_status so = compute_order(c, pcost, &order);
        if (so != NBODY_OK) return so;
    }
    nbody_status st = reset_walk_counters(c, reset_accumulators);
    if (st != NBODY_OK) return st;
    if (!geometric) {
        launch_group_alpha(c->stream, c->L.n, c->ds, P<int32_t>(c->grp_first),
                           P<int32_t>(c->grp_count), P<float>(c->aold_s), c->cfg.delta_acc,
                           P<float>(c->grp_alpha), c->nsm);
        c->kernels += 1;
    }
    while (!c->capturing && (int)c->wev.size() < c->wev_used + 2) {
        cudaEvent_t ev;
        NB_CUDA(c, cudaEventCreate(&ev));
        c->wev.push_back(ev);
    }
    WalkArgs a = walk_args(c);
    a.order = order;
    a.nactive = nactive;
    a.perm = perm;
    a.ax = ax;
    a.ay = ay;
    a.az = az;
    a.phi = ph;
    a.acc_sorted = acc_sorted;
    // inside a graph capture: event nodes (recorded at every replay)
    const bool gtime = c->capturing && c->gwev_used + 2 <= 4 && c->gwev[c->gwev_used];
    if (!c->capturing) NB_CUDA(c, cudaEventRecord(c->wev[c->wev_used], c->stream));
    if (gtime) NB_CUDA(c, cudaEventRecordWithFlags(c->gwev[c->gwev_used], c->stream, cudaEventRecordExternal));
    cudaError_t e = launch_walk(c->stream, a, walk_shape(c, geometric, phi, safe), c->nsm);
    if (e != cudaSuccess) return cuda_fail(c, e, "walk launch");
    if (!c->capturing) {
        NB_CUDA(c, cudaEventRecord(c->wev[c->wev_used + 1], c->stream));
        c->wev_used += 2;
    }
    if (gtime) {
        NB_CUDA(c, cudaEventRecordWithFlags(c->gwev[c->gwev_used + 1], c->stream, cudaEventRecordExternal));
        c->gwev_used += 2;
    }
    c->kernels += 1;
    if (!geometric) c->costs_valid = true;
    return NBODY_OK;
}

// After a synchronisation: total walk-kernel time of the recorded pairs.
float collect_walk_ms(nbody_ctx *c, int *launches) {
    float t = 0.0f;
    for (int k = 0; k + 1 < c->wev_used; k += 2) {
        float ms = 0.0f;
        if (cudaEventElapsedTime(&ms, c->wev[k], c->wev[k + 1]) == cudaSuccess) t += ms;
        else cudaGetLastError();  // a timing query must not leave an error behind
    }
    *launches = c->wev_used / 2;
    c->wev_used = 0;
    return t;
}


}  // namespace

// ============================================================================ ABI
extern "C" {

int32_t nbody_abi_version(void) { return NBODY_ABI_VERSION; }

void nbody_config_default(nbody_config *c) {
    if (!c) return;
    std::memset(c, 0, sizeof *c);
    c->G = 1.0f;
    c->eps = 1.0f / 64.0f;
    c->delta_acc = 1.0f / 512.0f;
    c->theta = 0.5f;
    c->leaf_cap = 16;
    c->group_size = 64;
    c->ipl = 3;
    c->list_depth = 256;
    c->stack_depth = 256;
    c->warps_per_block = 4;
    c->compensated = 2;
    c->want_potential = 0;
    c->schedule = NBODY_SCHED_MORTON;
    c->use_graph = 0;
    c->rebuild_interval = 1;
    c->quadrupole = 0;
    c->block_levels = 0;
    c->block_eta = 0.025f;
    c->walk_pipeline = 0;
}

nbody_status nbody_create(nbody_ctx **out, const nbody_config *cfg, void *cuda_stream) {
    if (!out) return fail(nullptr, NBODY_EINVAL, "out is NULL");
    *out = nullptr;
    nbody_config c;
    if (cfg) c = *cfg; else nbody_config_default(&c);
    std::string why;
    if (!config_ok(&c, why)) return fail(nullptr, NBODY_EINVAL, why);
    nbody_ctx *ctx = new (std::nothrow) nbody_ctx();
    if (!ctx) return fail(nullptr, NBODY_ENOMEM, "host allocation");
    ctx->cfg = c;
    ctx->stream = (cudaStream_t)cuda_stream;
    cudaError_t e = cudaGetDevice(&ctx->device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&ctx->nsm, cudaDevAttrMultiProcessorCount, ctx->device);
    if (e == cudaSuccess) e = cudaMalloc(&ctx->ds, sizeof(DevState));
    if (e == cudaSuccess) e = cudaMallocHost(&ctx->h_ds, sizeof(DevState));
    if (e == cudaSuccess) e = cudaMallocHost(&ctx->h_diag, 8 * sizeof(double));
    for (int k = 0; k < 4 && e == cudaSuccess; k++) e = cudaEventCreate(&ctx->ev[k]);
    if (e == cudaSuccess) e = cudaMemset(ctx->ds, 0, sizeof(DevState));
    if (e != cudaSuccess) {
        nbody_status st = cuda_fail(nullptr, e, "nbody_create");
        nbody_destroy(ctx);
        return st;
    }
    *out = ctx;
    return NBODY_OK;
}

nbody_status nbody_destroy(nbody_ctx *ctx) {
    if (!ctx) return NBODY_OK;
    cudaStreamSynchronize(ctx->stream);
    for (DevBuf *b : ctx->owned)
        if (b->p) cudaFree(b->p);
    if (ctx->ds) cudaFree(ctx->ds);
    if (ctx->h_ds) cudaFreeHost(ctx->h_ds);
    if (ctx->h_diag) cudaFreeHost(ctx->h_diag);
    for (auto &ev : ctx->ev)
        if (ev) cudaEventDestroy(ev);
    for (auto ev : ctx->wev) cudaEventDestroy(ev);
    for (auto ev : ctx->gwev)
        if (ev) cudaEventDestroy(ev);
    if (ctx->gexec) cudaGraphExecDestroy(ctx->gexec);
    if (ctx->gstream) cudaStreamDestroy(ctx->gstream);
    for (auto ev : ctx->evpool) cudaEventDestroy(ev);
    delete ctx;
    return NBODY_OK;
}

nbody_status nbody_set_config(nbody_ctx *ctx, const nbody_config *cfg) {
    if (!ctx || !cfg) return fail(ctx, NBODY_EINVAL, "NULL argument");
    std::string why;
    if (!config_ok(cfg, why)) return fail(ctx, NBODY_EINVAL, why);
    bool rebuild = cfg->leaf_cap != ctx->cfg.leaf_cap || cfg->group_size != ctx->cfg.group_size ||
                   cfg->G != ctx->cfg.G || cfg->eps != ctx->cfg.eps;
    ctx->cfg = *cfg;
    if (rebuild) ctx->built = false;
    return NBODY_OK;
}

nbody_status nbody_get_config(const nbody_ctx *ctx, nbody_config *cfg) {
    if (!ctx || !cfg) return NBODY_EINVAL;
    *cfg = ctx->cfg;
    return NBODY_OK;
}

nbody_status nbody_build(nbody_ctx *ctx, int64_t n, const float *x, const float *y,
                         const float *z, const float *m) {
    if (!ctx) return fail(nullptr, NBODY_EINVAL, "ctx is NULL");
    if (n < 1 || n >= ((int64_t)1 << 31)) return fail(ctx, NBODY_EINVAL, "n must be in 1..2^31-1");
    if (!x || !y || !z || !m) return fail(ctx, NBODY_EINVAL, "NULL array");
    ctx->built = false;
    return do_build(ctx, n, 1, nullptr, nullptr, x, y, z, m);
}

nbody_status nbody_refit(nbody_ctx *ctx, const float *x, const float *y, const float *z,
                         const float *m) {
    if (!ctx) return fail(nullptr, NBODY_EINVAL, "ctx is NULL");
    if (!x || !y || !z || !m) return fail(ctx, NBODY_EINVAL, "NULL array");
    if (!ctx->built) return fail(ctx, NBODY_ENOTBUILT, "nbody_refit before nbody_build");
    const int64_t n = ctx->L.n;
    const size_t fb = (size_t)n * 4;
    const void *dx, *dy, *dz, *dm;
    NB_CUDA(ctx, stage_in(ctx, 0, x, fb, &dx));
    NB_CUDA(ctx, stage_in(ctx, 1, y, fb, &dy));
    NB_CUDA(ctx, stage_in(ctx, 2, z, fb, &dz));
    NB_CUDA(ctx, stage_in(ctx, 3, m, fb, &dm));
    ctx->kernels = 0;
    NB_CUDA(ctx, cudaEventRecord(ctx->ev[0], ctx->stream));
    // the new positions into the build's sorted order (vals maps sorted
    // index -> caller index)
    launch_gather_pos4(ctx->stream, n, P<uint32_t>(ctx->vals), dx, dy, dz, false,
                       (const float *)dm, P<float4>(ctx->pos4));
    ctx->kernels += 1;
    nbody_status st = refit_tree_groups(ctx, ctx->L);
    if (st != NBODY_OK) return st;
    NB_CUDA(ctx, cudaEventRecord(ctx->ev[1], ctx->stream));
    st = read_status(ctx);
    if (st != NBODY_OK) return st;
    NB_CUDA(ctx, cudaEventElapsedTime(&ctx->last_ms_build, ctx->ev[0], ctx->ev[1]));
    ctx->last.ms_build = ctx->last_ms_build;
    ctx->last.kernels = ctx->kernels;
    return NBODY_OK;
}

int32_t nbody_rebuild_due(const float *cost_ms, int32_t m) {
    if (!cost_ms || m < 2) return 0;
    double sum = 0.0;
    for (int32_t i = 0; i < m; i++) sum += (double)cost_ms[i];
    return (double)cost_ms[m - 1] * (double)m > sum ? 1 : 0;
}

nbody_status nbody_build_batched(nbody_ctx *ctx, int32_t nsys, const int64_t *offsets,
                                 const float *eps_sys, const float *x, const float *y,
                                 const float *z, const float *m) {
    if (!ctx) return fail(nullptr, NBODY_EINVAL, "ctx is NULL");
    nbody_status st = check_systems(ctx, nsys, offsets, eps_sys);
    if (st != NBODY_OK) return st;
    if (!x || !y || !z || !m) return fail(ctx, NBODY_EINVAL, "NULL array");
    ctx->built = false;
    return do_build(ctx, offsets[nsys], nsys, offsets, eps_sys, x, y, z, m);
}

nbody_status nbody_walk(nbody_ctx *ctx, const float *a_old, float *ax, float *ay, float *az,
                        float *phi, nbody_stats *stats) {
    if (!ctx) return fail(nullptr, NBODY_EINVAL, "ctx is NULL");
    if (!ctx->built) return fail(ctx, NBODY_ENOTBUILT, "nbody_walk before nbody_build");
    if (!ax || !ay || !az) return fail(ctx, NBODY_EINVAL, "NULL output array");
    if (phi && !ctx->cfg.want_potential) return fail(ctx, NBODY_EINVAL, "phi requested but want_potential = 0");
    const int64_t n = ctx->L.n;
    const size_t fb = (size_t)n * 4;
    cudaStream_t s = ctx->stream;
    void *dax, *day, *daz, *dph;
    NB_CUDA(ctx, stage_out(ctx, 4, ax, fb, &dax));
    NB_CUDA(ctx, stage_out(ctx, 5, ay, fb, &day));
    NB_CUDA(ctx, stage_out(ctx, 6, az, fb, &daz));
    NB_CUDA(ctx, stage_out(ctx, 7, phi, fb, &dph));
    const bool safe = ctx->eps_zero;
    const bool want_phi = phi != nullptr;
    ctx->kernels = 0;
    ctx->wev_used = 0;
    char *dsb = reinterpret_cast<char *>(ctx->ds);
    NB_CUDA(ctx, cudaMemsetAsync(dsb + offsetof(DevState, status), 0, sizeof(int32_t), s));
    NB_CUDA(ctx, cudaEventRecord(ctx->ev[2], s));
    nbody_status st;
    if (a_old) {
        const void *dao;
        NB_CUDA(ctx, stage_in(ctx, 8, a_old, fb, &dao));
        launch_gather_f32(s, n, P<uint32_t>(ctx->vals), (const float *)dao, P<float>(ctx->aold_s));
        ctx->kernels += 1;
    } else {
        // bootstrap: geometric criterion first, its |a| feeds Eq. 2
        st = run_walk(ctx, true, false, safe, nullptr, nullptr, nullptr, nullptr, nullptr,
                      P<float4>(ctx->acc_s));
        if (st != NBODY_OK) return st;
        launch_acc_mag(s, n, P<float4>(ctx->acc_s), P<float>(ctx->aold_s));
        ctx->kernels += 1;
    }
    const bool have_pcost = ctx->costs_valid && ctx->pcost_walk.p;
    st = run_walk(ctx, false, want_phi, safe, (const int32_t *)P<uint32_t>(ctx->vals),
                  (float *)dax, (float *)day, (float *)daz, (float *)dph, nullptr, true,
                  have_pcost ? P<float>(ctx->pcost_walk) : nullptr);
    if (st != NBODY_OK) return st;
    if (ensure(ctx->pcost_walk, (size_t)n * 4) == cudaSuccess) {
        launch_spread_cost(s, &ctx->ds->ngroups, P<int32_t>(ctx->grp_first), P<int32_t>(ctx->grp_count),
                           P<int32_t>(ctx->grp_cost), P<float>(ctx->pcost_walk), ctx->nsm);
        ctx->kernels += 1;
    }
    NB_CUDA(ctx, cudaEventRecord(ctx->ev[3], s));
    NB_CUDA(ctx, stage_out_finish(ctx, ax, dax, fb));
    NB_CUDA(ctx, stage_out_finish(ctx, ay, day, fb));
    NB_CUDA(ctx, stage_out_finish(ctx, az, daz, fb));
    NB_CUDA(ctx, stage_out_finish(ctx, phi, dph, fb));
    st = read_status(ctx);
    float ms = 0.0f;
    if (cudaEventElapsedTime(&ms, ctx->ev[2], ctx->ev[3]) != cudaSuccess) cudaGetLastError();
    ctx->last.n_groups = ctx->h_ds->ngroups;
    ctx->last.interactions = (int64_t)ctx->h_ds->interactions;
    ctx->last.list_entries = (int64_t)ctx->h_ds->list_entries;
    ctx->last.quad_interactions = (int64_t)ctx->h_ds->quad_entries;
    ctx->last.walk_warps = ctx->walk_warps;
    ctx->last.max_stack = ctx->h_ds->max_stack;
    ctx->last.ms_walk = ms;
    ctx->last.ms_walk_kernel = collect_walk_ms(ctx, &ctx->last.walk_launches);
    ctx->last.kernels = ctx->kernels;
    if (stats) *stats = ctx->last;
    return st;
}

nbody_status nbody_direct(int64_t n, const float *x, const float *y, const float *z,
                          const float *m, float G, float eps, int32_t compensated, float *ax,
                          float *ay, float *az, float *phi, void *cuda_stream) {
    if (n < 1 || n >= ((int64_t)1 << 31)) return fail(nullptr, NBODY_EINVAL, "n must be in 1..2^31-1");
    if (!x || !y || !z || !m || !ax || !ay || !az) return fail(nullptr, NBODY_EINVAL, "NULL array");
    if (!(eps >= 0.0f) || !std::isfinite(eps) || !std::isfinite(G))
        return fail(nullptr, NBODY_EINVAL, "eps must be finite and >= 0");
    cudaStream_t s = (cudaStream_t)cuda_stream;
    const size_t fb = (size_t)n * 4;
    const float *in[4] = {x, y, z, m};
    float *out[4] = {ax, ay, az, phi};
    const float *din[4];
    float *dout[4];
    std::vector<void *> tmp;
    auto cleanup = [&]() {
        for (void *p : tmp) cudaFree(p);
    };
    for (int k = 0; k < 4; k++) {
        if (is_device_ptr(in[k])) {
            din[k] = in[k];
        } else {
            void *p = nullptr;
            cudaError_t e = cudaMalloc(&p, fb);
            if (e == cudaSuccess) e = cudaMemcpyAsync(p, in[k], fb, cudaMemcpyHostToDevice, s);
            if (e != cudaSuccess) { if (p) cudaFree(p); cleanup(); return cuda_fail(nullptr, e, "nbody_direct staging"); }
            tmp.push_back(p);
            din[k] = (const float *)p;
        }
        if (!out[k] || is_device_ptr(out[k])) {
            dout[k] = out[k];
        } else {
            void *p = nullptr;
            cudaError_t e = cudaMalloc(&p, fb);
            if (e != cudaSuccess) { cleanup(); return cuda_fail(nullptr, e, "nbody_direct staging"); }
            tmp.push_back(p);
            dout[k] = (float *)p;
        }
    }
    cudaError_t e = launch_direct(s, n, din[0], din[1], din[2], din[3], G, eps, compensated != 0,
                                  dout[0], dout[1], dout[2], dout[3]);
    for (int k = 0; k < 4 && e == cudaSuccess; k++)
        if (out[k] && dout[k] != out[k]) e = cudaMemcpyAsync(out[k], dout[k], fb, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    cleanup();
    if (e != cudaSuccess) return cuda_fail(nullptr, e, "nbody_direct");
    return NBODY_OK;
}

// Block (hierarchical) time steps, nsteps steps of dt with levels 0..K
// (step dt / 2^k).  The clock ticks in units of dt / 2^K; at tick 0 every
// particle takes the opening half kick of its level, and at each tick where a
// particle is active (its level's step ends there) all particles drift to the
// tick, the tree is rebuilt or refitted (rebuild_interval, per processed
// tick), the groups holding an active particle are walked, and the active
// particles take their closing half kick, a new level and -- except at the
// last tick -- the opening half kick of their next step.  Ticks at which no
// level ends are skipped (their drifts are merged into the next); the
// deepest occupied level is read back after every processed tick.
static nbody_status block_steps(nbody_ctx *ctx, const Layout &L, StepState *S, int &cur,
                                float4 *acc, float dt, int32_t nsteps, bool safe, int &rebuilds,
                                std::vector<int> &marks) {
    if (nsteps == 0) return NBODY_OK;  // no step: the state is returned as given
    cudaStream_t q = ctx->stream;
    const int64_t n = L.n;
    const int K = ctx->cfg.block_levels;
    const float eta = ctx->cfg.block_eta;
    int32_t *dmax = &ctx->ds->block_maxlvl, *dact = &ctx->ds->block_nactive;
    auto read_maxlvl = [&](int *out) -> nbody_status {
        NB_CUDA(ctx, cudaMemcpyAsync(&ctx->h_ds->block_maxlvl, dmax, sizeof(int32_t),
                                     cudaMemcpyDeviceToHost, q));
        NB_CUDA(ctx, cudaStreamSynchronize(q));
        *out = ctx->h_ds->block_maxlvl;
        return (*out >= 0 && *out <= K) ? NBODY_OK
                                        : fail(ctx, NBODY_ECUDA, "internal error: block level out of range");
    };
    NB_CUDA(ctx, cudaMemsetAsync(dmax, 0, sizeof(int32_t), q));
    launch_block_start(q, n, S[cur], acc, dt, K, eta, P<int64_t>(ctx->sys_off), L.nsys,
                       P<float>(ctx->sys_eps), dmax);
    ctx->kernels += 1;
    int kmax = 0;
    nbody_status st = read_maxlvl(&kmax);
    if (st != NBODY_OK) return st;
    const int64_t total = (int64_t)nsteps << K;
    const double tau = (double)dt / (double)(int64_t(1) << K);
    const int interval = ctx->cfg.rebuild_interval;
    std::vector<float> cycle;
    int64_t last = 0;
    int since = 0;
    bool first = true;
    for (int64_t T = 1; T <= total; T++) {
        if (T % (int64_t(1) << (K - kmax))) continue;
        const float span = (float)((double)(T - last) * tau);
        last = T;
        bool rebuild = first || interval == 1;
        if (!rebuild && interval > 1) rebuild = since >= interval;
        if (!rebuild && interval == 0)
            rebuild = since >= 32 || nbody_rebuild_due(cycle.data(), (int32_t)cycle.size()) != 0;
        if (rebuild) {
            since = 0;
            cycle.clear();
        }
        // the first rebuild sorts the caller's order; later ones the last build's
        const bool near_order = !first;
        first = false;
        // drift every particle to tick T (no kick: the kick factor is 0)
        launch_kick_drift(q, n, S[cur], acc, 0.0f, span, rebuild ? nullptr : P<float4>(ctx->pos4));
        ctx->kernels += 1;
        cudaEvent_t e0, e1, e2;
        NB_CUDA(ctx, pool_event(ctx, &e0));
        NB_CUDA(ctx, cudaEventRecord(e0, q));
        if (rebuild) {
            st = build_core(ctx, L, S[cur].x, S[cur].y, S[cur].z, true, S[cur].m, false,
                            near_order, near_order ? nullptr : first_sort_hint(ctx, L));
            if (st != NBODY_OK) return st;
            if (near_order) {
                launch_permute_state(q, n, P<uint32_t>(ctx->vals), S[cur], S[1 - cur], P<float4>(ctx->pos4));
                ctx->kernels += 1;
            } else {
                launch_permute_state_recs(q, n, P<uint32_t>(ctx->vals), S[cur], S[1 - cur],
                                          P<float4>(ctx->pos4), ctx->recs.p);
                ctx->kernels += 2;
            }
            cur = 1 - cur;
            st = build_tree_groups(ctx, L);
            rebuilds++;
        } else {
            st = refit_tree_groups(ctx, L);
        }
        if (st != NBODY_OK) return st;
        NB_CUDA(ctx, pool_event(ctx, &e1));
        NB_CUDA(ctx, cudaEventRecord(e1, q));
        NB_CUDA(ctx, cudaMemcpyAsync(ctx->aold_s.p, S[cur].aold, (size_t)n * 4,
                                     cudaMemcpyDeviceToDevice, q));
        NB_CUDA(ctx, cudaMemsetAsync(dact, 0, sizeof(int32_t), q));
        launch_block_active_groups(q, ctx->ds, P<int32_t>(ctx->grp_first), P<int32_t>(ctx->grp_count),
                                   S[cur].lvl, T, K, P<int32_t>(ctx->grp_order), dact, ctx->nsm);
        ctx->kernels += 1;
        st = run_walk(ctx, false, false, safe, nullptr, nullptr, nullptr, nullptr, nullptr, acc,
                      false, nullptr, P<int32_t>(ctx->grp_order), dact);
        if (st != NBODY_OK) return st;
        NB_CUDA(ctx, pool_event(ctx, &e2));
        NB_CUDA(ctx, cudaEventRecord(e2, q));
        marks.push_back(ctx->evused - 3);
        NB_CUDA(ctx, cudaMemsetAsync(dmax, 0, sizeof(int32_t), q));
        launch_block_kick(q, n, S[cur], acc, T, total, dt, K, eta, P<int64_t>(ctx->sys_off), L.nsys,
                          P<float>(ctx->sys_eps), dmax);
        ctx->kernels += 1;
        st = read_maxlvl(&kmax);
        if (st != NBODY_OK) return st;
        since++;
        if (interval == 0) {
            float c = 0.0f;
            NB_CUDA(ctx, cudaEventElapsedTime(&c, e0, e2));
            cycle.push_back(c);
        }
    }
    return NBODY_OK;
}

static nbody_status step_impl(nbody_ctx *ctx, int32_t nsys, const int64_t *offsets,
                              const float *eps_sys, int64_t n, double *x, double *y, double *z,
                              float *vx, float *vy, float *vz, const float *m, float *ax,
                              float *ay, float *az, float dt, int32_t nsteps, nbody_stats *stats) {
    if (!x || !y || !z || !vx || !vy || !vz || !m || !ax || !ay || !az)
        return fail(ctx, NBODY_EINVAL, "NULL array");
    if (nsteps < 0) return fail(ctx, NBODY_EINVAL, "nsteps must be >= 0");
    if (!std::isfinite(dt)) return fail(ctx, NBODY_EINVAL, "dt must be finite");
    ctx->built = false;
    cudaStream_t s = ctx->stream;
    Layout L = make_layout(n, nsys);
    cudaError_t e = ensure_capacity(ctx, n, nsys, L.levels);
    for (int b = 0; b < 2 && e == cudaSuccess; b++) {
        for (int k = 0; k < 3 && e == cudaSuccess; k++) e = ensure(ctx->st_buf[b][k], (size_t)n * 8);
        for (int k = 3; k < 10 && e == cudaSuccess; k++) e = ensure(ctx->st_buf[b][k], (size_t)n * 4);
        if (e == cudaSuccess && ctx->cfg.block_levels > 0) e = ensure(ctx->st_buf[b][10], (size_t)n);
    }
    if (e == cudaSuccess) e = ensure(ctx->recs, (size_t)n * 64);
    if (e != cudaSuccess) return fail(ctx, NBODY_ENOMEM, std::string("allocation: ") + cudaGetErrorString(e));
    std::vector<int64_t> off1 = {0, n};
    nbody_status st = upload_systems(ctx, nsys, offsets ? offsets : off1.data(), eps_sys);
    if (st != NBODY_OK) return st;
    const bool safe = any_zero_eps(ctx, nsys, eps_sys);
    ctx->L = L;  // the walk's bounds checks read the particle count from here
    StepState S[2];
    for (int b = 0; b < 2; b++) {
        S[b].x = P<double>(ctx->st_buf[b][0]);
        S[b].y = P<double>(ctx->st_buf[b][1]);
        S[b].z = P<double>(ctx->st_buf[b][2]);
        S[b].vx = P<float>(ctx->st_buf[b][3]);
        S[b].vy = P<float>(ctx->st_buf[b][4]);
        S[b].vz = P<float>(ctx->st_buf[b][5]);
        S[b].m = P<float>(ctx->st_buf[b][6]);
        S[b].aold = P<float>(ctx->st_buf[b][7]);
        S[b].id = P<uint32_t>(ctx->st_buf[b][8]);
        // the per-particle cost of the last walk is carried only for the
        // schedule that reads it
        S[b].pcost = ctx->cfg.schedule == NBODY_SCHED_LASTCOST ? P<float>(ctx->st_buf[b][9])
                                                               : nullptr;
        S[b].lvl = ctx->cfg.block_levels > 0 ? P<uint8_t>(ctx->st_buf[b][10]) : nullptr;
    }
    const size_t db = (size_t)n * 8, fb = (size_t)n * 4;
    const void *in[10];
    void *arr[10] = {x, y, z, vx, vy, vz, (void *)m, ax, ay, az};
    size_t sz[10] = {db, db, db, fb, fb, fb, fb, fb, fb, fb};
    // load_state reads each input once and the closing gather writes each
    // output once: page-locked host arrays are used in place
    bool direct[10];
    for (int k = 0; k < 10; k++)
        NB_CUDA(ctx, stage_once(ctx, k, arr[k], sz[k], &in[k], &direct[k]));
    float4 *acc = P<float4>(ctx->acc_s);
    ctx->kernels = 0;
    ctx->wev_used = 0;
    ctx->evused = 0;
    NB_CUDA(ctx, cudaMemsetAsync(ctx->ds, 0, sizeof(DevState), s));
    // the first step's opening kick and drift are applied by the state load
    // (shared steps; block steps start with their own kicks)
    bool loaded_kd = nsteps >= 1 && ctx->cfg.block_levels == 0;
    launch_load_state(s, n, (const double *)in[0], (const double *)in[1], (const double *)in[2],
                      (const float *)in[3], (const float *)in[4], (const float *)in[5],
                      (const float *)in[6], (const float *)in[7], (const float *)in[8],
                      (const float *)in[9], S[0], acc, loaded_kd, 0.5f * dt, dt,
                      loaded_kd ? ctx->recs.p : nullptr);
    // with the first kick-drift fused, the load also writes the records the
    // first step's sort gathers (its state exists only as records and x, y, z)
    bool loaded_recs = loaded_kd;
    ctx->kernels += 1;
    int cur = 0;
    std::vector<int> marks;  // per eager step: event indices (build start, build end, walk end)

    // One leapfrog step enqueued on ctx->stream.  With `timing`, phase
    // boundaries are recorded with pool events (eager steps only).  A step
    // either rebuilds the tree (keys, sort, state permutation, tree, groups)
    // or refits the current one (moments and group spheres at the drifted
    // positions, which the kick-drift writes to pos4 in place).
    int rebuilds = 0;
    // A step defers its closing half kick into the next step's kick-drift
    // pass (pending_kick): between eager steps, and between the two steps of
    // a graph; the graph's last step kicks on its own, so that every replay
    // starts from the same state.
    bool pending_kick = false, defer_in_capture = false;
    // near_order: the state is in the Morton order of this call's previous
    // build (every step but the call's first, whose state is in caller order)
    auto one_step = [&](bool timing, bool rebuild, bool near_order) -> nbody_status {
        cudaStream_t q = ctx->stream;
        if (loaded_kd) {  // done by the state load (the call's first step)
            loaded_kd = false;
        } else {
            launch_kick_drift(q, n, S[cur], acc, 0.5f * dt, dt,
                              rebuild ? nullptr : P<float4>(ctx->pos4), pending_kick ? 0.5f * dt : 0.0f);
            ctx->kernels += 1;
        }
        pending_kick = false;
        cudaEvent_t e0 = nullptr, e1 = nullptr, e2 = nullptr;
        if (timing) {
            NB_CUDA(ctx, pool_event(ctx, &e0));
            NB_CUDA(ctx, cudaEventRecord(e0, q));
        }
        nbody_status r;
        if (rebuild) {
            r = build_core(ctx, L, S[cur].x, S[cur].y, S[cur].z, true, S[cur].m, false, near_order,
                           near_order ? nullptr : first_sort_hint(ctx, L));
            if (r != NBODY_OK) return r;
            if (near_order) {
                launch_permute_state(q, n, P<uint32_t>(ctx->vals), S[cur], S[1 - cur],
                                     P<float4>(ctx->pos4));
            } else {  // the caller's order: a far-from-identity permutation
                launch_permute_state_recs(q, n, P<uint32_t>(ctx->vals), S[cur], S[1 - cur],
                                          P<float4>(ctx->pos4), ctx->recs.p, loaded_recs);
                ctx->kernels += loaded_recs ? 0 : 1;
            }
            loaded_recs = false;
            ctx->kernels += 1;
            cur = 1 - cur;
            r = build_tree_groups(ctx, L);
            rebuilds++;
        } else {
            r = refit_tree_groups(ctx, L);
        }
        if (r != NBODY_OK) return r;
        if (timing) {
            NB_CUDA(ctx, pool_event(ctx, &e1));
            NB_CUDA(ctx, cudaEventRecord(e1, q));
        }
        NB_CUDA(ctx, cudaMemcpyAsync(ctx->aold_s.p, S[cur].aold, fb, cudaMemcpyDeviceToDevice, q));
        r = run_walk(ctx, false, false, safe, nullptr, nullptr, nullptr, nullptr, nullptr, acc, false,
                     S[cur].pcost);
        if (r != NBODY_OK) return r;
        if (S[cur].pcost) {
            launch_spread_cost(q, &ctx->ds->ngroups, P<int32_t>(ctx->grp_first),
                               P<int32_t>(ctx->grp_count), P<int32_t>(ctx->grp_cost), S[cur].pcost,
                               ctx->nsm);
            ctx->kernels += 1;
        }
        if (timing) {
            NB_CUDA(ctx, pool_event(ctx, &e2));
            NB_CUDA(ctx, cudaEventRecord(e2, q));
            marks.push_back(ctx->evused - 3);
        }
        if ((ctx->capturing && !defer_in_capture) || dt == 0.0f) {
            launch_kick(q, n, S[cur], acc, 0.5f * dt);
            ctx->kernels += 1;
        } else {
            pending_kick = true;
        }
        return NBODY_OK;
    };

    int eager = nsteps;
    int graph_replays = 0;
    bool sorted_state = false;  // the state is in the Morton order of a build of this call
    // steps that may refit instead of rebuilding, and block steps, run eagerly
    if (ctx->cfg.use_graph && nsteps >= 3 && ctx->cfg.rebuild_interval == 1 &&
        ctx->cfg.block_levels == 0) {
        // The call's first step sorts the state from the caller's order: it
        // runs eagerly, and the graph's steps all find the state in the order
        // of the build before them.
        st = one_step(true, true, false);
        if (st != NBODY_OK) return st;
        if (pending_kick) {
            launch_kick(s, n, S[cur], acc, 0.5f * dt);
            ctx->kernels += 1;
            pending_kick = false;
        }
        sorted_state = true;
        // Two steps per graph: the sort's ping-pong buffers and the state
        // copies swap roles every step, so after two steps every pointer is
        // back where the capture found it and the graph can be replayed.
        GraphKey key;
        std::memset(&key, 0, sizeof key);  // padding too: keys are compared bytewise
        key.n = n;
        key.nsys = nsys;
        key.dt = dt;
        key.safe = safe;
        key.mlp_norm = ctx->mlp_norm_set;
        key.cfg = ctx->cfg;
        key.bufs[0] = ctx->keys.p;
        key.bufs[1] = ctx->vals.p;
        key.bufs[2] = S[0].x;
        key.bufs[3] = ctx->nodeA.p;
        key.bufs[4] = ctx->grp_first.p;
        key.bufs[5] = ctx->rs_temp.p;
        key.bufs[6] = ctx->pos4.p;
        key.bufs[7] = ctx->acc_s.p;
        if (!ctx->gstream)
            NB_CUDA(ctx, cudaStreamCreateWithFlags(&ctx->gstream, cudaStreamNonBlocking));
        if (!ctx->gexec || std::memcmp(&key, &ctx->gkey, sizeof key) != 0) {
            if (ctx->gexec) {
                cudaGraphExecDestroy(ctx->gexec);
                ctx->gexec = nullptr;
            }
            for (auto &ev : ctx->gwev)
                if (!ev) NB_CUDA(ctx, cudaEventCreate(&ev));
            ctx->gwev_used = 0;
            cudaStream_t saved = ctx->stream;
            ctx->stream = ctx->gstream;
            ctx->capturing = true;
            int64_t k0 = ctx->kernels;
            cudaGraph_t graph = nullptr;
            cudaError_t ce = cudaStreamBeginCapture(ctx->gstream, cudaStreamCaptureModeRelaxed);
            nbody_status r1 = NBODY_OK, r2 = NBODY_OK;
            if (ce == cudaSuccess) {
                defer_in_capture = true;
                r1 = one_step(false, true, true);
                defer_in_capture = false;
                if (r1 == NBODY_OK) r2 = one_step(false, true, true);
                cudaError_t ee = cudaStreamEndCapture(ctx->gstream, &graph);
                if (ce == cudaSuccess) ce = ee;
            }
            ctx->stream = saved;
            ctx->capturing = false;
            if (r1 != NBODY_OK) return r1;
            if (r2 != NBODY_OK) return r2;
            if (ce == cudaSuccess) ce = cudaGraphInstantiate(&ctx->gexec, graph, 0);
            if (graph) cudaGraphDestroy(graph);
            if (ce != cudaSuccess) return cuda_fail(ctx, ce, "step graph capture");
            ctx->gkernels = ctx->kernels - k0;
            ctx->gwev_pairs = ctx->gwev_used / 2;
            ctx->kernels = k0;
            ctx->gkey = key;
        }
        NB_CUDA(ctx, cudaEventRecord(ctx->ev[0], s));
        NB_CUDA(ctx, cudaStreamWaitEvent(ctx->gstream, ctx->ev[0], 0));
        for (int it = 1; it + 1 < nsteps; it += 2) {
            NB_CUDA(ctx, cudaGraphLaunch(ctx->gexec, ctx->gstream));
            ctx->kernels += ctx->gkernels;
            rebuilds += 2;
            graph_replays++;
        }
        NB_CUDA(ctx, cudaEventRecord(ctx->ev[1], ctx->gstream));
        NB_CUDA(ctx, cudaStreamWaitEvent(s, ctx->ev[1], 0));
        eager = (nsteps - 1) % 2;
    }
    if (ctx->cfg.block_levels > 0) {
        st = block_steps(ctx, L, S, cur, acc, dt, nsteps, safe, rebuilds, marks);
        if (st != NBODY_OK) return st;
        eager = 0;
    }
    // Rebuild schedule of the eager steps: every rebuild_interval-th step, or
    // (interval 0) when nbody_rebuild_due says the last step raised the mean
    // cost of the current cycle -- measured per step, so the stream is
    // synchronised after each step -- and at most every kAutoMaxInterval.
    constexpr int kAutoMaxInterval = 32;
    const int interval = ctx->cfg.rebuild_interval;
    std::vector<float> cycle;
    int since = 0;
    for (int it = 0; it < eager; it++) {
        bool rebuild = (it == 0 && eager == nsteps) || interval == 1;
        if (!rebuild && interval > 1) rebuild = since >= interval;
        if (!rebuild && interval == 0)
            rebuild = since >= kAutoMaxInterval ||
                      nbody_rebuild_due(cycle.data(), (int32_t)cycle.size()) != 0;
        if (rebuild) {
            since = 0;
            cycle.clear();
        }
        st = one_step(true, rebuild, sorted_state);
        if (st != NBODY_OK) return st;
        if (rebuild) sorted_state = true;
        since++;
        if (interval == 0) {
            const int k = marks.back();
            float c = 0.0f;
            NB_CUDA(ctx, cudaEventSynchronize(ctx->evpool[k + 2]));
            NB_CUDA(ctx, cudaEventElapsedTime(&c, ctx->evpool[k], ctx->evpool[k + 2]));
            cycle.push_back(c);
        }
    }
    // the last eager step's closing half kick is applied on the way out
    const float hclose = pending_kick ? 0.5f * dt : 0.0f;
    pending_kick = false;
    // the Morton order this call ends in starts the next call's first sort
    // (a call without steps ends in the caller's order: nothing to keep)
    if (nsteps > 0) {
        NB_CUDA(ctx, ensure(ctx->last_ids, (size_t)n * 4));
        NB_CUDA(ctx, cudaMemcpyAsync(ctx->last_ids.p, S[cur].id, (size_t)n * 4,
                                     cudaMemcpyDeviceToDevice, s));
        ctx->hint_n = n;
        ctx->hint_nsys = nsys;
    }
    // in[] are the device copies (the caller's arrays themselves when on the device)
    launch_store_state(s, n, S[cur], acc, (double *)in[0], (double *)in[1], (double *)in[2],
                       (float *)in[3], (float *)in[4], (float *)in[5], (float *)in[7],
                       (float *)in[8], (float *)in[9], ctx->recs.p, hclose);
    ctx->kernels += 2;
    for (int k = 0; k < 10; k++) {
        if (k == 6 || direct[k]) continue;
        NB_CUDA(ctx, cudaMemcpyAsync(arr[k], in[k], sz[k], cudaMemcpyDeviceToHost, s));
    }
    st = read_status(ctx);
    float ms_build = 0.0f, ms_walk = 0.0f;
    for (int k : marks) {
        float a = 0, b = 0;
        if (cudaEventElapsedTime(&a, ctx->evpool[k], ctx->evpool[k + 1]) != cudaSuccess ||
            cudaEventElapsedTime(&b, ctx->evpool[k + 1], ctx->evpool[k + 2]) != cudaSuccess) {
            cudaGetLastError();
            a = b = 0.0f;
        }
        ms_build += a;
        ms_walk += b;
    }
    ctx->L = L;
    ctx->last.n_nodes = ctx->h_ds->nnodes;
    ctx->last.n_groups = ctx->h_ds->ngroups;
    ctx->last.levels = L.levels;
    ctx->last.interactions = (int64_t)ctx->h_ds->interactions;
    ctx->last.list_entries = (int64_t)ctx->h_ds->list_entries;
    ctx->last.quad_interactions = (int64_t)ctx->h_ds->quad_entries;
    ctx->last.walk_warps = ctx->walk_warps;
    ctx->last.max_stack = ctx->h_ds->max_stack;
    ctx->last.ms_build = ms_build;
    ctx->last.ms_walk = ms_walk;
    ctx->last.ms_walk_kernel = collect_walk_ms(ctx, &ctx->last.walk_launches);
    if (graph_replays > 0) {  // the walks of the last graph replay (its event nodes)
        for (int k = 0; k < ctx->gwev_pairs; k++) {
            float ms = 0.0f;
            if (cudaEventElapsedTime(&ms, ctx->gwev[2 * k], ctx->gwev[2 * k + 1]) == cudaSuccess) {
                ctx->last.ms_walk_kernel += ms;
                ctx->last.walk_launches += 1;
            } else {
                cudaGetLastError();
            }
        }
    }
    ctx->last.kernels = ctx->kernels;
    ctx->last.rebuilds = rebuilds;
    if (stats) *stats = ctx->last;
    // the sorted state no longer matches a caller-order build
    ctx->built = false;
    return st;
}

nbody_status nbody_step(nbody_ctx *ctx, int64_t n, double *x, double *y, double *z, float *vx,
                        float *vy, float *vz, const float *m, float *ax, float *ay, float *az,
                        float dt, int32_t nsteps, nbody_stats *stats) {
    if (!ctx) return fail(nullptr, NBODY_EINVAL, "ctx is NULL");
    if (n < 1 || n >= ((int64_t)1 << 31)) return fail(ctx, NBODY_EINVAL, "n must be in 1..2^31-1");
    return step_impl(ctx, 1, nullptr, nullptr, n, x, y, z, vx, vy, vz, m, ax, ay, az, dt, nsteps,
                     stats);
}

nbody_status nbody_step_batched(nbody_ctx *ctx, int32_t nsys, const int64_t *offsets,
                                const float *eps_sys, double *x, double *y, double *z,
                                float *vx, float *vy, float *vz, const float *m, float *ax,
                                float *ay, float *az, float dt, int32_t nsteps,
                                nbody_stats *stats) {
    if (!ctx) return fail(nullptr, NBODY_EINVAL, "ctx is NULL");
    nbody_status st = check_systems(ctx, nsys, offsets, eps_sys);
    if (st != NBODY_OK) return st;
    return step_impl(ctx, nsys, offsets, eps_sys, offsets[nsys], x, y, z, vx, vy, vz, m, ax, ay,
                     az, dt, nsteps, stats);
}

nbody_status nbody_diagnostics(nbody_ctx *ctx, int64_t n, const double *x, const double *y,
                               const double *z, const float *vx, const float *vy,
                               const float *vz, const float *m, const float *phi, double *out) {
    if (!ctx) return fail(nullptr, NBODY_EINVAL, "ctx is NULL");
    if (n < 1 || n >= ((int64_t)1 << 31)) return fail(ctx, NBODY_EINVAL, "n must be in 1..2^31-1");
    if (!x || !y || !z || !vx || !vy || !vz || !m || !out) return fail(ctx, NBODY_EINVAL, "NULL array");
    const size_t db = (size_t)n * 8, fb = (size_t)n * 4;
    const void *in[8];
    const void *arr[8] = {x, y, z, vx, vy, vz, m, phi};
    size_t sz[8] = {db, db, db, fb, fb, fb, fb, fb};
    for (int k = 0; k < 8; k++) NB_CUDA(ctx, stage_in(ctx, k, arr[k], sz[k], &in[k]));
    cudaError_t e = ensure(ctx->diag_temp, diag_temp_bytes());
    if (e == cudaSuccess) e = ensure(ctx->diag_out, 8 * sizeof(double));
    if (e != cudaSuccess) return fail(ctx, NBODY_ENOMEM, "allocation");
    launch_diagnostics(ctx->stream, n, (const double *)in[0], (const double *)in[1],
                       (const double *)in[2], (const float *)in[3], (const float *)in[4],
                       (const float *)in[5], (const float *)in[6], (const float *)in[7],
                       ctx->diag_temp.p, P<double>(ctx->diag_out));
    NB_CUDA(ctx, cudaGetLastError());
    NB_CUDA(ctx, cudaMemcpyAsync(ctx->h_diag, ctx->diag_out.p, 8 * sizeof(double),
                                 cudaMemcpyDeviceToHost, ctx->stream));
    NB_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    std::memcpy(out, ctx->h_diag, 8 * sizeof(double));
    return NBODY_OK;
}

nbody_status nbody_get_group_costs(nbody_ctx *ctx, int32_t *counts, int64_t cap,
                                   int64_t *n_groups) {
    if (!ctx) return fail(nullptr, NBODY_EINVAL, "ctx is NULL");
    if (!counts || cap < 0 || !n_groups) return fail(ctx, NBODY_EINVAL, "bad argument");
    if (!ctx->grp_cost.p) return fail(ctx, NBODY_ENOTBUILT, "no walk yet");
    NB_CUDA(ctx, cudaMemcpyAsync(ctx->h_ds, ctx->ds, sizeof(DevState), cudaMemcpyDeviceToHost, ctx->stream));
    NB_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    int64_t ng = ctx->h_ds->ngroups;
    *n_groups = ng;
    int64_t k = std::min(ng, cap);
    if (k > 0) {
        cudaMemcpyKind kind = is_device_ptr(counts) ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
        NB_CUDA(ctx, cudaMemcpyAsync(counts, ctx->grp_cost.p, (size_t)k * 4, kind, ctx->stream));
        NB_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    }
    return NBODY_OK;
}

void nbody_tune_space_default(nbody_tune_space *sp) {
    if (!sp) return;
    std::memset(sp, 0, sizeof *sp);
    sp->n_leaf_cap = 2;
    sp->leaf_cap[0] = 8;
    sp->leaf_cap[1] = 16;
    sp->n_group_size = 3;
    sp->group_size[0] = 32;
    sp->group_size[1] = 64;
    sp->group_size[2] = 128;
    sp->n_ipl = 3;
    sp->ipl[0] = 2;
    sp->ipl[1] = 3;
    sp->ipl[2] = 4;
    sp->n_list_depth = 2;
    sp->list_depth[0] = 128;
    sp->list_depth[1] = 256;
    sp->n_warps_per_block = 3;
    sp->warps_per_block[0] = 2;
    sp->warps_per_block[1] = 4;
    sp->warps_per_block[2] = 8;
    sp->repeats = 2;
}

nbody_status nbody_autotune(nbody_ctx *ctx, int32_t nsys, const int64_t *offsets,
                            const float *eps_sys, const float *x, const float *y,
                            const float *z, const float *m, const float *a_old,
                            const nbody_tune_space *space, nbody_config *best, float *best_ms,
                            int32_t *n_tried) {
    if (!ctx) return fail(nullptr, NBODY_EINVAL, "ctx is NULL");
    nbody_tune_space sp;
    if (space) sp = *space; else nbody_tune_space_default(&sp);
    if (sp.n_leaf_cap < 1 || sp.n_leaf_cap > 4 || sp.n_group_size < 1 || sp.n_group_size > 6 ||
        sp.n_ipl < 1 || sp.n_ipl > 3 || sp.n_list_depth < 1 || sp.n_list_depth > 4 ||
        sp.n_warps_per_block < 1 || sp.n_warps_per_block > 4 || sp.repeats < 1)
        return fail(ctx, NBODY_EINVAL, "bad tune space");
    if (nsys < 1) return fail(ctx, NBODY_EINVAL, "nsys must be >= 1");
    int64_t n = 0;
    if (nsys == 1 && !offsets) {
        return fail(ctx, NBODY_EINVAL, "offsets is NULL (pass {0, n} for one system)");
    }
    nbody_status st = check_systems(ctx, nsys, offsets, eps_sys);
    if (st != NBODY_OK) return st;
    n = offsets[nsys];
    const nbody_config base = ctx->cfg;
    nbody_config bestc = base;
    float bestt = INFINITY;
    int tried = 0;
    // outputs of the timed walks (device scratch owned by the context)
    cudaError_t e = ensure(ctx->stage[9], (size_t)n * 4);
    if (e == cudaSuccess) e = ensure(ctx->stage[10], (size_t)n * 4);
    if (e == cudaSuccess) e = ensure(ctx->stage[11], (size_t)n * 4);
    if (e != cudaSuccess) return fail(ctx, NBODY_ENOMEM, "allocation");
    float *o0 = P<float>(ctx->stage[9]), *o1 = P<float>(ctx->stage[10]), *o2 = P<float>(ctx->stage[11]);
    for (int il = 0; il < sp.n_leaf_cap; il++)
        for (int ig = 0; ig < sp.n_group_size; ig++)
            for (int ii = 0; ii < sp.n_ipl; ii++) {
                nbody_config c = base;
                c.leaf_cap = sp.leaf_cap[il];
                c.group_size = sp.group_size[ig];
                c.ipl = sp.ipl[ii];
                if (c.group_size <= 8 * c.ipl) continue;  // slots beyond any useful tile
                std::string why;
                c.list_depth = sp.list_depth[0];
                c.warps_per_block = sp.warps_per_block[0];
                if (!config_ok(&c, why)) continue;
                ctx->cfg = c;
                st = nbody_build_batched(ctx, nsys, offsets, eps_sys, x, y, z, m);
                if (st != NBODY_OK) { ctx->cfg = base; return st; }
                const float tb = ctx->last.ms_build;
                for (int id = 0; id < sp.n_list_depth; id++)
                    for (int iw = 0; iw < sp.n_warps_per_block; iw++) {
                        nbody_config cw = c;
                        cw.list_depth = sp.list_depth[id];
                        cw.warps_per_block = sp.warps_per_block[iw];
                        if (!config_ok(&cw, why)) continue;
                        ctx->cfg = cw;  // walk-only parameters: the build stays valid
                        float tw = INFINITY;
                        for (int r = 0; r < sp.repeats; r++) {
                            nbody_stats s2;
                            st = nbody_walk(ctx, a_old, o0, o1, o2, nullptr, &s2);
                            if (st == NBODY_EOVERFLOW) break;  // too shallow a stack: skip
                            if (st != NBODY_OK) { ctx->cfg = base; return st; }
                            tw = std::min(tw, s2.ms_walk_kernel);
                        }
                        if (st == NBODY_EOVERFLOW) continue;
                        tried++;
                        if (tb + tw < bestt) {
                            bestt = tb + tw;
                            bestc = cw;
                        }
                    }
            }
    if (!tried) {
        ctx->cfg = base;
        return fail(ctx, NBODY_EINVAL, "no valid candidate in the tune space");
    }
    ctx->cfg = bestc;
    ctx->built = false;  // the last build used another candidate
    if (best) *best = bestc;
    if (best_ms) *best_ms = bestt;
    if (n_tried) *n_tried = tried;
    return NBODY_OK;
}

nbody_status nbody_export(nbody_ctx *ctx, int32_t what, void *dst, int64_t cap, int64_t *count) {
    if (!ctx) return fail(nullptr, NBODY_EINVAL, "ctx is NULL");
    if (!count || cap < 0 || (cap > 0 && !dst)) return fail(ctx, NBODY_EINVAL, "bad argument");
    if (!ctx->built) return fail(ctx, NBODY_ENOTBUILT, "no build to export");
    NB_CUDA(ctx, cudaMemcpyAsync(ctx->h_ds, ctx->ds, sizeof(DevState), cudaMemcpyDeviceToHost, ctx->stream));
    NB_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    const int64_t n = ctx->L.n, nn = ctx->h_ds->nnodes, ng = ctx->h_ds->ngroups;
    const void *src = nullptr;
    int64_t len = 0;
    size_t esz = 4;
    switch (what) {
        case NBODY_EXPORT_PERM: src = ctx->vals.p; len = n; break;
        case NBODY_EXPORT_KEYS: src = ctx->keys.p; len = n; esz = 8; break;
        case NBODY_EXPORT_NODE_LEVEL: src = ctx->node_level.p; len = nn; esz = 1; break;
        case NBODY_EXPORT_NODE_START: src = ctx->node_start.p; len = nn; break;
        case NBODY_EXPORT_NODE_COUNT: src = ctx->node_count.p; len = nn; break;
        case NBODY_EXPORT_NODE_PARENT: src = ctx->node_parent.p; len = nn; break;
        case NBODY_EXPORT_NODE_A: src = ctx->nodeA.p; len = nn; esz = 16; break;
        case NBODY_EXPORT_NODE_B: src = ctx->nodeB.p; len = nn; esz = 16; break;
        case NBODY_EXPORT_GROUP_FIRST: src = ctx->grp_first.p; len = ng; break;
        case NBODY_EXPORT_GROUP_COUNT: src = ctx->grp_count.p; len = ng; break;
        case NBODY_EXPORT_GROUP_SPHERE: src = ctx->grp_sphere.p; len = ng; esz = 16; break;
        case NBODY_EXPORT_NODE_Q:
            if (!ctx->cfg.quadrupole) return fail(ctx, NBODY_EINVAL, "quadrupoles are off");
            src = ctx->nodeQ.p; len = nn; esz = 32; break;
        case NBODY_EXPORT_SYS_BOX: {
            // SysBox is 32 bytes; export the first 16 (x0, y0, z0, L) of each
            *count = ctx->L.nsys;
            int64_t k = std::min<int64_t>(cap, ctx->L.nsys);
            if (k > 0) {
                cudaMemcpyKind kind = is_device_ptr(dst) ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
                NB_CUDA(ctx, cudaMemcpy2DAsync(dst, 16, ctx->sys_box.p, sizeof(SysBox), 16, (size_t)k,
                                               kind, ctx->stream));
                NB_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
            }
            return NBODY_OK;
        }
        default: return fail(ctx, NBODY_EINVAL, "unknown export");
    }
    *count = len;
    int64_t k = std::min(cap, len);
    if (k > 0) {
        cudaMemcpyKind kind = is_device_ptr(dst) ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
        NB_CUDA(ctx, cudaMemcpyAsync(dst, src, (size_t)k * esz, kind, ctx->stream));
        NB_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    }
    return NBODY_OK;
}

// ---------------------------------------------------------------- learned cost model
static_assert(NBODY_MLP_PARAMS == nb::kMlpParams, "parameter count");

static cudaError_t ensure_mlp_state(nbody_ctx *c) {
    cudaError_t e = ensure(c->mlp_w, kMlpParams * 4);
    if (e == cudaSuccess) e = ensure(c->mlp_m1, kMlpParams * 4);
    if (e == cudaSuccess) e = ensure(c->mlp_m2, kMlpParams * 4);
    if (e == cudaSuccess) e = ensure(c->mlp_wb, kMlpParams * 2);
    if (e == cudaSuccess) e = ensure(c->mlp_norm, 32 * 4);
    return e;
}

nbody_status nbody_mlp_set_params(nbody_ctx *ctx, const float *params) {
    if (!ctx || !params) return fail(ctx, NBODY_EINVAL, "NULL argument");
    cudaError_t e = ensure_mlp_state(ctx);
    if (e != cudaSuccess) return fail(ctx, NBODY_ENOMEM, "allocation");
    cudaMemcpyKind kind = is_device_ptr(params) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    NB_CUDA(ctx, cudaMemcpyAsync(ctx->mlp_w.p, params, kMlpParams * 4, kind, ctx->stream));
    NB_CUDA(ctx, cudaMemsetAsync(ctx->mlp_m1.p, 0, kMlpParams * 4, ctx->stream));
    NB_CUDA(ctx, cudaMemsetAsync(ctx->mlp_m2.p, 0, kMlpParams * 4, ctx->stream));
    launch_mlp_round(ctx->stream, P<float>(ctx->mlp_w), reinterpret_cast<__nv_bfloat16 *>(ctx->mlp_wb.p));
    NB_CUDA(ctx, cudaGetLastError());
    NB_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    ctx->mlp_t = 0;
    ctx->mlp_ready = true;
    ctx->mlp_norm_set = false;
    return NBODY_OK;
}

nbody_status nbody_mlp_get_params(nbody_ctx *ctx, float *params) {
    if (!ctx || !params) return fail(ctx, NBODY_EINVAL, "NULL argument");
    if (!ctx->mlp_ready) return fail(ctx, NBODY_EINVAL, "no MLP parameters set");
    cudaMemcpyKind kind = is_device_ptr(params) ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    NB_CUDA(ctx, cudaMemcpyAsync(params, ctx->mlp_w.p, kMlpParams * 4, kind, ctx->stream));
    NB_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    return NBODY_OK;
}

nbody_status nbody_mlp_train(nbody_ctx *ctx, int32_t epochs, float lr, int32_t batch, float *loss) {
    if (!ctx) return fail(nullptr, NBODY_EINVAL, "ctx is NULL");
    if (!ctx->mlp_ready) return fail(ctx, NBODY_EINVAL, "no MLP parameters set");
    if (!ctx->costs_valid) return fail(ctx, NBODY_EINVAL, "no walk since the last build");
    if (epochs < 1 || batch < 32 || batch > (1 << 16) || !(lr > 0.0f))
        return fail(ctx, NBODY_EINVAL, "epochs >= 1, 32 <= batch <= 65536, lr > 0");
    int64_t ng = 0;
    nbody_status st = host_ngroups(ctx, &ng);
    if (st != NBODY_OK) return st;
    if (ng < 1) return fail(ctx, NBODY_EINVAL, "no groups");
    cudaStream_t s = ctx->stream;
    const int64_t nbatches = (ng + batch - 1) / batch;
    const int maxb = (int)((ng / nbatches + 1 + 127) / 128) + 1;
    cudaError_t e = ensure_mlp_buffers(ctx);
    if (e == cudaSuccess) e = ensure(ctx->mlp_gpart, (size_t)maxb * kMlpParams * 4);
    if (e == cudaSuccess) e = ensure(ctx->mlp_lpart, (size_t)maxb * 4);
    if (e == cudaSuccess) e = ensure(ctx->mlp_loss, (size_t)nbatches * 4);
    if (e != cudaSuccess) return fail(ctx, NBODY_ENOMEM, "allocation");
    const int32_t *png = &ctx->ds->ngroups;
    ctx->kernels = 0;
    launch_features(ctx);
    if (!ctx->mlp_norm_set) {  // freeze feature and target statistics
        launch_mlp_target(s, png, P<int32_t>(ctx->grp_cost), nullptr, P<float>(ctx->target), ctx->nsm);
        launch_mlp_norm(s, png, P<float>(ctx->feat), P<float>(ctx->target), P<float>(ctx->mlp_norm));
        ctx->mlp_norm_set = true;
    }
    launch_mlp_target(s, png, P<int32_t>(ctx->grp_cost), P<float>(ctx->mlp_norm) + 16,
                      P<float>(ctx->target), ctx->nsm);
    __nv_bfloat16 *wb = reinterpret_cast<__nv_bfloat16 *>(ctx->mlp_wb.p);
    for (int ep = 0; ep < epochs; ep++)
        for (int64_t k = 0; k < nbatches; k++) {
            const int count = (int)((ng - 1 - k) / nbatches + 1);
            ctx->mlp_t += 1;
            e = launch_mlp_train_step(s, P<float>(ctx->feat), P<float>(ctx->target), k, nbatches,
                                      count, wb, P<float>(ctx->mlp_norm), P<float>(ctx->mlp_gpart),
                                      P<float>(ctx->mlp_lpart), nullptr,
                                      P<float>(ctx->mlp_loss) + k, P<float>(ctx->mlp_w),
                                      P<float>(ctx->mlp_m1), P<float>(ctx->mlp_m2), wb, lr,
                                      ctx->mlp_t, true);
            if (e != cudaSuccess) return cuda_fail(ctx, e, "mlp train step");
        }
    std::vector<float> h((size_t)nbatches);
    NB_CUDA(ctx, cudaMemcpyAsync(h.data(), ctx->mlp_loss.p, (size_t)nbatches * 4,
                                 cudaMemcpyDeviceToHost, s));
    NB_CUDA(ctx, cudaStreamSynchronize(s));
    double m = 0;
    for (float v : h) m += v;
    if (loss) *loss = (float)(m / (double)nbatches);
    return NBODY_OK;
}

nbody_status nbody_mlp_predict(nbody_ctx *ctx, float *pred, float *features, int64_t cap,
                               int64_t *n_groups) {
    if (!ctx || !n_groups || cap < 0) return fail(ctx, NBODY_EINVAL, "bad argument");
    if (!ctx->mlp_ready) return fail(ctx, NBODY_EINVAL, "no MLP parameters set");
    int64_t ng = 0;
    nbody_status st = host_ngroups(ctx, &ng);
    if (st != NBODY_OK) return st;
    *n_groups = ng;
    if (ensure_mlp_buffers(ctx) != cudaSuccess) return fail(ctx, NBODY_ENOMEM, "allocation");
    launch_features(ctx);
    const float *nrm = ctx->mlp_norm_set ? P<float>(ctx->mlp_norm) : nullptr;
    launch_mlp_forward(ctx->stream, &ctx->ds->ngroups, 0, P<float>(ctx->feat),
                       reinterpret_cast<const __nv_bfloat16 *>(ctx->mlp_wb.p), nrm,
                       nrm ? nrm + 16 : nullptr, P<float>(ctx->score), ctx->nsm);
    NB_CUDA(ctx, cudaGetLastError());
    const int64_t k = std::min(cap, ng);
    if (k > 0 && pred) {
        cudaMemcpyKind kind = is_device_ptr(pred) ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
        NB_CUDA(ctx, cudaMemcpyAsync(pred, ctx->score.p, (size_t)k * 4, kind, ctx->stream));
    }
    if (k > 0 && features) {
        cudaMemcpyKind kind = is_device_ptr(features) ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
        NB_CUDA(ctx, cudaMemcpyAsync(features, ctx->feat.p, (size_t)k * 8 * 4, kind, ctx->stream));
    }
    NB_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    return NBODY_OK;
}

nbody_status nbody_mlp_eval(int64_t n, const float *features, const float *targets,
                            const float *params, const float *norm, float *pred, float *grad,
                            float *loss, void *cuda_stream) {
    if (n < 1 || n > (1 << 20) || !features || !targets || !params)
        return fail(nullptr, NBODY_EINVAL, "bad argument (1 <= n <= 2^20, non-NULL inputs)");
    cudaStream_t s = (cudaStream_t)cuda_stream;
    const int nb = (int)((n + 127) / 128);
    // one device block: features, targets, params, norm, pred, grad, partials, loss, bf16 params
    const size_t fsz = (size_t)n * 8 * 4, tsz = (size_t)n * 4, psz = kMlpParams * 4;
    const size_t total = fsz + tsz + psz + 64 + tsz + psz + (size_t)nb * psz + (size_t)nb * 4 + 16 +
                         kMlpParams * 2 + 1024;
    char *buf = nullptr;
    cudaError_t e = cudaMalloc(&buf, total);
    if (e != cudaSuccess) return fail(nullptr, NBODY_ENOMEM, "allocation");
    auto align = [](size_t v) { return (v + 255) & ~(size_t)255; };
    size_t o = 0;
    float *dfeat = (float *)(buf + o); o = align(o + fsz);
    float *dtarget = (float *)(buf + o); o = align(o + tsz);
    float *dparams = (float *)(buf + o); o = align(o + psz);
    float *dnorm = (float *)(buf + o); o = align(o + 64);
    float *dpred = (float *)(buf + o); o = align(o + tsz);
    float *dgrad = (float *)(buf + o); o = align(o + psz);
    float *dgpart = (float *)(buf + o); o = align(o + (size_t)nb * psz);
    float *dlpart = (float *)(buf + o); o = align(o + (size_t)nb * 4);
    float *dloss = (float *)(buf + o); o = align(o + 16);
    __nv_bfloat16 *dwb = (__nv_bfloat16 *)(buf + o);
    auto h2d = [&](void *dst, const void *src, size_t b) {
        return cudaMemcpyAsync(dst, src, b, is_device_ptr(src) ? cudaMemcpyDeviceToDevice
                                                               : cudaMemcpyHostToDevice, s);
    };
    e = h2d(dfeat, features, fsz);
    if (e == cudaSuccess) e = h2d(dtarget, targets, tsz);
    if (e == cudaSuccess) e = h2d(dparams, params, psz);
    if (e == cudaSuccess && norm) e = h2d(dnorm, norm, 64);
    if (e == cudaSuccess) {
        launch_mlp_round(s, dparams, dwb);
        launch_mlp_forward(s, nullptr, n, dfeat, dwb, norm ? dnorm : nullptr, nullptr, dpred, 152);
        e = launch_mlp_train_step(s, dfeat, dtarget, 0, 1, (int)n, dwb, norm ? dnorm : nullptr,
                                  dgpart, dlpart, dgrad, dloss, nullptr, nullptr, nullptr, nullptr,
                                  0.0f, 1, false);
    }
    auto d2h = [&](void *dst, const void *src, size_t b) {
        return cudaMemcpyAsync(dst, src, b, is_device_ptr(dst) ? cudaMemcpyDeviceToDevice
                                                               : cudaMemcpyDeviceToHost, s);
    };
    if (e == cudaSuccess && pred) e = d2h(pred, dpred, tsz);
    if (e == cudaSuccess && grad) e = d2h(grad, dgrad, psz);
    if (e == cudaSuccess && loss) e = d2h(loss, dloss, 4);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    cudaFree(buf);
    if (e != cudaSuccess) return cuda_fail(nullptr, e, "nbody_mlp_eval");
    return NBODY_OK;
}

nbody_status nbody_sort_keys(nbody_ctx *ctx, int32_t method, const uint64_t *keys, int64_t n,
                             uint64_t *keys_out, int32_t *perm_out) {
    if (!ctx) return fail(nullptr, NBODY_EINVAL, "ctx is NULL");
    if (n < 1 || n >= ((int64_t)1 << 31)) return fail(ctx, NBODY_EINVAL, "n must be in 1..2^31-1");
    if (method != NBODY_SORT_RADIX && method != NBODY_SORT_NEAR_ORDER)
        return fail(ctx, NBODY_EINVAL, "unknown sort method");
    int dev = 0;
    NB_CUDA(ctx, cudaGetDevice(&dev));
    if (!on_device(keys, dev) || !on_device(keys_out, dev) || !on_device(perm_out, dev))
        return fail(ctx, NBODY_EINVAL, "keys, keys_out and perm_out must be memory of the "
                                       "context's device");
    cudaError_t e = ensure_capacity(ctx, n, 1, make_layout(n, 1).levels);
    if (e != cudaSuccess) return fail(ctx, NBODY_ENOMEM, std::string("allocation: ") + cudaGetErrorString(e));
    ctx->built = false;
    cudaStream_t s = ctx->stream;
    NB_CUDA(ctx, cudaMemsetAsync(ctx->ds, 0, sizeof(DevState), s));
    NB_CUDA(ctx, cudaMemcpyAsync(ctx->keys.p, keys, (size_t)n * 8, cudaMemcpyDeviceToDevice, s));
    bool alt = true;
    if (method == NBODY_SORT_NEAR_ORDER && nosort_fits(n))
        nosort(s, P<uint64_t>(ctx->keys), P<uint64_t>(ctx->keys_alt), P<uint32_t>(ctx->vals),
               P<uint32_t>(ctx->vals_alt), n, ctx->rs_temp.p, &ctx->ds->status);
    else
        alt = radix_sort(s, P<uint64_t>(ctx->keys), P<uint32_t>(ctx->vals),
                         P<uint64_t>(ctx->keys_alt), P<uint32_t>(ctx->vals_alt), n, 64,
                         ctx->rs_temp.p, false, &ctx->ds->status, ctx->nsm) != 0;
    NB_CUDA(ctx, cudaGetLastError());
    NB_CUDA(ctx, cudaMemcpyAsync(keys_out, alt ? ctx->keys_alt.p : ctx->keys.p, (size_t)n * 8,
                                 cudaMemcpyDeviceToDevice, s));
    NB_CUDA(ctx, cudaMemcpyAsync(perm_out, alt ? ctx->vals_alt.p : ctx->vals.p, (size_t)n * 4,
                                 cudaMemcpyDeviceToDevice, s));
    return read_status(ctx);
}

nbody_status nbody_selftest(int32_t which, void *cuda_stream) {
    if (which != NBODY_SELFTEST_SORT_WAIT) return fail(nullptr, NBODY_EINVAL, "unknown self-test");
    cudaStream_t s = (cudaStream_t)cuda_stream;
    int32_t *dstat = nullptr;
    cudaError_t e = cudaMalloc(&dstat, sizeof(int32_t));
    if (e != cudaSuccess) return cuda_fail(nullptr, e, "nbody_selftest");
    int32_t h = 0;
    e = cudaMemsetAsync(dstat, 0, sizeof(int32_t), s);
    if (e == cudaSuccess) e = radix_selftest_wait(s, dstat);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&h, dstat, sizeof h, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    cudaFree(dstat);
    if (e != cudaSuccess) return cuda_fail(nullptr, e, "nbody_selftest");
    if (h & kStatusTimeout) {
        set_stateless_error("self-test: the radix-sort look-back wait ran out as intended");
        return NBODY_ETIMEOUT;
    }
    return NBODY_OK;
}

nbody_status nbody_last_error(const nbody_ctx *ctx, char *buf, size_t len) {
    if (!buf || len == 0) return NBODY_EINVAL;
    const std::string &m = ctx ? ctx->err : g_last_error;
    size_t k = std::min(len - 1, m.size());
    std::memcpy(buf, m.data(), k);
    buf[k] = '\0';
    return NBODY_OK;
}

}  // extern "C"
