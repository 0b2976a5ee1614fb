#!/usr/bin/env python3
"""Benchmark of the gravitational octree step on a GB300.

Workload (default): the three-component galaxy with N = 2^23 equal-mass
particles (Hernquist bulge 15 %, exponential disk 10 %, NFW halo 75 %),
eps = 1/64, delta_acc = 2^-9, leapfrog dt = 1/256, the tree rebuilt every
step.  One step = kick-drift, bounding cube, Morton keys, radix sort, octree,
monopoles, groups, tree walk (Eq. 1 under the MAC of Eq. 2), kick.

Prints ONE JSON line (rank 0).  `value` is whole-job Ginteractions/s
(interactions = Eq. 1 kernel evaluations in the walk, 22 flops each);
`s_per_step` and the FP32 fraction of peak sit beside it.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

--impl reference times the FP64 CPU oracle (the deliberately plain
reference implementation) on the host cores, on a bounded sample.
Multi-GPU (torchrun): every rank runs its own replica of the workload; the
single large system does not shard (replicas only), so there is no
collective on the data path.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

METRIC = "s/step & Ginteractions/s at N=2^23, % GB300 FP32 peak, at stated force error"
UNIT = "Ginteractions/s"
FLOPS_PER_INTERACTION = 22  # 3 sub, 3 FMA (r^2+eps^2), rsqrt = 4, 3 mul, 3 FMA
EPS, DACC, DT = 1.0 / 64, 2.0 ** -9, 1.0 / 256
PHASE_STEPS = 8  # eager steps that time the phases when the timed steps replay a graph
FP32_LANES_PER_SM = 128

# DRAM traffic of walk_kernel from one single-pass ncu capture
# (dram__bytes_read.sum + dram__bytes_write.sum) of the N=2^23 galaxy's
# warm-up-step walk, per particle; at another N the launch is scaled by
# particles.  It is reported only while the walk source is the one the
# counters were taken on (sha256 of walk_impl.cuh).
WALK_TRAFFIC = {"bytes_per_particle": (230.617e6 + 110.988e6) / 8388608,
                "n_captured": 8388608,
                "walk_impl_sha256": "f45061adc710b78f6f6a1da075f2fc1840aeb28aed1bfb5370e2eeb20542bb67",
                "capture": "profiles/walk_kernel_traffic_galaxy_2e23.md"}


def walk_traffic(n):
    import hashlib
    src = os.path.join(ROOT, "paper_1811_02761_gb300", "csrc", "walk_impl.cuh")
    try:
        sha = hashlib.sha256(open(src, "rb").read()).hexdigest()
    except OSError:
        return None, "walk source not found"
    if sha != WALK_TRAFFIC["walk_impl_sha256"]:
        return None, "walk kernel changed since the ncu capture"
    note = WALK_TRAFFIC["capture"]
    if n != WALK_TRAFFIC["n_captured"]:
        note += f" (N={WALK_TRAFFIC['n_captured']}, scaled by particles)"
    return WALK_TRAFFIC["bytes_per_particle"] * n, note


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=32)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=("ours", "reference"), default="ours")
    ap.add_argument("--workload", choices=("galaxy", "batched", "learned", "precision", "scaling"),
                    default="galaxy",
                    help="galaxy: N=2^23 three-component galaxy (the headline); batched: 512 "
                         "independent Plummer/Hernquist systems, one forest per step; learned: "
                         "MLP-ordered walk queue at N=25*2^20; precision: delta_acc sweep, plain "
                         "vs compensated, error vs FP64 direct, FP64 energy/momentum drift; "
                         "scaling: the galaxy step from N=2^10 to N=25*2^20 with its breakdown")
    ap.add_argument("--nsys", type=int, default=512)
    ap.add_argument("--train-steps", type=int, default=20)
    ap.add_argument("--train-epochs", type=int, default=2)
    ap.add_argument("--schedules", action="store_true",
                    help="batched: also train the cost model and time each queue schedule")
    ap.add_argument("--autotune", action="store_true",
                    help="batched: also autotune leaf capacity, group size, i-particles per lane, "
                         "list depth and warps per CTA on the forest and time the tuned step")
    ap.add_argument("--per-system-steps", type=int, default=2,
                    help="batched: steps timed for the one-call-per-system comparison")
    ap.add_argument("--n", type=int, default=1 << 23)
    ap.add_argument("--quadrupole", type=int, default=0, choices=(0, 1),
                    help="galaxy: nodes carry quadrupoles (an extension beyond the paper's "
                         "monopoles); precision: add a quadrupole sweep")
    ap.add_argument("--use-graph", type=int, default=1, choices=(0, 1),
                    help="galaxy: replay the steps as a two-step CUDA graph (1, default) or "
                         "launch them eagerly (0)")
    ap.add_argument("--block-levels", type=int, default=0,
                    help="galaxy: block time steps with levels 0..K (step dt/2^k); 0 = shared step")
    ap.add_argument("--block-eta", type=float, default=0.025)
    ap.add_argument("--dt", type=float, default=DT, help="galaxy: the (largest) time step")
    ap.add_argument("--rebuild-interval", type=int, default=1,
                    help="galaxy: tree rebuilt every k-th step, refitted between (0: automatic, "
                         "by timing); the headline configuration rebuilds every step")
    ap.add_argument("--seed", type=int, default=2)
    ap.add_argument("--e2e-steps", type=int, default=4)
    ap.add_argument("--error-sample", type=int, default=4096,
                    help="seeded particles whose accelerations are checked against the FP64 direct sum")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--sweep-sample", type=int, default=1 << 16)
    ap.add_argument("--sweep-max", type=int, default=20)
    ap.add_argument("--drift-steps", type=int, default=256)
    ap.add_argument("--drift-every", type=int, default=32)
    ap.add_argument("--cpu-group-stride", type=int, default=1,
                    help="CPU baseline walks every k-th group of the full tree")
    return ap.parse_args()


def workload_config(n, rebuild_interval=1, dt=DT, block_levels=0, block_eta=0.025):
    rb = ("tree rebuilt every step" if rebuild_interval == 1 else
          "tree rebuilt when timing says so (refitted between)" if rebuild_interval == 0 else
          f"tree rebuilt every {rebuild_interval} steps (refitted between)")
    dts = "1/256" if dt == DT else f"{dt:g}"
    integ = (f"shared-step leapfrog dt={dts}" if block_levels == 0 else
             f"block-step leapfrog, levels dt/2^k for k=0..{block_levels}, dt={dts}, "
             f"criterion sqrt(2*{block_eta:g}*eps/|a|)")
    return {
        "workload": f"three-component galaxy N={n} (Hernquist bulge 15% a=0.6, exponential disk "
                    f"10% Rd=5.4 z0=0.6, NFW halo 75% rs=12 cut 10rs), eps=1/64, "
                    f"delta_acc=2^-9, {integ}, {rb}",
        "n": n,
        "flops_per_interaction": FLOPS_PER_INTERACTION,
        "l2": l2_note(n),
    }


def l2_note(n):
    """Whether one step's inputs exceed the 129 MB L2 (about 0.45 GB of particle state
    and 0.4 GB of tree at N = 2^23, in proportion to N)."""
    state, tree = 0.45 * n / (1 << 23), 0.4 * n / (1 << 23)
    if state + tree > 0.129:
        return f"inputs larger than L2 (particle state ~{state:.2g} GB, tree ~{tree:.2g} GB > 129 MB)"
    return (f"inputs smaller than L2 (~{1e3 * (state + tree):.2g} MB < 129 MB); "
            "L2 not flushed between steps")


# ---------------------------------------------------------------------------- clocks
class ClockSampler:
    FIELDS = ("uuid,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, uuid):
        self.uuid = uuid
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        for line in open(self.path):
            f = [c.strip() for c in line.split(",")]
            if len(f) < 9 or (self.uuid and self.uuid not in f[0]):
                continue
            rows.append(f)
        os.unlink(self.path)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        reasons = sorted({nm for r in rows for nm, v in zip(names, r[5:9]) if "Active" == v})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "samples": len(rows),
                "reasons": reasons}


def measured_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        return {}


# ---------------------------------------------------------------------------- oracle (CPU)
def oracle_small_timings():
    """The FP64 oracle on the N = 2^13 Plummer sphere: the direct sum on all
    cores and on one core, and the tree build + group walk (all cores)."""
    import ics
    import oracle
    p = ics.plummer(1 << 13, 1)
    x, y, z, m = (np.asarray(p[k], np.float64) for k in ("x", "y", "z", "m"))
    out = {"n": 1 << 13}
    for label, k in (("direct_all_cores_s", 0), ("direct_one_core_s", 1)):
        oracle.set_threads(k)
        t0 = time.perf_counter()
        oracle.direct(x, y, z, m, 1.0, 1.0 / 128, want_phi=False)
        out[label] = time.perf_counter() - t0
    oracle.set_threads(0)
    out["all_cores"] = oracle.threads()
    t0 = time.perf_counter()
    t = oracle.Tree(x, y, z, m, 21, 16)
    ax, ay, az, _, _ = t.walk(oracle.MAC_GROUP_GEO, 1.0, 1.0 / 128, 0.0, 0.5, 64, None,
                              want_phi=False)
    out["tree_build_walk_s"] = time.perf_counter() - t0
    return out


def cpu_oracle_sample(p, group_stride, a_old=None):
    """FP64 oracle: full tree build + walk of every group_stride-th group.
    Returns (interactions, walk_seconds, build_seconds, threads, ngroups_walked)."""
    import oracle
    x, y, z, m = (np.asarray(p[k], np.float64) for k in ("x", "y", "z", "m"))
    t0 = time.perf_counter()
    tree = oracle.Tree(x, y, z, m, 21, 16)
    t1 = time.perf_counter()
    f, c = tree.groups(64)
    sel = np.arange(0, f.size, group_stride)
    if a_old is None:  # bootstrap for the sampled groups, as the library does
        gx, gy, gz, _ = tree.walk_groups(sel, oracle.MAC_GROUP_GEO, 1.0, EPS, 0.0, 0.5, 64, None)
        a_old = np.nan_to_num(np.sqrt(gx ** 2 + gy ** 2 + gz ** 2), nan=1.0)
    t2 = time.perf_counter()
    _, _, _, nint = tree.walk_groups(sel, oracle.MAC_GROUP_ACC, 1.0, EPS, DACC, 0.5, 64, a_old)
    t3 = time.perf_counter()
    return int(nint[nint > 0].sum()), t3 - t2, t1 - t0, oracle.threads(), int(sel.size), int(f.size)


# ---------------------------------------------------------------------------- our arm
def oracle_force_error(final, sample, seed):
    """Relative error of the GPU accelerations against FP64 direct summation
    (the oracle) on `sample` seeded particles at the final positions."""
    import oracle
    xs, ms, ga = final
    tg = np.random.default_rng(seed).choice(ms.size, sample, replace=False)
    t0 = time.perf_counter()
    bx, by, bz, _ = oracle.direct_targets(*xs, ms, tg, 1.0, EPS)
    e = oracle.rel_err(*[a[tg].astype(np.float64) for a in ga], bx, by, bz)
    return {"p50": oracle.percentile_nearest_rank(e, 50),
            "p99": oracle.percentile_nearest_rank(e, 99), "max": float(e.max()),
            "sample": int(sample), "vs": "FP64 direct summation at the final positions",
            "oracle_s": time.perf_counter() - t0, "cores": oracle.threads()}


def run_ours(args, rank, world, local_rank):
    import torch
    import torch.distributed as dist

    import ics
    import paper_1811_02761_gb300 as nb

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    props = torch.cuda.get_device_properties(dev)
    nsm = props.multi_processor_count
    uuid = str(getattr(props, "uuid", "") or "")
    p = ics.galaxy(args.n, args.seed)
    n = args.n

    def D(a):
        return torch.from_numpy(np.ascontiguousarray(a)).to(dev)

    X64 = [D(p[k]) for k in ("x64", "y64", "z64")]
    V = [D(p[k]) for k in ("vx", "vy", "vz")]
    M = D(p["m"])
    A = [torch.empty(n, dtype=torch.float32, device=dev) for _ in range(3)]
    stream = torch.cuda.current_stream(dev)
    cfg = nb.nbody_config_default(eps=EPS, delta_acc=DACC, rebuild_interval=args.rebuild_interval,
                                  quadrupole=args.quadrupole, block_levels=args.block_levels,
                                  block_eta=args.block_eta, use_graph=args.use_graph)
    dt = args.dt
    ctx = nb.nbody_create(cfg, stream)
    try:
        # accelerations at t = 0 (bootstrap MAC), then warm-up steps
        nb.nbody_build(ctx, *[D(p[k]) for k in ("x", "y", "z")], M)
        nb.nbody_walk(ctx, None, *A)
        nb.nbody_step(ctx, *X64, *V, M, *A, dt, args.warmup)
        torch.cuda.synchronize(dev)
        if world > 1:
            dist.barrier()
        sampler = ClockSampler(uuid)
        sampler.start()
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize(dev)
        ev0.record(stream)
        st = nb.nbody_step(ctx, *X64, *V, M, *A, dt, args.steps)
        ev1.record(stream)
        torch.cuda.synchronize(dev)
        clocks = sampler.stop()
        if world > 1:
            dist.barrier()
        elapsed = ev0.elapsed_time(ev1) / 1e3
        inter = st.interactions
        t = torch.tensor([elapsed], dtype=torch.float64, device=dev)
        it = torch.tensor([inter], dtype=torch.float64, device=dev)
        if world > 1:
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            dist.all_reduce(it, op=dist.ReduceOp.SUM)
        elapsed_max, inter_all = float(t.item()), float(it.item())
        # the walk kernel's CUDA-event time inside the timed call: its eager
        # steps and, with the graph, the last replay's two walks (event nodes)
        walk_ms, walk_launches = st.ms_walk_kernel, st.walk_launches
        phase_ms, phase_steps = (st.ms_build, st.ms_walk), args.steps
        wcfg = nb.nbody_get_config(ctx)
        graph_used = (wcfg.use_graph and args.steps >= 3 and wcfg.rebuild_interval == 1
                      and wcfg.block_levels == 0)  # the library's condition for replays
        if graph_used:  # graph replays carry no phase events:
            # time the build and walk phases in eager steps
            c2 = nb.nbody_get_config(ctx)
            c2.use_graph = 0
            nb.nbody_set_config(ctx, c2)
            s3 = nb.nbody_step(ctx, *X64, *V, M, *A, dt, PHASE_STEPS)
            phase_ms, phase_steps = (s3.ms_build, s3.ms_walk), PHASE_STEPS
            c2.use_graph = 1
            nb.nbody_set_config(ctx, c2)

        # end-to-end through the C ABI with pinned host buffers
        hx = [a.cpu().pin_memory() for a in X64]
        hv = [a.cpu().pin_memory() for a in V]
        hm = M.cpu().pin_memory()
        ha = [a.cpu().pin_memory() for a in A]
        torch.cuda.synchronize(dev)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e2e_inter = 0
        e0.record(stream)
        w0 = time.perf_counter()
        for _ in range(args.e2e_steps):
            s2 = nb.nbody_step(ctx, *hx, *hv, hm, *ha, dt, 1)
            e2e_inter += s2.interactions
        e1.record(stream)
        torch.cuda.synchronize(dev)
        e2e_wall = time.perf_counter() - w0
        e2e_s = max(e0.elapsed_time(e1) / 1e3, e2e_wall)

        # final state on the host, for the oracle leg's force-error check
        final = None
        if rank == 0 and world == 1 and (not args.no_cpu_baseline or args.error_sample > 0):
            final = ([a.cpu().numpy().astype(np.float32).astype(np.float64) for a in X64],
                     M.cpu().numpy().astype(np.float64), [a.cpu().numpy() for a in A])
    finally:
        nb.nbody_destroy(ctx)

    if rank != 0:
        return None
    steps = args.steps
    s_per_step = elapsed_max / steps
    value = inter_all / elapsed_max / 1e9
    inter_per_step = inter / steps
    walk_avg_s = (walk_ms / max(walk_launches, 1)) / 1e3
    walk_tflops = FLOPS_PER_INTERACTION * inter_per_step / walk_avg_s / 1e12
    peaks = measured_peaks()
    sm_max = float(peaks.get("sm_max_mhz", 2070.0))
    peak_tflops = 2 * FP32_LANES_PER_SM * nsm * sm_max * 1e6 / 1e12
    med = clocks["sm_mhz"] if clocks and clocks.get("sm_mhz") else None
    peak_med = 2 * FP32_LANES_PER_SM * nsm * med * 1e6 / 1e12 if med else None
    whole_tflops = FLOPS_PER_INTERACTION * inter_per_step / s_per_step / 1e12
    traffic, traffic_note = walk_traffic(n)

    # oracle leg (rank 0, N = 1): the FP64 oracle tree walk on a bounded
    # sample, timed on the host cores, and the FP64 direct sum at the final
    # positions that states the force error of the GPU accelerations
    cpu, err = None, None
    if final is not None and args.error_sample > 0:
        err = oracle_force_error(final, args.error_sample, args.seed)
    if final is not None and not args.no_cpu_baseline:
        ni, walk_s, build_s, thr, nsel, ng = cpu_oracle_sample(p, args.cpu_group_stride)
        cpu = {"value": ni / walk_s / 1e9, "unit": UNIT, "cores": thr, "kind": "oracle",
               "sample": f"FP64 oracle tree walk (group-mode acceleration MAC) of "
                         f"{'every group' if args.cpu_group_stride == 1 else f'every {args.cpu_group_stride}-th group'} "
                         f"({nsel} of {ng} groups, {ni} interactions) of the same N={n} galaxy "
                         f"at its initial positions; oracle tree build {build_s:.2f} s timed "
                         f"separately",
               "build_s": build_s, "walk_s": walk_s, "small": oracle_small_timings()}

    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": steps,
        "warmup": args.warmup, "ms_per_step": s_per_step * 1e3, "s_per_step": s_per_step,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic (seeded three-component galaxy; stands in for the paper's M31 model)",
        "config": dict(workload_config(n, args.rebuild_interval, dt, args.block_levels,
                                       args.block_eta), parallelism=f"replicas x{world}",
                       walk=cfg.as_dict()),
        "interactions_per_step": inter_per_step,
        "whole_step_tflops": whole_tflops,
        "whole_step_fp32_peak_frac": whole_tflops / peak_tflops,
        "walk_ms_per_step": walk_ms / max(walk_launches, 1),
        "walk_timing": f"CUDA events around {walk_launches} walk launches inside the timed call "
                       f"(its eager steps and the last graph replay's two walks, event nodes of "
                       f"the graph)",
        "build_ms_per_step": phase_ms[0] / phase_steps,
        "walk_phase_ms_per_step": phase_ms[1] / phase_steps,
        "phase_timing": "eager steps (CUDA events per phase)" if not graph_used else
                        f"{PHASE_STEPS} extra eager steps after the timed graph replays (CUDA "
                        "events per phase; graph nodes carry no events; the first step of the "
                        "call also gathers the state from the caller's order)",
        "nodes": st.n_nodes, "groups": st.n_groups, "max_stack": st.max_stack,
        "rebuilds": int(st.rebuilds),
        "quadrupole": args.quadrupole,
        "block_levels": args.block_levels, "block_eta": args.block_eta, "dt": dt,
        "quad_interactions_per_step": st.quad_interactions / steps,
        "roofline": {"bound": "alu", "achieved": walk_tflops, "peak": peak_tflops,
                     "unit": "TFLOP/s", "frac": walk_tflops / peak_tflops, "traffic": traffic,
                     "traffic_note": traffic_note, "kernel": "walk_kernel",
                     "peak_note": f"FP32 2 x {FP32_LANES_PER_SM} lanes x {nsm} SMs x {sm_max:.0f} MHz "
                                  f"(max clock, MEASURED_PEAKS sm_max_mhz)",
                     "frac_at_median_clock": (walk_tflops / peak_med) if peak_med else None},
        "force_error": err,
        "cpu_baseline": cpu,
        "e2e": {"value": e2e_inter / e2e_s / 1e9, "unit": UNIT,
                "h2d_bytes_per_step": n * (3 * 8 + 7 * 4),
                "d2h_bytes_per_step": n * (3 * 8 + 6 * 4),
                "steps": args.e2e_steps,
                "note": "nbody_step(nsteps=1) per step on pinned host arrays: every call reads "
                        "the state from host memory and writes it back (the state load and the "
                        "closing gather use the page-locked arrays in place)"},
        "clocks": clocks,
        "gpu_launches": int(st.kernels),
    }
    return out


# ---------------------------------------------------------------------------- batched workload
def run_batched(args, rank, world, local_rank):
    """512 independent systems: one forest + one persistent walk per step
    (CUDA graph of two steps) against one nbody_step call per system.  With N
    ranks every rank takes whole systems, placed by predicted walk cost, and
    no collective touches the data path."""
    import torch
    import torch.distributed as dist

    import ics
    import paper_1811_02761_gb300 as nb

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    from paper_1811_02761_gb300.sharding import (local_csr, partition_systems, rank_loads,
                                                  system_costs)
    full = ics.batched(args.nsys, 4)
    placement, cost = "single rank: every system", None
    if world > 1:
        # predicted cost per system: its interactions in one walk of the whole
        # forest (every rank computes the same numbers, so the placement needs
        # no communication), then longest-processing-time placement by cost
        cost = batched_system_costs(full, dev)
        placement = "whole systems by predicted walk cost (interactions of a probe walk), LPT"
    parts_all = partition_systems(np.diff(full["offsets"]), world, cost)
    mine = parts_all[rank]
    off, idx = local_csr(full["offsets"], mine)
    parts = {k: full[k][idx] for k in ("x", "y", "z", "vx", "vy", "vz", "m")}
    sizes = np.diff(off)
    eps = full["eps"][mine]
    n = int(off[-1])

    def D(a):
        return torch.from_numpy(np.ascontiguousarray(a)).to(dev)

    X = [D(parts[k].astype(np.float64)) for k in ("x", "y", "z")]
    V = [D(parts[k]) for k in ("vx", "vy", "vz")]
    M = D(parts["m"])
    A = [torch.zeros(n, dtype=torch.float32, device=dev) for _ in range(3)]
    stream = torch.cuda.current_stream(dev)
    cfg = nb.nbody_config_default(delta_acc=DACC, use_graph=1)
    ctx = nb.nbody_create(cfg, stream)
    try:
        # initial accelerations: bootstrap walk of the forest
        nb.nbody_build_batched(ctx, off, eps, *[D(parts[k]) for k in ("x", "y", "z")], M)
        nb.nbody_walk(ctx, None, *A)
        nb.nbody_step_batched(ctx, off, eps, *X, *V, M, *A, DT, max(args.warmup, 2))
        torch.cuda.synchronize(dev)
        if world > 1:
            dist.barrier()
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        st = nb.nbody_step_batched(ctx, off, eps, *X, *V, M, *A, DT, args.steps)
        ev1.record(stream)
        torch.cuda.synchronize(dev)
        if world > 1:
            dist.barrier()
        elapsed = ev0.elapsed_time(ev1) / 1e3
    finally:
        nb.nbody_destroy(ctx)
    # the same systems, one nbody_step call per system and step
    ctx = nb.nbody_create(nb.nbody_config_default(delta_acc=DACC), stream)
    try:
        def one_pass(k):
            for j in range(len(sizes)):
                a, b = int(off[j]), int(off[j + 1])
                c2 = nb.nbody_config_default(delta_acc=DACC, eps=float(eps[j]))
                nb.nbody_set_config(ctx, c2)
                nb.nbody_step(ctx, *[t[a:b] for t in X], *[t[a:b] for t in V], M[a:b],
                              *[t[a:b] for t in A], DT, k)
        one_pass(1)
        torch.cuda.synchronize(dev)
        w0 = time.perf_counter()
        one_pass(args.per_system_steps)
        torch.cuda.synchronize(dev)
        per_sys = (time.perf_counter() - w0) / args.per_system_steps
    finally:
        nb.nbody_destroy(ctx)
    tuned = batched_autotune(args, off, eps, parts, stream, dev, elapsed / args.steps) \
        if args.autotune else None
    # schedules at the default parameters; with --autotune they add a run tuned
    # under the learned order itself
    sched = batched_schedules(args, off, eps, parts, stream, dev) if args.schedules else None
    t = torch.tensor([elapsed, float(st.interactions)], dtype=torch.float64, device=dev)
    if world > 1:
        tm = t[:1].clone()
        dist.all_reduce(tm, op=dist.ReduceOp.MAX)
        dist.all_reduce(t, op=dist.ReduceOp.SUM)
        t[0] = tm[0]
    if rank != 0:
        return None
    elapsed_max, inter_all = float(t[0].item()), float(t[1].item())
    s_per_step = elapsed_max / args.steps
    return {
        "metric": METRIC, "value": inter_all / elapsed_max / 1e9, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": s_per_step * 1e3,
        "s_per_step": s_per_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32",
        "data": "synthetic (seeded Plummer/Hernquist systems)",
        "config": {"workload": f"batched: {args.nsys} independent Plummer/Hernquist systems, "
                               f"N_s = 2^(10+6U), eps_s = 4/N_s^(1/3), delta_acc=2^-9, "
                               f"leapfrog dt=1/256; one forest and one persistent walk per step, "
                               f"CUDA graph of two steps",
                   "systems_this_rank": int(len(sizes)), "n_this_rank": n,
                   "parallelism": f"whole systems per rank x{world}",
                   "placement": placement,
                   "predicted_cost_per_rank": (rank_loads(parts_all, cost).tolist()
                                               if cost is not None else None),
                   "l2": "inputs larger than L2 (~8M particles)"},
        "per_system_launches": {"s_per_step": per_sys,
                                "note": "one nbody_step call (build + walk + kicks) per system "
                                        "and step, eager launches"},
        "speedup_vs_per_system": per_sys / s_per_step,
        "schedules": sched,
        "autotune": tuned,
        "interactions_per_step": float(st.interactions) / args.steps,
        "gpu_launches": int(st.kernels),
    }


def batched_system_costs(full, dev):
    """Interactions of every system in one acceleration-MAC walk of the whole
    forest (bootstrap walk for |a_old| first), from the walk's per-group log."""
    import torch

    import paper_1811_02761_gb300 as nb
    from paper_1811_02761_gb300.sharding import system_costs

    def D(a):
        return torch.from_numpy(np.ascontiguousarray(a)).to(dev)

    n = int(full["offsets"][-1])
    A = [torch.zeros(n, dtype=torch.float32, device=dev) for _ in range(3)]
    ctx = nb.nbody_create(nb.nbody_config_default(delta_acc=DACC), torch.cuda.current_stream(dev))
    try:
        nb.nbody_build_batched(ctx, full["offsets"], full["eps"],
                               *[D(full[k]) for k in ("x", "y", "z")], D(full["m"]))
        nb.nbody_walk(ctx, None, *A)
        amag = torch.sqrt(A[0] ** 2 + A[1] ** 2 + A[2] ** 2)
        nb.nbody_walk(ctx, amag, *A)
        first = nb.nbody_export(ctx, nb.EXPORT_GROUP_FIRST)
        count = nb.nbody_export(ctx, nb.EXPORT_GROUP_COUNT)
        costs = torch.zeros(first.size, dtype=torch.int32, device=dev)
        ng = nb.nbody_get_group_costs(ctx, costs)
        entries = costs[:ng].cpu().numpy()
    finally:
        nb.nbody_destroy(ctx)
    return system_costs(full["offsets"], first[:ng], count[:ng], entries)


def batched_autotune(args, off, eps, parts, stream, dev, default_s_per_step):
    """The autotuner's grid search (nbody_autotune: build + walk timed with
    CUDA events per candidate) on the batched forest, then the same graph
    steps as the default run with the tuned parameters."""
    import torch

    import paper_1811_02761_gb300 as nb

    def D(a):
        return torch.from_numpy(np.ascontiguousarray(a)).to(dev)

    n = int(off[-1])
    X32 = [D(parts[k]) for k in ("x", "y", "z")]
    X = [D(parts[k].astype(np.float64)) for k in ("x", "y", "z")]
    V = [D(parts[k]) for k in ("vx", "vy", "vz")]
    M = D(parts["m"])
    A = [torch.zeros(n, dtype=torch.float32, device=dev) for _ in range(3)]
    ctx = nb.nbody_create(nb.nbody_config_default(delta_acc=DACC, use_graph=1), stream)
    try:
        nb.nbody_build_batched(ctx, off, eps, *X32, M)
        nb.nbody_walk(ctx, None, *A)
        amag = torch.sqrt(A[0] ** 2 + A[1] ** 2 + A[2] ** 2).contiguous()
        w0 = time.perf_counter()
        best, ms, tried = nb.nbody_autotune(ctx, off, eps, *X32, M, amag)
        tune_s = time.perf_counter() - w0
        best.use_graph = 1
        nb.nbody_set_config(ctx, best)
        nb.nbody_build_batched(ctx, off, eps, *X32, M)
        nb.nbody_walk(ctx, None, *A)
        nb.nbody_step_batched(ctx, off, eps, *X, *V, M, *A, DT, max(args.warmup, 2))
        torch.cuda.synchronize(dev)
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        nb.nbody_step_batched(ctx, off, eps, *X, *V, M, *A, DT, args.steps)
        ev1.record(stream)
        torch.cuda.synchronize(dev)
        s_step = ev0.elapsed_time(ev1) / 1e3 / args.steps
    finally:
        nb.nbody_destroy(ctx)
    from paper_1811_02761_gb300.autotune import TUNED_FIELDS
    return {"tuned": {k: int(getattr(best, k)) for k in TUNED_FIELDS}, "candidates": tried,
            "search_s": tune_s, "best_build_walk_ms": ms, "s_per_step": s_step,
            "speedup_vs_default": default_s_per_step / s_step}


def batched_schedules(args, off, eps, parts, stream, dev, tuned=None):
    """The batched forest under each queue schedule, eager and in the step's
    CUDA graph (with `tuned`: the autotuner's parameters): the cost model is
    trained online on `train_steps` Morton-order steps, then `steps` steps run
    from the same state per schedule.  Final states must agree bit for bit."""
    import torch

    import ics
    import paper_1811_02761_gb300 as nb

    def D(a):
        return torch.from_numpy(np.ascontiguousarray(a)).to(dev)

    n = int(off[-1])
    X = [D(parts[k].astype(np.float64)) for k in ("x", "y", "z")]
    V = [D(parts[k]) for k in ("vx", "vy", "vz")]
    M = D(parts["m"])
    A = [torch.zeros(n, dtype=torch.float32, device=dev) for _ in range(3)]
    cfg0 = nb.nbody_config_default(delta_acc=DACC)
    for k, v in (tuned or {}).items():
        setattr(cfg0, k, v)
    ctx = nb.nbody_create(cfg0, stream)
    out, finals = {}, {}
    try:
        nb.nbody_build_batched(ctx, off, eps, *[D(parts[k]) for k in ("x", "y", "z")], M)
        nb.nbody_walk(ctx, None, *A)
        nb.nbody_mlp_set_params(ctx, ics.mlp_init(args.seed))
        losses = []
        for _ in range(args.train_steps):
            nb.nbody_step_batched(ctx, off, eps, *X, *V, M, *A, DT, 1)
            losses.append(nb.nbody_mlp_train(ctx, epochs=args.train_epochs, lr=2e-3, batch=4096))
        snap = [t.clone() for t in X + V + A]
        for name, sc, graph in (("morton", nb.SCHED_MORTON, 0), ("mlp", nb.SCHED_MLP, 0),
                                ("lastcost", nb.SCHED_LASTCOST, 0),
                                ("morton_graph", nb.SCHED_MORTON, 1), ("mlp_graph", nb.SCHED_MLP, 1)):
            for t, s0 in zip(X + V + A, snap):
                t.copy_(s0)
            cfg = nb.nbody_get_config(ctx)
            cfg.schedule, cfg.use_graph = sc, graph
            nb.nbody_set_config(ctx, cfg)
            if graph:  # capture outside the timed region
                nb.nbody_step_batched(ctx, off, eps, *X, *V, M, *A, DT, 2)
                for t, s0 in zip(X + V + A, snap):
                    t.copy_(s0)
            torch.cuda.synchronize(dev)
            ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            ev0.record(stream)
            st = nb.nbody_step_batched(ctx, off, eps, *X, *V, M, *A, DT, args.steps)
            ev1.record(stream)
            torch.cuda.synchronize(dev)
            out[name] = {"walk_ms_per_step": st.ms_walk_kernel / max(st.walk_launches, 1),
                         "s_per_step": ev0.elapsed_time(ev1) / 1e3 / args.steps}
            finals[name] = [t.cpu().numpy() for t in X + V + A]
        if args.autotune and tuned is None:
            # tune under the learned order: the autotuner's timed walks use the
            # context's schedule, so candidates are timed as they will run
            for t, s0 in zip(X + V + A, snap):
                t.copy_(s0)
            cfg = nb.nbody_get_config(ctx)
            cfg.schedule, cfg.use_graph = nb.SCHED_MLP, 1
            nb.nbody_set_config(ctx, cfg)
            amag = torch.sqrt(A[0] ** 2 + A[1] ** 2 + A[2] ** 2).contiguous()
            best, _, _ = nb.nbody_autotune(ctx, off, eps, *[x.float() for x in X], M, amag)
            best.schedule, best.use_graph = nb.SCHED_MLP, 1
            nb.nbody_set_config(ctx, best)
            nb.nbody_step_batched(ctx, off, eps, *X, *V, M, *A, DT, 2)
            for t, s0 in zip(X + V + A, snap):
                t.copy_(s0)
            torch.cuda.synchronize(dev)
            ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            ev0.record(stream)
            nb.nbody_step_batched(ctx, off, eps, *X, *V, M, *A, DT, args.steps)
            ev1.record(stream)
            torch.cuda.synchronize(dev)
            from paper_1811_02761_gb300.autotune import TUNED_FIELDS
            out["mlp_graph_tuned_under_mlp"] = {
                "s_per_step": ev0.elapsed_time(ev1) / 1e3 / args.steps,
                "parameters": {k: int(getattr(best, k)) for k in TUNED_FIELDS}}
    finally:
        nb.nbody_destroy(ctx)
    base = out["morton"]["walk_ms_per_step"]
    return {"runs": out, "parameters": "autotuned" if tuned else "defaults",
            "mlp_vs_morton_walk_speedup": base / out["mlp"]["walk_ms_per_step"],
            "mlp_graph_vs_morton_graph_step_speedup":
                out["morton_graph"]["s_per_step"] / out["mlp_graph"]["s_per_step"],
            "lastcost_vs_morton_walk_speedup": base / out["lastcost"]["walk_ms_per_step"],
            "bitwise_identical_final_states": all(
                np.array_equal(a, b) for k in ("mlp", "lastcost", "morton_graph", "mlp_graph")
                for a, b in zip(finals["morton"], finals[k])),
            "train_losses_first_last": [losses[0], losses[-1]] if losses else None}


def schedule_makespans(cost, pred, workers):
    """How much any queue order could gain: list scheduling of the groups
    (time taken as proportional to the logged list entries of each group)
    onto `workers` walk warps in Morton order, in descending predicted cost
    and in descending true cost, against the lower bound max(total / workers,
    largest group).  Locality effects are not modelled."""
    import heapq

    def makespan(order):
        h = [0.0] * workers
        for g in order:
            heapq.heapreplace(h, h[0] + cost[g])
        return max(h)

    lb = max(cost.sum() / workers, cost.max())
    return {"workers": workers, "groups": int(cost.size),
            "morton_over_bound": makespan(range(cost.size)) / lb,
            "predicted_order_over_bound": makespan(np.argsort(-pred, kind="stable")) / lb,
            "true_lpt_over_bound": makespan(np.argsort(-cost, kind="stable")) / lb,
            "note": "group time taken proportional to its list entries"}


# ---------------------------------------------------------------------------- learned schedule
def run_learned(args, rank, world, local_rank):
    """Galaxy at N = 25 * 2^20: the cost model is trained online on the first
    `train_steps` steps (Morton order), then the remaining steps run three
    times from the same state -- MLP-ordered queue, Morton order, last-step
    cost order -- and the walk-kernel times are compared.  The final states
    must agree bit for bit (the order never changes a group's result)."""
    import torch

    import ics
    import paper_1811_02761_gb300 as nb

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    n = args.n if args.n != (1 << 23) else 25 * (1 << 20)
    p = ics.galaxy(n, args.seed)

    def D(a):
        return torch.from_numpy(np.ascontiguousarray(a)).to(dev)

    X = [D(p[k]) for k in ("x64", "y64", "z64")]
    V = [D(p[k]) for k in ("vx", "vy", "vz")]
    M = D(p["m"])
    A = [torch.empty(n, dtype=torch.float32, device=dev) for _ in range(3)]
    stream = torch.cuda.current_stream(dev)
    ctx = nb.nbody_create(nb.nbody_config_default(eps=EPS, delta_acc=DACC), stream)
    out = {}
    try:
        nb.nbody_build(ctx, *[D(p[k]) for k in ("x", "y", "z")], M)
        nb.nbody_walk(ctx, None, *A)
        nb.nbody_mlp_set_params(ctx, ics.mlp_init(args.seed))
        losses = []
        t0 = time.perf_counter()
        for _ in range(args.train_steps):
            st_train = nb.nbody_step(ctx, *X, *V, M, *A, DT, 1)
            losses.append(nb.nbody_mlp_train(ctx, epochs=args.train_epochs, lr=2e-3, batch=4096))
        train_s = time.perf_counter() - t0
        pred, _ = nb.nbody_mlp_predict(ctx)
        cost = np.empty(pred.size, np.int32)
        nb.nbody_get_group_costs(ctx, cost)
        corr = float(np.corrcoef(pred, np.log2(np.maximum(cost, 1)))[0, 1])

        sched_model = schedule_makespans(cost.astype(np.float64), pred, int(st_train.walk_warps))
        snap = [t.clone() for t in X + V + A]
        runs = args.steps - args.train_steps
        finals = {}
        for name, sched in (("mlp", nb.SCHED_MLP), ("morton", nb.SCHED_MORTON),
                            ("lastcost", nb.SCHED_LASTCOST)):
            for t, s0 in zip(X + V + A, snap):
                t.copy_(s0)
            cfg = nb.nbody_get_config(ctx)
            cfg.schedule = sched
            nb.nbody_set_config(ctx, cfg)
            torch.cuda.synchronize(dev)
            ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            ev0.record(stream)
            st = nb.nbody_step(ctx, *X, *V, M, *A, DT, runs)
            ev1.record(stream)
            torch.cuda.synchronize(dev)
            out[name] = {"walk_ms_per_step": st.ms_walk_kernel / max(st.walk_launches, 1),
                         "s_per_step": ev0.elapsed_time(ev1) / 1e3 / runs,
                         "interactions_per_step": st.interactions / runs}
            finals[name] = [t.cpu().numpy() for t in X + V + A]
        same = all(np.array_equal(a, b) for k in ("morton", "lastcost")
                   for a, b in zip(finals["mlp"], finals[k]))
    finally:
        nb.nbody_destroy(ctx)
    if rank != 0:
        return None
    base = out["morton"]["walk_ms_per_step"]
    return {
        "metric": METRIC, "value": out["mlp"]["interactions_per_step"] / out["mlp"]["s_per_step"] / 1e9,
        "unit": UNIT, "n_gpus": world, "steps": args.steps, "warmup": args.train_steps,
        "ms_per_step": out["mlp"]["s_per_step"] * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic (seeded three-component galaxy)",
        "config": {"workload": f"learned scheduling: galaxy N={n}, {args.train_steps} training "
                               f"steps (Morton order, {args.train_epochs} epochs each), then "
                               f"{args.steps - args.train_steps} steps per schedule from the same state",
                   "n": n},
        "schedules": out,
        "mlp_vs_morton_walk_speedup": base / out["mlp"]["walk_ms_per_step"],
        "lastcost_vs_morton_walk_speedup": base / out["lastcost"]["walk_ms_per_step"],
        "bitwise_identical_final_states": same,
        "train": {"losses_first_last": [losses[0], losses[-1]], "seconds": train_s,
                  "pred_vs_cost_correlation": corr},
        "schedule_model": sched_model,
    }


# ---------------------------------------------------------------------------- N scaling
def run_scaling(args, rank, world, local_rank):
    """The galaxy step at N = 2^10, 2^12, ..., 2^24 and 25 * 2^20: s/step,
    walk and build time per step, interactions per particle and rate (the
    N dependence the paper measures in Sect. 4.1).  Rank 0 only."""
    import torch

    import ics
    import paper_1811_02761_gb300 as nb
    if rank != 0:
        return None
    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    props = torch.cuda.get_device_properties(dev)
    peaks = measured_peaks()
    peak = 2 * FP32_LANES_PER_SM * props.multi_processor_count * float(
        peaks.get("sm_max_mhz", 2070.0)) * 1e6 / 1e12
    sizes = [1 << k for k in range(10, 25, 2)] + [25 * (1 << 20)]
    rows = []
    stream = torch.cuda.current_stream(dev)

    def D(a):
        return torch.from_numpy(np.ascontiguousarray(a)).to(dev)

    for n in sizes:
        p = ics.galaxy(n, args.seed)
        X64 = [D(p[k]) for k in ("x64", "y64", "z64")]
        V = [D(p[k]) for k in ("vx", "vy", "vz")]
        M = D(p["m"])
        A = [torch.empty(n, dtype=torch.float32, device=dev) for _ in range(3)]
        ctx = nb.nbody_create(nb.nbody_config_default(eps=EPS, delta_acc=DACC), stream)
        try:
            nb.nbody_build(ctx, *[D(p[k]) for k in ("x", "y", "z")], M)
            nb.nbody_walk(ctx, None, *A)
            nb.nbody_step(ctx, *X64, *V, M, *A, DT, args.warmup)
            steps = max(args.steps, 4)
            ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize(dev)
            ev0.record(stream)
            st = nb.nbody_step(ctx, *X64, *V, M, *A, DT, steps)
            ev1.record(stream)
            torch.cuda.synchronize(dev)
        finally:
            nb.nbody_destroy(ctx)
        s = ev0.elapsed_time(ev1) / 1e3 / steps
        walk_ms = st.ms_walk_kernel / max(st.walk_launches, 1)
        ipp = st.interactions / steps / n
        rows.append({"n": n, "s_per_step": s, "walk_ms": walk_ms, "build_ms": st.ms_build / steps,
                     "interactions_per_particle": ipp,
                     "ginter_s": st.interactions / steps / s / 1e9,
                     "walk_fp32_peak_frac": FLOPS_PER_INTERACTION * ipp * n / (walk_ms / 1e3) / 1e12 / peak,
                     "groups": int(st.n_groups), "nodes": int(st.n_nodes)})
        del X64, V, M, A
        torch.cuda.empty_cache()
    head = next(r for r in rows if r["n"] == 1 << 24)
    return {
        "metric": METRIC, "value": head["ginter_s"], "unit": UNIT, "n_gpus": 1,
        "steps": max(args.steps, 4), "warmup": args.warmup, "ms_per_step": head["s_per_step"] * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic (seeded three-component galaxy)",
        "config": {"workload": "N scaling: galaxy N = 2^10 .. 2^24 and 25*2^20, eps=1/64, "
                               "delta_acc=2^-9, shared-step leapfrog dt=1/256; value is the N=2^24 row"},
        "rows": rows,
    }


# ---------------------------------------------------------------------------- precision sweep
def run_precision(args, rank, world, local_rank):
    """Precision sweep on the galaxy: one tree, walks at delta_acc = 2^-1 ..
    2^-sweep_max with plain and with compensated accumulation, each walk's
    per-particle relative acceleration error against FP64 direct summation
    (the oracle leg: the FP64 oracle on the host cores, run in a thread beside
    the GPU work) on sweep_sample seeded particles; then the FP64 energy and
    momentum drift of drift_steps leapfrog steps, plain and compensated, at
    delta_acc = 2^-9.  Only rank 0 runs it."""
    import threading

    import torch

    import ics
    import paper_1811_02761_gb300 as nb
    if rank != 0:
        return None
    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    n = args.n
    p = ics.galaxy(n, args.seed)
    tg = np.sort(np.random.default_rng(args.seed + 1).choice(n, args.sweep_sample, replace=False))

    ref = {}

    def oracle_leg():
        import oracle
        xs = [np.asarray(p[k], np.float64) for k in ("x", "y", "z", "m")]
        t0 = time.perf_counter()
        ref["b"] = oracle.direct_targets(*xs, tg, 1.0, EPS)[:3]
        ref["s"] = time.perf_counter() - t0
        ref["threads"] = oracle.threads()

    th = threading.Thread(target=oracle_leg, daemon=True)
    th.start()

    def D(a):
        return torch.from_numpy(np.ascontiguousarray(a)).to(dev)

    M = D(p["m"])
    stream = torch.cuda.current_stream(dev)
    ctx = nb.nbody_create(nb.nbody_config_default(eps=EPS, delta_acc=DACC), stream)
    rows, drift = [], {}
    try:
        A = [torch.empty(n, dtype=torch.float32, device=dev) for _ in range(3)]
        nb.nbody_build(ctx, *[D(p[k]) for k in ("x", "y", "z")], M)
        nb.nbody_walk(ctx, None, *A)
        amag = torch.sqrt(A[0] ** 2 + A[1] ** 2 + A[2] ** 2).contiguous()
        nb.nbody_walk(ctx, amag, *A)
        amag = torch.sqrt(A[0] ** 2 + A[1] ** 2 + A[2] ** 2).contiguous()
        tgd = torch.from_numpy(tg).to(dev)
        variants = [(0, 0), (1, 0)] + ([(0, 1)] if args.quadrupole else [])
        for k in range(1, args.sweep_max + 1):
            for comp, quad in variants:
                cfg = nb.nbody_get_config(ctx)
                cfg.delta_acc, cfg.compensated, cfg.quadrupole = 2.0 ** -k, comp, quad
                if quad != nb.nbody_get_config(ctx).quadrupole:
                    nb.nbody_set_config(ctx, cfg)
                    nb.nbody_build(ctx, *[D(p[k2]) for k2 in ("x", "y", "z")], M)
                while True:
                    nb.nbody_set_config(ctx, cfg)
                    try:
                        st = nb.nbody_walk(ctx, amag, *A)
                        break
                    except nb.NbodyError as e:
                        if e.status != nb.NBODY_EOVERFLOW or cfg.stack_depth >= 4096:
                            raise
                        cfg.stack_depth *= 2
                ms = st.ms_walk_kernel / max(st.walk_launches, 1)
                rows.append({"log2_delta_acc": -k, "compensated": comp, "quadrupole": quad,
                             "walk_ms": ms, "interactions": int(st.interactions),
                             "quad_interactions": int(st.quad_interactions),
                             "ginter_s": st.interactions / ms / 1e6,
                             "stack_depth": int(cfg.stack_depth), "max_stack": int(st.max_stack),
                             "a": [a[tgd].cpu().numpy().astype(np.float64) for a in A]})

        for comp in (0, 1):
            cfg = nb.nbody_config_default(eps=EPS, delta_acc=DACC, compensated=comp)
            nb.nbody_set_config(ctx, cfg)
            X64 = [D(p[k]) for k in ("x64", "y64", "z64")]
            V = [D(p[k]) for k in ("vx", "vy", "vz")]
            nb.nbody_build(ctx, *[x.float() for x in X64], M)
            nb.nbody_walk(ctx, None, *A)
            phi = torch.empty(n, dtype=torch.float32, device=dev)
            At = [torch.empty_like(a) for a in A]

            def diagnose():
                c2 = nb.nbody_get_config(ctx)
                c2.want_potential = 1
                nb.nbody_set_config(ctx, c2)
                nb.nbody_build(ctx, *[x.float() for x in X64], M)
                am = torch.sqrt(A[0] ** 2 + A[1] ** 2 + A[2] ** 2).contiguous()
                nb.nbody_walk(ctx, am, *At, phi)
                c2.want_potential = 0
                nb.nbody_set_config(ctx, c2)
                return nb.nbody_diagnostics(ctx, *X64, *V, M, phi)

            d0 = diagnose()
            hist, t_s, steps_done = [], 0.0, 0
            while steps_done < args.drift_steps:
                k = min(args.drift_every, args.drift_steps - steps_done)
                ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                ev0.record(stream)
                nb.nbody_step(ctx, *X64, *V, M, *A, DT, k)
                ev1.record(stream)
                torch.cuda.synchronize(dev)
                t_s += ev0.elapsed_time(ev1) / 1e3
                steps_done += k
                hist.append((steps_done, diagnose()))
            e0 = d0[0] + d0[1]
            pscale = np.sqrt(2.0 * d0[0] * float(M.double().sum()))
            drift[f"compensated={comp}"] = {
                "E0": e0, "steps": steps_done, "s_per_step": t_s / steps_done,
                "max_rel_dE": max(abs(d[0] + d[1] - e0) / abs(e0) for _, d in hist),
                "final_rel_dE": (hist[-1][1][0] + hist[-1][1][1] - e0) / abs(e0),
                "max_dP_over_rms_momentum": max(float(np.linalg.norm(d[2:5] - d0[2:5])) / pscale
                                                for _, d in hist),
                "max_rel_dL": max(float(np.linalg.norm(d[5:8] - d0[5:8]) /
                                        max(np.linalg.norm(d0[5:8]), 1e-300)) for _, d in hist),
                "every": args.drift_every}
    finally:
        nb.nbody_destroy(ctx)
    th.join()

    import oracle
    bx, by, bz = ref["b"]
    table = []
    for r in rows:
        e = oracle.rel_err(*r.pop("a"), bx, by, bz)
        r.update(p50=oracle.percentile_nearest_rank(e, 50), p99=oracle.percentile_nearest_rank(e, 99),
                 max=float(e.max()))
        table.append(r)
    head = next(r for r in table if r["log2_delta_acc"] == -9 and r["compensated"] == 0
                and r["quadrupole"] == 0)
    ni = tg.size * n
    return {
        "metric": METRIC, "value": head["ginter_s"], "unit": UNIT, "n_gpus": 1,
        "steps": 1, "warmup": 2, "ms_per_step": head["walk_ms"], "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic (seeded three-component galaxy)",
        "config": {"workload": f"precision sweep: galaxy N={n}, delta_acc 2^-1..2^-{args.sweep_max}, "
                               f"plain vs compensated FP32 accumulation, error vs FP64 direct on "
                               f"{tg.size} seeded particles; {args.drift_steps} leapfrog steps "
                               f"dt=1/256 for the FP64 energy/momentum drift", "n": n},
        "sweep": table, "drift": drift,
        "cpu_baseline": {"value": ni / ref["s"] / 1e9, "unit": UNIT, "cores": ref["threads"],
                         "kind": "oracle",
                         "sample": f"FP64 direct summation (oracle) for {tg.size} targets over all "
                                   f"{n} particles ({ni} interactions), run beside the GPU sweep"},
    }


# ---------------------------------------------------------------------------- reference arm
def run_reference(args, rank, world):
    if rank != 0:
        return None
    import ics
    import oracle
    p = ics.galaxy(args.n, args.seed)
    x, y, z, m = (np.asarray(p[k], np.float64) for k in ("x", "y", "z", "m"))
    t0 = time.perf_counter()
    tree = oracle.Tree(x, y, z, m, 21, 16)
    build_s = time.perf_counter() - t0
    f, c = tree.groups(64)
    stride = 32  # each step walks a different 1/32 of the groups (~0.2 s on 16 cores at 2^23)
    warm = np.arange(0, f.size, stride)
    gx, gy, gz, _ = tree.walk_groups(warm, oracle.MAC_GROUP_GEO, 1.0, EPS, 0.0, 0.5, 64, None)
    a_old = np.nan_to_num(np.sqrt(gx ** 2 + gy ** 2 + gz ** 2), nan=1.0)
    for _ in range(args.warmup):
        tree.walk_groups(warm, oracle.MAC_GROUP_ACC, 1.0, EPS, DACC, 0.5, 64, a_old)
    total_i, total_s = 0, 0.0
    for k in range(args.steps):
        sel = np.arange(k % stride, f.size, stride)
        gx, gy, gz, _ = tree.walk_groups(sel, oracle.MAC_GROUP_GEO, 1.0, EPS, 0.0, 0.5, 64, None)
        ao = np.nan_to_num(np.sqrt(gx ** 2 + gy ** 2 + gz ** 2), nan=1.0)
        t1 = time.perf_counter()
        _, _, _, nint = tree.walk_groups(sel, oracle.MAC_GROUP_ACC, 1.0, EPS, DACC, 0.5, 64, ao)
        total_s += time.perf_counter() - t1
        total_i += int(nint[nint > 0].sum())
    value = total_i / total_s / 1e9
    sample = (f"FP64 oracle tree walk of 1/{stride} of the groups of the N={args.n} galaxy per "
              f"step (a different slice each step); oracle tree built once ({build_s:.2f} s)")
    return {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": total_s / args.steps * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic (seeded three-component galaxy)",
            "config": workload_config(args.n),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": oracle.threads(),
                             "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0},
            "oracle_build_s": build_s}


def main():
    args = parse()
    rank = int(os.environ.get("RANK", 0))
    world = int(os.environ.get("WORLD_SIZE", 1))
    local_rank = int(os.environ.get("LOCAL_RANK", 0))
    if args.impl == "reference":
        out = run_reference(args, rank, world)
    else:
        if world > 1:
            import torch
            import torch.distributed as dist
            torch.cuda.set_device(local_rank)
            dist.init_process_group("nccl")
        if args.workload == "batched":
            out = run_batched(args, rank, world, local_rank)
        elif args.workload == "learned":
            out = run_learned(args, rank, world, local_rank)
        elif args.workload == "precision":
            out = run_precision(args, rank, world, local_rank)
        elif args.workload == "scaling":
            out = run_scaling(args, rank, world, local_rank)
        else:
            out = run_ours(args, rank, world, local_rank)
        if world > 1:
            import torch.distributed as dist
            dist.destroy_process_group()
    if out is not None:
        print(json.dumps(out), flush=True)


if __name__ == "__main__":
    main()
