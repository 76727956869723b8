#!/usr/bin/env python
"""HGMM build + register throughput on one GB300 (or N independent replicas).

Workload (one "step"): two consecutive frames of a simulated 64-beam spinning
LiDAR (0.2 deg azimuth step, +-15 deg elevation, 100 m range, N(0, 0.02^2) m
range noise) in a seeded synthetic urban scene (ground, 20 boxes of 5-20 m,
30 poles); the second frame after 1 m of forward motion and <= 2 deg of yaw.
A step builds the depth-4 GMM tree (4680 nodes, 8 EM iterations per level)
of the first frame and registers the second frame to it with 30 rounds of
the adaptive E-step (Algorithm 1) and the Mahalanobis M-step (Eq. 9-16).

value   = (target points + source points) per second through build +
          register, Mpts/s, summed over ranks (each rank registers its own
          independently seeded pair: weak scaling, no collective on the path)
e2e     = the same metric through hgmm_register_pair_host with pinned host
          buffers: host->device copies of both clouds and the device->host
          read of T inside the timed region
roofline: the kernel with the largest share of device time, its average
          CUDA-event duration (library event profiler, same stream) against
          its algorithmic work per launch
batched: 256 independent pairs (2k-200k points, depth 3/4) in one persistent
          cluster launch, pairs/s against the plain path looped over a subset
cpu_baseline / --impl reference: the FP64 numpy oracle on the same
          workload (full frames, depth 4, 30 rounds): one pair on one core,
          and one independently seeded pair per host core at once.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

DEPTH = 4
ITERS = 30
WORKLOAD = "lidar64_consecutive_frames_depth4_30it"
METRIC = "HGMM build+register Mpts/s"
L2_FLUSH_BYTES = 512 << 20

# algorithmic work per processed point for each kernel of the path
# (bytes of DRAM traffic a perfect kernel needs, FP32 flops with FMA = 2)
KERNEL_WORK = {
    "estep": {"bytes": 16, "flops": 355, "unit": "target point"},
    "assign": {"bytes": 20, "flops": 160, "unit": "target point"},
    "scatter": {"bytes": 44, "flops": 0, "unit": "target point"},
    "register": {"bytes": 16, "flops": None, "unit": "source point"},
}
REGISTER_TRAFFIC_BYTES = 1966336
DESCEND_FLOPS_PER_LEVEL = 8 * 18 + 8 * 2 + 8  # 8 child scores, 8 exp2 + sum, rcp
DESCEND_FLOPS_FIXED = 18 + 12  # transform, fixed-point conversion


def _peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


# ---------------------------------------------------------------- clocks
class Clocks:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200", "-i", str(self.index)],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
            out, _ = self.proc.communicate()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------- oracle leg
# One worker process runs a list of jobs: it generates every job's pair first,
# then times the FP64 oracle's build + registration of each (one thread).
ORACLE_WORKER = r"""
import json, sys, time
sys.path.insert(0, {root!r})
import numpy as np
from oracle import hgmm_oracle as O
from paper_1807_02587_gb300 import synth
jobs = {jobs!r}
pairs = []
for job in jobs:
    if job[0] == "lidar":
        p, depth = synth.lidar_pair(job[1]), 4
    else:  # ("primitive", seed, n, max_deg, depth)
        p, depth = synth.primitive_pair(job[1], job[2], max_deg=job[3]), job[4]
    pairs.append((p["tgt"].astype(np.float32).astype(np.float64),
                  p["src"].astype(np.float32).astype(np.float64), depth))
out = []
for tgt, src, depth in pairs:
    t0 = time.time()
    tree = O.build_tree(tgt, O.Params(depth=depth))
    T = O.register(tree, src, iters={iters})
    t1 = time.time()
    out.append({{"n": int(tgt.shape[0] + src.shape[0]), "start": t0, "end": t1,
                 "T": T.reshape(-1).tolist()}})
print(json.dumps(out))
"""


def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def oracle_pool(jobs, workers):
    """Run the oracle jobs on `workers` single-threaded processes at once
    (fresh interpreters: nothing is forked from a process that holds a CUDA
    context).  Returns the per-job results in job order and the wall time
    of the compute (first start to last end, generation excluded)."""
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")
    workers = max(1, min(workers, len(jobs)))
    chunks = [list(range(k, len(jobs), workers)) for k in range(workers)]
    procs = []
    for idx in chunks:
        code = ORACLE_WORKER.format(root=ROOT, jobs=[jobs[i] for i in idx], iters=ITERS)
        procs.append(subprocess.Popen([sys.executable, "-c", code], stdout=subprocess.PIPE,
                                      stderr=subprocess.PIPE, text=True, env=env))
    res = [None] * len(jobs)
    for idx, pr in zip(chunks, procs):
        out, err = pr.communicate()
        if pr.returncode != 0:
            raise RuntimeError("oracle worker failed: " + err[-2000:])
        for i, r in zip(idx, json.loads(out.strip().splitlines()[-1])):
            res[i] = r
    wall = max(r["end"] for r in res) - min(r["start"] for r in res)
    return res, wall


def oracle_sample_desc(cores):
    return ("FP64 numpy oracle on the bench's own workload: full LiDAR frames (float32-rounded), "
            "depth-4 tree, 8 EM iterations per level, 30 registration rounds; "
            f"{cores} single-threaded process(es) at once, one independently seeded pair each")


def cpu_baseline(seed):
    """The oracle on the bench workload: one pair on one core, then one pair
    per host core at once (the path shards by pairs: all cores = that many
    independent pairs)."""
    one, wall1 = oracle_pool([("lidar", seed)], 1)
    cores = host_cores()
    many, wall = oracle_pool([("lidar", seed + k) for k in range(cores)], cores)
    n_all = sum(r["n"] for r in many)
    return {"value": n_all / wall / 1e6, "unit": "Mpts/s", "cores": cores, "kind": "oracle",
            "sample": oracle_sample_desc(cores), "seconds": wall,
            "single_core": {"value": one[0]["n"] / wall1 / 1e6, "unit": "Mpts/s", "cores": 1,
                            "seconds": wall1, "pairs": 1}}


def reference_main(args, rank, world):
    if rank != 0:
        return 0
    cores = host_cores()
    if args.warmup:
        oracle_pool([("lidar", args.seed + 1000 + k) for k in range(args.warmup)], cores)
    res, wall = oracle_pool([("lidar", args.seed + k) for k in range(args.steps)], cores)
    n_tot = sum(r["n"] for r in res)
    val = n_tot / wall / 1e6
    line = {
        "impl": "reference", "metric": METRIC, "value": val, "unit": "Mpts/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * wall / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": WORKLOAD, "points_per_step": n_tot / args.steps, "depth": DEPTH,
                   "reg_iters": ITERS, "host_processes": min(cores, args.steps)},
        "cpu_baseline": {"value": val, "unit": "Mpts/s", "cores": min(cores, args.steps), "kind": "oracle",
                         "sample": oracle_sample_desc(min(cores, args.steps))
                         + f"; {args.steps} timed pairs after {args.warmup} untimed"},
        "e2e": {"value": val, "unit": "Mpts/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------- ranks
def rank_seed(seed, rank):
    """Weak scaling: every rank registers its own LiDAR pair (no data-path
    collective; the ranks only meet to time and to add up their work)."""
    return seed + rank


def aggregate_over_ranks(points, ms, e2e_ms, world, device):
    """Whole-job figures: points summed over the ranks, step times (device
    and end to end) the maximum over the ranks."""
    if world == 1:
        return points, ms, e2e_ms
    import torch
    import torch.distributed as dist
    p = torch.tensor([points], dtype=torch.float64, device=device)
    dist.all_reduce(p, op=dist.ReduceOp.SUM)
    m = torch.tensor([ms, e2e_ms], dtype=torch.float64, device=device)
    dist.all_reduce(m, op=dist.ReduceOp.MAX)
    return float(p[0]), float(m[0]), float(m[1])


# ---------------------------------------------------------------- GPU leg
def gpu_main(args, rank, world, local_rank):
    import torch
    import torch.distributed as dist
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local_rank)
    from paper_1807_02587_gb300 import binding as B
    from paper_1807_02587_gb300 import synth

    pair = synth.lidar_pair(rank_seed(args.seed, rank))
    tgt4 = synth.to_float4(pair["tgt"])
    src4 = synth.to_float4(pair["src"])
    n_t, n_s = tgt4.shape[0], src4.shape[0]
    tgt = torch.from_numpy(tgt4).cuda()
    src = torch.from_numpy(src4).cuda()
    tree = B.Tree(max(n_t, n_s), DEPTH)
    prm = B.params(flags=B.HGMM_FLAG_EM_COOPERATIVE if args.em_cooperative else 0)
    s = torch.cuda.Stream()
    T_out = torch.zeros((4, 4), dtype=torch.float64, device="cuda")

    def step():
        tree.build(tgt, DEPTH, prm, stream=s)
        tree.register(src, None, ITERS, stream=s, T_out=T_out)

    # correctness gate + warm-up (eager)
    step()
    tree.sync(s)
    T0 = T_out.cpu().numpy().copy()
    for _ in range(args.warmup):
        step()
    tree.sync(s)
    if args.ncu:
        # plain eager steps for an external profiler's launch list; no timing
        for _ in range(args.steps):
            step()
        tree.sync(s)
        print(json.dumps({"ncu_mode": True, "launches_per_step_expected": None}))
        return 0
    # per-kernel profile of two eager steps (event pairs around every launch)
    tree.profile(True)
    step()
    step()
    prof = tree.profile_read()
    tree.profile(False)
    launches_per_step = sum(c for _, c in prof.values()) // 2

    graph = None
    graph_note = "disabled"
    if not args.no_graph:
        try:
            graph = torch.cuda.CUDAGraph()
            with torch.cuda.graph(graph, stream=s):
                step()
            graph_note = "captured"
        except Exception as e:  # capture unsupported: time eager launches
            graph = None
            graph_note = f"capture failed ({type(e).__name__}: {str(e)[:120]}), eager launches"
            torch.cuda.synchronize()
    if graph is not None:
        T_out.zero_()
        torch.cuda.synchronize()
        with torch.cuda.stream(s):
            for _ in range(2):
                graph.replay()
        torch.cuda.synchronize()
        assert np.allclose(T_out.cpu().numpy(), T0, atol=1e-9), "graph replay changed the result"

    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device="cuda")
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    clocks = Clocks(local_rank)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    time.sleep(0.3)
    for k in range(args.steps):
        with torch.cuda.stream(s):
            flush.zero_()
        starts[k].record(s)
        with torch.cuda.stream(s):
            if graph is not None:
                graph.replay()
            else:
                step()
        ends[k].record(s)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    clk = clocks.stop()
    tree.sync(s)
    ms = [a.elapsed_time(b) for a, b in zip(starts, ends)]
    ms_step = float(np.mean(ms))

    # end to end through the host-buffer entry point
    tgt_h = torch.from_numpy(tgt4).pin_memory()
    src_h = torch.from_numpy(src4).pin_memory()
    for _ in range(2):
        B.hgmm_register_pair_host(tree.handle, tgt_h, src_h, DEPTH, prm, None, ITERS, stream=s)
    e2e_ms = []
    for _ in range(args.steps):
        with torch.cuda.stream(s):
            flush.zero_()
        s.synchronize()
        t0 = time.perf_counter()
        T_h = B.hgmm_register_pair_host(tree.handle, tgt_h, src_h, DEPTH, prm, None, ITERS, stream=s)
        e2e_ms.append(1e3 * (time.perf_counter() - t0))
    e2e_step = float(np.mean(e2e_ms))

    pts_tot, ms_max, e2e_max = aggregate_over_ranks(float(n_t + n_s), ms_step, e2e_step, world, "cuda")
    if rank != 0:
        dist.destroy_process_group()
        return 0

    # roofline of the dominant kernel
    hbm_peak, peak_kind = _peaks()
    sm_count = torch.cuda.get_device_properties(0).multi_processor_count
    clk_mhz = clk["sm_mhz"] or 2070.0
    fp32_peak_tflops = sm_count * 128 * 2 * clk_mhz * 1e6 / 1e12
    dom = max(prof, key=lambda k: prof[k][0])
    dom_ms = prof[dom][0] / max(prof[dom][1], 1)
    total_prof = sum(v[0] for v in prof.values())
    kernels = {k: {"ms_total_2steps": round(v[0], 4), "launches_2steps": v[1],
                   "share": round(v[0] / total_prof, 4)} for k, v in prof.items() if v[1]}
    roof = {"kernel": dom, "avg_launch_us": dom_ms * 1e3}
    work = KERNEL_WORK.get(dom)
    units = n_t if (work and work["unit"] == "target point") else n_s
    if dom == "register":
        # one launch runs all ITERS rounds of Algorithm 1 + the M-step
        lv = _descend_levels(B, tree, src4, DEPTH)
        flops_pt = DESCEND_FLOPS_FIXED + DESCEND_FLOPS_PER_LEVEL * lv
        units = n_s * ITERS
        roof.update(bound="alu", achieved=flops_pt * units / (dom_ms / 1e3) / 1e12,
                    peak=fp32_peak_tflops, unit="TFLOP/s",
                    note=f"FP32 flops/point {flops_pt:.0f} (avg {lv:.2f} levels visited); "
                         f"peak = {sm_count} SM x 128 lanes x 2 x {clk_mhz:.0f} MHz")
    elif work is not None and work["flops"] and \
            work["flops"] / work["bytes"] > fp32_peak_tflops * 1e12 / (hbm_peak * 1e9):
        roof.update(bound="alu", achieved=work["flops"] * units / (dom_ms / 1e3) / 1e12,
                    peak=fp32_peak_tflops, unit="TFLOP/s",
                    note=f"FP32 flops/point {work['flops']}; peak = {sm_count} SM x 128 x 2 x "
                         f"{clk_mhz:.0f} MHz")
    elif work is not None:
        roof.update(bound="hbm", achieved=work["bytes"] * units / (dom_ms / 1e3) / 1e9,
                    peak=hbm_peak, unit="GB/s", note=f"{peak_kind} HBM copy bandwidth")
    else:
        roof.update(bound="alu", achieved=None, peak=None, unit=None,
                    note="no algorithmic model for this kernel")
    if roof.get("achieved") is not None:
        roof["frac"] = roof["achieved"] / roof["peak"]
    # DRAM bytes (read + write) of one k_register launch on this workload, from
    # an ncu capture of the kernel as it is built now (None for other kernels)
    roof["traffic"] = REGISTER_TRAFFIC_BYTES if dom == "register" else None
    hbm_equiv = None
    if dom in KERNEL_WORK:
        hbm_equiv = KERNEL_WORK[dom]["bytes"] * units / (dom_ms / 1e3) / 1e9
    roof["hbm_gbs_equivalent"] = hbm_equiv

    configs = configs_section(args, B, synth, torch, prm)
    batched = None
    if not args.no_batched:
        batched = batched_section(args, B, synth, torch, prm)
    learned = None
    if not args.no_learned:
        learned = learned_section(args, B, torch)
    large = None
    if not args.no_large_build:
        large = large_build_section(args, B, torch)
    odometry = None
    if not args.no_odometry:
        odometry = odometry_section(args, B, torch)
    variants = None
    if not args.no_variants:
        variants = variants_section(args, B, torch, pair, tgt, src, fp32_peak_tflops)

    cpu = None
    if world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(args.seed)

    c = (np.trace(T0[:3, :3].T @ pair["T_gt"][:3, :3]) - 1.0) / 2.0
    rot_err = float(np.degrees(np.arccos(np.clip(c, -1.0, 1.0))))
    line = {
        "metric": METRIC, "value": pts_tot / (ms_max / 1e3) / 1e6, "unit": "Mpts/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_max,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": WORKLOAD, "n_target": n_t, "n_source": n_s, "depth": DEPTH,
                   "J": 8, "em_iters": prm.em_iters, "reg_iters": ITERS,
                   "l2": f"flushed between steps ({L2_FLUSH_BYTES >> 20} MB write)",
                   "cuda_graph": graph_note, "parallelism": f"replicas{world}"},
        "pairs_per_s": world / (ms_max / 1e3),
        "e2e": {"value": pts_tot / (e2e_max / 1e3) / 1e6, "unit": "Mpts/s",
                "h2d_bytes_per_step": int(16 * (n_t + n_s)), "d2h_bytes_per_step": 128,
                "ms_per_step": e2e_max},
        "gpu_launches": int(launches_per_step * args.steps),
        "launches_per_step": int(launches_per_step),
        "roofline": roof,
        "kernels": kernels,
        "configs": configs,
        "batched": batched,
        "learned": learned,
        "large_build": large,
        "odometry": odometry,
        "variants": variants,
        "cpu_baseline": cpu,
        "clocks": clk,
        "accuracy": {"rot_err_deg_vs_truth": rot_err,
                     "trans_err_m_vs_truth": float(np.linalg.norm(T0[:3, 3] - pair["T_gt"][:3, 3])),
                     "e2e_equals_device_path": bool(np.array_equal(T_h, T0))},
    }
    print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()
    return 0


def batched_section(args, B, synth, torch, prm):
    """Batched form on 256 plane/box/sphere pairs (2k-200k points, depth 3
    or 4, rotations <= 30 deg): pairs/s of the single persistent cluster
    launch against looping the plain single-pair path over a subset."""
    pairs = synth.batched_pairs(args.seed + 100, count=args.batch_pairs)
    tb = [synth.to_float4(p["tgt"]) for p in pairs]
    sb = [synth.to_float4(p["src"]) for p in pairs]
    t_off = np.concatenate([[0], np.cumsum([x.shape[0] for x in tb])]).astype(np.int64)
    s_off = (np.concatenate([[0], np.cumsum([x.shape[0] for x in sb])]) + t_off[-1]).astype(np.int64)
    depths = [p["depth"] for p in pairs]
    n = len(pairs)
    pts = torch.from_numpy(np.concatenate(tb + sb)).cuda()
    maxn = int(max(np.diff(t_off).max(), np.diff(s_off).max()))
    bat = B.Batch(maxn, 4, n)
    B.hgmm_batch_plan(bat.handle, t_off, s_off, depths)
    s = torch.cuda.Stream()
    T = torch.zeros((n, 16), dtype=torch.float64, device="cuda")
    st = torch.zeros(n, dtype=torch.int32, device="cuda")
    with torch.cuda.stream(s):
        tune_ms = B.hgmm_batch_autotune(bat.handle, pts, T, prm, None, ITERS, stream=s)
    shape, clusters = B.hgmm_batch_get_shape(bat.handle)
    build_shape, build_ms = B.hgmm_batch_get_build_shape(bat.handle)

    def run():
        B.hgmm_batch_register(bat.handle, pts, T, prm, None, ITERS, stream=s, pair_status=st)

    graph = torch.cuda.CUDAGraph()
    note = "captured"
    try:
        with torch.cuda.graph(graph, stream=s):
            run()
    except Exception as e:
        graph, note = None, f"capture failed ({type(e).__name__}), eager"
        torch.cuda.synchronize()
    for _ in range(2):
        with torch.cuda.stream(s):
            graph.replay() if graph is not None else run()
    torch.cuda.synchronize()
    e0 = [torch.cuda.Event(enable_timing=True) for _ in range(args.batch_steps)]
    e1 = [torch.cuda.Event(enable_timing=True) for _ in range(args.batch_steps)]
    for k in range(args.batch_steps):
        e0[k].record(s)
        with torch.cuda.stream(s):
            graph.replay() if graph is not None else run()
        e1[k].record(s)
    torch.cuda.synchronize()
    ms = float(np.mean([a.elapsed_time(b) for a, b in zip(e0, e1)]))
    Tb = T.cpu().numpy().reshape(n, 4, 4)
    status = st.cpu().numpy()

    def rot_err(Ta, Tb_):
        c = (np.trace(Ta[:3, :3].T @ Tb_[:3, :3]) - 1.0) / 2.0
        return float(np.degrees(np.arccos(np.clip(c, -1.0, 1.0))))

    ok_b = [rot_err(Tb[i], p["T_gt"]) <= 0.1 for i, p in enumerate(pairs)]
    # the plain path, one pair after another on one stream, over a subset
    sub = list(range(0, n, max(1, n // args.plain_pairs)))[: args.plain_pairs]
    tree = B.Tree(maxn, 4)
    outs = [torch.zeros((4, 4), dtype=torch.float64, device="cuda") for _ in sub]

    def plain():
        for j, i in enumerate(sub):
            tree.build(pts[t_off[i]:t_off[i + 1]], depths[i], prm, stream=s)
            tree.register(pts[s_off[i]:s_off[i + 1]], None, ITERS, stream=s, T_out=outs[j])

    with torch.cuda.stream(s):
        plain()
    torch.cuda.synchronize()
    a0 = torch.cuda.Event(enable_timing=True)
    a1 = torch.cuda.Event(enable_timing=True)
    a0.record(s)
    with torch.cuda.stream(s):
        plain()
    a1.record(s)
    torch.cuda.synchronize()
    plain_ms = a0.elapsed_time(a1)
    agree = np.array([rot_err(outs[j].cpu().numpy(), Tb[i]) for j, i in enumerate(sub)])
    ok_p = [rot_err(outs[j].cpu().numpy(), pairs[i]["T_gt"]) <= 0.1 for j, i in enumerate(sub)]
    ok_b_sub = np.array([ok_b[i] for i in sub])
    out = {
        "pairs": n, "points_per_side": int(t_off[-1]), "pairs_per_s": n / (ms / 1e3),
        "pairs_le_0p1deg_per_s": float(np.sum(ok_b)) / (ms / 1e3),
        "ms_per_batch": ms, "cluster_ctas": shape, "clusters": clusters,
        "autotune_ms_by_cluster_ctas_1_2_4_8": tune_ms, "graph": note,
        "build_shape_by_bucket": {f"bucket{k}_{lab}": {"warp_item_parents": int(build_shape[k][0]),
                                                       "mstep_cta_runs": int(build_shape[k][1]),
                                                       "offsets_cta_items": int(build_shape[k][2])}
                                  for k, lab in enumerate(("tgt_lt_20k", "tgt_20k_80k", "tgt_ge_80k"))},
        "autotune_ms_default_vs_tuned_build_shape": build_ms,
        "plain_pairs_per_s": len(sub) / (plain_ms / 1e3), "plain_subset": len(sub),
        "plain_pairs_le_0p1deg_per_s": float(np.sum(ok_p)) / (plain_ms / 1e3),
        "speedup_vs_plain": (n / (ms / 1e3)) / (len(sub) / (plain_ms / 1e3)),
        "success_rate_le_0p1deg": float(np.mean(ok_b)),
        "success_rate_le_0p1deg_subset": float(np.mean(ok_b_sub)),
        "plain_success_rate_le_0p1deg_subset": float(np.mean(ok_p)),
        "agree_with_plain_within_0p01deg_subset": float(np.mean(agree < 0.01)),
        "disagree_with_plain_gt_0p01deg_subset": int(np.sum(agree >= 0.01)),
        "pair_status_nonzero": int(np.sum(status != 0)),
    }
    if not args.no_cpu_baseline:
        # the FP64 oracle (build + register, free-running) on the same subset,
        # one pair per host process at once
        jobs = [("primitive", int(pairs[i]["seed"]), int(pairs[i]["src"].shape[0]), 30.0, depths[i])
                for i in sub]
        res, wall = oracle_pool(jobs, host_cores())
        To = [np.array(r["T"]).reshape(4, 4) for r in res]
        ok_o = np.array([rot_err(To[j], pairs[i]["T_gt"]) <= 0.1 for j, i in enumerate(sub)])
        vs_o = np.array([rot_err(To[j], Tb[i]) for j, i in enumerate(sub)])
        out["oracle_subset"] = {
            "success_rate_le_0p1deg": float(np.mean(ok_o)),
            "batched_within_0p01deg_of_oracle": float(np.mean(vs_o < 0.01)),
            "batched_within_0p01deg_of_oracle_where_oracle_succeeds":
                float(np.mean(vs_o[ok_o] < 0.01)) if ok_o.any() else None,
            "batched_vs_plain_disagreements_where_oracle_succeeds": int(np.sum((agree >= 0.01) & ok_o)),
            "host_processes": min(host_cores(), len(jobs)), "seconds": wall}
    return out


def configs_section(args, B, synth, torch, prm):
    """The other single-pair configurations, timed like the main step (CUDA
    graph of build + 30 rounds, L2 flushed between steps): the 10k-point
    corner scene at depth 3 (rotation <= 30 deg, t <= 0.1) and the
    640 x 480 structured-light depth pair at depth 4."""
    out = {}
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device="cuda")
    for key, pair, depth in (("corner10k_depth3_30it", synth.corner_pair(args.seed), 3),
                             ("depth640x480_depth4_30it", synth.depth_pair(args.seed), 4)):
        tgt = torch.from_numpy(synth.to_float4(pair["tgt"])).cuda()
        src = torch.from_numpy(synth.to_float4(pair["src"])).cuda()
        n_t, n_s = int(tgt.shape[0]), int(src.shape[0])
        tree = B.Tree(max(n_t, n_s), depth)
        s = torch.cuda.Stream()
        T_out = torch.zeros((4, 4), dtype=torch.float64, device="cuda")

        def step():
            tree.build(tgt, depth, prm, stream=s)
            tree.register(src, None, ITERS, stream=s, T_out=T_out)

        for _ in range(3):
            step()
        tree.sync(s)
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph, stream=s):
            step()
        reps = 10
        e0 = [torch.cuda.Event(enable_timing=True) for _ in range(reps)]
        e1 = [torch.cuda.Event(enable_timing=True) for _ in range(reps)]
        for k in range(reps):
            with torch.cuda.stream(s):
                flush.zero_()
            e0[k].record(s)
            with torch.cuda.stream(s):
                graph.replay()
            e1[k].record(s)
        torch.cuda.synchronize()
        tree.sync(s)
        ms = float(np.mean([a.elapsed_time(b) for a, b in zip(e0, e1)]))
        T = T_out.cpu().numpy()
        out[key] = {"n_target": n_t, "n_source": n_s, "depth": depth, "ms_per_pair": ms,
                    "mpts_per_s": (n_t + n_s) / (ms / 1e3) / 1e6,
                    "rot_err_deg_vs_truth": _rot_err(T[:3, :3], pair["T_gt"][:3, :3])}
    return out


# algorithmic FLOPs of the proposal network per pair (1280 -> 256 -> 256 -> 9)
MLP_FWD_FLOPS = 2 * (1280 * 256 + 256 * 256 + 256 * 9)
MLP_BWD_FLOPS = 2 * (256 * 9 + 9 * 256 + 256 * 256 + 256 * 256 + 256 * 1280)


def odometry_section(args, B, torch):
    """Frame-to-frame odometry over a LiDAR drive (each frame's tree is the
    model of the next frame, three yaw starts per frame): frames/s with the
    build of frame k overlapped with the registration of frame k on a second
    stream and without, and the trajectory's drift for the default lambda_c
    with three starts and with the constant-velocity start alone, and for
    lambda_c = 0."""
    from paper_1807_02587_gb300 import synth
    from paper_1807_02587_gb300.odometry import Odometry, chain
    seq = synth.lidar_sequence(args.seed + 11, frames=args.odometry_frames)
    dev = [torch.from_numpy(synth.to_float4(f)).cuda() for f in seq["frames"]]
    n = max(d.shape[0] for d in dev)
    F = len(dev)
    W_gt = np.linalg.inv(seq["W"][0]) @ seq["W"]
    path = float(np.sum(np.linalg.norm(np.diff(W_gt[:, :3, 3], axis=0), axis=1)))
    out = {"frames": F, "points_per_frame": int(np.mean([d.shape[0] for d in dev])), "path_m": path}
    for overlap in (True, False):
        odo = Odometry(n, depth=DEPTH, iters=ITERS, overlap=overlap)
        odo.run(dev)
        odo.sync()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        T = odo.run(dev)
        odo.sync()
        torch.cuda.synchronize()
        out["frames_per_s_overlap" if overlap else "frames_per_s_sequential"] = F / (time.perf_counter() - t0)
    for lam, yaws, key in ((None, (0.0, 3.0, -3.0), "default_lam_c"), (None, (0.0,), "default_lam_c_one_start"),
                           (0.0, (0.0, 3.0, -3.0), "lam_c_0")):
        prm = B.params(lam_c=lam) if lam is not None else None
        odo = Odometry(n, depth=DEPTH, iters=ITERS, prm=prm, yaw_starts_deg=yaws)
        T = odo.run(dev)
        odo.sync()
        Tn = T.cpu().numpy()
        W = chain(Tn)
        per = np.array([[_rot_err(Tn[k, :3, :3], seq["T_rel"][k][:3, :3]),
                         float(np.linalg.norm(Tn[k, :3, 3] - seq["T_rel"][k][:3, 3]))] for k in range(1, F)])
        out[key] = {"final_trans_err_m": float(np.linalg.norm(W[-1, :3, 3] - W_gt[-1, :3, 3])),
                    "final_rot_err_deg": _rot_err(W[-1, :3, :3], W_gt[-1, :3, :3]),
                    "per_frame_rot_err_deg_median": float(np.median(per[:, 0])),
                    "per_frame_trans_err_m_median": float(np.median(per[:, 1])),
                    "frames_rot_err_over_1deg": int(np.sum(per[:, 0] > 1.0))}
    return out


# FP32 operations per (point, component) pair and round of the flat
# registration: the score (3 sub, 15 for the triangular W (z - mu) and its
# squared norm) twice, the running log-sum (max, exp2, add), gamma (sub,
# exp2) and its four moments (add, 3 FMA)
FLAT_FLOPS_PER_PAIR = 2 * 18 + 3 + 2 + 7


def variants_section(args, B, torch, pair, tgt, src, fp32_peak_tflops):
    """Sec. 5's variants on the bench's LiDAR pair (depth 4, 30 rounds, tree
    built once): Adaptive (lambda_c = 0.01), GMM-Tree (lambda_c = 0), the
    descent variants of Sec. 4.1 (path-product gamma; multi-path descent
    pruned at tau), the full Eq. 7 M-step (scatter kept) and the flat GMM J=n (the tree's leaves; and after 4 EM
    iterations over all J):
    registration time (CUDA events, median of 3), error against the known
    motion, and for the flat model its (point, component) pair rate against
    the FP32 peak."""
    n = int(max(tgt.shape[0], src.shape[0]))
    tree = B.Tree(n, DEPTH)
    tree.build(tgt, DEPTH)
    tree.sync()
    extent = tree.root()["extent"]
    T_gt = pair["T_gt"]
    out = {"workload": WORKLOAD, "depth": DEPTH, "reg_iters": ITERS}

    def timed(fn, reps=3):
        s = torch.cuda.current_stream()
        ts = []
        res = None
        for _ in range(reps):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(s)
            res = fn()
            b.record(s)
            b.synchronize()
            ts.append(a.elapsed_time(b))
        return float(np.median(ts)), res

    def errs(T):
        T = T.cpu().numpy()
        return {"rot_err_deg": _rot_err(T[:3, :3], T_gt[:3, :3]),
                "trans_err_m": float(np.linalg.norm(T[:3, 3] - T_gt[:3, 3]))}

    for lam, key in ((-1.0, "adaptive"), (0.0, "gmm_tree")):
        ms, T = timed(lambda: tree.register(src, iters=ITERS, lam_c=lam))
        tree.sync()
        out[key] = {"ms": ms, **errs(T)}
    # descent variants (Sec. 4.1): path-product gamma, threshold-pruned paths
    for mode, tau, full, key in ((1, 0.0, False, "ml_path_product_gamma"), (2, 0.01, False, "multipath_tau_0.01"),
                                 (2, 0.1, False, "multipath_tau_0.1"), (0, 0.0, True, "full_eq7"),
                                 (0, 0.0, False, "algorithm1_via_variant_kernel")):
        ms, T = timed(lambda: tree.register_descent(src, mode, tau, iters=ITERS, full_eq7=full))
        tree.sync()
        out[key] = {"ms": ms, **errs(T)}
    flat = B.Flat(n, int(B.hgmm_node_count(DEPTH)))
    for em, key in ((0, "flat_leaves"), (4, "flat_em4")):
        flat.from_tree(tree)
        fit_ms, _ = timed(lambda: flat.fit(tgt, em), reps=1) if em else (0.0, None)
        flat.sync()
        J = flat.export()["J"]
        ms, T = timed(lambda: flat.register(src, iters=ITERS))
        flat.sync()
        pairs = float(src.shape[0]) * J * ITERS
        out[key] = {"J": J, "ms": ms, "fit_ms": fit_ms, **errs(T),
                    "point_component_pairs_per_s": pairs / (ms / 1e3),
                    "achieved_tflops": pairs * FLAT_FLOPS_PER_PAIR / (ms / 1e3) / 1e12,
                    "frac_of_fp32_peak": pairs * FLAT_FLOPS_PER_PAIR / (ms / 1e3) / 1e12 / fp32_peak_tflops}
    return out


def _rot_err(Ra, Rb):
    c = (np.trace(Ra.T @ Rb) - 1.0) / 2.0
    return float(np.degrees(np.arccos(np.clip(c, -1.0, 1.0))))


def large_cloud(n, seed):
    """An n-point plane/box/sphere cloud (float4 on the device), sampled on
    the host in eight chunks."""
    import torch
    from paper_1807_02587_gb300 import synth
    scene = synth.primitive_scene(synth.make_rng(seed + 1))
    parts = [synth._sample_primitives(synth.make_rng(seed + 10 + k), scene, n // 8, 0.005) for k in range(8)]
    return torch.from_numpy(synth.to_float4(np.concatenate(parts))).cuda()


def large_build_section(args, B, torch):
    """The build on a cloud far larger than L2 (HBM-resident points): the
    E-step's achieved point-read bandwidth against the measured HBM peak and
    its FP32 rate against the ALU peak, from the event profile of one build."""
    dev = large_cloud(args.large_points, args.seed)
    n = int(dev.shape[0])
    tree = B.Tree(n, 4)
    tree.build(dev, 4)
    tree.sync()
    tree.profile(True)
    tree.build(dev, 4)
    tree.sync()
    prof = tree.profile_read()
    tree.profile(False)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    tree.build(dev, 4)
    e1.record()
    tree.sync()
    es_ms, es_n = prof["estep"]
    per = es_ms / max(es_n, 1) / 1e3
    hbm, kind = _peaks()
    sm_count = torch.cuda.get_device_properties(0).multi_processor_count
    alu = sm_count * 128 * 2 * 2070e6 / 1e12
    # registration at this size: the cloud itself moved by a known motion
    # (2 degrees, 1 % of the extent), 10 rounds against its tree
    from paper_1807_02587_gb300 import synth
    extent = tree.root()["extent"]
    T_gt = synth.rigid(synth.axis_angle_matrix([1.0, -2.0, 3.0], np.deg2rad(2.0)), np.full(3, 0.01 * extent / np.sqrt(3)))
    Ti = torch.from_numpy(np.linalg.inv(T_gt)).to(device="cuda", dtype=torch.float32)
    src = dev.clone()
    src[:, :3] = dev[:, :3] @ Ti[:3, :3].T + Ti[:3, 3]
    iters = 10
    tree.register(src, iters=iters)
    tree.sync()
    r0, r1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    r0.record()
    T = tree.register(src, iters=iters)
    r1.record()
    tree.sync()
    reg_ms = r0.elapsed_time(r1)
    T = T.cpu().numpy()
    m = tree.reg_moments()  # levels visited: node depth of each point's last round
    lv = 1.0
    if m.size:
        offs = np.cumsum([0] + [8 ** (l + 1) for l in range(4)])
        w = np.array([m[offs[l]:offs[l + 1], 0].sum() for l in range(4)])
        lv = float((w * np.arange(1, 5)).sum() / max(w.sum(), 1e-30))
    flops_pt = 30 + 168 * lv
    register = {"rounds": iters, "ms": reg_ms, "us_per_round": reg_ms * 1e3 / iters,
                "gpts_per_s_per_round": n * iters / (reg_ms / 1e3) / 1e9,
                "point_read_GBps": 16 * n * iters / (reg_ms / 1e3) / 1e9,
                "levels_visited": lv, "fp32_TFLOPs": flops_pt * n * iters / (reg_ms / 1e3) / 1e12,
                "fp32_frac": flops_pt * n * iters / (reg_ms / 1e3) / 1e12 / alu,
                "rot_err_deg_vs_truth": _rot_err(T[:3, :3], T_gt[:3, :3]),
                "trans_err_rel_extent": float(np.linalg.norm(T[:3, 3] - T_gt[:3, 3]) / extent)}
    return {"points": n, "depth": 4, "build_ms": e0.elapsed_time(e1), "register": register,
            "estep_launches": es_n, "estep_us_per_launch": per * 1e6,
            "estep_point_read_GBps": 16 * n / per / 1e9, "hbm_peak_GBps": hbm, "peak_kind": kind,
            "estep_hbm_frac": 16 * n / per / 1e9 / hbm,
            "estep_TFLOPs": KERNEL_WORK["estep"]["flops"] * n / per / 1e12 if KERNEL_WORK["estep"]["flops"] else None,
            "fp32_peak_TFLOPs": alu,
            "kernels_ms": {k: round(v[0], 3) for k, v in prof.items() if v[1]}}


def learned_section(args, B, torch):
    """Learned pose proposal: the shipped network (trained on 100k pairs by
    paper_1807_02587_gb300.train_proposal) proposes, the plain method refines
    at depth 4 with the identity start as fallback; success (<= 0.1 deg) and
    pairs/s against the plain method from the identity on held-out pairs with
    SO(3)-uniform rotations.  Plus the network's tensor-core throughput."""
    from paper_1807_02587_gb300 import proposal as P
    path = os.path.join(ROOT, "paper_1807_02587_gb300", "weights", "proposal_mlp.npz")
    if not os.path.exists(path):
        return {"skipped": "no trained weights at paper_1807_02587_gb300/weights/proposal_mlp.npz"}
    params = np.load(path)["params"]
    big = 8192
    net = B.Mlp(big)
    B.hgmm_mlp_set_params(net.handle, params)
    ts = P.so3_test_pairs(args.seed + 31337, args.learned_pairs, args.learned_points)
    res = P.evaluate(net, ts, depth=4, iters=30, reps=3)
    # the network alone: one forward of a large batch, and one training step
    x = torch.randn((big, 1280), device="cuda").to(torch.bfloat16)
    y = torch.zeros((big, 9), dtype=torch.float32, device="cuda")
    lab = torch.zeros((big, 12), dtype=torch.float32, device="cuda")
    lab[:, [0, 4, 8]] = 1.0

    def timed(fn, reps=20):
        for _ in range(3):
            fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            fn()
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps / 1e3

    t_fwd = timed(lambda: B.hgmm_mlp_forward(net.handle, x, y))
    tb = 1024
    t_train = timed(lambda: B.hgmm_mlp_train_step(net.handle, x, lab, tb, lr=0.0))
    B.hgmm_mlp_set_params(net.handle, params)  # lr 0 left them unchanged; reset Adam state anyway
    bf16_peak = _bf16_peak()
    fwd_tf = MLP_FWD_FLOPS * big / t_fwd / 1e12
    res.update({
        "weights": "paper_1807_02587_gb300/weights/proposal_mlp.npz (train_proposal, 100k pairs)",
        "test_points": args.learned_points,
        "mlp": {"forward_batch": big, "forward_us": t_fwd * 1e6, "forward_tflops": fwd_tf,
                "train_step_batch": tb, "train_step_us": t_train * 1e6,
                "train_step_tflops": (MLP_FWD_FLOPS + MLP_BWD_FLOPS) * tb / t_train / 1e12,
                "bf16_peak_tflops": bf16_peak[0], "peak_kind": bf16_peak[1],
                "forward_frac": fwd_tf / bf16_peak[0]},
    })
    return res


def _bf16_peak():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            return float(json.load(f)["bf16_tflops"]), "measured burst (cuBLAS bf16)"
    return 1900.0, "fallback"


def _descend_levels(B, tree, src4, depth):
    """Average number of tree levels the descent visits per source point in
    the last round (from the association levels of the exported moments)."""
    m = tree.reg_moments()
    sizes = [8 ** (l + 1) for l in range(depth)]
    offs = np.cumsum([0] + sizes)
    mass = np.array([m[offs[l]:offs[l + 1], 0].sum() for l in range(depth)])
    if mass.sum() <= 0:
        return float(depth)
    return float(np.sum(mass * (np.arange(depth) + 1)) / mass.sum())


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["gpu", "reference"], default="gpu")
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--no-graph", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-batched", action="store_true")
    ap.add_argument("--batch-pairs", type=int, default=256)
    ap.add_argument("--batch-steps", type=int, default=3)
    ap.add_argument("--plain-pairs", type=int, default=32)
    ap.add_argument("--no-learned", action="store_true")
    ap.add_argument("--learned-pairs", type=int, default=256)
    ap.add_argument("--learned-points", type=int, default=50000)
    ap.add_argument("--profile-build", type=int, default=0, metavar="N",
                    help="only build the depth-4 tree of an N-point plane/box/sphere cloud 3 times, "
                         "for a profiler")
    ap.add_argument("--profile-register", type=int, default=0, metavar="N",
                    help="only register the N-point cloud, moved as in the large-build section, to its "
                         "depth-4 tree 3 times (10 rounds each), for a profiler")
    ap.add_argument("--no-large-build", action="store_true")
    ap.add_argument("--no-odometry", action="store_true")
    ap.add_argument("--no-variants", action="store_true")
    ap.add_argument("--em-cooperative", action="store_true",
                    help="build EM of each level in one cooperative launch (default: launches per iteration)")
    ap.add_argument("--profile-variants", action="store_true",
                    help="plain launches of the flat, multi-path and full Eq. 7 variants for a profiler")
    ap.add_argument("--odometry-frames", type=int, default=20)
    ap.add_argument("--large-points", type=int, default=16_000_000)
    ap.add_argument("--profile-mlp", action="store_true",
                    help="only run the proposal network (5 forwards of 8192 pairs, 3 training "
                         "steps of 1024), for a profiler")
    ap.add_argument("--profile-batch", type=int, default=0, metavar="P",
                    help="only run the batched launch on the first P pairs of the batched workload "
                         "(2 launches: warm-up, then the one to capture), for a profiler")
    ap.add_argument("--ncu", action="store_true",
                    help="only run warm-up + eager steps (for an ncu launch list)")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        return reference_main(args, rank, world)
    if args.profile_mlp:
        return profile_mlp_main()
    if args.profile_batch:
        return profile_batch_main(args)
    if args.profile_variants:
        return profile_variants_main(args)
    if args.profile_build:
        import torch
        from paper_1807_02587_gb300 import binding as B
        dev = large_cloud(args.profile_build, args.seed)
        tree = B.Tree(dev.shape[0], 4)
        for _ in range(3):
            tree.build(dev, 4)
        tree.sync()
        print(json.dumps({"profile_build": True, "points": int(dev.shape[0])}))
        return 0
    if args.profile_register:
        return profile_register_main(args)
    return gpu_main(args, rank, world, local_rank)


def profile_register_main(args):
    """Registration of a large cloud for an external profiler: the N-point
    plane/box/sphere cloud moved by the large-build section's motion (2
    degrees, 1 % of the extent), registered to its depth-4 tree 3 times with
    10 rounds.  A source of 2^20 points or more takes two k_register launches
    per call (the one-round launch that records the nodes, then the other
    nine rounds on the reordered source)."""
    import torch
    from paper_1807_02587_gb300 import binding as B
    from paper_1807_02587_gb300 import synth
    dev = large_cloud(args.profile_register, args.seed)
    n = int(dev.shape[0])
    tree = B.Tree(n, 4)
    tree.build(dev, 4)
    extent = tree.root()["extent"]
    T_gt = synth.rigid(synth.axis_angle_matrix([1.0, -2.0, 3.0], np.deg2rad(2.0)),
                       np.full(3, 0.01 * extent / np.sqrt(3)))
    Ti = torch.from_numpy(np.linalg.inv(T_gt)).to(device="cuda", dtype=torch.float32)
    src = dev.clone()
    src[:, :3] = dev[:, :3] @ Ti[:3, :3].T + Ti[:3, 3]
    for _ in range(3):
        T = tree.register(src, iters=10)
    tree.sync()
    T = T.cpu().numpy()
    print(json.dumps({"profile_register": True, "points": n,
                      "rot_err_deg_vs_truth": _rot_err(T[:3, :3], T_gt[:3, :3])}))
    return 0


def profile_variants_main(args):
    """Plain launches of the Sec. 5 / Sec. 4.1 variants on the bench's LiDAR
    pair for an external profiler: per variant two warm-up registrations of
    2 rounds, then one of 2 rounds (flat J=n from the depth-4 leaves; the
    multi-path descent at tau = 0.01; the full Eq. 7 M-step)."""
    import torch
    from paper_1807_02587_gb300 import binding as B
    from paper_1807_02587_gb300 import synth
    pair = synth.lidar_pair(args.seed)
    tgt = torch.from_numpy(synth.to_float4(pair["tgt"])).cuda()
    src = torch.from_numpy(synth.to_float4(pair["src"])).cuda()
    n = int(max(tgt.shape[0], src.shape[0]))
    tree = B.Tree(n, DEPTH)
    tree.build(tgt, DEPTH)
    flat = B.Flat(n, int(B.hgmm_node_count(DEPTH)))
    flat.from_tree(tree)
    for _ in range(3):
        flat.register(src, iters=2)
    flat.sync()
    for _ in range(3):
        tree.register_descent(src, B.HGMM_DESCENT_MULTIPATH, 0.01, iters=2)
    for _ in range(3):
        tree.register_descent(src, B.HGMM_DESCENT_ML_LOCAL, 0.0, iters=2, full_eq7=True)
    tree.sync()
    print(json.dumps({"profile_variants": True, "J": flat.export()["J"]}))
    return 0


def profile_batch_main(args):
    """The batched launch alone on the first P pairs of the bench's batched
    workload (same seed, depth, cluster shape 8), twice; prints the
    algorithmic bytes of one launch: every EM iteration of every level reads
    each target point (16 B), the hand-off reads it again and writes it, and
    every registration round reads each source point (16 B)."""
    import torch
    from paper_1807_02587_gb300 import binding as B
    from paper_1807_02587_gb300 import synth
    pairs = synth.batched_pairs(args.seed + 100, count=256)[: args.profile_batch]
    tb = [synth.to_float4(p["tgt"]) for p in pairs]
    sb = [synth.to_float4(p["src"]) for p in pairs]
    t_off = np.concatenate([[0], np.cumsum([x.shape[0] for x in tb])]).astype(np.int64)
    s_off = (np.concatenate([[0], np.cumsum([x.shape[0] for x in sb])]) + t_off[-1]).astype(np.int64)
    n = len(pairs)
    pts = torch.from_numpy(np.concatenate(tb + sb)).cuda()
    bat = B.Batch(int(max(np.diff(t_off).max(), np.diff(s_off).max())), 4, n)
    B.hgmm_batch_plan(bat.handle, t_off, s_off, [p["depth"] for p in pairs])
    B.hgmm_batch_set_shape(bat.handle, 8)
    T = torch.zeros((n, 16), dtype=torch.float64, device="cuda")
    prm = B.params()
    for _ in range(2):
        B.hgmm_batch_register(bat.handle, pts, T, prm, None, ITERS)
    torch.cuda.synchronize()
    nt = np.diff(t_off)
    ns = np.diff(s_off)
    depth = np.array([p["depth"] for p in pairs])
    estep = int(np.sum(16 * nt * prm.em_iters * depth))
    handoff = int(np.sum(2 * 16 * nt * depth))
    reg = int(np.sum(16 * ns * ITERS))
    print(json.dumps({"profile_batch": True, "pairs": n, "target_points": int(nt.sum()),
                      "source_points": int(ns.sum()), "device_bytes_inputs": int(pts.numel() * 4),
                      "algorithmic_bytes_per_launch": {"estep": estep, "handoff": handoff,
                                                       "register": reg, "total": estep + handoff + reg}}))
    return 0


def profile_mlp_main():
    import torch
    from paper_1807_02587_gb300 import binding as B
    params = np.load(os.path.join(ROOT, "paper_1807_02587_gb300", "weights", "proposal_mlp.npz"))["params"]
    net = B.Mlp(8192)
    B.hgmm_mlp_set_params(net.handle, params)
    g = torch.Generator(device="cuda")
    g.manual_seed(0)
    x = torch.randn((8192, 1280), device="cuda", generator=g).to(torch.bfloat16)
    y = torch.zeros((8192, 9), dtype=torch.float32, device="cuda")
    lab = torch.zeros((8192, 12), dtype=torch.float32, device="cuda")
    lab[:, [0, 4, 8]] = 1.0
    for _ in range(5):
        B.hgmm_mlp_forward(net.handle, x, y)
    for _ in range(3):
        B.hgmm_mlp_train_step(net.handle, x, lab, 1024, lr=0.0)
    B.hgmm_mlp_sync(net.handle)
    print(json.dumps({"profile_mlp": True, "y_finite": bool(torch.isfinite(y).all().item())}))
    return 0


if __name__ == "__main__":
    sys.exit(main())
