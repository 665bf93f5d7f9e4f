#!/usr/bin/env python3
"""Benchmark: loopy belief propagation edge-state message updates per second.

Workload (default): the 2D Ising grid 1000x1000 (1,998,000 pairwise factors,
7,992,000 edge-states), couplings J~U[-1,1] as [J,-J,-J,J], fields h~N(0,1), damping
0.5, 200 flooding iterations, FP32 messages. One step = one cold-start run at T=1
(sum-product) and one at T=0 (max-product), each followed by normalised beliefs and
the MAP decode. One update = one new factor-to-variable value for one edge-state in
one iteration, so a step is 2 x 200 x 7,992,000 updates.

Prints one JSON line. Under torchrun (N > 1) every rank runs its own replica (seed =
rank): the graph does not shard, so there is no collective on the data path; the
barrier and the max over ranks of the timed duration are the only communication.

--impl reference times the FP64 oracle (the plain CPU restatement of the method) on
the host cores on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import datetime
import hashlib
import json
import os
import re
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "LBP edge-state msg updates/s (batched vs per-graph) at 1e-4; p50/p99 serve latency"
UNIT = "edge-state updates/s"
NOMINAL_HBM_GBS = 7900.0  # GB300 HBM3e, nominal
FALLBACK_HBM_GBS = 6800.0
L2_FLUSH_BYTES = 512 << 20
PROFILE_PERIOD = 100  # per-pass CUDA events (graph event nodes) on every 100th iteration of the timed runs


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--side", type=int, default=1000)
    ap.add_argument("--iters", type=int, default=200)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-batch", action="store_true", help="skip the batched vs per-graph measurement")
    ap.add_argument("--batch-grids", type=int, default=256)
    ap.add_argument("--no-multi", action="store_true", help="skip the multi-evidence measurement")
    ap.add_argument("--no-grad", action="store_true", help="skip the gradient measurement")
    ap.add_argument("--no-deconv", action="store_true",
                    help="skip the deconvolution (1000 iterations) and 10x10 latency sections")
    ap.add_argument("--no-until", action="store_true", help="skip the batch's per-member early exit")
    ap.add_argument("--pool-probe", default="",
                    help="SIDE,RADIUS,SLACK: a short uncaptured run of a pool grid (large listed-"
                         "configuration factors, T=0) for ncu captures of its kernels")
    ap.add_argument("--batch-probe", type=int, default=0,
                    help="only run the batched workload for N iterations (3 runs, no CUDA graphs; for ncu)")
    ap.add_argument("--deconv-probe", type=int, default=0,
                    help="only run the deconvolution workload for N iterations (3 runs, no CUDA graphs; for ncu)")
    ap.add_argument("--small-probe", type=int, default=0,
                    help="only run N runs of the 10x10 grid workload (50 iterations, T=1, one launch each; for ncu)")
    ap.add_argument("--small-side", type=int, default=10,
                    help="with --small-probe: the grid's side (above 26 the run is one cluster launch)")
    ap.add_argument("--grad-probe", type=int, default=0,
                    help="run only N gradient calls of the gradient workload, CUDA graphs off (for ncu)")
    ap.add_argument("--pair-form", type=int, default=0,
                    help="with --batch-probe: the dense K-state pairwise kernel form (PGM_OPT_PAIR_FORM)")
    ap.add_argument("--no-serve", action="store_true", help="skip the serving measurement")
    ap.add_argument("--serve-rate", type=float, default=2000.0, help="mean Poisson arrival rate (requests/s)")
    ap.add_argument("--serve-duration", type=float, default=1.0, help="seconds of arrivals per serving run")
    ap.add_argument("--serve-slots", type=int, default=16)
    ap.add_argument("--cpu-iters", type=int, default=40, help="oracle iterations per T in the CPU baseline sample")
    ap.add_argument("--ref-iters", type=int, default=16, help="oracle iterations per T in one reference step")
    return ap.parse_args()


def workload_config(args, n_gpus):
    return {
        "workload": f"ising{args.side}x{args.side}",
        "description": f"2D Ising {args.side}x{args.side} binary, 4-neighbour pairwise enumeration factors, "
                       f"J~U[-1,1] as [J,-J,-J,J], h~N(0,1) as [-h,h], damping 0.5, {args.iters} iterations, "
                       "one T=1 (sum-product) and one T=0 (max-product) cold-start run per step",
        "iterations": args.iters,
        "temperatures": [1.0, 0.0],
        "damping": 0.5,
        "messages": "fp32 (log-ratio per edge inside a run on binary pairwise graphs)",
        "l2": f"flushed between timed steps ({L2_FLUSH_BYTES >> 20} MiB write)",
        "parallelism": f"replicas x{n_gpus}" if n_gpus > 1 else "single GPU",
    }


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        for k in ("hbm_gbs", "hbm_GBs", "hbm"):
            if k in d:
                return float(d[k]), "measured"
    except (OSError, ValueError):
        pass
    return FALLBACK_HBM_GBS, "fallback"


LR_KERNELS = ("k_pair2_lr", "k_var_slot4_lr", "k_var_csr_lr")


def kernel_source_hash(kernel: str) -> str:
    """sha256 (16 hex digits) of the source a kernel is built from: for the log-ratio
    kernels, kernels.cu's helper prelude (before the first section), its log-ratio
    section and the log-ratio launchers; for the others, the whole of kernels.cu."""
    with open(os.path.join(ROOT, "paper_2202_04110_gb300", "csrc", "kernels.cu")) as f:
        src = f.read()
    if kernel in LR_KERNELS:
        first = src.index("// =====")
        a = src.index("// Binary pairwise graphs: log-ratio messages (Plan::lr)")
        b = src.index("// Many evidence / potential sets on one binary pairwise graph")
        c = src.index("static cudaError_t launch_pdl(")
        d = src.index("cudaError_t launch_ms_prepare(")
        src = src[:first] + src[a:b] + src[c:d]
    return hashlib.sha256(src.encode()).hexdigest()[:16]


def profiled_traffic(kernel: str, workload: str):
    """dram bytes per launch recorded from an ncu capture in profiles/, if the kernel's
    source (kernel_source_hash) has not changed since."""
    path = os.path.join(ROOT, "profiles", f"{kernel}_{workload}.md")
    try:
        txt = open(path).read()
    except OSError:
        return None
    m = re.search(r"traffic_bytes_per_launch:\s*([0-9.eE+]+)", txt)
    h = re.search(r"source_sha256_16:\s*([0-9a-f]+)", txt)
    if not m or not h or h.group(1) != kernel_source_hash(kernel):
        return None
    return float(m.group(1))


class ClockSampler:
    """nvidia-smi samples during the timed region."""

    FIELDS = ("timestamp,index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.window = None

    def start(self):
        """Start sampling (every 20 ms); call before the warm-up so that sampling runs
        when the timed region begins."""
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "20"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None

    def mark(self, t0: float, t1: float):
        """The timed region in host wall-clock seconds (time.time())."""
        self.window = (t0, t1)

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
            out, _ = self.proc.communicate()
        rows = []
        for line in out.strip().splitlines():
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 10:
                continue
            try:
                ts = datetime.datetime.strptime(parts[0], "%Y/%m/%d %H:%M:%S.%f").timestamp()
                rows.append((ts, float(parts[2]), float(parts[3]), parts[6:10]))
            except ValueError:
                continue
        inside = [r for r in rows if self.window and self.window[0] <= r[0] <= self.window[1]]
        used, where = (inside, "timed region") if inside else (rows, "whole run (no sample fell in the timed region)")
        if not used:
            return None
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({nm for r in used for nm, val in zip(names, r[3]) if val.lower().startswith("active")})
        return {"sm_mhz": statistics.median(r[1] for r in used), "sm_max_mhz": max(r[2] for r in used),
                "reasons": reasons, "samples": len(used), "window": where}


def aggregate_ranks(dist, local_ms: float, updates_per_rank: float, device=None):
    """Whole-job throughput over replicas: the slowest rank's time (all-reduce MAX) and
    the updates of all ranks. Returns (max_ms, updates/s)."""
    world = dist.get_world_size() if dist is not None else 1
    ms = local_ms
    if dist is not None and world > 1:
        import torch
        t = torch.tensor([local_ms], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
    return ms, world * updates_per_rank / (ms / 1e3)


def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def cpu_sample(problem, iters: int):
    """Time the FP64 oracle on the host cores: `iters` iterations at T=1 and at T=0."""
    import oracle
    oracle.build()
    t0 = time.perf_counter()
    for T in (1.0, 0.0):
        oracle.run_bp(problem.graph, problem.log_pot, problem.evidence, T, problem.damping, iters)
    dt = time.perf_counter() - t0
    updates = 2 * iters * problem.graph.n_edge_states
    return updates / dt, dt, oracle.num_threads()


def run_reference(args):
    world, rank, _ = dist_setup()
    if rank != 0:
        return
    from paper_2202_04110_gb300 import workloads as W
    p = W.ising_large(0, T=1.0, side=args.side, n_iters=args.iters)
    vals = []
    for _ in range(args.warmup):
        cpu_sample(p, args.ref_iters)
    total_updates, total_s, cores = 0, 0.0, 1
    for _ in range(args.steps):
        v, dt, cores = cpu_sample(p, args.ref_iters)
        vals.append(v)
        total_updates += 2 * args.ref_iters * p.graph.n_edge_states
        total_s += dt
    value = total_updates / total_s
    sample = (f"{args.ref_iters} iterations at T=1 and {args.ref_iters} at T=0 per step on the full "
              f"{args.side}x{args.side} grid (FP64 oracle, OpenMP)")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total_s / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": workload_config(args, world),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def measure_batched(args, binding, W, torch, dev):
    """Batched vs per-graph on the uneven-graph workload: 256 Potts grids (side U{16..256},
    K in {2,4,8,16}, truncated-linear tables) plus the 784x500 RBM, T=1, damping 0.5,
    100 iterations. Batched = one graph of all members (one launch per kernel variant per
    pass, launch shapes autotuned, run replayed as a CUDA graph); per-graph = each member
    built and run on its own (same kernels, CUDA graphs per member)."""
    iters = 100
    batch, members = W.potts_rbm_batch(seed=0, n_grids=args.batch_grids, n_iters=iters)
    lp = torch.as_tensor(batch.log_pot).to(dev)
    ev = torch.as_tensor(batch.evidence).to(dev)
    gb = binding.Graph([m.graph for m in members])
    ES = gb.info["n_edge_states"]
    mb = gb.new_msgs()
    t0 = time.perf_counter()
    gb.autotune(lp, ev, 1.0, 0.5)
    tune_s = time.perf_counter() - t0
    stream = torch.cuda.current_stream()

    def timed(fn, reps):
        fn()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / 1e3 / reps

    def run_batched():
        mb.zero_()
        gb.run_bp(lp, ev, 1.0, 0.5, iters, mb)

    t_batched = timed(run_batched, 3)
    singles = []
    for i, m in enumerate(members):
        off = gb.member(i)
        g = binding.Graph(m.graph)
        lpi = lp[off["pot_off"]: off["pot_off"] + off["n_potentials"]]
        evi = ev[off["vs_off"]: off["vs_off"] + off["n_var_states"]]
        singles.append((g, lpi, evi, g.new_msgs()))

    def run_singles():
        for g, lpi, evi, mi in singles:
            mi.zero_()
            g.run_bp(lpi, evi, 1.0, 0.5, iters, mi)

    import numpy as np
    t_single = timed(run_singles, 2)
    upd = ES * iters
    launches = [dict(zip(("kind", "variant", "threads", "blocks"), x)) for x in gb.launches()]
    kernels = batched_kernel_rooflines(gb, members, lp, ev, iters)
    # f4 inside the batch: each member stops once its own residual is <= 1e-4 (checked
    # every 10 iterations, at most `iters`), the stopped members' factors are skipped
    out_ee = {}
    if not args.no_until:
        res_holder = {}

        def run_members():
            mb.zero_()
            res_holder["done"], _ = gb.run_bp_until_members(lp, ev, 1.0, 0.5, iters, 1e-4, 10, mb)

        t_members = timed(run_members, 3)
        done = res_holder["done"]
        member_es = np.array([gb.member(i)["n_edge_states"] for i in range(len(members))], np.int64)
        out_ee = {"early_exit_members": {
            "tol": 1e-4, "check_every": 10, "max_iters": iters, "ms_per_run": 1e3 * t_members,
            "speedup_vs_fixed": t_batched / t_members,
            "members_stopped_early": int((done < iters).sum()),
            "edge_state_updates_run_fraction": float((done * member_es).sum() / (iters * member_es.sum())),
            "call": "pgm_run_bp_until_members (edge-state iterations, conditional while node)"}}
    peak, _ = measured_peaks()
    it_bytes = sec8d_bytes(batch.graph)
    out_cpu = {}
    if not args.no_cpu_baseline:
        # the FP64 oracle on a seeded subset: the first 16 grids of the batch and the RBM
        import oracle
        oracle.build()
        sub = W.union(members[:16] + [members[-1]], name="subset")
        n_cpu = 3
        t0 = time.perf_counter()
        oracle.run_bp(sub.graph, sub.log_pot, sub.evidence, 1.0, 0.5, n_cpu)
        dt = time.perf_counter() - t0
        out_cpu = {"cpu_baseline": {"value": n_cpu * sub.graph.n_edge_states / dt, "unit": UNIT,
                                    "cores": oracle.num_threads(), "kind": "oracle",
                                    "sample": f"{n_cpu} iterations of the first 16 Potts grids and the RBM "
                                              f"({sub.graph.n_edge_states} edge-states), FP64, {dt:.1f} s"}}
    return {"workload": f"{args.batch_grids} Potts grids (side U{{16..256}}, K in {{2,4,8,16}}) + RBM 784x500, "
                        f"T=1, damping 0.5, {iters} iterations",
            "graphs": len(members), "edge_states": ES,
            "iteration_sec8d_bytes": it_bytes,
            "batched_iteration_frac": round(it_bytes / (t_batched / iters) / 1e9 / peak, 4),
            **out_cpu,
            "batched": upd / t_batched, "per_graph": upd / t_single, "unit": UNIT,
            "batched_ms_per_run": 1e3 * t_batched, "per_graph_ms_per_run": 1e3 * t_single,
            "speedup": t_single / t_batched, "autotune_s": round(tune_s, 2), "launch_shapes": launches,
            "kernels": kernels,
            "kernel_timing": "CUDA events around each launch of every 10th iteration of one batched run (event "
                             "nodes in its CUDA graph); an event pair includes the launch's latency",
            **out_ee}


# factor-pass variants of the dense K-state pairwise groups -> (K, kernel name)
PAIR_VARIANTS = {0: (2, "k_pair<2>"), 1: (4, "k_pair_group<4>"), 2: (8, "k_pair_group<8>"),
                 3: (16, "k_pair_group<16>"), 7: (4, "k_pair_thr<4>"), 8: (8, "k_pair_thr<8>"),
                 9: (16, "k_pair_thr<16>"), 11: (8, "k_pair_quad<8>"), 12: (16, "k_pair_quad<16>"),
                 13: (4, "k_pair_dir<4>"), 14: (8, "k_pair_dir<8>"), 15: (16, "k_pair_dir<16>")}


def batched_kernel_rooflines(gb, members, lp, ev, iters):
    """Per-launch CUDA-event times of one batched run and, for the dense pairwise factor
    launches, their algorithmic bytes and fraction of the HBM peak. A K-state pairwise
    factor moves 4 (2K old-message reads + 2K new-message writes + 2K belief gathers + 2
    edge indices) = 24 K + 8 bytes, plus its K^2 table when the table is its own."""
    import torch
    peak, _ = measured_peaks()
    fac_bytes = {}  # K -> bytes of all pairwise factors with K states
    for m in members:
        for grp in m.graph.enum_groups:
            if grp.arity != 2:
                continue
            K = int(m.graph.num_states[grp.vars[0, 0]]) if grp.vars.shape[0] else 0
            n = int(grp.vars.shape[0])
            fac_bytes[K] = fac_bytes.get(K, 0) + n * (24 * K + 8) + (0 if grp.shared else 4 * n * K * K)
    period = 10
    gb.set_profiling(period)
    mb = gb.new_msgs()
    gb.run_bp(lp, ev, 1.0, 0.5, iters, mb)
    torch.cuda.synchronize()
    lt = gb.launch_times()
    gb.set_profiling(0)
    out = []
    for (kind, variant, threads, blocks), (ms, cnt) in zip(gb.launches(), lt):
        if cnt == 0:
            continue
        us = 1e3 * ms / cnt
        d = {"kind": "factor" if kind == 1 else "variable", "variant": variant, "threads": threads,
             "blocks": blocks, "mean_launch_us": round(us, 2)}
        if kind == 1 and variant in PAIR_VARIANTS and PAIR_VARIANTS[variant][0] in fac_bytes:
            K, name = PAIR_VARIANTS[variant]
            d["kernel"] = name
            d["algorithmic_bytes_per_launch"] = fac_bytes[K]
            d["achieved_gbs"] = round(fac_bytes[K] / (us * 1e-6) / 1e9, 1)
            d["frac"] = round(fac_bytes[K] / (us * 1e-6) / 1e9 / peak, 4)
        out.append(d)
    return out


def measure_multi(args, binding, W, torch, dev):
    """Multi-evidence batching of one graph: a 256x256 Ising grid (couplings shared) with
    32 evidence sets (fields h ~ N(0,1) per sample), T=1, damping 0.5, `iters` iterations,
    all samples in one pgm_run_bp_multi call vs the same samples run one after another
    with pgm_run_bp (CUDA graphs)."""
    import numpy as np
    S, side = 32, 256
    p = W.ising_large(seed=0, T=1.0, side=side, n_iters=args.iters)
    g = binding.Graph(p.graph)
    ES, V = g.info["n_edge_states"], g.info["n_vars"]
    rng = np.random.default_rng(1)
    h = rng.standard_normal((S, V))
    ev = torch.as_tensor(np.stack([-h, h], axis=2).reshape(S, -1).astype(np.float32)).to(dev)
    lp = torch.as_tensor(p.log_pot).to(dev)
    msgs = torch.zeros(S, ES, device=dev)
    singles = [torch.zeros(ES, device=dev) for _ in range(S)]
    stream = torch.cuda.current_stream()

    def run_multi():
        msgs.zero_()
        g.run_bp_multi(lp, ev, 1.0, 0.5, args.iters, msgs)

    def run_singles():
        for s_ in range(S):
            singles[s_].zero_()
            g.run_bp(lp, ev[s_], 1.0, 0.5, args.iters, singles[s_])

    def timed(fn, reps):
        fn()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / 1e3 / reps

    t_multi = timed(run_multi, 3)
    t_single = timed(run_singles, 3)
    same = all(torch.equal(msgs[s_], singles[s_]) for s_ in range(S))
    upd = S * args.iters * ES
    # perturb-and-max-product: S samples (Gumbel-perturbed evidence, T=0, same iterations)
    u = rng.uniform(1e-12, 1.0, (S, g.info["n_var_states"]))
    noise = torch.as_tensor((-np.log(-np.log(u))).astype(np.float32)).to(dev)
    ev0 = ev[0].contiguous()
    t_pmp = timed(lambda: g.pmp_sample(lp, ev0, noise, 0.5, args.iters), 3)
    # a K-state graph: 32 evidence sets of a 96x96 Potts grid (K = 8), side by side
    pk = W.potts_grid(96, 8, 0, T=1.0, n_iters=100)
    gk = binding.Graph(pk.graph)
    ESk = gk.info["n_edge_states"]
    evk = torch.as_tensor((np.asarray(pk.evidence, np.float32)[None, :] +
                           rng.standard_normal((S, pk.graph.n_var_states)).astype(np.float32))).to(dev)
    lpk = torch.as_tensor(pk.log_pot).to(dev)
    mk = torch.zeros(S, ESk, device=dev)
    sk = [torch.zeros(ESk, device=dev) for _ in range(S)]

    def run_multi_k():
        mk.zero_()
        gk.run_bp_multi(lpk, evk, 1.0, 0.5, 100, mk)

    def run_singles_k():
        for s_ in range(S):
            sk[s_].zero_()
            gk.run_bp(lpk, evk[s_], 1.0, 0.5, 100, sk[s_])

    t_mk = timed(run_multi_k, 3)
    t_sk = timed(run_singles_k, 3)
    same_k = all(torch.equal(mk[s_], sk[s_]) for s_ in range(S))
    updk = S * 100 * ESk
    return {"workload": f"ising{side}x{side}, {S} evidence sets (h ~ N(0,1)), shared couplings, "
                        f"T=1, damping 0.5, {args.iters} iterations",
            "samples": S, "multi": upd / t_multi, "one_by_one": upd / t_single, "unit": UNIT,
            "multi_ms_per_call": 1e3 * t_multi, "one_by_one_ms": 1e3 * t_single,
            "speedup": t_single / t_multi, "bitwise_equal_to_single_runs": bool(same),
            "pmp_samples_per_s": S / t_pmp,
            "k_state": {"workload": f"potts96x96 K=8, {S} evidence sets, shared table, T=1, damping 0.5, "
                                    "100 iterations (samples as the second grid dimension)",
                        "multi": updk / t_mk, "one_by_one": updk / t_sk, "speedup": t_sk / t_mk,
                        "bitwise_equal_to_single_runs": bool(same_k)},
            "pmp": f"{S} perturb-and-max-product samples per call (Gumbel-perturbed evidence, T=0, "
                   f"{args.iters} iterations, MAP decode), pgm_pmp_sample"}


def measure_l2_free(args, binding, W, torch, dev):
    """Supplementary DRAM-bound run: a 4000x4000 Ising grid (1.9 GB working set against
    the 129 MB L2, so no iteration is served from L2), T=1, damping 0.5, 50 iterations
    from zero messages, CUDA events around each run (L2 is overwritten by the run
    itself). The same log-ratio kernels and byte accounting as the headline."""
    side, n_it = 4000, 50
    p = W.ising_large(seed=0, T=1.0, side=side, n_iters=n_it)
    g = binding.Graph(p.graph)
    I = g.info
    lp = torch.as_tensor(p.log_pot).to(dev)
    ev = torch.as_tensor(p.evidence).to(dev)
    m = g.new_msgs()
    stream = torch.cuda.current_stream()
    for _ in range(3):
        m.zero_()
        g.run_bp(lp, ev, 1.0, 0.5, n_it, m)
    torch.cuda.synchronize()
    times = []
    for _ in range(5):
        m.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        g.run_bp(lp, ev, 1.0, 0.5, n_it, m)
        e1.record(stream)
        torch.cuda.synchronize()
        times.append(e0.elapsed_time(e1) / 1e3)
    t = statistics.median(times)
    V, VS, E, F = I["n_vars"], I["n_var_states"], I["n_edges"], I["n_factors"]
    iter_bytes = (4 * (E + 2 * E + 3 * F) + 8 * V) + (4 * (4 * V + VS) + 8 * V)
    peak, _ = measured_peaks()
    it_s = t / n_it
    lr_on = g.get_option(binding.OPT_LOG_RATIO) > 0
    del m, g
    return {"workload": f"ising{side}x{side}, T=1, damping 0.5, {n_it} iterations (log-ratio path)",
            "value": n_it * I["n_edge_states"] / t, "unit": UNIT, "ms_per_run": 1e3 * t,
            "iteration_us": round(1e6 * it_s, 2), "iteration_algorithmic_bytes": iter_bytes,
            "achieved_gbs": round(iter_bytes / it_s / 1e9, 1), "frac": round(iter_bytes / it_s / 1e9 / peak, 4),
            "frac_of_nominal": round(iter_bytes / it_s / 1e9 / NOMINAL_HBM_GBS, 4),
            "log_ratio_path": lr_on}


def measure_large_enum(args, binding, W, torch, dev):
    """Large listed-configuration factors (block-per-factor kernel k_enum_block): grids of
    RCN-style pool variables (Sec. 5.2), K = (2r + 1)^2 offsets per variable, lateral
    factors listing the offset pairs within `slack` (one shared N(0,1) table), max-product
    T=0, damping 0.5, 50 iterations. Reported: edge-state updates/s of whole runs, and the
    factor pass's achieved HBM bandwidth (algorithmic bytes 4 (3 ksum + arity) per factor:
    old and new messages and the belief gather) from in-graph pass events."""
    out = []
    stream = torch.cuda.current_stream()
    n_it = 50
    for side, radius, slack in ((256, 3, 1), (128, 5, 2)):
        p = W.pool_grid(side, radius, slack, 0, T=0.0, n_iters=n_it)
        g = binding.Graph(p.graph)
        lp = torch.as_tensor(p.log_pot).to(dev)
        ev = torch.as_tensor(p.evidence).to(dev)
        m = g.new_msgs()
        for _ in range(3):
            m.zero_()
            g.run_bp(lp, ev, 0.0, 0.5, n_it, m)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        reps = 5
        e0.record(stream)
        for _ in range(reps):
            m.zero_()
            g.run_bp(lp, ev, 0.0, 0.5, n_it, m)
        e1.record(stream)
        torch.cuda.synchronize()
        t = e0.elapsed_time(e1) / 1e3 / reps
        g.set_profiling(1)
        m.zero_()
        g.run_bp(lp, ev, 0.0, 0.5, n_it, m)
        torch.cuda.synchronize()
        tv, tf, nv, nf = g.pass_times()
        g.set_profiling(0)
        grp = p.graph.enum_groups[0]
        K = int(p.graph.num_states[0])
        ksum = 2 * K
        fac_bytes = 4 * (3 * ksum + 2) * grp.n_fac
        f_ms = tf / max(nf, 1)
        ES = g.info["n_edge_states"]
        out.append({"workload": f"pool grid {side}x{side}, K={K}, {grp.n_cfg} of {K * K} pairs listed "
                                f"(slack {slack}), T=0, damping 0.5, {n_it} iterations",
                    "value": n_it * ES / t, "unit": UNIT, "ms_per_run": 1e3 * t,
                    "factor_pass_ms": f_ms, "var_pass_ms": tv / max(nv, 1),
                    "factor_pass_gbs": fac_bytes / (f_ms * 1e-3) / 1e9,
                    "launches": g.launches()})
    return out


def sec8d_bytes(fg, factor_groups=None):
    """The per-iteration minimum traffic of the method for a factor graph: 8 ES (read and
    write every factor-to-variable message) + 4 sum n_cfg (per-factor log-potentials; a
    shared table counts once) + 4 VS (evidence) + 4 E (edge index). With `factor_groups`
    (indices into enum_groups + logic_groups), the factor-side share of those groups
    only: their 8 ES + 4 n_cfg + 4 E."""
    import numpy as np
    k = fg.num_states.astype(np.int64)
    groups = [("enum", g) for g in fg.enum_groups] + [("logic", g) for g in fg.logic_groups]
    sel = range(len(groups)) if factor_groups is None else factor_groups
    total = 0
    for i in sel:
        kind, g = groups[i]
        if kind == "enum":
            es, e = int(k[g.vars].sum()), g.n_fac * g.arity
            total += 8 * es + 4 * e + 4 * (g.n_cfg if g.shared else g.n_cfg * g.n_fac)
        else:
            e = int(g.par_off[-1]) + g.n_fac
            total += 8 * 2 * e + 4 * e
    if factor_groups is None:
        total += 4 * int(k.sum())
    return total


def measure_deconv(args, binding, W, torch, dev):
    """Binary deconvolution with logical factors (the paper's Sec. 5.2 example; synthetic
    stand-in for its notebook data): 5 features 6x6, activations 10x10, 100 images 15x15,
    1,800,000 AND factors (fan-in 2) and 22,500 OR factors (fan-in 5..180), max-product T=0,
    damping 0.5, 1000 iterations from zero messages. Whole runs timed with CUDA events;
    per-launch times from in-graph events on every 50th iteration of one run; the FP64
    oracle timed on the host cores on a 10-iteration sample of the same graph."""
    import numpy as np
    n_it = 1000
    p = W.deconvolution(0, n_iters=n_it)
    fg = p.graph
    g = binding.Graph(fg)
    I = g.info
    ev = torch.as_tensor(p.evidence).to(dev)
    m = g.new_msgs()
    stream = torch.cuda.current_stream()
    for _ in range(2):
        m.zero_()
        g.run_bp(None, ev, 0.0, 0.5, n_it, m)
    torch.cuda.synchronize()
    times = []
    for _ in range(3):
        m.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        g.run_bp(None, ev, 0.0, 0.5, n_it, m)
        e1.record(stream)
        torch.cuda.synchronize()
        times.append(e0.elapsed_time(e1) / 1e3)
    t = statistics.median(times)
    period = 50
    g.set_profiling(period)
    m.zero_()
    g.run_bp(None, ev, 0.0, 0.5, n_it, m)
    torch.cuda.synchronize()
    lt = g.launch_times()
    g.set_profiling(0)
    launches = g.launches()
    peak, _ = measured_peaks()
    # the workload's parts: W (degree 10,000: block-per-variable pass), the AND group
    # (thread per factor) and the OR group (warp per factor)
    ks = fg.num_states.astype(np.int64)
    deg = np.zeros(fg.n_vars, np.int64)
    for lg_ in fg.logic_groups:
        np.add.at(deg, lg_.parents, 1)
        np.add.at(deg, lg_.child, 1)
    hi = deg > 64
    # implementation bytes per launch: the high-degree pass reads the variables' K d
    # messages and their incoming-edge index, writes and re-reads the tile totals (16 bytes
    # per tile and state) and writes each state's totals (16 bytes) and belief;
    # a logical factor reads its old messages, the beliefs of its edges (the totals of a
    # high-degree variable) and their index, and writes its messages
    n_hi_es = int((ks[hi] * deg[hi]).sum())
    and_g, or_g = fg.logic_groups[0], fg.logic_groups[1]
    e_and = int(and_g.par_off[-1]) + and_g.n_fac
    e_or = int(or_g.par_off[-1]) + or_g.n_fac
    d_hi = int(deg[hi].sum())
    n_tiles_st = int((ks[hi] * ((deg[hi] + 2047) // 2048)).sum())
    impl = {"k_var_hd": 4 * n_hi_es + 4 * d_hi + 32 * n_tiles_st + 20 * int(ks[hi].sum()),
            "k_logic_small": 4 * (4 * e_and + 2 * e_and + e_and),
            "k_logic_warp": 4 * (4 * e_or + 2 * e_or + e_or)}
    s8d = {"k_logic_small": sec8d_bytes(fg, [0]), "k_logic_warp": sec8d_bytes(fg, [1]),
           "k_var_hd": 4 * int(ks[hi].sum())}
    names = {(0, 1): "k_var_hd", (0, 2): "k_var_thread<2>", (0, 0): "k_var_thread",
             (1, 5): "k_logic_small", (1, 6): "k_logic_warp"}
    per = {}
    for (kind, variant, threads, blocks), (ms, cnt) in zip(launches, lt):
        name = names.get((kind, variant), f"kind{kind}_variant{variant}")
        if cnt == 0:
            continue
        us = 1e3 * ms / cnt
        d = {"mean_launch_us": round(us, 2), "threads": threads, "blocks": blocks}
        if name in impl:
            d["algorithmic_bytes_per_launch"] = impl[name]
            d["achieved_gbs"] = round(impl[name] / (us * 1e-6) / 1e9, 1)
            d["frac"] = round(impl[name] / (us * 1e-6) / 1e9 / peak, 4)
            d["sec8d_share_bytes"] = s8d[name]
            d["sec8d_frac"] = round(s8d[name] / (us * 1e-6) / 1e9 / peak, 4)
        per[name] = d
    it_s = t / n_it
    it_bytes = sec8d_bytes(fg)
    ES = I["n_edge_states"]
    out = {"workload": "deconvolution: 5 features 6x6, S 10x10, 100 images 15x15 (W 180, S 50,000, AND 1,800,000, "
                       "X 22,500 variables; 1,800,000 AND + 22,500 OR factors), T=0, damping 0.5, 1000 iterations",
           "edge_states": ES, "value": n_it * ES / t, "unit": UNIT, "ms_per_run": round(1e3 * t, 3),
           "iteration_us": round(1e6 * it_s, 2), "iteration_sec8d_bytes": it_bytes,
           "iteration_achieved_gbs": round(it_bytes / it_s / 1e9, 1),
           "iteration_frac": round(it_bytes / it_s / 1e9 / peak, 4),
           "kernels": per,
           "kernel_timing": f"CUDA events around each launch of every {period}th iteration of one run "
                            "(event nodes in its CUDA graph); an event pair includes the launch's latency"}
    if not args.no_cpu_baseline:
        import oracle
        oracle.build()
        n_cpu = 10
        t0 = time.perf_counter()
        oracle.run_bp(fg, p.log_pot, p.evidence, 0.0, 0.5, n_cpu)
        dt = time.perf_counter() - t0
        out["cpu_baseline"] = {"value": n_cpu * ES / dt, "unit": UNIT, "cores": oracle.num_threads(),
                               "kind": "oracle", "sample": f"{n_cpu} iterations of the full graph, FP64, {dt:.1f} s"}
    del m, g
    return out


def measure_small(args, binding, W, torch, dev):
    """Per-iteration latency of the 10x10 Ising grid (180 factors, 720 edge-states), T=1,
    damping 0.5, 50 iterations: CUDA events around 200 back-to-back pgm_run_bp calls (one
    CUDA graph replay each), and the FP64 oracle's time for the same run on the host; the
    same for a 64x64 grid (one cluster launch per run), each beside the multi-launch
    run."""
    stream = torch.cuda.current_stream()

    def per_run(p, small):
        lp = torch.as_tensor(p.log_pot).to(dev)
        ev = torch.as_tensor(p.evidence).to(dev)
        g = binding.Graph(p.graph)
        g.set_option(binding.OPT_SMALL_RUN, small)
        m = g.new_msgs()
        for _ in range(10):
            g.run_bp(lp, ev, 1.0, 0.5, p.n_iters, m)
        torch.cuda.synchronize()
        reps = 200
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            g.run_bp(lp, ev, 1.0, 0.5, p.n_iters, m)
        e1.record(stream)
        torch.cuda.synchronize()
        launches = 1 if g.get_option(binding.OPT_SMALL_RUN) else p.n_iters * g.info["launches_per_iter"] + 3
        return e0.elapsed_time(e1) / 1e3 / reps, launches, g.info["n_edge_states"]

    p = W.ising_small(0)
    t, launches, n_es = per_run(p, 1)  # the default: one block runs the whole run
    t_multi, launches_multi, _ = per_run(p, 0)
    out = {"workload": "ising10x10, T=1, damping 0.5, 50 iterations", "us_per_run": round(1e6 * t, 2),
           "us_per_iteration": round(1e6 * t / p.n_iters, 3),
           "value": p.n_iters * n_es / t, "unit": UNIT, "launches_per_run": launches,
           "multi_launch": {"us_per_run": round(1e6 * t_multi, 2), "launches_per_run": launches_multi,
                            "note": "PGM_OPT_SMALL_RUN 0: two launches per iteration"}}
    pm = W.ising_grid(64, 64, 0, T=1.0)  # 4,096 variables: one launch of an 8-block cluster
    tc, lc, n_es_m = per_run(pm, 1)
    tm, lm, _ = per_run(pm, 0)
    out["cluster_grid"] = {"workload": "ising64x64, T=1, damping 0.5, 50 iterations",
                           "us_per_run": round(1e6 * tc, 2), "value": pm.n_iters * n_es_m / tc, "unit": UNIT,
                           "launches_per_run": lc, "multi_launch_us_per_run": round(1e6 * tm, 2),
                           "multi_launch_launches_per_run": lm}
    if not args.no_cpu_baseline:
        import oracle
        oracle.build()
        t0 = time.perf_counter()
        n_rep = 0
        while n_rep < 200 and time.perf_counter() - t0 < 2.0:
            oracle.run_bp(p.graph, p.log_pot, p.evidence, 1.0, 0.5, p.n_iters)
            n_rep += 1
        dt = (time.perf_counter() - t0) / n_rep
        out["cpu_baseline"] = {"us_per_run": round(1e6 * dt, 2), "cores": oracle.num_threads(), "kind": "oracle",
                               "sample": f"{n_rep} runs of the full workload (FP64)"}
    return out


def measure_grad(args, binding, W, torch, dev):
    """The gradient of the serving + gradient configuration: L = sum(g * normalised
    log-beliefs) after 100 sum-product iterations (damping 0.5) of a 64x64 Ising grid,
    w.r.t. the log-potentials and the evidence (pgm_grad, reverse mode through the
    unrolled iterations, a message checkpoint every 10 iterations), against the forward
    run alone (pgm_run_bp + normalised beliefs)."""
    import numpy as np
    p = W.ising_grid(64, 64, 0, T=1.0, n_iters=100)
    g = binding.Graph(p.graph)
    lp = torch.as_tensor(p.log_pot).to(dev)
    ev = torch.as_tensor(p.evidence).to(dev)
    gnb = torch.as_tensor(np.random.default_rng(1).standard_normal(p.graph.n_var_states).astype(np.float32)).to(dev)
    msgs = g.new_msgs()
    stream = torch.cuda.current_stream()

    def forward():
        msgs.zero_()
        g.run_bp(lp, ev, 1.0, 0.5, 100, msgs)
        g.beliefs(ev, msgs, True)

    def backward():
        g.grad(lp, ev, 1.0, 0.5, 100, 10, gnb)

    def timed(fn, reps):
        for _ in range(3):
            fn()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps

    t_fwd = timed(forward, 20)
    t_grad = timed(backward, 20)
    return {"workload": "ising64x64, T=1, damping 0.5, 100 iterations, checkpoint every 10, "
                        "cotangent N(0,1) on the normalised log-beliefs",
            "grad_ms": t_grad, "forward_ms": t_fwd, "grad_over_forward": t_grad / t_fwd,
            "call": "pgm_grad (forward with checkpoints + reverse pass)"}


def measure_until(args, binding, W, torch, dev):
    """Early-exit runs (pgm_run_bp_until) on a 64x64 Ising grid, T=1, damping 0.5, up to
    400 iterations, residual checked every 10, tol 1e-6: the device loop (CUDA graph with a
    conditional while node) vs the host-checked chunks (CUDA graphs off)."""
    p = W.ising_grid(64, 64, 0, T=1.0)
    lp = torch.as_tensor(p.log_pot).to(dev)
    ev = torch.as_tensor(p.evidence).to(dev)
    out = {"workload": "ising64x64, T=1, damping 0.5, max 400 iterations, check every 10, tol 1e-6"}
    for name, graphs in (("device_loop", 1), ("host_checked", 0)):
        g = binding.Graph(p.graph)
        g.set_option(binding.OPT_CUDA_GRAPH, graphs)
        m = g.new_msgs()
        for _ in range(3):
            m.zero_()
            done, res = g.run_bp_until(lp, ev, 1.0, 0.5, 400, 1e-6, 10, m)
        t0 = time.perf_counter()
        for _ in range(10):
            m.zero_()
            done, res = g.run_bp_until(lp, ev, 1.0, 0.5, 400, 1e-6, 10, m)
        out[name + "_ms"] = (time.perf_counter() - t0) / 10 * 1e3
        out["iterations"] = done
    out["speedup"] = out["host_checked_ms"] / out["device_loop_ms"]
    return out


def serve_run(binding, templates, descs, arrivals, slots, budget, tol=None):
    """Submit `arrivals` on schedule to a server with `slots` in-flight requests; wait
    for all; latencies (s) and throughput (updates/s over first submission to last
    completion). With `tol`, each request may stop early (residual checked every 10
    iterations; its iteration count is the limit)."""
    srv = binding.Server(memory_budget_bytes=budget, max_in_flight=slots)
    # the templates' inputs, borrowed by every request (pgm_serve_submit_borrowed: no copy
    # at submission, so the submitter keeps up with the offered rate)
    import numpy as np
    lps = [np.ascontiguousarray(p.log_pot, np.float32) for p in templates]
    evs = [np.ascontiguousarray(p.evidence, np.float32) for p in templates]
    ids = []
    t0 = time.perf_counter()
    for t_arr, ti, iters in arrivals:
        now = time.perf_counter() - t0
        if t_arr > now:
            time.sleep(t_arr - now)
        p = templates[ti]
        ids.append(srv.submit(p.graph, lps[ti], evs[ti], p.T, 0.5, iters, desc=descs[ti], tol=tol, borrow=True))
    t_sub = time.perf_counter() - t0
    lat = []
    for i in ids:
        _, _, l = srv.wait(i, 600.0)
        lat.append(l)
    st = srv.stats()
    srv.close()
    lat = sorted(lat)
    q = lambda f: 1e3 * lat[min(len(lat) - 1, int(f * len(lat)))]
    n_ok = max(st["completed"], 1)
    return {"requests": len(ids), "p50_ms": round(q(0.50), 2), "p99_ms": round(q(0.99), 2),
            "mean_ms": round(1e3 * sum(lat) / len(lat), 2),
            "throughput": st["updates_done"] / st["span_s"] if st["span_s"] > 0 else None,
            "served_req_s": round(st["completed"] / st["span_s"], 1) if st["span_s"] > 0 else None,
            "offered_rate_achieved": round(len(ids) / t_sub, 1), "span_s": round(st["span_s"], 3),
            "arrival_window_s": round(arrivals[-1][0], 3) if arrivals else 0.0,
            # mean seconds per request in each stage (queue to a worker, host compile,
            # admission wait, device work: build, upload, iterations, read-back)
            "mean_stage_ms": {k: round(1e3 * st[k + "_s"] / n_ok, 3) for k in ("queue", "compile", "admit", "run")},
            "peak_bytes": st["peak_bytes"], "failed": st["failed"]}


def measure_serving(args, binding, W):
    """Serving workload: Poisson arrivals of grid requests (side U{16..512}, K in {2,4,16},
    T in {0,1}, 50-200 iterations, damping 0.5) drawn from 48 seeded templates; the
    continuous server (admission by slots and memory) against the FIFO baseline (one
    request at a time) on the same arrivals, and a load sweep."""
    templates = W.serving_templates(seed=0)
    descs = [binding.marshal_desc(p.graph) for p in templates]
    budget = 40 << 30
    rate, dur = args.serve_rate, args.serve_duration
    out = {"workload": "Poisson arrivals of Ising / Potts grid requests: side U{16..512}, K in {2,4,16}, "
                       "T in {0,1}, 50-200 iterations, damping 0.5 (48 seeded templates)",
           "rate_req_s": rate, "duration_s": dur, "slots": args.serve_slots, "memory_budget_bytes": budget,
           "latency": "submission to results in host memory", "unit": UNIT}
    warm = W.poisson_arrivals(99, 200.0, 0.1, len(templates))
    serve_run(binding, templates, descs, warm, args.serve_slots, budget)
    arr = W.poisson_arrivals(1, rate, dur, len(templates))
    out["continuous"] = serve_run(binding, templates, descs, arr, args.serve_slots, budget)
    out["fifo"] = serve_run(binding, templates, descs, arr, 1, budget)
    # f4: the same arrivals, each request stopping once its residual is <= 1e-4
    out["continuous_early_exit"] = serve_run(binding, templates, descs, arr, args.serve_slots, budget, tol=1e-4)
    out["continuous_early_exit"]["tol"] = 1e-4
    # a load sweep around the measured capacity (requests served per second while
    # saturated): at 0.25 / 0.5 / 0.75 of it the server keeps up (span close to the arrival
    # window), so p50 / p99 there are service latencies rather than queueing
    cap = out["continuous"]["served_req_s"] or rate
    out["capacity_req_s"] = cap
    out["sweep"] = []
    for f in (0.25, 0.5, 0.75, 1.0):
        a = W.poisson_arrivals(2, cap * f, dur, len(templates))
        r = serve_run(binding, templates, descs, a, args.serve_slots, budget)
        r["rate_req_s"] = round(cap * f, 1)
        r["fraction_of_capacity"] = f
        out["sweep"].append(r)
        if f == 0.25:  # with early exit (tol 1e-4) at the lowest load
            r = serve_run(binding, templates, descs, a, args.serve_slots, budget, tol=1e-4)
            r["rate_req_s"] = round(cap * f, 1)
            r["fraction_of_capacity"] = f
            r["tol"] = 1e-4
            out["sweep"].append(r)
    return out


def run_ours(args):
    import numpy as np
    import torch

    world, rank, local = dist_setup()
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        dist = None
        torch.cuda.set_device(0)
    dev = torch.device("cuda", torch.cuda.current_device())

    from paper_2202_04110_gb300 import binding, build
    from paper_2202_04110_gb300 import workloads as W
    build.build()
    p = W.ising_large(seed=rank, T=1.0, side=args.side, n_iters=args.iters)
    g = binding.Graph(p.graph)
    I = g.info
    lp = torch.as_tensor(p.log_pot).to(dev)
    ev = torch.as_tensor(p.evidence).to(dev)
    msgs = g.new_msgs()
    bel = torch.empty(I["n_var_states"], dtype=torch.float32, device=dev)
    dec = torch.empty(I["n_vars"], dtype=torch.int32, device=dev)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()
    temps = (1.0, 0.0)

    run_events = []  # CUDA events around each run (one CUDA graph replay) of the timed steps

    def step(record=False):
        for T in temps:
            msgs.zero_()
            if record:
                r0 = torch.cuda.Event(enable_timing=True)
                r1 = torch.cuda.Event(enable_timing=True)
                r0.record(stream)
            g.run_bp(lp, ev, T, 0.5, args.iters, msgs)
            if record:
                r1.record(stream)
                run_events.append((r0, r1))
            g.beliefs(ev, msgs, True, out=bel)
            g.decode(ev, msgs, out=dec)

    # clocks: nvidia-smi samples from before the warm-up on, kept inside the timed window
    sampler = ClockSampler(torch.cuda.current_device())
    sampler.start()
    # per-pass timing inside the timed runs: the captured CUDA graphs record events
    # around the variable and factor passes of every PROFILE_PERIOD-th iteration
    g.set_profiling(min(PROFILE_PERIOD, args.iters))
    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    g.pass_times()  # reset
    ES = I["n_edge_states"]
    updates_per_step = len(temps) * args.iters * ES
    # log-ratio iterations (binary pairwise graph): one number per edge during the run;
    # per run one pack, one table-differences and one unpack launch
    lr_min = g.get_option(binding.OPT_LOG_RATIO)
    lr = lr_min > 0 and args.iters >= lr_min
    launches_per_step = len(temps) * (args.iters * I["launches_per_iter"] + 2 + (3 if lr else 0))

    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    t_start = time.time()
    step_ms = []
    for _ in range(args.steps):
        flush.fill_(1.0)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        step(record=True)
        e1.record(stream)
        step_ms.append((e0, e1))
    torch.cuda.synchronize()
    sampler.mark(t_start, time.time())
    if dist is not None:
        dist.barrier()
    clocks = sampler.stop()
    var_ms, fac_ms, n_var, n_fac = g.pass_times()
    g.set_profiling(0)
    ms = [a.elapsed_time(b) for a, b in step_ms]
    total_ms, value = aggregate_ranks(dist, float(sum(ms)), updates_per_step * args.steps, dev)
    flags = g.flags(clear=True)

    # roofline of the dominant kernel: algorithmic bytes per launch / mean launch time
    V, VS, E = I["n_vars"], I["n_var_states"], I["n_edges"]
    n_cfg_total = 4 * I["n_factors"]
    F = I["n_factors"]
    if lr and I["max_degree"] <= 4:  # log-ratios in 4 slots per variable; per-variable totals Dv
        S = 4 * V
        fac_bytes = 4 * (E + 2 * E + 3 * F) + 8 * V  # slot index + d read/write + table differences + Dv
        var_bytes = 4 * (S + VS) + 8 * V             # d + evidence + Dv write (no index)
    elif lr:  # log-ratios in CSR order
        fac_bytes = 4 * (E + E + 2 * E + 3 * F)  # slot index + lam gather + d read/write + table differences
        var_bytes = 4 * (E + VS + E)             # d + evidence + lam write
    else:
        fac_bytes = 4 * (2 * ES + n_cfg_total + E + VS)  # m_old + m_new + log-potentials + edge index + beliefs
        var_bytes = 4 * (ES + 2 * VS + E)               # messages + evidence + beliefs + incoming-edge index
    # the method's minimum traffic per iteration (8 ES + 4 sum n_cfg + 4 VS + 4 E), split
    # into the factor pass's share (its messages, log-potentials and edge index) and the
    # variable pass's (evidence); the bytes the implementation above moves are reported
    # beside it (the log-ratio encoding keeps one number per edge and direction)
    impl_fac_bytes, impl_var_bytes = fac_bytes, var_bytes
    fac_bytes = sec8d_bytes(p.graph, [0])
    var_bytes = 4 * VS
    fac_avg_s = fac_ms / 1e3 / max(n_fac, 1)
    var_avg_s = var_ms / 1e3 / max(n_var, 1)
    peak, peak_src = measured_peaks()
    wl = f"ising{args.side}x{args.side}"
    fac_gbs = fac_bytes / fac_avg_s / 1e9
    var_gbs = var_bytes / var_avg_s / 1e9
    iter_bytes = fac_bytes + var_bytes
    run_ms = [a.elapsed_time(b) for a, b in run_events]
    iter_run_s = statistics.mean(run_ms) / 1e3 / args.iters  # includes the run's pack / unpack
    iter_s = (var_ms + fac_ms) / 1e3 / max(n_fac, 1)
    if lr:
        fac_name, var_name = "k_pair2_lr", ("k_var_slot4_lr" if I["max_degree"] <= 4 else "k_var_csr_lr")
    else:
        fac_name, var_name = "k_pair2", "variable_pass"
    fac_dom = fac_ms >= var_ms
    dominant, other = (fac_name, var_name) if fac_dom else (var_name, fac_name)
    dom_gbs, oth_gbs = (fac_gbs, var_gbs) if fac_dom else (var_gbs, fac_gbs)
    dom_bytes, oth_bytes = (fac_bytes, var_bytes) if fac_dom else (var_bytes, fac_bytes)
    dom_impl, oth_impl = (impl_fac_bytes, impl_var_bytes) if fac_dom else (impl_var_bytes, impl_fac_bytes)
    dom_s, oth_s = (fac_avg_s, var_avg_s) if fac_dom else (var_avg_s, fac_avg_s)
    roof = {"bound": "hbm", "kernel": dominant,
            "achieved": round(dom_gbs, 1),
            "peak": peak, "unit": "GB/s", "peak_source": f"{peak_src} HBM copy bandwidth",
            "frac": round(dom_gbs / peak, 4),
            "traffic": profiled_traffic(dominant, wl),
            "algorithmic_bytes_per_launch": dom_bytes,
            "algorithmic_bytes": "the factor pass's share of the per-iteration minimum 8 ES + 4 sum n_cfg + "
                                 "4 VS + 4 E (8 ES + 4 sum n_cfg + 4 E); the variable pass's share is 4 VS",
            "implementation_bytes_per_launch": dom_impl,
            "implementation_frac": round(dom_impl / dom_s / 1e9 / peak, 4),
            "mean_launch_us": round(1e6 * dom_s, 2),
            "other_kernels": {
                other: {"achieved": round(oth_gbs, 1), "frac": round(oth_gbs / peak, 4),
                        "algorithmic_bytes_per_launch": oth_bytes,
                        "implementation_bytes_per_launch": oth_impl,
                        "implementation_frac": round(oth_impl / oth_s / 1e9 / peak, 4),
                        "mean_launch_us": round(1e6 * oth_s, 2),
                        "traffic": profiled_traffic(other, wl)}},
            "kernel_timing": "CUDA events on the launching stream around the passes of every "
                             f"{min(PROFILE_PERIOD, args.iters)}th iteration of the timed runs (event nodes in their CUDA graphs)",
            "nominal_peak": NOMINAL_HBM_GBS, "frac_of_nominal": round(dom_gbs / NOMINAL_HBM_GBS, 4),
            "iteration": {"algorithmic_bytes": iter_bytes,
                          "implementation_bytes": impl_fac_bytes + impl_var_bytes,
                          "mean_us": round(1e6 * iter_run_s, 2),
                          "achieved": round(iter_bytes / iter_run_s / 1e9, 1),
                          "frac": round(iter_bytes / iter_run_s / 1e9 / peak, 4),
                          "frac_of_nominal": round(iter_bytes / iter_run_s / 1e9 / NOMINAL_HBM_GBS, 4),
                          "timing": "CUDA events around each pgm_run_bp call (one CUDA graph replay) "
                                    "of the timed steps / iterations; both passes back to back",
                          "sum_of_pass_events_us": round(1e6 * iter_s, 2)}}

    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": workload_config(args, world), "roofline": roof, "clocks": clocks,
            "gpu_launches": launches_per_step * args.steps, "device_flags": flags,
            "step_ms": [round(x, 3) for x in ms]}

    # end to end through the host-buffer C-ABI call (copies inside the timed region)
    if not args.no_e2e:
        lp_h = torch.empty(p.log_pot.size, dtype=torch.float32, pin_memory=True).numpy()
        ev_h = torch.empty(p.evidence.size, dtype=torch.float32, pin_memory=True).numpy()
        lp_h[:] = p.log_pot
        ev_h[:] = p.evidence
        bel_h = torch.empty(VS, dtype=torch.float32, pin_memory=True).numpy()
        dec_h = torch.empty(V, dtype=torch.int32, pin_memory=True).numpy()

        def e2e_step():
            for T in temps:
                g.infer_host(lp_h, ev_h, T, 0.5, args.iters, bel_h, dec_h)

        for _ in range(max(1, args.warmup)):
            e2e_step()
        if dist is not None:
            dist.barrier()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            e2e_step()
        dt = time.perf_counter() - t0
        if dist is not None:
            t = torch.tensor([dt], device=dev)
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            dt = float(t.item())
        line["e2e"] = {"value": world * updates_per_step * args.steps / dt, "unit": UNIT,
                       "h2d_bytes_per_step": len(temps) * 4 * (p.log_pot.size + p.evidence.size),
                       "d2h_bytes_per_step": len(temps) * 4 * (VS + V),
                       "call": "pgm_infer_host (pinned host buffers, blocking)"}

    # the further sections are single-GPU measurements: run at N = 1 only (at N > 1 the
    # line reports the replicas' headline)
    if not args.no_batch and world == 1:
        line["batched"] = measure_batched(args, binding, W, torch, dev)
    if not args.no_multi and world == 1:
        line["multi_evidence"] = measure_multi(args, binding, W, torch, dev)
    if not args.no_deconv and world == 1:
        line["deconvolution"] = measure_deconv(args, binding, W, torch, dev)
        line["small_grid"] = measure_small(args, binding, W, torch, dev)
    if not args.no_grad and world == 1:
        line["gradient"] = measure_grad(args, binding, W, torch, dev)
        line["early_exit"] = measure_until(args, binding, W, torch, dev)
        line["large_factors"] = measure_large_enum(args, binding, W, torch, dev)
        line["l2_free"] = measure_l2_free(args, binding, W, torch, dev)
    if not args.no_serve and world == 1:
        line["serving"] = measure_serving(args, binding, W)

    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        v, dt, cores = cpu_sample(p, args.cpu_iters)
        line["cpu_baseline"] = {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle",
                                "sample": f"{args.cpu_iters} iterations at T=1 and {args.cpu_iters} at T=0 on the "
                                          f"full {args.side}x{args.side} grid, FP64, {dt:.1f} s"}
        # the same oracle on one core (a quarter of the sample), for the per-core rate
        import oracle
        n_all = oracle.num_threads()
        oracle.set_num_threads(1)
        v1, dt1, _ = cpu_sample(p, max(1, args.cpu_iters // 4))
        oracle.set_num_threads(n_all)
        line["cpu_baseline"]["single_core"] = {"value": v1, "unit": UNIT, "cores": 1,
                                               "sample": f"{max(1, args.cpu_iters // 4)} iterations per T, "
                                                         f"FP64, {dt1:.1f} s"}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.barrier()
        dist.destroy_process_group()


def batch_probe(args):
    """A short, uncaptured run of the batched workload for ncu captures of its kernels:
    two warm-up runs and one measured run of `--batch-probe` iterations each, CUDA graphs
    off (one launch per kernel per pass). Prints one JSON line with the launch shapes."""
    import torch
    from paper_2202_04110_gb300 import binding, build
    from paper_2202_04110_gb300 import workloads as W
    build.build()
    batch, members = W.potts_rbm_batch(seed=0, n_grids=args.batch_grids, n_iters=100)
    lp = torch.as_tensor(batch.log_pot).cuda()
    ev = torch.as_tensor(batch.evidence).cuda()
    g = binding.Graph([m.graph for m in members])
    g.set_option(binding.OPT_CUDA_GRAPH, 0)
    g.set_option(binding.OPT_PAIR_FORM, args.pair_form)
    m = g.new_msgs()
    for _ in range(3):
        m.zero_()
        g.run_bp(lp, ev, 1.0, 0.5, args.batch_probe, m)
    torch.cuda.synchronize()
    # per-launch CUDA-event times of a fourth run (every iteration sampled)
    g.set_profiling(1)
    m.zero_()
    g.run_bp(lp, ev, 1.0, 0.5, args.batch_probe, m)
    torch.cuda.synchronize()
    lt = g.launch_times()
    g.set_profiling(0)
    times = [round(1e3 * ms / cnt, 2) if cnt else None for ms, cnt in lt]
    print(json.dumps({"batch_probe": args.batch_probe, "pair_form": args.pair_form,
                      "launches_per_iter": g.info["launches_per_iter"], "launch_shapes": g.launches(),
                      "mean_launch_us": times}))


def deconv_probe(args):
    """A short, uncaptured run of the deconvolution workload (T=0, damping 0.5) for ncu
    captures of its kernels: three runs of `--deconv-probe` iterations, CUDA graphs off.
    Prints one JSON line with the launch shapes."""
    import torch
    from paper_2202_04110_gb300 import binding, build
    from paper_2202_04110_gb300 import workloads as W
    build.build()
    p = W.deconvolution(0, n_iters=args.deconv_probe)
    ev = torch.as_tensor(p.evidence).cuda()
    g = binding.Graph(p.graph)
    g.set_option(binding.OPT_CUDA_GRAPH, 0)
    m = g.new_msgs()
    for _ in range(3):
        m.zero_()
        g.run_bp(None, ev, 0.0, 0.5, args.deconv_probe, m)
    torch.cuda.synchronize()
    print(json.dumps({"deconv_probe": args.deconv_probe, "launches_per_iter": g.info["launches_per_iter"],
                      "launch_shapes": g.launches()}))


def small_probe(args):
    """`--small-probe N` runs of the 10x10 Ising workload (T=1, damping 0.5, 50
    iterations: one k_lr_small launch each), or of a `--small-side` grid (one k_lr_small
    or k_lr_cluster launch each), CUDA graphs off, for ncu captures of the one-launch
    run. Prints one JSON line."""
    import torch
    from paper_2202_04110_gb300 import binding, build
    from paper_2202_04110_gb300 import workloads as W
    build.build()
    p = W.ising_small(0) if args.small_side == 10 else W.ising_grid(args.small_side, args.small_side, 0, T=1.0)
    lp = torch.as_tensor(p.log_pot).cuda()
    ev = torch.as_tensor(p.evidence).cuda()
    g = binding.Graph(p.graph)
    g.set_option(binding.OPT_CUDA_GRAPH, 0)
    m = g.new_msgs()
    for _ in range(args.small_probe):
        m.zero_()
        g.run_bp(lp, ev, 1.0, 0.5, p.n_iters, m)
    torch.cuda.synchronize()
    print(json.dumps({"small_probe": args.small_probe, "side": args.small_side,
                      "small_run": g.get_option(binding.OPT_SMALL_RUN),
                      "n_edge_states": g.info["n_edge_states"]}))


def grad_probe(args):
    """`--grad-probe N` gradient calls of the gradient workload (64x64 Ising, T=1, damping
    0.5, 100 iterations, a checkpoint every 10), CUDA graphs off, for an ncu launch list of
    the reverse pass. Prints one JSON line with the launches per call."""
    import numpy as np
    import torch
    from paper_2202_04110_gb300 import binding, build
    from paper_2202_04110_gb300 import workloads as W
    build.build()
    p = W.ising_grid(64, 64, 0, T=1.0, n_iters=100)
    g = binding.Graph(p.graph)
    g.set_option(binding.OPT_CUDA_GRAPH, 0)
    lp = torch.as_tensor(p.log_pot).cuda()
    ev = torch.as_tensor(p.evidence).cuda()
    gnb = torch.as_tensor(np.random.default_rng(1).standard_normal(p.graph.n_var_states).astype(np.float32)).cuda()
    for _ in range(args.grad_probe):
        g.grad(lp, ev, 1.0, 0.5, 100, 10, gnb)
    torch.cuda.synchronize()
    print(json.dumps({"grad_probe": args.grad_probe, "workload": "ising64x64, T=1, damping 0.5, 100 iterations, "
                      "checkpoint every 10", "launches_per_iter": g.info["launches_per_iter"]}))


def pool_probe(args):
    """A short, uncaptured run of a pool grid (`--pool-probe SIDE,RADIUS,SLACK`, T=0,
    damping 0.5) for ncu captures of the block-form enumeration kernel: three runs of 10
    iterations, CUDA graphs off. Prints one JSON line with the launch shapes."""
    import torch
    from paper_2202_04110_gb300 import binding, build
    from paper_2202_04110_gb300 import workloads as W
    build.build()
    side, radius, slack = (int(x) for x in args.pool_probe.split(","))
    p = W.pool_grid(side, radius, slack, 0, T=0.0, n_iters=10)
    lp = torch.as_tensor(p.log_pot).cuda()
    ev = torch.as_tensor(p.evidence).cuda()
    g = binding.Graph(p.graph)
    g.set_option(binding.OPT_CUDA_GRAPH, 0)
    m = g.new_msgs()
    for _ in range(3):
        m.zero_()
        g.run_bp(lp, ev, 0.0, 0.5, 10, m)
    torch.cuda.synchronize()
    print(json.dumps({"pool_probe": args.pool_probe, "n_factors": g.info["n_factors"],
                      "n_edge_states": g.info["n_edge_states"], "launch_shapes": g.launches()}))


def main():
    args = parse_args()
    if args.pool_probe:
        pool_probe(args)
    elif args.deconv_probe:
        deconv_probe(args)
    elif args.batch_probe:
        batch_probe(args)
    elif args.grad_probe:
        grad_probe(args)
    elif args.small_probe:
        small_probe(args)
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
