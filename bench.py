#!/usr/bin/env python
"""Benchmark of the per-step heat solve (IMEX Euler, Section 2) on the starfish workload:
unit disk minus 5 starfish holes (N_Gamma = 6 x 1024), adaptive quadtree to level 8 with
8 x 8 nodes per leaf (N_D = 257,728), Gaussian-sum forcing, dt = alpha^2 = 1e-3, p = 20.

One step = heat_step: B -> volume potential (adaptive multipole method) -> leaf
interpolation onto Gamma -> GMRES on the Nystrom system (tol 1e-10) -> double layer at
the nodes in Omega -> combine.  Metric: points * timesteps / s, points = N_D + N_Gamma.

  python bench.py [--gpus N --steps K --warmup W] [--prec mixed|fp64]
                  [--warm learned|previous|secant|zero] [--impl reference]

Default form: mixed precision with the learned GMRES start.  The network is trained before
the timed region on this geometry (2000 pairs from trajectories of 100 other Gaussian-sum
forcings, 200 validation pairs; reported under warm_start, not timed); the benchmark's own
forcing is not among them.

Timing: W untimed warm-up steps, then K steps, each bracketed by CUDA events on the
library's stream; between timed steps a 256 MB buffer is written (L2 flush, untimed).
`e2e` repeats the K steps, from the state the timed steps started in (so with the same GMRES
work), through the public API with host buffers: the step's inputs
(u, F, f, packed in one pinned buffer) are copied from host memory and the result u^{N+1}
is copied back inside the timed region.  With N > 1 (torchrun) every rank runs its own replica of the
problem (the single-problem path does not shard), the time is the max over ranks and
the value sums the points of all ranks.  --impl reference times the CPU oracle on a
bounded sample of the same workload (rank 0 only).
"""
import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import mh_workloads as W  # noqa: E402

METRIC = "points*timesteps/s per GB300 at rel-L2 err<=1e-6 vs FP64 oracle; % of roofline"
FP64_PEAK_TFLOPS = 1.25     # nominal GB300 binary64 rate (all pipes)
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12   # 152 SMs x 128 FP32 lanes x FMA x 2.07 GHz


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return json.load(fh)
    except OSError:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0, "fallback": True}


# where ClockSampler keeps its raw nvidia-smi samples (--clocks-dir); the summary goes into the JSON line
CLOCKS_DIR = tempfile.gettempdir()


class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""

    def __init__(self, device):
        self.device = device
        self.proc = None
        self.path = os.path.join(CLOCKS_DIR, f"clocks_{os.getpid()}.csv")

    def __enter__(self):
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={q}", "--format=csv,noheader,nounits",
                                          "-i", str(self.device), "-lms", "50"], stdout=self.fh,
                                         stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            self.fh.close()

    def summary(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as fh:
            for line in fh:
                f = [x.strip() for x in line.split(",")]
                if len(f) < 9:
                    continue
                try:
                    sm.append(float(f[1]))
                    mx = float(f[2])
                except ValueError:
                    continue
                for nm, v in zip(names, f[5:9]):
                    if v.lower().startswith("active"):
                        reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def aggregate_over_ranks(local_ms: float, points_per_rank: int, steps: int, dist=None, device=None):
    """Whole-job throughput of N independent replicas: the time is the maximum over ranks
    (each rank times its own K steps), the work is the sum of every rank's points * steps.
    Returns (value, max_ms)."""
    import torch
    total_ms = float(local_ms)
    world = 1
    if dist is not None and dist.is_initialized():
        world = dist.get_world_size()
        t = torch.tensor([total_ms], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total_ms = float(t.item())
    return points_per_rank * steps * world / (total_ms / 1e3), total_ms


def setup_problem(mh, ctx, wl, torch, dev):
    t0 = time.time()
    tree = mh.Tree(ctx, wl.box, wl.q, wl.min_level, wl.max_level, wl.forcing, wl.refine_tol)
    bnd = mh.Boundary(ctx, wl.curves, alpert_order=8)
    prob = mh.Problem(ctx, tree, bnd, wl.dt, wl.p, ext_mode=mh.MH_EXT_CONST, ext_const=wl.ext_const)
    torch.cuda.synchronize(dev)
    nodes = tree.nodes().cpu().numpy()
    F = wl.forcing(nodes)
    return tree, bnd, prob, nodes, F, time.time() - t0


def run_ours(args):
    import torch
    import paper_1007_5335_gb300 as mh

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device(f"cuda:{local}"))
    torch.cuda.set_device(local)
    dev = torch.device(f"cuda:{local}")
    wl = W.starfish_domain()
    prec = mh.MH_PREC_MIXED if args.prec == "mixed" else mh.MH_PREC_FP64
    ctx = mh.Context(local)
    tree, bnd, prob, nodes, F_np, t_setup = setup_problem(mh, ctx, wl, torch, dev)
    n_pts = tree.n_nodes + bnd.n
    F = torch.tensor(F_np, device=dev)
    f_next = torch.zeros(bnd.n, dtype=torch.float64, device=dev)     # f = 0 on every curve
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)

    # graph form (default): the step of this one problem is one CUDA graph launch through the
    # batch API (mh_batch_step), GMRES included (device-side loops, no host round trips); the
    # graph is recorded on fixed arrays at the first call
    batch = mh.Batch(ctx, [prob]) if args.graph else None
    ub = torch.zeros(tree.n_nodes, dtype=torch.float64, device=dev)
    sb = torch.zeros(bnd.n, dtype=torch.float64, device=dev)

    def run_steps(k, u, sigma, timed, prec_, graph=False):
        un = torch.empty_like(u)
        times, its = [], []
        if graph:
            ub.copy_(u)
            sb.copy_(sigma)
        for _ in range(k):
            if timed:
                flush.zero_()
                a = torch.cuda.Event(enable_timing=True)
                b = torch.cuda.Event(enable_timing=True)
                a.record()
            if graph:
                info = batch.step([ub], [F], [f_next], [sb], gmres_tol=1e-10, prec=prec_)[0]
            else:
                info = mh.heat_step(ctx, prob, u, F, f_next, un, sigma, gmres_tol=1e-10, prec=prec_)
            if timed:
                b.record()
                b.synchronize()
                times.append(a.elapsed_time(b))
            its.append(info.gmres_iterations)
            if not graph:
                u, un = un, u
        if graph:
            u.copy_(ub)
            sigma.copy_(sb)
        return u, times, its

    # learned start: trained on this geometry from solver trajectories of other forcings
    warm_modes = {"learned": mh.MH_WARM_LEARNED, "previous": mh.MH_WARM_PREVIOUS, "secant": mh.MH_WARM_SECANT,
                  "zero": mh.MH_WARM_ZERO}
    warm_mode = warm_modes[args.warm]
    net, warm_info = None, {"mode": args.warm}
    if warm_mode == mh.MH_WARM_LEARNED:
        net, warm_info = train_warm_start(mh, ctx, prob, bnd, nodes, f_next, prec, dev)

    def set_start(mode):
        prob.set_warm_start(mode, net, mh.MH_NET_BF16X2)

    # near-field tile: the fastest of the autotuner's three shapes on a few untimed steps
    tile_ms = {}
    for tile in (128, 256, 512):
        prob.set_near_tile(tile)
        ut = torch.zeros(tree.n_nodes, dtype=torch.float64, device=dev)
        st_ = torch.zeros(bnd.n, dtype=torch.float64, device=dev)
        _, tt, _ = run_steps(3, ut, st_, True, prec)
        tile_ms[tile] = float(np.median(tt))
    near_tile = min(tile_ms, key=tile_ms.get)
    prob.set_near_tile(near_tile)

    # accuracy of the headline form (precision + start) against the plain FP64 path
    # (previous-step start), same steps from u = 0
    u0 = torch.zeros(tree.n_nodes, dtype=torch.float64, device=dev)
    err = None
    if args.check_steps > 0 and (prec == mh.MH_PREC_MIXED or warm_mode != mh.MH_WARM_PREVIOUS):
        s64 = torch.zeros(bnd.n, dtype=torch.float64, device=dev)
        s32 = torch.zeros(bnd.n, dtype=torch.float64, device=dev)
        set_start(mh.MH_WARM_PREVIOUS)
        u64, _, _ = run_steps(args.check_steps, u0.clone(), s64, False, mh.MH_PREC_FP64)
        set_start(warm_mode)
        u32, _, _ = run_steps(args.check_steps, u0.clone(), s32, False, prec, args.graph)
        regions = prob.regions()
        ins = torch.tensor(regions == -1, device=dev)
        err = float(torch.linalg.norm((u32 - u64)[ins]) / torch.linalg.norm(u64[ins]))
    # GMRES iterations of the same steps with the previous-step start (context, untimed)
    if warm_mode != mh.MH_WARM_PREVIOUS:
        set_start(mh.MH_WARM_PREVIOUS)
        sp = torch.zeros(bnd.n, dtype=torch.float64, device=dev)
        _, _, its_prev = run_steps(args.warmup + args.steps, u0.clone(), sp, False, prec)
        warm_info["previous_start_gmres_iterations_mean"] = float(np.mean(its_prev[args.warmup:]))
    set_start(warm_mode)

    sigma = torch.zeros(bnd.n, dtype=torch.float64, device=dev)
    u, _, _ = run_steps(args.warmup, u0.clone(), sigma, False, prec, args.graph)
    launches0 = ctx.launches
    # the state the timed steps start from: the end-to-end steps below replay the same
    # trajectory from it (same solution, same previous density, so the same GMRES work; the
    # iteration count falls as the run goes on, and later steps would be cheaper)
    u_start, sigma_start = u.clone(), sigma.clone()
    if dist:
        dist.barrier()
    torch.cuda.synchronize(dev)
    with ClockSampler(local) as clk:
        torch.cuda.nvtx.range_push("timed_steps")      # lets a profiler select the timed region
        u, times, its = run_steps(args.steps, u, sigma, True, prec, args.graph)
        torch.cuda.nvtx.range_pop()
    torch.cuda.synchronize(dev)
    launches = ctx.launches - launches0
    value, total_ms = aggregate_over_ranks(sum(times), n_pts, args.steps, dist, dev)
    # the same number of steps again with the library's region timers on (a CUDA event pair on
    # the library's stream around every region): per-kernel durations for the roofline.  Kept
    # out of the headline region, whose steps run without the extra event records.
    ctx.profile(True)
    ctx.profile_read("gmres", reset=True)
    torch.cuda.synchronize(dev)
    with ClockSampler(local) as clk_prof:
        u, times_prof, _ = run_steps(args.steps, u, sigma, True, prec)
    torch.cuda.synchronize(dev)
    regions_ms = {}
    for r in REGION_NAMES:
        regions_ms[r] = ctx.profile_read(r)
    ctx.profile(False)
    # end to end through the API with host buffers: the step's inputs u, F, f sit in one pinned
    # host buffer and go over in one copy (one 4.2 MB copy costs less than three)
    nn_, ng_ = tree.n_nodes, bnd.n
    in_h = torch.empty(2 * nn_ + ng_, dtype=torch.float64).pin_memory()
    in_h[:nn_].copy_(u_start.cpu())
    in_h[nn_:2 * nn_].copy_(torch.from_numpy(F_np))
    in_h[2 * nn_:].zero_()
    u_h = in_h[:nn_]
    out_h = torch.empty(nn_, dtype=torch.float64).pin_memory()
    in_d = torch.empty(2 * nn_ + ng_, dtype=torch.float64, device=dev)
    ud, Fd, fd = in_d[:nn_], in_d[nn_:2 * nn_], in_d[2 * nn_:]
    und = torch.empty_like(u)
    e2e_batch = None
    if args.graph:   # the graph of the host-buffer form is recorded on these arrays (untimed)
        del batch
        e2e_batch = mh.Batch(ctx, [prob])
        ud.copy_(u)
        e2e_batch.step([ud], [Fd], [fd], [sigma], gmres_tol=1e-10, prec=prec)
    sigma.copy_(sigma_start)
    e2e_times, e2e_its = [], []
    for _ in range(args.steps):
        flush.zero_()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record()
        in_d.copy_(in_h, non_blocking=True)
        if args.graph:
            info = e2e_batch.step([ud], [Fd], [fd], [sigma], gmres_tol=1e-10, prec=prec)[0]
            out_h.copy_(ud, non_blocking=True)
        else:
            info = mh.heat_step(ctx, prob, ud, Fd, fd, und, sigma, gmres_tol=1e-10, prec=prec)
            out_h.copy_(und, non_blocking=True)
        b.record()
        b.synchronize()
        e2e_times.append(a.elapsed_time(b))
        e2e_its.append(info.gmres_iterations)
        u_h.copy_(out_h)
    e2e_value, e2e_ms = aggregate_over_ranks(sum(e2e_times), n_pts, args.steps, dist, dev)
    bytes_in = (2 * tree.n_nodes + bnd.n) * 8
    bytes_out = tree.n_nodes * 8
    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return
    peaks = _peaks()
    roof = roofline(regions_ms, tree, bnd, prob, prec, mh, peaks, args.steps)
    line = {
        "metric": METRIC,
        "value": value,
        "unit": "points*timesteps/s",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": total_ms / args.steps,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f32+f64" if prec == mh.MH_PREC_MIXED else "f64",
        "data": "synthetic",
        "config": {"workload": "starfish_domain: unit disk minus 5 starfish holes, N_Gamma=6144, "
                               "N_D=%d (adaptive tree levels 4-8, 8x8 GL nodes per leaf), dt=alpha^2=1e-3, p=20, "
                               "IMEX Euler, GMRES tol 1e-10" % tree.n_nodes,
                   "points": n_pts, "n_gamma": bnd.n, "n_d": tree.n_nodes, "precision": args.prec,
                   "l2": "flushed between timed steps (256 MB write, untimed)", "near_tile": near_tile,
                   "step_form": ("one CUDA graph launch per step (mh_batch_step of this problem)" if args.graph
                                 else "heat_step on the stream"),
                   "parallelism": "replicas" if world > 1 else "single"},
        "rel_l2_vs_fp64_path": err,
        "gmres_iterations": its,
        "warm_start": dict(warm_info, gmres_iterations_mean=float(np.mean(its))),
        "setup_s": t_setup,
        "e2e": {"value": e2e_value, "unit": "points*timesteps/s", "h2d_bytes_per_step": bytes_in,
                "d2h_bytes_per_step": bytes_out, "start": "the timed steps' starting state",
                "gmres_iterations_mean": float(np.mean(e2e_its))},
        "gpu_launches": launches,
        "profiled_ms_per_step": float(np.mean(times_prof)),
        "profiled_clocks": clk_prof.summary(),
        "regions_ms_per_step": {k: v[0] / args.steps for k, v in regions_ms.items()},
        "kernel_launches_per_step": {k: v[1] / args.steps for k, v in regions_ms.items()},
        "roofline": roof,
        "clocks": clk.summary(),
    }
    if args.cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(wl, budget_s=args.cpu_budget)
    print(json.dumps(line))
    if dist:
        dist.destroy_process_group()


# region: (bound, pipe, what); regions are timed by the library (mh_profile_read) with the
# algorithmic work it declares per launch: GEMV 4n^2 + 12n bytes (binary32) / 2n^2 flop;
# pair sums 68 flop per pair; contractions 2 R C flop per task.
KERNEL_REGIONS = {
    "bie_gemv32": ("hbm", None, "Nystrom operator GEMV, binary32 (Arnoldi iterations)"),
    "bie_gemv64": ("alu", "fp64", "Nystrom operator GEMV, binary64 (residuals, learned-start judge)"),
    "bie_gemvff": ("hbm", None, "Nystrom operator GEMV, float-float on A32 + a binary16 low part (mixed-precision "
                                "residuals, learned-start judge)"),
    "dlp_near": ("alu", "auto", "double-layer near-field pair sums (fine dipoles of neighbour leaves)"),
    "dlp_fine": ("alu", "auto", "16x upsampled pair sums at the normal-line auxiliary points"),
    "dlp_coarse": ("alu", "auto", "trapezoid pair sums"),
    "volume_contract": ("alu", "auto", "volume multipole contractions (near tables, P2M, M2L + P2L, L2P + M2P)"),
    "volume_chain": ("alu", "auto", "volume M2M / L2L level chains"),
    "dlp_fmm_contract": ("alu", "auto", "double-layer multipole contractions (dipole P2M, M2L + P2L, L2P + M2P)"),
    "dlp_fmm_chain": ("alu", "auto", "double-layer M2M / L2L level chains"),
    "volume_contract_tc": ("hbm", None, "volume contractions on the tensor cores (k_contract_tc: TF32 head/tail "
                                        "MMAs; binary32 sources, operators and products)"),
    "dlp_fmm_contract_tc": ("hbm", None, "double-layer contractions on the tensor cores (k_contract_tc)"),
}
# Regions that time a whole phase of several kernels (tensor-core launch, CUDA-core chunks of the
# operators with few tasks, ordered reduction): reported, but not candidates for the dominant
# kernel, which is the single-kernel region with the most time per step.
PHASE_REGIONS = {"volume_contract", "dlp_fmm_contract"}
# DRAM bytes (read + write) per launch of a region's kernel, from one-kernel ncu captures of the
# current kernels at the sizes the bench runs (dram__bytes_read.sum + dram__bytes_write.sum);
# the tensor-core figure is the mean over the four volume launches of one potential.
NCU_TRAFFIC = {"bie_gemv32": 153.77e6, "bie_gemvff": 230.31e6, "dlp_near": 19.97e6, "dlp_fine": 2.12e6,
               "volume_contract_tc": 4.71e6}
REGION_NAMES = tuple(KERNEL_REGIONS) + ("volume_apply", "dlp_fmm", "gmres", "dlp_evaluate", "warm_start", "warm_net",
                                        "bie_gemv64_gated")


def region_roofline(name, v, prec, mh, peaks):
    ms, launches, flops, nbytes = v
    bound, pipe, desc = KERNEL_REGIONS[name]
    avg_s = ms / max(launches, 1) / 1e3
    out = {"kernel": name, "what": desc, "bound": bound, "avg_launch_ms": avg_s * 1e3, "launches": launches,
           "traffic": NCU_TRAFFIC.get(name)}
    if bound == "hbm":
        achieved = nbytes / launches / avg_s / 1e9
        peak = peaks["hbm_gbs"]
        out.update({"achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                    "bytes_per_launch": nbytes / launches,
                    "peak_source": "measured (MEASURED_PEAKS.json hbm_gbs)"})
        if flops:
            out["tflops"] = flops / launches / avg_s / 1e12
    else:
        fp64 = pipe == "fp64" or (pipe == "auto" and prec != mh.MH_PREC_MIXED)
        achieved = flops / launches / avg_s / 1e12
        peak = FP64_PEAK_TFLOPS if fp64 else FP32_PEAK_TFLOPS
        out.update({"achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                    "flops_per_launch": flops / launches,
                    "peak_source": ("derived: binary64 nominal 1.25 TFLOP/s" if fp64 else
                                    "derived: binary32 152 SMs x 128 lanes x 2 flop x 2.07 GHz = 80.5 TFLOP/s")})
    return out


def roofline(regions_ms, tree, bnd, prob, prec, mh, peaks, steps):
    """Roofline of the dominant (longest) instrumented kernel region, and of every region."""
    cand = {k: v for k, v in regions_ms.items() if k in KERNEL_REGIONS and v[1] > 0}
    name = max((k for k in cand if k not in PHASE_REGIONS), key=lambda k: cand[k][0])
    dom = region_roofline(name, cand[name], prec, mh, peaks)
    dom["all_regions"] = {k: {kk: (round(vv, 4) if isinstance(vv, float) else vv)
                              for kk, vv in region_roofline(k, v, prec, mh, peaks).items()
                              if kk in ("bound", "avg_launch_ms", "achieved", "peak", "unit", "frac", "tflops")}
                          for k, v in sorted(cand.items(), key=lambda kv: -kv[1][0])}
    return dom


def train_warm_start(mh, ctx, prob, bnd, nodes, f_next, prec, dev, steps_per_forcing=20, adam_steps=200):
    """Network of the learned start: 2000 training pairs (100 Gaussian-sum forcings x 20 steps
    from u = 0, previous-step start), 200 validation pairs, closed-form start + Adam."""
    import torch
    from paper_1007_5335_gb300 import warmstart as wsg
    t0 = time.time()
    net = mh.Net(ctx, bnd, 256, 256)
    forc = lambda seeds: [torch.tensor(W.gaussian_forcing(s)(nodes), device=dev) for s in seeds]
    X, Y, _ = wsg.collect_samples(ctx, prob, net, forc(W.WARM_TRAIN_SEEDS), steps_per_forcing, f_next, prec=prec)
    Xv, Yv, _ = wsg.collect_samples(ctx, prob, net, forc(W.WARM_VALID_SEEDS), steps_per_forcing, f_next, prec=prec)
    torch.cuda.synchronize(dev)
    t1 = time.time()
    omega, idx = W.warm_start_draws(X.shape[0], net.width, adam_steps, 64)
    first, best, best_step = wsg.train(net, X, Y, Xv, Yv, torch.tensor(omega, device=dev),
                                       torch.tensor(idx, device=dev))
    torch.cuda.synchronize(dev)
    t2 = time.time()
    return net, {"mode": "learned", "arith": "bf16x2", "train_pairs": int(X.shape[0]), "valid_pairs": int(Xv.shape[0]),
                 "modes_per_curve": net.n_modes, "width": net.width, "sampling_s": t1 - t0, "training_s": t2 - t1,
                 "val_loss_closed_form": first, "val_loss_best": best, "adam_best_step": best_step,
                 "adam_steps": adam_steps}


def run_batch(args):
    """Batched workload: independent problems (1-8 starfish/ellipse holes, 256-2048 nodes per
    curve, alpha^2 log-uniform in [1e-4, 1e-2], adaptive trees) advanced by one CUDA graph launch
    per time step; multipole order and near-field tile from the autotuner per problem."""
    import torch
    import paper_1007_5335_gb300 as mh

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device(f"cuda:{local}"))
    torch.cuda.set_device(local)
    dev = torch.device(f"cuda:{local}")
    prec = mh.MH_PREC_MIXED if args.prec == "mixed" else mh.MH_PREC_FP64
    ctx = mh.Context(local)
    t0 = time.time()
    items, tune_s, choices = [], 0.0, []
    for i in range(args.batch_size):
        wl = W.batch_problem(i)
        tree = mh.Tree(ctx, wl.box, wl.q, wl.min_level, wl.max_level, wl.forcing, wl.refine_tol)
        bnd = mh.Boundary(ctx, wl.curves, alpert_order=8)
        nodes = tree.nodes().cpu().numpy()
        F = torch.tensor(wl.forcing(nodes), device=dev)
        f = torch.zeros(bnd.n, dtype=torch.float64, device=dev)
        p, tile, err = 16, 256, None
        if args.tune:
            t1 = time.time()
            p, tile, rep = mh.mh_autotune(ctx, tree, bnd, wl.dt, F, f, p_cand=(10, 16, 24), err_tol=1e-7, steps=3,
                                          prec=prec)
            tune_s += time.time() - t1
            err = {e.p: e.rel_err for e in rep[:3]}[p]
        prob = mh.Problem(ctx, tree, bnd, wl.dt, p, ext_mode=mh.MH_EXT_CONST, ext_const=wl.ext_const)
        prob.set_near_tile(tile)
        if args.batch_warm == "secant":
            prob.set_warm_start(mh.MH_WARM_SECANT)
        items.append(dict(wl=wl, tree=tree, bnd=bnd, prob=prob, F=F, f=f,
                          u=torch.zeros(tree.n_nodes, dtype=torch.float64, device=dev),
                          s=torch.zeros(bnd.n, dtype=torch.float64, device=dev)))
        choices.append({"p": p, "tile": tile, "alpha2": wl.alpha ** 2, "n_gamma": bnd.n, "n_d": tree.n_nodes,
                        "rel_err_vs_p_ref": err})
    torch.cuda.synchronize(dev)
    setup_s = time.time() - t0 - tune_s
    n_pts = sum(it["tree"].n_nodes + it["bnd"].n for it in items)
    batch = mh.Batch(ctx, [it["prob"] for it in items])
    U = [it["u"] for it in items]
    S = [it["s"] for it in items]
    Fs = [it["F"] for it in items]
    fs = [it["f"] for it in items]
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    for _ in range(args.warmup):                      # the first step records the graph
        batch.step(U, Fs, fs, S, gmres_tol=1e-10, prec=prec)
    times, its = [], []
    launches0 = ctx.launches
    if dist:
        dist.barrier()
    torch.cuda.synchronize(dev)
    with ClockSampler(local) as clk:
        torch.cuda.nvtx.range_push("timed_steps")
        for _ in range(args.steps):
            flush.zero_()
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record()
            infos = batch.step(U, Fs, fs, S, gmres_tol=1e-10, prec=prec)
            b.record()
            b.synchronize()
            times.append(a.elapsed_time(b))
            its.append(float(np.mean([x.gmres_iterations for x in infos])))
        torch.cuda.nvtx.range_pop()
    torch.cuda.synchronize(dev)
    launches = ctx.launches - launches0
    value, total_ms = aggregate_over_ranks(sum(times), n_pts, args.steps, dist, dev)
    # the same problems stepped one at a time with heat_step (host-synchronised GMRES), context
    seq_ms = []
    un = [torch.empty_like(u) for u in U]
    for _ in range(max(1, min(args.steps, 3))):
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record()
        for k, it in enumerate(items):
            mh.heat_step(ctx, it["prob"], U[k], Fs[k], fs[k], un[k], S[k], gmres_tol=1e-10, prec=prec)
            U[k].copy_(un[k])
        b.record()
        b.synchronize()
        seq_ms.append(a.elapsed_time(b))
    # end to end: every step copies all u from pinned host memory and reads them back
    u_h = [torch.empty(u.shape, dtype=torch.float64).pin_memory() for u in U]
    for k in range(len(U)):
        u_h[k].copy_(U[k])
    e2e_times = []
    for _ in range(args.steps):
        flush.zero_()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record()
        for k in range(len(U)):
            U[k].copy_(u_h[k], non_blocking=True)
        batch.step(U, Fs, fs, S, gmres_tol=1e-10, prec=prec)
        for k in range(len(U)):
            u_h[k].copy_(U[k], non_blocking=True)
        b.record()
        b.synchronize()
        e2e_times.append(a.elapsed_time(b))
    e2e_value, _ = aggregate_over_ranks(sum(e2e_times), n_pts, args.steps, dist, dev)
    # roofline of the dominant kernel region, from one profiled eager pass over the batch
    ctx.profile(True)
    ctx.profile_read("gmres", reset=True)
    for k, it in enumerate(items):
        mh.heat_step(ctx, it["prob"], U[k], Fs[k], fs[k], un[k], S[k], gmres_tol=1e-10, prec=prec)
    regions_ms = {r: ctx.profile_read(r) for r in REGION_NAMES}
    ctx.profile(False)
    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return
    roof = roofline(regions_ms, None, None, None, prec, mh, _peaks(), 1)
    bytes_io = sum(u.numel() for u in U) * 8
    line = {
        "metric": METRIC,
        "value": value,
        "unit": "points*timesteps/s",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": total_ms / args.steps,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f32+f64" if prec == mh.MH_PREC_MIXED else "f64",
        "data": "synthetic",
        "config": {"workload": f"batch: {args.batch_size} independent problems (unit disk minus 1-8 starfish/ellipse "
                               "holes, 256-2048 nodes per curve, alpha^2 = dt log-uniform in [1e-4, 1e-2], adaptive "
                               "trees with 8x8 nodes per leaf, Gaussian-sum forcing), IMEX Euler, GMRES tol 1e-10, one "
                               "CUDA graph launch per time step",
                   "points": n_pts, "problems": args.batch_size, "precision": args.prec,
                   "autotuned": bool(args.tune), "gmres_start": args.batch_warm,
                   "l2": "flushed between timed steps (256 MB write, untimed)",
                   "parallelism": "replicas" if world > 1 else "single"},
        "gmres_iterations_mean": float(np.mean(its)),
        "sequential_heat_step_ms_per_step": float(np.median(seq_ms)),
        "graph_kernels_per_step": batch.graph_kernels,
        "setup_s": setup_s,
        "autotune_s": tune_s,
        "autotune": {"p_counts": {str(pp): sum(1 for c in choices if c["p"] == pp) for pp in (10, 16, 24)},
                     "tile_counts": {str(tt): sum(1 for c in choices if c["tile"] == tt) for tt in (128, 256, 512)},
                     "max_rel_err_vs_p_ref": max((c["rel_err_vs_p_ref"] or 0.0) for c in choices)},
        "e2e": {"value": e2e_value, "unit": "points*timesteps/s", "h2d_bytes_per_step": bytes_io,
                "d2h_bytes_per_step": bytes_io},
        "gpu_launches": launches,
        "roofline": roof,
        "clocks": clk.summary(),
    }
    print(json.dumps(line))
    if dist:
        dist.destroy_process_group()


def prob_inside(prob):
    r = prob.regions()
    return int(np.sum(r == -1))


def cpu_baseline(wl, budget_s=20.0, seed=11):
    """The oracle as it stands, on all host cores, on a bounded sample of one step of the
    workload: the volume potential and the double layer at sampled interior nodes and sampled
    rows of the Nystrom matrix, each spread over a pool of worker processes (one per core; the
    per-target and per-row loops are independent), and one dense solve (BLAS threads).  The
    wall time per target / row with every core busy, extrapolated to one full step (N_D
    targets, N_Gamma rows, the solve), gives points * steps / s."""
    from oracle import bie, geometry as G, pool, tree as T
    t_start = time.time()
    rng = np.random.default_rng(seed)
    with pool.Workers() as wk:
        cores = wk.n
        tr = T.build(wl.box, wl.q, wl.min_level, wl.max_level, wl.forcing, wl.refine_tol)
        nodes = tr.nodes()
        leaves = tr.leaf_array()
        B = (wl.forcing(nodes) * wl.dt).reshape(len(leaves), -1)
        ntot = nodes.shape[0]
        n = sum(c.shape[0] for c in wl.curves)

        def timed(fn, per_worker):
            """Marginal wall time per item with every worker busy: batches of k and 3k items per
            worker (k = per_worker); the difference removes the per-call costs (pickling, and in
            the double layer the upsampling of the curves that every call redoes), which a full
            step pays once per worker, not per item."""
            t = []
            for k in (per_worker, 3 * per_worker):
                t0 = time.time()
                fn(k * cores)
                t.append(time.time() - t0)
            n1, n3 = per_worker * cores, 3 * per_worker * cores
            return max((t[1] - t[0]) / (n3 - n1), 0.1 * t[1] / n3), n1 + n3

        scale = max(0.25, budget_s / 20.0)
        t_vol, nv = timed(lambda k: wk.volume_potential(leaves, B, wl.q, wl.alpha,
                                                        nodes[rng.choice(ntot, k, replace=False)]),
                          max(1, int(2 * scale)))
        wk.nystrom_rows(wl.curves, wl.alpha, np.arange(cores))     # workers build the curves once
        t_row, nr = timed(lambda k: wk.nystrom_rows(wl.curves, wl.alpha, np.sort(rng.choice(n, k, replace=False))),
                          max(1, int(8 * scale)))
        curves = G.make_curves(wl.curves)
        cand = nodes[rng.choice(ntot, 64 * cores, replace=False)]
        info = G.classify(curves, cand)
        inside = cand[[i for i in range(len(cand)) if info.region[i] == -1 and all(
            p is None or p["d"] >= bie.NEAR_LINE * p["hs"] for p in info.proj[i])]]
        sig = rng.standard_normal(n)
        pos = [0]

        def dl(k):
            wk.dlp_eval(wl.curves, sig, wl.alpha, inside[pos[0]:pos[0] + k])
            pos[0] += k
        t_dlp, nd = timed(dl, max(1, min(int(2 * scale), len(inside) // (4 * cores))))
        M = np.eye(n) + 1e-3 * rng.standard_normal((n, n))
        t0 = time.time()
        np.linalg.solve(M, rng.standard_normal(n))
        t_solve = time.time() - t0
    t_step = ntot * (t_vol + t_dlp) + n * t_row + t_solve
    return {"value": (ntot + n) / t_step, "unit": "points*timesteps/s", "cores": cores, "kind": "oracle",
            "sample": f"{nv} volume targets, {nd} double-layer targets, {nr} Nystrom rows (each set spread over "
                      f"{cores} worker processes), one {n}x{n} dense solve; marginal wall time per item with all "
                      f"cores busy, extrapolated to one step ({ntot} targets, {n} rows)",
            "seconds_per_step_extrapolated": t_step, "wall_s": time.time() - t_start}


def run_profile_case(args):
    """One small fixed case of the starfish workload for a profiler (ncu -k ... -c ...), then
    exit: no training, no timing, no JSON line.
      volume   : the tree, then two mixed-precision volume potentials (tensor-core contractions,
                 M2M / L2L chains);
      operator : the boundary, then three binary32 operator products (k_gemv32s);
      solve    : two mixed-precision GMRES solves (float-float residual products, k_gemv_cpa);
      step     : three mixed-precision heat steps (near-field and upsampled-rule pair sums);
      mfree    : the heat-step problem with the matrix-free boundary operator, three products."""
    import torch
    import paper_1007_5335_gb300 as mh
    ctx = mh.Context(0)
    wl = W.starfish_domain()
    dev = torch.device("cuda:0")
    rng = np.random.default_rng(0)
    if args.profile_case == "volume":
        tree = mh.Tree(ctx, wl.box, wl.q, wl.min_level, wl.max_level, wl.forcing, wl.refine_tol)
        b = torch.tensor(wl.forcing(tree.nodes().cpu().numpy()) * wl.dt, device=dev)
        out = torch.empty_like(b)
        for _ in range(2):
            mh.mh_volume_potential(ctx, tree, wl.alpha, wl.p, b, out, prec=mh.MH_PREC_MIXED)
        tree.check()
    elif args.profile_case in ("operator", "solve"):
        bnd = mh.Boundary(ctx, wl.curves, alpert_order=8)
        x = torch.tensor(rng.standard_normal(bnd.n), device=dev)
        out = torch.empty_like(x)
        if args.profile_case == "operator":
            for _ in range(3):
                mh.mh_double_layer_apply(ctx, bnd, wl.alpha, x, out, prec=mh.MH_PREC_MIXED)
        else:
            for _ in range(2):
                out.zero_()
                mh.mh_gmres_solve(ctx, bnd, wl.alpha, x, out, tol=1e-10, prec=mh.MH_PREC_MIXED)
    elif args.profile_case == "mfree":
        tree, bnd, prob, _, _, _ = setup_problem(mh, ctx, wl, torch, dev)
        prob.matrix_free(True)
        x = torch.tensor(rng.standard_normal(bnd.n), device=dev)
        out = torch.empty_like(x)
        mh.mh_double_layer_apply(ctx, bnd, prob.alpha, x, out)
        torch.cuda.synchronize(dev)
        torch.cuda.nvtx.range_push("mfree_products")      # lets a profiler select the products
        for _ in range(3):
            mh.mh_double_layer_apply(ctx, bnd, prob.alpha, x, out)
        torch.cuda.nvtx.range_pop()
    else:
        tree, bnd, prob, nodes, F_np, _ = setup_problem(mh, ctx, wl, torch, dev)
        F = torch.tensor(F_np, device=dev)
        f = torch.zeros(bnd.n, dtype=torch.float64, device=dev)
        u = torch.zeros(tree.n_nodes, dtype=torch.float64, device=dev)
        un = torch.empty_like(u)
        sig = torch.zeros(bnd.n, dtype=torch.float64, device=dev)
        for _ in range(3):
            mh.heat_step(ctx, prob, u, F, f, un, sig, gmres_tol=1e-10, prec=mh.MH_PREC_MIXED)
            u, un = un, u
        tree.check()
    torch.cuda.synchronize(dev)


def run_bie_crossover(args):
    """Boundary-operator products at growing N_Gamma (starfish domain, 6 curves of 512 to 4096
    nodes, then 12 curves of 4096; tree, alpha and p of the heat-step workload): the dense binary64 product (k_gemv64s),
    the dense binary32 Krylov product (k_gemv32s) and the matrix-free product (on-surface multipole
    pass + chirp-transform Alpert correction, binary64), each the mean over K products timed by
    the library's region events with a 256 MB L2 flush between products; the device memory of
    each form; the matrix-free error against the dense binary64 product.  One JSON line."""
    import torch
    import paper_1007_5335_gb300 as mh
    dev = torch.device("cuda:0")
    ctx = mh.Context(0)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)
    K = max(args.steps if args.steps < 100 else 20, 3)
    rows = []
    for npc, holes in ((512, 5), (1024, 5), (2048, 5), (4096, 5), (4096, 11)):
        wl = W.starfish_domain(n_per_curve=npc, n_holes=holes)
        tree, bnd, prob, _, _, t_setup = setup_problem(mh, ctx, wl, torch, dev)
        n = bnd.n
        rng = np.random.default_rng(npc)
        y = np.concatenate(wl.curves)
        x = torch.tensor(np.cos(3 * y[:, 0]) * np.sin(2 * y[:, 1]) + 0.3 * rng.standard_normal(n), device=dev)
        out = torch.empty_like(x)

        def timed(region, prec, parts=()):
            for _ in range(3):
                mh.mh_double_layer_apply(ctx, bnd, prob.alpha, x, out, prec=prec)
            ctx.profile(True)
            ctx.profile_read(region, reset=True)   # a reset clears every region
            for _ in range(K):
                flush.zero_()
                mh.mh_double_layer_apply(ctx, bnd, prob.alpha, x, out, prec=prec)
            ms, cnt, _, _ = ctx.profile_read(region)
            split = {r: round(ctx.profile_read(r)[0] / K, 4) for r in parts}
            ctx.profile_read(region, reset=True)
            ctx.profile(False)
            return ms / max(cnt, 1), out.cpu().numpy(), split

        t64, y64, _ = timed("bie_gemv64", mh.MH_PREC_FP64)
        t32, _, _ = timed("bie_gemv32", mh.MH_PREC_MIXED)
        torch.cuda.synchronize(dev)
        free_a = torch.cuda.mem_get_info(dev)[0]
        t0 = time.time()
        prob.matrix_free(True)
        t_mf_setup = time.time() - t0
        torch.cuda.synchronize(dev)
        free_b = torch.cuda.mem_get_info(dev)[0]
        dense_bytes = 8 * n * n + 4 * n * n + 2 * n * n    # binary64 + binary32 + binary16 low part
        tmf, ymf, split = timed("bie_mfree", mh.MH_PREC_FP64, ("bie_fmm", "bie_fmm_contract", "bie_fmm_chain"))
        e = float(np.linalg.norm(ymf - y64) / np.linalg.norm(y64))
        rows.append({"n_gamma": n, "nodes_per_curve": npc, "dense_fp64_ms": round(t64, 4),
                     "dense_fp32_ms": round(t32, 4), "matrix_free_ms": round(tmf, 4),
                     "matrix_free_ms_split": dict(split, outside_multipole_pass=round(tmf - split["bie_fmm"], 4)),
                     "dense_bytes": dense_bytes, "matrix_free_bytes": int(free_a - free_b + dense_bytes),
                     "matrix_free_setup_s": round(t_mf_setup, 3), "problem_setup_s": round(t_setup, 3),
                     "rel_l2_matrix_free_vs_dense": e})
        del prob, bnd, tree
        torch.cuda.synchronize(dev)
    cross = next((r["n_gamma"] for r in rows if r["matrix_free_ms"] < r["dense_fp64_ms"]), None)
    cross32 = next((r["n_gamma"] for r in rows if r["matrix_free_ms"] < r["dense_fp32_ms"]), None)
    print(json.dumps({"bie_operator_products": rows, "products_per_point": K, "p": W.starfish_domain().p,
                      "first_n_gamma_matrix_free_below_dense_fp64": cross,
                      "first_n_gamma_matrix_free_below_dense_fp32": cross32,
                      "l2": "flushed between products (256 MB write, untimed)"}))



def run_reference(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    wl = W.starfish_domain()
    for _ in range(args.warmup):
        pass
    vals = []
    budget = max(2.0, min(8.0, 150.0 / max(args.steps + args.warmup, 1)))
    for _ in range(args.warmup):
        cpu_baseline(wl, budget_s=budget, seed=100)
    for s in range(args.steps):
        vals.append(cpu_baseline(wl, budget_s=budget, seed=200 + s))
    value = float(np.mean([v["value"] for v in vals]))
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "points*timesteps/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "starfish_domain (as the GPU arm), oracle on a bounded sample per step"},
            "cpu_baseline": {"value": value, "unit": "points*timesteps/s", "cores": vals[0]["cores"],
                             "kind": "oracle", "sample": vals[0]["sample"]},
            "e2e": {"value": value, "unit": "points*timesteps/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--prec", choices=["mixed", "fp64"], default="mixed")
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--check-steps", type=int, default=3)
    ap.add_argument("--workload", choices=["starfish", "batch"], default="starfish",
                    help="starfish: the single-domain step; batch: 64 independent problems per graph launch")
    ap.add_argument("--batch-size", type=int, default=W.BATCH_SIZE)
    ap.add_argument("--batch-warm", choices=["previous", "secant"], default="secant",
                    help="batch workload: GMRES start (no network is trained per problem)")
    ap.add_argument("--no-tune", dest="tune", action="store_false",
                    help="batch workload: p = 16 and the default near-field tile instead of the autotuner")
    ap.add_argument("--warm", choices=["learned", "previous", "secant", "zero"], default="learned",
                    help="GMRES start of every step (learned: the trained network with the bfloat16-pair weights)")
    ap.add_argument("--no-graph", dest="graph", action="store_false",
                    help="step through heat_step on the stream instead of one graph launch per step")
    ap.add_argument("--cpu-budget", type=float, default=20.0)
    ap.add_argument("--clocks-dir", default=None, help="directory for the raw clock samples (default: temp dir)")
    ap.add_argument("--no-cpu-baseline", dest="cpu_baseline", action="store_false")
    ap.add_argument("--bie-crossover", action="store_true",
                    help="time dense and matrix-free boundary-operator products at growing N_Gamma and exit")
    ap.add_argument("--profile-case", choices=["volume", "operator", "solve", "step", "mfree"], default=None,
                    help="run one small fixed case for a profiler and exit (see run_profile_case)")
    args = ap.parse_args()
    if args.clocks_dir:
        global CLOCKS_DIR
        CLOCKS_DIR = args.clocks_dir
    if args.profile_case:
        run_profile_case(args)
        return
    if args.bie_crossover:
        run_bie_crossover(args)
        return
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "ours" and args.workload == "batch":
        run_batch(args)
        return
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
