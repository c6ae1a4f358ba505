"""Benchmark: node relaxations/s to relative duality gap 1e-6 on GB300.

One step = one root-node relaxation of the least-squares workload
X 20000 x 50000 FP32 (Toeplitz correlation 0.9, k = 50, lambda2 = 0.1, SNR 3,
M = 2) solved to relative gap 1e-6 through the C ABI (fused X-pass + p-phase per
FISTA iteration, gap restarts, FP64 certification at the end), inputs resident
in HBM.  X (4 GB) is larger than L2, so no flush is needed between steps.

e2e: the same relaxation end to end through the public API from pinned host
buffers: X and y copied to the device, handle created (Lipschitz constant by a
Lanczos estimate), solved, beta copied back, handle destroyed.

Multi-GPU: one process per GPU (torchrun), each rank solves its own replica of
the workload; no data-path collective (the path shards by independent node
problems).  value = relaxations of all ranks / max over ranks of the timed span.

--impl reference times the FP64 CPU oracle (as it stands) on the host cores on a
bounded sample of the same workload (a few FISTA iterations on the full X), and
extrapolates to relaxations/s with the iteration count of the GPU solve.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

WORKLOAD = "ls_20000x50000_f32"
GAP_TOL = 1e-6
# FISTA iterations the GPU solve of WORKLOAD needs to reach GAP_TOL (measured on
# GB300 by this script's own arm; used by --impl reference to extrapolate).
GPU_ITERS_TO_GAP = {"ls_20000x50000_f32": 576}
METRIC = "node relaxations/s to rel. gap 1e-6 on 1 GB300; fused X-pass HBM GB/s vs peak"
PROFILE = os.path.join(ROOT, "profiles", "xstrip_ls_20000x50000_f32.md")


def max_over_ranks(ms, world, device="cpu"):
    """The slowest rank's time: every rank returns the maximum (one all-reduce;
    the only collective of a run, outside the timed region)."""
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(ms)], dtype=torch.float64, device=device)
    if world > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def throughput(units_per_rank, world, ms_max):
    """Whole-job units per second: every rank's units over the slowest rank's time."""
    return world * units_per_rank / (ms_max * 1e-3)


def env_rank():
    return int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")), \
        int(os.environ.get("LOCAL_RANK", "0"))


def measured_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return None


def kernel_source_hash():
    h = hashlib.sha256()
    for f in ("xstrip.cuh", "xpass.cuh", "common.cuh"):
        h.update(open(os.path.join(ROOT, "paper_2603_01306_gb300", "csrc", f), "rb").read())
    return h.hexdigest()[:16]


def profile_traffic(workload=WORKLOAD):
    """DRAM bytes per X-pass launch from the committed ncu summary (its
    "key: value" lines), or None when the kernel source changed since the
    counters were taken."""
    try:
        kv = {}
        for line in open(PROFILE):
            if ":" in line and not line.startswith(("#", " ", "|")):
                k, v = line.split(":", 1)
                kv[k.strip("- *`").strip()] = v.strip(" `\n")
    except Exception:
        return None
    if kv.get("kernel_source_hash") != kernel_source_hash():
        return None
    if workload != WORKLOAD:        # the summary's counters are of the headline workload
        return None
    try:
        return float(kv["dram_bytes_per_launch_full"])
    except Exception:
        return None


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def __enter__(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        if not self.path or not os.path.exists(self.path):
            return None
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        os.unlink(self.path)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "samples": len(sm),
                "reasons": sorted(reasons)}


def make_inputs(device, workload=WORKLOAD):
    import synth
    w = synth.WORKLOADS[workload]
    X, y = synth.make_problem_gpu(w, device=device)
    return w, X, y


def run_ours(args):
    import torch
    import torch.distributed as dist
    import paper_2603_01306_gb300 as relax

    rank, world, local = env_rank()
    torch.cuda.set_device(local)
    device = f"cuda:{local}"
    if args.workload == BNB_WORKLOAD:
        relax.load()
        if rank != 0:
            return None
        return {"metric": "branch and bound with the learned warm start vs the parent start", **run_bnb(device),
                "n_gpus": 1, "dtype": "f32", "data": "synthetic (seeded AR(1) Gaussian design)"}
    if args.workload == BATCH_WORKLOAD:
        # the batched-node workload alone (one JSON object, rank 0)
        relax.load()
        if rank != 0:
            return None
        return {"metric": "batched node relaxations/s to rel. gap 1e-6", **run_batch(device), "n_gpus": 1,
                "higher_is_better": True, "dtype": "f32", "data": "synthetic (seeded AR(1) Gaussian design)"}
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device(device))
    relax.load()
    w, X, y = make_inputs(device, args.workload)
    prec = {"f32": 0, "bf16": relax.binding.RELAX_BF16, "fp8": relax.binding.RELAX_FP8E4M3}[args.precision]
    esz = {"f32": 4, "bf16": 2, "fp8": 1}[args.precision]
    h = relax.Handle(X, y, loss=w.loss, k=w.k, lambda2=w.lambda2, M=w.M, timing=True, precision=prec)
    stream = torch.cuda.current_stream()
    beta = torch.empty(w.p, dtype=torch.float32, device=device)

    def step():
        _, res, code = h.solve(gap_tol=GAP_TOL, beta_out=beta)
        if code != 0:
            raise RuntimeError(f"solve status {relax.STATUS[code]}")
        return res

    for _ in range(args.warmup):
        step()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    results = []
    with ClockSampler(local) as clk:
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(args.steps):
            results.append(step())
        e1.record(stream)
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
    ms = e0.elapsed_time(e1)
    ms_max = max_over_ranks(ms, world, device)
    clocks = clk.summary()
    vs_fp32 = None
    if prec:
        # the same relaxation on the FP32 master X: the stored format's effect on the bound
        h32 = relax.Handle(X, y, loss=w.loss, k=w.k, lambda2=w.lambda2, M=w.M)
        _, r32, c32 = h32.solve(gap_tol=GAP_TOL)
        h32.close()
        rq = results[-1]
        vs_fp32 = {"fp32_status": relax.STATUS[c32], "fp32_dual_bound": r32.dual_bound, "fp32_iters": r32.iters,
                   "dual_bound": rq.dual_bound,
                   "rel_bound_diff": (rq.dual_bound - r32.dual_bound) / max(1.0, abs(r32.dual_bound)),
                   "note": "both bounds certified in FP64 on the FP32 master X; the stored format changes the "
                           "loop's products only"}
    # ---- end to end through the public API, from pinned host buffers
    X_h = torch.empty(tuple(X.shape), dtype=torch.float32).pin_memory()
    y_h = torch.empty(tuple(y.shape), dtype=torch.float32).pin_memory()
    X_h.copy_(X)
    y_h.copy_(y)
    beta_h = torch.empty(w.p, dtype=torch.float32).pin_memory()
    h.close()
    del X, y
    torch.cuda.empty_cache()
    torch.cuda.synchronize()
    e2e_steps = max(1, args.e2e_steps)
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        Xd = X_h.to(device, non_blocking=True)
        yd = y_h.to(device, non_blocking=True)
        he = relax.Handle(Xd, yd, loss=w.loss, k=w.k, lambda2=w.lambda2, M=w.M)
        _, res_e, code = he.solve(gap_tol=GAP_TOL, beta_out=beta)
        beta_h.copy_(beta, non_blocking=True)
        torch.cuda.synchronize()
        he.close()
        del Xd, yd
        if code != 0:
            raise RuntimeError(f"solve status {relax.STATUS[code]}")
    e2e_s = time.perf_counter() - t0
    if world > 1:
        dist.destroy_process_group()
    if rank != 0:
        return None
    iters = [r.iters for r in results]
    xp_ms = sum(r.xpass_ms for r in results)
    xp_n = sum(r.xpass_count for r in results)
    pp_ms = sum(r.pphase_ms for r in results)
    alg_bytes = w.n * w.p * esz + 4 * (w.n + w.p)      # X once (stored format) + y + beta
    if args.precision == "fp8":
        alg_bytes += 4 * w.p                               # per-column scales
    avg_ms = xp_ms / max(1, xp_n)
    achieved = alg_bytes / (avg_ms * 1e-3) / 1e9
    peaks = measured_peaks()
    peak = peaks["hbm_gbs"] if peaks else 6800.0
    traffic = profile_traffic(args.workload) if args.precision == "f32" else None
    value = throughput(args.steps, world, ms_max)
    line = {
        "metric": METRIC,
        "value": value,
        "unit": "relaxations/s",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": ms_max / args.steps,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": {"f32": "f32", "bf16": "bf16 X, f32 accumulation", "fp8": "fp8-e4m3 X, f32 accumulation"}[
            args.precision],
        "data": "synthetic (seeded AR(1) Gaussian design, generated on the device)",
        "config": {"workload": args.workload, "precision": args.precision, "n": w.n, "p": w.p, "k": w.k,
                   "lambda2": w.lambda2,
                   "rho": w.rho, "loss": w.loss, "M": w.M, "gap_tol": GAP_TOL, "snr": w.snr,
                   "l2": f"inputs larger than L2 (X is {w.n * w.p * esz / 1e9:.1f} GB as stored), no flush",
                   "parallelism": f"replicas x{world}" if world > 1 else "single GPU"},
        "iters_per_relaxation": iters,
        "certified_rel_gap": max(r.rel_gap for r in results),
        "dual_bound": results[-1].dual_bound,
        "lipschitz": results[-1].lipschitz,
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "traffic": traffic,
                     "kernel": "xstrip_kernel (fused X beta / link / X' r)",
                     "avg_launch_ms": avg_ms, "launches_timed": xp_n,
                     "algorithmic_bytes_per_launch": alg_bytes,
                     "peak_source": "MEASURED_PEAKS.json hbm_gbs (of measured)" if peaks
                     else "fallback 6800 GB/s (of fallback)"},
        "pphase_ms_per_iter": pp_ms / max(1, xp_n),
        "e2e": {"value": world * e2e_steps / e2e_s, "unit": "relaxations/s",
                "h2d_bytes_per_step": w.n * w.p * 4 + w.n * 4, "d2h_bytes_per_step": w.p * 4,
                "steps": e2e_steps,
                "note": "X, y from pinned host; handle create (Lanczos estimate of L), solve, beta to host, destroy"},
        "clocks": clocks,
        "gpu_launches": sum(r.launches for r in results),
    }
    if vs_fp32:
        line["vs_fp32_solve"] = vs_fp32
    if not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(X_h, y_h, w, results[-1].lipschitz, statistics.median(iters),
                                            args.cpu_sample_iters)
    if not args.no_batch:
        del X_h, y_h
        line["batch"] = run_batch(device)
    return line


BATCH_WORKLOAD = "batch256_5000x10000_f32"


def run_batch(device, workload=BATCH_WORKLOAD, reps=2, singles=16):
    """Batched node relaxations: the nodes of one tree share X (5000 x 10000,
    FP32); relax_solve_batch runs them in lockstep (X B and X' R GEMMs,
    per-node p-phase, converged nodes retire).  Reported against the plain
    FP32 single-node solve of the same nodes (the first `singles`)."""
    import numpy as np
    import torch
    import paper_2603_01306_gb300 as relax
    import synth
    w = synth.WORKLOADS[workload]
    nb = w.extra["nodes"]
    X, y = synth.make_problem_gpu(w, device=device)
    fix = np.stack([synth.node_fixings(w.p, 0, j, w.extra["j0_max"], w.extra["j1_max"], k=w.k) for j in range(nb)])
    fixd = torch.tensor(fix, device=device)
    h = relax.Handle(X, y, loss=w.loss, k=w.k, lambda2=w.lambda2, M=w.M)
    stream = torch.cuda.current_stream()
    times = []
    for r in range(reps):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        _, res, code = h.solve_batch(nb, fixings=fixd, gap_tol=GAP_TOL)
        e1.record(stream)
        torch.cuda.synchronize()
        times.append(e0.elapsed_time(e1) * 1e-3)
        if code not in (0, 4):   # ENOTCONV: reported below as uncertified nodes
            raise RuntimeError(f"batch status {relax.STATUS[code]}")
    t = min(times[1:]) if reps > 1 else times[0]
    it = [r.iters for r in res]
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    single_bounds = []
    for j in range(singles):
        _, r1, c1 = h.solve(fixings=fixd[j].contiguous(), gap_tol=GAP_TOL)
        single_bounds.append(r1.dual_bound)
    e1.record(stream)
    torch.cuda.synchronize()
    ts = e0.elapsed_time(e1) * 1e-3
    agree = max(abs(a - b.dual_bound) / abs(a) for a, b in zip(single_bounds, res))
    # the two products of a batched iteration alone (relax_batch_xpass on the
    # nodes' solutions), timed with CUDA events around the tensor-core launches
    betas, _, _ = h.solve_batch(nb, fixings=fixd, gap_tol=GAP_TOL)
    h.batch_xpass(betas, timing=True)
    ms = [h.batch_xpass(betas, timing=True)[2] for _ in range(5)]
    z_ms = statistics.median(m[0] for m in ms)
    g_ms = statistics.median(m[1] for m in ms)
    mma_flops = 6 * 2 * w.n * w.p * nb          # six BF16 plane products per FP32 product
    achieved = 2 * mma_flops / ((z_ms + g_ms) * 1e-3) / 1e12
    peaks = measured_peaks()
    peak = peaks["bf16_tflops"] if peaks else 1900.0
    h.close()
    certified = sum(1 for r in res if r.status == 0)
    return {"workload": workload, "nodes": nb, "value": certified / t, "unit": "node relaxations/s",
            "seconds": t, "nodes_certified": certified,
            "iters_min_med_max": [min(it), int(np.median(it)), max(it)],
            "polished_nodes": sum(1 for r in res if r.polish_iters > 0),
            "max_certified_rel_gap": max(r.rel_gap for r in res),
            "single_node_fp32": {"value": singles / ts, "unit": "node relaxations/s", "nodes": singles},
            "max_rel_bound_diff_vs_single": agree,
            "roofline": {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                         "frac": achieved / peak, "traffic": None,
                         "kernel": "bgemm_kernel (Z = X B', G = X' R on tcgen05, BF16 planes)",
                         "ms_per_product": [z_ms, g_ms],
                         "fp32_equivalent_tflops": 2 * 2 * w.n * w.p * nb / ((z_ms + g_ms) * 1e-3) / 1e12,
                         "flops_note": "achieved counts the BF16 MMA work (6 plane products x 2 n p nodes per "
                                       "product); fp32_equivalent_tflops counts 2 n p nodes per product",
                         "peak_source": "MEASURED_PEAKS.json bf16_tflops, burst (of measured)" if peaks
                         else "fallback 1900 TFLOP/s (of fallback)"},
            "products": "the library's tcgen05 kernel on BF16 planes of X, X' and the node operands "
                        "(FP32-accurate products, TMEM sums drained every 128 terms, FP64 sums of the K chunks); "
                        "each round of 16 iterations is one CUDA graph"}


BNB_WORKLOAD = "bnb_2000x5000_f32"


def run_bnb(device, workload=BNB_WORKLOAD, gen_nodes=60000, eval_nodes=60000, batch=64, epochs=3, seed=0):
    """The learned warm start at its configuration (X 2000 x 5000, rho 0.8,
    k 15, lambda2 0.2, LS): a batched best-first BnB from the parent start
    records its (parent, child) node solves; the network is trained on them on
    the device by the library's kernels (the last tenth of the pairs held
    out); then the BnB runs again from scratch with the parent start and with
    the learned start (Phi fallback), and both runs are reported: nodes,
    FISTA iterations, wall time, certified or not, incumbent and bound."""
    import numpy as np
    import torch
    import paper_2603_01306_gb300 as relax
    from paper_2603_01306_gb300 import bnb
    from paper_2603_01306_gb300.warmstart import WarmStartNet
    import synth
    w = synth.WORKLOADS[workload]
    X, y = synth.make_problem_gpu(w, device=device)
    h = relax.Handle(X, y, loss=w.loss, k=w.k, lambda2=w.lambda2, M=w.M)
    t0 = time.perf_counter()
    gen = bnb.run(h, w.k, max_nodes=gen_nodes, gap_tol=GAP_TOL, warm="parent", record=True, batch=batch)
    torch.cuda.synchronize()
    t_gen = time.perf_counter() - t0
    pairs = gen.pairs
    gen.pairs = []
    cut = int(0.9 * len(pairs))
    t0 = time.perf_counter()
    Ftr, Ttr = bnb.training_rows(h, pairs[:cut])
    Fte, Tte = bnb.training_rows(h, pairs[cut:])
    del pairs
    net = WarmStartNet(seed=seed, bf16=True)
    net.set_standardisation(Ftr[::97])
    mse_parent = net.loss_of(Fte, Tte)
    net.fit(Ftr, Ttr, epochs=epochs, batch=1 << 16, lr=1e-3, seed=seed)
    mse_learned = net.loss_of(Fte, Tte)
    torch.cuda.synchronize()
    t_train = time.perf_counter() - t0
    rows = int(Ftr.shape[0])
    del Ftr, Ttr, Fte, Tte
    runs = {}
    for warm in ("parent", "learned"):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        st = bnb.run(h, w.k, max_nodes=eval_nodes, gap_tol=GAP_TOL, warm=warm, net=net, batch=batch)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        runs[warm] = {"nodes": st.nodes, "iterations": st.iters, "seconds": dt, "nodes_per_s": st.nodes / dt,
                      "certified": st.certified, "incumbent": st.incumbent, "best_bound": st.best_bound,
                      "rel_gap": (st.incumbent - st.best_bound) / max(1.0, abs(st.incumbent)),
                      "learned_used": st.learned_used, "fallbacks": st.fallbacks,
                      "rule1_branch": st.cut_branch, "rule2_prune": st.cut_prune}
    h.close()
    return {"workload": workload, "n": w.n, "p": w.p, "k": w.k, "lambda2": w.lambda2, "rho": w.rho,
            "generation": {"nodes": gen.nodes, "seconds": t_gen, "certified": gen.certified},
            "training": {"rows": rows, "pairs": cut, "epochs": epochs, "seconds": t_train,
                         "heldout_mse_parent_start": mse_parent, "heldout_mse_learned_start": mse_learned},
            "bnb_parent_start": runs["parent"], "bnb_learned_start": runs["learned"],
            "iterations_ratio_learned_over_parent": runs["learned"]["iterations"] / max(1, runs["parent"]["iterations"])}


def oracle_sample(Xh, yh, w, L, sample_iters):
    """Time `sample_iters` FISTA iterations of the oracle on the full workload."""
    from oracle import solver
    t0 = time.perf_counter()
    solver.solve(Xh, yh, w.loss, w.k, w.lambda2, w.M, gap_tol=1e-300, L=L, max_iters=sample_iters)
    return time.perf_counter() - t0


def host_copy(X, y):
    import numpy as np
    Xh = np.empty(tuple(X.shape), dtype=np.float64)
    step = 1000
    for i in range(0, X.shape[0], step):
        Xh[i:i + step] = X[i:i + step].double().cpu().numpy()
    return Xh, y.double().cpu().numpy()


def cpu_cores():
    try:
        from threadpoolctl import threadpool_info
        n = [d.get("num_threads") for d in threadpool_info() if d.get("user_api") == "blas"]
        if n and n[0]:
            return int(n[0])
    except Exception:
        pass
    return os.cpu_count()


def cpu_baseline(X, y, w, L, iters_to_gap, sample_iters):
    Xh, yh = host_copy(X, y)
    secs = oracle_sample(Xh, yh, w, L, sample_iters)
    per_iter = secs / (sample_iters + 1)       # +1: the evaluation at the start point
    return {"value": 1.0 / (per_iter * iters_to_gap), "unit": "relaxations/s", "cores": cpu_cores(),
            "kind": "oracle",
            "sample": f"{sample_iters} oracle FISTA iterations (+ start evaluation) on the full "
                      f"{w.n}x{w.p} workload in FP64 ({secs:.1f} s), extrapolated to the GPU's "
                      f"{iters_to_gap:.0f} iterations to gap {GAP_TOL:g}"}


def run_reference(args):
    rank, world, local = env_rank()
    if rank != 0:
        return None
    import torch
    device = f"cuda:{local}"
    torch.cuda.set_device(local)
    w, X, y = make_inputs(device, args.workload)   # synthetic inputs only; the timed work runs on the host
    Xh, yh = host_copy(X, y)
    del X, y
    torch.cuda.empty_cache()
    from oracle import solver
    L = 2.0 * solver.spectral_norm_sq(Xh, iters=30) * 1.01
    iters_to_gap = GPU_ITERS_TO_GAP.get(args.workload) or args.ref_iters
    for _ in range(args.warmup):
        oracle_sample(Xh, yh, w, L, 1)
    t0 = time.perf_counter()
    tot = 0.0
    for _ in range(args.steps):
        tot += oracle_sample(Xh, yh, w, L, args.cpu_sample_iters)
    wall = time.perf_counter() - t0
    per_iter = tot / (args.steps * (args.cpu_sample_iters + 1))
    value = 1.0 / (per_iter * iters_to_gap)
    return {"impl": "reference", "metric": METRIC, "value": value, "unit": "relaxations/s",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": wall * 1e3 / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": args.workload, "n": w.n, "p": w.p, "k": w.k, "lambda2": w.lambda2,
                       "rho": w.rho, "loss": w.loss, "M": w.M, "gap_tol": GAP_TOL, "snr": w.snr},
            "cpu_baseline": {"value": value, "unit": "relaxations/s", "cores": cpu_cores(),
                             "kind": "oracle",
                             "sample": f"each step {args.cpu_sample_iters} oracle FISTA iterations on "
                                       f"the full workload, extrapolated to {iters_to_gap} iterations"},
            "e2e": {"value": value, "unit": "relaxations/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--workload", default=WORKLOAD,
                    help="synthetic workload (ls_4000x50000_f32: the counter-capture case; "
                         "batch256_5000x10000_f32: the batched-node measurement alone)")
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--cpu-sample-iters", type=int, default=12)
    ap.add_argument("--e2e-steps", type=int, default=2)
    ap.add_argument("--ref-iters", type=int, default=2000)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-batch", action="store_true", help="skip the batched-node measurement")
    ap.add_argument("--precision", choices=["f32", "bf16", "fp8"], default="f32",
                    help="storage format of X in the loop (BF16, or FP8-e4m3 with per-column scales)")
    args = ap.parse_args()
    if args.impl == "reference":
        line = run_reference(args)
    else:
        line = run_ours(args)
    if line is not None:
        print(json.dumps(line), flush=True)


if __name__ == "__main__":
    main()
