#!/usr/bin/env python3
"""Benchmark of the SVD-compressed M2L translation on GB300.

One step = one batched compressed M2L apply (V^T compression, offset-grouped
core products over the interaction lists, U expansion; five kernel
launches) over every level 2..6 of the synthetic 2,097,152-point sphere
workload (depth 6, p = 8, n = 296,
eps = 1e-7, d = 0.1, one right-hand side), i.e. 1,158,296 box-pair
translations.  Inputs are resident in HBM when the timed region starts and
L2 is flushed (a 256 MB write) before every timed step.

Prints ONE JSON line (rank 0).  Besides the throughput it reports the
tensor roofline of the core kernel (tracing with CUDA events), an end-to-end
number through the public API with pinned host buffers, the plain FP32
dense M2L on the same GPU, the adjoint, stage 2 (Sec. 3.2), the complete
evaluation of the workload's point potentials with the compressed passes
(Sec. 3.3; key "fmm"), SM clocks sampled during the timed region, and the
FP64 oracle timed on the host cores (cpu_baseline).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

With N > 1 (launched by torchrun) every rank runs an independent replica
of the workload (weak scaling: the M2L of independent FMM instances needs
no data exchange) and the slowest rank's time is reported.
``--impl reference`` times the FP64 oracle on the host cores instead.
"""
from __future__ import annotations

import argparse
import hashlib
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

METRIC = "M2L box-pair translations/s and % tensor roofline vs dense M2L, rel err ≤1e-6"
UNIT = "box-pair translations/s"
WORKLOAD = "sphere2m_p8"
LEVELS = range(2, 7)
L2_FLUSH_BYTES = 256 << 20


def env_int(name, default):
    try:
        return int(os.environ.get(name, default))
    except ValueError:
        return default


def workload_desc(pairs, r, r_pad, precision):
    return {
        "workload": "sphere2m_p8: 2,097,152 points uniform on the unit sphere (normalised Gaussian, seed 0), "
                    "uniform octree depth 6 with empty boxes skipped, levels 2-6, p=8 (n=296), eps=1e-7, d=0.1, "
                    "Laplace 1/(4 pi r), 1 right-hand side, upward-equivalent densities N(0,1)",
        "pairs_per_step": pairs,
        "rank_r": r,
        "r_pad": r_pad,
        "precision": precision,
        "l2": "flushed before every timed step (256 MB write)",
        "scaling_units": "independent replicas, one per GPU",
    }


# ---------------------------------------------------------------------------
# clocks
# ---------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("uuid,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, uuid):
        self.uuid = uuid
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(prefix="clocks_", suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        time.sleep(0.3)

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"], "samples": 0}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons, n = [], [], set(), 0
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            if self.uuid and self.uuid not in parts[0] and parts[0] not in self.uuid:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            n += 1
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": n}


# ---------------------------------------------------------------------------
# the FP64 oracle on the host cores
# ---------------------------------------------------------------------------
_ORACLE_FACTORS = {}


def oracle_sample(wl, seconds_budget):
    """Time the FP64 oracle's compressed M2L on a bounded slice of the
    workload (its precompute, like the library's, is not timed); returns
    (pairs, seconds, description)."""
    import numpy as np

    import synth
    from oracle import geometry as geo
    from oracle import m2l as om

    key = (wl.p, wl.d, wl.eps)
    if key not in _ORACLE_FACTORS:
        _ORACLE_FACTORS[key] = om.svd_factors(wl.p, wl.d, wl.eps)
    f = _ORACLE_FACTORS[key]
    done_pairs, spent, parts = 0, 0.0, []
    for level in LEVELS:
        box = wl.tree.levels[level]
        tg, sr, ok = geo.interaction_lists(box)
        q = synth.random_box_densities(box.shape[0], 1, f.U.shape[0], 1000 + level)[:, 0].astype(np.float64)
        # whole level if the budget allows, else the first targets that fit
        est = tg.size / 1.5e5
        if spent + est > seconds_budget and done_pairs > 0:
            frac = max(0.0, (seconds_budget - spent) / est)
            if frac < 0.02:
                break
            nt = max(1, int(frac * box.shape[0]))
            sel = tg < nt
            tg, sr, ok = tg[sel], sr[sel], ok[sel]
            parts.append(f"level {level}: targets 0..{nt - 1} ({tg.size} pairs)")
        else:
            parts.append(f"level {level}: all {tg.size} pairs")
        t0 = time.perf_counter()
        om.m2l_svd(box, level, wl.tree.r0, f, q, (tg, sr, ok))
        spent += time.perf_counter() - t0
        done_pairs += tg.size
        if spent > seconds_budget:
            break
    return done_pairs, spent, "oracle.m2l.m2l_svd (NumPy FP64, BLAS) on " + "; ".join(parts)


_ORACLE_DENSE = {}


def oracle_dense_sample(wl, seconds_budget):
    """Time the FP64 oracle's uncompressed M2L (Eq. (4) through the 316
    unit matrices, grouped by offset) on the first targets of the finest
    level that fit the budget; returns (pairs, seconds, description)."""
    import numpy as np

    import synth
    from oracle import geometry as geo
    from oracle import m2l as om

    key = (wl.p, wl.d)
    if key not in _ORACLE_DENSE:
        _ORACLE_DENSE[key] = om.unit_m2l_matrices(wl.p, wl.d)
    K = _ORACLE_DENSE[key]
    level = max(LEVELS)
    box = wl.tree.levels[level]
    tg, sr, ok = geo.interaction_lists(box)
    q = synth.random_box_densities(box.shape[0], 1, K.shape[1], 2000 + level)[:, 0].astype(np.float64)
    nt = max(1, box.shape[0] // 64)
    done, spent, used = 0, 0.0, nt
    while nt <= box.shape[0]:
        sel = tg < nt
        t0 = time.perf_counter()
        om.m2l_dense_unit(box, level, wl.tree.r0, K, q, (tg[sel], sr[sel], ok[sel]))
        done, spent, used = int(sel.sum()), time.perf_counter() - t0, nt
        if spent > seconds_budget / 4:
            break
        nt *= 2
    return done, spent, (f"oracle.m2l.m2l_dense_unit (NumPy FP64, BLAS) on level {level}, targets 0..{used - 1} "
                         f"({done} pairs)")


def oracle_single_thread(seconds_budget):
    """The compressed oracle sample again in a child process whose BLAS runs
    one thread (the thread count is fixed when NumPy loads); returns the
    child's (pairs, seconds, description) or None."""
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")
    code = ("import json, sys; sys.path.insert(0, %r); import bench, synth; "
            "wl = synth.workload(bench.WORKLOAD); print(json.dumps(bench.oracle_sample(wl, %r)))"
            % (ROOT, float(seconds_budget)))
    try:
        out = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True,
                             timeout=600).stdout.strip().splitlines()
        return tuple(json.loads(out[-1])) if out else None
    except (subprocess.TimeoutExpired, OSError, ValueError):
        return None


def job_throughput(local_ms: float, local_units: float, steps: int, device, world: int):
    """Whole-job throughput of weak-scaled replicas: the units every rank
    processed, summed, over the slowest rank's time (max over ranks).
    Returns (units per second, max_ms, summed units)."""
    import torch

    t = torch.tensor([float(local_ms)], dtype=torch.float64, device=device)
    u = torch.tensor([float(local_units)], dtype=torch.float64, device=device)
    if world > 1:
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        torch.distributed.all_reduce(u, op=torch.distributed.ReduceOp.SUM)
    max_ms, units = float(t.item()), float(u.item())
    return units * steps / (max_ms / 1e3), max_ms, units


def run_reference(args, rank):
    if rank != 0:
        return
    import synth

    wl = synth.workload(WORKLOAD)
    budget = max(2.0, min(20.0, 150.0 / max(1, args.steps + args.warmup)))
    for _ in range(args.warmup):
        oracle_sample(wl, budget)
    pairs = secs = 0.0
    desc = ""
    for _ in range(args.steps):
        p, s, desc = oracle_sample(wl, budget)
        pairs += p
        secs += s
    value = pairs / secs
    cores = os.cpu_count()
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * secs / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": workload_desc(None, None, None, "fp64 oracle"),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": desc},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# our arm
# ---------------------------------------------------------------------------
def kernel_source_hash():
    """Hash of the sources of the bench's dominant kernel (core_stage_kernel)."""
    h = hashlib.sha256()
    for f in ("kernels_core.cu", "umma_ptx.h"):
        h.update(open(os.path.join(ROOT, "paper_1211_2517_gb300", "csrc", f), "rb").read())
    return h.hexdigest()[:16]


def recorded_traffic():
    """DRAM bytes per core launch from the committed ncu summary, when it was
    taken on the current kernel source (else None)."""
    path = os.path.join(ROOT, "profiles", "m2l_core_sphere2m_p8_traffic.json")
    try:
        rec = json.load(open(path))
    except (OSError, ValueError):
        return None
    if rec.get("kernel_source_sha256_16") != kernel_source_hash():
        return None
    return rec.get("dram_bytes_per_step_core")


def run_ours(args, rank, world, local_rank):
    import torch

    import __graft_entry__

    if rank == 0:
        __graft_entry__.build()
    if world > 1:
        torch.distributed.barrier()
    import numpy as np

    import synth
    from paper_1211_2517_gb300 import M2LPlan

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        pass
    bf16_peak = peaks.get("bf16_tflops", 1900.0)
    peak_src = "measured" if "bf16_tflops" in peaks else "fallback"

    wl = synth.workload(WORKLOAD, seed=rank)
    tree = wl.tree
    plan = M2LPlan(wl.p, wl.eps, wl.d, args.precision)
    pairs = {}
    for l in LEVELS:
        pairs[l] = plan.set_level(l, tree.levels[l], tree.r0)
    total_pairs = sum(pairs.values())
    n, r, rp = plan.n, plan.r, plan.r_pad
    # the levels' densities back to back (one batched apply per step)
    q_all = torch.from_numpy(np.concatenate(
        [synth.random_box_densities(tree.levels[l].shape[0], 1, n, 100 + l)[:, 0] for l in LEVELS])).to(dev)
    out_all = torch.empty_like(q_all)
    lo, hi = min(LEVELS), max(LEVELS)
    offs, row = {}, 0
    for l in LEVELS:
        offs[l] = (row, row + tree.levels[l].shape[0])
        row = offs[l][1]
    q = {l: q_all[a:b] for l, (a, b) in offs.items()}
    out = {l: out_all[a:b] for l, (a, b) in offs.items()}
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()

    def step(adjoint=False):
        plan.apply_levels(q_all, lo, hi, out=out_all, adjoint=adjoint)

    def step_per_level(fn):
        for l in LEVELS:
            fn(q[l], l, out=out[l])

    def timed(fn_step, k):
        evs = []
        for _ in range(k):
            flush.fill_(1.0)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            fn_step()
            e1.record(stream)
            evs.append((e0, e1))
        torch.cuda.synchronize()
        return sum(a.elapsed_time(b) for a, b in evs)

    # core launch variant for this workload (untimed; the same arithmetic for
    # every candidate)
    tune = None
    if args.precision != "fp32" and not args.no_autotune:
        tune = plan.autotune(q_all, lo, hi, reps=5, out=out_all)
    for _ in range(args.warmup):
        step()
    plan.sync()

    # ---- timed region --------------------------------------------------
    uuid = str(getattr(torch.cuda.get_device_properties(dev), "uuid", ""))
    sampler = ClockSampler(uuid)
    sampler.start()
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_push("timed_steps")
    total_ms = timed(step, args.steps)
    torch.cuda.nvtx.range_pop()
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    clocks = sampler.stop()
    plan.sync()
    value, max_ms, job_pairs = job_throughput(total_ms, total_pairs, args.steps, dev, world)
    # split + compression (the f16x3 compression writes the core's FP16
    # pieces itself), core, split + expansion, over all levels
    launches_per_step = 5

    # ---- roofline of the core kernel (traced pass, same conditions) -----
    k_prof = min(args.steps, 20)
    plan.profile(True)
    timed(step, k_prof)
    stage_ms, traced = plan.profile_read()
    plan.profile(False)
    core_ms = stage_ms["core"] / k_prof
    flops_step = 2.0 * r * r * total_pairs
    achieved = flops_step / (core_ms / 1e3) / 1e12
    issued = {"split6": 6, "split3": 3, "bf16": 1, "f16x3": 3}.get(args.precision, 0) * 2.0 * rp * rp * total_pairs
    traffic = recorded_traffic()
    roofline = {
        "bound": "tensor", "achieved": achieved, "peak": bf16_peak, "unit": "TFLOP/s",
        "frac": achieved / bf16_peak, "traffic": traffic,
        "kernel": {1: "core_resident_kernel (A-resident split6 core, K~_o in column blocks)",
                   2: "umma_kernel<A_GATHER,E_RED> (offset-grouped core, partials of 2 K-chunks drained)",
                   3: "umma_kernel<A_GATHER,E_RED> (offset-grouped core, partials of 1 K-chunk drained)",
                   6: "umma_kernel<A_GATHER,E_RED> (offset-grouped core, partials of 3 K-chunks drained)",
                   9: "umma_kernel<A_GATHER,E_RED> (offset-grouped core, partials of 2 K-chunks, 2 per MMA step)",
                   10: "umma_kernel<A_GATHER,E_RED> (offset-grouped core, partials of 3 K-chunks, 2 per MMA step)",
                   11: "umma_kernel<A_GATHER,E_RED> (offset-grouped core, partials of 3 K-chunks, 3 per MMA step)",
                   12: "umma_kernel<A_GATHER,E_RED> (offset-grouped core, partials of 3 K-chunks, 3 per MMA step, "
                       "rows reduced without a transpose)",
                   13: "core_stage_kernel (offset-grouped core, partials of 3 K-chunks drained into registers, rows "
                       "staged in shared memory and reduced into p~ by TMA bulk reductions)"}.get(
                       (tune or {}).get("variant"), "umma_kernel<A_GATHER,E_RED> (offset-grouped core)"),
        "core_dtype": {"f16x3": "fp16 pieces x fp16 pieces, fp32 accumulate (3 products)",
                       "split6": "bf16 pieces, fp32 accumulate (6 products)"}.get(args.precision, args.precision),
        "algorithmic_flops_per_step": flops_step,
        "flops_per_unit": f"2 r^2 = {2 * r * r} per box pair (r = {r})",
        "launches_per_step": 1,
        "core_ms_per_step": core_ms,
        "stage_ms_per_step": {k: v / k_prof for k, v in stage_ms.items()},
        "issued_tensor_tflops": issued / (core_ms / 1e3) / 1e12 if issued else None,
        "peak_source": f"{peak_src} bf16 dense burst (MEASURED_PEAKS.json bf16_tflops); dense fp16 has the same "
                       "nominal rate (ratio 1)" if args.precision == "f16x3" else
                       f"{peak_src} bf16 dense burst (MEASURED_PEAKS.json bf16_tflops)",
    }

    # ---- end to end through the public API with pinned host buffers: the
    # library's host-buffer apply copies the rows in and the results out in
    # chunks that overlap its compression and expansion ---------------------
    hq = q_all.cpu().pin_memory()
    hp = torch.empty_like(hq).pin_memory()

    def e2e_step():
        plan.apply_levels_host(hq, lo, hi, out=hp)

    for _ in range(3):
        e2e_step()
    k_e2e = min(args.steps, 50)
    e2e_ms = timed(e2e_step, k_e2e)
    h2d = hq.numel() * 4
    e2e_value, _, _ = job_throughput(e2e_ms, total_pairs, k_e2e, dev, world)
    e2e = {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": h2d,
           "api": "kifmm_m2l_apply_levels_host (pinned host buffers, copies in 4 chunks on the plan's copy stream)"}

    # ---- adjoint and the plain FP32 dense M2L on the same GPU -----------
    k_small = min(args.steps, 10)
    step(adjoint=True)
    adj_ms = timed(lambda: step(adjoint=True), k_small)
    step_per_level(plan.apply_dense)
    dense_ms = timed(lambda: step_per_level(plan.apply_dense), max(2, min(k_small, 5)))
    dense_value = total_pairs * max(2, min(k_small, 5)) / (dense_ms / 1e3)
    # the same uncompressed M2L on the tensor cores at the compressed path's accuracy
    dense_tc = None
    if args.precision == "f16x3":
        step_per_level(plan.apply_dense_tc)
        plan.sync()
        k_tc = max(2, min(k_small, 10))
        tc_ms = timed(lambda: step_per_level(plan.apply_dense_tc), k_tc)
        plan.sync()
        dense_tc = {"value": total_pairs * k_tc / (tc_ms / 1e3), "unit": UNIT, "ms_per_step": tc_ms / k_tc,
                    "precision": "f16x3 (the compressed path's arithmetic)", "flops_per_unit": f"2 n^2 = {2 * n * n}",
                    "tflops_algorithmic": 2.0 * n * n * total_pairs / (tc_ms / k_tc / 1e3) / 1e12,
                    "parity": "tests/test_gpu_m2l.py::test_dense_tensor_core_parity (1e-6 against the FP64 dense M2L)"}
    per_gpu_value = total_pairs * args.steps / (total_ms / 1e3)
    plan.sync()

    # ---- the BF16 split (split6) on the same workload: the FP16 split's
    # counterpart, and the plan that stage 2 and the point-source evaluation
    # (BF16 modes) run on ----------------------------------------------------
    plan6, split6 = plan, None
    legs = {"split6", "noalloc", "stage2", "fmm", "yukawa", "torus", "batch64"} if args.legs == "all" else \
        set(x for x in args.legs.split(",") if x and x != "none")
    if args.precision == "f16x3" and legs & {"split6", "noalloc", "stage2"}:
        plan6 = M2LPlan(wl.p, wl.eps, wl.d, "split6")
        for l in LEVELS:
            plan6.set_level(l, tree.levels[l], tree.r0)
        if not args.no_autotune:
            plan6.autotune(q_all, lo, hi, reps=5, out=out_all)
        for _ in range(3):
            plan6.apply_levels(q_all, lo, hi, out=out_all)
        plan6.sync()
        k6 = min(args.steps, 50)
        s6_ms = timed(lambda: plan6.apply_levels(q_all, lo, hi, out=out_all), k6)
        plan6.profile(True)
        timed(lambda: plan6.apply_levels(q_all, lo, hi, out=out_all), min(k6, 20))
        s6_stage, _ = plan6.profile_read()
        plan6.profile(False)
        split6 = {"value": total_pairs * k6 / (s6_ms / 1e3), "unit": UNIT, "ms_per_step": s6_ms / k6,
                  "stage_ms_per_step": {k: v / min(k6, 20) for k, v in s6_stage.items()},
                  "core_tflops_algorithmic": flops_step / (s6_stage["core"] / min(k6, 20) / 1e3) / 1e12}

    def step6():
        plan6.apply_levels(q_all, lo, hi, out=out_all)

    # ---- the allocation-free apply beside kifmm_m2l_apply: level 6 of the
    # workload (its scratch fits the 64 MiB static array), split6 -----------
    noalloc = None
    if args.precision != "fp32" and "noalloc" in legs:
        import ctypes

        from paper_1211_2517_gb300 import _lib

        lv = max(LEVELS)
        xq, yo = q[lv], out[lv]
        strm = ctypes.c_void_p(stream.cuda_stream)

        def na_step():
            _lib.check("kifmm_m2l_apply_noalloc", _lib.lib().kifmm_m2l_apply_noalloc(
                plan6._h, 0, lv, 1, ctypes.c_void_p(xq.data_ptr()), ctypes.c_void_p(yo.data_ptr()), 0.0, strm))

        for _ in range(3):
            na_step()
            plan6.apply(xq, lv, out=yo)
        plan6.sync()
        k_na = min(args.steps, 50)
        na_ms = timed(na_step, k_na)
        ap_ms = timed(lambda: plan6.apply(xq, lv, out=yo), k_na)
        plan6.sync()
        noalloc = {"level": lv, "pairs": pairs[lv], "precision": "split6",
                   "ms_per_apply": na_ms / k_na, "apply_ms_per_apply": ap_ms / k_na,
                   "value": pairs[lv] * k_na / (na_ms / 1e3), "unit": UNIT,
                   "note": "kifmm_m2l_apply_noalloc against kifmm_m2l_apply on the same level and plan"}

    # ---- stage 2 (Sec. 3.2): per-offset low-rank cores, c2 = 10 ----------
    plan_main = plan
    stage2 = None
    if args.precision != "fp32" and "stage2" in legs:
        plan, plan_main = plan6, plan
        step_main = step
        step = step6
        c2 = 10.0
        plan.set_stage2(c2)
        ranks = plan.stage2_ranks()
        for _ in range(3):
            step()
        plan.sync()
        k_s2 = min(args.steps, 50)
        s2_ms = timed(step, k_s2)
        plan.profile(True)
        timed(step, min(k_s2, 20))
        s2_stage, _ = plan.profile_read()
        plan.profile(False)
        plan.set_stage2(0.0)
        stage2 = {"c2": c2, "eps2": c2 * wl.eps / r, "ranks_min_mean_max": [int(ranks.min()), float(ranks.mean()),
                                                                         int(ranks.max())],
                  "value": total_pairs * k_s2 / (s2_ms / 1e3), "unit": UNIT, "ms_per_step": s2_ms / k_s2,
                  "core_ms_per_step": s2_stage["core"] / min(k_s2, 20), "precision": "split6",
                  "parity": "tests/test_gpu_m2l.py::test_stage2_parity against the oracle's two-product M2L"}
        plan, step = plan_main, step_main
        if args.precision == "f16x3":
            # the same c2 on the headline plan's f16x3 arithmetic, against its
            # single-stage core
            plan.set_stage2(c2)
            for _ in range(3):
                step()
            plan.sync()
            f_ms = timed(step, k_s2)
            plan.profile(True)
            timed(step, min(k_s2, 20))
            f_stage, _ = plan.profile_read()
            plan.profile(False)
            plan.set_stage2(0.0)
            plan.profile(True)
            timed(step, min(k_s2, 20))
            one_stage, _ = plan.profile_read()
            plan.profile(False)
            plan.sync()
            stage2["f16x3"] = {"value": total_pairs * k_s2 / (f_ms / 1e3), "unit": UNIT, "ms_per_step": f_ms / k_s2,
                               "core_ms_per_step": f_stage["core"] / min(k_s2, 20),
                               "single_stage_core_ms_per_step": one_stage["core"] / min(k_s2, 20),
                               "parity": "tests/test_gpu_m2l.py::test_stage2_parity[f16x3]"}

    # ---- complete evaluation for the workload's points (Sec. 4 with the
    # compressed passes of Sec. 3.3): near field + S~, M~, M2L, L~, T~ ------
    fmm = None
    if args.precision != "fp32" and "fmm" in legs:
        from paper_1211_2517_gb300 import PointFMM

        ftree = PointFMM(plan_main, wl.points, wl.depth)
        qd = torch.tensor(wl.densities, dtype=torch.float32, device=dev)
        pot = torch.empty_like(qd)
        for parts in (3, 1, 2):
            for _ in range(3):
                ftree.evaluate(qd, parts, out=pot)
        k_f = min(args.steps, 20)
        torch.cuda.nvtx.range_push("fmm_evaluate")
        f_ms = timed(lambda: ftree.evaluate(qd, 3, out=pot), k_f)
        torch.cuda.nvtx.range_pop()
        near_ms = timed(lambda: ftree.evaluate(qd, 1, out=pot), k_f)
        far_ms = timed(lambda: ftree.evaluate(qd, 2, out=pot), k_f)
        info = ftree.info()
        npts = wl.points.shape[0]
        # the same points as dipoles with their outward normals (double layer, Sec. 4)
        ftree.set_normals(wl.points / np.linalg.norm(wl.points, axis=1, keepdims=True))
        for _ in range(3):
            ftree.evaluate(qd, 3, out=pot)
        dl_ms = timed(lambda: ftree.evaluate(qd, 3, out=pot), k_f)
        dl_near_ms = timed(lambda: ftree.evaluate(qd, 1, out=pot), k_f)
        ftree.set_normals(None)
        fmm = {"value": npts * k_f / (f_ms / 1e3), "unit": "points/s (potential at every point from all others)",
               "ms_per_evaluate": f_ms / k_f, "near_ms": near_ms / k_f, "far_ms": far_ms / k_f,
               "m2l_precision": args.precision,
               "points": npts, "depth": info["depth"], "leaves": info["leaves"], "m2l_pairs": info["m2l_pairs"],
               "near_pairs": info["near_pairs"],
               "near_pairs_per_s": info["near_pairs"] * k_f / (near_ms / 1e3),
               "double_layer": {"value": npts * k_f / (dl_ms / 1e3), "unit": "points/s",
                                "ms_per_evaluate": dl_ms / k_f, "near_ms": dl_near_ms / k_f,
                                "sources": "the same points as dipoles, outward unit normals",
                                "parity": "tests/test_gpu_fmm.py::test_double_layer_matches_oracle"},
               "parity": "tests/test_gpu_fmm.py: within 1e-6 relative L2 of the FP64 oracle's compressed FMM and "
                         "of the direct sum"}
        ftree.close()

    # ---- a non-homogeneous kernel (Sec. 3.1's O(L) precompute): the Yukawa
    # kernel exp(-kappa r) / (4 pi r), one plan per level, the same levels and
    # densities as the headline --------------------------------------------
    yukawa = None
    if args.precision != "fp32" and not args.no_yukawa and "yukawa" in legs:
        try:
            kappa = 3.0
            t0 = time.time()
            yplans = {}
            for l in LEVELS:
                yp = M2LPlan(wl.p, wl.eps, wl.d, args.precision, "yukawa", kappa, tree.r0 / (1 << l))
                yp.set_level(l, tree.levels[l], tree.r0)
                yplans[l] = yp
            setup_s = time.time() - t0
            from paper_1211_2517_gb300 import apply_batch

            # the five level plans as one batch: one grouped core launch,
            # replayed from a CUDA graph
            yitems = [{"plan": yp, "level_lo": l, "level_hi": l, "x": q[l], "out": out[l]}
                      for l, yp in yplans.items()]

            def ystep():
                torch.cuda.nvtx.range_push("yukawa_step")
                apply_batch(yitems, use_graph=True)
                torch.cuda.nvtx.range_pop()

            for _ in range(3):
                ystep()
            torch.cuda.synchronize()
            k_y = min(args.steps, 20)
            y_ms = timed(ystep, k_y)
            yukawa = {"value": total_pairs * k_y / (y_ms / 1e3), "unit": UNIT, "ms_per_step": y_ms / k_y,
                      "mode": "one batch of the level plans (one grouped core launch) from a CUDA graph",
                      "kappa": kappa, "ranks_by_level": {str(l): yp.r for l, yp in yplans.items()},
                      "precompute_s_all_levels": setup_s, "precision": args.precision,
                      "parity": "tests/test_gpu_m2l.py::test_yukawa_per_level_plans, ::test_yukawa_levels_one_batch"}
            for yp in yplans.values():
                yp.close()
        except Exception as exc:  # a secondary leg: reported, the headline line still prints
            yukawa = {"error": f"{type(exc).__name__}: {exc}"}

    # ---- the p = 10 torus and the 64-instance batch -------------------------
    torus = batch64 = None
    if args.precision != "fp32" and not args.no_extra and "torus" in legs:
        try:
            torus = torus_measure(args, dev, min(args.steps, 50), bf16_peak)
        except Exception as exc:  # a secondary leg: reported, the headline line still prints
            torus = {"error": f"{type(exc).__name__}: {exc}"}
    if args.precision != "fp32" and not args.no_extra and "batch64" in legs:
        try:
            kb = min(args.steps, 10)
            bv, bms, bpairs, bach, _ = batch64_measure(args, rank, world, dev, kb, 3, False)
            batch64 = {"value": bv, "unit": UNIT, "ms_per_step": bms / kb, "pairs_per_step": bpairs,
                       "steps": kb, "precision": args.precision, "workload": BATCH64_DESC,
                       "roofline": {"bound": "tensor", "achieved": bach, "peak": bf16_peak, "unit": "TFLOP/s",
                                    "frac": bach / bf16_peak, "flops_per_unit": "2 r^2 per box pair and rhs",
                                    "time": "whole batch (compression, core and expansion of three operators)"},
                       "parity": "tests/test_gpu_m2l.py::test_batch64_full_config",
                       "arithmetic": "the batch64 workload is stated in FP32; the batch runs the plan's "
                                     f"tensor-core arithmetic ({args.precision}), which meets the FP32 gate of 1e-6 "
                                     "against the oracle"}
        except Exception as exc:
            batch64 = {"error": f"{type(exc).__name__}: {exc}"}

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": max_ms / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": {"f16x3": "f16", "fp32": "f32"}.get(args.precision, "bf16"), "data": "synthetic",
        "config": dict(workload_desc(total_pairs, r, rp, args.precision),
                       core_variant=({k: tune[k] for k in ("n_chunk", "contiguous", "variant")} if tune else "default")),
        "roofline": roofline,
        "clocks": clocks,
        "e2e": e2e,
        "gpu_launches": launches_per_step * args.steps,
        "dense_fp32_baseline": {"value": dense_value, "unit": UNIT,
                                "speedup_compressed_over_dense": per_gpu_value / dense_value,
                                "note": "plain FP32 CUDA-core kernel; dense_tensor_core is the equal-accuracy comparison"},
        "dense_tensor_core": dict(dense_tc, speedup_compressed_over_dense=per_gpu_value / dense_tc["value"])
        if dense_tc else None,
        "adjoint": {"value": total_pairs * k_small / (adj_ms / 1e3), "unit": UNIT},
        "split6": split6,
        "stage2": stage2,
        "fmm": fmm,
        "yukawa_per_level": yukawa,
        "torus4m_p10": torus,
        "noalloc": noalloc,
        "batch64": batch64,
        "parity": "tests/test_gpu_m2l.py: f16x3, split6 and fp32 within 1e-6 relative L2 of the FP64 oracle",
    }

    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cp, cs, cdesc = oracle_sample(wl, 20.0)
        line["cpu_baseline"] = {"value": cp / cs, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
                                "sample": cdesc}
        one = oracle_single_thread(10.0)
        if one:
            line["cpu_baseline"]["single_thread"] = {"value": one[0] / one[1], "unit": UNIT, "cores": 1,
                                                     "sample": one[2]}
        dp, ds, ddesc = oracle_dense_sample(wl, 10.0)
        line["cpu_baseline"]["dense"] = {"value": dp / ds, "unit": UNIT, "cores": os.cpu_count(),
                                         "kind": "oracle, uncompressed M2L", "sample": ddesc}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if plan6 is not plan:
        plan6.close()
    plan.close()


def torus_measure(args, dev, steps, peak):
    """The 4,194,304-point torus (R = 1, r = 0.3), depth 6, p = 10,
    eps = 1e-8 (r = 271, r_pad = 272: the core splits N in two parts), levels
    2-6 in one apply per step; the core's roofline with 2 r^2 FLOPs per pair."""
    import numpy as np
    import torch

    import synth
    from paper_1211_2517_gb300 import M2LPlan

    wl = synth.workload("torus4m_p10", seed=0)
    tree = wl.tree
    plan = M2LPlan(wl.p, wl.eps, wl.d, args.precision)
    pairs = sum(plan.set_level(l, tree.levels[l], tree.r0) for l in LEVELS)
    q_all = torch.from_numpy(np.concatenate(
        [synth.random_box_densities(tree.levels[l].shape[0], 1, plan.n, 700 + l)[:, 0] for l in LEVELS])).to(dev)
    out = torch.empty_like(q_all)
    lo, hi = min(LEVELS), max(LEVELS)
    tune = plan.autotune(q_all, lo, hi, reps=3, out=out) if not args.no_autotune else None
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()

    def timed(k):
        evs = []
        for _ in range(k):
            flush.fill_(1.0)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            plan.apply_levels(q_all, lo, hi, out=out)
            e1.record(stream)
            evs.append((e0, e1))
        torch.cuda.synchronize()
        return sum(a.elapsed_time(b) for a, b in evs)

    timed(3)
    ms = timed(steps)
    plan.profile(True)
    kp = min(steps, 20)
    timed(kp)
    st, _ = plan.profile_read()
    plan.profile(False)
    plan.sync()
    core_ms = st["core"] / kp
    achieved = 2.0 * plan.r * plan.r * pairs / (core_ms / 1e3) / 1e12
    res = {"value": pairs * steps / (ms / 1e3), "unit": UNIT, "ms_per_step": ms / steps, "pairs_per_step": pairs,
           "rank_r": plan.r, "r_pad": plan.r_pad, "precision": args.precision,
           "core_ms_per_step": core_ms, "stage_ms_per_step": {k: v / kp for k, v in st.items()},
           "roofline": {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                        "frac": achieved / peak, "flops_per_unit": f"2 r^2 = {2 * plan.r * plan.r} per box pair"},
           "core_variant": {k: tune[k] for k in ("n_chunk", "contiguous", "variant")} if tune else "default",
           "workload": "torus4m_p10: 4,194,304 points area-uniform on a torus R=1 r=0.3 (seed 0), depth 6, levels "
                       "2-6, p=10 (n=488), eps=1e-8, d=0.1, 1 rhs, N(0,1) upward-equivalent densities",
           "parity": "tests/test_gpu_m2l.py::test_full_size_torus_p10_sampled and the p = 10 parity tests"}
    plan.close()
    return res


def batch64_measure(args, rank, world, dev, steps, warmup, sample_clocks):
    """64 ellipsoid instances (N log-uniform 5e4-1e6, depth 3-6,
    p in {6, 8, 10}, 16 rhs), all M2L levels, one grouped batch replayed from a
    CUDA graph per step (rank k takes instances 64 k .. 64 k + 63).  Returns
    (units per second over all ranks, slowest rank's ms, units, achieved
    TFLOP/s, clocks)."""
    import torch

    import synth
    from paper_1211_2517_gb300 import M2LPlan, apply_batch

    plans = {p: M2LPlan(p, 1e-7, 0.1, args.precision) for p in (6, 8, 10)}
    items, pairs, flops = [], 0, 0.0
    for j in range(64):
        i = 64 * rank + j
        wl = synth.ellipsoid_instance(i)
        plan = plans[wl.p]
        for l in range(2, wl.depth + 1):
            np_ = plan.set_level(l, wl.tree.levels[l], wl.tree.r0, instance=i)
            pairs += np_ * 16
            flops += 2.0 * plan.r * plan.r * np_ * 16
        nb = sum(wl.tree.levels[l].shape[0] for l in range(2, wl.depth + 1))
        x = torch.from_numpy(synth.random_box_densities32(nb, 16, plan.n, 5000 + i)).to(dev)
        items.append({"plan": plan, "instance": i, "level_lo": 2, "level_hi": wl.depth, "x": x,
                      "out": torch.empty_like(x)})
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()
    for _ in range(warmup):
        apply_batch(items, use_graph=True)
    torch.cuda.synchronize()
    sampler = None
    if sample_clocks:
        sampler = ClockSampler(str(getattr(torch.cuda.get_device_properties(dev), "uuid", "")))
        sampler.start()
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    evs = []
    for _ in range(steps):
        flush.fill_(1.0)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.nvtx.range_push("batch64_step")
        e0.record(stream)
        apply_batch(items, use_graph=True)
        e1.record(stream)
        torch.cuda.nvtx.range_pop()
        evs.append((e0, e1))
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    clocks = sampler.stop() if sampler else None
    total_ms = sum(a.elapsed_time(b) for a, b in evs)
    value, max_ms, units = job_throughput(total_ms, pairs, steps, dev, world)
    achieved = flops / (total_ms / steps / 1e3) / 1e12
    for plan in plans.values():
        plan.close()
    return value, max_ms, pairs, achieved, clocks


BATCH64_DESC = ("batch64: 64 ellipsoid instances (axes U[0.5,2], N log-uniform 5e4-1e6, depth U{3..6}, "
                "p U{6,8,10}, eps 1e-7, d 0.1), 16 rhs each, N(0,1) upward-equivalent densities, all M2L levels "
                "in one grouped batch replayed from a CUDA graph")


def run_batch64(args, rank, world, local_rank):
    import torch

    import __graft_entry__

    if rank == 0:
        __graft_entry__.build()
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    value, max_ms, pairs, achieved, clocks = batch64_measure(args, rank, world, dev, args.steps, args.warmup, True)
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        pass
    bf16_peak = peaks.get("bf16_tflops", 1900.0)
    line = {
        "metric": METRIC, "value": value, "unit": UNIT,
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": max_ms / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": {"f16x3": "f16", "fp32": "f32"}.get(args.precision, "bf16"), "data": "synthetic",
        "config": {"workload": BATCH64_DESC, "pairs_per_step": pairs, "precision": args.precision,
                   "l2": "flushed before every timed step (256 MB write)"},
        "roofline": {"bound": "tensor", "achieved": achieved, "peak": bf16_peak, "unit": "TFLOP/s",
                     "frac": achieved / bf16_peak, "traffic": None,
                     "kernel": "whole batch (compression, core and expansion of three operators)",
                     "flops_per_unit": "2 r^2 per box pair and rhs"},
        # per operator: split + compression, split + expansion; one grouped core
        # launch where the plans allow it (f16x3, split3, bf16), else one per operator
        "clocks": clocks, "e2e": None, "gpu_launches": (13 if args.precision != "split6" else 15) * args.steps,
        "cpu_baseline": None,
    }
    if rank == 0:
        print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", choices=("ours", "reference"), default="ours")
    ap.add_argument("--precision", choices=("f16x3", "split6", "split3", "bf16", "fp32"), default="f16x3")
    ap.add_argument("--no-autotune", action="store_true", help="use the plan's default core variant")
    ap.add_argument("--no-cpu-baseline", action="store_true", help="skip the timed oracle leg")
    ap.add_argument("--no-yukawa", action="store_true", help="skip the per-level Yukawa leg")
    ap.add_argument("--no-extra", action="store_true", help="skip the torus4m_p10 and batch64 legs")
    ap.add_argument("--legs", default="all",
                    help="secondary legs to run besides the headline step, comma-separated from split6, noalloc, "
                         "stage2, fmm, yukawa, torus, batch64; 'all' (default) or 'none' (profiler runs)")
    ap.add_argument("--workload", choices=("sphere2m_p8", "batch64"), default="sphere2m_p8",
                    help="sphere2m_p8: the headline configuration; batch64: the 64-instance mixed batch")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)
    world = env_int("WORLD_SIZE", 1)
    rank = env_int("RANK", 0)
    local_rank = env_int("LOCAL_RANK", 0)
    if args.impl == "reference":
        run_reference(args, rank)
        return
    if world > 1:
        import torch

        torch.cuda.set_device(local_rank)
        torch.distributed.init_process_group("nccl")
    try:
        if args.workload == "batch64":
            run_batch64(args, rank, world, local_rank)
        else:
            run_ours(args, rank, world, local_rank)
    finally:
        if world > 1:
            import torch

            torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
