"""Benchmark of the layered-media Helmholtz FMM evaluation on GB300.

Default workload: the three-layer medium (interfaces z = 0, -1.2; k = 0.8,
1.2, 1.6; eps = 1, 2, 3) with N = 32,768 particles split evenly over the cubes
[-1,1]^2 x {[0.1,1.1], [-1.1,-0.1], [-2.3,-1.3]}, charges U[0,1], targets =
sources, p = 8, leaf 64, FP64 throughout.  One step = one full evaluation
(classification, trees, lists, translation operators looked up in the
handle's per-geometry cache, upward and downward passes, near field, sum),
inputs resident in device memory.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--no-large] [--no-surrogate] [--no-tables] [--no-cpu-baseline]

Extra keys of the JSON line:
  mixed      the same workload in the mixed-precision form (FMM_MIXED)
  surrogate  count-only reaction trees (FMM_TREE_COUNTS), so that the
             reaction components have a near field: FP64 with the quadrature
             near field, then the mixed + surrogate form (FMM_MIXED |
             FMM_SURROGATE) with the network trained on the near-field box
  large      N = 2^20, p = 10, complex charges: FP64 and mixed forms
  tables     the reaction M2L from tabulated integrals (FMM_TABLES): table
             build at create, evaluations with a new geometry every step
             with and without the tables, error against the oracle values
  paper_table  the paper's timing study (Sec. 4, Table 1): irregular domains,
             p = 4, N = 618,256 .. 2,861,288; all components, the 3
             free-space ones and the 3 reaction ones the table selects
  errors     each form against oracle values stored in
             tests/golden/oracle_values_full.npz (written offline by
             tests/golden/make_golden_full.py from the oracle alone)

Multi-GPU (torchrun): every rank evaluates its own independent problem of the
same size (weak scaling, no data-path collective); the barrier and the
max-over-ranks time use torch.distributed.  With --split components the
ranks share ONE problem instead: each evaluates a contiguous range of its
components (chosen from the work estimate of one all-component evaluation)
and the potentials are summed along the ranks in component order
(paper_1902_05132_gb300.distributed.chain_sum over NCCL), inside the timed
step (strong scaling).  --impl reference times the CPU
oracle (the only reference implementation this project has) on a bounded
sample of the same workload, on all host cores.
"""
import argparse
import json
import multiprocessing as mp
import os
import platform
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

WORKLOADS = {
    # the configuration the metric is quoted on (default)
    "three-layer-32768": dict(name="three-layer N=32768 p=8 leaf=64", n=32768, p=8, leaf=64, complex=False),
    # the large configuration of the mixed-precision form: N = 2^20, p = 10, complex charges
    "three-layer-1M": dict(name="three-layer N=1048576 p=10 leaf=64 complex charges", n=1048576, p=10, leaf=64,
                           complex=True),
}
WORKLOAD = WORKLOADS["three-layer-32768"]
METRIC = "FMM particles/sec at rel L2 err 1e-6 (FP64)"
L2_BYTES = 129 * 1024 * 1024
GOLDEN = os.path.join(ROOT, "tests", "golden", "oracle_values_full.npz")
# DRAM bytes (read + write) of the M2L product launches of one evaluation,
# per (workload, form), from an ncu capture of the current kernels (absent once
# a kernel changes); the capture command is in the kernel's profile summary.
NCU_TRAFFIC = {
    # k_zrot (autotuned tile) + k_zgemm_res
    ("three-layer N=32768 p=8 leaf=64", "fp64"): 94.662144e6 + 43.065088e6 + 806.672384e6 + 646.199040e6,
    ("three-layer N=32768 p=8 leaf=64", "mixed"): 1260.710e6 + 755.058432e6,
}


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def aggregate(total_ms, steps, n_per_rank, ws, device):
    """Whole-job time and throughput: the slowest rank's time of the timed
    steps (max over ranks), and the units all ranks processed per second
    (each rank evaluates its own problem of n_per_rank particles)."""
    if ws > 1:
        import torch
        import torch.distributed as dist
        t = torch.tensor([total_ms], device=device, dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total_ms = float(t.item())
    ms_per_step = total_ms / steps
    return ms_per_step, ws * n_per_rank / (ms_per_step * 1e-3)


def _clock_sampler(path, dev):
    q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
    try:
        return subprocess.Popen(["nvidia-smi", f"--id={dev}", f"--query-gpu={q}", "--format=csv,noheader,nounits",
                                 "-lms", "200"], stdout=open(path, "w"), stderr=subprocess.DEVNULL)
    except Exception:
        return None


def _clock_summary(path):
    sm, mx, reasons = [], [], set()
    names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
    try:
        for line in open(path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
    except OSError:
        pass
    if not sm:
        return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"]}
    return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
            "samples": len(sm)}


def _hbm_peak():
    """HBM bandwidth: the measured copy figure of this machine, else the fallback."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"]), "measured copy bandwidth (of measured)"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback 6.8 TB/s (of fallback)"


def _tensor_peak():
    """Dense FP16 tensor peak: the measured bf16 burst figure of this machine
    (FP16 and BF16 run at the same nominal rate), else the fallback."""
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            return float(json.load(f)["bf16_tflops"]), "measured bf16 dense burst x 1 (fp16 nominal ratio) (of measured)"
    except (OSError, KeyError, ValueError):
        return 1900.0, "fallback 1.9 PFLOP/s bf16 dense (of fallback)"


def _cpu_model():
    try:
        for line in open("/proc/cpuinfo"):
            if line.lower().startswith(("model name", "cpu model")):
                return line.split(":", 1)[1].strip()
    except OSError:
        pass
    return platform.processor() or platform.machine()


def _golden():
    try:
        return np.load(GOLDEN)
    except OSError:
        return None


def _rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b)))


def timed_evals(torch, solver, src, q, tgt, out, steps, warmup, flush, stream, nvtx=None):
    """Warm-up, then `steps` evaluations each timed with CUDA events on the
    evaluation stream, the L2 flushed before each; returns (ms list, stats).
    `nvtx` names a range around the timed evaluations (for a profiler)."""
    for _ in range(max(3, warmup)):
        solver.eval(src, q, tgt, out=out)
    ms, stats = [], []
    if nvtx:
        torch.cuda.nvtx.range_push(nvtx)
    for _ in range(steps):
        flush.fill_(1.0)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        solver.eval(src, q, tgt, out=out)
        e1.record(stream)
        e1.synchronize()
        ms.append(e0.elapsed_time(e1))
        stats.append(solver.stats())
    if nvtx:
        torch.cuda.nvtx.range_pop()
    return ms, stats


STAGES = ["tree", "operators", "upward", "m2l", "l2p", "near_free", "near_reac", "sum"]


def _stage_ms(stats):
    return {k: statistics.mean(s["gpu_ms_" + k] for s in stats) for k in STAGES}


def _oracle_worker(args):
    n, seed, p, leaf, complex_charges, idx = args
    sys.path.insert(0, ROOT)
    from oracle import green
    from oracle.media import Medium
    from paper_1902_05132_gb300 import workloads as wl
    w = wl.three_layer(n=n, seed=seed, p=p, leaf=leaf, complex_charges=complex_charges)
    m = Medium(w["k"], w["d"], w["eps"])
    green.direct_sum(m, w["src"], w["q"], w["tgt"], targets=idx)
    return len(idx)


def cpu_oracle_sample(n_targets, cores=None, seed=0):
    """Time the oracle as it stands (FP64 direct sum with Sommerfeld
    quadrature) at n_targets sampled targets of the workload against all its
    sources, the targets spread over `cores` worker processes (spawn, one
    thread each).  Returns (targets per second, seconds, cores)."""
    from paper_1902_05132_gb300 import workloads as wl
    cores = cores or os.cpu_count() or 1
    cores = max(1, min(cores, n_targets))
    sel = wl.sample_targets(WORKLOAD["n"], n_targets, seed=3)
    parts = [c for c in np.array_split(sel, cores) if len(c)]
    for var in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ[var] = "1"
    ctx = mp.get_context("spawn")
    with ctx.Pool(len(parts)) as pool:
        args = [(WORKLOAD["n"], seed, WORKLOAD["p"], WORKLOAD["leaf"], WORKLOAD["complex"], c) for c in parts]
        empty = np.zeros(0, dtype=np.int64)                 # imports done in every worker before timing
        pool.map(_oracle_worker, [a[:-1] + (empty,) for a in args], chunksize=1)
        t = time.perf_counter()
        done = sum(pool.map(_oracle_worker, args, chunksize=1))
        sec = time.perf_counter() - t
    return done / sec, sec, len(parts)


def run_reference(args):
    ws, rank, _ = _dist()
    if rank != 0:
        return
    cores = os.cpu_count() or 1
    n_sample = max(cores, 2 * cores * 32768 // WORKLOAD["n"])
    vals, secs = [], []
    used = 1
    for _ in range(args.steps):
        v, s, used = cpu_oracle_sample(n_sample, cores)
        vals.append(v)
        secs.append(s)
    value = statistics.median(vals)
    sample = (f"oracle direct sum (FP64, Sommerfeld quadrature) at {n_sample} sampled targets of the "
              f"{WORKLOAD['name']} workload against all its sources per step, spread over {used} worker processes "
              f"on {cores} host cores ({_cpu_model()})")
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": "particles/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * statistics.median(secs),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD["name"], "sample_targets": n_sample},
        "cpu_baseline": {"value": value, "unit": "particles/s", "cores": used, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": "particles/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }))


def mixed_leg(pkg, torch, w, src, q, tgt, ref_out, args, flush, stream, ws):
    """The mixed-precision form on the same workload: throughput, error
    against the FP64 path, roofline of the tensor-core M2L product."""
    n = len(w["tgt"])
    mixed = pkg.LayeredFMM(w["k"], w["d"], w["eps"], p=w["p"], leaf=w["leaf"], mixed=True)
    out_m = torch.empty_like(ref_out)
    mms, mst = timed_evals(torch, mixed, src, q, tgt, out_m, args.steps, args.warmup, flush, stream,
                           nvtx="timed_mixed")
    mixed.close()
    m_ms = statistics.mean(mms)
    tc_ms = statistics.mean(s["gpu_ms_m2l_gemm"] for s in mst)
    tc_flops = mst[-1]["m2l_tensor_flops"]
    bf16_peak, peak_src = _tensor_peak()
    tc_achieved = tc_flops / (tc_ms * 1e-3) / 1e12
    tc_bytes = mst[-1]["m2l_tc_bytes"]
    tc_gbs = tc_bytes / (tc_ms * 1e-3) / 1e9
    hbm_peak, hbm_src = _hbm_peak()
    res = {
        "value": ws * n / (m_ms * 1e-3), "unit": "particles/s", "ms_per_step": m_ms,
        "rel_l2_vs_fp64_path": float(torch.linalg.vector_norm(out_m - ref_out) / torch.linalg.vector_norm(ref_out)),
        "dtype": "f16 hi/lo -> f32 (M2L), f64 elsewhere", "stage_ms": _stage_ms(mst),
        # the product moves ~70 flop per byte, below the FP16 tensor balance
        # point (peak flops / HBM bandwidth ~ 280): it is bounded by HBM
        "roofline": {"bound": "hbm", "kernel": "k_m2l_tc", "achieved": tc_gbs, "peak": hbm_peak, "unit": "GB/s",
                     "frac": tc_gbs / hbm_peak, "traffic": NCU_TRAFFIC.get((w["name"], "mixed")),
                     "kernel_ms": tc_ms, "algorithmic_gb": tc_bytes / 1e9, "peak_source": hbm_src,
                     "tensor": {"achieved": tc_achieved, "peak": bf16_peak, "unit": "TFLOP/s",
                                "frac": tc_achieved / bf16_peak, "executed_tflop": tc_flops / 1e12,
                                "peak_source": peak_src},
                     "algorithmic_fp64_equiv_tflop": mst[-1]["m2l_gemm_flops"] / 1e12},
    }
    return res, out_m


def surrogate_leg(pkg, torch, w, src, q, tgt, ref_out, args, flush, stream, ws, gold):
    """Count-only reaction trees (FMM_TREE_COUNTS): the reaction components
    get a near field.  FP64 with the quadrature there (the method without
    the network), then the surrogate trained on the (rho, zt, zs) box that
    near field needs, and the mixed + surrogate form timed on the same trees;
    last FP64 with the near-field kernel from the tables (FMM_TABLES)."""
    n = len(w["tgt"])
    out = torch.empty_like(ref_out)
    plain = pkg.LayeredFMM(w["k"], w["d"], w["eps"], p=w["p"], leaf=w["leaf"], tree_counts=True)
    qms, qst = timed_evals(torch, plain, src, q, tgt, out, max(1, args.steps // 2), 1, flush, stream)
    out_q = out.clone()
    plain.close()
    st_q = qst[-1]
    box = dict(rho_max=1.001 * st_q["reac_near_rho_max"], z_min=0.999 * st_q["reac_near_z_min"],
               z_max=1.001 * st_q["reac_near_z_max"])
    ms_surr = pkg.LayeredFMM(w["k"], w["d"], w["eps"], p=w["p"], leaf=w["leaf"], tree_counts=True, mixed=True,
                             surrogate=True)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    err, ok = ms_surr.train_surrogate(**box, samples=262144, steps=8000, bound=1e-5, seed=5)
    train_s = time.perf_counter() - t0
    judged = err[err >= 0]
    sms, sst = timed_evals(torch, ms_surr, src, q, tgt, out, args.steps, args.warmup, flush, stream,
                           nvtx="timed_mixed_surrogate")
    ms_surr.close()
    st_s = sst[-1]
    # FP64 with the tabulated near-field kernel (FMM_TABLES): no network, no quadrature
    tab = pkg.LayeredFMM(w["k"], w["d"], w["eps"], p=w["p"], leaf=w["leaf"], tree_counts=True, tables=True)
    out_t = torch.empty_like(ref_out)
    tms, tst = timed_evals(torch, tab, src, q, tgt, out_t, args.steps, args.warmup, flush, stream,
                           nvtx="timed_tables_near")
    tab.close()
    st_t = tst[-1]
    res = {
        "trees": "count-only reaction trees (FMM_TREE_COUNTS)",
        "fp64_quadrature": {"value": ws * n / (statistics.mean(qms) * 1e-3), "ms_per_step": statistics.mean(qms),
                            "near_reac_ms": statistics.mean(s["gpu_ms_near_reac"] for s in qst),
                            "n_reac_pairs": st_q["n_reac_pairs"], "n_reac_nodes": st_q["n_reac_nodes"],
                            "rel_l2_vs_fp64_path": _rel(out_q.cpu().numpy(), ref_out.cpu().numpy())},
        "training": {"box": box, "samples_per_component": 262144, "steps": 8000, "train_s": train_s,
                     "components": int((err >= 0).any(axis=1).sum()),
                     "heldout_rel_rms_median": float(np.median(judged)), "heldout_rel_rms_max": float(judged.max()),
                     "cells_within_1e-5": int(ok.sum()), "cells": int(judged.size)},
        "mixed_surrogate": {"value": ws * n / (statistics.mean(sms) * 1e-3), "unit": "particles/s",
                            "ms_per_step": statistics.mean(sms), "stage_ms": _stage_ms(sst),
                            "surrogate_pairs": st_s["n_reac_surr_pairs"], "reac_pairs": st_s["n_reac_pairs"],
                            "surrogate_fraction": st_s["n_reac_surr_pairs"] / max(1, st_s["n_reac_pairs"]),
                            "rel_l2_vs_fp64_path": _rel(out.cpu().numpy(), ref_out.cpu().numpy())},
        "fp64_tables": {"value": ws * n / (statistics.mean(tms) * 1e-3), "unit": "particles/s",
                        "ms_per_step": statistics.mean(tms),
                        "near_reac_ms": statistics.mean(s["gpu_ms_near_reac"] for s in tst),
                        "table_pairs": st_t["n_reac_table_pairs"], "reac_pairs": st_t["n_reac_pairs"],
                        "rel_l2_vs_fp64_quadrature": _rel(out_t.cpu().numpy(), out_q.cpu().numpy()),
                        "rel_l2_vs_fp64_path": _rel(out_t.cpu().numpy(), ref_out.cpu().numpy())},
    }
    if gold is not None:
        sel = gold["three_layer_sel2000"]
        res["fp64_tables"]["rel_l2_vs_oracle_direct_2000"] = _rel(out_t.cpu().numpy()[sel],
                                                                  gold["three_layer_direct2000"])
        res["mixed_surrogate"]["rel_l2_vs_oracle_direct_2000"] = _rel(out.cpu().numpy()[sel],
                                                                      gold["three_layer_direct2000"])
        res["fp64_quadrature"]["rel_l2_vs_oracle_direct_2000"] = _rel(out_q.cpu().numpy()[sel],
                                                                      gold["three_layer_direct2000"])
    return res


def large_leg(pkg, torch, dev, args, flush, stream, gold):
    """N = 2^20, p = 10, complex charges: FP64 and mixed forms, each against
    the oracle direct sum at the stored sampled targets."""
    from paper_1902_05132_gb300 import workloads
    spec = WORKLOADS["three-layer-1M"]
    w = workloads.three_layer(n=spec["n"], p=spec["p"], leaf=spec["leaf"], complex_charges=True)
    src = torch.tensor(w["src"], device=dev)
    q = torch.tensor(w["q"], device=dev)
    tgt = torch.tensor(w["tgt"], device=dev)
    n = len(w["tgt"])
    res = {"workload": spec["name"]}
    outs = {}
    for form, kw in (("fp64", {}), ("mixed", {"mixed": True})):
        s = pkg.LayeredFMM(w["k"], w["d"], w["eps"], p=w["p"], leaf=w["leaf"], **kw)
        out = torch.empty(n, dtype=torch.complex128, device=dev)
        ms, st = timed_evals(torch, s, src, q, tgt, out, max(2, args.steps // 2), 3, flush, stream)
        s.close()
        r = {"value": n / (statistics.mean(ms) * 1e-3), "unit": "particles/s", "ms_per_step": statistics.mean(ms),
             "stage_ms": _stage_ms(st), "m2l_kernel_ms": statistics.mean(x["gpu_ms_m2l_gemm"] for x in st)}
        if form == "fp64":
            peak = pkg.measure_fp64_peak() / 1e3
            ach = st[-1]["m2l_gemm_flops"] / (r["m2l_kernel_ms"] * 1e-3) / 1e12
            r["roofline"] = {"bound": "alu", "kernel": "k_zrot + k_zgemm_res", "achieved": ach, "peak": peak,
                             "unit": "TFLOP/s", "frac": ach / peak, "traffic": None}
        else:
            hbm, _ = _hbm_peak()
            gbs = st[-1]["m2l_tc_bytes"] / (r["m2l_kernel_ms"] * 1e-3) / 1e9
            r["roofline"] = {"bound": "hbm", "kernel": "k_m2l_tc", "achieved": gbs, "peak": hbm, "unit": "GB/s",
                             "frac": gbs / hbm, "traffic": None}
        outs[form] = out.cpu().numpy()
        if gold is not None:
            sel = gold["three_layer_1m_sel"]
            r["rel_l2_vs_oracle_direct"] = _rel(outs[form][sel], gold["three_layer_1m_direct"])
            r["oracle_targets"] = int(len(sel))
        res[form] = r
    res["mixed"]["rel_l2_vs_fp64_path"] = _rel(outs["mixed"], outs["fp64"])
    return res


# the paper's Table 1 (Sec. 4): N, free-space time (all 3 components) and
# reaction time (3 selected components) on 36 Xeon E5-2699 v4 cores, p = 4
PAPER_TABLE_36 = {618256: (2.29, 2.74), 1128556: (5.00, 3.21), 1862568: (11.45, 3.59), 2861288: (12.60, 3.90)}


def tables_leg(pkg, torch, w, src, q, tgt, out, args, flush, stream, gold):
    """Tabulated reaction M2L integrals (FMM_TABLES, Sec. 3.5): table build at
    create, then evaluations whose geometry changes every step (all points
    moved by a few 1e-4 along a fixed random direction field, so every box
    width and hence every translation operator is new), with and without
    the tables; the error of the tables path against the stored oracle values."""
    rng = np.random.default_rng(7)
    field = torch.tensor(rng.uniform(-1.0, 1.0, size=tuple(src.shape)), device=src.device)
    field[:, 2] *= 0.5
    t0 = time.perf_counter()
    tab = pkg.LayeredFMM(w["k"], w["d"], w["eps"], p=w["p"], leaf=w["leaf"], tables=True)
    create_s = time.perf_counter() - t0
    st0 = tab.stats()
    res = {"create_s": create_s, "build_ms": st0["ms_tables"], "table_bytes": st0["table_bytes"]}
    tab.eval(src, q, tgt, out=out)
    if gold is not None:
        res["rel_l2_vs_oracle_direct_2000"] = _rel(out.cpu().numpy()[gold["three_layer_sel2000"]],
                                                   gold["three_layer_direct2000"])
        res["rel_l2_vs_oracle_fmm_200"] = _rel(out.cpu().numpy()[gold["three_layer_fmm_sel"]],
                                               gold["three_layer_fmm200"])

    def moving(solver, steps, j0):
        ms, stats = [], []
        for j in range(steps):
            s_j = src + (j0 + j + 1) * 2e-4 * field
            flush.fill_(1.0)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            solver.eval(s_j, q, s_j, out=out)
            e1.record(stream)
            e1.synchronize()
            ms.append(e0.elapsed_time(e1))
            stats.append(solver.stats())
        return ms, stats

    n = len(w["tgt"])
    ms, stats = moving(tab, max(3, args.steps), 0)
    res["moving_geometry"] = {
        "value": n / (statistics.mean(ms) * 1e-3), "unit": "particles/s", "ms_per_step": statistics.mean(ms),
        "operators_ms": statistics.mean(s["gpu_ms_operators"] for s in stats),
        "table_classes_per_step": stats[-1]["n_reac_table_classes"],
        "quadrature_nodes": stats[-1]["n_reac_T_nodes"]}
    tab.close()
    quad = pkg.LayeredFMM(w["k"], w["d"], w["eps"], p=w["p"], leaf=w["leaf"])
    quad.eval(src, q, tgt, out=out)
    msq, statsq = moving(quad, 2, 100)
    res["moving_geometry_quadrature"] = {
        "value": n / (statistics.mean(msq) * 1e-3), "unit": "particles/s", "ms_per_step": statistics.mean(msq),
        "operators_ms": statistics.mean(s["gpu_ms_operators"] for s in statsq),
        "reaction_classes_per_step": statsq[-1]["n_reac_classes"]}
    quad.close()
    return res


def paper_table_leg(pkg, torch, dev, flush, stream):
    """The paper's timing study (Sec. 4, Table 1) on its own workload: the
    irregular domains of workloads.paper_domains scaled to the table's N,
    p = 4, FP64.  Times all 19 components, the 3 free-space components, and
    the 3 reaction components the table selects (u_00^{up up}, u_11^{up up},
    u_22^{down down}: components 3, 9 and 18 of the library's order)."""
    from paper_1902_05132_gb300 import workloads
    rows = []
    for n, (t_free36, t_reac36) in PAPER_TABLE_36.items():
        base = np.array([912, 640, 1296], dtype=float)
        counts = np.floor(n * base / base.sum()).astype(int)
        counts[0] += n - counts.sum()
        w = workloads.paper_domains(counts=tuple(int(c) for c in counts), p=4, leaf=64)
        src = torch.tensor(w["src"], device=dev)
        q = torch.tensor(w["q"], device=dev)
        tgt = torch.tensor(w["tgt"], device=dev)
        out = torch.empty(n, dtype=torch.complex128, device=dev)
        row = {"n": n}
        for name, ranges in (("all", [(0, -1)]), ("free3", [(0, 3)]), ("reac3", [(3, 1), (9, 1), (18, 1)])):
            tot = 0.0
            for first, count in ranges:
                s = pkg.LayeredFMM(w["k"], w["d"], w["eps"], p=4, leaf=64)
                s.set_components(first, count)
                ms, _ = timed_evals(torch, s, src, q, tgt, out, 2, 1, flush, stream)
                s.close()
                tot += statistics.mean(ms)
            row[name + "_ms"] = tot
        row["particles_per_s"] = n / (row["all_ms"] * 1e-3)
        row["free3_particles_per_s"] = n / (row["free3_ms"] * 1e-3)
        row["paper_36_cores_s"] = {"free3": t_free36, "reac3": t_reac36,
                                   "free3_particles_per_s": n / t_free36}
        rows.append(row)
        del src, q, tgt, out
    return {"workload": "paper domains (Sec. 4), k=(1.2,1.5,1.8), p=4, leaf 64, FP64; the paper's times are "
                        "2x Xeon E5-2699 v4, 36 cores (context only)", "rows": rows}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-surrogate", action="store_true")
    ap.add_argument("--no-large", action="store_true")
    ap.add_argument("--no-paper-table", action="store_true")
    ap.add_argument("--no-tables", action="store_true")
    ap.add_argument("--workload", default="three-layer-32768", choices=sorted(WORKLOADS))
    ap.add_argument("--split", default="problems", choices=["problems", "components"])
    args = ap.parse_args()
    global WORKLOAD
    WORKLOAD = WORKLOADS[args.workload]
    if args.impl == "reference":
        return run_reference(args)

    import torch

    import paper_1902_05132_gb300 as pkg
    from paper_1902_05132_gb300 import _build, workloads

    ws, rank, local = _dist()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    _build.build()
    split = args.split == "components" and ws > 1
    w = workloads.three_layer(n=WORKLOAD["n"], seed=0 if split else rank, p=WORKLOAD["p"], leaf=WORKLOAD["leaf"],
                              complex_charges=WORKLOAD["complex"])
    solver = pkg.LayeredFMM(w["k"], w["d"], w["eps"], p=w["p"], leaf=w["leaf"])
    src = torch.tensor(w["src"], device=dev)
    q = torch.tensor(w["q"], device=dev)
    tgt = torch.tensor(w["tgt"], device=dev)
    out = torch.empty(len(w["tgt"]), dtype=torch.complex128, device=dev)
    flush = torch.empty(2 * L2_BYTES // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream(dev)
    step = None
    if split:
        from paper_1902_05132_gb300 import distributed
        solver.eval(src, q, tgt, out=out)                    # plan: work of every component
        work = torch.tensor(solver.component_work(), dtype=torch.float64, device=dev)
        dist.broadcast(work, src=0)
        first, count = distributed.partition(work.cpu().tolist(), ws)[rank]
        solver.set_components(first, count)
        part = torch.empty_like(out)

        def step():
            solver.eval(src, q, tgt, out=part)
            distributed.chain_sum(out, solver.add_components, rank, ws, dist,
                                  own_result=part if rank == 0 else None)
    else:
        def step():
            solver.eval(src, q, tgt, out=out)
    for _ in range(max(3, args.warmup)):
        step()
    torch.cuda.synchronize()
    clock_dir = os.environ.get("FMM_BENCH_CLOCKS_DIR") or tempfile.mkdtemp(prefix="fmm_bench_")
    os.makedirs(clock_dir, exist_ok=True)
    clock_path = os.path.join(clock_dir, f"bench_clocks_r{rank}.csv")
    sampler = _clock_sampler(clock_path, local)
    time.sleep(0.3)
    if ws > 1:
        dist.barrier()
    torch.cuda.synchronize()
    ms, stage = [], []
    launches = 0
    torch.cuda.nvtx.range_push("timed")      # lets a profiler select the timed steps
    for _ in range(args.steps):
        flush.fill_(1.0)                      # evict the L2 between steps
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        step()
        e1.record(stream)
        e1.synchronize()
        ms.append(e0.elapsed_time(e1))
        st = solver.stats()
        stage.append(st)
        launches += st["n_launches"]
    torch.cuda.nvtx.range_pop()
    torch.cuda.synchronize()
    if ws > 1:
        dist.barrier()
    if sampler:
        sampler.terminate()
        sampler.wait()
    n = len(w["tgt"])
    ms_per_step, value = aggregate(sum(ms), args.steps, n, ws, dev)
    if split:                     # one problem shared by all ranks: N particles per step
        value /= ws
        if rank == 0:
            print(json.dumps({
                "metric": METRIC, "value": value, "unit": "particles/s", "n_gpus": ws, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "strong",
                "vs_baseline": None, "dtype": "f64", "data": "synthetic",
                "config": {"workload": WORKLOAD["name"], "parallelism": f"components of one problem over {ws} GPUs, "
                           "chain sum of the potentials in component order (NCCL)",
                           "l2": "flushed between steps (256 MB write)"},
                "clocks": _clock_summary(clock_path), "gpu_launches": launches}))
        dist.destroy_process_group()
        return

    # first evaluation of a fresh solver: translation operators not cached yet
    cold = pkg.LayeredFMM(w["k"], w["d"], w["eps"], p=w["p"], leaf=w["leaf"])
    flush.fill_(1.0)
    torch.cuda.synchronize()
    c0, c1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    c0.record(stream)
    cold.eval(src, q, tgt, out=out)
    c1.record(stream)
    c1.synchronize()
    cst = cold.stats()
    cold_info = {"ms": c0.elapsed_time(c1), "operators_ms": cst["gpu_ms_operators"],
                 "reaction_classes": cst["n_reac_classes"], "free_operators": cst["n_free_ops"],
                 "particles_per_s": n / (c0.elapsed_time(c1) * 1e-3)}
    cold.close()

    # end to end through the public API with host buffers (pinned)
    hs = torch.tensor(w["src"]).pin_memory().numpy()
    hq = torch.tensor(w["q"]).pin_memory().numpy()
    ht = torch.tensor(w["tgt"]).pin_memory().numpy()
    solver.eval_host(hs, hq, ht)
    e2e_ms = []
    for _ in range(args.steps):
        flush.fill_(1.0)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        res = solver.eval_host(hs, hq, ht)
        e2e_ms.append(1e3 * (time.perf_counter() - t0))
    e2e_value = ws * n / (statistics.mean(e2e_ms) * 1e-3)
    h2d = hs.nbytes + hq.nbytes + ht.nbytes
    d2h = res.nbytes

    # roofline of the dominant kernels: the M2L translations (k_zrot for
    # free-space classes in rotation form, k_zgemm_res for reaction classes),
    # timed by the library's CUDA events around their launches on the
    # evaluation's stream; FP64 pipe peak measured on this GPU now
    gemm_ms = statistics.mean(s["gpu_ms_m2l_gemm"] for s in stage)
    gemm_flops = stage[-1]["m2l_gemm_flops"]
    peak = pkg.measure_fp64_peak() / 1e3
    achieved = gemm_flops / (gemm_ms * 1e-3) / 1e12
    result = {
        "metric": METRIC, "value": value, "unit": "particles/s", "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD["name"], "medium": "3 layers, d=(0,-1.2), k=(0.8,1.2,1.6), eps=(1,2,3)",
                   "l2": "flushed between steps (256 MB write)", "parallelism": f"independent problem per GPU x{ws}",
                   "operators": "translation operators cached in the handle per geometry (warm); a new geometry "
                                "pays cold_first_eval"},
        "clocks": _clock_summary(clock_path),
        "e2e": {"value": e2e_value, "unit": "particles/s", "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
        "gpu_launches": launches,
        "roofline": {"bound": "alu", "kernel": "k_zrot + k_zgemm_res", "achieved": achieved, "peak": peak,
                     "unit": "TFLOP/s", "frac": achieved / peak,
                     "traffic": NCU_TRAFFIC.get((WORKLOAD["name"], "fp64")),
                     "per": "the M2L translation launches of one evaluation (free-space and reaction classes)",
                     "kernel_ms": gemm_ms, "algorithmic_tflop": gemm_flops / 1e12,
                     "peak_source": "FP64 FMA throughput measured on this GPU by the library's probe (of measured)"},
        "stage_ms": _stage_ms(stage),
        "m2l_autotune": {"kernel": "k_zrot", "column_tile": stage[-1]["tune_zrot_kc"],
                         "threads": stage[-1]["tune_zrot_threads"],
                         "candidates": stage[-1]["tune_zrot_candidates"],
                         "chosen_ms": stage[-1]["tune_zrot_ms"], "fixed_rule_ms": stage[-1]["tune_zrot_rule_ms"]},
        "cold_first_eval": cold_info,
        "counts": {k: stage[-1][k] for k in ("n_components", "n_boxes", "n_v_pairs", "n_v_pairs_reac", "n_free_pairs",
                                             "n_reac_pairs", "n_reac_nodes", "n_reac_classes", "n_reac_T_nodes")},
    }
    gold = _golden() if WORKLOAD["n"] == 32768 and not WORKLOAD["complex"] and rank == 0 else None
    ref_out = out.clone()
    if gold is not None:
        sel = gold["three_layer_sel2000"]
        result["errors"] = {"fp64_vs_oracle_direct_2000": _rel(ref_out.cpu().numpy()[sel],
                                                               gold["three_layer_direct2000"]),
                            "fp64_vs_oracle_fmm_200": _rel(ref_out.cpu().numpy()[gold["three_layer_fmm_sel"]],
                                                           gold["three_layer_fmm200"])}
    result["mixed"], out_m = mixed_leg(pkg, torch, w, src, q, tgt, ref_out, args, flush, stream, ws)
    if gold is not None:
        result["errors"]["mixed_vs_oracle_direct_2000"] = _rel(out_m.cpu().numpy()[gold["three_layer_sel2000"]],
                                                               gold["three_layer_direct2000"])
    if not args.no_tables and ws == 1:
        result["tables"] = tables_leg(pkg, torch, w, src, q, tgt, torch.empty_like(out), args, flush, stream, gold)
    if not args.no_surrogate:
        result["surrogate"] = surrogate_leg(pkg, torch, w, src, q, tgt, ref_out, args, flush, stream, ws, gold)
    if not args.no_large and ws == 1:
        result["large"] = large_leg(pkg, torch, dev, args, flush, stream, _golden())
    if not args.no_paper_table and ws == 1:
        result["paper_table"] = paper_table_leg(pkg, torch, dev, flush, stream)
    if rank == 0 and not args.no_cpu_baseline and ws == 1:
        cores = os.cpu_count() or 1
        n_sample = max(cores, 2 * cores * 32768 // WORKLOAD["n"])   # about 10-30 s of oracle work in all
        v, sec, used = cpu_oracle_sample(n_sample, cores)
        result["cpu_baseline"] = {"value": v, "unit": "particles/s", "cores": used, "kind": "oracle",
                                  "sample": f"oracle direct sum (FP64, Sommerfeld quadrature) at {n_sample} sampled "
                                            f"targets of the same workload against all {n} sources, spread over "
                                            f"{used} worker processes on {cores} host cores ({_cpu_model()}), "
                                            f"{sec:.1f} s"}
    if rank == 0:
        print(json.dumps(result))
    if ws > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
