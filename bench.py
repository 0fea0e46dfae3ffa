"""Throughput of the slice-sweep transport path on GB300.

Default workload (one step = the whole hot path once): square lattice t = 1,
M = 64 orbitals per slice, L = 512 slices, two clean leads of width 64,
Anderson disorder W = 2, 1024 midpoint energies in (-3.9, 3.9) x 8 disorder
seeds = 8192 instances.  Each step computes the lead self-energies for every
energy (transverse-mode solver, FP64), runs the mixed-precision sweep for all
instances and returns T for each.  Metric: T(E) points/s (instances/s), with
slice-updates/s beside it, the plain FP64 GPU sweep timed on a one-wave
subset, and the CPU oracle timed on a bounded sample.

python bench.py [--gpus N] [--steps K] [--warmup W] [--impl knit|reference]
Under torchrun (N > 1) every rank runs its own copy of the workload with
energies shifted by rank (weak scaling); no data-path collective.
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

M, L, W = 64, 512, 2.0
NE, NS = 1024, 8
METRIC = "T(E) points/s (mixed sweep, |dT| <= 1e-6 vs FP64)"
WORKLOAD = "square M=64 L=512 W=2, 1024 energies x 8 seeds, two clean leads"
PEAKS = os.path.join(ROOT, "MEASURED_PEAKS.json")
# DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) of one launch of
# the sweep kernel on this workload, for the kernel as it stands: taken on the
# 152-instance profile case (one kernel, one launch: 1.387 MB) and scaled by
# instances to 8192 (the traffic is per instance: parameters and self-energy
# blocks); set to None whenever the kernel changes until it is measured again
SWEEP_TRAFFIC_BYTES = 1.387008e6 * 8192 / 152
L2_BYTES = 126 * 1024 * 1024


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    return ws, rank


def _clock_sampler():
    try:
        return subprocess.Popen(
            ["nvidia-smi", "--query-gpu=index,clocks.sm,clocks.max.sm,power.draw,"
             "clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
             "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
             "clocks_event_reasons.sw_power_cap", "--format=csv,noheader,nounits", "-lms", "200"],
            stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
    except Exception:
        return None


def _smi_index(dev_index, seen):
    """nvidia-smi's index of CUDA device dev_index: through
    CUDA_VISIBLE_DEVICES when it lists plain indices, else the same number;
    the only index sampled when that one is absent."""
    want = str(dev_index)
    vis = [x.strip() for x in os.environ.get("CUDA_VISIBLE_DEVICES", "").split(",") if x.strip()]
    if dev_index < len(vis) and vis[dev_index].isdigit():
        want = vis[dev_index]
    if want not in seen and len(seen) == 1:
        want = next(iter(seen))
    return want


def _clock_summary(proc, dev_index):
    if proc is None:
        return None
    proc.terminate()
    try:
        out, _ = proc.communicate(timeout=5)
    except Exception:
        proc.kill()
        out, _ = proc.communicate()
    return _parse_clocks(out, dev_index)


def _parse_clocks(out, dev_index):
    sm, mx, reasons = [], [], set()
    names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
    rows = [[x.strip() for x in line.split(",")] for line in out.splitlines()]
    rows = [f for f in rows if len(f) >= 9]
    want = _smi_index(dev_index, {f[0] for f in rows})
    for f in rows:
        if f[0] != want:
            continue
        try:
            sm.append(float(f[1]))
            mx.append(float(f[2]))
        except ValueError:
            continue
        for n, v in zip(names, f[5:9]):
            if v.lower() == "active":
                reasons.add(n)
    if not sm:
        return None
    return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "samples": len(sm),
            "reasons": sorted(reasons)}


def _peaks():
    try:
        with open(PEAKS) as f:
            return json.load(f)
    except Exception:
        return {}


# iterations per launch of each peak loop (a few ms each on GB300)
PEAK_ITERS = {"mma_bf16_tflops": 40000, "mma_tf32_tflops": 40000, "dfma_tflops": 2000,
              "ffma_tflops": 20000, "mma_bf16_pattern_tflops": 8000,
              "mma_tf32_pattern_tflops": 8000}


def measure_peaks(knit, torch, stream, nsm, reps=5):
    """The library's own peak loops (tcgen05 kind::f16 and kind::tf32 dense
    MMA, FP64 and FP32 FMA), each timed with CUDA events on `stream` over
    `reps` launches after one warm-up launch (median), with the SM clock
    sampled during the loops.  Returns TFLOP/s per kind."""
    kinds = {"mma_bf16_tflops": knit.KNIT_PEAK_MMA_BF16, "mma_tf32_tflops": knit.KNIT_PEAK_MMA_TF32,
             "dfma_tflops": knit.KNIT_PEAK_DFMA, "ffma_tflops": knit.KNIT_PEAK_FFMA,
             "mma_bf16_pattern_tflops": knit.KNIT_PEAK_MMA_RESIDUAL,
             "mma_tf32_pattern_tflops": knit.KNIT_PEAK_MMA_RESIDUAL_TF32}
    out = {}
    clocks = _clock_sampler()
    for name, kind in kinds.items():
        knit.knit_peak_probe(kind, PEAK_ITERS[name], nsm, stream=stream, check=True)
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
              for _ in range(reps)]
        flop = 0.0
        with torch.cuda.stream(stream):
            for a, b in ev:
                a.record(stream)
                flop = knit.knit_peak_probe(kind, PEAK_ITERS[name], nsm, stream=stream)
                b.record(stream)
        torch.cuda.synchronize()
        ms = statistics.median(a.elapsed_time(b) for a, b in ev)
        out[name] = flop / (ms / 1e3) / 1e12
    out["clocks"] = _clock_summary(clocks, torch.cuda.current_device())
    out["nsm"] = nsm
    # the roofline denominators: the higher of the two tensor-core loops per type
    out["mma_bf16_single_tflops"] = out["mma_bf16_tflops"]
    out["mma_tf32_single_tflops"] = out["mma_tf32_tflops"]
    out["mma_bf16_tflops"] = max(out["mma_bf16_tflops"], out["mma_bf16_pattern_tflops"])
    out["mma_tf32_tflops"] = max(out["mma_tf32_tflops"], out["mma_tf32_pattern_tflops"])
    out["how"] = ("own loops (csrc/peaks.cu), one CTA per SM, one thread issuing back-to-back "
                  "tcgen05.mma, M=128: (a) N=256 on one operand pair into two accumulators in "
                  "turn, (b) the wide sweep's residual chunk (three A tiles, N=256 and "
                  "N=192/128/64 into staggered accumulators); mma_*_tflops = the higher of "
                  "(a) and (b) (K=16 bf16 / K=8 tf32); 8 x 256 threads per SM with 8 "
                  f"independent FMA chains each; CUDA events, median of {reps} launches "
                  "after a warm-up")
    return out


def cpu_baseline(E, seeds, budget_s=15.0):
    """The oracle's slice sweep on all host cores over a bounded sample of the
    workload's instances; returns instances/s and what was sampled."""
    import oracle
    from paper_1010_2627_gb300 import inputs
    ss = inputs.square(M, L)
    nthr = oracle.max_threads()
    # one instance per core at a time, up to 16 per core or ~budget seconds
    idx = np.linspace(0, len(E) - 1, 16 * nthr).astype(int)
    Es = E[idx]
    sd = np.asarray([seeds[i % len(seeds)] for i in range(len(idx))], np.uint64)
    Sig = np.stack([oracle.sigma_square(M, 1.0, e) for e in Es])
    done, t0 = 0, time.perf_counter()
    while done < len(Es):
        n = nthr
        sl = slice(done, done + n)
        oracle.rgf_batch(ss.H0, ss.V, L, Es[sl], sd[sl], np.full(n, W), Sig[sl], Sig[sl],
                         np.arange(n), nthreads=nthr)
        done += n
        if time.perf_counter() - t0 > budget_s:
            break
    dt = time.perf_counter() - t0
    return {"value": done / dt, "unit": "T(E) points/s", "cores": nthr, "kind": "oracle",
            "sample": f"{done} instances of the same workload (M={M}, L={L}, W={W}), "
                      f"energies spread over the grid, oracle slice sweep (FP64, own LU), "
                      f"OpenMP over instances, {dt:.1f} s",
            "slice_updates_per_s": done * L / dt}


def run_reference(args):
    ws, rank = _dist()
    if rank != 0:
        return
    from paper_1010_2627_gb300 import inputs
    E = inputs.energy_grid(-3.9, 3.9, NE)
    seeds = np.arange(NS, dtype=np.uint64)
    times, vals, step_ms = [], [], []
    for k in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        r = cpu_baseline(E, seeds, budget_s=8.0)
        if k >= args.warmup:
            step_ms.append(1e3 * (time.perf_counter() - t0))
            vals.append(r["value"])
            times.append(r)
    v = statistics.median(vals)
    # one step = one bounded sample of the workload's instances (measured);
    # the whole 8192-instance workload at this rate is only extrapolated
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "T(E) points/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": statistics.median(step_ms),
            "step": "a bounded sample of the workload (see cpu_baseline.sample), timed",
            "full_workload_ms_extrapolated": 1e3 * NE * NS / v,
            "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "instances": NE * NS, "flush": "n/a (CPU)"},
            "cpu_baseline": {"value": v, "unit": "T(E) points/s", "cores": times[-1]["cores"],
                             "kind": "oracle", "sample": times[-1]["sample"]},
            "e2e": {"value": v, "unit": "T(E) points/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_knit(args):
    import torch
    ws, rank = _dist()
    if ws > 1:
        import torch.distributed as dist
        local = int(os.environ.get("LOCAL_RANK", rank))
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    dev = torch.cuda.current_device()
    from paper_1010_2627_gb300 import build, inputs, knit
    build.build()
    knit.load()

    from paper_1010_2627_gb300 import shard
    nsm = torch.cuda.get_device_properties(dev).multi_processor_count
    pk = measure_peaks(knit, torch, torch.cuda.current_stream(), nsm)
    ss = inputs.square(M, L)
    # weak scaling: the global grid has NE energies per rank, rank r takes
    # every ws-th energy (its own 1024-energy shard of the same interval)
    E = inputs.energy_grid(-3.9, 3.9, NE * ws)[shard.interleave(NE * ws, ws, rank)]
    seeds = np.arange(NS, dtype=np.uint64)
    n = NE * NS
    sysk = knit.System(ss)
    stream = torch.cuda.Stream()
    dE = torch.tensor(E, device="cuda")
    ds = torch.tensor(seeds.astype(np.int64), device="cuda")
    dT = torch.empty(n, dtype=torch.float64, device="cuda")
    dst = torch.empty(n, dtype=torch.int32, device="cuda")
    flush = torch.empty(2 * L2_BYTES // 4, dtype=torch.float32, device="cuda")

    def step(precision=knit.KNIT_MIXED):
        knit.knit_transmission(sysk.handle, dE, ds, W, precision, dT, dst, nE=NE, nS=NS,
                               stream=stream)

    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            flush.fill_(1.0)
            step()
    torch.cuda.synchronize()
    assert (dst.cpu().numpy() == 0).all(), "instance status != 0 in warm-up"

    # ---- timed region: K steps, L2 flushed before each (outside its events)
    if ws > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    clocks = _clock_sampler()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    with torch.cuda.stream(stream):
        for k in range(args.steps):
            flush.fill_(float(k))
            ev[k][0].record(stream)
            step()
            ev[k][1].record(stream)
    torch.cuda.synchronize()
    step_ms = [a.elapsed_time(b) for a, b in ev]
    total_ms = sum(step_ms)
    if ws > 1:
        t = torch.tensor([total_ms], device="cuda")
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        total_ms = float(t.item())
    clk = _clock_summary(clocks, dev)
    T_mixed = dT.cpu().numpy().reshape(NE, NS).copy()
    st = dst.cpu().numpy()
    gathered = None
    if ws > 1:
        # every rank's T in the global (energy, seed) order, once, on the host
        def agather(obj):
            out = [None] * ws
            torch.distributed.all_gather_object(out, obj)
            return out
        rows = shard.interleave(NE * ws, ws, rank)
        idx = (rows[:, None] * NS + np.arange(NS)[None, :]).ravel()
        gathered = int(len(shard.gather(T_mixed.ravel(), idx, NE * ws * NS, agather)))
    ms_per_step = total_ms / args.steps
    value = ws * n / (ms_per_step / 1e3)

    peaks = _peaks()
    # ---- the sweep kernel alone (Sigma precomputed): average launch duration
    SL = torch.empty(NE * M * M * 2, dtype=torch.float64, device="cuda")
    knit.knit_lead_selfenergy(sysk.handle, 0, dE, SL, stream=stream)
    torch.cuda.synchronize()
    kev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in range(3)]
    with torch.cuda.stream(stream):
        for a, b in kev:
            flush.fill_(2.0)
            a.record(stream)
            knit.knit_transmission_sigma(sysk.handle, dE, ds, W, SL, SL, knit.KNIT_MIXED, dT, dst,
                                         nE=NE, nS=NS, stream=stream)
            b.record(stream)
    torch.cuda.synchronize()
    sweep_ms = statistics.mean(a.elapsed_time(b) for a, b in kev)
    alg_flop = 16.0 * M ** 3 * L * n          # 16 M^3 real flop per slice-update
    achieved_tflops = alg_flop / (sweep_ms / 1e3) / 1e12
    # executed tensor-core work per slice, in 128 x 64 x 16 MMA units: the
    # residual's 18 digit products x 8 K-chunks, the Gauss-Jordan's 9 term
    # products x 8 panels (M / 8 panels of 8 columns) and the refinement
    # product's 6 term products x 4 K-chunks at N = 128 (every slice but the
    # ~0.07 % that take the error-free CUDA-core product)
    tc_flop = (18 * 8 + 9 * (M // 8) + 6 * 4 * 2) * 2.0 * 128 * 64 * 16 * L * n
    tc_tflops = tc_flop / (sweep_ms / 1e3) / 1e12

    # ---- plain FP64 GPU sweep on a one-wave subset (same energies/seeds grid)
    nsub_e = 19                                # 19 energies x 8 seeds = 152 instances
    sub = np.linspace(0, NE - 1, nsub_e).astype(int)
    dEs = torch.tensor(E[sub], device="cuda")
    dTs = torch.empty(nsub_e * NS, dtype=torch.float64, device="cuda")
    dsts = torch.empty(nsub_e * NS, dtype=torch.int32, device="cuda")
    REPS = 5   # each side timed as the median of 5 launches after a warm-up

    def median_ms(precision, out):
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
               for _ in range(REPS)]
        with torch.cuda.stream(stream):
            knit.knit_transmission(sysk.handle, dEs, ds, W, precision, out, dsts, nE=nsub_e,
                                   nS=NS, stream=stream)   # warm-up (lead modes cached)
            for a, b in evs:
                a.record(stream)
                knit.knit_transmission(sysk.handle, dEs, ds, W, precision, out, dsts, nE=nsub_e,
                                       nS=NS, stream=stream)
                b.record(stream)
        torch.cuda.synchronize()
        return statistics.median(a.elapsed_time(b) for a, b in evs)

    fp64_ms = median_ms(knit.KNIT_FP64, dTs)
    fp64_rate = nsub_e * NS / (fp64_ms / 1e3)
    fp64_tflops = 16.0 * M ** 3 * L * nsub_e * NS / (fp64_ms / 1e3) / 1e12
    # the same subset through the CUDA-core residual path of the mixed sweep
    dTc = torch.empty(nsub_e * NS, dtype=torch.float64, device="cuda")
    cc_rate = nsub_e * NS / (median_ms(knit.KNIT_MIXED_CUDACORE, dTc) / 1e3)
    T64 = dTs.cpu().numpy().reshape(nsub_e, NS)
    ek = 2 * np.cos(np.arange(1, M + 1) * np.pi / (M + 1))
    nch = np.array([max(1, int(np.sum(np.abs(e - ek) < 2))) for e in E[sub]])
    mixed_vs_fp64 = float(np.max(np.abs(T_mixed[sub] - T64) / nch[:, None]))

    # ---- end to end through the public API with host buffers
    Eh = np.ascontiguousarray(E)
    Th = np.empty(n)
    sth = np.empty(n, np.int32)
    e2e_ms = []
    for k in range(max(2, min(args.steps, 3))):
        flush.fill_(3.0)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        knit.knit_transmission(sysk.handle, Eh, seeds, W, knit.KNIT_MIXED, Th, sth)
        e2e_ms.append((time.perf_counter() - t0) * 1e3)
    e2e_val = ws * n / (statistics.mean(e2e_ms) / 1e3)

    launches_per_step = 4     # modes self-energy, status combine, status fill, mixed sweep
    line = {
        "metric": METRIC, "value": value, "unit": "T(E) points/s", "n_gpus": ws,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_per_step,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "c64 inversion + bf16-digit tensor-core residual (f32 accumulate)", "data": "synthetic",
        "config": {"workload": WORKLOAD, "M": M, "L": L, "W": W, "energies": NE, "seeds": NS,
                   "instances_per_gpu": n, "precision": "mixed",
                   "flush": "L2 flushed before every timed step (252 MB write)"},
        "slice_updates_per_s": value * L,
        "fp64_sweep": {"value": fp64_rate, "unit": "T(E) points/s",
                       "sample": f"{nsub_e} energies x {NS} seeds, one wave, median of {REPS} "
                                 f"launches", "ms": fp64_ms,
                       "mixed_speedup": value / ws / fp64_rate,
                       "roofline": {"bound": "fp64", "achieved": fp64_tflops,
                                    "peak": pk["dfma_tflops"], "unit": "TFLOP/s",
                                    "frac": fp64_tflops / pk["dfma_tflops"],
                                    "note": "16 M^3 flop per slice-update over the measured "
                                            "DFMA peak (own loop, csrc/peaks.cu); includes "
                                            "the lead solve of the subset"},
                       "mixed_cudacore_residual_rate": cc_rate,
                       "max_abs_dT_mixed_vs_fp64_over_nch": mixed_vs_fp64},
        "roofline": {"bound": "tensor", "kernel": "knit_sweep_mixed_tc_kernel",
                     "achieved": achieved_tflops, "peak": pk["mma_tf32_tflops"],
                     "unit": "TFLOP/s", "frac": achieved_tflops / pk["mma_tf32_tflops"],
                     "traffic": SWEEP_TRAFFIC_BYTES,
                     "note": "algorithmic 16 M^3 flop per slice-update (the method's complex "
                             "inversion plus product) over the measured dense TF32 tensor peak "
                             "(own tcgen05 kind::tf32 loop, csrc/peaks.cu), the contraction "
                             "type of a complex64 sweep; kernel timed alone with CUDA events",
                     "kernel_ms": sweep_ms,
                     "fp32_alu": {"peak": pk["ffma_tflops"],
                                  "frac": achieved_tflops / pk["ffma_tflops"],
                                  "note": "the same rate over the measured FP32 FMA peak (the "
                                          "Gauss-Jordan pivot chain and the digit splitting "
                                          "run on the CUDA cores)"},
                     "tensor_pipe": {"executed_tflops": tc_tflops,
                                     "peak": pk["mma_bf16_tflops"],
                                     "frac": tc_tflops / pk["mma_bf16_tflops"],
                                     "note": "bf16 products per slice: the residual's 18 digit "
                                             "products x 8 K-chunks, the Gauss-Jordan panel "
                                             "updates' 9 term products x 8 panels and the "
                                             "refinement product's 6 term products x 4 K-chunks "
                                             "(N = 128), in units of a 128 x 64 x 16 MMA, over "
                                             "the measured bf16 MMA peak (own loop)"}},
        "peaks_measured": pk,
        "e2e": {"value": e2e_val, "unit": "T(E) points/s", "h2d_bytes_per_step": 8 * NE + 8 * NS,
                "d2h_bytes_per_step": 12 * n, "ms": statistics.mean(e2e_ms)},
        "gpu_launches": launches_per_step * args.steps,
        "clocks": clk,
        "peaks_file": {k: peaks.get(k) for k in ("hbm_gbs", "bf16_tflops", "sm_max_mhz")},
        "status_nonzero": int((st != 0).sum()),
    }
    if gathered is not None:
        line["results_gathered"] = gathered
    if rank == 0 and args.cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(E, seeds) if ws == 1 else None
    if rank == 0:
        print(json.dumps(line), flush=True)
    sysk.close()
    if ws > 1:
        torch.distributed.destroy_process_group()


def run_uneven(args):
    """Uneven batch: 4096 square-lattice instances, M in {32,48,64,96,128},
    L in {128,...,2048}, W ~ U[0,4], E ~ U(-3.9,3.9), seed = index, drawn from
    a sampler seeded 12345; one plan, mixed precision (widths 33..64 on the
    tensor-core kernel of sweep_mixed_tc.cu, 32 and below on the CUDA-core
    one, 65..128 on the tensor-core kernel of sweep_mixed_tc128.cu).  One step
    = lead self-energies + sweeps for all instances.  Beside it: the
    algorithmic rate over the measured TF32 peak, a stratified subset of 64
    instances (the shortest of each width) checked against the oracle, and
    the oracle's rate on that subset."""
    import torch
    from paper_1010_2627_gb300 import build, inputs, knit, shard
    ws, rank = _dist()
    if ws > 1:
        import torch.distributed as dist
        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", rank)))
        dist.init_process_group("nccl")
    build.build()
    knit.load()
    nsm = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    pk = measure_peaks(knit, torch, torch.cuda.current_stream(), nsm)
    inst_all = inputs.uneven_instances(4096)
    n_all = len(inst_all["M"])
    # several GPUs: the fixed batch split by cost M^3 L, longest first
    # (strong scaling), each rank one plan over its share
    owner = shard.lpt(inst_all["M"].astype(np.float64) ** 3 * inst_all["L"], ws)
    mine = np.flatnonzero(owner == rank)
    inst = {k: v[mine] for k, v in inst_all.items()}
    keys = sorted(set(zip(inst["M"].tolist(), inst["L"].tolist())))
    systems = [knit.System(inputs.square(m, l)) for m, l in keys]
    sys_index = np.array([keys.index((m, l)) for m, l in zip(inst["M"], inst["L"])], np.int32)
    batch = knit.Batch(systems, sys_index, precision=knit.KNIT_MIXED)
    n = len(sys_index)
    stream = torch.cuda.Stream()
    dE = torch.tensor(inst["E"], device="cuda")
    ds = torch.tensor(inst["seeds"].astype(np.int64), device="cuda")
    dW = torch.tensor(inst["W"], device="cuda")
    dT = torch.empty(n, dtype=torch.float64, device="cuda")
    dst = torch.empty(n, dtype=torch.int32, device="cuda")
    flush = torch.empty(2 * L2_BYTES // 4, dtype=torch.float32, device="cuda")
    # CTAs per SM per kernel variant: own CUDA-event timings, cached as JSON
    cache = os.path.join(os.path.dirname(os.path.abspath(__file__)), "paper_1010_2627_gb300",
                         "_build", "autotune_uneven.json")
    t0 = time.perf_counter()
    tuned = batch.autotune(inst["E"], inst["seeds"], inst["W"], cache=cache)
    tune_s = time.perf_counter() - t0

    def step():
        knit.knit_batch_transmission(batch.handle, dE, ds, dW, dT, dst, stream=stream)

    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            flush.fill_(1.0)
            step()
    torch.cuda.synchronize()
    if ws > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    clocks = _clock_sampler()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    with torch.cuda.stream(stream):
        for k in range(args.steps):
            flush.fill_(float(k))
            ev[k][0].record(stream)
            step()
            ev[k][1].record(stream)
    torch.cuda.synchronize()
    ms = statistics.mean(a.elapsed_time(b) for a, b in ev)
    if ws > 1:
        t = torch.tensor([ms], device="cuda")
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        ms = float(t.item())
    clk = _clock_summary(clocks, torch.cuda.current_device())
    T_mine = dT.cpu().numpy()
    st_mine = dst.cpu().numpy()
    if ws > 1:
        # every rank's results in the caller's instance order, once, on the host
        def agather(obj):
            out = [None] * ws
            torch.distributed.all_gather_object(out, obj)
            return out
        T = shard.gather(T_mine, mine, n_all, agather)
        st = shard.gather(st_mine, mine, n_all, agather)
    else:
        T, st = T_mine, st_mine
    inst, n = inst_all, n_all
    # the same step captured once in a CUDA graph and replayed (the plan only
    # enqueues kernels once its buffers exist)
    graph = {}
    try:
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=stream):
            step()
        gev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
               for _ in range(args.steps)]
        with torch.cuda.stream(stream):
            for k in range(args.steps):
                flush.fill_(float(k))
                gev[k][0].record(stream)
                g.replay()
                gev[k][1].record(stream)
        torch.cuda.synchronize()
        gms = statistics.mean(a.elapsed_time(b) for a, b in gev)
        graph = {"ms_per_step": gms, "value": n / (gms / 1e3),
                 "same_T": bool(np.array_equal(dT.cpu().numpy(), T_mine))}
    except Exception as exc:   # capture refused: report, keep the stream numbers
        graph = {"error": str(exc)[:200]}
    slices = int(inst["L"].sum())
    flop = float((16.0 * inst["M"].astype(np.float64) ** 3 * inst["L"]).sum())
    achieved = flop / (ms / 1e3) / 1e12
    Ms = inst["M"]
    line = {
        "metric": "T(E) points/s (uneven batch)", "value": n / (ms / 1e3),
        "unit": "T(E) points/s", "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms, "higher_is_better": True, "scaling": "strong", "vs_baseline": None,
        "dtype": "c64 inversion + bf16-digit tensor-core residual (f32 accumulate)",
        "data": "synthetic",
        "config": {"workload": "uneven square batch, 4096 instances, M in {32..128}, "
                               "L in {128..2048}, W ~ U[0,4]", "systems": len(keys),
                   "instances_by_kernel": {"mixed CUDA-core, M <= 32": int((Ms <= 32).sum()),
                                           "mixed tensor-core, 33 <= M <= 64":
                                               int(((Ms > 32) & (Ms <= 64)).sum()),
                                           "mixed tensor-core, 65 <= M <= 128": int((Ms > 64).sum())},
                   "flush": "L2 flushed before every timed step"},
        "slice_updates_per_s": slices / (ms / 1e3),
        "roofline": {"bound": "tensor", "achieved": achieved, "peak": pk["mma_tf32_tflops"],
                     "unit": "TFLOP/s", "frac": achieved / pk["mma_tf32_tflops"], "traffic": None,
                     "note": "sum of 16 M^3 L over the batch / step time (leads included) over "
                             "the measured dense TF32 tensor peak (own loop)"},
        "clocks": clk, "peaks_measured": pk,
        "kernel_variants": [{"kind": k, "Mmax": m, "instances": c, "max_ctas_per_sm": x,
                             "ctas_per_sm": tuned[q]} for q, (k, m, c, x) in enumerate(batch.buckets())],
        "autotune_s": tune_s, "cuda_graph": graph,
        "status_nonzero": int((st != 0).sum())}
    if ws > 1:
        line["sharding"] = "LPT by M^3 L over ranks, results gathered to rank 0"
    if rank != 0:
        batch.close()
        torch.distributed.destroy_process_group()
        return
    # stratified subset: the 13 (12 for the last width) shortest instances of each width
    import oracle
    sub = []
    for m in sorted(set(Ms.tolist())):
        ids = np.flatnonzero(Ms == m)
        sub += ids[np.argsort(inst["L"][ids], kind="stable")][:13].tolist()
    sub = np.array(sub[:64])
    nthr = oracle.max_threads()
    worst, t0, n_or, sl_or = 0.0, time.perf_counter(), 0, 0
    for m in sorted(set(Ms[sub].tolist())):
        for l in sorted(set(inst["L"][sub][Ms[sub] == m].tolist())):
            ids = sub[(Ms[sub] == m) & (inst["L"][sub] == l)]
            ss = inputs.square(m, l)
            Sg = np.stack([oracle.sigma_square(m, 1.0, e) for e in inst["E"][ids]])
            To, sto = oracle.rgf_batch(ss.H0, ss.V, l, inst["E"][ids], inst["seeds"][ids],
                                       inst["W"][ids], Sg, Sg, np.arange(len(ids)), nthreads=nthr)
            ek = 2 * np.cos(np.arange(1, m + 1) * np.pi / (m + 1))
            for q, i in enumerate(ids):
                nch = max(1, int(np.sum(np.abs(inst["E"][i] - ek) < 2)))
                worst = max(worst, abs(T[i] - To[q]) / nch)
            n_or += len(ids)
            sl_or += len(ids) * l
    dt = time.perf_counter() - t0
    line["oracle_subset"] = {"instances": int(n_or), "max_abs_dT_over_nch": worst,
                             "tolerance": 1e-6, "pass": bool(worst <= 1e-6)}
    if args.cpu_baseline:
        line["cpu_baseline"] = {"value": n_or / dt, "unit": "T(E) points/s", "cores": nthr,
                                "kind": "oracle", "slice_updates_per_s": sl_or / dt,
                                "sample": f"the {n_or}-instance stratified subset (shortest of "
                                          f"each width), oracle slice sweep (FP64, own LU), "
                                          f"OpenMP over instances, {dt:.1f} s"}
    print(json.dumps(line), flush=True)
    batch.close()
    if ws > 1:
        torch.distributed.destroy_process_group()


def run_profile_case(args):
    """Small case for ncu captures: square lattice of width --profile-M
    (default 64), L = --profile-L (default 64), W = 2, 19 energies x 8 seeds
    (one wave of 152 instances), two mixed sweeps and one FP64 sweep (FP64
    skipped above width 64, where it takes seconds).  --profile-lattice
    armchair: the graphene ribbon of the same row width and length instead
    (t = 2.7, W = 1, 19 energies in (-2, 2)), above width 128 run by
    half-rows; --profile-lattice bdg: the spinful BdG bar of --profile-M / 4
    sites (mu = -1, Delta = 0.1, alpha = 0.2, W = 1, 19 energies in
    (-0.2, 0.2), normal leads)."""
    import torch
    from paper_1010_2627_gb300 import build, inputs, knit
    build.build()
    knit.load()
    Lp, Mp = args.profile_L, args.profile_M
    honeycomb = args.profile_lattice == "armchair"
    nambu = args.profile_lattice == "bdg"
    if honeycomb:
        ss, E, Wp = inputs.armchair(Mp, Lp), inputs.energy_grid(-2.0, 2.0, 19), 1.0
    elif nambu:
        ss = inputs.bdg(Mp // 4, Lp, mu=-1.0, delta=0.1, alpha=0.2)
        E, Wp = inputs.energy_grid(-0.2, 0.2, 19), 1.0
    else:
        ss, E, Wp = inputs.square(Mp, Lp), inputs.energy_grid(-3.9, 3.9, 19), W
    seeds = np.arange(NS, dtype=np.uint64)
    sysk = knit.System(ss)
    runs = (knit.KNIT_MIXED, knit.KNIT_MIXED) + ((knit.KNIT_FP64,) if Mp <= 64 else ())
    for precision in runs:
        T, st = sysk.transmission(E, seeds, W=Wp, precision=precision)
        if (st != 0).any():
            bad = np.argwhere(st != 0)
            print(json.dumps({"case": "profile", "status": {int(c): int((st == c).sum()) for c in np.unique(st)
                                                            if c != 0},
                              "energies": sorted({float(E[e]) for e, _ in bad})}), flush=True)
        assert honeycomb or nambu or (st == 0).all()
    torch.cuda.synchronize()
    print(json.dumps({"case": "profile", "M": Mp, "L": Lp, "instances": 19 * NS,
                      "T_mean": float(T.mean())}))
    sysk.close()


def run_ldos_case(args):
    """LDOS through the sewing pass, mixed vs FP64: square M=64, L=512, W=2,
    38 energies x 8 seeds (two waves of 152 instances), saving_level 8 (one
    checkpoint every 8 slices, the slices between recomputed).  One step = the
    whole LDOS call for all instances; reports LDOS points/s (instances/s) and
    the largest difference between the two precisions."""
    import torch
    from paper_1010_2627_gb300 import build, inputs, knit
    build.build()
    knit.load()
    ss = inputs.square(M, L)
    ne, save = 38, 8
    E = inputs.energy_grid(-3.9, 3.9, ne)
    seeds = np.arange(NS, dtype=np.uint64)
    n = ne * NS
    sysk = knit.System(ss)
    stream = torch.cuda.Stream()
    dE = torch.tensor(E, device="cuda")
    ds = torch.tensor(seeds.astype(np.int64), device="cuda")
    out = {}
    for name, prec in (("mixed", knit.KNIT_MIXED), ("fp64", knit.KNIT_FP64)):
        dL = torch.empty(n * L * M, dtype=torch.float64, device="cuda")
        dst = torch.empty(n, dtype=torch.int32, device="cuda")

        def step():
            knit.knit_ldos(sysk.handle, dE, ds, W, save, dL, None, dst, nE=ne, nS=NS,
                           stream=stream, precision=prec)

        with torch.cuda.stream(stream):
            for _ in range(max(1, args.warmup)):
                step()
        torch.cuda.synchronize()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
              for _ in range(args.steps)]
        with torch.cuda.stream(stream):
            for k in range(args.steps):
                ev[k][0].record(stream)
                step()
                ev[k][1].record(stream)
        torch.cuda.synchronize()
        ms = statistics.mean(a.elapsed_time(b) for a, b in ev)
        out[name] = (n / (ms / 1e3), ms, dL.cpu().numpy(), int((dst != 0).sum().item()))
    diff = float(np.abs(out["mixed"][2] - out["fp64"][2]).max() / np.abs(out["fp64"][2]).max())
    print(json.dumps({
        "metric": "LDOS points/s (sewing pass, mixed vs FP64)", "value": out["mixed"][0],
        "unit": "LDOS points/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": out["mixed"][1], "higher_is_better": True, "dtype": "c64 forward + "
        "double-float sewing", "data": "synthetic",
        "config": {"workload": f"square M={M} L={L} W={W}, {ne} energies x {NS} seeds, "
                               f"saving_level {save}"},
        "fp64": {"value": out["fp64"][0], "ms": out["fp64"][1]},
        "mixed_speedup": out["mixed"][0] / out["fp64"][0],
        "max_abs_dldos_over_max_ldos": diff,
        "status_nonzero": out["mixed"][3] + out["fp64"][3]}), flush=True)
    sysk.close()


def run_bdg_case(args):
    """Spinful BdG bar: 32 sites x 4 (spin x Nambu) = 128 orbitals per slice,
    L = 2048, mu = -1, t = 1, Delta = 0.1 in the system, Rashba alpha = 0.2,
    normal leads, W = 1 seed 0, 2048 midpoint energies in (-0.2, 0.2).  One
    step = lead self-energies (FP64 decimation of the leads' electron sector
    in its two mode blocks, the hole sector its particle-hole image) + mixed
    sweep (tensor-core kernel, 4 x 4 block couplings) for all energies.  Beside it: the lead solve and the sweep timed apart (the
    sweep's roofline over the measured TF32 peak), the FP64 sweep on 16
    energies, particle-hole symmetry of the total transmission T(E) = T(-E)
    for one disorder realisation, and the oracle on a bounded sample."""
    import torch
    from paper_1010_2627_gb300 import build, inputs, knit
    build.build()
    knit.load()
    nsm = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    pk = measure_peaks(knit, torch, torch.cuda.current_stream(), nsm)
    ne, Lb, Mb = args.bdg_energies, 2048, 128
    b = inputs.bdg(32, Lb, mu=-1.0, t=1.0, delta=0.1, alpha=0.2)
    E = inputs.energy_grid(-0.2, 0.2, ne)
    seeds = np.array([0], np.uint64)
    sysk = knit.System(b)
    T, st = sysk.transmission(E[:8], seeds, W=1.0, precision=knit.KNIT_MIXED)   # warm-up
    clocks = _clock_sampler()
    times = []
    for _ in range(args.steps):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        T, st = sysk.transmission(E, seeds, W=1.0, precision=knit.KNIT_MIXED)
        times.append(time.perf_counter() - t0)
    sec = statistics.mean(times)
    # the two parts apart: lead self-energies, then the sweep with them given
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    SL = sysk.lead_selfenergy(0, E, method=knit.KNIT_LEAD_DECIMATION)[0]
    SR = sysk.lead_selfenergy(1, E, method=knit.KNIT_LEAD_DECIMATION)[0]
    lead_sec = time.perf_counter() - t0
    dE = torch.tensor(E, device="cuda")
    dS = torch.tensor(seeds.astype(np.int64), device="cuda")
    dSL = torch.tensor(np.ascontiguousarray(SL).view(np.float64), device="cuda")
    dSR = torch.tensor(np.ascontiguousarray(SR).view(np.float64), device="cuda")
    dT = torch.empty(ne, dtype=torch.float64, device="cuda")
    dst = torch.empty(ne, dtype=torch.int32, device="cuda")
    a, bb = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    knit.knit_transmission_sigma(sysk.handle, dE, dS, 1.0, dSL, dSR, knit.KNIT_MIXED, dT, dst,
                                 nE=ne, nS=1)
    bb.record()
    torch.cuda.synchronize()
    sweep_ms = a.elapsed_time(bb)
    clk = _clock_summary(clocks, torch.cuda.current_device())
    achieved = 16.0 * Mb ** 3 * Lb * ne / (sweep_ms / 1e3) / 1e12
    sub = np.linspace(0, ne - 1, 16).astype(int)
    t0 = time.perf_counter()
    Tf, stf = sysk.transmission(E[sub], seeds, W=1.0, precision=knit.KNIT_FP64)
    fsec = time.perf_counter() - t0
    both = (st[:, 0] == 0) & (st[::-1, 0] == 0)   # energies mirror pairwise on this grid
    ph = float(np.abs(T[both, 0] - T[::-1, 0][both]).max())
    line = {
        "metric": "T(E) points/s (BdG mixed sweep incl. leads)", "value": ne / sec,
        "unit": "T(E) points/s", "n_gpus": 1, "steps": args.steps, "warmup": 1,
        "ms_per_step": 1e3 * sec, "higher_is_better": True,
        "dtype": "c64 inversion + bf16-digit tensor-core residual and products (f32 accumulate)",
        "data": "synthetic",
        "config": {"workload": f"BdG 32 sites x 4, L={Lb}, mu=-1, Delta=0.1, alpha=0.2, W=1 "
                               f"seed 0, {ne} energies in (-0.2, 0.2), normal leads"},
        "slice_updates_per_s": ne * Lb / sec,
        "lead_selfenergies_s": lead_sec, "sweep_s": sweep_ms / 1e3,
        "lead_blocks": sysk.info()[1],
        "roofline": {"bound": "tensor", "kernel": "knit_sweep_mixed_tc128_kernel",
                     "achieved": achieved, "peak": pk["mma_tf32_tflops"], "unit": "TFLOP/s",
                     "frac": achieved / pk["mma_tf32_tflops"], "traffic": None,
                     "note": "16 M^3 flop per slice-update over the sweep alone (Sigma given), "
                             "over the measured dense TF32 tensor peak (own loop)"},
        "fp64_sweep": {"value": len(sub) / fsec, "energies": len(sub), "seconds": fsec},
        "max_abs_dT_mixed_vs_fp64_over_nch": float(
            np.abs(T[sub, 0] - Tf[:, 0]).max() / max(1.0, float(np.abs(Tf).max()))),
        "particle_hole_max_abs_T_minus_T_mirror": ph,
        "particle_hole_pairs": int(both.sum()) // 2,
        "clocks": clk, "peaks_measured": pk,
        "status_nonzero": int((st != 0).sum() + (stf != 0).sum()),
        "status_mixed": {int(c): int((st == c).sum()) for c in np.unique(st) if c != 0},
        "status_fp64": {int(c): int((stf == c).sum()) for c in np.unique(stf) if c != 0},
        "energies_status_nonzero": [float(E[k]) for k in np.nonzero(st[:, 0] != 0)[0][:8]]}
    if args.cpu_baseline:
        # the oracle's slice sweep (FP64, own LU) on all host cores, with the
        # GPU's lead self-energies, on 16 energies of a 256-slice copy of the bar
        import oracle
        Ls = 256
        nthr = oracle.max_threads()
        idx = np.linspace(0, ne - 1, 16).astype(int)
        t0 = time.perf_counter()
        To, sto = oracle.rgf_batch(b.H0, b.V, Ls, E[idx], np.zeros(16, np.uint64), np.ones(16),
                                   SL[idx], SR[idx], np.arange(16), block=4, sign=b.sign,
                                   nthreads=nthr)
        dt = time.perf_counter() - t0
        line["cpu_baseline"] = {"value": 16 * Ls / dt, "unit": "slice-updates/s", "cores": nthr,
                                "kind": "oracle",
                                "sample": f"16 energies of a {Ls}-slice copy of the bar, "
                                          f"oracle slice sweep (FP64), OpenMP, {dt:.1f} s; the "
                                          f"GPU runs {ne * Lb / sec:.0f} slice-updates/s incl. leads"}
    print(json.dumps(line), flush=True)
    sysk.close()


def run_graphene_case(args):
    """Graphene armchair ribbon: honeycomb lattice t = 2.7 as a brick wall of
    256 sites per row, L = 1024 rows, on-site disorder uniform in [-0.5, 0.5]
    (W = 1, seed 0), 8192 midpoint energies in (-2, 2), clean ribbon leads
    (period 2).  One step = both lead self-energies (the leads' two-slice
    supercells decimated block by block in the basis of transverse modes) +
    the KNIT_MIXED sweep, which the library runs on the half-row chain (128
    orbitals, 2048 slices, tensor-core kernel), host E in, host T out.
    Beside it: leads and sweep timed apart on the device (the sweep's roofline
    over the measured TF32 peak), the FP64 row sweep on 16 energies, the
    oracle on an 8-row copy, and the oracle's speed on a bounded sample."""
    import torch
    import oracle
    from paper_1010_2627_gb300 import build, inputs, knit
    build.build()
    knit.load()
    nsm = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    pk = measure_peaks(knit, torch, torch.cuda.current_stream(), nsm)
    ne, Lg, Mg, Wg = args.graphene_energies, args.graphene_L, 256, 1.0
    ss = inputs.armchair(Mg, Lg)
    E = inputs.energy_grid(-2.0, 2.0, ne)
    seeds = np.array([0], np.uint64)
    t0 = time.perf_counter()
    sysk = knit.System(ss)
    create_s = time.perf_counter() - t0
    kind, blocks = sysk.info(knit.KNIT_MIXED)
    T, st = sysk.transmission(E[:8], seeds, W=Wg, precision=knit.KNIT_MIXED)   # warm-up
    clocks = _clock_sampler()
    times = []
    for _ in range(args.steps):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        T, st = sysk.transmission(E, seeds, W=Wg, precision=knit.KNIT_MIXED)
        times.append(time.perf_counter() - t0)
    sec = statistics.mean(times)
    # the two parts apart, on the device: lead self-energies, then the sweep
    MM = Mg * Mg
    dE = torch.tensor(E, device="cuda")
    dS = torch.tensor(seeds.astype(np.int64), device="cuda")
    dSL = torch.empty(2 * MM * ne, dtype=torch.float64, device="cuda")
    dSR = torch.empty(2 * MM * ne, dtype=torch.float64, device="cuda")
    dT = torch.empty(ne, dtype=torch.float64, device="cuda")
    dst = torch.empty(ne, dtype=torch.int32, device="cuda")
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
    ev[0].record()
    knit.knit_lead_selfenergy(sysk.handle, 0, dE, dSL)
    knit.knit_lead_selfenergy(sysk.handle, 1, dE, dSR)
    ev[1].record()
    knit.knit_transmission_sigma(sysk.handle, dE, dS, Wg, dSL, dSR, knit.KNIT_MIXED, dT, dst,
                                 nE=ne, nS=1)
    ev[2].record()
    torch.cuda.synchronize()
    lead_ms, sweep_ms = ev[0].elapsed_time(ev[1]), ev[1].elapsed_time(ev[2])
    clk = _clock_summary(clocks, torch.cuda.current_device())
    # the learned warm start for both leads (20 000 decimation samples each,
    # the library's own training kernels), then the leads' self-energies
    # through it (Newton per mode block, decimation where it does not settle)
    learned = {}
    try:
        t0 = time.perf_counter()
        rng = np.random.default_rng(20)
        models = tuple(knit.LeadModel(sysk, p, rng.uniform(-2.0, 2.0, 20000), epochs=60, batch=256,
                                      lr=1e-3, seed=p + 1) for p in (0, 1))
        train_s = time.perf_counter() - t0
        opts = knit._opts(knit.KNIT_LEAD_LEARNED, models=(models[0].handle, models[1].handle))
        dSLl = torch.empty_like(dSL)
        dSRl = torch.empty_like(dSR)
        knit.knit_lead_selfenergy(sysk.handle, 0, dE, dSLl, opts)   # warm-up
        ev[0].record()
        knit.knit_lead_selfenergy(sysk.handle, 0, dE, dSLl, opts)
        knit.knit_lead_selfenergy(sysk.handle, 1, dE, dSRl, opts)
        ev[1].record()
        torch.cuda.synchronize()
        lead_l_ms = ev[0].elapsed_time(ev[1])
        dmax = max(float((dSLl - dSL).abs().max()), float((dSRl - dSR).abs().max()))
        learned = {"training_s": train_s, "samples_per_lead": 20000, "epochs": 60,
                   "lead_selfenergies_s": lead_l_ms / 1e3,
                   "decimation_lead_selfenergies_s": lead_ms / 1e3,
                   "max_abs_dSigma_vs_decimation": dmax}
        for m in models:
            m.close()
    except Exception as exc:
        learned = {"error": str(exc)[:200]}
    Th = Mg // 2
    achieved = 16.0 * Th ** 3 * (2 * Lg) * ne / (sweep_ms / 1e3) / 1e12
    sub = np.linspace(0, ne - 1, 16).astype(int)
    t0 = time.perf_counter()
    Tf, stf = sysk.transmission(E[sub], seeds, W=Wg, precision=knit.KNIT_FP64)
    fsec = time.perf_counter() - t0
    sysk.close()
    # the oracle's row sweep on an 8-row copy with the GPU's lead self-energies
    Lo, Eo = 8, E[np.linspace(0, ne - 1, 4).astype(int)]
    so = inputs.armchair(Mg, Lo)
    ko = knit.System(so)
    oSL, oSR = ko.lead_selfenergy(0, Eo)[0], ko.lead_selfenergy(1, Eo)[0]
    To_gpu, sto_gpu = ko.transmission(Eo, seeds, W=Wg, precision=knit.KNIT_MIXED)
    ko.close()
    nthr = oracle.max_threads()
    To, sto = oracle.rgf_batch(so.H0, so.V, Lo, Eo, np.zeros(len(Eo), np.uint64),
                               np.full(len(Eo), Wg), oSL, oSR, np.arange(len(Eo)), nthreads=nthr)
    line = {
        "metric": "T(E) points/s (graphene mixed sweep incl. leads)", "value": ne / sec,
        "unit": "T(E) points/s", "n_gpus": 1, "steps": args.steps, "warmup": 1,
        "ms_per_step": 1e3 * sec, "higher_is_better": True,
        "dtype": "c64 inversion + bf16-digit tensor-core residual and products (f32 accumulate)",
        "data": "synthetic",
        "config": {"workload": f"graphene armchair ribbon t=2.7, {Mg} sites per row, L={Lg} rows, "
                               f"W=1 (uniform [-0.5, 0.5]) seed 0, {ne} energies in (-2, 2), "
                               f"clean ribbon leads"},
        "sweep_kernel": {knit.KNIT_SWEEP_MIXED_HALF_ROWS: "half-row chain on the tensor-core "
                         "kernel (128 orbitals, 2L slices)"}.get(kind, kind),
        "lead_blocks": blocks, "system_create_s": create_s,
        "row_slice_updates_per_s": ne * Lg / sec,
        "lead_selfenergies_s": lead_ms / 1e3, "sweep_s": sweep_ms / 1e3,
        "roofline": {"bound": "tensor", "kernel": "knit_sweep_mixed_tc128_kernel",
                     "achieved": achieved, "peak": pk["mma_tf32_tflops"], "unit": "TFLOP/s",
                     "frac": achieved / pk["mma_tf32_tflops"], "traffic": None,
                     "note": "16 M^3 flop per half-row slice-update (M = 128, 2L slices) over "
                             "the sweep alone (Sigma given), over the measured dense TF32 "
                             "tensor peak (own loop)"},
        "learned_leads": learned,
        "fp64_row_sweep": {"value": len(sub) / fsec, "energies": len(sub), "seconds": fsec},
        "max_abs_dT_mixed_vs_fp64": float(np.abs(T[sub, 0] - Tf[:, 0]).max()),
        "oracle_subset": {"rows": Lo, "energies": len(Eo),
                          "max_abs_dT": float(np.abs(To_gpu[:, 0] - To).max()),
                          "status_nonzero": int((sto != 0).sum() + (sto_gpu != 0).sum())},
        "clocks": clk, "peaks_measured": pk,
        "status_nonzero": int((st != 0).sum() + (stf != 0).sum()),
        "status_mixed": {int(c): int((st == c).sum()) for c in np.unique(st) if c != 0}}
    if args.cpu_baseline:
        # the oracle's row sweep (FP64, own LU) on all host cores, 16 energies
        # of a 16-row copy with the GPU's lead self-energies
        Lc = 16
        sc_ = inputs.armchair(Mg, Lc)
        t0 = time.perf_counter()
        oracle.rgf_batch(sc_.H0, sc_.V, Lc, np.repeat(Eo, 4), np.zeros(16, np.uint64),
                         np.full(16, Wg), oSL, oSR, np.repeat(np.arange(4), 4), nthreads=nthr)
        dt = time.perf_counter() - t0
        line["cpu_baseline"] = {"value": 16 * Lc / dt, "unit": "row slice-updates/s",
                                "cores": nthr, "kind": "oracle",
                                "sample": f"16 instances of a {Lc}-row copy of the ribbon, oracle "
                                          f"row sweep (FP64), OpenMP, {dt:.1f} s; the GPU runs "
                                          f"{ne * Lg / sec:.0f} row slice-updates/s incl. leads"}
    print(json.dumps(line), flush=True)


def run_eigen_case(args):
    """Transmission eigenvalues and shot noise on the bench workload (square
    M=64, L=512, W=2, 1024 energies x 8 seeds, mixed sweep): one step = lead
    self-energies, the sweep with G_LL stored, Gamma_R^{1/2} per energy, the
    Hermitian matrix per instance and its FP64 Jacobi eigenvalues, for all
    8192 instances, outputs in device memory.  Beside it: the same call for
    T alone, so the eigenvalue pipeline's own cost reads as the difference."""
    import torch
    from paper_1010_2627_gb300 import build, inputs, knit
    build.build()
    knit.load()
    ss = inputs.square(M, L)
    E = inputs.energy_grid(-3.9, 3.9, NE)
    seeds = np.arange(NS, dtype=np.uint64)
    n = NE * NS
    sysk = knit.System(ss)
    stream = torch.cuda.Stream()
    dE = torch.tensor(E, device="cuda")
    ds = torch.tensor(seeds.astype(np.int64), device="cuda")
    dtau = torch.empty(n * M, dtype=torch.float64, device="cuda")
    dnoise = torch.empty(n, dtype=torch.float64, device="cuda")
    dT = torch.empty(n, dtype=torch.float64, device="cuda")
    dst = torch.empty(n, dtype=torch.int32, device="cuda")

    def eig_step():
        knit.knit_transmission_eigenvalues(sysk.handle, dE, ds, W, knit.KNIT_MIXED, dtau, dnoise,
                                           dT, dst, nE=NE, nS=NS, stream=stream)

    def t_step():
        knit.knit_transmission(sysk.handle, dE, ds, W, knit.KNIT_MIXED, dT, dst, nE=NE, nS=NS,
                               stream=stream)

    res = {}
    for name, fn in (("eig", eig_step), ("T", t_step)):
        with torch.cuda.stream(stream):
            for _ in range(max(1, args.warmup)):
                fn()
        torch.cuda.synchronize()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
              for _ in range(args.steps)]
        with torch.cuda.stream(stream):
            for k in range(args.steps):
                ev[k][0].record(stream)
                fn()
                ev[k][1].record(stream)
        torch.cuda.synchronize()
        res[name] = statistics.mean(a.elapsed_time(b) for a, b in ev)
    eig_step()
    torch.cuda.synchronize()
    tau = dtau.cpu().numpy().reshape(n, M)
    noise = dnoise.cpu().numpy()
    T = dT.cpu().numpy()
    st = dst.cpu().numpy()
    ok = (st == 0) & (T > 0.5)
    print(json.dumps({
        "metric": "T(E) points/s with transmission eigenvalues and shot noise (mixed sweep)",
        "value": n / (res["eig"] / 1e3), "unit": "T(E) points/s", "n_gpus": 1,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": res["eig"],
        "higher_is_better": True, "dtype": "c64 sweep + FP64 eigenvalues", "data": "synthetic",
        "config": {"workload": f"square M={M} L={L} W={W}, {NE} energies x {NS} seeds, "
                               "eigenvalues of every instance"},
        "T_only_ms_per_step": res["T"],
        "eigenvalue_pipeline_ms": res["eig"] - res["T"],
        "max_abs_sum_tau_minus_T": float(np.abs(tau.sum(axis=1) - T)[st == 0].max()),
        "tau_range": [float(tau[st == 0].min()), float(tau[st == 0].max())],
        "mean_fano_T_gt_half": float(np.mean(noise[ok] / T[ok])) if ok.any() else None,
        "status_nonzero": int((st != 0).sum())}), flush=True)
    sysk.close()


def run_lesser_case(args):
    """Lead-resolved lesser function (FP64 sewing pass with the column towards
    the right lead): square M=64, L=512, W=2, 38 energies x 8 seeds (two
    waves of 152 instances), saving_level 8.  One step = the whole call for
    all instances: densities injected by each lead and left-injected bond
    currents for every slice.  Beside it: the FP64 LDOS call on the same
    instances, and the largest violation of current conservation
    (sum_x jx[n][x] = T for every slice interface)."""
    import torch
    from paper_1010_2627_gb300 import build, inputs, knit
    build.build()
    knit.load()
    ss = inputs.square(M, L)
    ne, save = 38, 8
    E = inputs.energy_grid(-3.9, 3.9, ne)
    seeds = np.arange(NS, dtype=np.uint64)
    n = ne * NS
    sysk = knit.System(ss)
    nedge = knit.knit_system_num_edges(sysk.handle)
    stream = torch.cuda.Stream()
    dE = torch.tensor(E, device="cuda")
    ds = torch.tensor(seeds.astype(np.int64), device="cuda")
    rl = torch.empty(n * L * M, dtype=torch.float64, device="cuda")
    rr = torch.empty(n * L * M, dtype=torch.float64, device="cuda")
    jx = torch.empty(n * (L - 1) * M, dtype=torch.float64, device="cuda")
    jt = torch.empty(n * L * nedge, dtype=torch.float64, device="cuda")
    dT = torch.empty(n, dtype=torch.float64, device="cuda")
    dst = torch.empty(n, dtype=torch.int32, device="cuda")
    dL = torch.empty(n * L * M, dtype=torch.float64, device="cuda")

    def lesser_step():
        knit.knit_lesser(sysk.handle, dE, ds, W, save, rl, rr, jx, jt, dT, dst, nE=ne, nS=NS,
                         stream=stream)

    def ldos_step():
        knit.knit_ldos(sysk.handle, dE, ds, W, save, dL, None, None, nE=ne, nS=NS,
                       stream=stream, precision=knit.KNIT_FP64)

    res = {}
    for name, fn in (("lesser", lesser_step), ("ldos", ldos_step)):
        with torch.cuda.stream(stream):
            for _ in range(max(1, args.warmup)):
                fn()
        torch.cuda.synchronize()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
              for _ in range(args.steps)]
        with torch.cuda.stream(stream):
            for k in range(args.steps):
                ev[k][0].record(stream)
                fn()
                ev[k][1].record(stream)
        torch.cuda.synchronize()
        res[name] = statistics.mean(a.elapsed_time(b) for a, b in ev)
    lesser_step()
    torch.cuda.synchronize()
    T = dT.cpu().numpy()
    st = dst.cpu().numpy()
    cons = np.abs(jx.cpu().numpy().reshape(n, L - 1, M).sum(axis=2) - T[:, None])
    sumrule = np.abs((rl + rr - dL).cpu().numpy()).max()
    print(json.dumps({
        "metric": "lesser-function points/s (injected densities + bond currents, FP64)",
        "value": n / (res["lesser"] / 1e3), "unit": "instances/s", "n_gpus": 1,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": res["lesser"],
        "higher_is_better": True, "dtype": "f64", "data": "synthetic",
        "config": {"workload": f"square M={M} L={L} W={W}, {ne} energies x {NS} seeds, "
                               f"saving_level {save}"},
        "fp64_ldos_ms_per_step": res["ldos"],
        "max_abs_current_conservation": float(cons[st == 0].max()),
        "max_abs_rhoL_plus_rhoR_minus_ldos": float(sumrule),
        "status_nonzero": int((st != 0).sum())}), flush=True)
    sysk.close()


def hall_bar(Lx=96, Ly=32, w_side=16, W_dis=1.0, seed=4):
    """A disordered four-terminal bar as a site graph (square lattice, t = 1,
    on-site U[-W/2, W/2] from a seeded generator): lead 0 on the left column,
    lead 1 on the right column, leads 2 and 3 on the middle w_side sites of
    the top and bottom edges."""
    rng = np.random.default_rng(seed)
    N = Lx * Ly
    H = np.zeros((N, N), np.complex128)
    for x in range(Lx):
        for y in range(Ly):
            s = x * Ly + y
            H[s, s] = W_dis * (rng.random() - 0.5)
            if y + 1 < Ly:
                H[s, s + 1] = H[s + 1, s] = 1.0
            if x + 1 < Lx:
                H[s, s + Ly] = H[s + Ly, s] = 1.0
    x0 = (Lx - w_side) // 2
    leads = [np.arange(Ly), (Lx - 1) * Ly + np.arange(Ly),
             np.array([x * Ly + Ly - 1 for x in range(x0, x0 + w_side)]),
             np.array([x * Ly for x in range(x0, x0 + w_side)])]
    return H, leads


def graph_flop(widths, w0):
    """Algorithmic FP64 flops of the knitting sweep per energy (8 per complex
    FMA): per slice the inverse (w^3), V g V^dagger (w_{k-1}^2 w + w^2 w_{k-1}),
    and the two carried blocks G_{0,k}, G_{k,0} (2 (w0 w_{k-1} w + w0 w^2))."""
    f = 0.0
    for k, w in enumerate(widths):
        f += w ** 3
        if k:
            p = widths[k - 1]
            f += p * p * w + w * w * p + 2 * (w0 * p * w + w0 * w * w)
    return 8.0 * f


def run_graph_case(args):
    """Multi-terminal transmission matrix of a disordered four-terminal bar
    (96 x 32 sites, leads of 32, 32, 16 and 16 sites; the knitting sweep over
    an arbitrary geometry, FP64): one step = T_kl for every pair of leads at
    256 energies, self-energies and outputs in device memory.  Beside it: the
    oracle's dense solve on a bounded sample of energies."""
    import torch
    from paper_1010_2627_gb300 import build, inputs, knit
    build.build()
    knit.load()
    H, leads = hall_bar()
    ne = 256
    E = inputs.energy_grid(-3.5, 3.5, ne)
    g = knit.Graph(H, leads=leads)
    widths, _ = g.slices()
    sig = []
    for l in leads:
        S = knit.System(inputs.square(len(l), 2)).lead_selfenergy(0, E, method=knit.KNIT_LEAD_MODES)[0]
        sig.append(torch.tensor(S, device="cuda"))
    P = len(leads)
    stream = torch.cuda.Stream()
    dE = torch.tensor(E, device="cuda")
    dTm = torch.empty(ne * P * P, dtype=torch.float64, device="cuda")
    dst = torch.empty(ne, dtype=torch.int32, device="cuda")

    def step():
        knit.knit_graph_conductance(g.handle, dE, sig, dTm, dst, nE=ne, stream=stream)

    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            step()
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    with torch.cuda.stream(stream):
        for k in range(args.steps):
            ev[k][0].record(stream)
            step()
            ev[k][1].record(stream)
    torch.cuda.synchronize()
    ms = statistics.mean(a.elapsed_time(b) for a, b in ev)
    Tm = dTm.cpu().numpy().reshape(ne, P, P)
    st = dst.cpu().numpy()
    flop = graph_flop([int(w) for w in widths], len(leads[0])) * ne
    achieved = flop / (ms / 1e3) / 1e12
    nsm = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    pk = measure_peaks(knit, torch, torch.cuda.current_stream(), nsm)
    line = {
        "metric": "multi-terminal T_kl energies/s (knitting over an arbitrary geometry, FP64)",
        "value": ne / (ms / 1e3), "unit": "energies/s", "n_gpus": 1, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": f"disordered four-terminal bar 96 x 32 (W = 1), leads 32/32/16/16 "
                               f"sites, {ne} energies", "slices": len(widths),
                   "max_slice_width": int(max(widths))},
        "roofline": {"bound": "fp64", "achieved": achieved, "peak": pk["dfma_tflops"],
                     "unit": "TFLOP/s", "frac": achieved / pk["dfma_tflops"],
                     "traffic": None,
                     "note": "algorithmic flops from the slice widths (graph_flop) over the "
                             "measured DFMA peak (own loop, csrc/peaks.cu)"},
        "peaks_measured": pk,
        "buttiker_sum_rule_max": float(np.abs(Tm.sum(axis=2) - Tm.sum(axis=1))[st == 0].max()),
        "status_nonzero": int((st != 0).sum())}
    if args.cpu_baseline:
        import oracle
        t0, done = time.perf_counter(), 0
        worst = 0.0
        for e in np.linspace(0, ne - 1, 4).astype(int):
            To = oracle.transmission_matrix(H, E[e], leads, [s[e].cpu().numpy() for s in sig])
            worst = max(worst, float(np.abs(To - Tm[e]).max()))
            done += 1
            if time.perf_counter() - t0 > 20.0:
                break
        dt = time.perf_counter() - t0
        line["cpu_baseline"] = {"value": done / dt, "unit": "energies/s",
                                "cores": os.cpu_count(), "kind": "oracle",
                                "sample": f"{done} energies, dense numpy inverse, {dt:.1f} s"}
        line["max_abs_dT_vs_oracle"] = worst
    print(json.dumps(line), flush=True)
    g.close()


def run_peaks_case(args):
    """The peak loops alone (one JSON line)."""
    import torch
    from paper_1010_2627_gb300 import build, knit
    build.build()
    knit.load()
    nsm = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    pk = measure_peaks(knit, torch, torch.cuda.current_stream(), nsm, reps=max(3, args.steps))
    pk["case"] = "peaks"
    pk["driver_file"] = {k: _peaks().get(k) for k in ("hbm_gbs", "bf16_tflops",
                                                        "bf16_tflops_sustained")}
    print(json.dumps(pk), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--case", default="bench",
                    choices=["bench", "peaks", "profile", "uneven", "ldos", "bdg", "eigen", "lesser",
                             "graph", "graphene"])
    ap.add_argument("--bdg-energies", dest="bdg_energies", type=int, default=2048)
    ap.add_argument("--graphene-energies", dest="graphene_energies", type=int, default=8192)
    ap.add_argument("--graphene-L", dest="graphene_L", type=int, default=1024)
    ap.add_argument("--profile-L", dest="profile_L", type=int, default=64)
    ap.add_argument("--profile-M", dest="profile_M", type=int, default=64)
    ap.add_argument("--profile-lattice", dest="profile_lattice", default="square",
                    choices=["square", "armchair", "bdg"])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="knit", choices=["knit", "reference"])
    ap.add_argument("--no-cpu-baseline", dest="cpu_baseline", action="store_false")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.case == "profile":
        run_profile_case(args)
    elif args.case == "peaks":
        run_peaks_case(args)
    elif args.case == "uneven":
        run_uneven(args)
    elif args.case == "ldos":
        run_ldos_case(args)
    elif args.case == "bdg":
        run_bdg_case(args)
    elif args.case == "eigen":
        run_eigen_case(args)
    elif args.case == "graph":
        run_graph_case(args)
    elif args.case == "graphene":
        run_graphene_case(args)
    elif args.case == "lesser":
        run_lesser_case(args)
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_knit(args)


if __name__ == "__main__":
    main()
