#!/usr/bin/env python
"""Benchmark of the chi0 / E_c hot path on one GB300 (or N replicas).

Metric: chi0 TFLOP/s (algorithmic Hermitian rank-k flops 4 NG (NG+1) K nw per
q-point, summed over the step) and seconds per q-point with all frequencies,
mixed precision against plain FP64 on the same GPU, and the E_c relative error
of the mixed mode against the FP64 mode.

Workload: the bulk-solid configuration (9 bohr cubic box, 40^3 grid, 2x2x2
k-mesh, 8 q-points, 16 occupied + 1200 empty bands, 20 Ha orbitals, NG ~ 1200,
16 frequencies, 3 PAW atoms x 13 projectors), seeded synthetic data.  One step
is one E_c evaluation over all 8 q-points: wavefunctions to the grid, pair
densities + PAW, rank-k update, FP64 log-det and quadrature.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
With --gpus N > 1 it expects torchrun.  By default the 8 q-points of one step
are split over the ranks (shard.shard_qpoints, balanced by NG^2 x pairs); each
rank evaluates its share with its own context, E_c is the sum of one scalar per
rank (shard.sharded_energy) and no collective touches the data path: total
work is fixed, so the line says "scaling": "strong".  With --replicas every
rank runs the whole step on its own copy of the workload instead (weak
scaling).  Rank 0 prints one JSON line with the whole-job throughput.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "chi0 TFLOP/s and s per q (all iw), mixed vs FP64 on 1 GB300; E_c rel. error"
WORKLOAD = "bulk 9 bohr box, 40^3 grid, 2x2x2 k, 8 q, 16 occ + 1200 empty bands, NG~1200, 16 iw, 3x13 PAW projectors"
OPTICAL_QDIR = (1.0, 1.0, 1.0)
WORKLOAD_SLAB = ("slab 9.4x8.1x40 bohr, 48x40x200 grid, 4x2x1 k, 120 occ + 3000 empty bands, NG~3000, 16 iw, "
                 "16x18 + 2x8 PAW projectors")
CLOCK_FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
                "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
                "clocks_event_reasons.sw_power_cap")


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return d, "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0, "sm_max_mhz": 2070.0}, "fallback"


class ClockSampler:
    """nvidia-smi samples (every 200 ms) of SM clock and throttle reasons during the timed region."""

    def __init__(self, device: int):
        self.device = device
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.device), f"--query-gpu={CLOCK_FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            self.t.join(timeout=2)

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            for nm, val in zip(names, parts[4:8]):
                if val.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


HERK_DEVICE_END = "// ---------------------------------------------------------------- operand preparation"


def herk_traffic():
    """DRAM bytes per launch of the rank-k kernel from the committed ncu summary,
    or None when the kernel's device code (the source up to its operand
    preparation section) has changed since the counters were taken."""
    import hashlib
    p = os.path.join(ROOT, "profiles", "herk_tc_traffic.json")
    try:
        with open(p) as f:
            d = json.load(f)
        with open(os.path.join(ROOT, d["source"])) as f:
            src = f.read()
        h = hashlib.sha256(src[:src.index(HERK_DEVICE_END)].encode()).hexdigest()
    except (OSError, KeyError, ValueError):
        return None
    if h != d.get("device_code_sha256"):
        return None
    return float(d["dram_bytes_read_per_launch"] + d["dram_bytes_write_per_launch"])


def pd_flops(grid_points, ks):
    """Algorithmic pair-density flops, FFT convention (6 N_r + 5 N_r log2 N_r per pair)."""
    import math
    return float(sum(k * (6.0 * n + 5.0 * n * math.log2(n)) for n, k in zip(grid_points, ks)))


def rankk_flops(ngs, ks, nw):
    return float(sum(4.0 * ng * (ng + 1) * k * nw for ng, k in zip(ngs, ks)))


def make_workload(config="bulk"):
    from paper_1307_8052_gb300 import synthetic as syn
    return syn.config2() if config == "slab" else syn.config1()


def workload_qpoints(args, p):
    """q-points of one step: all 8 for the bulk workload; for the slab the
    ``--slab-q`` q-points from (0, 1/2, 0) on (8 transitions each)."""
    if args.config == "slab":
        return list(range(1, 1 + args.slab_q))
    return list(range(len(p.qpoints)))


def pairs_per_q(p):
    out = []
    for qp in p.qpoints:
        k = 0
        for ik, ikp in zip(qp.k_of, qp.kq_of):
            k += int(np.sum(p.sets[ik].f > 0)) * int(np.sum(p.sets[ikp].f < 1))
        out.append(k)
    return out


def cpu_sample(p, steps=1, warmup=0, iq=3, nocc=4, nemp=1200):
    """Time the oracle on a bounded sample of the workload: chi0 of q-point iq from
    the first transition with nocc occupied x nemp empty bands (all G, all iw)."""
    import oracle as o
    from paper_1307_8052_gb300 import synthetic as syn
    qp = p.qpoints[iq]
    no = int(np.sum(p.sets[0].f > 0))
    sets = []
    for s in p.sets:
        keep = np.r_[np.arange(no - nocc, no), np.arange(no, no + nemp)]
        sets.append(syn.OrbitalSet(s.k_red, s.miller, s.C[keep], s.eps[keep], s.f[keep], s.P[keep]))
    sub = syn.Problem(p.name, p.config, p.cell, p.grid, p.ecut_wf, p.ecut_chi, p.spin_factor, p.nk_bz, sets,
                      [syn.QPoint(qp.q_red, qp.k_of[:1], qp.kq_of[:1], qp.G0[:1], 1.0)], p.nw, p.paw)
    gm = o.g_sphere(p.cell, qp.q_red, p.ecut_chi)
    Q = syn.paw_Q(p.paw, p.cell, qp.q_red, gm)
    om, _ = o.frequency_grid(p.nw)
    flops = rankk_flops([len(gm)], [nocc * nemp], p.nw)
    times = []
    for i in range(warmup + steps):
        t0 = time.perf_counter()
        o.chi0(sub, 0, om, Q)
        if i >= warmup:
            times.append(time.perf_counter() - t0)
    try:
        from threadpoolctl import threadpool_info
        cores = max([d.get("num_threads", 1) for d in threadpool_info()] + [1])
    except Exception:
        cores = os.cpu_count()
    t = float(np.mean(times))
    return {"value": flops / t / 1e12, "unit": "TFLOP/s", "cores": int(cores), "kind": "oracle",
            "sample": f"chi0 of q={tuple(float(x) for x in qp.q_red)}, first k-transition, {nocc} occupied x {nemp} "
                      f"empty bands, all G and iw ({flops / 1e12:.4f} TFLOP algorithmic, {t:.2f} s per sample)"}, times


def cpu_sample_for(args, p, steps=1, warmup=0):
    if args.config == "slab":
        return cpu_sample(p, steps, warmup, iq=1, nocc=2, nemp=100)
    return cpu_sample(p, steps, warmup)


def run_reference(args):
    """Reference arm: the CPU FP64 oracle as it stands, on the host cores."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    p = make_workload(args.config)
    base, times = cpu_sample_for(args, p, steps=args.steps, warmup=args.warmup)
    t = float(np.mean(times))
    line = {"impl": "reference", "metric": METRIC, "value": base["value"], "unit": "TFLOP/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": t * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD_SLAB if args.config == "slab" else WORKLOAD, "sample": base["sample"]},
            "cpu_baseline": base,
            "e2e": {"value": base["value"], "unit": "TFLOP/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def run_ours(args):
    import torch
    from paper_1307_8052_gb300 import binding as b
    from paper_1307_8052_gb300 import shard
    from paper_1307_8052_gb300 import synthetic as syn
    from paper_1307_8052_gb300.build import build

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    torch.cuda.set_device(local)
    if rank == 0:
        build()
    if dist:
        dist.barrier()
    b.load()
    stream = torch.cuda.current_stream()

    p = make_workload(args.config)
    iqs_all = workload_qpoints(args, p)
    om, W = b.rpa_gauss_legendre(p.nw, 1.0)
    Kall = pairs_per_q(p)

    # q = 0 of the bulk mesh carries the optical-limit head and wings (Eqs. 12-14)
    optical_all = [i for i in iqs_all if np.all(p.qpoints[i].q_red == 0)] if args.config == "bulk" else []

    def make_ctx(precision, qs):
        ctx = b.rpa_create(p.cell, p.grid, p.ecut_chi, p.spin_factor, p.nk_bz, precision, device=local,
                           stream=stream.cuda_stream)
        ngs = b.load_problem(ctx, p, qs=qs,
                             paw_Q=lambda iq, gm: syn.paw_Q(p.paw, p.cell, p.qpoints[iq].q_red, gm))
        for iq in optical_all:
            if iq in qs:
                b.rpa_set_optical(ctx, iq, OPTICAL_QDIR, p.paw.nproj, syn.paw_Qnabla(p.paw, p.config))
        if args.paw_tc:
            b.rpa_set_tuning(ctx, b.RPA_TUNE_PAW_TC, 1)
        if args.tc_pair is not None:
            b.rpa_set_tuning(ctx, b.RPA_TUNE_TC_PAIR, args.tc_pair)
        return ctx, ngs

    # every rank loads every q-point of the step (the response spheres give the
    # cost of each), then evaluates the share shard.shard_qpoints assigns it,
    # or the whole step with --replicas
    ctx, ngs_all = make_ctx(args.precision, iqs_all)
    costs = [float(ng) ** 2 * Kall[iq] for ng, iq in zip(ngs_all, iqs_all)]
    shards = shard.partition(iqs_all, costs, world, args.replicas)
    iqs = shards[rank]
    nq = len(iqs)
    wq = [p.qpoints[i].weight for i in iqs]
    Kq = [Kall[i] for i in iqs]
    ngs = [ngs_all[iqs_all.index(i)] for i in iqs]
    # whole-job work: every rank's share (replicas: world copies of the step)
    job_flops = float(sum(rankk_flops([ngs_all[iqs_all.index(i)] for i in part], [Kall[i] for i in part], p.nw)
                          for part in shards))
    flops = rankk_flops(ngs, Kq, p.nw)
    b.rpa_set_profiling(ctx, True)

    def barrier():
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        torch.cuda.synchronize()

    def max_over_ranks(x):
        return shard.max_over_ranks(x, device="cuda")

    wq_all = [p.qpoints[i].weight for i in iqs_all]

    def evaluate(qs, wqs):
        return b.rpa_energy(ctx, qs, wqs, om, W)[0]

    def step():
        # this rank's share (or the whole step with --replicas); E_c summed over the ranks
        return shard.sharded_step(evaluate, iqs_all, costs, wq_all, rank, world, device="cuda",
                                  replicas=args.replicas)

    for _ in range(args.warmup):
        step()
    barrier()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    stage_ms = np.zeros(b.RPA_NSTAGES)
    launches = np.zeros(b.RPA_NSTAGES, dtype=np.int64)
    with ClockSampler(local) as clk:
        e0.record(stream)
        for _ in range(args.steps):
            E = step()
            ms, nl = b.rpa_get_profile(ctx)
            stage_ms += ms
            launches += nl
        e1.record(stream)
        barrier()
    t_step = e0.elapsed_time(e1) / args.steps / 1e3
    t_step = max_over_ranks(t_step)
    value = job_flops / t_step / 1e12

    # end to end through the public API from pinned host buffers
    pinned = []
    for s in p.sets:
        pinned.append((torch.from_numpy(s.C).pin_memory(), torch.from_numpy(s.P).pin_memory()))
    Qpin = {}
    for iq in iqs:
        gm = b.rpa_gvectors(ctx, iq)
        Qpin[iq] = torch.from_numpy(syn.paw_Q(p.paw, p.cell, p.qpoints[iq].q_red, gm)).pin_memory()
    h2d = sum(c.numel() * 16 + pp.numel() * 16 for c, pp in pinned) + sum(q.numel() * 16 for q in Qpin.values())
    h2d += sum(s.miller.nbytes + s.eps.nbytes + s.f.nbytes for s in p.sets)
    d2h = 8 * (1 + nq * p.nw)

    def e2e_step():
        for i, s in enumerate(p.sets):
            b.rpa_set_orbitals(ctx, i, s.k_red, s.miller, pinned[i][0], s.eps, s.f)
            b.rpa_set_paw(ctx, i, p.paw.nproj, pinned[i][1])
        for iq in iqs:
            b.rpa_set_paw_Q(ctx, iq, p.paw.nproj, Qpin[iq])
        return step()

    t_e2e = float("nan")
    # the end-to-end figure is the plain API path: stage profiling off
    b.rpa_set_profiling(ctx, False)
    if not args.no_e2e:
        e2e_step()
        barrier()
        e0.record(stream)
        for _ in range(args.steps):
            e2e_step()
        e1.record(stream)
        barrier()
        t_e2e = max_over_ranks(e0.elapsed_time(e1) / args.steps / 1e3)

    # plain FP64 form, and the FP32 mode, on one q-point (rank 0) for the
    # mixed-vs-FP64 statement: time per q, TFLOP/s, E_c error against FP64
    modes = {}
    if rank == 0 and args.fp64_q >= 0 and args.config == "bulk":
        iq = args.fp64_q
        pos = iqs_all.index(iq)
        fq = rankk_flops([ngs_all[pos]], [Kall[iq]], p.nw)
        Emix, tmix = b.rpa_energy(ctx, [iq], [1.0], om, W)
        for mode in ("fp64", "fp32"):
            if mode == "fp32" and args.no_fp32:
                continue
            cm, _ = make_ctx(mode, [iq])
            if mode == "fp32":
                b.rpa_energy(cm, [iq], [1.0], om, W)  # one untimed warm-up (the FP64 run is long enough without)
            b.rpa_set_profiling(cm, True)
            torch.cuda.synchronize()
            e0.record(stream)
            Em, tm = b.rpa_energy(cm, [iq], [1.0], om, W)
            e1.record(stream)
            torch.cuda.synchronize()
            sm_ = e0.elapsed_time(e1) / 1e3
            msm, _ = b.rpa_get_profile(cm)
            b.rpa_destroy(cm)
            modes[mode] = {"q": iq, "s_per_q": sm_, "chi0_tflops": fq / sm_ / 1e12, "rankk_ms": msm[2],
                           "logdet_ms": msm[3], "E_c_q": Em, "terms": tm}
        if "fp64" in modes:
            E64, t64 = modes["fp64"]["E_c_q"], modes["fp64"].pop("terms")
            modes["fp64"].update({"speedup_mixed_vs_fp64": modes["fp64"]["s_per_q"] / (t_step / max(nq, 1)),
                                  "ec_q_fp64": E64, "ec_q_mixed": Emix,
                                  "ec_rel_error": abs(Emix - E64) / abs(E64),
                                  "terms_max_rel_error": float(np.max(np.abs(tmix - t64)) / np.max(np.abs(t64)))})
            if "fp32" in modes:
                t32 = modes["fp32"].pop("terms")
                E32 = modes["fp32"]["E_c_q"]
                modes["fp32"].update({"ec_rel_error_vs_fp64": abs(E32 - E64) / abs(E64),
                                      "terms_max_rel_error_vs_fp64":
                                          float(np.max(np.abs(t32 - t64)) / np.max(np.abs(t64))),
                                      "speedup_vs_fp64": modes["fp64"]["s_per_q"] / modes["fp32"]["s_per_q"]})

    peaks, peak_kind = load_peaks()
    herk_ms = stage_ms[2] / args.steps
    peak_sus = None
    if args.precision in ("bf16x2", "bf16x3"):
        peak = peaks.get("bf16_tflops_sustained" if args.sustained else "bf16_tflops")
        peak_sus = peaks.get("bf16_tflops_sustained")
        bound = "tensor"
    else:
        sm_mhz = peaks.get("sm_max_mhz", 2070.0)
        peak = (152 * 128 * 2 * sm_mhz * 1e6 / 1e12) if args.precision == "fp32" else 1.05
        bound = "alu"
    achieved = flops / (herk_ms / 1e3) / 1e12 if herk_ms > 0 else None
    fp32_peak = 152 * 128 * 2 * peaks.get("sm_max_mhz", 2070.0) * 1e6 / 1e12
    pd_fl = pd_flops([int(np.prod(p.grid))] * len(Kq), Kq)
    base = None
    if rank == 0 and not args.no_cpu:
        base, _ = cpu_sample_for(args, p, steps=1, warmup=0)
    b.rpa_destroy(ctx)
    if rank != 0:
        return
    stage_names = ["wf_to_grid", "pair_density_paw", "rankk_kernel", "logdet", "other", "rankk_operand_prep"]
    mixed = args.precision in ("fp32", "bf16x2", "bf16x3")
    terms = {"bf16x2": 2, "bf16x3": 3}.get(args.precision)
    line = {
        "metric": METRIC, "value": value, "unit": "TFLOP/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": t_step * 1e3, "higher_is_better": True,
        "scaling": "weak" if (args.replicas or world == 1) else "strong",
        "vs_baseline": None, "dtype": {"fp64": "f64", "fp32": "f32", "bf16x2": "bf16x2->f32",
                                       "bf16x3": "bf16x3->f32"}[args.precision],
        "data": "synthetic",
        "config": {"workload": WORKLOAD_SLAB if args.config == "slab" else WORKLOAD, "precision": args.precision,
                   "q_points": len(iqs_all), "NG": ngs_all,
                   "optical_limit": (f"q=0 head and wings along {OPTICAL_QDIR}" if optical_all else None),
                   "paw_product": "tensor cores" if args.paw_tc else "CUDA cores (FP32)",
                   "rankk": (f"tcgen05 split bfloat16 ({terms} terms per operand, FP32 accumulation in TMEM, "
                             "FP32 register folds, FP64 chi0)" if terms else
                             "CUDA cores, FP32 with compensated folds into FP64 chi0" if args.precision == "fp32"
                             else "CUDA cores, FP64"),
                   "logdet": ("blocked Cholesky, float-float trailing update (~44 bits) with FP64 pivots, "
                              "FP64 diagonal blocks and inverses, one-panel look-ahead" if mixed else
                              "blocked Cholesky, FP64 throughout"),
                   "quadrature": "FP64 Gauss-Legendre, 16 nodes mapped to [0, inf)",
                   "pairs_per_q": [Kall[i] for i in iqs_all], "nw": p.nw,
                   "l2": "inputs larger than L2 (grids >= 1.2 GB, pair densities + rank-k operands >= 3.5 GB per block)",
                   "parallelism": (f"replicas x{world}" if args.replicas or world == 1 else
                                   f"q-points sharded over {world} ranks (no data-path collective): "
                                   + "; ".join(f"rank {r}: q {part}" for r, part in enumerate(shards)))},
        "s_per_q": t_step / max(nq, 1),
        "E_c": E,
        "stage_ms_per_step": {n: float(m / args.steps) for n, m in zip(stage_names, stage_ms)},
        "fp64": modes.get("fp64"),
        "fp32": modes.get("fp32"),
        "e2e": {"value": job_flops / t_e2e / 1e12, "unit": "TFLOP/s", "h2d_bytes_per_step": int(h2d),
                "d2h_bytes_per_step": int(d2h), "ms_per_step": t_e2e * 1e3},
        "gpu_launches": int(launches.sum()),
        "roofline_pair_density": {
            "bound": "alu", "kernels": "pd_stageA/B/C + PAW (Eqs. 4, 6, 10)",
            "achieved": pd_fl / (stage_ms[1] / args.steps / 1e3) / 1e12 if stage_ms[1] > 0 else None,
            "peak": fp32_peak, "unit": "TFLOP/s",
            "frac": (pd_fl / (stage_ms[1] / args.steps / 1e3) / 1e12) / fp32_peak if stage_ms[1] > 0 else None,
            "flops_convention": "6 N_r + 5 N_r log2 N_r per pair on the caller's grid (FFT count)",
            "peak_source": "derived: 152 SM x 128 FP32 lanes x 2 x max clock"},
        "roofline": {"bound": bound, "kernel": "rank-k update (Eq. 17)", "achieved": achieved, "peak": peak,
                     "unit": "TFLOP/s", "frac": achieved / peak if achieved else None,
                     "peak_sustained": peak_sus,
                     "frac_sustained": (achieved / peak_sus) if (achieved and peak_sus) else None,
                     "issued_frac": ((achieved * {2: 3, 3: 6}[terms] / peak) if (achieved and terms) else None),
                     "issued_note": "hardware bf16 products per algorithmic product: 3 (two terms) or 6 (three)",
                     "traffic": herk_traffic() if (bound == "tensor" and args.config == "bulk") else None,
                     "traffic_note": "ncu DRAM read+write bytes of one launch of the profiling case (one k-block, "
                                     "NG 1180); null once the kernel's device code differs from the captured one",
                     "peak_source": (f"{peak_kind} (bf16 burst; frac_sustained uses the sustained figure)"
                                     if bound == "tensor" else "derived: 152 SM x 128 FP32 lanes x 2 x max clock")},
        "clocks": clk.summary(),
        "cpu_baseline": base,
    }
    print(json.dumps(line))


def run_backward(args):
    """Gradient workload: the bulk geometry at one q = (1/2, 0, 0) with all 8
    k-points and 16 occupied + 1200 empty bands per set; one step is
    rpa_energy_backward for dE_c/dchi0, dE_c/dC and dE_c/dP of every set (the
    forward pass included), outputs in device memory."""
    import torch
    from paper_1307_8052_gb300 import binding as b
    from paper_1307_8052_gb300 import synthetic as syn
    from paper_1307_8052_gb300.build import build

    torch.cuda.set_device(0)
    build()
    b.load()
    stream = torch.cuda.current_stream()
    p = syn.config1()
    iq = [i for i, qp in enumerate(p.qpoints) if np.allclose(qp.q_red, [0.5, 0.0, 0.0])][0]
    om, W = b.rpa_gauss_legendre(p.nw, 1.0)
    ctx = b.rpa_create(p.cell, p.grid, p.ecut_chi, p.spin_factor, p.nk_bz, args.precision,
                       stream=stream.cuda_stream)
    ng = b.load_problem(ctx, p, qs=[iq], paw_Q=lambda i, gm: syn.paw_Q(p.paw, p.cell, p.qpoints[i].q_red, gm))[0]
    b.rpa_set_tuning(ctx, b.RPA_TUNE_GAMMA, args.gamma)
    K = pairs_per_q(p)[iq]
    dev = torch.device("cuda")
    dC = [torch.zeros(s.C.shape, dtype=torch.complex128, device=dev) for s in p.sets]
    dP = [torch.zeros(s.P.shape, dtype=torch.complex128, device=dev) for s in p.sets]
    dchi = [torch.zeros((p.nw, ng, ng), dtype=torch.complex128, device=dev)]
    sets = list(range(len(p.sets)))
    wq = [p.qpoints[iq].weight]

    def step():
        return b.rpa_energy_backward(ctx, [iq], wq, om, W, 1.0, sets, dC, dP, dchi)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    b.rpa_set_profiling(ctx, True)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    stage_ms = np.zeros(b.RPA_NSTAGES)
    with ClockSampler(0) as clk:
        e0.record(stream)
        for _ in range(args.steps):
            E = step()
            stage_ms += b.rpa_get_profile(ctx)[0]
        e1.record(stream)
        torch.cuda.synchronize()
    t = e0.elapsed_time(e1) / args.steps / 1e3
    b.rpa_destroy(ctx)
    f_fwd = rankk_flops([ng], [K], p.nw)
    f_bwd = 8.0 * ng * ng * K * p.nw  # N-bar = 2 sum_w w Gamma_w n: one complex NG x NG by NG x K product per w
    stage_names = ["wf_to_grid", "pair_density_paw", "rankk_kernel", "logdet", "other_and_adjoint",
                   "rankk_operand_prep"]
    line = {"metric": "E_c gradient (dE/dchi0, dE/dC, dE/dP incl. forward) TFLOP/s on 1 GB300",
            "value": (f_fwd + f_bwd) / t / 1e12, "unit": "TFLOP/s", "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": t * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": args.precision, "data": "synthetic",
            "config": {"workload": "gradient: bulk 9 bohr box, 40^3 grid, q=(1/2,0,0), 8 k, 16 occ + 1200 empty "
                                   "bands, NG %d, 16 iw, 3x13 PAW" % ng, "pairs": K,
                       "flops": {"forward_rankk": f_fwd, "adjoint_nbar": f_bwd},
                       "dE_dchi0": {0: "FP64 from the Cholesky factor", 1: "FP32 product form",
                                    2: "float-float products"}[args.gamma]},
            "E_c_q": E, "stage_ms_per_step": {n: float(m / args.steps) for n, m in zip(stage_names, stage_ms)},
            "clocks": clk.summary()}
    print(json.dumps(line))


def run_batched(args):
    """Batched workload: ``--instances`` (q, cell) instances of uneven sizes
    (NG ~ U[400, 3000], n_occ ~ U[8, 120], n_unocc ~ NG, 16 frequencies, PAW),
    evaluated (a) as plain sequential rpa_energy calls, (b) as one CUDA graph of
    every instance's own launches and (c) as one CUDA graph built around
    persistent rank-k launches that pull (block, tile, frequency) items of all
    instances from a device queue.  Launch shapes come from the autotuner, one
    greedy search per (NG, pairs) size class, applied to every instance of that
    class; the persistent form keeps the per-instance pair-density shapes and
    runs its rank-k items with one pipeline shape."""
    import torch
    from paper_1307_8052_gb300 import autotune as at
    from paper_1307_8052_gb300 import binding as b
    from paper_1307_8052_gb300 import synthetic as syn
    from paper_1307_8052_gb300.build import build

    torch.cuda.set_device(0)
    build()
    b.load()
    t0 = time.perf_counter()
    rng_kw = {"ng_range": (400, 900), "nocc_range": (8, 32)} if args.small else {}
    probs = [syn.config3_instance(i, **rng_kw) for i in range(args.instances)]
    gen_s = time.perf_counter() - t0
    stream = torch.cuda.Stream()
    om, W = b.rpa_gauss_legendre(16, 1.0)
    ctxs, flops, ngs, pairs = [], [], [], []
    for p in probs:
        ctx = b.rpa_create(p.cell, p.grid, p.ecut_chi, p.spin_factor, p.nk_bz, args.precision,
                           stream=stream.cuda_stream)
        b.rpa_set_tuning(ctx, b.RPA_TUNE_OPERAND_MB, 512)
        ng = b.load_problem(ctx, p, paw_Q=lambda iq, gm, p=p: syn.paw_Q(p.paw, p.cell, p.qpoints[iq].q_red, gm))[0]
        b.rpa_set_frequencies(ctx, om)
        k = int(np.sum(p.sets[0].f > 0)) * int(np.sum(p.sets[1].f < 1))
        ctxs.append(ctx)
        ngs.append(ng)
        pairs.append(k)
        flops.append(rankk_flops([ng], [k], 16))
    total = float(sum(flops))
    sync = stream.synchronize
    # one greedy search per size class, applied to every instance of the class
    t0 = time.perf_counter()
    bt = at.BucketTuner(args.precision, sync=sync)
    for ctx, ng, k in zip(ctxs, ngs, pairs):
        bt.tune(ctx, ng, k, [0], [1.0], om, W)
    tune_s = time.perf_counter() - t0

    def sequential():
        for ctx in ctxs:
            b.rpa_energy(ctx, [0], [1.0], om, W)

    sequential()
    sync()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for _ in range(args.steps):
        sequential()
    ev1.record(stream)
    sync()
    t_seq = ev0.elapsed_time(ev1) / args.steps / 1e3

    def graph_time():
        g = b.rpa_graph_create(ctxs, [[0]] * len(ctxs))
        try:
            b.rpa_graph_launch(g)
            sync()
            ev0.record(stream)
            for _ in range(args.steps):
                b.rpa_graph_launch(g)
            ev1.record(stream)
            sync()
            t = ev0.elapsed_time(ev1) / args.steps / 1e3
            E = [b.rpa_energy_collect(ctx, [1.0], W, 1)[0] for ctx in ctxs]
        finally:
            b.rpa_graph_destroy(g)
        return t, E

    b.rpa_set_tuning(ctxs[0], b.RPA_TUNE_BATCH_PERSIST, 0)
    t_graph, E_graph = graph_time()
    persist = args.precision == "bf16x2"
    t_pers, E_pers = None, None
    if persist:
        # the persistent form runs every rank-k item with one pipeline shape
        for ctx in ctxs:
            b.rpa_set_tuning(ctx, b.RPA_TUNE_TC_PIPE, 0)
            b.rpa_set_tuning(ctx, b.RPA_TUNE_TC_FUSE, 0)
        b.rpa_set_tuning(ctxs[0], b.RPA_TUNE_BATCH_PERSIST, 1)
        t_pers, E_pers = graph_time()
    free_gb = torch.cuda.mem_get_info()[0] / 1e9
    for ctx in ctxs:
        b.rpa_destroy(ctx)
    t_best = min(t for t in (t_graph, t_pers) if t is not None)
    line = {"metric": METRIC + " (batched instances)", "value": total / t_best / 1e12, "unit": "TFLOP/s",
            "n_gpus": 1, "steps": args.steps, "warmup": 1, "ms_per_step": t_best * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": args.precision, "data": "synthetic",
            "config": {"workload": f"{len(ctxs)} (q, cell) instances, "
                                   + ("NG 400-900, n_occ 8-32" if args.small else "NG 400-3000, n_occ 8-120")
                                   + ", n_unocc ~ NG, 16 iw, 3x13 PAW, one CUDA graph", "NG": ngs, "pairs": pairs,
                       "generation_s": gen_s, "flops": total, "device_free_gb_at_end": free_gb},
            "sequential": {"value": total / t_seq / 1e12, "ms_per_step": t_seq * 1e3},
            "graph_per_instance": {"value": total / t_graph / 1e12, "ms_per_step": t_graph * 1e3},
            "graph_persistent": (None if t_pers is None else
                                 {"value": total / t_pers / 1e12, "ms_per_step": t_pers * 1e3,
                                  "E_c_max_diff_vs_per_instance": float(max(abs(a - c) for a, c in
                                                                            zip(E_pers, E_graph)))}),
            "speedup_vs_sequential": t_seq / t_best,
            "autotune": {"buckets": len(bt.table), "tune_s": tune_s,
                         "table": {str(k): {str(p): v for p, v in val.items()} for k, val in bt.table.items()}},
            "E_c_sum": float(np.sum(E_pers if E_pers is not None else E_graph))}
    print(json.dumps(line))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--precision", choices=["fp64", "fp32", "bf16x2", "bf16x3"], default="bf16x2")
    ap.add_argument("--fp64-q", type=int, default=3, help="q-point timed in plain FP64 (-1: skip)")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-fp32", action="store_true", help="skip the FP32-mode q-point")
    ap.add_argument("--replicas", action="store_true",
                    help="N > 1: every rank runs the whole step (weak scaling) instead of a share of its q-points")
    ap.add_argument("--sustained", action="store_true")
    ap.add_argument("--no-e2e", action="store_true", help="skip the end-to-end (host buffer) measurement")
    ap.add_argument("--config", choices=["bulk", "slab", "batched", "backward"], default="bulk")
    ap.add_argument("--slab-q", type=int, default=1, help="q-points per step of the slab workload")
    ap.add_argument("--paw-tc", action="store_true",
                    help="PAW product on the tensor cores (split modes; faster for many projectors, larger E_c error)")
    ap.add_argument("--tc-pair", type=int, choices=[0, 1, 2], default=None,
                    help="rank-k launch paired over frequencies (TMA multicast of the shared operand); "
                         "default: the library's")
    ap.add_argument("--instances", type=int, default=64)
    ap.add_argument("--small", action="store_true",
                    help="--config batched: small instances only (NG 400-900, n_occ 8-32)")
    ap.add_argument("--gamma", type=int, choices=[0, 1, 2], default=2,
                    help="--config backward: dE/dchi0 in FP64 (0), FP32 product form (1) or float-float (2)")
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
    elif args.config == "batched":
        run_batched(args)
    elif args.config == "backward":
        run_backward(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
