#!/usr/bin/env python3
"""Benchmark of the FFT bispectrum-multipole estimator (arXiv:1708.05303, Sec. 3.1).

One step = one full bsp_compute on one synthetic realisation: shell/Legendre
filter + batched inverse 3-D FFTs of every field + contraction of all valid
bins + FP64 reduction and normalisation.  Workload: 512^3 grid, L = 1000
Mpc/h, 64 shells of width 2 k_f from k_f, l = 0, 2, 4 (25 424 bins x 3).
The triangle counts are geometry only; they are computed once before the
timed region.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line (rank 0).  Under torchrun every rank runs its own
independent realisation (replicas; no collective on the data path) and the
value is the bins all ranks finished divided by the slowest rank's time.
``--impl reference`` times the FP64 CPU oracle instead, on a bounded sample
of the same workload: ms_per_step is the measured sample time, and the bins/s
value is extrapolated to the whole step (labelled as such in the line).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "B_0,2,4 bins/s at 512^3, 64 shells; split-BF16 vs FP32 speedup at 1e-5 err"
BOX = 1000.0
SEED = 1708 + 2          # the 512^3 workload's seed
FP32_LANES_PER_SM = 128
N_SM = 152


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--n", type=int, default=512)
    ap.add_argument("--shells", type=int, default=64)
    ap.add_argument("--width", type=float, default=2.0, help="shell width in k_f")
    ap.add_argument("--prec", default="split_f16", choices=["fp32", "split_bf16", "split_f16", "bf16"])
    ap.add_argument("--no-fp32-compare", action="store_true",
                    help="skip timing the plain FP32 CUDA-core contraction beside the split path")
    ap.add_argument("--chunk", type=int, default=0, help="tensor-core FP32 accumulation chunk (points)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-precision-compare", action="store_true",
                    help="skip timing split-BF16 and plain BF16 beside the benchmarked path")
    ap.add_argument("--no-modal", action="store_true", help="skip the 512^3 / 50-mode modal entry")
    ap.add_argument("--no-batch", action="store_true", help="skip the 512-mock uneven-grid batch entry")
    ap.add_argument("--batch-mocks", type=int, default=512)
    return ap.parse_args()


def workload(n, shells, width=2.0):
    from paper_1708_05303_gb300.synth import linear_edges

    edges = linear_edges(shells, width)
    desc = ("%d^3 grid, L=%g Mpc/h, sigma_g=0.3 quadratic+Kaiser field, %d shells of width %g k_f from k_f, "
            "l=0,2,4" % (n, BOX, shells, width))
    return edges, desc


def make_input(n):
    from paper_1708_05303_gb300.synth import FieldModel, make_field

    dk, _ = make_field(FieldModel(n=n, box=BOX, sigma_g=0.3), SEED)
    return dk


class Clocks:
    """nvidia-smi sampling during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.idx = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.idx), "--query-gpu=" + self.FIELDS,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9:
                rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


def cpu_sample(dk, n, edges, n_fields=1, n_bins=4):
    """Time the oracle on a bounded sample of the step and extrapolate: one
    Hermitian completion, ``n_fields`` filtered fields (own FP64 FFT) and
    ``n_bins`` triple sums over all n^3 points; the step needs 3 x n_shells
    fields and 3 x n_bins_valid sums (the counts are geometry, excluded on
    both sides)."""
    import numpy as np

    import oracle

    oracle.build()
    t0 = time.perf_counter()
    full = oracle.full_from_half(dk.astype(np.complex128), n)
    t_full = time.perf_counter() - t0
    masks = oracle.shell_masks(n, edges)
    mu = oracle.mu_grid(n)
    ns = len(edges) - 1
    fields = []
    t0 = time.perf_counter()
    for i in range(n_fields):
        a = ns - 1 - i
        fields.append(oracle.real_field(full, oracle.legendre_weight(2, mu) * masks[a]))
    t_field = (time.perf_counter() - t0) / n_fields
    while len(fields) < 3:
        fields.append(fields[-1])
    t0 = time.perf_counter()
    oracle.sum3(fields, [(0, 1, 2)] * n_bins)
    t_bin = (time.perf_counter() - t0) / n_bins
    return dict(t_full=t_full, t_field=t_field, t_bin=t_bin, cores=oracle.num_threads(),
                measured_s=t_full + n_fields * t_field + n_bins * t_bin,
                sample="%d^3: Hermitian completion + %d filtered field(s) + %d triple sums, extrapolated to "
                       "%d fields + all bin sums" % (n, n_fields, n_bins, 3 * ns))


def run_reference(args):
    """The oracle as it stands, on this host's cores: each step times one
    bounded sample of the step (Hermitian completion, one filtered field,
    four triple sums over all n^3 points).  ms_per_step is that measured
    sample time; the bins/s value is the full step extrapolated from it
    (3 x n_shells fields and 3 x n_bins triple sums), reported with the
    extrapolated step time under its own key."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    import oracle

    edges, desc = workload(args.n, args.shells, args.width)
    dk = make_input(args.n)
    cand = oracle.candidate_triplets(args.shells)
    # valid bins of this geometry (no triangle can reach a > b + c + 2 for width-2 shells without wrap)
    nb = sum(1 for (a, b, c) in cand if edges[a] < edges[b + 1] + edges[c + 1])
    total_out = 3 * nb
    measured, full = [], []
    info = None
    for it in range(args.warmup + args.steps):
        info = cpu_sample(dk, args.n, edges)
        if it >= args.warmup:
            measured.append(info["measured_s"])
            full.append(info["t_full"] + 3 * args.shells * info["t_field"] + total_out * info["t_bin"])
    t_meas = statistics.median(measured)
    t_full = statistics.median(full)
    v = total_out / t_full
    line = {"metric": METRIC, "value": v, "unit": "bins/s", "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": t_meas * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
            "config": {"workload": desc, "bins": nb, "outputs": total_out},
            "step_is_sample": True,
            "extrapolated": {"ms_per_full_step": t_full * 1e3, "value_is_extrapolated": True,
                             "how": "sample seconds scaled to 3 x n_shells fields and 3 x n_bins triple sums"},
            "cpu_baseline": {"kind": "oracle", "value": v, "unit": "bins/s", "cores": info["cores"],
                             "sample": info["sample"], "measured_s": t_meas},
            "e2e": {"value": v, "unit": "bins/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    import numpy as np
    import torch

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    from paper_1708_05303_gb300 import build as B

    B.build()
    from paper_1708_05303_gb300 import bsp
    from paper_1708_05303_gb300.dist import max_over_ranks

    edges, desc = workload(args.n, args.shells, args.width)
    dk = make_input(args.n)
    t0 = time.perf_counter()
    est = bsp.Bispectrum(args.n, BOX, edges, (0, 2, 4), prec=args.prec, host_staging=not args.no_e2e)
    if args.chunk:
        bsp.bsp_set_accumulation_chunk(est.plan, args.chunk)
    torch.cuda.synchronize()
    t_counts = time.perf_counter() - t0
    nbins = len(est.bins)
    outputs = 3 * nbins
    d = torch.from_numpy(dk).cuda()
    stream = torch.cuda.current_stream()
    for _ in range(args.warmup):
        est.compute(d)
    torch.cuda.synchronize()

    def barrier():
        if world > 1:
            torch.distributed.barrier()

    clocks = Clocks(local)
    bsp.bsp_set_profiling(est.plan, True)
    barrier()
    torch.cuda.synchronize()
    clocks.start()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for _ in range(args.steps):
        est.compute(d)
    ev1.record(stream)
    torch.cuda.synchronize()
    barrier()
    ck = clocks.stop()
    ms = ev0.elapsed_time(ev1) / args.steps
    phase, ncalls, launches = bsp.bsp_phase_times(est.plan)
    bsp.bsp_set_profiling(est.plan, False)
    phase = [p / max(ncalls, 1) for p in phase]
    ms = max_over_ranks(ms, device="cuda")   # the slowest rank's time
    value = outputs * world / (ms / 1e3)

    # power-spectrum multipoles on the same shells (Eq. PowSpecMultipole): one pass over the
    # pruned half spectrum, HBM-bound; algorithmic bytes = the complex64 modes read
    est.power(d)
    torch.cuda.synchronize()
    p0, p1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    reps = 20
    p0.record(stream)
    for _ in range(reps):
        est.power(d)
    p1.record(stream)
    torch.cuda.synchronize()
    pw_ms = p0.elapsed_time(p1) / reps
    Kp = 0
    while (Kp + 1) ** 2 < edges[-1] ** 2:
        Kp += 1
    nKp, nKzp = (min(args.n, 2 * Kp + 1), min(args.n // 2 + 1, Kp + 1))
    pw_bytes = nKp * nKp * nKzp * 8.0
    # skew-spectrum multipoles on the same shells: inverse FFT of delta, square,
    # forward FFT, shell-averaged cross spectrum (separate workspace)
    import ctypes as _ct
    _sb = _ct.c_size_t()
    bsp.load().bsp_skew_workspace_size(est.plan, _ct.byref(_sb))
    sws = torch.empty(_sb.value, dtype=torch.uint8, device="cuda")
    est.skew(d, ws=sws)
    torch.cuda.synchronize()
    s0, s1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    s0.record(stream)
    for _ in range(5):
        est.skew(d, ws=sws)
    s1.record(stream)
    torch.cuda.synchronize()
    sk_ms = s0.elapsed_time(s1) / 5
    del sws
    # integrated-bispectrum multipoles (Sec. 3.4) on the same shells over 8^3
    # sub-cubes: inverse FFT of delta, 512 batched sub-cube forward FFTs,
    # cube-mean-weighted shell sums (separate workspace)
    ib_m = 8 if args.n % 8 == 0 and args.n // 8 >= 8 else 2
    bsp.load().bsp_ib_workspace_size(est.plan, ib_m, _ct.byref(_sb))
    iws = torch.empty(_sb.value, dtype=torch.uint8, device="cuda")
    est.integrated(d, ib_m, ws=iws)
    torch.cuda.synchronize()
    s0.record(stream)
    for _ in range(5):
        est.integrated(d, ib_m, ws=iws)
    s1.record(stream)
    torch.cuda.synchronize()
    ib_ms = s0.elapsed_time(s1) / 5
    del iws
    sk_bytes = skew_alg_bytes(args.n, edges)
    ib_bytes = ib_alg_bytes(args.n, edges, ib_m)
    # density input stage (CIC + interlacing + forward FFT) on the particle workload's
    # shape: 256^3 grid, 4 Mi particles (uniform positions: the cost does not depend on them)
    dn, dnp = 256, 4 * 2 ** 20
    dpos = torch.rand((dnp, 3), device="cuda", dtype=torch.float32,
                      generator=torch.Generator(device="cuda").manual_seed(SEED)) * BOX
    dws = None
    _, _ = bsp.density_from_particles(dpos, dn, BOX)
    torch.cuda.synchronize()
    _nb = _ct.c_size_t()
    bsp.load().bsp_density_workspace_size(dn, _ct.byref(_nb))
    dws = torch.empty(_nb.value, dtype=torch.uint8, device="cuda")
    bsp.density_from_particles(dpos, dn, BOX, ws=dws)
    torch.cuda.synchronize()
    q0, q1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    q0.record(stream)
    for _ in range(5):
        bsp.density_from_particles(dpos, dn, BOX, ws=dws)
    q1.record(stream)
    torch.cuda.synchronize()
    den_ms = q0.elapsed_time(q1) / 5
    nh = dn * dn * (dn // 2 + 1)
    # algorithmic bytes: positions, two grids written (atomics) and read, the two
    # spectra written by the z pass, read + written by the y and x passes, read by
    # the combine, and the output written
    den_bytes = dnp * 12.0 + 2 * dn ** 3 * 4 * 2 + 2 * nh * 8 * 5 + nh * 8
    del dpos, dws
    # end to end through the C ABI with host buffers (pinned), copies inside the timed region
    e2e = None
    if not args.no_e2e:
        host = torch.from_numpy(np.ascontiguousarray(dk)).pin_memory()
        Bh = torch.empty((3, nbins), dtype=torch.float64).pin_memory()
        est.compute_host(host.numpy(), Bh.numpy())
        barrier()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            est.compute_host(host.numpy(), Bh.numpy())
        dt = (time.perf_counter() - t0) / args.steps
        barrier()
        dt = max_over_ranks(dt, device="cuda")
        e2e = {"value": outputs * world / dt, "unit": "bins/s", "h2d_bytes_per_step": int(host.numel() * 8),
               "d2h_bytes_per_step": int(Bh.numel() * 8)}

    # roofline of the dominant phase
    n3 = float(args.n) ** 3
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        pass
    fft_ms, con_ms, red_ms = phase
    stats = bsp.bsp_plan_stats(est.plan)
    # measured FP32 FMA throughput of this GPU (the CUDA-core path's peak)
    try:
        fp32_peak, fp32_peak_ms = bsp.bsp_fp32_fma_peak()
    except Exception:
        fp32_peak, fp32_peak_ms = None, None
    flop = 2.0 * n3 * outputs
    issued = 2.0 * n3 * stats["issued_macs_per_point"]
    if con_ms >= fft_ms and args.prec == "fp32":
        clk = 2070.0
        peak = fp32_peak or N_SM * FP32_LANES_PER_SM * 2 * clk * 1e6 / 1e12
        ach = flop / (con_ms / 1e3) / 1e12
        roof = {"kernel": "k_contract_cc (FP32 CUDA-core contraction)", "bound": "alu", "achieved": ach,
                "peak": peak, "unit": "TFLOP/s", "frac": ach / peak, "traffic": None,
                "peak_source": ("measured: bsp_fp32_fma_peak (FMA chains, all SMs, CUDA events)" if fp32_peak
                                else "derived: 152 SMs x 128 FP32 lanes x 2 flop x 2070 MHz"),
                "algorithmic": "2 n^3 flop per (bin, l): %.3e flop per launch" % flop,
                "issued_frac": (issued / (con_ms / 1e3) / 1e12) / peak}
    elif con_ms >= fft_ms:
        peak = peaks.get("bf16_tflops_sustained", 1700.0)
        # DRAM bytes per launch: ncu capture of this kernel at 160^3 with the same bins,
        # schedule and default 64-point chunk (11.385 GB read + 0.597 GB written per
        # launch) scaled by the points
        traffic = (11.982e9 * (args.n / 160.0) ** 3
                   if (args.shells, args.prec, args.chunk) == (64, "split_f16", 0) else None)
        ach = flop / (con_ms / 1e3) / 1e12
        roof = {"kernel": "k_contract_tc (tcgen05 split-product contraction)", "bound": "tensor",
                "achieved": ach, "peak": peak, "unit": "TFLOP/s", "frac": ach / peak, "traffic": traffic,
                "traffic_unit": "bytes per launch (dram read + write)",
                "peak_source": ("MEASURED_PEAKS.json bf16_tflops_sustained (dense FP16 and BF16 run at the same "
                                "rate)" if peaks else "fallback 1700 TFLOP/s sustained"),
                "algorithmic": "2 n^3 flop per (bin, l): %.3e flop per launch" % flop,
                "issued_tflops": issued / (con_ms / 1e3) / 1e12,
                "issued_frac": (issued / (con_ms / 1e3) / 1e12) / peak}
    else:
        g = fft_alg_bytes(args.n, edges)
        ach = g / (fft_ms / 1e3) / 1e9
        peak = peaks.get("hbm_gbs", 6800.0)
        roof = {"kernel": "k_pass1/2/3 (filter + inverse FFT)", "bound": "hbm", "achieved": ach, "peak": peak,
                "unit": "GB/s", "frac": ach / peak, "traffic": None,
                "peak_source": "MEASURED_PEAKS.json hbm_gbs" if peaks else "fallback 6800 GB/s",
                "algorithmic": "%.3e bytes per step" % g}
    roof["schedule"] = stats
    line = {"metric": METRIC, "value": value, "unit": "bins/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": {"fp32": "f32", "split_bf16": "bf16x3", "split_f16": "f16x3", "bf16": "bf16"}[args.prec],
            "data": "synthetic",
            "config": {"workload": desc, "bins": nbins, "outputs": outputs, "precision": args.prec,
                       "parallelism": "replicas" if world > 1 else "single",
                       "l2": "inputs larger than L2 (delta(k) %.0f MB, fields %.0f GB)"
                             % (dk.nbytes / 1e6, 3 * args.shells * n3 * 4 / 1e9),
                       "counts_s": round(t_counts, 3)},
            "phases_ms": {"filter_fft": fft_ms, "contraction": con_ms, "reduce": red_ms},
            "roofline": roof, "e2e": e2e, "gpu_launches": launches * args.steps, "clocks": ck,
            "density_stage": {"ms": den_ms, "grid": dn, "particles": dnp,
                              "particles_per_s": dnp / (den_ms / 1e3), "algorithmic_bytes": den_bytes,
                              "achieved_gbs": den_bytes / (den_ms / 1e3) / 1e9,
                              "frac_hbm": den_bytes / (den_ms / 1e3) / 1e9 / peaks.get("hbm_gbs", 6800.0)},
            "skew_spectrum": {"ms": sk_ms, "shells_per_s": args.shells * 3 / (sk_ms / 1e3),
                              "algorithmic_bytes": sk_bytes, "achieved_gbs": sk_bytes / (sk_ms / 1e3) / 1e9,
                              "frac_hbm": sk_bytes / (sk_ms / 1e3) / 1e9 / peaks.get("hbm_gbs", 6800.0)},
            "integrated_bispectrum": {"ms": ib_ms, "subcubes": ib_m ** 3, "subcube_side": args.n // ib_m,
                                      "shells_per_s": args.shells * 3 / (ib_ms / 1e3),
                                      "algorithmic_bytes": ib_bytes,
                                      "achieved_gbs": ib_bytes / (ib_ms / 1e3) / 1e9,
                                      "frac_hbm": ib_bytes / (ib_ms / 1e3) / 1e9 / peaks.get("hbm_gbs", 6800.0)},
            "power_multipoles": {"ms": pw_ms, "shells_per_s": args.shells * 3 / (pw_ms / 1e3),
                                 "algorithmic_bytes": pw_bytes, "achieved_gbs": pw_bytes / (pw_ms / 1e3) / 1e9,
                                 "frac_hbm": pw_bytes / (pw_ms / 1e3) / 1e9 / peaks.get("hbm_gbs", 6800.0)}}
    # the plain FP32 CUDA-core path on the same input (shared counts and workspace),
    # for the split-vs-FP32 speedup and the largest departure between the two
    if args.prec != "fp32" and not args.no_fp32_compare:
        ref = bsp.Bispectrum(args.n, BOX, edges, (0, 2, 4), prec="fp32", counts_from=est, ws=est.ws)
        ref.compute(d)
        torch.cuda.synchronize()
        bsp.bsp_set_profiling(ref.plan, True)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        k32 = 2
        e0.record(stream)
        for _ in range(k32):
            ref.compute(d)
        e1.record(stream)
        torch.cuda.synchronize()
        ms32 = e0.elapsed_time(e1) / k32
        ph32, nc32, _ = bsp.bsp_phase_times(ref.plan)
        bsp.bsp_set_profiling(ref.plan, False)
        ph32 = [p / max(nc32, 1) for p in ph32]
        Bs = est.compute(d).clone()
        Bf = ref.compute(d)
        rms = torch.sqrt(torch.mean(Bf * Bf, dim=1, keepdim=True))
        dev = torch.max(torch.abs(Bs - Bf) / torch.maximum(torch.abs(Bf), rms)).item()
        line["fp32_compare"] = {"ms_per_step": ms32, "contraction_ms": ph32[1], "filter_fft_ms": ph32[0],
                                "speedup_step": ms32 / ms, "speedup_contraction": ph32[1] / con_ms,
                                "max_rel_dev_vs_fp32": dev, "steps": k32,
                                "fp32_contraction_tflops": flop / (ph32[1] / 1e3) / 1e12,
                                "fp32_peak_tflops_measured": fp32_peak,
                                "fp32_frac_of_measured_peak": (flop / (ph32[1] / 1e3) / 1e12 / fp32_peak
                                                               if fp32_peak else None)}
        gg = golden_gate(est.bins, Bf.cpu().numpy(), args.n, args.shells, args.width)
        if gg:
            line["fp32_compare"].update(gg)
        if not args.no_precision_compare:
            line["precision_compare"] = precision_compare(args, est, d, stream, Bf.clone(), ph32[1], edges)
        ref.close()
        del ref
    # cuFFT as a timed comparison only (never on the path): a full, unpruned
    # C2R transform of one n^3 field beside this library's per-field filter +
    # pruned inverse FFT + 16-bit split
    line["cufft_compare"] = cufft_compare(d, args.n, fft_ms / (3 * args.shells), stream)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        info = cpu_sample(dk, args.n, edges)
        step_s = info["t_full"] + 3 * args.shells * info["t_field"] + outputs * info["t_bin"]
        line["cpu_baseline"] = {"value": outputs / step_s, "unit": "bins/s", "cores": info["cores"],
                                "kind": "oracle", "sample": info["sample"], "measured_s": info["measured_s"],
                                "value_is_extrapolated": True}
    line["fp32_peak"] = {"tflops": fp32_peak, "ms": fp32_peak_ms,
                         "how": "bsp_fp32_fma_peak: 1024 threads per SM, 8 FMA chains each, CUDA events"}
    est.close()
    del est, d
    torch.cuda.empty_cache()
    if not args.no_modal and world == 1:
        try:
            line["modal"] = modal_bench(args, stream)
        except Exception as e:   # reported, not fatal: the headline line still prints
            line["modal"] = {"error": "%s: %s" % (type(e).__name__, str(e)[:300])}
        torch.cuda.empty_cache()
    if not args.no_batch and world == 1:
        try:
            line["batch"] = batch_bench(args, stream)
        except Exception as e:
            line["batch"] = {"error": "%s: %s" % (type(e).__name__, str(e)[:300])}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


GOLDEN = os.path.join(ROOT, "tests", "golden", "fullsize_512_64shells.json")


def golden_gate(bins, B, n, shells, width):
    """Gate error |dB| / max(|B|, rms_l) of B [3][n_bins] on the bins of the
    committed FP64-oracle sample (tests/golden), where it covers this
    workload; rms_l is taken over all bins of B.  None if not applicable."""
    try:
        g = json.load(open(GOLDEN))
    except Exception:
        return None
    from paper_1708_05303_gb300.synth import linear_edges

    if g["n"] != n or g["seed"] != SEED or list(g["edges"]) != list(linear_edges(shells, width)):
        return None
    import numpy as np

    V, n3 = BOX ** 3, float(n) ** 3
    idx = {tuple(int(v) for v in t): i for i, t in enumerate(bins)}
    rms = np.sqrt(np.mean(B ** 2, axis=1))
    worst = 0.0
    for j, t in enumerate(g["bins"]):
        i = idx[tuple(t)]
        for li in range(3):
            Bo = g["T"][li][j] / (V * n3 * g["counts"][j])
            worst = max(worst, abs(B[li, i] - Bo) / max(abs(Bo), rms[li]))
    return {"gate_vs_oracle": worst, "oracle_bins": len(g["bins"])}


def precision_compare(args, est, d, stream, B_fp32, con_fp32_ms, edges):
    """split-BF16 and plain BF16 contractions on the same input, counts and
    workspace as the benchmarked plan: contraction time, speedup over the
    plain FP32 CUDA-core path, error against the FP64 oracle's sample, and
    the largest departure from FP32 over every output."""
    import torch
    from paper_1708_05303_gb300 import bsp

    out = {}
    rms = torch.sqrt(torch.mean(B_fp32 * B_fp32, dim=1, keepdim=True))
    for prec in ("split_f16", "split_bf16", "bf16"):
        if prec == args.prec:
            p, own = est, False
        else:
            p, own = bsp.Bispectrum(args.n, BOX, edges, (0, 2, 4), prec=prec, counts_from=est, ws=est.ws), True
        p.compute(d)
        torch.cuda.synchronize()
        bsp.bsp_set_profiling(p.plan, True)
        for _ in range(2):
            p.compute(d)
        torch.cuda.synchronize()
        ph, nc, _ = bsp.bsp_phase_times(p.plan)
        bsp.bsp_set_profiling(p.plan, False)
        B = p.compute(d)
        dev = torch.max(torch.abs(B - B_fp32) / torch.maximum(torch.abs(B_fp32), rms)).item()
        ent = {"contraction_ms": ph[1] / max(nc, 1), "step_ms": sum(ph) / max(nc, 1),
               "speedup_contraction_vs_fp32": con_fp32_ms / (ph[1] / max(nc, 1)) if con_fp32_ms else None,
               "max_rel_dev_vs_fp32": dev, "gated": prec == "split_f16"}
        gg = golden_gate(p.bins, B.cpu().numpy(), args.n, args.shells, args.width)
        if gg:
            ent.update(gg)
        out[prec] = ent
        if own:
            p.close()
    return out


def modal_bench(args, stream, reps=2):
    """The modal estimator's workload (Sec. 3.5): 512^3, 50 shifted-Legendre
    modes on [k_f, 0.3 h/Mpc] over sqrt(k P(k)), l = 0, 2, 4, 22 100 raw
    projections per l, on the benchmarked precision."""
    import torch
    from paper_1708_05303_gb300 import bsp
    from paper_1708_05303_gb300.synth import FieldModel, make_field

    n, nm, kmax = args.n, 50, 0.3
    kf = 2 * math.pi / BOX
    model = FieldModel(n=n, box=BOX, sigma_g=0.3)
    dk, amp = make_field(model, 1708 + 3)
    R = bsp.bsp_modal_radial_powerlaw(n, BOX, nm, kf, kmax, amp, model.n_s, True)
    d = torch.from_numpy(dk).cuda()
    m = bsp.Modal(n, BOX, R, (0, 2, 4), prec=args.prec)
    m.compute(d)
    torch.cuda.synchronize()
    bsp.bsp_set_profiling(m.plan, True)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(reps):
        m.compute(d)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / reps
    ph, nc, nl = bsp.bsp_phase_times(m.plan)
    bsp.bsp_set_profiling(m.plan, False)
    ph = [v / max(nc, 1) for v in ph]
    st = bsp.bsp_plan_stats(m.plan) if hasattr(bsp, "bsp_plan_stats") else {}
    status = bsp.bsp_device_status(m.plan)
    m.close()
    ntrip = nm * (nm + 1) * (nm + 2) // 6
    # sums the plan computes: T^l(a; b >= c) for every a and l, and U(a; b >= c) for l = 4
    sums = 3 * nm * nm * (nm + 1) // 2 + nm * nm * (nm + 1) // 2
    flop = 2.0 * float(n) ** 3 * sums
    peak = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))).get("bf16_tflops_sustained", 1700.0) \
        if os.path.exists(os.path.join(ROOT, "MEASURED_PEAKS.json")) else 1700.0
    ach = flop / (ph[1] / 1e3) / 1e12
    return {"ms": ms, "phases_ms": {"filter_fft": ph[0], "contraction": ph[1], "assemble": ph[2]},
            "modes_1d": nm, "triplets_per_l": ntrip, "projections_per_s": 3 * ntrip / (ms / 1e3),
            "fields": 3 * nm, "contraction_sums": sums, "device_status": status,
            "roofline": {"bound": "tensor", "achieved": ach, "peak": peak, "unit": "TFLOP/s", "frac": ach / peak,
                         "algorithmic": "2 n^3 flop per sum, T^l(a; b >= c) for all a and l plus U: %.3e flop"
                                        % flop}}


def _mock_input(m):
    """Half spectrum of mock m of the uneven-grid ensemble (inputs only)."""
    from paper_1708_05303_gb300.synth import make_field, mock_model

    model, seed = mock_model(m, BATCH_SIZES)
    dk, _ = make_field(model, seed)
    return BATCH_SIZES.index(model.n), dk


BATCH_SIZES = (96, 128, 160)


def batch_bench(args, stream):
    """512 mocks of 96^3, 128^3 and 160^3 grids (own n_s, f per mock), 24
    shells of width k_f, l = 0, 2, 4 (a 4962-vector per mock) through the
    batch runner: CUDA graphs per size, autotuned schedule, H2D copies of the
    next mock overlapped with the current one; then the FP64 covariance.
    Timed on the FP32 path (the one that meets 1e-5 on these fields) and on
    the split-FP16 tensor-core path beside it."""
    import multiprocessing as mp

    import torch
    from paper_1708_05303_gb300 import bsp
    from paper_1708_05303_gb300.synth import linear_edges

    edges = linear_edges(24, 1.0)
    nm = args.batch_mocks
    t0 = time.perf_counter()
    ctx = mp.get_context("spawn")
    with ctx.Pool(min(16, os.cpu_count() or 4)) as pool:
        inputs = pool.map(_mock_input, range(nm), chunksize=4)
    t_gen = time.perf_counter() - t0
    counts_s = {}
    for n in BATCH_SIZES:
        t0 = time.perf_counter()
        e = bsp.Bispectrum(n, BOX, edges, (0, 2, 4), prec="fp32")
        torch.cuda.synchronize()
        counts_s[str(n)] = round(time.perf_counter() - t0, 3)
        e.close()
        del e
    hosts = [torch.from_numpy(dk).pin_memory() for _, dk in inputs]
    idx = [si for si, _ in inputs]
    out = {"mocks": nm, "sizes": list(BATCH_SIZES), "shells": 24, "counts_s": counts_s,
           "input_generation_s": round(t_gen, 1)}
    for prec in ("fp32", "split_f16"):
        t0 = time.perf_counter()
        batch = bsp.Batch(BATCH_SIZES, BOX, edges, (0, 2, 4), prec=prec, autotune=True)
        t_prep = time.perf_counter() - t0
        batch.run(hosts[:6], idx[:6])
        torch.cuda.synchronize()
        rows = torch.empty((nm, 3 * batch.nbins), dtype=torch.float64, device="cuda")
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        batch.run(hosts, idx, rows=rows)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        c0, c1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        c0.record(stream)
        mean, cov = batch.covariance(rows)
        c1.record(stream)
        torch.cuda.synchronize()
        ent = {"ms": ms, "mocks_per_s": nm / (ms / 1e3), "per_size_graph_ms": batch.tuning["ms"],
               "tuning": batch.tuning, "prepare_s": round(t_prep, 3), "covariance_ms": c0.elapsed_time(c1),
               "covariance_finite": bool(torch.isfinite(cov).all().item())}
        out["bins"], out["vector"] = batch.nbins, 3 * batch.nbins
        if prec == "fp32":
            out.update(ent)
            out["precision"] = "fp32"
        else:
            out["split_f16"] = ent
        batch.close()
        del rows, mean, cov
    return out


def cufft_compare(delta_k, n, ours_ms_per_field, stream=None, reps=10):
    """Time torch.fft.irfftn (cuFFT) on the n^3 half spectrum: the full
    complex-to-real transform of one field, no filter and no pruning.  Any
    failure is reported in the result instead of raised."""
    import torch

    try:
        dev = delta_k.device
        out = None
        for _ in range(3):
            out = torch.fft.irfftn(delta_k, s=(n, n, n), dim=(0, 1, 2))
        if dev.type != "cuda":
            return {"error": "no CUDA device"}
        st = stream if stream is not None else torch.cuda.current_stream()
        with torch.cuda.stream(st):
            torch.cuda.synchronize()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(st)
            for _ in range(reps):
                out = torch.fft.irfftn(delta_k, s=(n, n, n), dim=(0, 1, 2))
            b.record(st)
            torch.cuda.synchronize()
        ms = a.elapsed_time(b) / reps
        del out
        return {"cufft_ms_per_field": ms, "ours_ms_per_field": ours_ms_per_field,
                "what": "cuFFT (torch.fft.irfftn): full unpruned C2R of one %d^3 field, FP32; ours: shell/Legendre "
                        "filter + pruned C2R + hi/lo split of one field (filter_fft phase / fields per step)" % n}
    except Exception as e:   # a comparison only: never fail the run for it
        return {"error": "%s: %s" % (type(e).__name__, str(e)[:200])}


def fft_alg_bytes(n, edges):
    """Algorithmic HBM bytes of the filter + inverse FFT phase per step: per
    field, the nonzero input modes it reads (complex64), the pruned
    intermediates written and read once (complex64), and the real output."""
    K = 0
    emax = edges[-1]
    while (K + 1) ** 2 < emax ** 2:
        K += 1
    nK = min(n, 2 * K + 1)
    nKz = min(n // 2 + 1, K + 1)
    nf = 3 * (len(edges) - 1)
    per = 8 * (nK * nK * nKz) + 2 * 8 * (nK * n * nKz) + 2 * 8 * (n * n * nKz) + 4 * n ** 3
    return float(nf * per)


def raw_fft_bytes(n):
    """HBM bytes of the unpruned inverse real FFT of delta (all modes but the
    mean): the half spectrum read, the two complex64 intermediates written and
    read once, the FP32 field written."""
    h = 8 * n * n * (n // 2 + 1)
    return float(5 * h + 4 * n ** 3)


def power_read_bytes(n, edges, m=1):
    """Complex64 modes the shell sums read: the box |f| <= K of each of the
    m^3 spectra of side n/m (K from the top edge, in units of the box's k_f)."""
    s = n // m
    K = 0
    while (K + 1) ** 2 * m * m < edges[-1] ** 2:
        K += 1
    nK, nKz = min(s, 2 * K + 1), min(s // 2 + 1, K + 1)
    return float(8 * m ** 3 * nK * nK * nKz)


def skew_alg_bytes(n, edges):
    """Skew spectrum: inverse FFT, the forward FFT of the square (field read,
    spectrum written, then read and written by each of two passes), the cross
    sums reading delta and Q."""
    h = 8 * n * n * (n // 2 + 1)
    return raw_fft_bytes(n) + 4 * n ** 3 + 5 * h + 2 * power_read_bytes(n, edges)


def ib_alg_bytes(n, edges, m):
    """Integrated bispectrum: inverse FFT, the sub-cube forward FFTs (field
    read, m^3 spectra written, then read and written by each of two passes),
    the weighted sums reading the sub-cube spectra."""
    s = n // m
    hs = 8 * m ** 3 * s * s * (s // 2 + 1)
    return raw_fft_bytes(n) + 4 * n ** 3 + 5 * hs + power_read_bytes(n, edges, m)


if __name__ == "__main__":
    sys.exit(main())
