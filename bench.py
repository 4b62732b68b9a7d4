#!/usr/bin/env python3
"""Benchmark of the adaptive-precision EAM/ACE molecular-dynamics step on GB300.

Workload: the nanoindentation-shaped slab of 100x100x100 FCC cells (4,000,000
copper-like atoms, x/y periodic, bottom 3 layers fixed, spherical indenter),
parameter set Hyb2, lambda and the precise-atom queue updated every 10 MD steps,
mixed precision (FP32 potentials, FP64 integration and energy sums).

One bench step = one lambda period = 10 velocity-Verlet steps through ap_step
(neighbour rebuild, classification, EAM for all atoms, ACE for the precise queue,
indenter, integration).  Metric: atom-steps/s = N_atoms x MD steps / time.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

Under torchrun each rank runs an independent replica (the path has no exchange
step on one GPU per system); value = atoms x steps over all ranks / max time.
"""
from __future__ import annotations

import argparse
import dataclasses
import json
import math
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import ap_inputs as I  # noqa: E402

MD_PER_STEP = 10
METRIC = "atom-steps/s adaptive vs full-ACE on 1 GB300 at <=10 meV/A force error"
# The step's three largest kernels are instrumented (CUDA events around each launch);
# `roofline` describes the one with the most measured time, `rooflines` all three.
#
# Algorithmic FLOPs of the ACE force stage k_ace_adjoint, per neighbour pair within r_c
# and per precise atom (FMA = 2): per pair the radial functions and derivatives (~100),
# the solid harmonics and gradients for l <= 4 (~400), the two 8-term contractions and
# the accumulations for 25 (l, m) (~1040) and the scatter (~40); per atom
# u = W^T dE/dA / N0 (~3300).
ADJ_FLOP_PER_PAIR = 1580
ADJ_FLOP_PER_ATOM = 3300
# Algorithmic FLOPs of k_ace_basis: per pair g (~30), Y (~70), the normalisation (~10)
# and the G = g^T Y accumulation over 8 x 25 (l, m, k) (400); per atom A = W G (3200)
# and the nu = 1, 2 energy and gradient (~3800).
BASIS_FLOP_PER_PAIR = 510
BASIS_FLOP_PER_ATOM = 7000
# The whole ACE evaluation (k_ace_basis + k_ace_nu3 + k_ace_adjoint): per atom add the
# nu = 3 monomials (~11400).
ACE_FLOP_PER_PAIR = ADJ_FLOP_PER_PAIR + BASIS_FLOP_PER_PAIR
ACE_FLOP_PER_ATOM = ADJ_FLOP_PER_ATOM + BASIS_FLOP_PER_ATOM + 11400
# DRAM bytes (read + write) per launch on this workload, from an ncu capture of the
# current kernels on the 500k-atom case (60,000 precise atoms), scaled to 4,000,000 atoms
# and 240,000 precise atoms (profiles/dram_traffic_slab50_mixed.md):
#   k_ace_basis    45.2 MB read + 120.4 MB written (the pair records, 16 B per pair);
#   k_ace_adjoint  185.6 MB read (mostly the basis kernel's pair records) + 2.4 MB written;
#   k_eam_force    146.0 MB read + 8.2 MB written.
ADJ_TRAFFIC_BYTES = 188.0e6 * 240000 / 60000
BASIS_TRAFFIC_BYTES = 165.6e6 * 240000 / 60000
EAM_FORCE_TRAFFIC_BYTES = 154.2e6 * 4000000 / 500000
# FP32 SIMT peak from unit counts: SMs (read from the device) x 128 FP32 lanes x 2 flop x the
# maximum SM clock; reported for context beside the measured FFMA peak (ap_probe_peak), which
# is the denominator of the ALU rooflines.
FP32_LANES_PER_SM = 128
SM_MAX_GHZ = 2.07
MMA_TILE_FLOP = 2 * 16 * 8 * 8       # one m16n8k8 tensor-core tile
# Algorithmic bytes of one k_eam_force launch: the row entries it walks (4 B each; per
# atom the prefix up to the last entry inside r_c) plus, per atom, its own shadow,
# (lambda xi', lambda), xi and prefix length (16 + 8 + 8 + 4 B), its force and E^f
# (24 + 8 B), and one read of its shadow and q as some other atom's neighbour (24 B):
# 4 E_walked + 92 n.  The ncu traffic above matches it: no DRAM byte is read twice.
EAM_FORCE_BYTES_PER_ENTRY = 4
EAM_FORCE_BYTES_PER_ATOM = 92


def measured_peaks(dev_index: int):
    """FP32 FFMA and warp-level TF32 MMA peaks of this GPU, measured now by the library's
    probe (best of 5 timed runs, SM clock read during the probe), and the derived FP32 figure."""
    import torch
    import paper_2411_03002_gb300 as ap
    sms = torch.cuda.get_device_properties(dev_index).multi_processor_count
    ffma, mhz_f = ap.probe_peak(ap.PEAK_FFMA)
    tf32, mhz_t = ap.probe_peak(ap.PEAK_TF32_MMA)
    return {"fp32_tflops": ffma, "fp32_sm_mhz": mhz_f, "tf32_mma_tflops": tf32, "tf32_sm_mhz": mhz_t, "sms": sms,
            "fp32_derived_tflops": sms * FP32_LANES_PER_SM * 2 * SM_MAX_GHZ * 1e9 / 1e12,
            "source": "measured by ap_probe_peak on this GPU before the timed region (FFMA chains; mma.sync "
                      "m16n8k8 TF32 tiles)"}


def kernel_rooflines(ctx, prof, n, hbm_gbs, hbm_src, peaks):
    """Roofline objects of the instrumented kernels from the step's own CUDA-event timers."""
    ph = prof["phases"]
    pairs, atoms = prof["ace_pairs"], prof["ace_atoms"]
    fp32 = peaks["fp32_tflops"]
    alu_src = ("measured FFMA peak (ap_probe_peak, %d SMs at %.0f MHz; %.1f TFLOP/s derived from unit counts at "
               "2.07 GHz)" % (peaks["sms"], peaks["fp32_sm_mhz"], peaks["fp32_derived_tflops"]))
    out = {}
    for name, key, fpp, fpa, traffic in (("k_ace_basis", "ace_basis", BASIS_FLOP_PER_PAIR, BASIS_FLOP_PER_ATOM,
                                          BASIS_TRAFFIC_BYTES),
                                         ("k_ace_adjoint", "ace_adjoint", ADJ_FLOP_PER_PAIR, ADJ_FLOP_PER_ATOM,
                                          ADJ_TRAFFIC_BYTES)):
        ms, calls = ph[key]
        tf = (fpp * pairs + fpa * atoms) / (ms / 1e3) / 1e12 if ms > 0 else 0.0
        out[name] = {"bound": "alu", "achieved": tf, "peak": fp32, "unit": "TFLOP/s",
                     "frac": tf / fp32, "traffic": traffic, "peak_source": alu_src,
                     "ms_per_launch": ms / max(1, calls), "ms_total": ms, "launches": calls,
                     "pairs_per_launch": pairs / max(1, calls), "atoms_per_launch": atoms / max(1, calls)}
    ms, calls = ph["ace_basis"]
    if ms > 0 and prof.get("ace_mma", 0) > 0:      # tensor-pipe use of the basis kernel
        tcf = MMA_TILE_FLOP * prof["ace_mma"]
        out["k_ace_basis"]["tensor"] = {
            "mma_tiles_per_launch": prof["ace_mma"] / max(1, calls), "achieved": tcf / (ms / 1e3) / 1e12,
            "peak": peaks["tf32_mma_tflops"], "unit": "TFLOP/s",
            "frac": tcf / (ms / 1e3) / 1e12 / peaks["tf32_mma_tflops"],
            "peak_source": "measured mma.sync m16n8k8 TF32 rate (ap_probe_peak)",
            "note": "issued MMA flops incl. the 3xTF32 split and padding of 25 (l, m) rows to 32"}
    ms, calls = ph["eam_force"]
    walked = ctx.neighbor_total(2)            # row entries the last force pass walked
    b = EAM_FORCE_BYTES_PER_ENTRY * walked + EAM_FORCE_BYTES_PER_ATOM * n
    gbs = b / (ms / max(1, calls) / 1e3) / 1e9 if ms > 0 else 0.0
    out["k_eam_force"] = {"bound": "hbm", "achieved": gbs, "peak": hbm_gbs, "unit": "GB/s", "frac": gbs / hbm_gbs,
                          "traffic": EAM_FORCE_TRAFFIC_BYTES, "peak_source": hbm_src,
                          "algorithmic_bytes_per_launch": b, "row_entries_walked": walked,
                          "row_entries_total": ctx.neighbor_total(0), "ms_per_launch": ms / max(1, calls),
                          "ms_total": ms, "launches": calls}
    return out


def curve_at(points, kx, x, ky):
    """ky at kx = x, interpolated linearly along the points ordered by precise fraction (the
    first crossing); None when x lies outside the range the points cover."""
    pts = sorted(points, key=lambda p: p["precise_fraction"])
    for a, b in zip(pts, pts[1:]):
        if (a[kx] - x) * (b[kx] - x) <= 0 and a[kx] != b[kx]:
            t = (x - a[kx]) / (b[kx] - a[kx])
            return a[ky] + t * (b[ky] - a[ky])
    return None


def dominant_kernel(rooflines):
    """The instrumented kernel with the most measured time in the timed region."""
    return max(rooflines, key=lambda k: rooflines[k]["ms_total"])


def hbm_peak():
    """(GB/s, source) from MEASURED_PEAKS.json, else the profiling recipe's fallback."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return float(json.load(fh)["hbm_gbs"]), "measured (MEASURED_PEAKS.json hbm_gbs)"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback (6.8 TB/s)"


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=5)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--ncell", type=int, default=100)
    p.add_argument("--mode", default="adaptive", choices=["adaptive", "full-ace", "full-eam"])
    p.add_argument("--precision", default="mixed", choices=["mixed", "fp64"])
    p.add_argument("--no-extras", action="store_true", help="skip full-ACE/full-EAM, error and CPU baseline legs")
    p.add_argument("--skin", type=float, default=0.7, help="neighbour-list skin (A)")
    p.add_argument("--rebuild", default="skin", choices=["lambda", "skin"],
                   help="list rebuilds in the timed run: at every lambda update, or on the skin criterion "
                        "(checked after every drift; a lambda update keeps the lists while no atom has moved "
                        "more than 0.45 skin)")
    p.add_argument("--thermostat", action="store_true", help="local thermostat (Appendix C) in the timed run")
    p.add_argument("--deterministic", action="store_true",
                   help="fixed-point ACE force reduction (bitwise reproducible) in the timed run")
    p.add_argument("--detector", default="csp", choices=["csp", "selector"],
                   help="detector behind lambda_0 in the timed run (centro-symmetry or the stored selector)")
    return p.parse_args()


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def max_over_ranks(ms: float, ws: int, device) -> float:
    """The whole job's time for N independent replicas: the slowest rank's (ms)."""
    if ws <= 1:
        return ms
    import torch
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return float(t.item())


def job_rate(units_per_rank: float, ws: int, ms: float) -> float:
    """Whole-job throughput: the units every rank processed over the slowest rank's time."""
    return units_per_rank * ws / (ms / 1e3)


def hyb_for(mode: str, hyb: I.HybridParams) -> I.HybridParams:
    import dataclasses
    if mode == "full-ace":       # every changeable atom detected: lambda = 0
        return dataclasses.replace(hyb, csp_lo=-2.0, csp_hi=-1.0)
    if mode == "full-eam":       # no atom detected: lambda = 1
        return dataclasses.replace(hyb, csp_lo=1e30, csp_hi=2e30)
    return hyb


# ----------------------------------------------------------------------------- clocks
class Clocks:
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, device: int):
        self.device = device
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                                          "-lms", "200", "-i", str(self.device)], stdout=subprocess.PIPE,
                                         stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        out, _ = self.proc.communicate(timeout=10)
        sm, mx, reasons = [], [], set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for line in out.strip().splitlines():
            f = [t.strip() for t in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for k, nm in enumerate(names):
                if f[5 + k].lower().startswith("active"):
                    reasons.add(nm)
        loaded = [s for s in sm if s > 0.5 * max(mx)] if mx else []
        return {"sm_mhz": statistics.median(loaded) if loaded else (statistics.median(sm) if sm else None),
                "sm_max_mhz": max(mx) if mx else None, "reasons": sorted(reasons), "samples": len(sm)}


# ----------------------------------------------------------------------------- oracle baseline
def oracle_sample(hyb: I.HybridParams, reps: int = 1):
    """Time the oracle on a bounded sample of the workload: a laterally periodic
    6x6x100-cell column (14,400 atoms) of the same slab, one MD step's force work
    (classification + hybrid EAM/ACE forces + indenter) per repetition."""
    import oracle as O
    w = I.config_c5(100, hyb=hyb, nxy=6)
    ch = (w.fixed == 0).astype(np.uint8)
    eam, ace = I.eam_params(0), O.ACE(I.ace_for_config(5))
    times = []
    for _ in range(reps):
        st = O.LambdaState(w.n, hyb.n_csp_avg, hyb.n_lam_avg)
        t0 = time.perf_counter()
        lam, *_ = O.classify(st, w.x, w.box, hyb, changeable=ch)
        e, f, _, _ = O.hybrid(w.x, w.box, lam, eam, ace)
        O.indenter(w.x, w.indenter.center0, w.indenter.radius, w.indenter.k)
        times.append(time.perf_counter() - t0)
    return w.n, times, O.num_threads()


def reference_arm(args, ws, rank):
    if rank != 0:
        return
    hyb = hyb_for(args.mode, I.HYB2)
    n, times, cores = oracle_sample(hyb, reps=args.warmup + args.steps)
    timed = times[args.warmup:]
    v = n * len(timed) / sum(timed)
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "atom-steps/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * sum(timed) / len(timed),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": "6x6x100-cell column (14,400 atoms) of the 100^3-cell nanoindentation slab, "
                                   "Hyb2, one MD step of force work per step (FP64 CPU oracle)"},
            "cpu_baseline": {"value": v, "unit": "atom-steps/s", "cores": cores, "kind": "oracle",
                             "sample": "14,400-atom column, classification + hybrid forces + indenter"},
            "e2e": {"value": v, "unit": "atom-steps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ----------------------------------------------------------------------------- GPU arm
def c2_record(dev, nsteps: int = 200):
    """The 32,000-atom adaptive-MD slab (20^3 FCC cells, x/y periodic, a 0.3 A-disordered
    hemisphere of 15 A under the top surface, Hyb1, lambda every 10 steps, lists rebuilt every
    5 steps) for 200 MD steps of 1 fs from 300 K, in FP64 and in mixed precision from the same
    start: rates, total-energy drift and the largest difference between the two precisions'
    final forces and positions.  The oracle comparison of the same runs' final forces is a test
    (tests/test_gpu_md.py)."""
    import torch
    import paper_2411_03002_gb300 as ap
    w = I.config_c2()
    out = {"workload": "FCC slab 20^3 cells (32,000 atoms), x/y periodic, 0.3 A-disordered 15 A hemisphere, "
                       "Hyb1, lambda every 10 steps, %d MD steps of 1 fs from 300 K" % nsteps}
    final = {}
    for pname, p in (("fp64", ap.PREC_FP64), ("mixed", ap.PREC_MIXED)):
        cfg = ap.make_config(I.eam_params(0), I.ace_for_config(2), w.hyb, precision=p, dt=w.dt, lambda_every=10,
                             rebuild_every=5)
        c = ap.Context(cfg)
        x, v = torch.as_tensor(w.x, device=dev).clone(), torch.as_tensor(w.v, device=dev).clone()
        f = torch.zeros_like(x)
        lam = torch.empty(w.n, dtype=torch.float64, device=dev)
        m = torch.as_tensor(w.mass, device=dev)
        c.build_neighbors(x, w.box)
        s0 = c.step(x, v, f, m, None, lam, 0)
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(torch.cuda.current_stream())
        s1 = c.step(x, v, f, m, None, lam, nsteps)
        b.record(torch.cuda.current_stream())
        torch.cuda.synchronize()
        t = a.elapsed_time(b)
        out[pname] = {"atom_steps_s": w.n * nsteps / (t / 1e3), "precise_fraction": s1.n_precise / w.n,
                      "drift_eV_per_atom": (s1.e_pot + s1.e_kin - s0.e_pot - s0.e_kin) / w.n}
        final[pname] = (x.clone(), f.clone())
        c.close()
        del c
    (x64, f64), (x32, f32) = final["fp64"], final["mixed"]
    out["mixed_vs_fp64"] = {
        "force_max_meV_A": float(torch.linalg.vector_norm(f32 - f64, dim=1).max().item() * 1e3),
        "force_rms_meV_A": float(torch.sqrt(((f32 - f64) ** 2).mean()).item() * 1e3),
        "position_p99_A": float(torch.quantile(torch.linalg.vector_norm(x32 - x64, dim=1), 0.99).item())}
    return out


def run_ours(args, ws, rank, local):
    import torch
    import paper_2411_03002_gb300 as ap
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    prec = ap.PREC_MIXED if args.precision == "mixed" else ap.PREC_FP64
    w = I.config_c5(args.ncell, hyb=I.HYB2)
    hyb = hyb_for(args.mode, w.hyb)
    eam, acep = I.eam_params(0), I.ace_for_config(5)

    sel = np.load(os.path.join(ROOT, "paper_2411_03002_gb300", "selector_cu.npz"))

    def new_ctx(h, p=prec, detector=ap.DETECT_CSP, thermostat=False, p_lo=None, p_hi=None, deterministic=False,
                rebuild=None):
        rebuild = args.rebuild if rebuild is None else rebuild
        c = ap.Context(ap.make_config(eam, acep, h, precision=p, indenter=w.indenter, lambda_every=MD_PER_STEP,
                                      dt=w.dt, skin=args.skin, detector=detector,
                                      rebuild_every=ap.REBUILD_SKIN if rebuild == "skin" else 0,
                                      sel_p_lo=float(sel["p_lo"]) if p_lo is None else p_lo,
                                      sel_p_hi=float(sel["p_hi"]) if p_hi is None else p_hi,
                                      thermostat=thermostat or args.thermostat,
                                      deterministic=deterministic or args.deterministic))
        if detector == ap.DETECT_SELECTOR:
            c.sel_set_model(sel["params"], sel["mu"], sel["inv_sigma"])
        return c

    def tensors():
        return (torch.as_tensor(w.x, device=dev).clone(), torch.as_tensor(w.v, device=dev).clone(),
                torch.zeros((w.n, 3), dtype=torch.float64, device=dev), torch.as_tensor(w.mass, device=dev),
                torch.as_tensor(w.fixed, device=dev), torch.empty(w.n, dtype=torch.float64, device=dev))

    def barrier():
        torch.cuda.synchronize()
        if ws > 1:
            torch.distributed.barrier()
            torch.cuda.synchronize()

    peaks = measured_peaks(local)
    free0 = torch.cuda.mem_get_info(local)[0]
    ctx = new_ctx(hyb, detector=ap.DETECT_SELECTOR if args.detector == "selector" else ap.DETECT_CSP)
    x, v, f, mass, fixed, lam = tensors()
    ctx.build_neighbors(x, w.box)
    stats = ctx.step(x, v, f, mass, fixed, lam, 0)
    for _ in range(args.warmup):
        stats = ctx.step(x, v, f, mass, fixed, lam, MD_PER_STEP)
    stats_start = stats
    footprint_gb = (free0 - torch.cuda.mem_get_info(local)[0]) / 1e9   # library scratch + the run's own state
    barrier()
    ctx.profile_enable(True)
    clocks = Clocks(local)
    clocks.start()
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        stats = ctx.step(x, v, f, mass, fixed, lam, MD_PER_STEP)
    e1.record(stream)
    barrier()
    ck = clocks.stop()
    ms = e0.elapsed_time(e1)
    prof = ctx.profile_read()
    ms = max_over_ranks(ms, ws, dev)
    atom_steps = w.n * MD_PER_STEP * args.steps * ws
    value = job_rate(w.n * MD_PER_STEP * args.steps, ws, ms)
    ace_ms, ace_calls = prof["phases"]["ace"]
    flops = ACE_FLOP_PER_PAIR * prof["ace_pairs"] + ACE_FLOP_PER_ATOM * prof["ace_atoms"]
    hbm_gbs, hbm_src = hbm_peak()
    rooflines = kernel_rooflines(ctx, prof, w.n, hbm_gbs, hbm_src, peaks)
    dominant = dominant_kernel(rooflines)
    sub = ("ace_adjoint", "eam_force", "ace_basis")
    top = {k: v for k, v in prof["phases"].items() if k not in sub}   # the sub-phases are inside ace / eam
    phase_share = {k: round(m / max(1e-9, sum(p[0] for p in top.values())), 4) for k, (m, c) in top.items()}

    # end-to-end through the public call with host buffers (pinned), copies inside the timed region
    xh, vh, fh = x.cpu().pin_memory(), v.cpu().pin_memory(), f.cpu().pin_memory()
    lamh = lam.cpu().pin_memory()
    barrier()
    e2, e3 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e2.record(stream)
    for _ in range(args.steps):
        x.copy_(xh, non_blocking=True)
        v.copy_(vh, non_blocking=True)
        f.copy_(fh, non_blocking=True)
        ctx.step(x, v, f, mass, fixed, lam, MD_PER_STEP)
        xh.copy_(x, non_blocking=True)
        vh.copy_(v, non_blocking=True)
        fh.copy_(f, non_blocking=True)
        lamh.copy_(lam, non_blocking=True)
    e3.record(stream)
    barrier()
    ms_e2e = max_over_ranks(e2.elapsed_time(e3), ws, dev)
    h2d = 3 * w.n * 3 * 8
    d2h = 3 * w.n * 3 * 8 + w.n * 8

    drift = (stats.e_pot + stats.e_kin - stats_start.e_pot - stats_start.e_kin) / w.n

    def timed_mode(make, steps):
        """One mode of the comparison on the same workload and GPU: a fresh context, one
        warm-up bench step, then `steps` timed bench steps with their own clock record."""
        c = make()
        x2, v2, f2, m2, fx2, l2 = tensors()
        c.build_neighbors(x2, w.box)
        c.step(x2, v2, f2, m2, fx2, l2, 0)
        s0 = c.step(x2, v2, f2, m2, fx2, l2, MD_PER_STEP)
        torch.cuda.synchronize()
        ck2 = Clocks(local)
        ck2.start()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(steps):
            s1 = c.step(x2, v2, f2, m2, fx2, l2, MD_PER_STEP)
        b.record(stream)
        torch.cuda.synchronize()
        clk = ck2.stop()
        t = a.elapsed_time(b)
        out = {"atom_steps_s": w.n * MD_PER_STEP * steps / (t / 1e3), "ms_per_step": t / steps, "steps": steps,
               "precise_fraction": s1.n_precise / w.n, "rebuilds": s1.rebuilds - s0.rebuilds,
               "kept_updates": s1.kept - s0.kept,
               "drift_eV_per_atom": (s1.e_pot + s1.e_kin - s0.e_pot - s0.e_kin) / w.n, "clocks": clk}
        if s1.th_corrected or s1.th_refused:
            out["thermostat"] = {"corrections": s1.th_corrected, "refused": s1.th_refused,
                                 "corrected_energy_eV": s1.th_energy}
        c.close()
        del c, x2, v2, f2, m2, fx2, l2
        torch.cuda.empty_cache()
        return out

    def rms_max(d):
        return {"rms_meV_A": float(torch.sqrt((d * d).mean()).item() * 1e3) if d.numel() else None,
                "max_meV_A": float(torch.linalg.vector_norm(d, dim=1).max().item() * 1e3) if d.numel() else None,
                "atoms": int(d.shape[0])}

    extras = {}
    cpu = None
    if rank == 0 and not args.no_extras:
        lam0 = ctx.get_lambda_state()["lam0"]
        detected = lam0 < 1.0
        xs, lams = x.clone(), lam.clone()
        ctx.close()
        del ctx
        torch.cuda.empty_cache()
        # force error against full ACE at the timed run's final positions and lambda, in both
        # precisions: on the detected set (the paper's defect and surface atoms), on {lambda = 0}
        # and on every precise atom; full EAM (lambda = 1 everywhere) on the detected set
        allq = torch.arange(w.n, dtype=torch.int32, device=dev)
        na = torch.tensor([w.n], dtype=torch.int64, device=dev)
        q = torch.nonzero(lams < 1.0).flatten().to(torch.int32)
        nq = torch.tensor([q.numel()], dtype=torch.int64, device=dev)
        z = torch.zeros_like(lams)
        ferr = {}
        for pname, p in (("mixed", ap.PREC_MIXED), ("fp64", ap.PREC_FP64)):
            ev = new_ctx(hyb, p=p)
            ev.build_neighbors(xs, w.box)
            _, fh_ = ev.eval_eam(xs, lams)
            _, fh_ = ev.eval_ace(xs, lams, q, nq, f=fh_)
            _, fa_ = ev.eval_eam(xs, z)
            _, fa_ = ev.eval_ace(xs, z, allq, na, f=fa_)
            _, fe_ = ev.eval_eam(xs, torch.ones_like(lams))
            ferr[pname] = {"adaptive_vs_full_ace": {"detected": rms_max((fh_ - fa_)[detected]),
                                                    "lambda0": rms_max((fh_ - fa_)[lams == 0.0]),
                                                    "precise": rms_max((fh_ - fa_)[lams < 1.0])},
                           "full_eam_vs_full_ace": {"detected": rms_max((fe_ - fa_)[detected])}}
            ev.close()
            if pname == "mixed":
                fh_m, fa_m, fe_m = fh_, fa_, fe_
            del ev, fh_, fa_, fe_
            torch.cuda.empty_cache()
        extras["force_error"] = ferr
        fh_, fa_, fe_ = fh_m, fa_m, fe_m
        mobile = torch.as_tensor(w.fixed, device=dev) == 0
        # scored region: mobile atoms with no fixed (always-EAM) atom inside the ACE cutoff,
        # since no detector can remove the error that the fixed layers contribute
        z_fixed = float(w.x[w.fixed != 0, 2].max()) if (w.fixed != 0).any() else -1e30
        scored = mobile & (torch.as_tensor(w.x[:, 2], device=dev) > z_fixed + float(acep.rc))
        pos = (torch.linalg.vector_norm(fa_ - fe_, dim=1) > float(sel["tau"])) & scored
        dp = (fh_ - fa_)[pos]
        # the same positions classified by the selector instead of CSP, and both detectors over
        # a set of switching zones: precise fraction against the force error on the atoms whose
        # full-ACE and full-EAM forces differ by more than the selector's label threshold
        def detector_point(detector, h, p_lo, p_hi):
            es = new_ctx(h, detector=detector, p_lo=p_lo, p_hi=p_hi)
            es.build_neighbors(xs, w.box)
            lam_s, q_s, n_s = es.classify(xs, mobile.to(torch.uint8))
            _, fs_ = es.eval_eam(xs, lam_s)
            _, fs_ = es.eval_ace(xs, lam_s, q_s, n_s, f=fs_)
            ds = (fs_ - fa_)[pos]
            out = {"r_lo": h.r_lo, "r_hi": h.r_hi, "precise_fraction": float((lam_s < 1.0).float().mean().item()),
                   "force_err_rms_meV_A_label_positive": float(torch.sqrt((ds * ds).mean()).item() * 1e3)}
            es.close()
            del es, fs_
            return out
        pareto = {"csp": [], "selector": []}
        for r_lo, r_hi in ((8.0, 20.0), (6.0, 14.0), (5.0, 12.0), (4.0, 10.0), (4.0, 8.0), (3.0, 6.0)):
            hz = dataclasses.replace(hyb, r_lo=r_lo, r_hi=r_hi)
            pareto["csp"].append(detector_point(ap.DETECT_CSP, hz, 0.0, 0.0))
            pareto["selector"].append(dict(detector_point(ap.DETECT_SELECTOR, hz, 0.9, 0.95), p_lo=0.9, p_hi=0.95))
        deployed = detector_point(ap.DETECT_SELECTOR, hyb, float(sel["p_lo"]), float(sel["p_hi"]))
        csp_ref = pareto["csp"][0]                       # the timed run's detector and zone
        err_key = "force_err_rms_meV_A_label_positive"
        extras["selector"] = {
            "model": "paper_2411_03002_gb300/selector_cu.npz (p_lo %.2f, p_hi %.2f)" % (sel["p_lo"], sel["p_hi"]),
            "label_positive_fraction_of_scored": float((pos.sum() / scored.sum()).item()),
            "precise_fraction": deployed["precise_fraction"],
            "force_err_rms_meV_A_label_positive": deployed["force_err_rms_meV_A_label_positive"],
            "csp_force_err_rms_meV_A_label_positive": float(torch.sqrt((dp * dp).mean()).item() * 1e3),
            "csp_precise_fraction": float((lams < 1.0).float().mean().item()),
            "matched": {"csp_hyb2": csp_ref,
                        "selector_error_at_csp_cost": curve_at(pareto["selector"], "precise_fraction",
                                                               csp_ref["precise_fraction"], err_key),
                        "selector_cost_at_csp_error": curve_at(pareto["selector"], err_key, csp_ref[err_key],
                                                               "precise_fraction"),
                        "csp_error_at_deployed_selector_cost": curve_at(pareto["csp"], "precise_fraction",
                                                                        deployed["precise_fraction"], err_key)},
            "pareto": pareto,
        }
        del fa_, fe_, fh_, fh_m, fa_m, fe_m
        torch.cuda.empty_cache()
        # the comparison of the paper's nanoindentation run: adaptive (mixed, the timed run above;
        # FP64), full ACE and full EAM, plus the selector detector and the local thermostat, on the
        # same GPU and workload, each timed over the same number of bench steps
        modes = {"adaptive_mixed": {"atom_steps_s": value / ws, "ms_per_step": ms / args.steps,
                                    "steps": args.steps, "precise_fraction": stats.n_precise / w.n,
                                    "rebuilds": stats.rebuilds - stats_start.rebuilds,
                                    "kept_updates": stats.kept - stats_start.kept,
                                    "drift_eV_per_atom": drift, "clocks": ck}}
        other_rebuild = "lambda" if args.rebuild == "skin" else "skin"
        for name, make in (("adaptive_fp64", lambda: new_ctx(hyb, p=ap.PREC_FP64)),
                           ("full_ace", lambda: new_ctx(hyb_for("full-ace", w.hyb))),
                           ("full_eam", lambda: new_ctx(hyb_for("full-eam", w.hyb))),
                           ("adaptive_selector", lambda: new_ctx(hyb, detector=ap.DETECT_SELECTOR)),
                           ("adaptive_deterministic", lambda: new_ctx(hyb, deterministic=True)),
                           ("adaptive_rebuild_" + other_rebuild, lambda: new_ctx(hyb, rebuild=other_rebuild)),
                           ("adaptive_thermostat", lambda: new_ctx(hyb, thermostat=True))):
            modes[name] = timed_mode(make, args.steps)
        extras["modes"] = modes
        extras["selector"]["atom_steps_s"] = modes["adaptive_selector"]["atom_steps_s"]
        extras["speedup_vs_full_ace"] = value / ws / modes["full_ace"]["atom_steps_s"]
        extras["c2"] = c2_record(dev)
        if ws == 1:
            n_s, times, cores = oracle_sample(w.hyb, reps=1)
            cpu = {"value": n_s / times[0], "unit": "atom-steps/s", "cores": cores, "kind": "oracle",
                   "sample": "6x6x100-cell column (14,400 atoms) of the same slab, one MD step of force work "
                             "(classification + hybrid forces + indenter), FP64 oracle"}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "atom-steps/s", "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32" if prec == ap.PREC_MIXED else "f64", "data": "synthetic",
            "config": {"workload": f"nanoindentation-shaped FCC slab {args.ncell}^3 cells ({w.n} atoms), Hyb2 "
                                   f"(r_lambda 8/20 A), {args.mode}, {args.precision} precision"
                                   + (", selector detector" if args.detector == "selector" else "")
                                   + (", local thermostat" if args.thermostat else "")
                                   + (", fixed-point ACE forces" if args.deterministic else "")
                                   + (", lists rebuilt on the skin criterion" if args.rebuild == "skin" else ""),
                       "atoms": w.n, "md_steps_per_step": MD_PER_STEP, "lambda_every": MD_PER_STEP,
                       "precision": "FP32 potentials, FP64 integration and energy sums" if prec == ap.PREC_MIXED
                       else "FP64", "l2": "inputs larger than L2 (no flush)",
                       "parallelism": f"replicas x{ws}" if ws > 1 else "1 GPU"},
            "precise_fraction": stats.n_precise / w.n, "n_precise": stats.n_precise, "n_detected": stats.n_detected,
            "memory": {"device_gb": footprint_gb, "what": "device memory taken by the context and the run's x, v, f, "
                                                        "mass, fixed, lambda after warm-up (cudaMemGetInfo)"},
            "drift_eV_per_atom": drift,
            "lists": {"rebuild": args.rebuild, "rebuilds": stats.rebuilds - stats_start.rebuilds,
                      "kept_updates": stats.kept - stats_start.kept, "lambda_updates": args.steps},
            "e2e": {"value": atom_steps / (ms_e2e / 1e3), "unit": "atom-steps/s", "h2d_bytes_per_step": h2d,
                    "d2h_bytes_per_step": d2h},
            "gpu_launches": prof["kernels"],
            "roofline": dict(rooflines[dominant], kernel=dominant + " (the kernel with the most time in the step)"),
            "rooflines": rooflines,
            "peaks": peaks,
            "ace_all_kernels": {"tflops": flops / (ace_ms / 1e3) / 1e12 if ace_ms > 0 else 0.0,
                                "ms_per_call": ace_ms / max(1, ace_calls)},
            "phase_share": phase_share,
            "clocks": ck,
            "cpu_baseline": cpu,
            **extras,
        }
        print(json.dumps(line), flush=True)
    if ws > 1:
        torch.distributed.destroy_process_group()


def main():
    args = parse()
    ws, rank, local = dist_env()
    if args.impl == "reference":
        reference_arm(args, ws, rank)
        return
    run_ours(args, ws, rank, local)


if __name__ == "__main__":
    main()
