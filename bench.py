"""Benchmark: H_eff evaluations per second of the energy-minimising hysteresis
sweep on the 2000 x 1000 x 20 nm film (512 x 256 x 4 cells), one GB300.

A step is one field value of the sweep: set the field, minimise to the stop
rule (max |m x H| / Ms < 1e-5) from the previous state -- the whole device
path: x-FFT with the fused step, y-z convolution, x-inverse with the local
terms and BB sums (its last CTA picks the step size and applies the stop
rule), looped on the device by a CUDA graph.  `value` = effective-field evaluations per second over the K timed
steps (inputs resident in HBM), L2 flushed between steps.  `e2e` is the same
through the C ABI with the magnetisation in pinned host memory (copied in and
out inside every step).  Under torchrun each rank runs an independent replica
(a single minimisation does not shard); value sums the ranks' evaluations over
the slowest rank's time.  By default the line also carries the other
precision (FP32 beside FP64) on the same field values, each with the roofline
of its dominant kernel.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--precision fp64|fp32]
  python bench.py --impl reference   # the CPU oracle on the same workload and metric
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "H_eff evals/s & hysteresis-loop time (512x256x4 film) FP32 vs FP64, %HBM peak"
UNIT = "H_eff evals/s"
PEAKS_FILE = os.path.join(ROOT, "MEASURED_PEAKS.json")
# nominal FMA lanes per SM per clock (the measured rates come from mm_probe_fma)
FP64_FMA_PER_SM_CLK = 2
FP32_FMA_PER_SM_CLK = 128
# the timed steps' field values are far from switching; a whole loop needs more evaluations there
LOOP_NOTE = ("field values x the mean time of the timed steps; the whole loop, timed by --full-loop, takes longer: "
             "near the switching field a value needs thousands of evaluations")
DW_ADD_INSTRUCTIONS = 11      # FP32 instructions of one double-word (float pair) addition
PRECISIONS = {"fp64": 0, "fp32": 1, "f32x2": 2}   # mm.MM_FP64, mm.MM_FP32, mm.MM_F32X2
DTYPE_LABEL = {"fp64": "f64", "fp32": "f32", "f32x2": "f32x2 (double-word) fields, FFT, convolution and local terms"}


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def measured_peaks():
    try:
        with open(PEAKS_FILE) as f:
            return json.load(f)
    except OSError:
        return {}


class ClockSampler:
    """nvidia-smi samples (every 100 ms) of SM clock and throttle reasons during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.idx = gpu_index
        self.proc = None
        self.path = None

    def __enter__(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.idx), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100", "-f", self.path], stdout=subprocess.DEVNULL, stderr=subprocess.DEVNULL)
        except (OSError, ValueError):
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        if not self.path or not os.path.exists(self.path):
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        os.unlink(self.path)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm)}


def algorithmic_model(info, esz):
    """Bytes and flops per launch of each kernel stage as the kernels run them.

    Bytes: compulsory traffic of the pass structure -- xfwd reads m_k and g_k
    and writes m_{k+1} and the x-spectrum; yz reads/writes the spectrum and
    reads the tensor spectra; xinv reads the spectrum, m_{k+1}, m_k and g_k and
    writes g_{k+1} (its last CTA also sums the per-CTA partials and picks tau).  Flops: real arithmetic of the radix-8 Stockham transforms
    with zero-padding pruning, the tensor product and the local terms."""
    nx, ny, nz, Px, Py, Pz = (info[k] for k in ("nx", "ny", "nz", "px", "py", "pz"))
    N = nx * ny * nz
    F = 3 * N * esz
    W = info["spectrum_bytes"]
    T = info["tensor_bytes"]
    Hx = Px // 2
    C = Hx + 1

    def fft_flops(L, half_in, half_out):
        if L <= 1:
            return 0
        lg = L.bit_length() - 1
        passes = []
        if lg % 3 == 1:
            passes.append(2)
        elif lg % 3 == 2:
            passes.append(4)
        passes += [8] * (lg // 3)
        if L < 8:
            passes = [L]
        dft = {2: (4, 0), 4: (16, 8), 8: (56, 40)}
        fl = 0
        ns = 1
        for i, R in enumerate(passes):
            full, pruned = dft[R]
            fl += (L // R) * (pruned if (i == 0 and half_in) else full)
            if ns > 1:
                fl += (L // R) * (R - 1) * 6 * (0.5 if (i == len(passes) - 1 and half_out) else 1)
            ns *= R
        return fl

    x_rows = 3 * ny * nz
    unpack = 10 * C
    f_xfwd = x_rows * (fft_flops(Hx, True, False) + unpack) + N * 3 * 8
    f_xinv = x_rows * (fft_flops(Hx, False, True) + unpack) + N * 90
    model = {
        "xfwd_step": {"bytes": 3 * F + W, "flops": f_xfwd},
        "xinv_local_bb": {"bytes": W + 4 * F, "flops": f_xinv},
    }
    if info.get("bulk_layout"):
        # bulk layout: y forward (W -> W2), z convolution in place in W2
        # (reads and writes the nz rows, reads the tensor), y inverse (W2 -> W)
        W2 = C * nz * Py * 3 * 2 * esz
        model["y_fwd"] = {"bytes": W + W2, "flops": C * 3 * nz * fft_flops(Py, True, False)}
        model["z_conv"] = {"bytes": 2 * W2 + T,
                           "flops": C * Py * (3 * (fft_flops(Pz, True, False) + fft_flops(Pz, False, True)) + Pz * 36)}
        model["y_inv"] = {"bytes": W2 + W, "flops": C * 3 * nz * fft_flops(Py, False, True)}
    else:
        # z direction as a direct convolution per (kx, ky): nz^2 source/target
        # pairs of the real-even part (20 flops) and nz(nz-1) pairs of the
        # imaginary-odd part (16 flops)
        zc = nz * nz * 20 + nz * (nz - 1) * 16
        f_yz = C * (3 * nz * (fft_flops(Py, True, False) + fft_flops(Py, False, True)) + Py * zc)
        model["yz_conv"] = {"bytes": 2 * W + T, "flops": f_yz}
    return model


def survey_flops(info):
    """Flops per launch of each stage under the workload's reference flop
    model: 2.5 L log2 L per real and 5 L log2 L per complex transform of
    length L (padded), 36 flops per frequency for the symmetric tensor
    product, 200 flops per cell for the local terms, torque, step and
    step-size sums.  At 512 x 256 x 4 (padded 1024 x 512 x 8) this is
    x 0.157 + y 0.284 + z 0.189 + product 0.076 + local 0.105 = 0.81 GFLOP per
    evaluation.  The kernels execute fewer flops (zero inputs and discarded
    outputs pruned, the film z direction as a direct sum); this model is the
    algorithmic count the roofline is quoted against."""
    import math
    nx, ny, nz, Px, Py, Pz = (info[k] for k in ("nx", "ny", "nz", "px", "py", "pz"))
    C = Px // 2 + 1
    lg = lambda L: math.log2(L) if L > 1 else 0.0
    x_half = 3 * ny * nz * 2.5 * Px * lg(Px)          # one real transform per row
    y_one = 3 * C * nz * 5 * Py * lg(Py)              # one direction of the y transforms
    z_both = 2 * 3 * C * Py * 5 * Pz * lg(Pz)
    prod = 36 * C * Py * Pz
    local = 200 * nx * ny * nz
    out = {"xfwd_step": x_half, "xinv_local_bb": x_half + local}
    if info.get("bulk_layout"):
        out.update({"y_fwd": y_one, "z_conv": z_both + prod, "y_inv": y_one})
    else:
        out["yz_conv"] = 2 * y_one + z_both + prod
    return out


KERNEL_SOURCES = ("fft.cuh", "dfloat.cuh", "field_kernels.cuh")  # the device code of the film field kernels


def kernel_source_hash():
    """sha256 (first 16 hex) of the sources of the film field kernels with
    comments and whitespace removed, to tell whether a committed ncu summary
    still describes the kernels that run (an edit of a comment, or of host
    code elsewhere, does not change them)."""
    import hashlib
    import re
    h = hashlib.sha256()
    for name in KERNEL_SOURCES:
        f = os.path.join(ROOT, "paper_1405_2728_gb300", "csrc", name)
        with open(f, encoding="utf-8") as fh:
            text = fh.read()
        text = re.sub(r"/\*.*?\*/", " ", text, flags=re.S)  # block comments
        text = re.sub(r"//[^\n]*", " ", text)               # line comments
        h.update(re.sub(r"\s+", "", text).encode())
    return h.hexdigest()[:16]


def load_traffic(stage, workload, precision):
    """DRAM bytes per launch of a stage from the committed ncu summary
    (profiles/ncu_<workload>_<precision>.md), or None when there is none or the
    kernels changed since it was captured."""
    path = os.path.join(ROOT, "profiles", f"ncu_{workload}_{precision}.md")
    try:
        text = open(path).read()
    except OSError:
        return None
    if f"`{kernel_source_hash()}`" not in text:
        return None
    for line in text.splitlines():
        parts = line.split()
        if len(parts) == 3 and parts[0] == "traffic_bytes_per_launch" and parts[1] == stage:
            return int(parts[2])
    return None


def combine_ranks(evals, ms, e2e_evals, e2e_ms, ws, device):
    """Whole-job figures of independent replicas: evaluations summed over the
    ranks, times taken from the slowest rank (max), for both legs."""
    if ws <= 1:
        return float(evals), float(ms), float(e2e_evals), float(e2e_ms)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(evals), float(ms), float(e2e_evals), float(e2e_ms)], dtype=torch.float64, device=device)
    s = t.clone()
    dist.all_reduce(s, op=dist.ReduceOp.SUM)
    mx = t.clone()
    dist.all_reduce(mx, op=dist.ReduceOp.MAX)
    return s[0].item(), mx[1].item(), s[2].item(), mx[3].item()


def oracle_rate(w, seconds_budget=15.0, max_evals=40):
    """Oracle (float64 numpy/scipy, quad tensor) H_eff+step iterations per second
    on a bounded sample of the workload, on this host's cores."""
    from oracle import micromag as om
    from paper_1405_2728_gb300 import inputs
    oprob = om.Problem(w.nx, w.ny, w.nz, w.dx, w.dy, w.dz, Ms=w.Ms, A=w.A, K=w.K)
    workers = os.cpu_count() or 1
    demag = om.Demag(oprob, workers=workers)
    m = w.initial_m()
    H = w.fields()[0]
    om.minimize(oprob, m, H, demag, tol=0.0, max_iter=0)  # warm (1 evaluation)
    evals, t0 = 0, time.perf_counter()
    n = 1
    while evals < max_evals and time.perf_counter() - t0 < seconds_budget:
        r = om.minimize(oprob, m, H, demag, tol=0.0, max_iter=n)
        evals += r.heff_evals
        m = r.m
    dt = time.perf_counter() - t0
    return evals / dt, evals, workers, dt


def cufft_demag_ms(info, tdt, dev, reps=20):
    """Comparison baseline, not product: the demagnetising convolution of one
    field evaluation done with cuFFT (torch.fft) on the same zero-padded grid
    -- three real-to-complex 3-D FFTs, the symmetric 3x3 tensor product with
    six stored real spectra, three complex-to-real inverses and the unpadding
    -- timed with CUDA events.  The tensor values are random (the time does
    not depend on them).  Returns ms per evaluation."""
    import torch
    nx, ny, nz, Px, Py, Pz = (info[k] for k in ("nx", "ny", "nz", "px", "py", "pz"))
    g = torch.Generator(device=dev).manual_seed(7)
    m = torch.rand((3, nz, ny, nx), device=dev, dtype=tdt, generator=g)
    N = torch.rand((6, Pz, Py, Px // 2 + 1), device=dev, dtype=tdt, generator=g)
    xx, yy, zz, xy, xz, yz = N

    def one():
        mh = torch.fft.rfftn(m, s=(Pz, Py, Px), dim=(1, 2, 3))
        h0 = xx * mh[0] + xy * mh[1] + xz * mh[2]
        h1 = xy * mh[0] + yy * mh[1] + yz * mh[2]
        h2 = xz * mh[0] + yz * mh[1] + zz * mh[2]
        H = torch.fft.irfftn(torch.stack((h0, h1, h2)), s=(Pz, Py, Px), dim=(1, 2, 3))
        return H[:, :nz, :ny, :nx].contiguous()

    for _ in range(3):
        one()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    a.record()
    for _ in range(reps):
        one()
    b.record()
    torch.cuda.synchronize()
    return a.elapsed_time(b) / reps


def run_full_loop(args, w, prob, m, F, opts, stream, tdt, esz, info, dev):
    """One whole hysteresis loop: every field value of the workload's sweep in
    one mm_hysteresis_sweep call from the seeded start, timed with CUDA
    events (after W untimed field values on the same problem as warm-up)."""
    import torch
    from paper_1405_2728_gb300 import inputs, mm
    m_init = m.clone()
    mm.mm_hysteresis_sweep(prob, m, F[: args.warmup], opts=opts, stream=stream)   # warm-up
    m.copy_(m_init)
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    sampler = ClockSampler(int(str(dev).split(":")[-1] or 0))
    with sampler:
        torch.cuda.synchronize()
        a.record(stream)
        st, mavg, res = mm.mm_hysteresis_sweep(prob, m, F, opts=opts, stream=stream)
        b.record(stream)
        torch.cuda.synchronize()
    sec = a.elapsed_time(b) / 1e3
    evals = sum(r.heff_evals for r in res)
    hhat = F[int(np.argmax(np.linalg.norm(F, axis=1)))]
    hhat = hhat / np.linalg.norm(hhat)
    line = {"metric": METRIC, "value": evals / sec, "unit": UNIT, "n_gpus": 1, "steps": 1, "warmup": 1,
            "ms_per_step": sec * 1e3, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": DTYPE_LABEL[args.precision], "data": "synthetic",
            "config": {"workload": w.name, "cells": [w.nx, w.ny, w.nz], "precision": args.precision,
                       "step": f"one whole loop: {len(F)} field values minimised to tol {w.tol:g}",
                       "tau_rule": args.tau_rule},
            "loop_time_s": sec, "loop_evals": int(evals),
            "converged_field_values": int(sum(r.converged for r in res)), "field_values": len(F),
            "status": int(st), "gpu_launches": int(sum(r.kernel_launches for r in res)),
            "clocks": sampler.summary()}
    h = (F @ hhat) * inputs.MU0 * 1e3
    p = mavg @ hhat
    nd = 1
    while nd < len(h) and h[nd] < h[nd - 1]:
        nd += 1
    sw = [float(h[i]) for i in range(1, nd) if p[i] < 0]
    line["H_sw_mT"] = sw[0] if sw else None
    print(json.dumps(line))
    prob.close()
    return 0


def measure_mixed_loop(w, dev, hi_name, tol_lo, max_iter, warmup):
    """One whole loop with mm_hysteresis_sweep_mixed (per field value FP32 to
    tol_lo, then hi_name, FP64 or f32x2, to the workload's tolerance), timed
    with CUDA events after a warm-up over the first field values.  Returns
    the loop's time, evaluations, switching field and clocks."""
    import torch
    from paper_1405_2728_gb300 import inputs, mm
    grid = mm.make_grid(w.nx, w.ny, w.nz, w.dx, w.dy, w.dz)
    mat = mm.make_material(w.Ms, w.A, w.K, K_cell=w.K_cell, u_cell=w.u_cell)
    lo = mm.mm_setup_geometry(grid, mat, mm.MM_FP32)
    hi = mm.mm_setup_geometry(grid, mat, PRECISIONS[hi_name])
    F = w.fields()
    o_lo = mm.make_opts(tol=tol_lo, max_iter=20000)
    o_hi = mm.make_opts(tol=w.tol, max_iter=max_iter)
    stream = torch.cuda.current_stream(dev)
    m0 = torch.from_numpy(w.initial_m()).to(device=dev, dtype=torch.float64).contiguous()
    m = m0.clone()
    mm.mm_hysteresis_sweep_mixed(lo, hi, m, F[:warmup], opts_lo=o_lo, opts_hi=o_hi, stream=stream)
    m.copy_(m0)
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    sampler = ClockSampler(int(str(dev).split(":")[-1] or 0))
    with sampler:
        torch.cuda.synchronize()
        a.record(stream)
        st, mavg, rl, rh = mm.mm_hysteresis_sweep_mixed(lo, hi, m, F, opts_lo=o_lo, opts_hi=o_hi, stream=stream)
        b.record(stream)
        torch.cuda.synchronize()
    sec = a.elapsed_time(b) / 1e3
    ev_lo, ev_hi = sum(r.heff_evals for r in rl), sum(r.heff_evals for r in rh)
    hhat = F[int(np.argmax(np.linalg.norm(F, axis=1)))]
    hhat = hhat / np.linalg.norm(hhat)
    h = (F @ hhat) * inputs.MU0 * 1e3
    p = mavg @ hhat
    nd = 1
    while nd < len(h) and h[nd] < h[nd - 1]:
        nd += 1
    sw = [float(h[i]) for i in range(1, nd) if p[i] < 0]
    lo.close()
    hi.close()
    return {"loop_time_s": sec, "loop_evals_fp32": int(ev_lo), "loop_evals_fp64": int(ev_hi),
            "converged_field_values": int(sum(r.converged for r in rh)), "field_values": len(F),
            "status": int(st), "H_sw_mT": sw[0] if sw else None,
            "gpu_launches": int(sum(r.kernel_launches for r in rl) + sum(r.kernel_launches for r in rh)),
            "clocks": sampler.summary()}


def run_mixed_loop(args, w, dev):
    """One whole loop with mm_hysteresis_sweep_mixed: per field value FP32 to
    --mixed-tol, then --mixed-hi to the workload's tolerance."""
    if args.mixed_tol is None:
        args.mixed_tol = 1e-4 if args.mixed_hi == "f32x2" else 3e-5
    r = measure_mixed_loop(w, dev, args.mixed_hi, args.mixed_tol, args.max_iter, args.warmup)
    F = w.fields()
    line = {"metric": METRIC, "value": (r["loop_evals_fp32"] + r["loop_evals_fp64"]) / r["loop_time_s"], "unit": UNIT,
            "n_gpus": 1, "steps": 1, "warmup": 1, "ms_per_step": r["loop_time_s"] * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32+" + DTYPE_LABEL[args.mixed_hi], "data": "synthetic",
            "config": {"workload": w.name, "cells": [w.nx, w.ny, w.nz], "precision": "mixed",
                       "step": f"one whole loop: {len(F)} field values, FP32 to tol {args.mixed_tol:g} "
                               f"then {args.mixed_hi} to tol {w.tol:g}"},
            **r}
    print(json.dumps(line))
    return 0


def run_precision_compare(args, w, dev):
    """The precision extension's comparison: one whole loop of the workload's
    sweep (the first --values field values) in FP32 and in FP64 from the same
    seeded start, each timed with CUDA events, and every FP32 result (<m>,
    energy per field value, the switching field) compared with the FP64 one."""
    import torch
    from paper_1405_2728_gb300 import inputs, mm
    grid = mm.make_grid(w.nx, w.ny, w.nz, w.dx, w.dy, w.dz)
    mat = mm.make_material(w.Ms, w.A, w.K, K_cell=w.K_cell, u_cell=w.u_cell)
    F = w.fields()
    if args.values:
        F = F[: args.values]
    opts = mm.make_opts(tol=w.tol, max_iter=args.max_iter)
    stream = torch.cuda.current_stream(dev)
    runs = {}
    sampler = ClockSampler(int(str(dev).split(":")[-1] or 0))
    with sampler:
        for name, prec, dt in (("fp64", mm.MM_FP64, torch.float64), ("fp32", mm.MM_FP32, torch.float32)):
            prob = mm.mm_setup_geometry(grid, mat, prec)
            m = torch.from_numpy(w.initial_m()).to(device=dev, dtype=dt).contiguous()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            a.record(stream)
            st, mavg, res = mm.mm_hysteresis_sweep(prob, m, F, opts=opts, stream=stream)
            b.record(stream)
            torch.cuda.synchronize()
            runs[name] = {"sec": a.elapsed_time(b) / 1e3, "mavg": mavg, "res": res, "status": int(st)}
            prob.close()
    hhat = F[int(np.argmax(np.linalg.norm(F, axis=1)))]
    hhat = hhat / np.linalg.norm(hhat)
    h = (F @ hhat) * inputs.MU0
    top = int(np.argmax(h))                  # ramp 0 -> +max, then +max -> -max

    def switching(mv):
        p = mv @ hhat
        idx = [i for i in range(top + 1, len(h)) if h[i] < 0 and p[i] < 0]
        return float(h[idx[0]]) if idx else None

    def remanence(mv):
        idx = [i for i in range(top + 1, len(h)) if abs(h[i]) < 1e-12]
        return float(mv[idx[0]] @ hhat) if idx else None

    d = np.abs(runs["fp32"]["mavg"] - runs["fp64"]["mavg"]).max(axis=1)
    e64 = np.array([r.energy for r in runs["fp64"]["res"]])
    e32 = np.array([r.energy for r in runs["fp32"]["res"]])
    de = np.abs(e32 - e64) / np.maximum(np.abs(e64), 1e-300)
    out = {}
    for name, r in runs.items():
        ev = sum(x.heff_evals for x in r["res"])
        out[name] = {"loop_time_s": r["sec"], "loop_evals": int(ev), "evals_per_s": ev / r["sec"],
                     "converged_field_values": int(sum(x.converged for x in r["res"])), "status": r["status"],
                     "H_sw_T": switching(r["mavg"]), "M_r": remanence(r["mavg"])}
    line = {"metric": METRIC, "value": out["fp32"]["evals_per_s"], "unit": UNIT, "n_gpus": 1, "steps": 1,
            "warmup": 0, "ms_per_step": out["fp32"]["loop_time_s"] * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32 (compared with f64)", "data": "synthetic",
            "config": {"workload": w.name, "cells": [w.nx, w.ny, w.nz], "precision": "fp32 vs fp64",
                       "step": f"one loop of {len(F)} field values in each precision, tol {w.tol:g}"},
            "fp64": out["fp64"], "fp32": out["fp32"],
            "fp32_vs_fp64": {"max_abs_dmavg": float(d.max()), "median_abs_dmavg": float(np.median(d)),
                             "values_within_1e-3": int((d <= 1e-3).sum()), "field_values": len(F),
                             "max_rel_denergy": float(de.max()), "median_rel_denergy": float(np.median(de)),
                             "loop_time_ratio_fp64_over_fp32": out["fp64"]["loop_time_s"] / out["fp32"]["loop_time_s"]},
            "clocks": sampler.summary()}
    print(json.dumps(line))
    return 0


def all_workloads(inputs):
    return {**inputs.WORKLOADS, **inputs.BULK_WORKLOADS}


def run_batch(args, ws, rank, local, dev):
    """64 films of uneven size (inputs.batch_films), FP64, each with its own
    +-50 mT sweep in 2 mT steps.  A step is one field value for every film:
    K field values for all 64 films in one mm_batch_sweep call, timed for each
    way of running a batch -- the branch graph (the default: one graph launch,
    an independent branch per film with its own nested minimiser loop), the
    grouped launches (one graph launch, one grouped launch per kernel stage
    over the films still running) and a stream per film -- against the same K
    field values swept film by film with mm_hysteresis_sweep.  The sequential
    sweeps run first and the grouped batch last, because making a grouped
    batch harmonises the members' tiles.  The L2 is flushed before each timed
    call."""
    import torch
    from paper_1405_2728_gb300 import inputs, mm
    films = inputs.batch_films(64)
    prec = PRECISIONS.get(args.precision, mm.MM_FP64)
    tdt = torch.float32 if prec == mm.MM_FP32 else torch.float64
    probs = [mm.mm_setup_geometry(mm.make_grid(w.nx, w.ny, w.nz, w.dx, w.dy, w.dz),
                                  mm.make_material(w.Ms, w.A, w.K), prec) for w in films]
    F = films[0].fields()
    opts = mm.make_opts(tol=films[0].tol, max_iter=200000)
    stream = torch.cuda.current_stream(dev)
    flush = torch.empty(int(256 * 2**20) // 4, dtype=torch.float32, device=dev)
    K, W = args.steps, args.warmup

    def fresh():
        return [torch.from_numpy(w.initial_m()).to(device=dev, dtype=tdt) for w in films]

    def timed(fn):
        flush.zero_()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        a.record(stream)
        out = fn()
        b.record(stream)
        torch.cuda.synchronize()
        return out, a.elapsed_time(b)

    sampler = ClockSampler(local)
    results = {}
    with sampler:
        ms = fresh()

        def seq(i0, k):
            ev = 0
            for p, m in zip(probs, ms):
                st, _, res = mm.mm_hysteresis_sweep(p, m, F[: i0 + k], start=i0, opts=opts, stream=stream)
                ev += sum(res[j].heff_evals for j in range(i0, i0 + k))
            return ev
        seq(0, W)
        ev_s, t_s = timed(lambda: seq(W, K))
        kinds = [("branches", mm.MM_BATCH_BRANCHES), ("streams", mm.MM_BATCH_STREAMS)]
        if prec != mm.MM_F32X2:   # grouped launches serve FP64 and FP32 films only
            kinds.append(("grouped", mm.MM_BATCH_GROUPED))
        for name, kind in kinds:
            batch = mm.mm_batch_create(probs, kind)
            ms = fresh()

            def bsweep(i0, k):
                st, _, res = mm.mm_batch_sweep(batch, ms, F[: i0 + k], start=i0, opts=opts, stream=stream)
                ev_f = [sum(r[j].heff_evals for j in range(i0, i0 + k)) for r in res]
                if kind == mm.MM_BATCH_GROUPED:   # 3 grouped stage kernels and the advance kernel per iteration
                    launches = 1 + 4 * max(ev_f)
                else:                            # per film: 3 kernels per iteration, init and record per value
                    launches = sum(3 * e + 2 * k for e in ev_f)
                return sum(ev_f), launches
            bsweep(0, W)
            (ev_b, launches), t_b = timed(lambda: bsweep(W, K))
            results[name] = {"value": ev_b / (t_b / 1e3), "unit": UNIT, "ms_per_step": t_b / K,
                             "evals_per_step": ev_b / K, "speedup_vs_sequential": t_s / t_b,
                             "gpu_launches": int(launches)}
            batch.close()
    clocks = sampler.summary()
    if rank != 0:
        return 0
    head = results["branches"]
    cells = [w.ncells for w in films]
    line = {
        "metric": METRIC, "value": head["value"], "unit": UNIT, "n_gpus": ws, "steps": K, "warmup": W,
        "ms_per_step": head["ms_per_step"], "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": DTYPE_LABEL.get(args.precision, "f64"), "data": "synthetic",
        "config": {"workload": "batch64_films", "films": len(films), "cells_min_max_sum": [min(cells), max(cells), sum(cells)],
                   "precision": args.precision,
                   "step": "one field value of the +-50 mT / 2 mT sweep for all 64 films, tol 1e-5; the K timed "
                           "steps are one mm_batch_sweep call",
                   "l2": "flushed before each timed call (256 MiB write)",
                   "parallelism": "one graph launch per sweep call, an independent branch per film (each with its "
                                  "own nested device-side minimiser loop)"},
        "sequential": {"value": ev_s / (t_s / 1e3), "unit": UNIT, "ms_per_step": t_s / K, "evals_per_step": ev_s / K},
        "batch_kinds": results,
        "evals_per_step": head["evals_per_step"],
        "loop_time_s_extrapolated": {"batched": len(F) * head["ms_per_step"] / 1e3, "sequential": len(F) * t_s / K / 1e3},
        "loop_time_note": LOOP_NOTE,
        "gpu_launches": head["gpu_launches"], "clocks": clocks,
    }
    print(json.dumps(line))
    for p in probs:
        p.close()
    return 0


def run_adjoint(args, dev):
    """Implicit adjoint of the differentiation extension on the 128 x 64 x 2
    film with per-cell K: relax at 0 mT from +x saturation (+50 mT first, as
    the sweeps start), then time mm_adjoint_dK for d<m_x>/dK (CG to a relative
    residual of 1e-11, one graph launch per solve) with CUDA events; W untimed
    solves first.  Reports ms per solve and per CG iteration."""
    import torch
    from paper_1405_2728_gb300 import inputs, mm
    w = inputs.film_128x64x2_random_K()
    grid = mm.make_grid(w.nx, w.ny, w.nz, w.dx, w.dy, w.dz)
    prob = mm.mm_setup_geometry(grid, mm.make_material(w.Ms, w.A, 0.0, K_cell=w.K_cell), mm.MM_FP64)
    m = torch.from_numpy(w.initial_m()).to(device=dev, dtype=torch.float64).contiguous()
    mm.mm_minimize(prob, m, w.fields()[0], mm.make_opts(tol=1e-10, max_iter=400000))
    st, r = mm.mm_minimize(prob, m, (0.0, 0.0, 0.0), mm.make_opts(tol=1e-14, max_iter=400000))
    dJdm = torch.zeros_like(m)
    dJdm[0] = 1.0 / w.ncells
    out = torch.empty(m.shape[1:], dtype=torch.float64, device=dev)
    stream = torch.cuda.current_stream(dev)
    for _ in range(args.warmup):
        mm.mm_adjoint_dK(prob, m, (0.0, 0.0, 0.0), dJdm, out, tol=1e-11, max_iter=200000, stream=stream)
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    its = []
    torch.cuda.synchronize()
    a.record(stream)
    for _ in range(args.steps):
        sta, it, res = mm.mm_adjoint_dK(prob, m, (0.0, 0.0, 0.0), dJdm, out, tol=1e-11, max_iter=200000,
                                        stream=stream)
        its.append(it)
    b.record(stream)
    torch.cuda.synchronize()
    ms = a.elapsed_time(b) / args.steps
    kt = mm.mm_kernel_times(prob, m, (0.0, 0.0, 0.0), reps=30, stream=stream)
    line = {"metric": "adjoint d<m_x>/dK solve time (128x64x2 film, per-cell K)", "value": ms, "unit": "ms/solve",
            "higher_is_better": False, "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
            "dtype": "f64", "data": "synthetic",
            "config": {"workload": w.name, "cells": [w.nx, w.ny, w.nz], "cg_tol": 1e-11,
                       "relaxed_to": "max|m x H|/Ms < 1e-14 at 0 mT"},
            "cg_iterations": its, "ms_per_cg_iteration": ms / max(1, its[-1]), "status": int(sta),
            "relaxation_status": int(st), "field_evaluation_ms": sum(kt.values()),
            "gpu_launches_per_solve": int(6 + 8 * its[-1] + 1)}
    print(json.dumps(line))
    prob.close()
    return 0


def run_reference(args, ws, rank):
    """The oracle as it stands, on this host's cores: one minimisation of
    K iterations at the workload's first field value (tol 0, so it never
    stops early), every field evaluation counted, after W untimed ones."""
    if rank != 0:
        return 0
    from paper_1405_2728_gb300 import inputs
    if args.workload not in inputs.WORKLOADS:
        print(json.dumps({"impl": "reference", "unavailable": f"the oracle reference arm covers the film workloads "
                          f"{sorted(inputs.WORKLOADS)}; {args.workload} needs hours of quad-precision tensor setup"}))
        return 0
    w = inputs.WORKLOADS[args.workload]()
    from oracle import micromag as om
    oprob = om.Problem(w.nx, w.ny, w.nz, w.dx, w.dy, w.dz, Ms=w.Ms, A=w.A, K=w.K)
    workers = os.cpu_count() or 1
    demag = om.Demag(oprob, workers=workers)
    m = w.initial_m()
    H = w.fields()[0]
    m = om.minimize(oprob, m, H, demag, tol=0.0, max_iter=args.warmup - 1).m   # W evaluations
    t0 = time.perf_counter()
    r = om.minimize(oprob, m, H, demag, tol=0.0, max_iter=args.steps)       # K steps: K + 1 evaluations
    dt = time.perf_counter() - t0
    evals = r.heff_evals
    value = evals / dt
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": w.name, "cells": [w.nx, w.ny, w.nz], "precision": args.precision,
                                            "step": "one oracle minimiser iteration (field evaluation + step)"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": workers, "kind": "oracle",
                             "sample": f"one oracle minimisation of {args.steps} iterations ({evals} field "
                                       f"evaluations) at {w.name}, first field value"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--precision", default="fp64", choices=["fp64", "fp32", "f32x2", "mixed"],
                    help="mixed: FP32 minimisation to --mixed-tol, then FP64 to the final tolerance (with --full-loop)")
    ap.add_argument("--mixed-tol", type=float, default=None,
                    help="hand-over tolerance of --precision mixed (default: 3e-5 before FP64, 1e-4 before f32x2, "
                         "the fastest of those measured for each)")
    ap.add_argument("--mixed-hi", default="fp64", choices=["fp64", "f32x2"],
                    help="precision of the second (final-tolerance) phase of --precision mixed")
    ap.add_argument("--workload", default="film_512x256x4")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-loop", action="store_true",
                    help="leave out the measured whole loop of the default 512x256x4 line (about a minute)")
    ap.add_argument("--adjoint", action="store_true",
                    help="time the implicit adjoint (differentiation extension) on the 128x64x2 film instead")
    ap.add_argument("--only", action="store_true",
                    help="measure only --precision (by default the line also carries the other precision)")
    ap.add_argument("--tau-rule", default="alternate", choices=["alternate", "adaptive"],
                    help="step-size rule of the minimiser (Section 2 alternation, or the adaptive switch)")
    ap.add_argument("--full-loop", action="store_true",
                    help="time one whole hysteresis loop (every field value, one sweep call) instead of K steps")
    ap.add_argument("--compare-precisions", action="store_true",
                    help="one loop in FP32 and one in FP64 on the workload, every FP32 result compared with FP64")
    ap.add_argument("--values", type=int, default=0,
                    help="with --compare-precisions: only the first VALUES field values of the sweep")
    ap.add_argument("--max-iter", type=int, default=200000,
                    help="iteration cap per field value (a bounded step for very slow workloads)")
    ap.add_argument("--profile-stages", type=int, default=0,
                    help="only set up the workload and launch each kernel stage this many times (for ncu)")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    ws, rank, local = dist_env()

    import torch
    import torch.distributed as dist
    if args.impl == "reference":
        return run_reference(args, ws, rank)

    if ws > 1:
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    from paper_1405_2728_gb300 import build as mmbuild
    mmbuild.build()
    from paper_1405_2728_gb300 import inputs, mm

    if args.workload == "batch64":
        return run_batch(args, ws, rank, local, dev)
    if args.adjoint:
        return run_adjoint(args, dev)
    w = all_workloads(inputs)[args.workload]()
    if args.compare_precisions:
        return run_precision_compare(args, w, dev)
    if args.precision == "mixed":
        if not args.full_loop:
            ap.error("--precision mixed is measured as a whole loop: add --full-loop")
        return run_mixed_loop(args, w, dev)
    prec = PRECISIONS[args.precision]
    tdt = torch.float32 if prec == mm.MM_FP32 else torch.float64
    esz = 4 if prec == mm.MM_FP32 else 8
    grid = mm.make_grid(w.nx, w.ny, w.nz, w.dx, w.dy, w.dz)
    prob = mm.mm_setup_geometry(grid, mm.make_material(w.Ms, w.A, w.K, K_cell=w.K_cell, u_cell=w.u_cell), prec)
    info = mm.mm_problem_info(prob)
    F = w.fields()
    hdir = F[int(np.argmax(np.linalg.norm(F, axis=1)))]
    hdir = hdir / np.linalg.norm(hdir)
    opts = mm.make_opts(tol=w.tol, max_iter=args.max_iter,
                        tau_rule=mm.MM_TAU_ADAPTIVE if args.tau_rule == "adaptive" else mm.MM_TAU_ALTERNATE)
    stream = torch.cuda.current_stream(dev)
    m = torch.from_numpy(w.initial_m()).to(device=dev, dtype=tdt).contiguous()
    flush = torch.empty(int(256 * 2**20) // 4, dtype=torch.float32, device=dev)  # > 2x L2

    if args.full_loop:
        return run_full_loop(args, w, prob, m, F, opts, stream, tdt, esz, info, dev)

    if args.profile_stages > 0:
        print(json.dumps(mm.mm_kernel_times(prob, m, F[0], reps=args.profile_stages, stream=stream)))
        prob.close()
        return 0

    def field_step(p, buf, i):
        st, _, res = mm.mm_hysteresis_sweep(p, buf, F[: i + 1], start=i, opts=opts, stream=stream)
        return st, res[i]

    def timed_steps(p, buf, first, K):
        """K field values starting at index `first`, L2 flushed before each,
        CUDA events around each on the launching stream."""
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(K)]
        n_ev = n_launch = 0
        sts = []
        torch.cuda.synchronize()
        for j in range(K):
            flush.zero_()
            evs[j][0].record(stream)
            st, r = field_step(p, buf, (first + j) % len(F))
            evs[j][1].record(stream)
            n_ev += r.heff_evals
            n_launch += r.kernel_launches
            sts.append(st)
        torch.cuda.synchronize()
        return sum(a.elapsed_time(b) for a, b in evs), n_ev, n_launch, sts

    for i in range(args.warmup):
        field_step(prob, m, i)
    torch.cuda.synchronize()
    if ws > 1:
        dist.barrier()

    K = args.steps
    sampler = ClockSampler(local)
    t_wall = time.perf_counter()
    with sampler:
        ms, evals, launches, statuses = timed_steps(prob, m, args.warmup, K)
    t_wall = time.perf_counter() - t_wall
    if ws > 1:
        dist.barrier()
    clocks = sampler.summary()

    # end to end through the C ABI with the magnetisation in pinned host memory
    mh = torch.empty(m.shape, dtype=tdt, pin_memory=True)
    mh.copy_(m.cpu())
    e2e_evals = 0
    e2e_ms = 0.0
    for j in range(K):
        i = (args.warmup + K + j) % len(F)
        flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        st, r = field_step(prob, mh, i)   # host buffer: H2D in, minimise, D2H out inside the call
        e2e_ms += 1e3 * (time.perf_counter() - t0)
        e2e_evals += r.heff_evals

    evals_all, ms_max, e2e_all, e2e_max = combine_ranks(evals, ms, e2e_evals, e2e_ms, ws, dev)
    if rank != 0:
        dist.destroy_process_group() if ws > 1 else None
        return 0

    n_sm = torch.cuda.get_device_properties(dev).multi_processor_count
    peaks = measured_peaks()
    fma = mm.mm_probe_fma()
    sm_mhz = clocks.get("sm_mhz") or peaks.get("sm_max_mhz") or 2070.0

    def roofline(p, pname, buf, at_field):
        """Roofline of the dominant kernel stage of problem p: per-stage CUDA
        event times over 30 repetitions on the launching stream."""
        kt = mm.mm_kernel_times(p, buf, F[at_field], reps=30, stream=stream)
        inf = mm.mm_problem_info(p)
        e = 4 if pname == "fp32" else 8
        model = algorithmic_model(inf, e)
        sflops = survey_flops(inf)
        dom = max(kt, key=kt.get)
        sec = kt[dom] * 1e-3
        gbs = model[dom]["bytes"] / sec / 1e9
        hbm = peaks.get("hbm_gbs")
        if pname == "f32x2":
            # double-word arithmetic on the FP32 pipes: one double-word add
            # (the bulk of an FFT) takes 11 FP32 instructions, a product 6
            peak = fma["fp32"] / 2 / DW_ADD_INSTRUCTIONS
            ach = sflops[dom] / sec / 1e12
            roof = {"bound": "alu", "achieved": ach, "peak": peak, "unit": "TFLOP/s (double-word)",
                    "frac": ach / peak,
                    "peak_source": f"measured FP32 FMA throughput {fma['fp32']:.1f} TFLOP/s = {fma['fp32'] / 2:.1f} T "
                                   f"instructions/s, / {DW_ADD_INSTRUCTIONS} instructions per double-word add",
                    "flop_model": "workload reference model (2.5/5 L log2 L per real/complex transform, 36 per "
                                  "frequency, 200 per cell)",
                    "vs_fp64_fma_peak": ach / fma["fp64"]}
        elif pname == "fp64":
            derived = n_sm * FP64_FMA_PER_SM_CLK * 2 * sm_mhz * 1e6 / 1e12
            peak = fma["fp64"]
            ach = sflops[dom] / sec / 1e12
            roof = {"bound": "alu", "achieved": ach, "peak": peak, "unit": "TFLOP/s", "frac": ach / peak,
                    "peak_source": f"measured FP64 FMA throughput (mm_probe_fma, {n_sm} SMs): {peak:.3f} TFLOP/s; "
                                   f"nominal {n_sm} SMs x {FP64_FMA_PER_SM_CLK} FMA/clk x 2 flop at "
                                   f"{sm_mhz:.0f} MHz = {derived:.3f}",
                    "flop_model": "workload reference model (2.5/5 L log2 L per real/complex transform, 36 per "
                                  "frequency, 200 per cell)",
                    "executed_flops_frac": model[dom]["flops"] / sec / 1e12 / peak}
        else:
            peak = hbm or 6800.0
            roof = {"bound": "hbm", "achieved": gbs, "peak": peak, "unit": "GB/s", "frac": gbs / peak,
                    "peak_source": "measured copy bandwidth (MEASURED_PEAKS.json)" if hbm else "fallback 6.8 TB/s",
                    "fp32_alu_frac": sflops[dom] / sec / 1e12 / fma["fp32"]}
        roof["kernel"] = dom
        roof["traffic"] = load_traffic(dom, w.name, pname)
        roof["algorithmic_bytes"] = model[dom]["bytes"]
        roof["algorithmic_flops"] = sflops[dom]
        roof["hbm_frac_of_measured"] = gbs / (hbm or 6800.0)
        roof["stage_ms"] = kt
        return roof, kt

    value = evals_all / (ms_max / 1e3)
    e2e_value = e2e_all / (e2e_max / 1e3)
    roof, ktimes = roofline(prob, args.precision, m, args.warmup)

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": K, "warmup": args.warmup,
        "ms_per_step": ms_max / K, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": DTYPE_LABEL[args.precision], "data": "synthetic",
        "config": {"workload": w.name, "cells": [w.nx, w.ny, w.nz], "padded": [info["px"], info["py"], info["pz"]],
                   "precision": args.precision,
                   "step": f"one field value of the {len(F)}-value sweep minimised to tol {w.tol:g}"
                           + (f", at most {args.max_iter} iterations" if args.max_iter < 200000 else ""),
                   "fields_mT": [round(float(F[(args.warmup + j) % len(F)] @ hdir) * inputs.MU0 * 1e3, 3) for j in range(K)],
                   "l2": "flushed between steps (256 MiB write)", "parallelism": f"replicas{ws}"},
        "evals_per_step": evals / K, "wall_s": t_wall,
        "loop_time_s_extrapolated": (len(F) * evals / K) / value,
        "loop_time_note": LOOP_NOTE,
        "statuses": statuses,
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": int(3 * w.ncells * esz + 24),
                "d2h_bytes_per_step": int(3 * w.ncells * esz + 64)},
        "gpu_launches": int(launches),
        "clocks": clocks,
        "roofline": roof,
        "n_sm": n_sm,
        "fma_peaks_tflops": fma,
    }
    # the other precision of the metric on the same workload and field values
    other = [] if args.only else [q for q in ("fp64", "fp32", "f32x2") if q != args.precision]
    for q in other:
        qprec = PRECISIONS[q]
        qdt = torch.float32 if q == "fp32" else torch.float64
        qp = mm.mm_setup_geometry(grid, mm.make_material(w.Ms, w.A, w.K, K_cell=w.K_cell, u_cell=w.u_cell), qprec)
        qm = torch.from_numpy(w.initial_m()).to(device=dev, dtype=qdt).contiguous()
        for i in range(args.warmup):
            field_step(qp, qm, i)
        qsampler = ClockSampler(local)
        with qsampler:
            qms, qev, qla, qst = timed_steps(qp, qm, args.warmup, K)
        qroof, _ = roofline(qp, q, qm, args.warmup)
        qinfo = mm.mm_problem_info(qp)
        line[q] = {"value": qev / (qms / 1e3), "unit": UNIT, "dtype": DTYPE_LABEL[q],
                   "ms_per_step": qms / K, "evals_per_step": qev / K, "statuses": qst, "gpu_launches": int(qla),
                   "loop_time_s_extrapolated": len(F) * (qms / K) / 1e3, "roofline": qroof, "clocks": qsampler.summary(),
                   "launch_shape": {k: qinfo[k] for k in ("x_fwd_tile_rows", "x_tile_rows", "yz_batch_rows")}}
        qp.close()
    if ws == 1:
        ours = sum(ktimes.values())
        theirs = cufft_demag_ms(info, tdt, dev)
        line["cufft_comparison"] = {
            "demag_convolution_ms": theirs, "ours_full_evaluation_ms": ours,
            "note": "torch.fft (cuFFT) demag convolution alone vs this library's whole evaluation "
                    "(step, convolution, local terms, step-size sums); comparison only"}
    if not args.no_loop and ws == 1 and not args.only and args.workload == "film_512x256x4":
        # the metric's loop time, measured: the fastest loop of FP64 accuracy (FP32, then
        # double-word from a 1e-4 hand-over), every field value of the sweep in one call
        line["loop_measured"] = {"sweep": "mm_hysteresis_sweep_mixed, FP32 then f32x2 (hand-over tol 1e-4)",
                                 **measure_mixed_loop(w, dev, "f32x2", 1e-4, args.max_iter, args.warmup)}
    if not args.no_cpu_baseline and ws == 1 and args.workload in inputs.BULK_WORKLOADS:
        line["cpu_baseline"] = {"value": None, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
                                "sample": "not run: the oracle's quad-precision tensor on the (n+1)^3 lattice of "
                                          "a 256^3 cube takes hours of host time"}
    elif not args.no_cpu_baseline and ws == 1:
        rate, n_ev, cores, dt = oracle_rate(w)
        line["cpu_baseline"] = {"value": rate, "unit": UNIT, "cores": cores, "kind": "oracle",
                                "sample": f"{n_ev} oracle H_eff+step iterations at {w.name} in {dt:.1f} s"}
    print(json.dumps(line))
    prob.close()
    if ws > 1:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
