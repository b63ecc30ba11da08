"""Benchmark of the residual-projection chirplet matching pursuit on GB300.

Default workload (one step = one whole decomposition, all orders):
  EEG-like window, N = 512 samples at fs = 256 Hz, 5 random chirplets plus
  pink noise at 10 dB SNR, searched over the 128 tc x 64 fc x 8 logDt x
  32 c = 2,097,152-atom grid (FP32 dictionary, 4.3 GB, resident in HBM),
  20 matching-pursuit orders, FP32 GEMV search (one channel per GPU).
With the tensor-core search built, the same line also reports the batched
BF16 search of 64 such channels ("bf16_batched").

Metric: chirplet projections/s = channels * atoms * orders / time, plus MP
atoms/s = channels * orders / time.  The dictionary (4.3 GB) is larger than
L2, so no flush is needed between steps.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun every rank decomposes its own channel (weak scaling, no
collective on the data path); the timing is the max over ranks.
--impl reference times the FP64 CPU oracle on a bounded sample of the same
workload (the reference arm of this comparison).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import re
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "chirplet projections/s and MP atoms/s: BF16-TC batched vs FP32 plain, % roofline"
UNIT = "projections/s"
WORKLOAD = "eeg_like_fp32_1ch_n512_fs256_grid128x64x8x32_k2097152_p20"
PROFILES = os.path.join(ROOT, "profiles")


def _env_rank():
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("LOCAL_RANK", "0")),
            int(os.environ.get("WORLD_SIZE", "1")))


def _measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return d, "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


def _source_hash(files):
    h = hashlib.sha256()
    for f in files:
        with open(os.path.join(ROOT, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def _profile_traffic(summary_name, kernel_files):
    """DRAM bytes per launch recorded in a committed ncu summary, or None if
    absent or if the kernel sources changed since it was taken."""
    path = os.path.join(PROFILES, summary_name)
    if not os.path.exists(path):
        return None
    text = open(path).read()
    m = re.search(r"traffic_bytes_per_launch:\s*([0-9.eE+]+)", text)
    h = re.search(r"source_sha256_16:\s*([0-9a-f]+)", text)
    if not m or not h or h.group(1) != _source_hash(kernel_files):
        return None
    return float(m.group(1))


class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""

    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.QUERY}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self._t = threading.Thread(target=self._read, daemon=True)
            self._t.start()
            time.sleep(0.3)
        except (FileNotFoundError, OSError):
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc is not None:
            time.sleep(0.2)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.lines:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx = float(parts[2])
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        if not sm:
            return None
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


# ---------------------------------------------------------------------------
# Reference arm / CPU baseline: the FP64 oracle on a bounded sample
# ---------------------------------------------------------------------------
def _oracle_sample(tc_cols: int, orders: int):
    import oracle
    from paper_2607_16629_gb300 import synth
    full = synth.grid_eeg()
    sub = synth.Grid(full.n_samples, full.fs, synth.Axis(full.tc.lo, full.tc.step, tc_cols), full.fc,
                     full.logdt, full.c)
    s, _ = synth.eeg_like_signal(2, 0)
    D, _ = oracle.dictionary(sub)
    t0 = time.perf_counter()
    oracle.mp(D, s, orders)
    dt = time.perf_counter() - t0
    return sub.n_atoms * orders / dt, sub.n_atoms, dt


def cpu_baseline(target_s: float = 12.0):
    import oracle
    cores = oracle.max_threads()
    # calibrate on 2 tc columns (32,768 atoms), then size the sample
    rate, _, _ = _oracle_sample(2, 2)
    per_col = 16384 * 20 / rate
    cols = int(max(2, min(128, target_s / per_col)))
    rate, K, dt = _oracle_sample(cols, 20)
    # the same oracle on one core, on a smaller sample (about 2-3 s)
    oracle.set_threads(1)
    try:
        cols1 = int(max(1, min(16, 2.5 / (per_col * cores))))
        rate1, K1, dt1 = _oracle_sample(cols1, 20)
    finally:
        oracle.set_threads(cores)
    return {"value": rate, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"FP64 oracle MP, 20 orders over the first {cols} of 128 tc columns "
                      f"({K} of 2,097,152 atoms), N=512; {dt:.1f} s timed; dictionary build excluded",
            "one_core": {"value": rate1, "unit": UNIT, "cores": 1,
                         "sample": f"the same, over {cols1} tc columns ({K1} atoms); {dt1:.1f} s timed"}}


def run_reference(args):
    rank, _, world = _env_rank()
    if rank != 0:
        return
    import oracle
    cores = oracle.max_threads()
    cols = 4  # 65,536 atoms per step, 20 orders: a bounded sample of the workload
    for _ in range(args.warmup):
        _oracle_sample(cols, 20)
    rates, times = [], []
    for _ in range(args.steps):
        r, K, dt = _oracle_sample(cols, 20)
        rates.append(r)
        times.append(dt)
    value = float(np.sum([16384 * cols * 20 for _ in times]) / np.sum(times))
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000 * float(np.mean(times)),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": WORKLOAD, "sample_atoms": 16384 * cols},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": f"FP64 oracle MP, 20 orders over {16384 * cols} of 2,097,152 atoms "
                                       f"per step, N=512, dictionary build excluded"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# Our arm
# ---------------------------------------------------------------------------
def run_ours(args):
    import torch
    import torch.distributed as dist

    from paper_2607_16629_gb300 import act, synth

    from paper_2607_16629_gb300.sharding import channels_for_rank, max_over_ranks

    rank, local_rank, world = _env_rank()
    if world > 1:
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    stream = torch.cuda.current_stream(dev)

    grid = synth.grid_eeg()
    P = 20
    (channel,) = channels_for_rank(1, world, rank)  # weak scaling: one EEG-like channel per GPU
    sig_np, _ = synth.eeg_like_signal(2, channel)
    K = grid.n_atoms
    h = act.act_grid_create(grid, local_rank)
    build_ev = (torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
    build_ev[0].record(stream)
    act.act_dictionary_build(h, act.ACT_DICT_FP32, stream)
    build_ev[1].record(stream)
    torch.cuda.synchronize(dev)
    build_ms = build_ev[0].elapsed_time(build_ev[1])

    sig = torch.tensor(sig_np[None, :], dtype=torch.float32, device=dev)
    act.act_autotune(h, sig, 1, stream)
    gemv_ctas, _, _ = act.act_get_tuning(h)
    atoms = torch.empty((1, P, act.ATOM_BYTES), dtype=torch.uint8, device=dev)
    coef = torch.empty((1, P), dtype=torch.float32, device=dev)
    resid = torch.empty((1, grid.n_samples), dtype=torch.float32, device=dev)
    energy = torch.empty((1, P + 1), dtype=torch.float64, device=dev)

    def step():
        act.act_decompose(h, sig, 1, P, atoms, coef, resid, energy, stream)

    def timed(steps):
        """CUDA-event time of `steps` decompositions, barrier-bracketed, max over ranks."""
        torch.cuda.synchronize(dev)
        if world > 1:
            dist.barrier()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(steps):
            step()
        e1.record(stream)
        torch.cuda.synchronize(dev)
        if world > 1:
            dist.barrier()
        return max_over_ranks(e0.elapsed_time(e1), dev)

    for _ in range(max(3, args.warmup)):
        step()
    with ClockSampler(local_rank) as clk:
        ms = timed(args.steps)
    # the same steps again with a CUDA event pair around every search launch
    # inside the graph: average GEMV duration for the roofline
    act.act_set_profiling(h, True)
    for _ in range(2):
        step()
    search_ms, search_n = 0.0, 0
    for _ in range(args.steps):
        step()
        _, core_i, n_i, kernels = act.act_profile_read(h)  # waits for this step's events
        search_ms += core_i
        search_n += n_i
    act.act_set_profiling(h, False)
    st = act.act_grid_status(h, stream)
    if st != act.ACT_OK:
        raise RuntimeError(f"device status {act.status_name(st)}")
    units = world * K * P * args.steps
    value = units / (ms / 1e3)

    # dominant kernel: the FP32 GEMV (events around each launch inside the graph)
    peaks, peak_kind = _measured_peaks()
    gemv_bytes = K * grid.n_samples * 4 + grid.n_samples * 4
    avg_ms = search_ms / max(1, search_n)
    achieved = gemv_bytes / (avg_ms / 1e3) / 1e9
    if gemv_ctas == -1:  # the bulk-copy streaming GEMV won the autotune
        gemv_kernel = "k_gemv_stream<4> (FP32 GEMV, TMA bulk-copy stream, fused argmax)"
        traffic = _profile_traffic("gemv_stream_eeg_k2097152_n512.md",
                                   ["paper_2607_16629_gb300/csrc/act_gemv_stream.cu",
                                    "paper_2607_16629_gb300/csrc/act_device.cuh"])
    else:
        gemv_kernel = "k_gemv<4,1> (FP32 GEMV + fused argmax)"
        traffic = _profile_traffic("gemv_argmax_eeg_k2097152_n512.md",
                                   ["paper_2607_16629_gb300/csrc/act_gemv.cu",
                                    "paper_2607_16629_gb300/csrc/act_device.cuh"])
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                "frac": achieved / peaks["hbm_gbs"], "traffic": traffic,
                "kernel": gemv_kernel, "autotuned_gemv_ctas": gemv_ctas,
                "peak_source": f"{peak_kind} hbm_gbs",
                "algorithmic_bytes_per_launch": gemv_bytes, "avg_launch_ms": avg_ms,
                "launches_timed": search_n,
                "timing": "CUDA event pair around every GEMV launch inside the graph, over a second pass "
                          "of the same steps right after the headline pass (which carries no event nodes)"}

    # end to end through the C ABI with host buffers (copies inside the region)
    hs = torch.tensor(sig_np[None, :], dtype=torch.float32).pin_memory()
    ha = torch.empty((1, P, act.ATOM_BYTES), dtype=torch.uint8).pin_memory()
    hc = torch.empty((1, P), dtype=torch.float32).pin_memory()
    hr = torch.empty((1, grid.n_samples), dtype=torch.float32).pin_memory()
    he = torch.empty((1, P + 1), dtype=torch.float64).pin_memory()
    for _ in range(3):
        act.act_decompose(h, hs, 1, P, ha, hc, hr, he, stream)
    torch.cuda.synchronize(dev)
    if world > 1:
        dist.barrier()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        act.act_decompose(h, hs, 1, P, ha, hc, hr, he, stream)
    torch.cuda.synchronize(dev)
    e2e_s = max_over_ranks(time.perf_counter() - t0, dev)
    e2e = {"value": world * K * P * args.steps / e2e_s, "unit": UNIT,
           "h2d_bytes_per_step": hs.numel() * 4,
           "d2h_bytes_per_step": ha.numel() + hc.numel() * 4 + hr.numel() * 4 + he.numel() * 8}
    act.act_destroy(h)
    fp32_picks = atoms.clone()

    shift = None
    if not args.no_shift:
        shift = bench_shift(args, dev, stream, ms / args.steps, fp32_picks, clk.summary(), peaks, peak_kind)
    bf16 = None
    if not args.no_bf16:
        bf16 = bench_bf16(args, dev, stream, peaks, peak_kind)
    ragged = None
    if not args.no_ragged:
        ragged = bench_ragged(args, dev, stream, peaks, peak_kind)
    refine = None
    if not args.no_refine:
        refine = bench_refine(args, dev, stream, peaks, peak_kind)
    small = None
    if not args.no_small:
        small = bench_small_check(args, dev, stream)
    lem = None
    if not args.no_lem:
        lem = bench_lem(args, dev, stream, peaks, peak_kind)

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                "config": {"workload": WORKLOAD, "channels_per_gpu": 1, "n_samples": grid.n_samples,
                           "fs_hz": grid.fs, "grid_atoms": K, "orders": P,
                           "dictionary": "FP32 4.29 GB stored in HBM", "search": "FP32 GEMV + fused argmax",
                           "l2": "inputs larger than L2 (4.3 GB dictionary streamed every order); no flush",
                           "parallelism": f"{world} independent channel(s), one per GPU"},
                "atoms_per_s": world * P * args.steps / (ms / 1e3),
                "dictionary_build_ms": build_ms,
                "roofline": roofline, "e2e": e2e, "gpu_launches": kernels * args.steps,
                "clocks": clk.summary()}
        if shift is not None:
            line["template_shift"] = shift
        if bf16 is not None:
            line["bf16_batched"] = bf16
        if ragged is not None:
            line["ragged_uneven_batch"] = ragged
        if refine is not None:
            line["offgrid_refinement"] = refine
        if lem is not None:
            line["hierarchical_lem"] = lem
        if small is not None:
            line["small_check"] = small
        line["targets"] = _targets(roofline, shift, bf16)
        if not args.no_cpu_baseline and world == 1:
            line["cpu_baseline"] = cpu_baseline()
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def _targets(roofline, shift, bf16):
    """The two throughput targets next to the fractions this run measured:
    the FP32 GEMV against the HBM roofline (>= 0.70), and the batched BF16
    search on tensor cores against the dense BF16 peak (>= 0.50).  For 64
    EEG-like channels the tensor-core search is the template form (BF16
    templates x shifted BF16 residual rows, FP32 accumulate, FP32 rescore);
    the stored-dictionary BF16 GEMM is HBM-bound at that batch (2 B flop per
    2 bytes of dictionary = 64 flop/byte, below the tensor ridge), so its
    fraction is stated against HBM."""
    out = {"fp32_gemv_hbm": {"target": 0.70, "frac": roofline.get("frac"), "kernel": roofline.get("kernel"),
                             "peak": "measured hbm_gbs"}}
    ch64 = (shift or {}).get("channels_64")
    if ch64:
        r = ch64["roofline"]
        out["bf16_batched_tensor"] = {"target": 0.50, "frac": r["frac"], "executed_frac": r.get("mma_frac"),
                                      "kernel": r["kernel"], "peak": r["peak_source"],
                                      "ms_per_step": ch64["tensor_ms_per_step"]}
    if bf16:
        r = bf16["roofline"]
        out["bf16_dense_gemm_hbm"] = {"frac": r["frac"], "tensor_frac": r["tensor_frac_of_bf16_peak"],
                                      "kernel": r["kernel"], "ms_per_step": bf16["ms_per_step"],
                                      "note": "64 flop/byte at 64 channels: bound by HBM, not by the tensor pipe"}
    return out


def _time_decompose(act, torch, h, sig, P, steps, stream, dev):
    """ms per decomposition (clean pass), then a profiled pass: average search
    and dominant-kernel ms per order, kernels per call; and the outputs."""
    B, L = sig.shape
    out = [torch.empty((B, P, act.ATOM_BYTES), dtype=torch.uint8, device=dev),
           torch.empty((B, P), dtype=torch.float32, device=dev),
           torch.empty((B, L), dtype=torch.float32, device=dev),
           torch.empty((B, P + 1), dtype=torch.float64, device=dev)]
    for _ in range(3):
        act.act_decompose(h, sig, B, P, *out, stream)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize(dev)
    e0.record(stream)
    for _ in range(steps):
        act.act_decompose(h, sig, B, P, *out, stream)
    e1.record(stream)
    torch.cuda.synchronize(dev)
    ms = e0.elapsed_time(e1) / steps
    act.act_set_profiling(h, True)
    act.act_decompose(h, sig, B, P, *out, stream)
    search, core, n = 0.0, 0.0, 0
    for _ in range(max(2, steps // 4)):
        act.act_decompose(h, sig, B, P, *out, stream)
        s_i, c_i, n_i, kernels = act.act_profile_read(h)
        search += s_i
        core += c_i
        n += n_i
    act.act_set_profiling(h, False)
    st = act.act_grid_status(h, stream)
    if st != act.ACT_OK:
        raise RuntimeError(act.status_name(st))
    return ms, search / max(1, n), core / max(1, n), kernels, n, [o.clone() for o in out]


def _tc_mma_flops(grid, B):
    """MMA flops one tensor-core template GEMM executes for B channels: the
    library's row tiling (Bg channels x Jt time centres per 128-row tile,
    only the 64-lag chunks the tile's windows touch), over 256-template
    tiles (128 when those would leave SMs idle, the same count of flops)."""
    S, tc0, Ntc, L = int(grid.tc.step), int(grid.tc.lo), grid.tc.count, grid.n_samples
    T = grid.fc.count * grid.logdt.count * grid.c.count
    t_pad = (T + 255) // 256 * 256
    bg = 1
    while bg < B and bg < 16:
        bg <<= 1
    n2 = 1
    while n2 < Ntc:
        n2 <<= 1
    jt = min(128 // bg, n2)
    n_cb = (B + 128 // jt - 1) // (128 // jt)
    span0 = S * (Ntc - 1)
    chunks = 0
    for g in range((Ntc + jt - 1) // jt):
        jf, jl = g * jt, min(g * jt + jt, Ntc) - 1
        chunks += ((L - 1 + span0 - S * jf) // 64 - (span0 - S * jl) // 64 + 1) * n_cb
    return 2.0 * 128 * t_pad * 64 * chunks


def bench_shift(args, dev, stream, fp32_ms_per_step, fp32_atoms, clocks, peaks, peak_kind):
    """Template dictionary (no atom rows stored; every atom formed in-kernel
    from its (fc, logDt, c) template) on the headline workload (one EEG-like
    channel, 2,097,152 atoms, 20 orders) and on 64 EEG-like channels: the
    FP32 template search (CUDA cores) and the tensor-core template search
    (BF16 tcgen05 GEMM + exact FP32 rescore), whose selections are checked
    equal bit for bit."""
    import torch

    from paper_2607_16629_gb300 import act, synth
    grid = synth.grid_eeg()
    P, K, L = 20, grid.n_atoms, grid.n_samples
    sig1 = torch.tensor(synth.eeg_like_signal(2, 0)[0][None, :], dtype=torch.float32, device=dev)
    w3 = synth.workload_c3()
    B = w3.signals.shape[0]
    sig64 = torch.tensor(w3.signals, dtype=torch.float32, device=dev)
    steps = args.steps
    h = act.act_grid_create(grid, dev.index)
    try:
        b0, b1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        b0.record(stream)
        act.act_dictionary_build(h, act.ACT_DICT_RECOMPUTE, stream)
        b1.record(stream)
        torch.cuda.synchronize(dev)
        build_ms = b0.elapsed_time(b1)
        act.act_autotune(h, sig1, 1, stream)
        lags, warps, stages, ctas_per_sm = act.act_get_shift_tuning(h)
        act.act_set_search(h, act.ACT_SEARCH_SHIFT)
        f1 = _time_decompose(act, torch, h, sig1, P, steps, stream, dev)
        act.act_set_search(h, act.ACT_SEARCH_SHIFT_BF16)
        t1 = _time_decompose(act, torch, h, sig1, P, steps, stream, dev)
        st0 = act.act_bf16_stats(h)
        t64 = _time_decompose(act, torch, h, sig64, P, max(3, steps // 4), stream, dev)
        st1 = act.act_bf16_stats(h)
        act.act_set_search(h, act.ACT_SEARCH_SHIFT)
        f64 = _time_decompose(act, torch, h, sig64, P, 2, stream, dev)
    finally:
        act.act_destroy(h)
    same_fp32 = all(torch.equal(a, b) for a, b in zip(f1[5], t1[5])) and \
        all(torch.equal(a, b) for a, b in zip(f64[5], t64[5]))
    same_gemv = bool(torch.equal(act.atom_indices(f1[5][0]), act.atom_indices(fp32_atoms)))
    T = grid.fc.count * grid.logdt.count * grid.c.count
    S, Ntc = int(grid.tc.step), grid.tc.count
    rows = (Ntc + 31) // 32 * 32 + (L + S - 1) // S - 1
    kt = (L - 1 + S * (Ntc - 1) + 1 + 63) // 64 * 64
    tpl_bytes = T * S * rows * 4 + 2 * T * ((Ntc + 31) // 32 * 32) * 4 + T * kt * 2
    props = torch.cuda.get_device_properties(dev)
    sm_mhz = clocks.get("sm_max_mhz") or 2070.0
    alu_peak = props.multi_processor_count * 128 * 2 * sm_mhz * 1e6 / 1e12
    alu = 2.0 * K * L / (f1[2] / 1e3) / 1e12
    tc_peak = peaks["bf16_tflops_sustained"]
    alg64 = 2.0 * B * K * L / (t64[2] / 1e3) / 1e12
    mma_flops = _tc_mma_flops(grid, B)
    mma64 = mma_flops / (t64[2] / 1e3) / 1e12
    fb = [y - x for x, y in zip(st0, st1)]
    return {"workload": "eeg_like_n512_k2097152_p20: 1 channel (the headline signal) and 64 channels",
            "value": K * P / (t1[0] / 1e3), "unit": UNIT, "ms_per_step": t1[0],
            "search": "tensor-core template search (default for a template build)",
            "speedup_vs_fp32_gemv": fp32_ms_per_step / t1[0],
            "same_selections_as_fp32_gemv": same_gemv,
            "tensor_equals_fp32_template_search_bit_for_bit": bool(same_fp32),
            "template_build_ms": build_ms, "template_bytes": int(tpl_bytes),
            "fp32_dictionary_bytes": K * L * 4,
            "fp32_template_search": {
                "ms_per_step": f1[0], "value": K * P / (f1[0] / 1e3), "unit": UNIT,
                "tuning": {"lags_per_thread": lags, "warps": warps, "stages": stages, "ctas_per_sm": ctas_per_sm},
                "roofline": {"bound": "alu", "achieved": alu, "peak": alu_peak, "unit": "TFLOP/s",
                             "frac": alu / alu_peak,
                             "traffic": _profile_traffic("shift_search_eeg_k2097152_n512.md",
                                                         ["paper_2607_16629_gb300/csrc/act_shift.cu",
                                                          "paper_2607_16629_gb300/csrc/act_device.cuh"]),
                             "kernel": "k_shift_search (FP32 FMA, templates in shared memory)",
                             "algorithmic_flops_per_launch": 2.0 * K * L, "avg_launch_ms": f1[2],
                             "launches_timed": f1[4],
                             "peak_source": f"{props.multi_processor_count} SMs x 128 FP32 FMA/clk x 2 flop x "
                                            f"{sm_mhz:.0f} MHz (maximum SM clock)"}},
            "tensor_template_search_1ch": {"ms_per_step": t1[0], "search_ms_per_order": t1[1],
                                           "rows_gemm_ms_per_order": t1[2], "kernels_per_call": t1[3]},
            "channels_64": {
                "tensor_ms_per_step": t64[0], "tensor_value": B * K * P / (t64[0] / 1e3),
                "fp32_template_ms_per_step": f64[0], "fp32_template_value": B * K * P / (f64[0] / 1e3),
                "unit": UNIT, "search_ms_per_order": t64[1], "rows_gemm_ms_per_order": t64[2],
                "resolved_items_fallbacks": fb,
                "roofline": {"bound": "tensor", "achieved": alg64, "peak": tc_peak, "unit": "TFLOP/s",
                             "frac": alg64 / tc_peak,
                             "traffic": _profile_traffic("shift_gemm_tc_eeg_b64.md",
                                                         ["paper_2607_16629_gb300/csrc/act_shift_tc.cu",
                                                          "paper_2607_16629_gb300/csrc/act_tc.cuh",
                                                          "paper_2607_16629_gb300/csrc/act_device.cuh"]),
                             "kernel": "k_shift_rows + k_shift_gemm<256> (BF16 tcgen05, scaled tile maxima)",
                             "algorithmic_flops_per_launch": 2.0 * B * K * L,
                             "mma_flops_per_launch": mma_flops, "mma_tflops": mma64,
                             "mma_frac": mma64 / tc_peak, "avg_launch_ms": t64[2],
                             "peak_source": f"{peak_kind} bf16_tflops_sustained",
                             "note": "each 128-row tile (16 channels x 8 time centres) multiplies the 64-lag "
                                     "chunks its windows touch (9 of Kt / 64 = 16): achieved counts 2 K L flops "
                                     "per channel, mma_tflops everything the tensor cores execute; timed by an "
                                     "event pair around the shifted-row build and the GEMM"}}}


def bench_bf16(args, dev, stream, peaks, peak_kind):
    """64 EEG-like channels, BF16 tensor-core search with FP32 rescore,
    against the plain FP32 path run channel by channel."""
    import torch

    from paper_2607_16629_gb300 import act, synth
    w = synth.workload_c3()
    B, P, K, L = w.signals.shape[0], w.n_atoms, w.grid.n_atoms, w.grid.n_samples
    h = act.act_grid_create(w.grid, dev.index)
    try:
        act.act_dictionary_build(h, act.ACT_DICT_BF16, stream)
    except act.ActError as e:
        act.act_destroy(h)
        return {"status": f"unavailable: {e}"}
    sig = torch.tensor(w.signals, dtype=torch.float32, device=dev)
    out = [torch.empty((B, P, act.ATOM_BYTES), dtype=torch.uint8, device=dev),
           torch.empty((B, P), dtype=torch.float32, device=dev),
           torch.empty((B, L), dtype=torch.float32, device=dev),
           torch.empty((B, P + 1), dtype=torch.float64, device=dev)]
    act.act_set_search(h, act.ACT_SEARCH_BF16)
    tune_ms = act.act_autotune(h, sig, B, stream)
    gemv_ctas, tile_atoms, stages_used = act.act_get_tuning(h)
    steps = max(3, args.steps // 2)
    for _ in range(3):
        act.act_decompose(h, sig, B, P, *out, stream)
    torch.cuda.synchronize(dev)
    c0, s0, f0 = act.act_bf16_stats(h)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        act.act_decompose(h, sig, B, P, *out, stream)
    e1.record(stream)
    torch.cuda.synchronize(dev)
    ms = e0.elapsed_time(e1)
    c1, s1, f1 = act.act_bf16_stats(h)
    # second pass with event pairs inside the graph: search and GEMM times per order
    act.act_set_profiling(h, True)
    act.act_decompose(h, sig, B, P, *out, stream)
    search_ms = gemm_ms = 0.0
    search_n = 0
    for _ in range(steps):
        act.act_decompose(h, sig, B, P, *out, stream)
        a, g_ms, n_i, kernels = act.act_profile_read(h)
        search_ms += a
        gemm_ms += g_ms
        search_n += n_i
    # plain FP32 comparator: the same 64 channels, one FP32 GEMV decomposition each,
    # with the GEMV tuned for one channel
    act.act_set_search(h, act.ACT_SEARCH_FP32)
    act.act_set_profiling(h, False)
    act.act_autotune(h, sig[:1].contiguous(), 1, stream)
    one = [o[:1].contiguous() for o in out]
    act.act_decompose(h, sig[:1].contiguous(), 1, P, *one, stream)
    torch.cuda.synchronize(dev)
    f_e0, f_e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    f_e0.record(stream)
    for b in range(B):
        act.act_decompose(h, sig[b:b + 1], 1, P, *one, stream)
    f_e1.record(stream)
    torch.cuda.synchronize(dev)
    fp32_ms = f_e0.elapsed_time(f_e1)
    act.act_destroy(h)
    value = B * K * P * steps / (ms / 1e3)
    avg = search_ms / max(1, search_n)
    avg_gemm = gemm_ms / max(1, search_n)
    bytes_per = K * L * 2
    flops_per = 2.0 * K * L * B
    bw = bytes_per / (avg_gemm / 1e3) / 1e9
    tflops = flops_per / (avg_gemm / 1e3) / 1e12
    return {"workload": f"eeg_like_bf16_{B}ch_n512_grid128x64x8x32_k2097152_p20", "value": value, "unit": UNIT,
            "atoms_per_s": B * P * steps / (ms / 1e3), "ms_per_step": ms / steps, "steps": steps,
            "dtype": "bf16 x bf16 -> f32 (tensor cores), f32 tile rescan",
            "roofline": {"bound": "hbm", "kernel": "k_gemm_tilemax (tcgen05 BF16 GEMM + per-tile and per-block maxima)",
                         "achieved": bw, "peak": peaks["hbm_gbs"], "unit": "GB/s", "frac": bw / peaks["hbm_gbs"],
                         "traffic": _profile_traffic("gemm_tilemax_bf16_eeg_b64.md",
                                                     ["paper_2607_16629_gb300/csrc/act_gemm.cu",
                                                      "paper_2607_16629_gb300/csrc/act_tc.cuh",
                                                      "paper_2607_16629_gb300/csrc/act_device.cuh"]),
                         "peak_source": f"{peak_kind} hbm_gbs", "avg_gemm_ms": avg_gemm,
                         "algorithmic_bytes_per_launch": bytes_per,
                         "tensor_tflops": tflops,
                         "tensor_frac_of_bf16_peak": tflops / peaks["bf16_tflops_sustained"],
                         "tensor_peak_source": f"{peak_kind} bf16_tflops_sustained",
                         "avg_search_ms_per_order": avg,
                         "search_frac_of_hbm_roofline": bytes_per / (avg / 1e3) / 1e9 / peaks["hbm_gbs"]},
            "autotuned": {"tile_atoms": tile_atoms, "stages": stages_used, "search_ms_per_order": tune_ms},
            "orders_resolved_by_block_rescan": c1 - c0, "blocks_rescanned": s1 - s0,
            "orders_full_fp32_fallback": f1 - f0,
            "fp32_plain_per_channel": {"value": B * K * P / (fp32_ms / 1e3), "ms": fp32_ms},
            "speedup_vs_fp32_plain": (B * K * P * steps / (ms / 1e3)) / (B * K * P / (fp32_ms / 1e3)),
            "gpu_launches": kernels * steps}


def _ragged_run(act, torch, synth, sigs, lengths, offsets, P, dict_mode, steps, dev, stream):
    """One ragged plan over per-length grids built with dict_mode: ms per
    decomposition of all channels, build seconds, device bytes held by the
    grids and the plan, plan info, and the selected flat indices."""
    handles = {}
    torch.cuda.synchronize(dev)
    free0 = torch.cuda.mem_get_info(dev)[0]
    t0 = time.perf_counter()
    try:
        for L in lengths:
            h = act.act_grid_create(synth.grid_emg(L), dev.index)
            handles[L] = h
            act.act_dictionary_build(h, dict_mode, stream)
        torch.cuda.synchronize(dev)
        build_s = time.perf_counter() - t0
        flat = torch.tensor(np.concatenate(sigs).astype(np.float32), device=dev)
        for L in lengths:  # tune each length group on its own channels
            idx = [i for i, x in enumerate(sigs) if len(x) == L]
            grp = torch.tensor(np.stack([sigs[i] for i in idx]).astype(np.float32), device=dev)
            act.act_autotune(handles[L], grp, len(idx), stream)
        plan = act.act_ragged_plan_create([handles[L] for L in lengths], offsets, P)
        try:
            C = len(sigs)
            out = [torch.empty((C, P, act.ATOM_BYTES), dtype=torch.uint8, device=dev),
                   torch.empty((C, P), dtype=torch.float32, device=dev),
                   torch.empty((int(offsets[-1]),), dtype=torch.float32, device=dev),
                   torch.empty((C, P + 1), dtype=torch.float64, device=dev)]
            act.act_ragged_decompose(plan, flat, *out, stream)
            torch.cuda.synchronize(dev)
            used = free0 - torch.cuda.mem_get_info(dev)[0]
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(steps):
                act.act_ragged_decompose(plan, flat, *out, stream)
            e1.record(stream)
            torch.cuda.synchronize(dev)
            ms = e0.elapsed_time(e1) / steps
            for L in lengths:
                st = act.act_grid_status(handles[L], stream)
                if st != act.ACT_OK:
                    raise RuntimeError(act.status_name(st))
            groups, kernels = act.act_ragged_plan_info(plan)
            idx_out = act.atom_indices(out[0]).cpu().numpy()
        finally:
            act.act_ragged_plan_destroy(plan)
    finally:
        for h in handles.values():
            act.act_destroy(h)
    return ms, build_s, int(used), groups, kernels, idx_out


def bench_ragged(args, dev, stream, peaks, peak_kind):
    """Uneven batch: 256 EMG-like signals, N uniform in {256, 512, 1024, 2048}
    at fs = 500 Hz, each over the 256 x 96 x 8 x 24 = 4,718,592-atom grid of
    its length, 30 orders, all length groups in one CUDA graph.  Two builds:
    template dictionaries (atoms generated in-kernel from per-(fc, logDt, c)
    templates, tensor-core template search), the configuration's own
    "generated in-kernel" reading; and stored BF16 + FP32 dictionaries (108 GB)
    with the dense BF16 tensor-core search."""
    import torch

    from paper_2607_16629_gb300 import act, synth
    sigs, grids_py, P = synth.workload_c4()
    lengths = sorted({int(len(x)) for x in sigs})
    offsets = np.concatenate([[0], np.cumsum([len(x) for x in sigs])]).astype(np.int64)
    steps = max(2, args.steps // 10)
    C = len(sigs)
    K = synth.grid_emg(256).n_atoms
    t_ms, t_build, t_bytes, groups, kernels, t_idx = _ragged_run(act, torch, synth, sigs, lengths, offsets, P,
                                                                  act.ACT_DICT_RECOMPUTE, steps, dev, stream)
    d_ms, d_build, d_bytes, _, d_kernels, d_idx = _ragged_run(act, torch, synth, sigs, lengths, offsets, P,
                                                               act.ACT_DICT_BF16, steps, dev, stream)
    bf16_bytes = sum(K * L * 2 for L in lengths)
    counts = {L: sum(1 for x in sigs if len(x) == L) for L in lengths}
    return {"workload": "emg_like_ragged_256ch_n256-2048_fs500_grid256x96x8x24_k4718592_p30",
            "value": C * K * P / (t_ms / 1e3), "unit": UNIT, "atoms_per_s": C * P / (t_ms / 1e3),
            "ms_per_step": t_ms, "steps": steps, "channels_per_length": counts,
            "search": "template dictionaries, tensor-core template search (atoms generated in-kernel)",
            "dictionary_build_s": t_build, "device_bytes": t_bytes, "length_groups": groups,
            "gpu_launches": kernels * steps,
            "stored_bf16_dictionaries": {
                "value": C * K * P / (d_ms / 1e3), "unit": UNIT, "ms_per_step": d_ms,
                "dictionary_build_s": d_build, "device_bytes": d_bytes, "gpu_launches": d_kernels * steps,
                "hbm_frac_of_bf16_dictionary_stream": bf16_bytes * P / (d_ms / 1e3) / 1e9 / peaks["hbm_gbs"],
                "same_selections_as_template_search": float(np.mean(d_idx == t_idx)),
                "dtype": "bf16 x bf16 -> f32 (tensor cores), f32 tile rescan"},
            "dtype": "bf16 x bf16 -> f32 (tensor cores), f32 rescore"}


def bench_small_check(args, dev, stream):
    """The 16,384-atom check workload (N = 256, fs = 128 Hz, 3 on-grid atoms
    plus white noise, 5 orders): its 16.8 MB FP32 dictionary stays in L2,
    so a decomposition is bound by kernel latency, not HBM; reported as us
    per order and projections/s (FP32 GEMV search, the autotuned launch)."""
    import torch

    from paper_2607_16629_gb300 import act, synth
    w = synth.workload_c1()
    B, P, K, L = w.signals.shape[0], w.n_atoms, w.grid.n_atoms, w.grid.n_samples
    h = act.act_grid_create(w.grid, dev.index)
    try:
        act.act_dictionary_build(h, act.ACT_DICT_FP32, stream)
        sig = torch.tensor(w.signals, dtype=torch.float32, device=dev)
        act.act_autotune(h, sig, B, stream)
        out = [torch.empty((B, P, act.ATOM_BYTES), dtype=torch.uint8, device=dev),
               torch.empty((B, P), dtype=torch.float32, device=dev),
               torch.empty((B, L), dtype=torch.float32, device=dev),
               torch.empty((B, P + 1), dtype=torch.float64, device=dev)]
        for _ in range(5):
            act.act_decompose(h, sig, B, P, *out, stream)
        reps = 200
        torch.cuda.synchronize(dev)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            act.act_decompose(h, sig, B, P, *out, stream)
        e1.record(stream)
        torch.cuda.synchronize(dev)
        ms = e0.elapsed_time(e1) / reps
        st = act.act_grid_status(h, stream)
        if st != act.ACT_OK:
            raise RuntimeError(act.status_name(st))
        gemv = act.act_get_tuning(h)[0]
    finally:
        act.act_destroy(h)
    return {"workload": "plain_fp32_1ch_n256_fs128_grid32x16x4x8_k16384_p5", "value": B * K * P / (ms / 1e3),
            "unit": UNIT, "ms_per_step": ms, "us_per_order": 1e3 * ms / P, "steps": reps,
            "bound": "latency (the 16.8 MB dictionary is L2-resident)",
            "gemv": "bulk-copy stream" if gemv == -1 else f"load-streaming, {gemv} CTAs",
            "l2": "dictionary smaller than L2: every step after the first reads it from L2"}


def _refine_runs(act, torch, w, dict_mode, steps_list, n, dev, stream):
    B, P, K, L = w.signals.shape[0], w.n_atoms, w.grid.n_atoms, w.grid.n_samples
    torch.cuda.synchronize(dev)
    free0 = torch.cuda.mem_get_info(dev)[0]
    h = act.act_grid_create(w.grid, dev.index)
    try:
        act.act_dictionary_build(h, dict_mode, stream)
        sig = torch.tensor(w.signals, dtype=torch.float32, device=dev)
        act.act_autotune(h, sig, B, stream)
        out = [torch.empty((B, P, act.ATOM_BYTES), dtype=torch.uint8, device=dev),
               torch.empty((B, P), dtype=torch.float32, device=dev),
               torch.empty((B, L), dtype=torch.float32, device=dev),
               torch.empty((B, P + 1), dtype=torch.float64, device=dev)]
        res = {}
        for steps in steps_list:
            act.act_set_refinement(h, steps)
            act.act_decompose(h, sig, B, P, *out, stream)
            torch.cuda.synchronize(dev)
            used = free0 - torch.cuda.mem_get_info(dev)[0]
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(n):
                act.act_decompose(h, sig, B, P, *out, stream)
            e1.record(stream)
            torch.cuda.synchronize(dev)
            ms = e0.elapsed_time(e1) / n
            st = act.act_grid_status(h, stream)
            if st != act.ACT_OK:
                raise RuntimeError(act.status_name(st))
            en = out[3].cpu().numpy()
            res[steps] = {"ms_per_step": ms, "projections_per_s": B * K * P / (ms / 1e3),
                          "mean_normalised_residue": float(np.mean(en[:, -1] / en[:, 0])), "device_bytes": int(used),
                          "coefs": out[1].clone()}
    finally:
        act.act_destroy(h)
    return res


def bench_refine(args, dev, stream, peaks, peak_kind):
    """Radar-like workload: 32 channels, N = 1024, fs = 1 kHz, 4 off-grid
    chirplets each, 256 x 128 x 8 x 32 = 8,388,608-atom grid, 10 orders, each
    grid selection followed by 20 BFGS iterations of off-grid refinement on
    the GPU; compared with the grid-only search on the same signals.  Atoms
    generated in-kernel from a template dictionary (tensor-core template
    search), the configuration's "recomputed in-kernel" reading; and, for
    comparison, the stored FP32 + BF16 dictionary (51 GB) with the dense BF16
    search."""
    import torch

    from paper_2607_16629_gb300 import act, synth
    w = synth.workload_c5()
    B, P = w.signals.shape[0], w.n_atoms
    n = max(2, args.steps // 10)
    t = _refine_runs(act, torch, w, act.ACT_DICT_RECOMPUTE, (0, 20), n, dev, stream)
    d = _refine_runs(act, torch, w, act.ACT_DICT_BF16, (20,), n, dev, stream)
    extra_ms = t[20]["ms_per_step"] - t[0]["ms_per_step"]
    same = bool(torch.equal(t[20]["coefs"], d[20]["coefs"]))
    for r in (t[0], t[20], d[20]):
        r.pop("coefs")
    return {"workload": "radar_like_32ch_n1024_fs1000_grid256x128x8x32_k8388608_p10_bfgs20",
            "value": t[20]["projections_per_s"], "unit": UNIT, "ms_per_step": t[20]["ms_per_step"],
            "search": "template dictionary, tensor-core template search (atoms generated in-kernel)",
            "grid_only": t[0], "refined": t[20],
            "bfgs_iterations_per_s": B * P * 20 / (max(extra_ms, 1e-6) / 1e3),
            "refinement_ms_per_order": extra_ms / P,
            "stored_dictionary_refined": d[20],
            "same_coefficients_as_stored_dictionary": same,
            "dtype": "bf16 search + f32 rescore; refinement f32 samples, f64 sums"}


def bench_lem(args, dev, stream, peaks, peak_kind):
    """Hierarchical (LEM-inspired) search without a dictionary against the
    dense search, on 64 EEG-like channels (N = 512, fs = 256 Hz) over the
    2,097,152-atom grid's box, 20 orders, each selection refined by 20 BFGS
    iterations: time, device memory and normalised residue (the trade-off of
    the paper's Table 7)."""
    import torch

    from paper_2607_16629_gb300 import act, synth
    w = synth.workload_c3()
    B, P, L = w.signals.shape[0], w.n_atoms, w.grid.n_samples
    sig = torch.tensor(w.signals, dtype=torch.float32, device=dev)
    out = [torch.empty((B, P, act.ATOM_BYTES), dtype=torch.uint8, device=dev),
           torch.empty((B, P), dtype=torch.float32, device=dev),
           torch.empty((B, L), dtype=torch.float32, device=dev),
           torch.empty((B, P + 1), dtype=torch.float64, device=dev)]
    res = {}
    for name in ("lem", "dense_bf16"):
        torch.cuda.synchronize(dev)
        free0 = torch.cuda.mem_get_info(dev)[0]
        h = act.act_grid_create(w.grid, dev.index)
        try:
            if name == "lem":
                act.act_set_search(h, act.ACT_SEARCH_LEM)
            else:
                act.act_dictionary_build(h, act.ACT_DICT_BF16, stream)
                act.act_set_search(h, act.ACT_SEARCH_BF16)
            act.act_set_refinement(h, 20)
            act.act_decompose(h, sig, B, P, *out, stream)
            torch.cuda.synchronize(dev)
            used = free0 - torch.cuda.mem_get_info(dev)[0]
            n = max(2, args.steps // 10)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(n):
                act.act_decompose(h, sig, B, P, *out, stream)
            e1.record(stream)
            torch.cuda.synchronize(dev)
            st = act.act_grid_status(h, stream)
            if st != act.ACT_OK:
                raise RuntimeError(act.status_name(st))
            en = out[3].cpu().numpy()
            res[name] = {"ms_per_step": e0.elapsed_time(e1) / n, "device_bytes": int(used),
                         "mean_normalised_residue": float(np.mean(en[:, -1] / en[:, 0]))}
        finally:
            act.act_destroy(h)
    return {"workload": "eeg_like_64ch_n512_box128x64x8x32_p20_bfgs20", "lem": res["lem"],
            "dense_bf16": res["dense_bf16"],
            "lem_settings": "paper EEG settings: top_k 4, 2 levels, steps (64,2,2,5)/(32,1,1,2.5)/(16,.5,.5,.5), "
                            "radius (2,2,1,2), 2048 LHS samples"}


def run_profile_case(args):
    """Small, self-checking cases for ncu captures: a few launches of one
    search kernel on a dictionary larger than L2 but a few GB at most.
      gemv_small: FP32 GEMV over 1,048,576 EEG-grid atoms (2.1 GB), 1 channel.
      bf16_small: BF16 GEMM search over the same atoms, 64 channels."""
    import torch

    from paper_2607_16629_gb300 import act, synth
    if args.case in ("shift_eeg", "shift_tc_eeg"):
        return run_shift_case(args)
    if args.case in ("lem_eeg", "refine_radar"):
        return run_offgrid_case(args)
    full = synth.grid_eeg()
    grid = synth.Grid(full.n_samples, full.fs, synth.Axis(full.tc.lo, full.tc.step, 64), full.fc, full.logdt,
                      full.c)
    B = 1 if args.case == "gemv_small" else 64
    sig = torch.tensor(np.stack([synth.eeg_like_signal(2, b)[0] for b in range(B)]), dtype=torch.float32,
                       device="cuda")
    h = act.act_grid_create(grid, 0)
    try:
        act.act_dictionary_build(h, act.ACT_DICT_FP32 if B == 1 else act.ACT_DICT_BF16)
        act.act_set_search(h, act.ACT_SEARCH_FP32 if B == 1 else act.ACT_SEARCH_BF16)
        if B == 1 and args.gemv == "stream":
            act.act_set_tuning(h, -1)
        for _ in range(args.steps):
            act.decompose(h, sig, 3)
        torch.cuda.synchronize()
        st = act.act_grid_status(h)
        if st != act.ACT_OK:
            raise RuntimeError(act.status_name(st))
    finally:
        act.act_destroy(h)
    print(json.dumps({"case": args.case, "atoms": grid.n_atoms, "channels": B, "ok": True}))


def run_shift_case(args):
    """Template search on the full 2,097,152-atom EEG-like grid, 3 orders per
    step: --channels EEG-like channels (1 or 64), the FP32 search (shift_eeg)
    or the tensor-core one (shift_tc_eeg).  Templates take 100 MB; with 64
    channels the shifted residual rows add 17 MB."""
    import torch

    from paper_2607_16629_gb300 import act, synth
    grid = synth.grid_eeg()
    B = args.channels
    sig_np = synth.workload_c3().signals[:B] if B > 1 else synth.eeg_like_signal(2, 0)[0][None, :]
    sig = torch.tensor(sig_np, dtype=torch.float32, device="cuda")
    h = act.act_grid_create(grid, 0)
    try:
        act.act_dictionary_build(h, act.ACT_DICT_RECOMPUTE)
        act.act_set_search(h, act.ACT_SEARCH_SHIFT_BF16 if args.case == "shift_tc_eeg" else act.ACT_SEARCH_SHIFT)
        if args.shift_tuning:
            act.act_set_shift_tuning(h, *(int(v) for v in args.shift_tuning.split("x")))
        for _ in range(args.steps):
            _, _, _, energy = act.decompose(h, sig, 3)
        torch.cuda.synchronize()
        st = act.act_grid_status(h)
        if st != act.ACT_OK:
            raise RuntimeError(act.status_name(st))
        e = energy.cpu().numpy()
        assert np.all(np.diff(e, axis=1) <= 0.0)
        tuning = act.act_get_shift_tuning(h)
    finally:
        act.act_destroy(h)
    print(json.dumps({"case": args.case, "atoms": grid.n_atoms, "channels": B, "tuning": tuning, "ok": True}))


def run_offgrid_case(args):
    """Off-grid cases, 2 orders per step with 20 BFGS iterations each:
      lem_eeg: hierarchical search (no dictionary) on --channels EEG-like
        channels (N = 512) over the 2,097,152-atom grid's box;
      refine_radar: tensor-core template search + refinement on 32
        radar-like channels (N = 1024, 8,388,608-atom grid)."""
    import torch

    from paper_2607_16629_gb300 import act, synth
    if args.case == "lem_eeg":
        w = synth.workload_c3()
        sig_np = w.signals[:args.channels]
    else:
        w = synth.workload_c5()
        sig_np = w.signals
    sig = torch.tensor(sig_np, dtype=torch.float32, device="cuda")
    h = act.act_grid_create(w.grid, 0)
    try:
        if args.case == "lem_eeg":
            act.act_set_search(h, act.ACT_SEARCH_LEM)
        else:
            act.act_dictionary_build(h, act.ACT_DICT_RECOMPUTE)
        act.act_set_refinement(h, 20)
        for _ in range(args.steps):
            _, _, _, energy = act.decompose(h, sig, 2)
        torch.cuda.synchronize()
        st = act.act_grid_status(h)
        if st != act.ACT_OK:
            raise RuntimeError(act.status_name(st))
        e = energy.cpu().numpy()
        assert np.all(np.diff(e, axis=1) <= 0.0)
    finally:
        act.act_destroy(h)
    print(json.dumps({"case": args.case, "channels": int(sig.shape[0]), "ok": True}))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=30)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-bf16", action="store_true")
    ap.add_argument("--no-ragged", action="store_true")
    ap.add_argument("--no-refine", action="store_true")
    ap.add_argument("--no-lem", action="store_true")
    ap.add_argument("--no-shift", action="store_true")
    ap.add_argument("--no-small", action="store_true")
    ap.add_argument("--channels", type=int, default=1, help="channels for the shift_* and lem_eeg cases (1 or up to 64)")
    ap.add_argument("--gemv", default="stream", choices=["stream", "load"],
                    help="FP32 GEMV of the gemv_small case: bulk-copy streaming or load-streaming")
    ap.add_argument("--shift-tuning", default="", help="JxW, JxWxS or JxWxSxC for --case shift_eeg (default: the build's)")
    ap.add_argument("--case", default="default",
                    choices=["default", "gemv_small", "bf16_small", "shift_eeg", "shift_tc_eeg", "lem_eeg",
                             "refine_radar"],
                    help="small single-kernel cases for profiler captures (not bench lines)")
    args = ap.parse_args()
    if args.case != "default":
        run_profile_case(args)
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
