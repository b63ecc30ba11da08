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


def _profile_value(summary_name, key, kernel_files):
    """A number recorded as `key: value` in a committed ncu summary, or None
    if absent or if the kernel sources changed since it was taken."""
    path = os.path.join(PROFILES, summary_name)
    if not os.path.exists(path):
        return None
    text = open(path).read()
    m = re.search(re.escape(key) + r":\s*([0-9.eE+]+)", text)
    h = re.search(r"source_sha256_16:\s*([0-9a-f]+)", text)
    if not m or not h or h.group(1) != _source_hash(kernel_files):
        return None
    return float(m.group(1))


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


def _lockstep_stats(score_fn, grid, rs, idx, coef, energy, gap_tol=1e-5):
    """Order-by-order comparison with the FP64 oracle from the GPU's own
    residuals rs[k] (Sec. III-A, Eq. (4)): whether the GPU picked the
    oracle's argmax (a near-tie, relative top-2 gap <= gap_tol, accepts
    either), and the relative error of c_k and |r_{k+1}|^2 against the FP64
    values for the GPU's pick."""
    import oracle
    same = ties = bad = 0
    ce = ee = 0.0
    for k in range(len(idx)):
        r = np.asarray(rs[k], dtype=np.float64)
        sc = score_fn(r, k)
        best, second = oracle.select(sc)
        a = abs(sc[best])
        gap = (a - abs(sc[second])) / a if a > 0 else 0.0
        if idx[k] == best:
            same += 1
        elif gap <= gap_tol:
            ties += 1
        else:
            bad += 1
        c_ref = sc[idx[k]]
        g, _ = oracle.atom(*oracle.atom_params(grid, int(idx[k])), grid.fs, grid.n_samples)
        e_ref = float(np.sum((r - c_ref * g) ** 2))
        ce = max(ce, abs(float(coef[k]) - c_ref) / max(abs(c_ref), 1e-300))
        ee = max(ee, abs(float(energy[k]) - e_ref) / max(e_ref, 1e-300))
    return {"orders": len(idx), "same_atom": same, "near_ties": ties, "violations": bad,
            "max_coef_rel_err": ce, "max_energy_rel_err": ee}


def _merge(stats):
    out = {"orders": 0, "same_atom": 0, "near_ties": 0, "violations": 0, "max_coef_rel_err": 0.0,
           "max_energy_rel_err": 0.0}
    for st in stats:
        for key in ("orders", "same_atom", "near_ties", "violations"):
            out[key] += st[key]
        for key in ("max_coef_rel_err", "max_energy_rel_err"):
            out[key] = max(out[key], st[key])
    return out


def oracle_checks(checks):
    """Error of every section's results against the FP64 oracle, on a bounded
    sample of channels and orders (the GPU data was collected by the sections
    after their timed regions).  Returns one entry per section."""
    import oracle
    from paper_2607_16629_gb300 import synth
    res = {}
    t_all = time.perf_counter()
    eeg = [k for k in ("headline", "bf16_batched", "template_shift_64ch") if k in checks]
    if eeg:
        t0 = time.perf_counter()
        D, _ = oracle.dictionary(synth.grid_eeg())
        build_s = time.perf_counter() - t0
        for key in eeg:
            c = checks[key]
            t0 = time.perf_counter()
            stats = []
            for j, b in enumerate(c["channels"]):
                stats.append(_lockstep_stats(lambda r, k: D @ r, c["grid"], [x[j] for x in c["rs"]], c["idx"][j],
                                             c["coef"][j], c["energy"][j]))
            res[key] = dict(_merge(stats), channels=c["channels"],
                            sample=f"channels {c['channels']}, every order, all 2,097,152 atoms scored by the "
                                   f"oracle's FP64 dictionary (built once in {build_s:.1f} s)",
                            seconds=time.perf_counter() - t0)
        del D
    if "ragged_uneven_batch" in checks:
        c = checks["ragged_uneven_batch"]
        t0 = time.perf_counter()
        stats = []
        for j, g in enumerate(c["grids"]):
            stats.append(_lockstep_stats(lambda r, k, g=g: oracle.scores_grid(g, r), g, c["rs"][j], c["idx"][j],
                                         c["coef"][j], c["energy"][j]))
        res["ragged_uneven_batch"] = dict(
            _merge(stats), channels=c["channels"],
            sample=f"channels {c['channels']} (windows 256 and 512) of the batch, first {len(c['idx'][0])} orders "
                   f"of a chained one-order plan, all 4,718,592 atoms regenerated and scored by the oracle",
            seconds=time.perf_counter() - t0)
    if "offgrid_refinement" in checks:
        c = checks["offgrid_refinement"]
        g = c["grid"]
        w, lo, hi = oracle.refine_box(g)
        t0 = time.perf_counter()
        same = bad = 0
        th_err = ce = ee = 0.0
        for j in range(len(c["channels"])):
            for k in range(c["idx"].shape[1]):
                r = np.asarray(c["rs"][k][j], dtype=np.float64)
                sc = oracle.scores_grid(g, r)
                best, second = oracle.select(sc)
                a = abs(sc[best])
                gap = (a - abs(sc[second])) / a if a > 0 else 0.0
                pick = int(c["idx"][j, k])
                same += pick == best
                bad += pick != best and gap > 1e-5
                th, _ = oracle.refine(oracle.atom_params(g, pick), g.fs, r, c["steps"], w, lo, hi)
                gg, _ = oracle.atom(*th, g.fs, g.n_samples)
                c_ref = float(gg @ r)
                e_ref = float(np.sum((r - c_ref * gg) ** 2))
                th_err = max(th_err, float(np.max(np.abs(c["theta"][j, k] - th) / w)))
                ce = max(ce, abs(float(c["coef"][j, k]) - c_ref) / abs(c_ref))
                ee = max(ee, abs(float(c["energy"][j, k]) - e_ref) / e_ref)
        n = c["idx"].size
        res["offgrid_refinement"] = {
            "orders": int(n), "same_grid_atom": int(same), "violations": int(bad),
            "max_theta_err_grid_steps": th_err, "max_coef_rel_err": ce, "max_energy_rel_err": ee,
            "channels": c["channels"],
            "sample": f"channel {c['channels']}, first {c['idx'].shape[1]} orders of chained one-order calls: the "
                      f"oracle scores all 8,388,608 atoms, then runs its FP64 BFGS ({c['steps']} iterations) from "
                      f"the GPU's grid pick",
            "seconds": time.perf_counter() - t0}
    if "hierarchical_lem" in checks:
        c = checks["hierarchical_lem"]
        g = c["grid"]
        axes = [g.tc, g.fc, g.logdt, g.c]
        lo = np.array([min(a.lo, a.lo + (a.count - 1) * a.step) for a in axes])
        hi = np.array([max(a.lo, a.lo + (a.count - 1) * a.step) for a in axes])
        w, blo, bhi = oracle.refine_box(g)
        steps = ((64, 2, 2, 5), (32, 1, 1, 2.5), (16, 0.5, 0.5, 0.5))
        n_coarse = int(np.prod([max(1.0, np.ceil((h_ - l_) / s_)) for l_, h_, s_ in zip(lo, hi, steps[0])]))
        params = oracle.lem_params(n_coarse, 4, 2, steps, (2, 2, 1, 2))
        t0 = time.perf_counter()
        ce = ee = 0.0
        first_div = []
        for j, b in enumerate(c["channels"]):
            th, co, _, en = oracle.mp_lem(params, lo, hi, w, blo, bhi, g.fs, c["signals"][j], c["P"], c["steps"],
                                          c["seed"], b)
            ce = max(ce, float(np.max(np.abs(np.abs(c["coef"][j]) - np.abs(co)) / np.abs(co))))
            ee = max(ee, float(np.max(np.abs(c["energy"][j] - en) / en)))
            d = np.max(np.abs(c["theta"][j] - th) / w, axis=1)
            first_div.append(int(np.argmax(d > 1e-3)) if np.any(d > 1e-3) else c["P"])
        res["hierarchical_lem"] = {
            "orders": len(c["channels"]) * c["P"], "max_abs_coef_rel_err": ce, "max_energy_rel_err": ee,
            "orders_before_parameters_differ_1e-3_steps": first_div, "channels": c["channels"],
            "sample": f"channels {c['channels']}, all {c['P']} orders: the oracle runs the same hierarchical search "
                      f"(same SplitMix64 draws) and FP64 BFGS ({c['steps']} iterations) on its own trajectory",
            "seconds": time.perf_counter() - t0}
    res["_seconds"] = time.perf_counter() - t_all
    return res


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
    if args.headline_gemv == "stream":
        act.act_set_tuning(h, -1)  # the bulk-copy streaming GEMV (the autotuner's pick on an idle GPU)
    else:
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
    checks = {"headline": dict(kind="lockstep", grid=grid, channels=[channel],
                               **_chain(act, torch, h, sig_np[None, :], P, dev, stream))}
    act.act_destroy(h)
    fp32_picks = atoms.clone()

    shift = None
    if not args.no_shift:
        shift = bench_shift(args, dev, stream, ms / args.steps, fp32_picks, clk.summary(), peaks, peak_kind, checks)
    bf16 = None
    if not args.no_bf16:
        bf16 = bench_bf16(args, dev, stream, peaks, peak_kind, checks)
    ragged = None
    if not args.no_ragged:
        ragged = bench_ragged(args, dev, stream, peaks, peak_kind, checks)
    refine = None
    if not args.no_refine:
        refine = bench_refine(args, dev, stream, peaks, peak_kind, checks)
    small = None
    if not args.no_small:
        small = bench_small_check(args, dev, stream)
    context = None
    if not args.no_context:
        context = bench_paper_context(args, dev, stream)
    lem = None
    if not args.no_lem:
        lem = bench_lem(args, dev, stream, peaks, peak_kind, checks)
    sweep = None
    if not args.no_sweep:
        sweep = bench_sweep(args, dev, stream, peaks, peak_kind)

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
        if context is not None:
            line["paper_epoch_context"] = context
        if sweep is not None:
            line["channel_sweep"] = sweep
        line["targets"] = _targets(roofline, shift, bf16)
        if not args.no_cpu_baseline and world == 1:
            # the oracle leg: the CPU baseline, then the error of every
            # section's results against the FP64 oracle
            line["cpu_baseline"] = cpu_baseline()
            oc = oracle_checks(checks)
            line["oracle_check"] = oc["headline"]
            if "template_shift" in line and "template_shift_64ch" in oc:
                line["template_shift"]["channels_64"]["oracle_check"] = oc["template_shift_64ch"]
            for key in ("bf16_batched", "ragged_uneven_batch", "offgrid_refinement", "hierarchical_lem"):
                if key in line and key in oc:
                    line[key]["oracle_check"] = oc[key]
            line["oracle_check"]["all_sections_seconds"] = oc["_seconds"]
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


def _chain(act, torch, h, sig_np, P, dev, stream):
    """P one-order decompositions of the channels sig_np [B][L], each fed the
    residual of the one before: the residual entering every order (float32
    [P+1][B][L]), and the selected flat index, coefficient and |r_{k+1}|^2 of
    every order ([B][P]).  This is what the FP64 oracle checks order by order
    (from the GPU's own residual, Sec. III-A lock-step)."""
    B, L = sig_np.shape
    r = torch.tensor(np.asarray(sig_np, dtype=np.float32), device=dev)
    rs, idx, coef, en, th = [r.cpu().numpy()], [], [], [], []
    for _ in range(P):
        a, c, res, e = (torch.empty((B, 1, act.ATOM_BYTES), dtype=torch.uint8, device=dev),
                        torch.empty((B, 1), dtype=torch.float32, device=dev),
                        torch.empty((B, L), dtype=torch.float32, device=dev),
                        torch.empty((B, 2), dtype=torch.float64, device=dev))
        act.act_decompose(h, r, B, 1, a, c, res, e, stream)
        torch.cuda.synchronize(dev)
        idx.append(act.atom_indices(a).cpu().numpy()[:, 0])
        th.append(act.atom_params(a).cpu().numpy()[:, 0])
        coef.append(c.cpu().numpy()[:, 0])
        en.append(e.cpu().numpy()[:, 1])
        r = res
        rs.append(r.cpu().numpy())
    st = act.act_grid_status(h, stream)
    if st != act.ACT_OK:
        raise RuntimeError(act.status_name(st))
    return {"rs": np.stack(rs), "idx": np.stack(idx, 1), "coef": np.stack(coef, 1), "energy": np.stack(en, 1),
            "theta": np.stack(th, 1)}


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
    while bg < B and bg < 32:
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


def bench_shift(args, dev, stream, fp32_ms_per_step, fp32_atoms, clocks, peaks, peak_kind, checks):
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
        pairs64 = act.act_get_cta_pairs(h, B)
        # the same search with one SM per MMA (cta_group::1), for comparison
        act.act_set_cta_pairs(h, False)
        s64 = _time_decompose(act, torch, h, sig64, P, 2, stream, dev)
        act.act_set_cta_pairs(h, True)
        act.act_set_search(h, act.ACT_SEARCH_SHIFT)
        f64 = _time_decompose(act, torch, h, sig64, P, 2, stream, dev)
        act.act_set_search(h, act.ACT_SEARCH_SHIFT_BF16)
        chans = [0, 21, 42, 63]
        checks["template_shift_64ch"] = dict(kind="lockstep", grid=grid, channels=chans,
                                             **_chain(act, torch, h, w3.signals[chans], P, dev, stream))
    finally:
        act.act_destroy(h)
    same_fp32 = all(torch.equal(a, b) for a, b in zip(f1[5], t1[5])) and \
        all(torch.equal(a, b) for a, b in zip(f64[5], t64[5])) and \
        all(torch.equal(a, b) for a, b in zip(s64[5], t64[5]))
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
    tc_peak = peaks["bf16_tflops"]  # burst: the timed region is a few ms, not a seconds-long loop
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
                "cta_pairs": pairs64, "single_sm_rows_gemm_ms_per_order": s64[2],
                "resolved_items_fallbacks": fb,
                "roofline": {"bound": "tensor", "achieved": alg64, "peak": tc_peak, "unit": "TFLOP/s",
                             "frac": alg64 / tc_peak,
                             "traffic": _profile_traffic("shift_gemm_tc_eeg_b64.md",
                                                         ["paper_2607_16629_gb300/csrc/act_shift_tc.cu",
                                                          "paper_2607_16629_gb300/csrc/act_tc.cuh",
                                                          "paper_2607_16629_gb300/csrc/act_device.cuh"]),
                             "kernel": "k_shift_rows + k_shift_gemm<256, pair> (BF16 tcgen05 on CTA pairs, "
                                       "scaled tile maxima)",
                             "algorithmic_flops_per_launch": 2.0 * B * K * L,
                             "mma_flops_per_launch": mma_flops, "mma_tflops": mma64,
                             "mma_frac": mma64 / tc_peak, "avg_launch_ms": t64[2],
                             "peak_source": f"{peak_kind} bf16_tflops (burst: a decomposition takes ms)",
                             "note": "each 128-row tile (32 channels x 4 time centres) multiplies the 64-lag "
                                     "chunks its windows touch (9 of Kt / 64 = 16): achieved counts 2 K L flops "
                                     "per channel, mma_tflops everything the tensor cores execute; timed by an "
                                     "event pair around the shifted-row build and the GEMM"}}}


def bench_bf16(args, dev, stream, peaks, peak_kind, checks):
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
    act.act_set_profiling(h, False)
    chans = [0, 21, 42, 63]
    checks["bf16_batched"] = dict(kind="lockstep", grid=w.grid, channels=chans,
                                  **_chain(act, torch, h, w.signals[chans], P, dev, stream))
    # plain FP32 comparator: the same 64 channels, one FP32 GEMV decomposition each,
    # with the GEMV tuned for one channel
    act.act_set_search(h, act.ACT_SEARCH_FP32)
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
                         "tensor_frac_of_bf16_peak": tflops / peaks["bf16_tflops"],
                         "tensor_peak_source": f"{peak_kind} bf16_tflops (burst)",
                         "avg_search_ms_per_order": avg,
                         "search_frac_of_hbm_roofline": bytes_per / (avg / 1e3) / 1e9 / peaks["hbm_gbs"]},
            "autotuned": {"tile_atoms": tile_atoms, "stages": stages_used, "search_ms_per_order": tune_ms},
            "orders_resolved_by_block_rescan": c1 - c0, "blocks_rescanned": s1 - s0,
            "orders_full_fp32_fallback": f1 - f0,
            "fp32_plain_per_channel": {"value": B * K * P / (fp32_ms / 1e3), "ms": fp32_ms},
            "speedup_vs_fp32_plain": (B * K * P * steps / (ms / 1e3)) / (B * K * P / (fp32_ms / 1e3)),
            "gpu_launches": kernels * steps}


def _ragged_run(act, torch, synth, sigs, lengths, offsets, P, dict_mode, steps, dev, stream, chain=None):
    """One ragged plan over per-length grids built with dict_mode: ms per
    decomposition of all channels, build seconds, device bytes held by the
    grids and the plan, plan info, and the selected flat indices.  With
    chain = (orders, channels): a one-order plan over the same grids is also
    chained that many orders, and the residual entering every order of the
    listed channels is returned for the oracle check."""
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
        payload = None
        if chain:
            n_ord, chans = chain
            plan1 = act.act_ragged_plan_create([handles[L] for L in lengths], offsets, 1)
            try:
                o1 = [torch.empty((C, 1, act.ATOM_BYTES), dtype=torch.uint8, device=dev),
                      torch.empty((C, 1), dtype=torch.float32, device=dev), None,
                      torch.empty((C, 2), dtype=torch.float64, device=dev)]
                r = flat
                rs, idx, coef, en = [r.cpu().numpy()], [], [], []
                for _ in range(n_ord):
                    o1[2] = torch.empty_like(flat)
                    act.act_ragged_decompose(plan1, r, *o1, stream)
                    torch.cuda.synchronize(dev)
                    idx.append(act.atom_indices(o1[0]).cpu().numpy()[:, 0])
                    coef.append(o1[1].cpu().numpy()[:, 0])
                    en.append(o1[3].cpu().numpy()[:, 1])
                    r = o1[2]
                    rs.append(r.cpu().numpy())
            finally:
                act.act_ragged_plan_destroy(plan1)
            payload = {"kind": "lockstep_ragged", "channels": list(chans),
                       "grids": [synth.grid_emg(len(sigs[c])) for c in chans],
                       "rs": [[x[offsets[c]:offsets[c + 1]] for x in rs] for c in chans],
                       "idx": np.stack(idx, 1)[chans], "coef": np.stack(coef, 1)[chans],
                       "energy": np.stack(en, 1)[chans]}
    finally:
        for h in handles.values():
            act.act_destroy(h)
    return ms, build_s, int(used), groups, kernels, idx_out, payload


def bench_ragged(args, dev, stream, peaks, peak_kind, checks):
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
    # the oracle check takes the first channel of window 256 and of window 512
    chk = [next(i for i, x in enumerate(sigs) if len(x) == L) for L in (256, 512)]
    t_ms, t_build, t_bytes, groups, kernels, t_idx, payload = _ragged_run(
        act, torch, synth, sigs, lengths, offsets, P, act.ACT_DICT_RECOMPUTE, steps, dev, stream, chain=(3, chk))
    checks["ragged_uneven_batch"] = payload
    d_ms, d_build, d_bytes, _, d_kernels, d_idx, _ = _ragged_run(act, torch, synth, sigs, lengths, offsets, P,
                                                                  act.ACT_DICT_BF16, steps, dev, stream)
    bf16_bytes = sum(K * L * 2 for L in lengths)
    counts = {L: sum(1 for x in sigs if len(x) == L) for L in lengths}
    # algorithmic flops of the projections P = D X^T: 2 K N per channel and order
    flops = 2.0 * K * float(sum(len(x) for x in sigs)) * P
    achieved = flops / (t_ms / 1e3) / 1e12
    return {"workload": "emg_like_ragged_256ch_n256-2048_fs500_grid256x96x8x24_k4718592_p30",
            "value": C * K * P / (t_ms / 1e3), "unit": UNIT, "atoms_per_s": C * P / (t_ms / 1e3),
            "ms_per_step": t_ms, "steps": steps, "channels_per_length": counts,
            "search": "template dictionaries, tensor-core template search (atoms generated in-kernel)",
            "dictionary_build_s": t_build, "device_bytes": t_bytes, "length_groups": groups,
            "gpu_launches": kernels * steps,
            "roofline": {"bound": "tensor", "achieved": achieved, "peak": peaks["bf16_tflops"], "unit": "TFLOP/s",
                         "frac": achieved / peaks["bf16_tflops"], "traffic": None,
                         "kernel": "whole decomposition (shifted rows + k_shift_gemm + flag + rescore + update, "
                                   "four length groups as graph branches)",
                         "algorithmic_flops_per_step": flops,
                         "peak_source": f"{peak_kind} bf16_tflops (burst: a decomposition takes tens of ms)",
                         "note": "achieved = 2 K sum(N_i) flops per order x 30 orders / the event-timed "
                                 "decomposition, every kernel of the step included: a lower bound on the "
                                 "GEMM's own fraction"},
            "stored_bf16_dictionaries": {
                "value": C * K * P / (d_ms / 1e3), "unit": UNIT, "ms_per_step": d_ms,
                "dictionary_build_s": d_build, "device_bytes": d_bytes, "gpu_launches": d_kernels * steps,
                "hbm_frac_of_bf16_dictionary_stream": bf16_bytes * P / (d_ms / 1e3) / 1e9 / peaks["hbm_gbs"],
                "same_selections_as_template_search": float(np.mean(d_idx == t_idx)),
                "dtype": "bf16 x bf16 -> f32 (tensor cores), f32 tile rescan"},
            "dtype": "bf16 x bf16 -> f32 (tensor cores), f32 rescore"}


def bench_paper_context(args, dev, stream):
    """Context only, no ratio formed: the setting of the paper's 1-s EEG
    epoch timings (Sec. IV-B/C: Table 2's EEG ranges with the time-centre
    step raised from 16 to 32 samples, i.e. tc 0..256 step 32, fc 0.5..15 Hz
    step 0.5, logDt -4..1 step 0.5, c -10..10 Hz/s step 0.5, half-open:
    92,800 atoms; N = 256 at 256 Hz; order 10) on one synthetic EEG-like
    epoch.  The paper's per-epoch times there (CPU 0.019 s, CuPy hybrid
    0.009 s, PyTorch hybrid 0.007 s on an RTX 5070 with an i9-14900K) are of
    a Python pipeline that refines every order by BFGS on the CPU and moves
    data between host and device; here: the grid-only decomposition, the
    same with 20 BFGS iterations per order on the GPU, and the latter with
    the epoch and results in host memory (copies inside the timing)."""
    import torch

    from paper_2607_16629_gb300 import act, synth
    desc = act.act_grid_from_ranges(256, 256.0, (0, 256, 32), (0.5, 15, 0.5), (-4, 1, 0.5), (-10, 10, 0.5))
    L, P = 256, 10
    sig_np = synth.eeg_like_signal(6, 0, n_samples=L, fs=256.0)[0][None, :].astype(np.float32)
    h = act.act_grid_create(desc, dev.index)
    try:
        K, _ = act.act_grid_size(h)
        act.act_dictionary_build(h, act.ACT_DICT_FP32, stream)
        sig = torch.tensor(sig_np, device=dev)
        out = [torch.empty((1, P, act.ATOM_BYTES), dtype=torch.uint8, device=dev),
               torch.empty((1, P), dtype=torch.float32, device=dev),
               torch.empty((1, L), dtype=torch.float32, device=dev),
               torch.empty((1, P + 1), dtype=torch.float64, device=dev)]
        host = [torch.empty(t.shape, dtype=t.dtype).pin_memory() for t in out]
        hsig = torch.tensor(sig_np).pin_memory()

        def timed(args_out, signal, reps=100):
            for _ in range(5):
                act.act_decompose(h, signal, 1, P, *args_out, stream)
            torch.cuda.synchronize(dev)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(reps):
                act.act_decompose(h, signal, 1, P, *args_out, stream)
            e1.record(stream)
            torch.cuda.synchronize(dev)
            st = act.act_grid_status(h, stream)
            if st != act.ACT_OK:
                raise RuntimeError(act.status_name(st))
            return e0.elapsed_time(e1) / reps

        grid_ms = timed(out, sig)
        act.act_set_refinement(h, 20)
        refined_ms = timed(out, sig)
        refined_host_ms = timed(host, hsig)
        coef = host[1].numpy()[0]
        energy = host[3].numpy()[0]
    finally:
        act.act_destroy(h)
    return {"workload": "paper_1s_eeg_epoch_setting_n256_fs256_grid8x29x10x40_k92800_p10",
            "atoms": K, "orders": P,
            "grid_only_ms_per_epoch": grid_ms, "refined_ms_per_epoch": refined_ms,
            "refined_host_buffers_ms_per_epoch": refined_host_ms,
            "normalised_residue_refined": float(energy[-1] / energy[0]),
            "first_coefficient": float(coef[0]),
            "paper_per_epoch_s": {"cpu": 0.019, "cupy_hybrid": 0.009, "torch_hybrid": 0.007},
            "note": "context only: the paper's times are of its own pipeline (real Bitbrain EEG epochs, CPU BFGS "
                    "to its own stopping rule, host transfers, Python) on an RTX 5070 + i9-14900K"}


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
        reps = 200

        def timed():
            for _ in range(5):
                act.act_decompose(h, sig, B, P, *out, stream)
            torch.cuda.synchronize(dev)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(reps):
                act.act_decompose(h, sig, B, P, *out, stream)
            e1.record(stream)
            torch.cuda.synchronize(dev)
            st = act.act_grid_status(h, stream)
            if st != act.ACT_OK:
                raise RuntimeError(act.status_name(st))
            return e0.elapsed_time(e1) / reps

        fused_ctas = act.act_get_fused(h, B)
        ms = timed()  # the default: one cooperative launch per decomposition
        act.act_set_fused(h, 0)
        ms_kernels = timed()  # the GEMV and update kernels of every order, in the grid's graph
        gemv = act.act_get_tuning(h)[0]
    finally:
        act.act_destroy(h)
    return {"workload": "plain_fp32_1ch_n256_fs128_grid32x16x4x8_k16384_p5", "value": B * K * P / (ms / 1e3),
            "unit": UNIT, "ms_per_step": ms, "us_per_order": 1e3 * ms / P, "steps": reps,
            "bound": "latency (the 16.8 MB dictionary is L2-resident)",
            "form": f"single cooperative launch per decomposition, {fused_ctas} CTAs (act_set_fused)",
            "per_order_kernels": {"us_per_order": 1e3 * ms_kernels / P,
                                  "gemv": "bulk-copy stream" if gemv == -1 else f"load-streaming, {gemv} CTAs"},
            "l2": "dictionary smaller than L2: every step after the first reads it from L2"}


def _refine_runs(act, torch, w, dict_mode, steps_list, n, dev, stream, chain=None):
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
            if chain and steps > 0:
                n_ord, chans = chain
                res["chain"] = dict(kind="lockstep_refined", grid=w.grid, channels=list(chans), steps=steps,
                                    **_chain(act, torch, h, w.signals[chans], n_ord, dev, stream))
    finally:
        act.act_destroy(h)
    return res


def bench_refine(args, dev, stream, peaks, peak_kind, checks):
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
    t = _refine_runs(act, torch, w, act.ACT_DICT_RECOMPUTE, (0, 20), n, dev, stream, chain=(2, [0]))
    checks["offgrid_refinement"] = t.pop("chain")
    d = _refine_runs(act, torch, w, act.ACT_DICT_BF16, (20,), n, dev, stream)
    extra_ms = t[20]["ms_per_step"] - t[0]["ms_per_step"]
    # k_refine against the instruction-issue roof: its warp instructions per
    # launch (ncu) over the refinement time of one order
    files = ["paper_2607_16629_gb300/csrc/act_refine.cu", "paper_2607_16629_gb300/csrc/act_ff.cuh",
             "paper_2607_16629_gb300/csrc/act_device.cuh"]
    inst = _profile_value("refine_radar_b32.md", "inst_executed_per_launch", files)
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    issue_peak = sms * 4 * 2.07  # G warp-instructions/s at the maximum SM clock
    ref_ms = extra_ms / P
    refine_roof = {"bound": "alu", "unit": "G warp-inst/s", "peak": issue_peak,
                   "achieved": (inst / (ref_ms / 1e3) / 1e9) if inst else None,
                   "frac": (inst / (ref_ms / 1e3) / 1e9 / issue_peak) if inst else None,
                   "traffic": _profile_traffic("refine_radar_b32.md", files),
                   "kernel": "k_refine (BFGS on -|<g(theta), r>|, float-float sums)",
                   "inst_executed_per_launch": inst, "avg_launch_ms": ref_ms,
                   "peak_source": f"issue roof: {sms} SMs x 4 schedulers x 1 warp-instruction/clk x 2.07 GHz",
                   "timing": "refined minus grid-only decomposition time, per order (event-timed)"}
    same = bool(torch.equal(t[20]["coefs"], d[20]["coefs"]))
    for r in (t[0], t[20], d[20]):
        r.pop("coefs")
    return {"workload": "radar_like_32ch_n1024_fs1000_grid256x128x8x32_k8388608_p10_bfgs20",
            "value": t[20]["projections_per_s"], "unit": UNIT, "ms_per_step": t[20]["ms_per_step"],
            "search": "template dictionary, tensor-core template search (atoms generated in-kernel)",
            "grid_only": t[0], "refined": t[20],
            "bfgs_iterations_per_s": B * P * 20 / (max(extra_ms, 1e-6) / 1e3),
            "refinement_ms_per_order": extra_ms / P,
            "roofline": refine_roof,
            "stored_dictionary_refined": d[20],
            "same_coefficients_as_stored_dictionary": same,
            "dtype": "bf16 search + f32 rescore; refinement f32 samples, f64 sums"}


def bench_lem(args, dev, stream, peaks, peak_kind, checks):
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
            if name == "lem":
                chans = [0, 1]
                checks["hierarchical_lem"] = dict(kind="lem_trajectory", grid=w.grid, channels=chans,
                                                  signals=w.signals[chans], P=P, steps=20, seed=0,
                                                  theta=act.atom_params(out[0]).cpu().numpy()[chans],
                                                  coef=out[1].cpu().numpy()[chans], energy=en[chans])
                # the hierarchical search's own time per order (event pairs in the graph)
                act.act_set_profiling(h, True)
                act.act_decompose(h, sig, B, P, *out, stream)
                search_ms, _, n_ord, _ = act.act_profile_read(h)
                act.act_set_profiling(h, False)
                res[name]["search_ms_per_order"] = search_ms / max(1, n_ord)
        finally:
            act.act_destroy(h)
    # candidates scored per channel and order: the coarse Latin hypercube
    # plus two levels of top_k x 375 neighbours (2,048 + 2 x 1,500 on this machine)
    cand = 2048 + 2 * 4 * 375
    samples = cand * B * L
    files = ["paper_2607_16629_gb300/csrc/act_lem.cu", "paper_2607_16629_gb300/csrc/act_ff.cuh",
             "paper_2607_16629_gb300/csrc/act_device.cuh"]
    ips = _profile_value("lem_score_eeg_b64.md", "inst_per_sample", files)
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    roof = sms * 4 * 32 * 2.07 / ips if ips else None  # G samples/s at the issue roof
    got = samples / (res["lem"]["search_ms_per_order"] / 1e3) / 1e9
    lem_roof = {"bound": "alu", "unit": "G samples/s", "achieved": got, "peak": roof,
                "frac": got / roof if roof else None,
                "traffic": _profile_traffic("lem_score_eeg_b64.md", files),
                "kernel": "hierarchical search per order (k_lem_lhs, k_lem_score x 3 levels, k_lem_topk, k_lem_neigh)",
                "samples_per_order": samples, "inst_per_sample": ips,
                "peak_source": f"issue roof of k_lem_score: {sms} SMs x 4 schedulers x 32 lanes x 2.07 GHz / "
                               "its warp instructions per sample (ncu)",
                "timing": "event pair around the whole hierarchical search of every order in the graph: a lower "
                          "bound on the scoring kernel's own fraction"}
    return {"workload": "eeg_like_64ch_n512_box128x64x8x32_p20_bfgs20", "lem": res["lem"],
            "dense_bf16": res["dense_bf16"], "roofline": lem_roof,
            "lem_settings": "paper EEG settings: top_k 4, 2 levels, steps (64,2,2,5)/(32,1,1,2.5)/(16,.5,.5,.5), "
                            "radius (2,2,1,2), 2048 LHS samples"}


def bench_sweep(args, dev, stream, peaks, peak_kind):
    """Channel sweep of both tensor-core searches on the 2,097,152-atom
    EEG-like grid (N = 512): B in {1, 8, 32, 64, 128, 256, 512, 1024}
    EEG-like channels (seeds of config 3, channel b), 3 orders per
    decomposition.  Per B: the whole search per order and its GEMM part (CUDA
    event pairs inside the graph), the GEMM's algorithmic tensor throughput
    2 B K N / t against the burst BF16 peak, and for the dense dictionary its
    stream rate 2 K Lb / t against the HBM copy peak (the batch at which the
    GEMM turns from HBM- to tensor-bound, Sec. V-A's channel scaling)."""
    import torch

    from paper_2607_16629_gb300 import act, synth
    grid = synth.grid_eeg()
    K, L, P = grid.n_atoms, grid.n_samples, 3
    Bs = [1, 8, 32, 64, 128, 256, 512, 1024]
    sig_all = torch.tensor(np.stack([synth.eeg_like_signal(3, b)[0] for b in range(max(Bs))]),
                           dtype=torch.float32, device=dev)
    tc_peak = peaks["bf16_tflops"]
    out = {"workload": "eeg_like_n512_k2097152_p3_channel_sweep", "orders": P,
           "peak_source": f"{peak_kind} bf16_tflops (burst) and hbm_gbs", "dense_bf16": [], "template_bf16": []}
    for name, build, search in (("dense_bf16", act.ACT_DICT_BF16, act.ACT_SEARCH_BF16),
                                ("template_bf16", act.ACT_DICT_RECOMPUTE, act.ACT_SEARCH_SHIFT_BF16)):
        h = act.act_grid_create(grid, dev.index)
        try:
            act.act_dictionary_build(h, build, stream)
            act.act_set_search(h, search)
            for B in Bs:
                sig = sig_all[:B].contiguous()
                ms, search_ms, core_ms, _, _, _ = _time_decompose(act, torch, h, sig, P, 3, stream, dev)
                tflops = 2.0 * B * K * L / (core_ms / 1e3) / 1e12
                row = {"channels": B, "ms_per_decomposition": ms, "search_ms_per_order": search_ms,
                       "gemm_ms_per_order": core_ms, "gemm_tflops_algorithmic": tflops,
                       "tensor_frac": tflops / tc_peak}
                if name == "dense_bf16":
                    gbs = 2.0 * K * L / (core_ms / 1e3) / 1e9
                    row.update({"gemm_gbs": gbs, "hbm_frac": gbs / peaks["hbm_gbs"]})
                else:
                    mma = _tc_mma_flops(grid, B) / (core_ms / 1e3) / 1e12
                    row.update({"gemm_tflops_executed": mma, "executed_tensor_frac": mma / tc_peak})
                out[name].append(row)
        finally:
            act.act_destroy(h)
    return out


def run_profile_case(args):
    """Small, self-checking cases for ncu captures: a few launches of one
    search kernel on a dictionary larger than L2 but a few GB at most.
      gemv_small: FP32 GEMV over 1,048,576 EEG-grid atoms (2.1 GB), 1 channel.
      bf16_small: BF16 GEMM search over the same atoms, 64 channels.
      fused_check: the 16,384-atom check workload (5 orders), one cooperative
        launch per decomposition."""
    import torch

    from paper_2607_16629_gb300 import act, synth
    if args.case == "fused_check":
        w = synth.workload_c1()
        sig = torch.tensor(w.signals[:1], dtype=torch.float32, device="cuda")
        h = act.act_grid_create(w.grid, 0)
        try:
            act.act_dictionary_build(h, act.ACT_DICT_FP32)
            ctas = act.act_get_fused(h, 1)
            assert ctas > 0
            for _ in range(args.steps):
                atoms, _, _, energy = act.decompose(h, sig, w.n_atoms)
            torch.cuda.synchronize()
            st = act.act_grid_status(h)
            if st != act.ACT_OK:
                raise RuntimeError(act.status_name(st))
            assert np.all(np.diff(energy.cpu().numpy(), axis=1) <= 0.0)
        finally:
            act.act_destroy(h)
        print(json.dumps({"case": args.case, "atoms": w.grid.n_atoms, "channels": 1, "ctas": ctas, "ok": True}))
        return
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
    ap.add_argument("--no-context", action="store_true")
    ap.add_argument("--no-sweep", action="store_true")
    ap.add_argument("--channels", type=int, default=1, help="channels for the shift_* and lem_eeg cases (1 or up to 64)")
    ap.add_argument("--headline-gemv", default="auto", choices=["auto", "stream"],
                    help="the headline's FP32 GEMV: autotuned, or the bulk-copy stream fixed (for profiler runs, "
                         "under which the autotuner's timings are not representative)")
    ap.add_argument("--gemv", default="stream", choices=["stream", "load"],
                    help="FP32 GEMV of the gemv_small case: bulk-copy streaming or load-streaming")
    ap.add_argument("--shift-tuning", default="", help="JxW, JxWxS or JxWxSxC for --case shift_eeg (default: the build's)")
    ap.add_argument("--case", default="default",
                    choices=["default", "gemv_small", "bf16_small", "fused_check", "shift_eeg", "shift_tc_eeg",
                             "lem_eeg", "refine_radar"],
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
