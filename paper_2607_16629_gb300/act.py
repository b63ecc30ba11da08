"""Python binding of the C ABI in include/act.h (argument marshalling only).

Every function here has the name of the C entry point it calls and does
nothing but convert arguments: tensors become raw pointers, the current torch
stream becomes a cudaStream_t, and a non-OK status becomes an ActError.  All
arithmetic runs inside libact.so.  There is no CPU fallback: if the library
has not been built, the first call raises.
"""
from __future__ import annotations

import ctypes
import os
import threading
from typing import Optional

PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(PKG, "libact.so")

ACT_OK = 0
ACT_ERR_INVALID_ARG = 1
ACT_ERR_OOM = 2
ACT_ERR_CUDA = 3
ACT_ERR_NONFINITE = 4
ACT_ERR_DEVICE_TIMEOUT = 5
ACT_ERR_NOT_BUILT = 6
ACT_ERR_UNSUPPORTED = 7

ACT_DICT_AUTO, ACT_DICT_FP32, ACT_DICT_BF16, ACT_DICT_RECOMPUTE = 0, 1, 2, 3
ACT_SEARCH_AUTO, ACT_SEARCH_FP32, ACT_SEARCH_BF16, ACT_SEARCH_LEM, ACT_SEARCH_SHIFT, ACT_SEARCH_SHIFT_BF16 = range(6)

# Every symbol include/act.h declares (checked by the CPU tests).
EXPORTS = (
    "act_status_string", "act_last_error_message", "act_grid_from_ranges", "act_grid_create",
    "act_grid_size", "act_dictionary_build", "act_set_search", "act_decompose", "act_project",
    "act_dictionary_rows", "act_grid_status", "act_set_profiling", "act_profile_read",
    "act_bf16_stats", "act_destroy", "act_search_noalloc", "act_autotune", "act_get_tuning", "act_set_tuning",
    "act_ragged_plan_create", "act_ragged_decompose", "act_ragged_plan_info", "act_ragged_plan_destroy",
    "act_set_refinement", "act_chirplet_score", "act_set_lem", "act_set_shift_tuning", "act_get_shift_tuning",
    "act_dictionary_mode", "act_set_memory_budget", "act_set_wait_limit", "act_inject_alloc_failure",
    "act_set_cta_pairs", "act_get_cta_pairs", "act_set_fused", "act_get_fused",
)


class act_axis(ctypes.Structure):
    _fields_ = [("lo", ctypes.c_double), ("step", ctypes.c_double), ("count", ctypes.c_int32)]


class act_grid_desc(ctypes.Structure):
    _fields_ = [("n_samples", ctypes.c_int32), ("fs", ctypes.c_double), ("tc", act_axis),
                ("fc", act_axis), ("logdt", act_axis), ("c", act_axis)]


class act_atom(ctypes.Structure):
    _fields_ = [("tc", ctypes.c_double), ("fc", ctypes.c_double), ("logdt", ctypes.c_double),
                ("c", ctypes.c_double), ("flat_index", ctypes.c_int64)]


ATOM_BYTES = ctypes.sizeof(act_atom)  # 40


class act_lem_params(ctypes.Structure):
    _fields_ = [("n_coarse", ctypes.c_int32), ("top_k", ctypes.c_int32), ("levels", ctypes.c_int32),
                ("steps", (ctypes.c_double * 4) * 3), ("radius", ctypes.c_int32 * 4), ("seed", ctypes.c_uint64)]


class ActError(RuntimeError):
    def __init__(self, status: int, call: str, detail: str = ""):
        self.status = status
        msg = f"{call} -> {status_name(status)}"
        if detail:
            msg += f" ({detail})"
        super().__init__(msg)


_lock = threading.Lock()
_lib = None
_P = ctypes.c_void_p


def load_library(path: str = LIB_PATH):
    """Loads libact.so (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(path):
            raise RuntimeError(f"{path} is missing: build it with __graft_entry__.build() "
                               "(the CUDA library is required; there is no CPU fallback)")
        lib = ctypes.CDLL(path)
        lib.act_status_string.restype = ctypes.c_char_p
        lib.act_status_string.argtypes = [ctypes.c_int]
        lib.act_last_error_message.restype = ctypes.c_char_p
        lib.act_last_error_message.argtypes = []
        d3 = ctypes.POINTER(ctypes.c_double)
        lib.act_grid_from_ranges.argtypes = [ctypes.c_int32, ctypes.c_double, d3, d3, d3, d3,
                                             ctypes.POINTER(act_grid_desc)]
        lib.act_grid_create.argtypes = [ctypes.POINTER(act_grid_desc), ctypes.c_int32, ctypes.POINTER(_P)]
        lib.act_grid_size.argtypes = [_P, ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int32)]
        lib.act_dictionary_build.argtypes = [_P, ctypes.c_int, _P]
        lib.act_set_search.argtypes = [_P, ctypes.c_int]
        lib.act_decompose.argtypes = [_P, _P, ctypes.c_int32, ctypes.c_int32, _P, _P, _P, _P, _P]
        lib.act_project.argtypes = [_P, _P, ctypes.c_int32, _P, _P]
        lib.act_dictionary_rows.argtypes = [_P, ctypes.c_int64, ctypes.c_int64, _P, _P]
        lib.act_grid_status.argtypes = [_P, _P]
        lib.act_set_profiling.argtypes = [_P, ctypes.c_int32]
        lib.act_profile_read.argtypes = [_P, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double),
                                         ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_int32)]
        lib.act_bf16_stats.argtypes = [_P, ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int64),
                                       ctypes.POINTER(ctypes.c_int64)]
        lib.act_search_noalloc.argtypes = [_P, ctypes.c_int64, ctypes.c_int32, _P, ctypes.c_int32, _P, _P, _P]
        lib.act_autotune.argtypes = [_P, _P, ctypes.c_int32, _P, ctypes.POINTER(ctypes.c_double)]
        lib.act_get_tuning.argtypes = [_P, ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_int32),
                                       ctypes.POINTER(ctypes.c_int32)]
        lib.act_set_tuning.argtypes = [_P, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32]
        lib.act_ragged_plan_create.argtypes = [_P, ctypes.c_int32, _P, ctypes.c_int32, ctypes.c_int32,
                                               ctypes.POINTER(_P)]
        lib.act_ragged_decompose.argtypes = [_P, _P, _P, _P, _P, _P, _P]
        lib.act_ragged_plan_info.argtypes = [_P, ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_int32)]
        lib.act_ragged_plan_destroy.argtypes = [_P]
        lib.act_ragged_plan_destroy.restype = None
        lib.act_set_refinement.argtypes = [_P, ctypes.c_int32]
        lib.act_chirplet_score.argtypes = [ctypes.c_int32, ctypes.c_double, _P, _P, ctypes.c_int32, _P, _P, _P, _P]
        lib.act_set_lem.argtypes = [_P, ctypes.POINTER(act_lem_params)]
        lib.act_set_shift_tuning.argtypes = [_P, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32]
        lib.act_get_shift_tuning.argtypes = [_P] + [ctypes.POINTER(ctypes.c_int32)] * 4
        lib.act_dictionary_mode.argtypes = [_P, ctypes.POINTER(ctypes.c_int32)]
        lib.act_set_memory_budget.argtypes = [_P, ctypes.c_uint64]
        lib.act_set_wait_limit.argtypes = [_P, ctypes.c_int64]
        lib.act_inject_alloc_failure.argtypes = [ctypes.c_int32]
        lib.act_set_cta_pairs.argtypes = [_P, ctypes.c_int32]
        lib.act_get_cta_pairs.argtypes = [_P, ctypes.c_int32, ctypes.POINTER(ctypes.c_int32)]
        lib.act_set_fused.argtypes = [_P, ctypes.c_int32]
        lib.act_get_fused.argtypes = [_P, ctypes.c_int32, ctypes.POINTER(ctypes.c_int32)]
        lib.act_destroy.argtypes = [_P]
        lib.act_destroy.restype = None
        for name in EXPORTS:
            if name not in ("act_status_string", "act_last_error_message", "act_destroy",
                            "act_ragged_plan_destroy"):
                getattr(lib, name).restype = ctypes.c_int
        _lib = lib
        return lib


def status_name(status: int) -> str:
    try:
        return load_library().act_status_string(int(status)).decode()
    except Exception:  # library absent: still give a readable message
        return f"status {status}"


def _check(status: int, call: str):
    if status != ACT_OK:
        detail = load_library().act_last_error_message().decode()
        raise ActError(status, call, detail)


def _ptr(x) -> Optional[int]:
    """Raw address of a tensor (device or host) or an int; None for None."""
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):
        if not x.is_contiguous():
            raise ValueError("tensors passed to libact must be contiguous")
        return x.data_ptr()
    if hasattr(x, "ctypes"):
        return x.ctypes.data
    raise TypeError(f"cannot pass {type(x)} to libact")


def _stream(stream) -> Optional[int]:
    if stream is None:
        import torch
        if torch.cuda.is_available():
            return torch.cuda.current_stream().cuda_stream
        return None
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


# ---------------------------------------------------------------------------
# Entry points (same names as the C ABI)
# ---------------------------------------------------------------------------
def act_grid_from_ranges(n_samples: int, fs: float, tc, fc, logdt, c) -> act_grid_desc:
    out = act_grid_desc()
    arrs = [(ctypes.c_double * 3)(*map(float, r)) for r in (tc, fc, logdt, c)]
    _check(load_library().act_grid_from_ranges(int(n_samples), float(fs), *arrs, ctypes.byref(out)),
           "act_grid_from_ranges")
    return out


def grid_desc(grid) -> act_grid_desc:
    """act_grid_desc from any object with n_samples, fs and tc/fc/logdt/c axes
    carrying lo, step and count."""
    d = act_grid_desc()
    d.n_samples = int(grid.n_samples)
    d.fs = float(grid.fs)
    for name in ("tc", "fc", "logdt", "c"):
        ax = getattr(grid, name)
        setattr(d, name, act_axis(float(ax.lo), float(ax.step), int(ax.count)))
    return d


def act_grid_create(desc, device: int = 0) -> int:
    if not isinstance(desc, act_grid_desc):
        desc = grid_desc(desc)
    h = _P()
    _check(load_library().act_grid_create(ctypes.byref(desc), int(device), ctypes.byref(h)), "act_grid_create")
    return h.value


def act_grid_size(grid: int):
    k = ctypes.c_int64()
    lp = ctypes.c_int32()
    _check(load_library().act_grid_size(grid, ctypes.byref(k), ctypes.byref(lp)), "act_grid_size")
    return k.value, lp.value


def act_dictionary_build(grid: int, mode: int = ACT_DICT_FP32, stream=None) -> None:
    _check(load_library().act_dictionary_build(grid, int(mode), _stream(stream)), "act_dictionary_build")


def act_set_search(grid: int, mode: int) -> None:
    _check(load_library().act_set_search(grid, int(mode)), "act_set_search")


def act_decompose(grid: int, signals, channels: int, n_atoms: int, atoms_out=None, coeffs_out=None,
                  residuals_out=None, energy_out=None, stream=None) -> None:
    _check(load_library().act_decompose(grid, _ptr(signals), int(channels), int(n_atoms), _ptr(atoms_out),
                                        _ptr(coeffs_out), _ptr(residuals_out), _ptr(energy_out),
                                        _stream(stream)), "act_decompose")


def act_project(grid: int, signals, channels: int, scores, stream=None) -> None:
    _check(load_library().act_project(grid, _ptr(signals), int(channels), _ptr(scores), _stream(stream)),
           "act_project")


def act_dictionary_rows(grid: int, first: int, count: int, out, stream=None) -> None:
    _check(load_library().act_dictionary_rows(grid, int(first), int(count), _ptr(out), _stream(stream)),
           "act_dictionary_rows")


def act_grid_status(grid: int, stream=None) -> int:
    """Device-side status since the last call (ACT_OK, ACT_ERR_NONFINITE, ...)."""
    return int(load_library().act_grid_status(grid, _stream(stream)))


def act_set_profiling(grid: int, enable: bool) -> None:
    _check(load_library().act_set_profiling(grid, 1 if enable else 0), "act_set_profiling")


def act_profile_read(grid: int):
    """(search_ms, core_ms, orders, kernels_per_call) of the last act_decompose."""
    ms = ctypes.c_double()
    core = ctypes.c_double()
    n = ctypes.c_int32()
    k = ctypes.c_int32()
    _check(load_library().act_profile_read(grid, ctypes.byref(ms), ctypes.byref(core), ctypes.byref(n),
                                           ctypes.byref(k)), "act_profile_read")
    return ms.value, core.value, n.value, k.value


def act_bf16_stats(grid: int):
    """(resolved, items_rescanned, fallbacks) counts of the tensor-core searches."""
    a = ctypes.c_int64()
    r = ctypes.c_int64()
    b = ctypes.c_int64()
    _check(load_library().act_bf16_stats(grid, ctypes.byref(a), ctypes.byref(r), ctypes.byref(b)),
           "act_bf16_stats")
    return a.value, r.value, b.value


def act_search_noalloc(dictionary, n_atoms: int, row_stride: int, residuals, channels: int, best_index,
                       best_score, stream=None) -> None:
    """FP32 search over a caller-owned dictionary without any allocation
    (see include/act.h)."""
    _check(load_library().act_search_noalloc(_ptr(dictionary), int(n_atoms), int(row_stride), _ptr(residuals),
                                             int(channels), _ptr(best_index), _ptr(best_score), _stream(stream)),
           "act_search_noalloc")


def act_autotune(grid: int, signals, channels: int, stream=None) -> float:
    """Picks the fastest launch configuration for these signals; returns ms per order."""
    ms = ctypes.c_double()
    _check(load_library().act_autotune(grid, _ptr(signals), int(channels), _stream(stream), ctypes.byref(ms)),
           "act_autotune")
    return ms.value


def act_get_tuning(grid: int):
    """(gemv_ctas, bf16_tile_atoms, bf16_stages) in use."""
    a = ctypes.c_int32()
    b = ctypes.c_int32()
    c = ctypes.c_int32()
    _check(load_library().act_get_tuning(grid, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c)),
           "act_get_tuning")
    return a.value, b.value, c.value


def act_set_tuning(grid: int, gemv_ctas: int = 0, bf16_tile_atoms: int = 0, bf16_stages: int = 0) -> None:
    _check(load_library().act_set_tuning(grid, int(gemv_ctas), int(bf16_tile_atoms), int(bf16_stages)),
           "act_set_tuning")


def act_set_shift_tuning(grid: int, lags_per_thread: int, warps: int, stages: int = 2, ctas_per_sm: int = 0) -> None:
    _check(load_library().act_set_shift_tuning(grid, int(lags_per_thread), int(warps), int(stages), int(ctas_per_sm)),
           "act_set_shift_tuning")


def act_get_shift_tuning(grid: int):
    """(lags_per_thread, warps, stages, ctas_per_sm) of the template search."""
    v = [ctypes.c_int32() for _ in range(4)]
    _check(load_library().act_get_shift_tuning(grid, *(ctypes.byref(x) for x in v)), "act_get_shift_tuning")
    return tuple(x.value for x in v)


def act_ragged_plan_create(grids, offsets, n_atoms: int) -> int:
    """Plan for channels of uneven length: grids (handles, one per length),
    offsets (host int64 sequence of channels+1 sample offsets)."""
    import numpy as np
    hs = (_P * len(grids))(*grids)
    off = np.ascontiguousarray(np.asarray(offsets, dtype=np.int64))
    h = _P()
    _check(load_library().act_ragged_plan_create(ctypes.cast(hs, _P), len(grids), off.ctypes.data, len(off) - 1,
                                                 int(n_atoms), ctypes.byref(h)), "act_ragged_plan_create")
    return h.value


def act_ragged_decompose(plan: int, signals, atoms_out=None, coeffs_out=None, residuals_out=None, energy_out=None,
                         stream=None) -> None:
    _check(load_library().act_ragged_decompose(plan, _ptr(signals), _ptr(atoms_out), _ptr(coeffs_out),
                                               _ptr(residuals_out), _ptr(energy_out), _stream(stream)),
           "act_ragged_decompose")


def act_ragged_plan_info(plan: int):
    g = ctypes.c_int32()
    k = ctypes.c_int32()
    _check(load_library().act_ragged_plan_info(plan, ctypes.byref(g), ctypes.byref(k)), "act_ragged_plan_info")
    return g.value, k.value


def act_ragged_plan_destroy(plan: int) -> None:
    if plan:
        load_library().act_ragged_plan_destroy(plan)


def act_set_refinement(grid: int, steps: int) -> None:
    _check(load_library().act_set_refinement(grid, int(steps)), "act_set_refinement")


def act_chirplet_score(n_samples: int, fs: float, theta, residuals, channels: int, score, grad_theta=None,
                       atoms=None, stream=None) -> None:
    _check(load_library().act_chirplet_score(int(n_samples), float(fs), _ptr(theta), _ptr(residuals), int(channels),
                                             _ptr(score), _ptr(grad_theta), _ptr(atoms), _stream(stream)),
           "act_chirplet_score")


def act_set_lem(grid: int, n_coarse: int = 0, top_k: int = 4, levels: int = 2,
                steps=((64, 2, 2, 5), (32, 1, 1, 2.5), (16, 0.5, 0.5, 0.5)), radius=(2, 2, 1, 2),
                seed: int = 0) -> None:
    p = act_lem_params()
    p.n_coarse, p.top_k, p.levels, p.seed = int(n_coarse), int(top_k), int(levels), int(seed)
    for l in range(3):
        for a in range(4):
            p.steps[l][a] = float(steps[min(l, len(steps) - 1)][a])
    for a in range(4):
        p.radius[a] = int(radius[a])
    _check(load_library().act_set_lem(grid, ctypes.byref(p)), "act_set_lem")


def act_dictionary_mode(grid: int) -> int:
    """The dictionary mode the last build made (ACT_DICT_FP32, _BF16 or _RECOMPUTE)."""
    m = ctypes.c_int32()
    _check(load_library().act_dictionary_mode(grid, ctypes.byref(m)), "act_dictionary_mode")
    return m.value


def act_set_memory_budget(grid: int, n_bytes: int) -> None:
    _check(load_library().act_set_memory_budget(grid, int(n_bytes)), "act_set_memory_budget")


def act_set_wait_limit(grid: int, ns: int) -> None:
    _check(load_library().act_set_wait_limit(grid, int(ns)), "act_set_wait_limit")


def act_set_cta_pairs(grid: int, enable: bool) -> None:
    """Whether the tensor-core template GEMM may pair SMs (cta_group::2)."""
    _check(load_library().act_set_cta_pairs(grid, 1 if enable else 0), "act_set_cta_pairs")


def act_get_cta_pairs(grid: int, channels: int) -> bool:
    """Whether a `channels`-channel tensor-core template search runs its GEMM on CTA pairs."""
    used = ctypes.c_int32(0)
    _check(load_library().act_get_cta_pairs(grid, int(channels), ctypes.byref(used)), "act_get_cta_pairs")
    return bool(used.value)


def act_set_fused(grid: int, ctas_per_sm: int) -> None:
    """CTAs per SM of the single-launch decomposition of small FP32 dictionaries (0: never)."""
    _check(load_library().act_set_fused(grid, int(ctas_per_sm)), "act_set_fused")


def act_get_fused(grid: int, channels: int) -> int:
    """CTAs of the single launch a `channels`-channel decomposition takes (0: per-order kernels)."""
    ctas = ctypes.c_int32(0)
    _check(load_library().act_get_fused(grid, int(channels), ctypes.byref(ctas)), "act_get_fused")
    return int(ctas.value)


def act_inject_alloc_failure(nth: int) -> None:
    """Makes the nth device allocation of the library from now on fail once (0 disarms)."""
    _check(load_library().act_inject_alloc_failure(int(nth)), "act_inject_alloc_failure")


def act_destroy(grid: int) -> None:
    if grid:
        load_library().act_destroy(grid)


# ---------------------------------------------------------------------------
# Output helpers (views over the raw buffers act_decompose fills)
# ---------------------------------------------------------------------------
def atoms_to_dict(buf) -> dict:
    """Splits an act_atom buffer (uint8 tensor/ndarray of B*P*40 bytes,
    host memory) into numpy arrays of fields."""
    import numpy as np
    dt = np.dtype([("tc", "<f8"), ("fc", "<f8"), ("logdt", "<f8"), ("c", "<f8"), ("flat_index", "<i8")])
    arr = np.frombuffer(bytes(memoryview(buf.numpy() if hasattr(buf, "numpy") else buf)), dtype=dt)
    return {name: arr[name].copy() for name in dt.names}


def decompose(grid: int, signals, n_atoms: int, stream=None):
    """Calls act_decompose on a [channels][n_samples] float32 tensor and
    returns freshly allocated outputs on the signals' device:
    (atoms uint8 [B, P, 40], coeffs float32 [B, P], residuals float32 [B, L],
    energy float64 [B, P+1])."""
    import torch
    sig = signals.contiguous()
    if sig.dtype != torch.float32:
        raise TypeError("signals must be float32")
    B, L = sig.shape
    dev = sig.device
    atoms = torch.empty((B, n_atoms, ATOM_BYTES), dtype=torch.uint8, device=dev)
    coeffs = torch.empty((B, n_atoms), dtype=torch.float32, device=dev)
    resid = torch.empty((B, L), dtype=torch.float32, device=dev)
    energy = torch.empty((B, n_atoms + 1), dtype=torch.float64, device=dev)
    act_decompose(grid, sig, B, n_atoms, atoms, coeffs, resid, energy, stream=stream)
    return atoms, coeffs, resid, energy


def atom_indices(atoms) -> "object":
    """flat_index field of an act_atom tensor [.., 40] as int64 (same device)."""
    import torch
    return atoms.reshape(-1, ATOM_BYTES)[:, 32:40].contiguous().view(torch.int64).reshape(atoms.shape[:-1])


def atom_params(atoms) -> "object":
    """(tc, fc, logdt, c) fields of an act_atom tensor [.., 40] as float64 [.., 4]."""
    import torch
    return atoms.reshape(-1, ATOM_BYTES)[:, 0:32].contiguous().view(torch.float64).reshape(
        *atoms.shape[:-1], 4)
