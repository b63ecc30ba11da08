"""FP64 CPU oracle for chirplet matching pursuit (test infrastructure only).

Only the test suite, the smoke check and the benchmark's CPU-baseline leg may
import this package.  The product path never does, and this package never
imports the CUDA implementation.  The arithmetic lives in ``act_oracle.c``
(plain C, double precision); this module only builds it with gcc and
marshals numpy arrays through ctypes.

See ``act_oracle.c`` for the passages of the paper each function follows and
for the readings taken where the paper is silent.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from typing import Optional, Tuple

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "act_oracle.c")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

_dp = ctypes.POINTER(ctypes.c_double)


class LemParams(ctypes.Structure):
    """Settings of the hierarchical search (Sec. VII-A): LHS samples of the
    coarse level, candidates kept per level, refinement levels, the step of
    each level per axis (tc, fc, logDt, c) and the neighbourhood half-width
    in steps per axis."""
    _fields_ = [("n_coarse", ctypes.c_int), ("top_k", ctypes.c_int), ("levels", ctypes.c_int),
                ("steps", (ctypes.c_double * 4) * 3), ("radius", ctypes.c_int * 4)]
_i64p = ctypes.POINTER(ctypes.c_int64)
_u8p = ctypes.POINTER(ctypes.c_uint8)


def build(force: bool = False) -> str:
    """Compile act_oracle.c into liboracle.so (gcc, -O2, OpenMP)."""
    stale = (not os.path.exists(_LIB_PATH)
             or os.path.getmtime(_LIB_PATH) < max(os.path.getmtime(_SRC), os.path.getmtime(__file__)))
    if force or stale:
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fPIC", "-shared", "-fopenmp", "-o", tmp, _SRC, "-lm"]
        subprocess.check_call(cmd)
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        build()
        lib = ctypes.CDLL(_LIB_PATH)
        lib.act_oracle_set_threads.argtypes = [ctypes.c_int]
        lib.act_oracle_max_threads.restype = ctypes.c_int
        lib.act_oracle_range_count.argtypes = [ctypes.c_double] * 3
        lib.act_oracle_range_count.restype = ctypes.c_int64
        lib.act_oracle_atom_params.argtypes = [_dp, _i64p, ctypes.c_int64, _dp, _dp, _dp, _dp]
        lib.act_oracle_atom_complex.argtypes = [ctypes.c_double] * 5 + [ctypes.c_int, _dp, _dp]
        lib.act_oracle_atom.argtypes = [ctypes.c_double] * 5 + [ctypes.c_int, _dp]
        lib.act_oracle_atom.restype = ctypes.c_int
        lib.act_oracle_dictionary.argtypes = [_dp, _i64p, ctypes.c_int, ctypes.c_double, _dp, _u8p]
        lib.act_oracle_dictionary.restype = ctypes.c_int64
        lib.act_oracle_scores.argtypes = [_dp, ctypes.c_int64, ctypes.c_int, _dp, _dp]
        lib.act_oracle_scores_grid.argtypes = [_dp, _i64p, ctypes.c_int, ctypes.c_double, _dp, _dp]
        lib.act_oracle_select.argtypes = [_dp, ctypes.c_int64, _i64p, _i64p]
        lib.act_oracle_mp.argtypes = [_dp, ctypes.c_int64, ctypes.c_int, _dp, ctypes.c_int, _i64p,
                                      _dp, _dp, _dp]
        lib.act_oracle_mp.restype = ctypes.c_int
        lib.act_oracle_mp_grid.argtypes = [_dp, _i64p, ctypes.c_int, ctypes.c_double, _dp,
                                           ctypes.c_int, _i64p, _dp, _dp, _dp, _dp]
        lib.act_oracle_mp_grid.restype = ctypes.c_int
        lib.act_oracle_score_grad.argtypes = [_dp, ctypes.c_double, ctypes.c_int, _dp, _dp, _dp]
        lib.act_oracle_score_grad.restype = ctypes.c_int
        lib.act_oracle_refine.argtypes = [_dp, ctypes.c_double, ctypes.c_int, _dp, ctypes.c_int, _dp, _dp, _dp]
        lib.act_oracle_refine.restype = ctypes.c_double
        lib.act_oracle_mp_refine.argtypes = [_dp, _i64p, ctypes.c_int, ctypes.c_double, _dp, ctypes.c_int,
                                             ctypes.c_int, _i64p, _dp, _dp, _dp, _dp]
        lib.act_oracle_mp_refine.restype = ctypes.c_int
        lib.act_oracle_splitmix64_at.argtypes = [ctypes.c_uint64, ctypes.c_uint64]
        lib.act_oracle_splitmix64_at.restype = ctypes.c_uint64
        lib.act_oracle_lhs.argtypes = [_dp, _dp, ctypes.c_int, ctypes.c_uint64, ctypes.c_int, ctypes.c_int, _dp]
        lib.act_oracle_lem_topk.argtypes = [_dp, _dp, ctypes.c_int, ctypes.c_int, _dp, _dp]
        lib.act_oracle_lem_topk.restype = ctypes.c_int
        lib.act_oracle_lem_neighbours.argtypes = [_dp, ctypes.c_int, _dp, ctypes.POINTER(ctypes.c_int), _dp, _dp, _dp]
        lib.act_oracle_lem_neighbours.restype = ctypes.c_int
        lib.act_oracle_lem_select.argtypes = [ctypes.POINTER(LemParams), _dp, _dp, ctypes.c_double, ctypes.c_int,
                                              _dp, ctypes.c_uint64, ctypes.c_int, ctypes.c_int, _dp, _dp]
        lib.act_oracle_lem_select.restype = ctypes.c_int
        lib.act_oracle_mp_lem.argtypes = [ctypes.POINTER(LemParams), _dp, _dp, _dp, _dp, _dp, ctypes.c_double,
                                          ctypes.c_int, _dp, ctypes.c_int, ctypes.c_int, ctypes.c_uint64,
                                          ctypes.c_int, _dp, _dp, _dp, _dp]
        lib.act_oracle_mp_lem.restype = ctypes.c_int
        _lib = lib
        return lib


def _d(a: np.ndarray):
    return a.ctypes.data_as(_dp)


def _i(a: np.ndarray):
    return a.ctypes.data_as(_i64p)


def _grid_arrays(grid) -> Tuple[np.ndarray, np.ndarray]:
    axes = np.array([grid.tc.lo, grid.tc.step, grid.fc.lo, grid.fc.step, grid.logdt.lo,
                     grid.logdt.step, grid.c.lo, grid.c.step], dtype=np.float64)
    counts = np.array([grid.tc.count, grid.fc.count, grid.logdt.count, grid.c.count],
                      dtype=np.int64)
    return axes, counts


def set_threads(n: int) -> None:
    _load().act_oracle_set_threads(int(n))


def max_threads() -> int:
    return int(_load().act_oracle_max_threads())


def range_count(start: float, stop: float, step: float) -> int:
    """Values in the half-open range [start, stop) with the given step (Table 2)."""
    return int(_load().act_oracle_range_count(float(start), float(stop), float(step)))


def atom_params(grid, flat: int) -> Tuple[float, float, float, float]:
    axes, counts = _grid_arrays(grid)
    out = [ctypes.c_double() for _ in range(4)]
    _load().act_oracle_atom_params(_d(axes), _i(counts), int(flat), *[ctypes.byref(o) for o in out])
    return tuple(o.value for o in out)


def atom_complex(tc, fc, logdt, c, fs, n_samples) -> np.ndarray:
    """Eq. (1) with its prefactor, sampled at t = n / fs (complex128)."""
    re = np.empty(n_samples)
    im = np.empty(n_samples)
    _load().act_oracle_atom_complex(tc, fc, logdt, c, fs, int(n_samples), _d(re), _d(im))
    return re + 1j * im


def atom(tc, fc, logdt, c, fs, n_samples) -> Tuple[np.ndarray, bool]:
    """Unit-norm real dictionary atom; returns (g, degenerate)."""
    g = np.empty(n_samples)
    d = _load().act_oracle_atom(tc, fc, logdt, c, fs, int(n_samples), _d(g))
    return g, bool(d)


def dictionary(grid) -> Tuple[np.ndarray, np.ndarray]:
    """D[K][n_samples] (float64) and the degenerate-atom mask."""
    axes, counts = _grid_arrays(grid)
    K = int(np.prod(counts))
    D = np.empty((K, grid.n_samples))
    deg = np.zeros(K, dtype=np.uint8)
    _load().act_oracle_dictionary(_d(axes), _i(counts), int(grid.n_samples), float(grid.fs), _d(D),
                                  deg.ctypes.data_as(_u8p))
    return D, deg.astype(bool)


def scores(D: np.ndarray, r: np.ndarray) -> np.ndarray:
    D = np.ascontiguousarray(D, dtype=np.float64)
    r = np.ascontiguousarray(r, dtype=np.float64)
    out = np.empty(D.shape[0])
    _load().act_oracle_scores(_d(D), D.shape[0], D.shape[1], _d(r), _d(out))
    return out


def scores_grid(grid, r: np.ndarray) -> np.ndarray:
    axes, counts = _grid_arrays(grid)
    r = np.ascontiguousarray(r, dtype=np.float64)
    out = np.empty(int(np.prod(counts)))
    _load().act_oracle_scores_grid(_d(axes), _i(counts), int(grid.n_samples), float(grid.fs), _d(r),
                                   _d(out))
    return out


def select(sc: np.ndarray) -> Tuple[int, int]:
    """(best, runner_up) under the selection rule (lowest index on ties)."""
    sc = np.ascontiguousarray(sc, dtype=np.float64)
    b = ctypes.c_int64()
    s = ctypes.c_int64()
    _load().act_oracle_select(_d(sc), sc.shape[0], ctypes.byref(b), ctypes.byref(s))
    return int(b.value), int(s.value)


def mp(D: np.ndarray, s: np.ndarray, P: int):
    """MP over a stored dictionary -> (idx[P], coef[P], residual, energy[P+1])."""
    D = np.ascontiguousarray(D, dtype=np.float64)
    s = np.ascontiguousarray(s, dtype=np.float64)
    idx = np.empty(P, dtype=np.int64)
    coef = np.empty(P)
    r = np.empty(D.shape[1])
    en = np.empty(P + 1)
    rc = _load().act_oracle_mp(_d(D), D.shape[0], D.shape[1], _d(s), int(P), _i(idx), _d(coef), _d(r),
                               _d(en))
    if rc != 0:
        raise MemoryError("oracle MP allocation failed")
    return idx, coef, r, en


def mp_grid(grid, s: np.ndarray, P: int):
    """MP with atoms regenerated from the grid at every order
    -> (idx[P], coef[P], residual, energy[P+1], gap[P])."""
    axes, counts = _grid_arrays(grid)
    s = np.ascontiguousarray(s, dtype=np.float64)
    idx = np.empty(P, dtype=np.int64)
    coef = np.empty(P)
    r = np.empty(grid.n_samples)
    en = np.empty(P + 1)
    gap = np.empty(P)
    rc = _load().act_oracle_mp_grid(_d(axes), _i(counts), int(grid.n_samples), float(grid.fs), _d(s),
                                    int(P), _i(idx), _d(coef), _d(r), _d(en), _d(gap))
    if rc != 0:
        raise MemoryError("oracle MP allocation failed")
    return idx, coef, r, en, gap


def score_grad(theta, fs, r):
    """(s, ds/dtheta[4]) of the unit-norm real chirplet at continuous theta."""
    th = np.ascontiguousarray(theta, dtype=np.float64)
    r = np.ascontiguousarray(r, dtype=np.float64)
    sc = ctypes.c_double()
    g = np.empty(4)
    _load().act_oracle_score_grad(_d(th), float(fs), int(r.shape[0]), _d(r), ctypes.byref(sc), _d(g))
    return sc.value, g


def refine(theta, fs, r, steps, w, lo, hi):
    """BFGS refinement of theta from the grid start (returns (theta*, J*))."""
    th = np.array(theta, dtype=np.float64)
    r = np.ascontiguousarray(r, dtype=np.float64)
    J = _load().act_oracle_refine(_d(th), float(fs), int(r.shape[0]), _d(r), int(steps),
                                  _d(np.ascontiguousarray(w, dtype=np.float64)),
                                  _d(np.ascontiguousarray(lo, dtype=np.float64)),
                                  _d(np.ascontiguousarray(hi, dtype=np.float64)))
    return th, J


def refine_box(grid):
    """(scales, lo, hi) the refinement uses for a grid: the grid steps and
    the grid box widened by one step on each side."""
    axes = [grid.tc, grid.fc, grid.logdt, grid.c]
    w, lo, hi = [], [], []
    for a in axes:
        st = abs(a.step)
        first, last = a.lo, a.lo + (a.count - 1) * a.step
        w.append(st if st > 0 else 1.0)
        lo.append(min(first, last) - st if st > 0 else first)
        hi.append(max(first, last) + st if st > 0 else first)
    return np.array(w), np.array(lo), np.array(hi)


def mp_refine(grid, s, P, steps):
    """MP with off-grid refinement -> (idx[P], coef[P], theta[P][4], residual, energy[P+1])."""
    axes, counts = _grid_arrays(grid)
    s = np.ascontiguousarray(s, dtype=np.float64)
    idx = np.empty(P, dtype=np.int64)
    coef = np.empty(P)
    th = np.empty((P, 4))
    r = np.empty(grid.n_samples)
    en = np.empty(P + 1)
    rc = _load().act_oracle_mp_refine(_d(axes), _i(counts), int(grid.n_samples), float(grid.fs), _d(s), int(P),
                                      int(steps), _i(idx), _d(coef), _d(th), _d(r), _d(en))
    if rc != 0:
        raise MemoryError("oracle MP allocation failed")
    return idx, coef, th, r, en


def lem_params(n_coarse, top_k, levels, steps, radius) -> LemParams:
    p = LemParams()
    p.n_coarse, p.top_k, p.levels = int(n_coarse), int(top_k), int(levels)
    for l in range(3):
        for a in range(4):
            p.steps[l][a] = float(steps[min(l, len(steps) - 1)][a])
    for a in range(4):
        p.radius[a] = int(radius[a])
    return p


def splitmix64_at(seed: int, n: int) -> int:
    """The n-th output of SplitMix64 seeded with `seed`."""
    return int(_load().act_oracle_splitmix64_at(int(seed), int(n)))


def lhs(lo, hi, n, seed, channel, order) -> np.ndarray:
    out = np.empty((n, 4))
    _load().act_oracle_lhs(_d(np.ascontiguousarray(lo, dtype=np.float64)),
                           _d(np.ascontiguousarray(hi, dtype=np.float64)), int(n), int(seed), int(channel),
                           int(order), _d(out))
    return out


def lem_topk(cand, score, k):
    """The k best candidates by |score| (lowest index on ties), a parameter
    vector equal to one already kept skipped -> (kept[m][4], kept_score[m])."""
    cand = np.ascontiguousarray(cand, dtype=np.float64)
    score = np.ascontiguousarray(score, dtype=np.float64)
    kept = np.empty((k, 4))
    ks = np.empty(k)
    m = _load().act_oracle_lem_topk(_d(cand), _d(score), int(score.shape[0]), int(k), _d(kept), _d(ks))
    return kept[:m], ks[:m]


def lem_neighbours(kept, step, radius, lo, hi):
    """Neighbourhood candidates of the kept parameter vectors (Sec. VII-A):
    every offset -R..R steps per axis (c fastest), clamped to [lo, hi]."""
    kept = np.ascontiguousarray(kept, dtype=np.float64).reshape(-1, 4)
    per = int(np.prod([2 * r + 1 for r in radius]))
    out = np.empty((kept.shape[0] * per, 4))
    R = (ctypes.c_int * 4)(*[int(r) for r in radius])
    f = lambda a: _d(np.ascontiguousarray(a, dtype=np.float64))
    n = _load().act_oracle_lem_neighbours(_d(kept), int(kept.shape[0]), f(step), R, f(lo), f(hi), _d(out))
    return out[:n]


def lem_select(params: LemParams, lo, hi, fs, r, seed, channel, order):
    """Hierarchical selection before BFGS -> (theta[4], score)."""
    th = np.empty(4)
    sc = np.empty(1)
    r = np.ascontiguousarray(r, dtype=np.float64)
    rc = _load().act_oracle_lem_select(ctypes.byref(params), _d(np.ascontiguousarray(lo, dtype=np.float64)),
                                       _d(np.ascontiguousarray(hi, dtype=np.float64)), float(fs), int(r.shape[0]),
                                       _d(r), int(seed), int(channel), int(order), _d(th), _d(sc))
    if rc != 0:
        raise MemoryError("oracle LEM allocation failed")
    return th, float(sc[0])


def mp_lem(params: LemParams, lo, hi, scale, box_lo, box_hi, fs, s, P, steps, seed, channel):
    """MP with hierarchical selection (+ BFGS) -> (theta[P][4], coef[P], residual, energy[P+1])."""
    s = np.ascontiguousarray(s, dtype=np.float64)
    L = s.shape[0]
    th = np.empty((P, 4))
    coef = np.empty(P)
    r = np.empty(L)
    en = np.empty(P + 1)
    f = lambda a: _d(np.ascontiguousarray(a, dtype=np.float64))
    rc = _load().act_oracle_mp_lem(ctypes.byref(params), f(lo), f(hi), f(scale), f(box_lo), f(box_hi), float(fs),
                                   int(L), _d(s), int(P), int(steps), int(seed), int(channel), _d(th), _d(coef),
                                   _d(r), _d(en))
    if rc != 0:
        raise MemoryError("oracle LEM allocation failed")
    return th, coef, r, en
