"""GPU parity of the FP32 path (atom generation, projection, GEMV argmax,
update, CUDA-graph loop) against the FP64 oracle, through the C ABI."""
import numpy as np
import pytest
import torch

import oracle
from paper_2607_16629_gb300 import act, synth
from parity_helpers import (ATOL_REL, RTOL, check_lockstep, full_dictionary, gpu_decompose,
                            gpu_residual_chain)

pytestmark = pytest.mark.gpu

# Atom accuracy: FP32 cospi/exp of FP64-formed arguments, FP32 scaling.
ATOM_ATOL = 1e-6


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    act.load_library()


class Grid:
    """Context manager: a built FP32 grid handle."""

    def __init__(self, grid, mode=act.ACT_DICT_FP32):
        self.grid, self.mode = grid, mode

    def __enter__(self):
        self.h = act.act_grid_create(self.grid, 0)
        act.act_dictionary_build(self.h, self.mode)
        return self.h

    def __exit__(self, *a):
        act.act_destroy(self.h)


def _rows(h, grid, first, count):
    out = torch.empty((count, grid.n_samples), dtype=torch.float32, device="cuda")
    act.act_dictionary_rows(h, first, count, out)
    torch.cuda.synchronize()
    return out.cpu().numpy().astype(np.float64)


def eeg_small():
    """EEG-like grid with every range of the full one but 32 x 16 x 8 x 32 =
    131,072 atoms (not a multiple of the rows one GEMV pass covers)."""
    return synth.scaled_grid(synth.grid_eeg(), tc_count=32, fc_count=16)


# ---------------------------------------------------------------------------
# Atoms
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("name,grid", [
    ("small", synth.grid_small_test()),
    ("c1", synth.grid_c1()),
    ("emg200", synth.scaled_grid(synth.Grid(200, 2000.0, synth.Axis(0, 32, 7), synth.Axis(20, 10, 43),
                                            synth.Axis(-4, 0.3, 14), synth.Axis(-10, 0.75, 27)), fc_count=11)),
    ("radar1024", synth.scaled_grid(synth.grid_radar(), tc_count=8, fc_count=8, c_count=8)),
])
def test_atoms_match_oracle(name, grid):
    D, deg = oracle.dictionary(grid)
    with Grid(grid) as h:
        K, Lp = act.act_grid_size(h)
        assert K == grid.n_atoms
        G = _rows(h, grid, 0, K)
    assert np.max(np.abs(G - D)) <= ATOM_ATOL
    norms = np.linalg.norm(G, axis=1)
    assert np.max(np.abs(norms[~deg] - 1.0)) <= 1e-6


def test_atoms_full_eeg_grid_sampled():
    """All 2,097,152 atoms of the EEG-like grid; sampled rows vs the oracle."""
    grid = synth.grid_eeg()
    rng = np.random.default_rng(5)
    rows = np.unique(np.concatenate([rng.integers(0, grid.n_atoms, 300), [0, grid.n_atoms - 1]]))
    with Grid(grid) as h:
        for i in rows:
            g = _rows(h, grid, int(i), 1)[0]
            ref, _ = oracle.atom(*oracle.atom_params(grid, int(i)), grid.fs, grid.n_samples)
            assert np.max(np.abs(g - ref)) <= ATOM_ATOL, i


# ---------------------------------------------------------------------------
# Projection P = D X^T
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("B", [1, 3, 6])
def test_projection_matches_oracle(B):
    grid = eeg_small()
    sig = synth.random_signals(11, B, grid.n_samples)
    D, _ = oracle.dictionary(grid)
    with Grid(grid) as h:
        scores = torch.empty((B, grid.n_atoms), dtype=torch.float32, device="cuda")
        act.act_project(h, torch.tensor(sig, dtype=torch.float32, device="cuda"), B, scores)
        torch.cuda.synchronize()
        got = scores.cpu().numpy()
    for b in range(B):
        x = sig[b].astype(np.float32).astype(np.float64)
        ref = D @ x
        assert np.max(np.abs(got[b] - ref)) <= 2e-6 * np.linalg.norm(x)


# ---------------------------------------------------------------------------
# Matching pursuit
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("name,grid,P", [
    ("small", synth.grid_small_test(), 8),
    ("c1", synth.grid_c1(), 5),
    ("eeg_small", None, 12),
])
def test_mp_lockstep(name, grid, P):
    if grid is None:
        grid = eeg_small()
    if name == "c1":
        s = synth.workload_c1().signals[0]
    elif name == "small":
        s = synth.random_signals(21, 1, grid.n_samples)[0]
    else:
        s, _ = synth.eeg_like_signal(2, 7)
    D, _ = oracle.dictionary(grid)
    with Grid(grid) as h:
        idx, par, coef, resid, energy = gpu_decompose(h, s[None, :], P)
        rs, cidx, ccoef = gpu_residual_chain(h, s, P)
    # chained one-order calls reproduce the P-order graph bit for bit
    assert np.array_equal(cidx, idx[0]) and np.array_equal(ccoef, coef[0])
    assert np.array_equal(rs[-1], resid[0])
    check_lockstep(lambda r: D @ r, rs, idx[0], coef[0], energy[0], lambda i: D[i])
    for k in range(P):
        assert par[0, k] == pytest.approx(oracle.atom_params(grid, idx[0, k]), abs=0)


def test_mp_matches_oracle_trajectory_c1():
    """Whole C1 decomposition vs the oracle's own trajectory."""
    w = synth.workload_c1()
    D, _ = oracle.dictionary(w.grid)
    s = w.signals[0].astype(np.float32).astype(np.float64)
    o_idx, o_coef, o_r, o_en = oracle.mp(D, s, w.n_atoms)
    with Grid(w.grid) as h:
        idx, _, coef, resid, energy = gpu_decompose(h, w.signals, w.n_atoms)
    assert np.array_equal(idx[0], o_idx)
    np.testing.assert_allclose(coef[0], o_coef, rtol=RTOL)
    np.testing.assert_allclose(energy[0], o_en, rtol=RTOL)
    np.testing.assert_allclose(resid[0], o_r, atol=ATOL_REL * np.linalg.norm(s) * 4)


def test_multichannel_equals_single_channel_runs():
    """B channels in one call (channel groups of 4 plus a ragged group) give
    bit-identical results to B one-channel calls."""
    grid = synth.grid_c1()
    sig = synth.random_signals(31, 7, grid.n_samples)
    with Grid(grid) as h:
        idx, _, coef, resid, energy = gpu_decompose(h, sig, 6)
        for b in range(7):
            i1, _, c1, r1, e1 = gpu_decompose(h, sig[b:b + 1], 6)
            assert np.array_equal(i1[0], idx[b]) and np.array_equal(c1[0], coef[b])
            assert np.array_equal(r1[0], resid[b]) and np.array_equal(e1[0], energy[b])


def test_host_buffers_match_device_buffers():
    grid = synth.grid_c1()
    sig = synth.random_signals(41, 3, grid.n_samples)
    with Grid(grid) as h:
        a = gpu_decompose(h, sig, 5, host=False)
        b = gpu_decompose(h, sig, 5, host=True)
    for x, y in zip(a, b):
        assert np.array_equal(x, y)


def test_repeat_runs_are_deterministic():
    grid = eeg_small()
    s, _ = synth.eeg_like_signal(2, 3)
    with Grid(grid) as h:
        a = gpu_decompose(h, s[None, :], 10)
        b = gpu_decompose(h, s[None, :], 10)
    for x, y in zip(a, b):
        assert np.array_equal(x, y)


def test_energy_identity_and_monotone_on_gpu():
    grid = eeg_small()
    s, _ = synth.eeg_like_signal(2, 4)
    with Grid(grid) as h:
        idx, _, coef, resid, energy = gpu_decompose(h, s[None, :], 20)
    e0 = energy[0, 0]
    for k in range(21):
        assert abs(e0 - (np.sum(coef[0, :k].astype(np.float64) ** 2) + energy[0, k])) <= 1e-5 * e0
    assert np.all(np.diff(energy[0]) <= 1e-7 * e0)


# ---------------------------------------------------------------------------
# Edge cases
# ---------------------------------------------------------------------------
def test_lone_on_grid_atom_recovered():
    grid = synth.grid_c1()
    for j, a in [(0, 1.3), (9999, -0.7), (grid.n_atoms - 1, 2.0)]:
        g, _ = oracle.atom(*oracle.atom_params(grid, j), grid.fs, grid.n_samples)
        with Grid(grid) as h:
            idx, _, coef, resid, energy = gpu_decompose(h, (a * g)[None, :], 1)
        assert idx[0, 0] == j
        assert abs(coef[0, 0] - a) <= 1e-5 * abs(a)
        assert np.linalg.norm(resid[0]) <= 1e-5 * abs(a)


def test_zero_signal_selects_index_zero():
    grid = synth.grid_small_test()
    with Grid(grid) as h:
        idx, _, coef, resid, energy = gpu_decompose(h, np.zeros((2, grid.n_samples)), 3)
    assert not idx.any() and not coef.any() and not resid.any() and not energy.any()


def test_nonfinite_signal_is_reported():
    grid = synth.grid_small_test()
    s = np.ones((1, grid.n_samples), dtype=np.float32)
    s[0, 5] = np.nan
    with Grid(grid) as h:
        sig = torch.tensor(s, device="cuda")
        act.decompose(h, sig, 2)
        assert act.act_grid_status(h) == act.ACT_ERR_NONFINITE
        assert act.act_grid_status(h) == act.ACT_OK  # cleared


def test_invalid_calls():
    grid = synth.grid_small_test()
    h = act.act_grid_create(grid, 0)
    try:
        sig = torch.zeros((1, grid.n_samples), device="cuda")
        with pytest.raises(act.ActError) as e:
            act.decompose(h, sig, 2)
        assert e.value.status == act.ACT_ERR_NOT_BUILT
        act.act_dictionary_build(h, act.ACT_DICT_FP32)
        with pytest.raises(act.ActError) as e:
            act.act_decompose(h, sig, 0, 2)
        assert e.value.status == act.ACT_ERR_INVALID_ARG
        with pytest.raises(act.ActError) as e:
            act.act_dictionary_build(h, act.ACT_DICT_RECOMPUTE)
        assert e.value.status == act.ACT_ERR_UNSUPPORTED
    finally:
        act.act_destroy(h)


@pytest.mark.parametrize("L", [1, 37, 128, 200, 385, 1000, 2048])
def test_window_lengths(L):
    """Row strides 128..2048 and ragged window lengths."""
    fs = 500.0
    grid = synth.Grid(L, fs, synth.Axis(0.0, max(L / 6.0, 1.0), 6), synth.Axis(20, 35, 6),
                      synth.Axis(-4.0, 0.5, 3), synth.Axis(-50, 50, 3))
    s = synth.random_signals(51, 1, L)[0]
    D, _ = oracle.dictionary(grid)
    with Grid(grid) as h:
        idx, _, coef, resid, energy = gpu_decompose(h, s[None, :], 4)
        rs, cidx, ccoef = gpu_residual_chain(h, s, 4)
    assert np.array_equal(cidx, idx[0])
    check_lockstep(lambda r: D @ r, rs, idx[0], coef[0], energy[0], lambda i: D[i])


@pytest.mark.parametrize("gemv", ["load_stream", "bulk_stream"])
def test_full_eeg_grid_lockstep_all_orders(gemv):
    """The 2,097,152-atom EEG-like workload at full size, all 20 orders, in
    both FP32 GEMV forms (the benchmark times the bulk-copy streaming GEMV):
    every order is checked against the oracle scoring every atom of its FP64
    dictionary from the GPU's own residual."""
    w = synth.workload_c2()
    P = w.n_atoms
    s = w.signals[0]
    D = full_dictionary(w.grid)
    with Grid(w.grid) as h:
        if gemv == "bulk_stream":
            act.act_set_tuning(h, -1)
        idx, _, coef, resid, energy = gpu_decompose(h, s[None, :], P)
        rs, cidx, ccoef = gpu_residual_chain(h, s, P)
    assert np.array_equal(cidx, idx[0]) and np.array_equal(ccoef, coef[0])
    ties = check_lockstep(lambda r: D @ r, rs, cidx, ccoef, energy[0], lambda i: D[i])
    print(f"{gemv}: {ties} near-ties in {P} orders")
    # every order: energy identity and monotone residual
    e0 = energy[0, 0]
    for k in range(P + 1):
        assert abs(e0 - (np.sum(coef[0, :k].astype(np.float64) ** 2) + energy[0, k])) <= 1e-5 * e0
    assert np.all(np.diff(energy[0]) <= 1e-7 * e0)


def test_degenerate_atoms_match_oracle():
    """Atoms centred far outside the window (tc = 5000 samples, Dt well under a
    sample) underflow to zero on both sides and are never selected."""
    grid = synth.Grid(64, 100.0, synth.Axis(20.0, 4980.0, 2), synth.Axis(10.0, 5.0, 2),
                      synth.Axis(-6.0, 0.5, 2), synth.Axis(0.0, 1.0, 2))
    D, deg = oracle.dictionary(grid)
    assert deg.sum() == 8 and not deg[:8].any()
    s = synth.random_signals(33, 1, grid.n_samples)[0]
    with Grid(grid) as h:
        G = _rows(h, grid, 0, grid.n_atoms)
        idx, _, coef, _, _ = gpu_decompose(h, s[None, :], 3)
    assert not G[deg].any()
    assert np.max(np.abs(G - D)) <= ATOM_ATOL
    assert not deg[idx[0]].any()
    o_idx, o_coef, _, _ = oracle.mp(D, s.astype(np.float32).astype(np.float64), 3)
    assert np.array_equal(idx[0], o_idx)


@pytest.mark.parametrize("name,grid", [
    ("c1", synth.grid_c1()),
    ("eeg_small", None),
    ("l2048", synth.Grid(2048, 500.0, synth.Axis(0.0, 300.0, 7), synth.Axis(20, 35, 6),
                         synth.Axis(-4.0, 0.5, 3), synth.Axis(-50, 50, 3))),
    ("l37", synth.Grid(37, 500.0, synth.Axis(0.0, 6.0, 6), synth.Axis(20, 35, 6), synth.Axis(-4.0, 0.5, 3),
                       synth.Axis(-50, 50, 3))),
])
def test_streaming_gemv_gives_the_same_bits(name, grid):
    """The bulk-copy streaming GEMV scores rows in the load-streaming GEMV's
    order: every output of a decomposition is identical, for one and several
    channels."""
    if grid is None:
        grid = eeg_small()
    sig = synth.random_signals(61, 3, grid.n_samples)
    with Grid(grid) as h:
        act.act_set_fused(h, 0)  # one channel too: the per-order GEMV kernels
        ref1 = gpu_decompose(h, sig[:1], 6)
        ref3 = gpu_decompose(h, sig, 6)
        act.act_set_tuning(h, -1)
        assert act.act_get_tuning(h)[0] == -1
        for ref, s in ((ref1, sig[:1]), (ref3, sig)):
            got = gpu_decompose(h, s, 6)
            for a, b in zip(ref, got):
                assert np.array_equal(a, b)
        with pytest.raises(act.ActError):
            act.act_set_tuning(h, -2)
