"""GPU parity of the BF16 tensor-core search (tcgen05 GEMM reduced to tile
and 32-atom block maxima, error-bounded selection of blocks, FP32 rescan of
the flagged blocks, FP32 full search as the last resort) through the C ABI.

The error bound makes the BF16 search return exactly the FP32 search's
selection, so its outputs must equal the FP32 path's bit for bit, and the
same order-by-order checks against the FP64 oracle apply."""
import numpy as np
import pytest
import torch

import oracle
from paper_2607_16629_gb300 import act, synth
from parity_helpers import check_lockstep

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    act.load_library()


class Bf16Grid:
    def __init__(self, grid):
        self.grid = grid

    def __enter__(self):
        self.h = act.act_grid_create(self.grid, 0)
        act.act_dictionary_build(self.h, act.ACT_DICT_BF16)
        act.act_set_search(self.h, act.ACT_SEARCH_BF16)
        return self.h

    def __exit__(self, *a):
        act.act_destroy(self.h)


def run(h, sig, P, mode):
    act.act_set_search(h, mode)
    atoms, coef, resid, energy = act.decompose(h, torch.tensor(sig, dtype=torch.float32, device="cuda"), P)
    torch.cuda.synchronize()
    st = act.act_grid_status(h)
    assert st == act.ACT_OK, act.status_name(st)
    return (act.atom_indices(atoms).cpu().numpy(), coef.cpu().numpy(), resid.cpu().numpy(),
            energy.cpu().numpy())


def chain(h, sig, P):
    """Residuals entering each order for all channels (one-order BF16 calls)."""
    rs = [np.asarray(sig, dtype=np.float32)]
    idx, coef = [], []
    for _ in range(P):
        i, c, r, _ = run(h, rs[-1], 1, act.ACT_SEARCH_BF16)
        idx.append(i[:, 0])
        coef.append(c[:, 0])
        rs.append(r)
    return rs, np.stack(idx, 1), np.stack(coef, 1)


def lockstep_all(D, rs, idx, coef):
    ties = 0
    for b in range(idx.shape[0]):
        ties += check_lockstep(lambda r: D @ r, [r[b] for r in rs], idx[b], coef[b])
    return ties


@pytest.mark.parametrize("name,grid,B,P", [
    ("tiny_k36_l32", synth.grid_small_test(), 3, 4),
    ("c1_k16384_l256", synth.grid_c1(), 16, 5),
])
def test_bf16_lockstep_small(name, grid, B, P):
    sig = np.concatenate([synth.workload_c1(min(B, 4)).signals if grid.n_samples == 256 else
                          synth.random_signals(61, min(B, 4), grid.n_samples),
                          synth.random_signals(62, B - min(B, 4), grid.n_samples)])
    D, _ = oracle.dictionary(grid)
    with Bf16Grid(grid) as h:
        c0, s0, f0 = act.act_bf16_stats(h)
        i_full, c_full, r_full, e_full = run(h, sig, P, act.ACT_SEARCH_BF16)
        rs, idx, coef = chain(h, sig, P)
        c1, s1, f1 = act.act_bf16_stats(h)
    assert np.array_equal(idx, i_full) and np.array_equal(coef, c_full)
    assert np.array_equal(rs[-1], r_full)
    assert (c1 - c0) + (f1 - f0) == 2 * B * P
    assert s1 - s0 >= c1 - c0  # at least one block per resolved selection
    lockstep_all(D, rs, idx, coef)


def test_bf16_matches_fp32_search_eeg():
    """64 EEG-like channels on a 131,072-atom EEG grid (512 tiles over the
    persistent CTAs, both accumulator buffers in use): the BF16 search and
    the FP32 search agree order by order, and both match the oracle."""
    grid = synth.scaled_grid(synth.grid_eeg(), tc_count=32, fc_count=16)
    sig = np.stack([synth.eeg_like_signal(3, b)[0] for b in range(64)])
    D, _ = oracle.dictionary(grid)
    P = 6
    with Bf16Grid(grid) as h:
        ib, cb, rb, eb = run(h, sig, P, act.ACT_SEARCH_BF16)
        i32, c32, r32, e32 = run(h, sig, P, act.ACT_SEARCH_FP32)
        rs, idx, coef = chain(h, sig, P)
        cert, rescan, fb = act.act_bf16_stats(h)
    for x, y in zip((ib, cb, rb, eb), (i32, c32, r32, e32)):
        assert np.array_equal(x, y)
    lockstep_all(D, rs, idx, coef)
    print(f"resolved {cert} blocks {rescan} fallback {fb}")


@pytest.mark.parametrize("grid,full_search", [
    (synth.grid_c1(), False),                                           # 512 blocks: all rescanned
    (synth.scaled_grid(synth.grid_eeg(), tc_count=32, fc_count=16), True),  # 4,096 blocks: full search
])
def test_bf16_zero_channel(grid, full_search):
    """An all-zero channel flags every block (all scores tie at 0): with at
    most 512 blocks they are all rescanned, beyond that the channel takes the
    FP32 full search.  Either way it selects index 0 with coefficient 0 and
    the other channels are unaffected."""
    sig = synth.random_signals(81, 3, grid.n_samples)
    sig[1] = 0.0
    with Bf16Grid(grid) as h:
        c0, t0, f0 = act.act_bf16_stats(h)
        idx, coef, resid, energy = run(h, sig, 3, act.ACT_SEARCH_BF16)
        c1, t1, f1 = act.act_bf16_stats(h)
        i32, c32, r32, e32 = run(h, sig, 3, act.ACT_SEARCH_FP32)
    assert (f1 - f0 == 3) == full_search
    assert not idx[1].any() and not coef[1].any()
    assert np.array_equal(idx, i32) and np.array_equal(coef, c32)


@pytest.mark.parametrize("B", [1, 128])
def test_bf16_channel_counts(B):
    grid = synth.grid_c1()
    sig = synth.random_signals(71, B, grid.n_samples)
    with Bf16Grid(grid) as h:
        ib, cb, rb, eb = run(h, sig, 2, act.ACT_SEARCH_BF16)
        i32, c32, r32, e32 = run(h, sig, 2, act.ACT_SEARCH_FP32)
    for x, y in zip((ib, cb, rb, eb), (i32, c32, r32, e32)):
        assert np.array_equal(x, y)


def test_bf16_rejects_more_than_128_channels():
    grid = synth.grid_small_test()
    with Bf16Grid(grid) as h:
        with pytest.raises(act.ActError) as e:
            act.decompose(h, torch.zeros((129, grid.n_samples), device="cuda"), 1)
        assert e.value.status == act.ACT_ERR_UNSUPPORTED


def test_bf16_full_eeg_grid_64_channels():
    """The 64-channel EEG-like workload on the full 2,097,152-atom grid in the
    benchmark's launch configuration: first order of every channel checked
    against the oracle on sampled atoms plus its selected atom, and the
    whole run against the FP32 search."""
    w = synth.workload_c3()
    P = 4
    with Bf16Grid(w.grid) as h:
        ib, cb, rb, eb = run(h, w.signals, P, act.ACT_SEARCH_BF16)
        i32, c32, r32, e32 = run(h, w.signals, P, act.ACT_SEARCH_FP32)
        cert, rescan, fb = act.act_bf16_stats(h)
    for x, y in zip((ib, cb, rb, eb), (i32, c32, r32, e32)):
        assert np.array_equal(x, y)
    rng = np.random.default_rng(3)
    sample = rng.integers(0, w.grid.n_atoms, 2000)
    for b in range(0, 64, 8):
        s = w.signals[b].astype(np.float32).astype(np.float64)
        g, _ = oracle.atom(*w.grid.params_of(int(ib[b, 0])), w.grid.fs, w.grid.n_samples)
        best = abs(g @ s)
        assert abs(cb[b, 0] - g @ s) <= 1e-5 * best
        for i in sample[:200]:
            gi, _ = oracle.atom(*w.grid.params_of(int(i)), w.grid.fs, w.grid.n_samples)
            assert abs(gi @ s) <= best * (1 + 1e-5)
    e0 = eb[:, 0]
    for k in range(P + 1):
        assert np.all(np.abs(e0 - (np.sum(cb[:, :k].astype(np.float64) ** 2, axis=1) + eb[:, k])) <= 1e-5 * e0)
    print(f"resolved {cert} blocks {rescan} fallback {fb}")


@pytest.mark.parametrize("L,fs", [(600, 500.0), (1024, 1000.0), (2048, 500.0)])
def test_bf16_long_windows_stream_the_residual(L, fs):
    """Windows longer than 512 samples stream the residual chunks with the
    dictionary chunks instead of keeping them resident; the selection still
    equals the FP32 search's on every output."""
    grid = synth.Grid(L, fs, synth.Axis(0.0, L / 16.0, 16), synth.Axis.linspace(20.0, 200.0, 12),
                      synth.Axis.linspace(-4.0, -1.5, 4), synth.Axis.linspace(-100.0, 100.0, 8))
    sig = np.stack([synth.emg_like_signal(b, L, fs)[0] for b in range(12)])
    with Bf16Grid(grid) as h:
        ib, cb, rb, eb = run(h, sig, 4, act.ACT_SEARCH_BF16)
        i32, c32, r32, e32 = run(h, sig, 4, act.ACT_SEARCH_FP32)
    for x, y in zip((ib, cb, rb, eb), (i32, c32, r32, e32)):
        assert np.array_equal(x, y)


@pytest.mark.parametrize("tile,stages", [(128, 2), (128, 0), (256, 2)])
def test_bf16_tile_widths_and_depths(tile, stages):
    """Every tensor-core configuration the autotuner may pick (tile width x
    pipeline depth) returns the FP32 search's results bit for bit."""
    grid = synth.scaled_grid(synth.grid_eeg(), tc_count=16, fc_count=16)
    sig = np.stack([synth.eeg_like_signal(3, b)[0] for b in range(20)])
    with Bf16Grid(grid) as h:
        act.act_set_tuning(h, 0, tile, stages)
        g, bn, st = act.act_get_tuning(h)
        assert bn == tile and (stages == 0 or st == stages)
        ib, cb, rb, eb = run(h, sig, 4, act.ACT_SEARCH_BF16)
        i32, c32, r32, e32 = run(h, sig, 4, act.ACT_SEARCH_FP32)
    for x, y in zip((ib, cb, rb, eb), (i32, c32, r32, e32)):
        assert np.array_equal(x, y)


def test_autotune_keeps_results():
    grid = synth.scaled_grid(synth.grid_eeg(), tc_count=16, fc_count=16)
    sig = np.stack([synth.eeg_like_signal(3, b)[0] for b in range(20)])
    with Bf16Grid(grid) as h:
        before = run(h, sig, 3, act.ACT_SEARCH_BF16)
        ms = act.act_autotune(h, torch.tensor(sig, dtype=torch.float32, device="cuda"), 20)
        assert ms > 0
        g, bn, st = act.act_get_tuning(h)
        assert bn in (128, 256) and st >= 2 and g > 0
        after = run(h, sig, 3, act.ACT_SEARCH_BF16)
        with pytest.raises(act.ActError):
            act.act_set_tuning(h, 0, 64, 0)
    for x, y in zip(before, after):
        assert np.array_equal(x, y)


def test_two_bf16_grids_with_different_windows_coexist():
    """Two BF16 grids with different shared-memory configurations (resident
    and streamed residual) can be used alternately."""
    ga = synth.scaled_grid(synth.grid_emg(256), tc_count=16, fc_count=8, logdt_count=4, c_count=8)
    gb = synth.scaled_grid(synth.grid_emg(2048), tc_count=16, fc_count=8, logdt_count=4, c_count=8)
    with Bf16Grid(ga) as ha, Bf16Grid(gb) as hb:
        for h, g, seed in ((ha, ga, 0), (hb, gb, 1), (ha, ga, 2)):
            sig = np.stack([synth.emg_like_signal(seed * 10 + b, g.n_samples)[0] for b in range(5)])
            x = run(h, sig, 3, act.ACT_SEARCH_BF16)
            y = run(h, sig, 3, act.ACT_SEARCH_FP32)
            for u, v in zip(x, y):
                assert np.array_equal(u, v)
