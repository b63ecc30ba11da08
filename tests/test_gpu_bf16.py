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
from parity_helpers import check_lockstep, full_dictionary

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


@pytest.mark.parametrize("B,L,tile", [(129, 512, 256), (256, 512, 128), (300, 1024, 256)])
def test_bf16_more_than_128_channels(B, L, tile):
    """More than one 128-channel row tile (the residual rows streamed with the
    dictionary chunks, the last tile ragged): the selection still equals the
    FP32 search's on every output, and lock-step against the oracle holds on
    a sample of channels from every row tile."""
    fs = 256.0 if L == 512 else 1000.0
    base = synth.grid_eeg(L, fs) if L == 512 else synth.grid_radar(L, fs)
    grid = synth.scaled_grid(base, tc_count=16, fc_count=16, c_count=16)
    sig = synth.random_signals(72, B, grid.n_samples)
    sig[::7] += np.stack([synth.eeg_like_signal(4, b, L, fs)[0] for b in range(0, B, 7)])
    P = 3
    D, _ = oracle.dictionary(grid)
    with Bf16Grid(grid) as h:
        act.act_set_tuning(h, 0, tile, 0)
        ib, cb, rb, eb = run(h, sig, P, act.ACT_SEARCH_BF16)
        i32, c32, r32, e32 = run(h, sig, P, act.ACT_SEARCH_FP32)
        for x, y in zip((ib, cb, rb, eb), (i32, c32, r32, e32)):
            assert np.array_equal(x, y)
        rs, idx, coef = chain(h, sig, P)       # one-order calls over all row tiles
    assert np.array_equal(idx, ib) and np.array_equal(coef, cb)
    for b in sorted({0, 127, 128, B - 1} | set(range(5, B, 41))):
        check_lockstep(lambda r: D @ r, [r[b] for r in rs], idx[b], coef[b])


def test_bf16_full_eeg_grid_64_channels():
    """The 64-channel EEG-like workload on the full 2,097,152-atom grid in the
    benchmark's launch configuration, all 20 orders: the whole run equals the
    FP32 search's, and eight channels (one from every group of eight) are
    checked order by order against the oracle scoring every atom of its FP64
    dictionary from the GPU's own residuals."""
    w = synth.workload_c3()
    P = w.n_atoms
    D = full_dictionary(w.grid)
    chans = list(range(0, 64, 8))
    with Bf16Grid(w.grid) as h:
        ib, cb, rb, eb = run(h, w.signals, P, act.ACT_SEARCH_BF16)
        i32, c32, r32, e32 = run(h, w.signals, P, act.ACT_SEARCH_FP32)
        cert, rescan, fb = act.act_bf16_stats(h)
        rs, idx, coef = chain(h, w.signals, P)
    for x, y in zip((ib, cb, rb, eb), (i32, c32, r32, e32)):
        assert np.array_equal(x, y)
    assert np.array_equal(idx, ib) and np.array_equal(coef, cb)
    ties = 0
    for k in range(P):
        R = np.stack([rs[k][b] for b in chans], axis=1).astype(np.float64)
        S = D @ R                                   # every atom's score, every sampled channel
        for j, b in enumerate(chans):
            ties += check_lockstep(lambda r, col=S[:, j]: col, [rs[k][b]], idx[b, k:k + 1], coef[b, k:k + 1])
    e0 = eb[:, 0]
    for k in range(P + 1):
        assert np.all(np.abs(e0 - (np.sum(cb[:, :k].astype(np.float64) ** 2, axis=1) + eb[:, k])) <= 1e-5 * e0)
    print(f"resolved {cert} blocks {rescan} fallback {fb}; {ties} near-ties in {len(chans) * P} checks")


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
