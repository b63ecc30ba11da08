"""GPU checks of the tensor-core template search (ACT_SEARCH_SHIFT_BF16).

The BF16 tcgen05 GEMM only narrows the search: every (time centre,
template tile) that the BF16 error bound cannot exclude is rescored with the
FP32 template search's own arithmetic, and a channel with too many such
items is searched in full by the FP32 template search itself (over a device
queue of such channels).  So the whole decomposition must
equal ACT_SEARCH_SHIFT's bit for bit, and through it the oracle parity of
tests/test_gpu_shift.py carries over; one lock-step check against the
oracle is repeated here directly."""
import numpy as np
import pytest
import torch

import oracle
from paper_2607_16629_gb300 import act, synth
from parity_helpers import check_lockstep, gpu_decompose, gpu_residual_chain

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    act.load_library()


def eeg_small():
    return synth.scaled_grid(synth.grid_eeg(), tc_count=32, fc_count=16)


def ragged():
    return synth.Grid(203, 500.0, synth.Axis(-3.0, 5.0, 37), synth.Axis(20.0, 35.0, 5),
                      synth.Axis(-4.0, 0.5, 3), synth.Axis(-60.0, 20.0, 7))


GRIDS = [
    ("c1", synth.grid_c1()),
    ("eeg_small", eeg_small()),
    ("ragged", ragged()),
    ("dense_tc", synth.Grid(96, 256.0, synth.Axis(0.0, 1.0, 96), synth.Axis(4.0, 9.0, 3),
                            synth.Axis(-3.0, 0.6, 4), synth.Axis(-20.0, 40.0, 2))),
    ("radar_scaled", synth.scaled_grid(synth.grid_radar(), fc_count=4, logdt_count=2, c_count=4)),
    ("emg2048_scaled", synth.scaled_grid(synth.grid_emg(2048), fc_count=8, logdt_count=2, c_count=4)),
]


def both(grid, sig, P, refine=0):
    """(FP32 template search, tensor-core template search) outputs and the
    tensor-core run's (resolved, items, fallbacks) counts."""
    h = act.act_grid_create(grid, 0)
    try:
        act.act_dictionary_build(h, act.ACT_DICT_RECOMPUTE)
        act.act_set_refinement(h, refine)
        act.act_set_search(h, act.ACT_SEARCH_SHIFT)
        a = gpu_decompose(h, sig, P)
        act.act_set_search(h, act.ACT_SEARCH_SHIFT_BF16)
        s0 = act.act_bf16_stats(h)
        b = gpu_decompose(h, sig, P)
        s1 = act.act_bf16_stats(h)
    finally:
        act.act_destroy(h)
    return a, b, tuple(y - x for x, y in zip(s0, s1))


def assert_same(a, b):
    for x, y in zip(a, b):
        assert np.array_equal(x, y)


@pytest.mark.parametrize("name,grid", GRIDS)
def test_equals_fp32_template_search(name, grid):
    sig = synth.random_signals(91, 3, grid.n_samples)
    a, b, (resolved, items, fallbacks) = both(grid, sig, 6)
    assert_same(a, b)
    assert resolved + fallbacks == 3 * 6 and items >= resolved


def test_eeg_like_channels_full_grid():
    """64 EEG-like channels on the 2,097,152-atom grid: the batched case the
    tensor cores are for; few items per channel-order, no fallbacks."""
    w = synth.workload_c3()
    a, b, (resolved, items, fallbacks) = both(w.grid, w.signals, 4)
    assert_same(a, b)
    assert resolved == 64 * 4 and fallbacks == 0
    assert items < 64 * 4 * 16


def odd_tiles():
    """100 whole-sample time centres (step 4) over the EEG templates: at 32
    channels the rows form 25 tiles of 32 channels x 4 time centres, an odd
    count, so the last CTA pair has a second tile without rows."""
    g = synth.grid_eeg()
    return synth.Grid(g.n_samples, g.fs, synth.Axis(0.0, 4.0, 100), g.fc, g.logdt, g.c)


@pytest.mark.parametrize("name,grid_fn,B", [
    ("eeg_8ch", synth.grid_eeg, 8),            # pairs of tiles 16 time centres apart (one channel block)
    ("eeg_64ch", synth.grid_eeg, 64),          # pairs of channel blocks at the same time centres
    ("eeg_130ch", synth.grid_eeg, 130),        # 5 channel blocks, the last with 2 channels
    ("odd_tiles_32ch", odd_tiles, 32),         # 25 row tiles: the last pair's second tile is empty
])
def test_cta_pairs_equal_single_sm(name, grid_fn, B):
    """The paired-SM GEMM (cta_group::2, M = 256 over two CTAs' row tiles)
    and the single-SM GEMM give the same decomposition bit for bit, and both
    equal the FP32 template search's."""
    grid = grid_fn()
    sig = np.stack([synth.eeg_like_signal(4, 300 + b)[0] for b in range(B)]).astype(np.float32)
    P = 3
    h = act.act_grid_create(grid, 0)
    try:
        act.act_dictionary_build(h, act.ACT_DICT_RECOMPUTE)
        act.act_set_search(h, act.ACT_SEARCH_SHIFT)
        ref = gpu_decompose(h, sig, P)
        act.act_set_search(h, act.ACT_SEARCH_SHIFT_BF16)
        assert act.act_get_cta_pairs(h, B)
        paired = gpu_decompose(h, sig, P)
        act.act_set_cta_pairs(h, False)
        assert not act.act_get_cta_pairs(h, B)
        single = gpu_decompose(h, sig, P)
        act.act_set_cta_pairs(h, True)
        again = gpu_decompose(h, sig, P)
    finally:
        act.act_destroy(h)
    assert_same(paired, single)
    assert_same(paired, ref)
    assert_same(again, paired)


def test_cta_pairs_not_used_where_they_do_not_apply():
    h = act.act_grid_create(synth.grid_eeg(), 0)
    try:
        assert not act.act_get_cta_pairs(h, 64)  # no template build yet
        act.act_dictionary_build(h, act.ACT_DICT_RECOMPUTE)
        assert not act.act_get_cta_pairs(h, 1)   # one row tile
        assert act.act_get_cta_pairs(h, 64)
        with pytest.raises(act.ActError):
            act.act_get_cta_pairs(h, 0)
    finally:
        act.act_destroy(h)


def test_lockstep_against_oracle():
    grid = eeg_small()
    s, _ = synth.eeg_like_signal(2, 7)
    D, _ = oracle.dictionary(grid)
    h = act.act_grid_create(grid, 0)
    try:
        act.act_dictionary_build(h, act.ACT_DICT_RECOMPUTE)
        act.act_set_search(h, act.ACT_SEARCH_SHIFT_BF16)
        idx, _, coef, _, energy = gpu_decompose(h, s[None, :], 10)
        rs, cidx, ccoef = gpu_residual_chain(h, s, 10)
    finally:
        act.act_destroy(h)
    assert np.array_equal(cidx, idx[0])
    check_lockstep(lambda r: D @ r, rs, idx[0], coef[0], energy[0], lambda i: D[i])


def test_zero_signal_takes_the_fallback():
    """All scores 0: every item ties, the channel has too many items and is
    searched in full (index 0 wins)."""
    grid = eeg_small()
    a, b, (resolved, items, fallbacks) = both(grid, np.zeros((2, grid.n_samples), np.float32), 2)
    assert_same(a, b)
    assert fallbacks == 4 and np.all(b[0] == 0)


def test_fallback_queue_holds_only_the_overflowed_channels():
    """Zero channels among EEG-like ones: only the zero channels overflow, the
    full FP32 search runs over the queue of those channels alone, and every
    channel's decomposition still equals the FP32 template search's."""
    grid = eeg_small()
    sig = np.stack([synth.eeg_like_signal(2, 40 + b)[0] for b in range(6)]).astype(np.float32)
    sig[1] = 0.0
    sig[4] = 0.0
    P = 3
    a, b, (resolved, items, fallbacks) = both(grid, sig, P)
    assert_same(a, b)
    assert fallbacks == 2 * P and resolved == 4 * P
    assert np.all(b[0][[1, 4]] == 0)


def test_one_channel_many_time_centres():
    """One channel over 512 time centres and 18,432 templates (rows tile as
    1 channel x 128 time centres): the tile width falls back to 128 templates
    when 256 would leave room for fewer than two stages beside the scale rows."""
    grid = synth.Grid(2048, 500.0, synth.Axis(0.0, 4.0, 512), synth.Axis.linspace(20.0, 200.0, 96),
                      synth.Axis.linspace(-4.0, -1.5, 8), synth.Axis.linspace(-100.0, 100.0, 24))
    sig = synth.random_signals(97, 1, grid.n_samples)
    a, b, (resolved, items, fallbacks) = both(grid, sig, 3)
    assert_same(a, b)
    assert resolved + fallbacks == 3


def test_refinement_after_tensor_core_search():
    grid = eeg_small()
    sig = np.stack([synth.eeg_like_signal(2, 90 + b)[0] for b in range(2)]).astype(np.float32)
    a, b, _ = both(grid, sig, 5, refine=20)
    assert_same(a, b)


def test_ragged_plan():
    grids = [synth.scaled_grid(synth.grid_emg(n), fc_count=6, logdt_count=2, c_count=4) for n in (256, 1024)]
    lens = [1024, 256, 1024, 256, 256]
    sigs = [synth.random_signals(95 + i, 1, n)[0] for i, n in enumerate(lens)]
    offsets = np.concatenate([[0], np.cumsum(lens)]).astype(np.int64)
    hs = [act.act_grid_create(g, 0) for g in grids]
    try:
        for h in hs:
            act.act_dictionary_build(h, act.ACT_DICT_RECOMPUTE)
            act.act_set_search(h, act.ACT_SEARCH_SHIFT_BF16)
        plan = act.act_ragged_plan_create(hs, offsets, 4)
        try:
            C = len(lens)
            atoms = torch.empty((C, 4, act.ATOM_BYTES), dtype=torch.uint8, device="cuda")
            coef = torch.empty((C, 4), dtype=torch.float32, device="cuda")
            flat = torch.tensor(np.concatenate(sigs), dtype=torch.float32, device="cuda")
            act.act_ragged_decompose(plan, flat, atoms, coef)
            torch.cuda.synchronize()
            idx = act.atom_indices(atoms).cpu().numpy()
            coef = coef.cpu().numpy()
        finally:
            act.act_ragged_plan_destroy(plan)
        for c, n in enumerate(lens):
            h = hs[0] if n == 256 else hs[1]
            act.act_set_search(h, act.ACT_SEARCH_SHIFT)
            i1, _, c1, _, _ = gpu_decompose(h, sigs[c][None, :], 4)
            act.act_set_search(h, act.ACT_SEARCH_SHIFT_BF16)
            assert np.array_equal(i1[0], idx[c]) and np.array_equal(c1[0], coef[c])
    finally:
        for h in hs:
            act.act_destroy(h)


def test_not_available_without_templates():
    grid = ragged()
    h = act.act_grid_create(grid, 0)
    try:
        act.act_dictionary_build(h, act.ACT_DICT_FP32)
        act.act_set_search(h, act.ACT_SEARCH_SHIFT_BF16)
        with pytest.raises(act.ActError):
            gpu_decompose(h, synth.random_signals(1, 1, grid.n_samples), 1)
    finally:
        act.act_destroy(h)
