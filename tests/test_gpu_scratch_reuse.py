"""Work buffers and recorded CUDA graphs: growing a grid's buffers must never
leave a cached graph pointing at freed memory, and a ragged plan must not
share reallocatable memory with its grids.

Each sequence below changes the channel count of one search back and forth on
a grid whose base buffers are already large enough, so that only the
search's own scratch (hierarchical-search candidates, tensor-core search
maxima, shifted residual rows) grows.  Every call must give exactly what a
fresh grid gives for the same input (the MP loop of Fig. 1, Eq. (4))."""
import numpy as np
import pytest
import torch

from paper_2607_16629_gb300 import act, synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    act.load_library()


def _run(h, sig, P):
    atoms, coef, resid, energy = act.decompose(h, torch.tensor(sig, dtype=torch.float32, device="cuda"), P)
    torch.cuda.synchronize()
    st = act.act_grid_status(h)
    assert st == act.ACT_OK, act.status_name(st)
    return tuple(t.cpu().numpy() for t in (atoms, coef, resid, energy))


def _fresh(grid, build, mode, sig, P, setup=None):
    h = act.act_grid_create(grid, 0)
    try:
        act.act_dictionary_build(h, build)
        act.act_set_search(h, mode)
        if setup:
            setup(h)
        return _run(h, sig, P)
    finally:
        act.act_destroy(h)


def _same(a, b, what):
    for x, y, name in zip(a, b, ("atoms", "coeffs", "residuals", "energies")):
        assert np.array_equal(x, y), f"{what}: {name} differ from a fresh grid's"


def _sequence(grid, build, mode, counts, P, big=64, setup=None):
    """On one grid: the FP32-sized base buffers for `big` channels first,
    then `mode` with each channel count of `counts` in turn, each compared
    with a fresh grid."""
    sigs = {B: synth.random_signals(90 + B, B, grid.n_samples) for B in set(counts) | {big}}
    ref = {B: _fresh(grid, build, mode, sigs[B], P, setup) for B in set(counts)}
    h = act.act_grid_create(grid, 0)
    try:
        act.act_dictionary_build(h, build)
        if setup:
            setup(h)
        # base buffers for `big` channels (a search without scratch of its own)
        act.act_set_search(h, act.ACT_SEARCH_SHIFT if build == act.ACT_DICT_RECOMPUTE else act.ACT_SEARCH_FP32)
        _run(h, sigs[big], P)
        act.act_set_search(h, mode)
        for i, B in enumerate(counts):
            _same(_run(h, sigs[B], P), ref[B], f"call {i} ({B} channels)")
    finally:
        act.act_destroy(h)


def test_template_tensor_search_channels_1_64_1():
    grid = synth.scaled_grid(synth.grid_eeg(), tc_count=32, fc_count=16)
    _sequence(grid, act.ACT_DICT_RECOMPUTE, act.ACT_SEARCH_SHIFT_BF16, [1, 64, 1, 64], 3)


def test_dense_tensor_search_channels_1_130_1():
    grid = synth.scaled_grid(synth.grid_eeg(), tc_count=16, fc_count=16)
    _sequence(grid, act.ACT_DICT_BF16, act.ACT_SEARCH_BF16, [1, 130, 1], 3, big=130)


def test_hierarchical_search_channels_2_4_2():
    grid = synth.scaled_grid(synth.grid_eeg(), tc_count=16, fc_count=16)

    def small_lem(h):
        act.act_set_lem(h, n_coarse=256)
    _sequence(grid, act.ACT_DICT_FP32, act.ACT_SEARCH_LEM, [2, 4, 2], 2, big=64, setup=small_lem)


def test_ragged_plan_unaffected_by_larger_grid_calls():
    """A plan keeps its own scratch: a later, larger act_decompose on one of
    its grids neither breaks nor changes it."""
    lens = [256, 512, 256, 512, 512]
    grids = {L: synth.scaled_grid(synth.grid_emg(L), tc_count=16, fc_count=8) for L in set(lens)}
    handles = {}
    try:
        for L, g in grids.items():
            handles[L] = act.act_grid_create(g, 0)
            act.act_dictionary_build(handles[L], act.ACT_DICT_RECOMPUTE)
        sig = [synth.random_signals(70 + i, 1, L)[0] for i, L in enumerate(lens)]
        flat = torch.tensor(np.concatenate(sig), dtype=torch.float32, device="cuda")
        offsets = np.concatenate([[0], np.cumsum(lens)])
        plan = act.act_ragged_plan_create([handles[L] for L in sorted(handles)], offsets, 3)
        try:
            C, P = len(lens), 3

            def run_plan():
                atoms = torch.empty((C, P, act.ATOM_BYTES), dtype=torch.uint8, device="cuda")
                coef = torch.empty((C, P), dtype=torch.float32, device="cuda")
                res = torch.empty_like(flat)
                en = torch.empty((C, P + 1), dtype=torch.float64, device="cuda")
                act.act_ragged_decompose(plan, flat, atoms, coef, res, en)
                torch.cuda.synchronize()
                return tuple(t.cpu().numpy() for t in (atoms, coef, res, en))

            before = run_plan()
            # the grid of length 512 now runs 200 channels: its own scratch grows
            _run(handles[512], synth.random_signals(5, 200, 512), 2)
            after = run_plan()
            _same(after, before, "ragged plan after a larger call on its grid")
        finally:
            act.act_ragged_plan_destroy(plan)
    finally:
        for h in handles.values():
            act.act_destroy(h)
