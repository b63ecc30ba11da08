"""GPU checks that the two forms of the per-order CUDA graph give the same
bits.  With profiling on, event nodes sit between the search kernels, so
no kernel there is a programmatic dependent of the one before; without
profiling the template searches' kernels are chained as programmatic
dependents (each waits on its predecessor inside the kernel).  The
decomposition must not depend on which form ran, for every search mode,
with and without refinement."""
import numpy as np
import pytest
import torch

from paper_2607_16629_gb300 import act, synth
from parity_helpers import gpu_decompose

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    act.load_library()


def eeg_small():
    return synth.scaled_grid(synth.grid_eeg(), tc_count=32, fc_count=16)


def both_forms(h, sig, P):
    act.act_set_profiling(h, False)
    plain = gpu_decompose(h, sig, P)
    act.act_set_profiling(h, True)
    profiled = gpu_decompose(h, sig, P)
    _, _, orders, kernels = act.act_profile_read(h)
    act.act_set_profiling(h, False)
    assert orders == P and kernels > 0
    return plain, profiled


@pytest.mark.parametrize("build,mode", [
    (act.ACT_DICT_RECOMPUTE, act.ACT_SEARCH_SHIFT_BF16),
    (act.ACT_DICT_RECOMPUTE, act.ACT_SEARCH_SHIFT),
    (act.ACT_DICT_BF16, act.ACT_SEARCH_BF16),
    (act.ACT_DICT_BF16, act.ACT_SEARCH_FP32),
])
@pytest.mark.parametrize("refine", [0, 10])
def test_profiled_graph_equals_plain_graph(build, mode, refine):
    grid = eeg_small()
    sig = np.stack([synth.eeg_like_signal(2, 60 + b)[0] for b in range(5)]).astype(np.float32)
    h = act.act_grid_create(grid, 0)
    try:
        act.act_dictionary_build(h, build)
        act.act_set_search(h, mode)
        act.act_set_refinement(h, refine)
        plain, profiled = both_forms(h, sig, 6)
    finally:
        act.act_destroy(h)
    for x, y in zip(plain, profiled):
        assert np.array_equal(x, y)


def test_profiled_graph_equals_plain_graph_hierarchical():
    grid = eeg_small()
    sig = np.stack([synth.eeg_like_signal(2, 70 + b)[0] for b in range(3)]).astype(np.float32)
    h = act.act_grid_create(grid, 0)
    try:
        act.act_set_search(h, act.ACT_SEARCH_LEM)
        act.act_set_refinement(h, 5)
        plain, profiled = both_forms(h, sig, 4)
    finally:
        act.act_destroy(h)
    for x, y in zip(plain, profiled):
        assert np.array_equal(x, y)
