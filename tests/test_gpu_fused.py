"""The single-launch decomposition of small FP32 dictionaries (Fig. 1's
loop, Eq. (4)) against the per-order GEMV and update kernels (bit for bit)
and against the FP64 oracle (lock-step), through the C ABI."""
import numpy as np
import pytest
import torch

from paper_2607_16629_gb300 import act, synth
from parity_helpers import check_lockstep, full_dictionary, gpu_decompose, gpu_residual_chain

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    act.load_library()


def _both_forms(grid, signals, P, ctas_per_sm=(2,)):
    """Outputs with the per-order kernels, then with the single launch at
    each CTAs-per-SM setting (asserting that it is the one taken)."""
    B = signals.shape[0]
    h = act.act_grid_create(grid, 0)
    try:
        act.act_dictionary_build(h, act.ACT_DICT_FP32)
        act.act_set_fused(h, 0)
        assert act.act_get_fused(h, B) == 0
        ref = gpu_decompose(h, signals, P)
        outs = []
        for c in ctas_per_sm:
            act.act_set_fused(h, c)
            assert act.act_get_fused(h, B) > 0
            outs.append(gpu_decompose(h, signals, P))  # device buffers: the kernel alone
            # host buffers: the same kernel inside the grid's graph, then copies
            outs.append(gpu_decompose(h, signals, P, host=True))
    finally:
        act.act_destroy(h)
    return ref, outs


def _assert_same(ref, out):
    for a, b, name in zip(ref, out, ("index", "params", "coef", "residual", "energy")):
        assert np.array_equal(a, b), f"{name} differs"


def _signals(grid, B, seed):
    rng = np.random.default_rng(seed)
    return rng.standard_normal((B, grid.n_samples)).astype(np.float32)


@pytest.mark.parametrize("seed,B,P", [(None, 1, 5), (None, 1, 1), (3, 1, 12), (4, 1, 40), (5, 2, 7), (6, 2, 1)])
def test_single_launch_equals_per_order_kernels_c1(seed, B, P):
    """16,384 atoms, N = 256: the outputs of both forms are identical (the
    check workload's signal, and white-noise signals)."""
    w = synth.workload_c1()
    grid = w.grid
    sig = w.signals[:1] if seed is None else _signals(grid, B, seed)
    ref, outs = _both_forms(grid, np.asarray(sig, dtype=np.float32), P, ctas_per_sm=(1, 2, 4))
    for out in outs:
        _assert_same(ref, out)


@pytest.mark.parametrize("name,grid", [
    # N = 200: the padded row (256) is longer than the window
    ("n200", synth.scaled_grid(synth.Grid(200, 2000.0, synth.Axis(0, 32, 7), synth.Axis(20, 10, 43),
                                          synth.Axis(-4, 0.3, 14), synth.Axis(-10, 0.75, 27)), fc_count=11)),
    # 12,288 atoms (25 MB; not a multiple of the rows one pass of the grid covers), N = 512
    ("eeg12k", synth.scaled_grid(synth.grid_eeg(), tc_count=12, fc_count=4, c_count=32)),
])
def test_single_launch_equals_per_order_kernels(name, grid):
    sig = _signals(grid, 2, 7)
    ref, outs = _both_forms(grid, sig, 9)
    _assert_same(ref, outs[0])


def test_single_launch_paper_epoch_setting():
    """The paper's EEG ranges (Table 2) at a coarser time-centre step:
    tc 0..256 step 128, 23,200 atoms (23.8 MB), N = 256, 10 orders."""
    desc = act.act_grid_from_ranges(256, 256.0, (0, 256, 128), (0.5, 15, 0.5), (-4, 1, 0.5), (-10, 10, 0.5))
    sig = synth.eeg_like_signal(6, 0, n_samples=256, fs=256.0)[0][None, :].astype(np.float32)
    h = act.act_grid_create(desc, 0)
    try:
        K, _ = act.act_grid_size(h)
        assert K == 23200
        act.act_dictionary_build(h, act.ACT_DICT_FP32)
        act.act_set_fused(h, 0)
        ref = gpu_decompose(h, sig, 10)
        act.act_set_fused(h, 2)
        assert act.act_get_fused(h, 1) > 0
        out = gpu_decompose(h, sig, 10)
    finally:
        act.act_destroy(h)
    _assert_same(ref, out)


def test_single_launch_lockstep_against_oracle():
    """Order by order against the FP64 oracle on the 16,384-atom grid: the
    residual entering each order comes from chained one-order calls (each a
    single launch of one order)."""
    w = synth.workload_c1()
    grid, P = w.grid, 12
    sig = np.asarray(w.signals[:1], dtype=np.float32)
    D = full_dictionary(grid)
    h = act.act_grid_create(grid, 0)
    try:
        act.act_dictionary_build(h, act.ACT_DICT_FP32)
        assert act.act_get_fused(h, 1) > 0
        idx, _, coef, resid, energy = gpu_decompose(h, sig, P)
        rs, idx_c, coef_c = gpu_residual_chain(h, sig[0], P)
    finally:
        act.act_destroy(h)
    assert np.array_equal(idx[0], idx_c) and np.array_equal(coef[0], coef_c)
    ties = check_lockstep(lambda r: D @ r, rs, idx[0], coef[0], energy[0], lambda i: D[i])
    assert ties <= 1
    # the returned residual is the last one of the chain
    assert np.array_equal(resid[0], rs[P])


def test_single_launch_not_used_where_it_does_not_apply():
    w = synth.workload_c1()
    h = act.act_grid_create(w.grid, 0)
    try:
        act.act_dictionary_build(h, act.ACT_DICT_FP32)
        assert act.act_get_fused(h, 1) > 0
        assert act.act_get_fused(h, 2) > 0
        assert act.act_get_fused(h, 3) == 0          # more channels: the per-order kernels
        act.act_set_refinement(h, 4)
        assert act.act_get_fused(h, 1) == 0          # refinement runs its own kernels
        act.act_set_refinement(h, 0)
        act.act_set_profiling(h, True)
        assert act.act_get_fused(h, 1) == 0          # per-order events need per-order kernels
        act.act_set_profiling(h, False)
        act.act_set_search(h, act.ACT_SEARCH_LEM)
        assert act.act_get_fused(h, 1) == 0
        act.act_set_search(h, act.ACT_SEARCH_AUTO)
        assert act.act_get_fused(h, 1) > 0
        with pytest.raises(RuntimeError):
            act.act_set_fused(h, -1)
    finally:
        act.act_destroy(h)
    # a larger dictionary (1 GiB) takes the per-order kernels
    big = synth.scaled_grid(synth.grid_eeg(), tc_count=64, fc_count=32)
    h = act.act_grid_create(big, 0)
    try:
        act.act_dictionary_build(h, act.ACT_DICT_FP32)
        assert act.act_get_fused(h, 1) == 0
    finally:
        act.act_destroy(h)


def test_single_launch_optional_outputs():
    """Outputs the caller leaves out (null pointers) are not written; the
    ones it asks for equal those of a call that asks for everything."""
    w = synth.workload_c1()
    P = 6
    sig = torch.tensor(np.asarray(w.signals[:1], dtype=np.float32), device="cuda")
    h = act.act_grid_create(w.grid, 0)
    try:
        act.act_dictionary_build(h, act.ACT_DICT_FP32)
        assert act.act_get_fused(h, 1) > 0
        atoms, coef, resid, energy = act.decompose(h, sig, P)
        for keep in ("atoms", "coef", "resid", "energy"):
            out = {"atoms": torch.zeros_like(atoms), "coef": torch.zeros_like(coef),
                   "resid": torch.zeros_like(resid), "energy": torch.zeros_like(energy)}
            args = [out[k] if k == keep else None for k in ("atoms", "coef", "resid", "energy")]
            act.act_decompose(h, sig, 1, P, *args)
            torch.cuda.synchronize()
            assert act.act_grid_status(h) == act.ACT_OK
            ref = {"atoms": atoms, "coef": coef, "resid": resid, "energy": energy}[keep]
            assert torch.equal(out[keep], ref), keep
    finally:
        act.act_destroy(h)


def test_single_launch_reports_nonfinite_input():
    w = synth.workload_c1()
    s = np.asarray(w.signals[:1], dtype=np.float32).copy()
    s[0, 17] = np.inf
    h = act.act_grid_create(w.grid, 0)
    try:
        act.act_dictionary_build(h, act.ACT_DICT_FP32)
        assert act.act_get_fused(h, 1) > 0
        act.decompose(h, torch.tensor(s, device="cuda"), 3)
        assert act.act_grid_status(h) == act.ACT_ERR_NONFINITE
        assert act.act_grid_status(h) == act.ACT_OK  # read and cleared
        # the next clean call is clean
        act.decompose(h, torch.tensor(np.asarray(w.signals[:1], dtype=np.float32), device="cuda"), 3)
        assert act.act_grid_status(h) == act.ACT_OK
    finally:
        act.act_destroy(h)


def test_single_launch_many_orders():
    """300 orders (the key slots rotate 100 times; the per-order graph has
    600 kernels): both forms equal bit for bit, the energy never rises and
    the energy identity holds."""
    w = synth.workload_c1()
    sig = _signals(w.grid, 1, 21)
    ref, outs = _both_forms(w.grid, sig, 300)
    for out in outs:
        _assert_same(ref, out)
    _, _, coef, _, energy = ref
    e0 = energy[0, 0]
    assert np.all(np.diff(energy[0]) <= 1e-7 * e0)
    assert abs(e0 - (np.sum(coef[0].astype(np.float64) ** 2) + energy[0, -1])) <= 1e-5 * e0
