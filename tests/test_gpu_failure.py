"""Failure paths, made without faulting the GPU.

* Bounded device waits: with a grid's wait limit at 0 every pipeline wait
  polls once, so the first copy or consumer that is not already done makes
  the kernel give up.  The kernel records ACT_ERR_DEVICE_TIMEOUT, lets the
  copies it issued land, releases its tensor memory and exits; the next call
  with the default limit must be clean and give a fresh grid's result.
* Out of memory (the one failure mode the paper discusses, Sec. IV-C): the
  library's allocations are made to fail on the host; the call reports
  ACT_ERR_OOM and the grid stays usable.
* ACT_DICT_AUTO: stored FP32 rows when they fit the memory budget, the
  template dictionary when they do not (whole-sample time centres), OOM when
  neither form fits."""
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
    yield
    act.act_inject_alloc_failure(0)


def _run(h, sig, P):
    atoms, coef, resid, energy = act.decompose(h, torch.tensor(sig, dtype=torch.float32, device="cuda"), P)
    torch.cuda.synchronize()
    return act.act_grid_status(h), tuple(t.cpu().numpy() for t in (atoms, coef, resid, energy))


def _grid(build, search, grid, tuning=None):
    h = act.act_grid_create(grid, 0)
    act.act_dictionary_build(h, build)
    act.act_set_search(h, search)
    if tuning:
        tuning(h)
    return h


EEG_SMALL = synth.scaled_grid(synth.grid_eeg(), tc_count=64, fc_count=32)  # 524,288 atoms, 1 GB FP32


@pytest.mark.parametrize("name,build,search,tuning,must_time_out", [
    ("fp32_bulk_stream", act.ACT_DICT_FP32, act.ACT_SEARCH_FP32, lambda h: act.act_set_tuning(h, -1), True),
    ("fp32_load_stream", act.ACT_DICT_FP32, act.ACT_SEARCH_FP32, lambda h: act.act_set_tuning(h, 152), True),
    ("bf16_dense", act.ACT_DICT_BF16, act.ACT_SEARCH_BF16, None, True),
    ("bf16_templates", act.ACT_DICT_RECOMPUTE, act.ACT_SEARCH_SHIFT_BF16, None, True),
    # the FP32 template search stages L2-resident templates: a poll may find
    # every copy already landed, so a timeout is likely but not certain
    ("fp32_templates", act.ACT_DICT_RECOMPUTE, act.ACT_SEARCH_SHIFT, None, False),
])
def test_wait_limit_zero_times_out_then_recovers(name, build, search, tuning, must_time_out):
    B, P = 4, 3
    sig = np.stack([synth.eeg_like_signal(3, ch)[0] for ch in range(B)])
    h = _grid(build, search, EEG_SMALL, tuning)
    ref_h = _grid(build, search, EEG_SMALL, tuning)
    try:
        st_ref, ref = _run(ref_h, sig, P)
        assert st_ref == act.ACT_OK
        act.act_set_wait_limit(h, 0)
        st, _ = _run(h, sig, P)
        if must_time_out:
            assert st == act.ACT_ERR_DEVICE_TIMEOUT, act.status_name(st)
        else:
            assert st in (act.ACT_OK, act.ACT_ERR_DEVICE_TIMEOUT), act.status_name(st)
        assert act.act_grid_status(h) == act.ACT_OK  # read and cleared
        act.act_set_wait_limit(h, 2_000_000_000)
        st, out = _run(h, sig, P)
        assert st == act.ACT_OK, act.status_name(st)
        for x, y in zip(out, ref):
            assert np.array_equal(x, y)
    finally:
        act.act_destroy(h)
        act.act_destroy(ref_h)


def test_wait_limit_zero_paired_template_gemm():
    """The paired-SM template GEMM (a cluster of two CTAs): both CTAs give up,
    wait for each other, release their tensor memory and exit; the next call
    is clean and equal to a fresh grid's."""
    B, P = 16, 2
    grid = synth.grid_eeg()
    sig = np.stack([synth.eeg_like_signal(3, ch)[0] for ch in range(B)])
    h = _grid(act.ACT_DICT_RECOMPUTE, act.ACT_SEARCH_SHIFT_BF16, grid)
    ref_h = _grid(act.ACT_DICT_RECOMPUTE, act.ACT_SEARCH_SHIFT_BF16, grid)
    try:
        assert act.act_get_cta_pairs(h, B)
        st_ref, ref = _run(ref_h, sig, P)
        assert st_ref == act.ACT_OK
        act.act_set_wait_limit(h, 0)
        st, _ = _run(h, sig, P)
        assert st == act.ACT_ERR_DEVICE_TIMEOUT, act.status_name(st)
        assert act.act_grid_status(h) == act.ACT_OK
        act.act_set_wait_limit(h, 2_000_000_000)
        st, out = _run(h, sig, P)
        assert st == act.ACT_OK, act.status_name(st)
        for x, y in zip(out, ref):
            assert np.array_equal(x, y)
    finally:
        act.act_destroy(h)
        act.act_destroy(ref_h)


def test_negative_wait_limit_rejected():
    h = act.act_grid_create(synth.grid_small_test(), 0)
    try:
        with pytest.raises(act.ActError) as e:
            act.act_set_wait_limit(h, -1)
        assert e.value.status == act.ACT_ERR_INVALID_ARG
    finally:
        act.act_destroy(h)


@pytest.mark.parametrize("build,search", [
    (act.ACT_DICT_FP32, act.ACT_SEARCH_FP32),
    (act.ACT_DICT_BF16, act.ACT_SEARCH_BF16),
    (act.ACT_DICT_RECOMPUTE, act.ACT_SEARCH_SHIFT_BF16),
])
def test_injected_allocation_failures(build, search):
    """Each allocation of a build, then of a first decomposition, is made to
    fail in turn (the 1st, the 2nd, ...); each failing call returns
    ACT_ERR_OOM, and the same grid then builds and decomposes exactly like a
    fresh one."""
    grid = synth.scaled_grid(synth.grid_eeg(), tc_count=16, fc_count=16)
    B, P = 3, 3
    sig = synth.random_signals(11, B, grid.n_samples)
    ref_h = _grid(build, search, grid)
    try:
        st, ref = _run(ref_h, sig, P)
        assert st == act.ACT_OK
    finally:
        act.act_destroy(ref_h)
    h = act.act_grid_create(grid, 0)
    try:
        act.act_set_search(h, search)
        # the build: fail the n-th allocation for n = 1, 2, ... until it succeeds
        for n in range(1, 12):
            act.act_inject_alloc_failure(n)
            try:
                act.act_dictionary_build(h, build)
                ok = True
            except act.ActError as e:
                assert e.status == act.ACT_ERR_OOM
                ok = False
            act.act_inject_alloc_failure(0)
            if ok:
                break
            with pytest.raises(act.ActError) as e:  # nothing is kept from a failed build
                act.act_decompose(h, torch.zeros((1, grid.n_samples), device="cuda"), 1, 1)
            assert e.value.status == act.ACT_ERR_NOT_BUILT
        act.act_dictionary_build(h, build)
        # the decomposition's buffers: the n-th allocation fails
        for n in range(1, 30):
            act.act_inject_alloc_failure(n)
            try:
                st, out = _run(h, sig, P)
                failed = False
            except act.ActError as e:
                assert e.status == act.ACT_ERR_OOM
                failed = True
            act.act_inject_alloc_failure(0)
            if not failed:
                break
            # a grid that failed to grow is usable: a fresh attempt succeeds
            st, out = _run(h, sig, P)
            assert st == act.ACT_OK
            for x, y in zip(out, ref):
                assert np.array_equal(x, y)
            act.act_destroy(h)
            h = act.act_grid_create(grid, 0)
            act.act_set_search(h, search)
            act.act_dictionary_build(h, build)
        st, out = _run(h, sig, P)
        assert st == act.ACT_OK
        for x, y in zip(out, ref):
            assert np.array_equal(x, y)
    finally:
        act.act_inject_alloc_failure(0)
        act.act_destroy(h)


def test_auto_dictionary_choice():
    whole = synth.scaled_grid(synth.grid_eeg(), tc_count=32, fc_count=16)     # tc step 16 samples
    frac = synth.scaled_grid(synth.grid_eeg(), tc_count=48, fc_count=16)      # tc step 10.67 samples
    B, P = 2, 3
    sig = synth.random_signals(12, B, 512)
    h = act.act_grid_create(whole, 0)
    try:
        act.act_dictionary_build(h, act.ACT_DICT_AUTO)       # fits: stored FP32 rows
        assert act.act_dictionary_mode(h) == act.ACT_DICT_FP32
        st, fp32 = _run(h, sig, P)
        assert st == act.ACT_OK
        act.act_set_memory_budget(h, 64 << 20)               # rows 268 MB > 64 MB > templates 26 MB
        act.act_dictionary_build(h, act.ACT_DICT_AUTO)
        assert act.act_dictionary_mode(h) == act.ACT_DICT_RECOMPUTE
        st, tpl = _run(h, sig, P)
        assert st == act.ACT_OK
        # the template search scores (sum r u) / |u| instead of sum r (u / |u|):
        # equal selections except within FP32 rounding of a tie
        assert np.mean(act.atom_indices(torch.tensor(tpl[0])).numpy() ==
                       act.atom_indices(torch.tensor(fp32[0])).numpy()) >= 0.8
        act.act_set_memory_budget(h, 1 << 10)                # nothing fits
        with pytest.raises(act.ActError) as e:
            act.act_dictionary_build(h, act.ACT_DICT_AUTO)
        assert e.value.status == act.ACT_ERR_OOM
        with pytest.raises(act.ActError) as e:
            act.act_dictionary_mode(h)
        assert e.value.status == act.ACT_ERR_NOT_BUILT
    finally:
        act.act_destroy(h)
    h = act.act_grid_create(frac, 0)
    try:
        act.act_set_memory_budget(h, 1 << 20)                # fractional centres: no template form
        with pytest.raises(act.ActError) as e:
            act.act_dictionary_build(h, act.ACT_DICT_AUTO)
        assert e.value.status == act.ACT_ERR_OOM
        act.act_set_memory_budget(h, 0)
        act.act_dictionary_build(h, act.ACT_DICT_AUTO)
        assert act.act_dictionary_mode(h) == act.ACT_DICT_FP32
    finally:
        act.act_destroy(h)


def test_wait_limit_zero_single_launch():
    """The single-launch decomposition of a small FP32 dictionary: with the
    wait limit at 0 every CTA but the last to arrive gives up at the first
    grid barrier and raises the abort flag, which ends the others' waits;
    the next call is clean and equal to a fresh grid's."""
    w = synth.workload_c1()
    B, P = 2, 4
    sig = np.stack([w.signals[0], w.signals[0][::-1]]).astype(np.float32)
    h = _grid(act.ACT_DICT_FP32, act.ACT_SEARCH_FP32, w.grid)
    ref_h = _grid(act.ACT_DICT_FP32, act.ACT_SEARCH_FP32, w.grid)
    try:
        assert act.act_get_fused(h, B) > 1
        st_ref, ref = _run(ref_h, sig, P)
        assert st_ref == act.ACT_OK
        act.act_set_wait_limit(h, 0)
        st, _ = _run(h, sig, P)
        assert st == act.ACT_ERR_DEVICE_TIMEOUT, act.status_name(st)
        assert act.act_grid_status(h) == act.ACT_OK
        act.act_set_wait_limit(h, 2_000_000_000)
        st, out = _run(h, sig, P)
        assert st == act.ACT_OK, act.status_name(st)
        for x, y in zip(out, ref):
            assert np.array_equal(x, y)
    finally:
        act.act_destroy(h)
        act.act_destroy(ref_h)
