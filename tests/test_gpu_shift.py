"""GPU parity of the template dictionary (ACT_DICT_RECOMPUTE) and its
shift-correlation search (ACT_SEARCH_SHIFT) against the FP64 oracle.

No atom rows exist on this path: every atom is formed in-kernel as a window
of its (fc, logDt, c) template, because the real atom of Eq. (1) depends on
n - tc only.  The oracle still scores every atom by its plain definition
(each atom generated and normalised on its own), so these tests check the
translation argument and the kernel together.  Tolerances as for the FP32
path: same atom unless the oracle's top two differ by less than 1e-5
relative, coefficients and energies within 1e-5 relative; scores within
4e-6 |x| (one FP32 accumulation chain of L products per score)."""
import numpy as np
import pytest
import torch

import oracle
from paper_2607_16629_gb300 import act, synth
from parity_helpers import check_lockstep, gpu_decompose, gpu_residual_chain

pytestmark = pytest.mark.gpu

SCORE_TOL = 4e-6


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    act.load_library()


class Templates:
    """Context manager: a grid handle with a template dictionary."""

    def __init__(self, grid, refine=0):
        self.grid, self.refine = grid, refine

    def __enter__(self):
        self.h = act.act_grid_create(self.grid, 0)
        act.act_dictionary_build(self.h, act.ACT_DICT_RECOMPUTE)
        act.act_set_search(self.h, act.ACT_SEARCH_SHIFT)  # the FP32 template search (AUTO picks tensor cores)
        if self.refine:
            act.act_set_refinement(self.h, self.refine)
        return self.h

    def __exit__(self, *a):
        act.act_destroy(self.h)


def eeg_small():
    """Every range of the EEG-like grid, 32 x 16 x 8 x 32 = 131,072 atoms
    (tc step 16 samples)."""
    return synth.scaled_grid(synth.grid_eeg(), tc_count=32, fc_count=16)


def ragged():
    """Negative first tc, 37 time centres 5 samples apart running past the
    window's end, a window of 203 samples (not a multiple of the step) and
    105 templates (not a multiple of 32)."""
    return synth.Grid(203, 500.0, synth.Axis(-3.0, 5.0, 37), synth.Axis(20.0, 35.0, 5),
                      synth.Axis(-4.0, 0.5, 3), synth.Axis(-60.0, 20.0, 7))


GRIDS = [
    ("c1", synth.grid_c1()),
    ("eeg_small", eeg_small()),
    ("ragged", ragged()),
    ("dense_tc", synth.Grid(96, 256.0, synth.Axis(0.0, 1.0, 96), synth.Axis(4.0, 9.0, 3),
                            synth.Axis(-3.0, 0.6, 4), synth.Axis(-20.0, 40.0, 2))),
    ("radar_scaled", synth.scaled_grid(synth.grid_radar(), fc_count=4, logdt_count=2, c_count=4)),
]


def project(h, sig):
    B = sig.shape[0]
    K, _ = act.act_grid_size(h)
    scores = torch.empty((B, K), dtype=torch.float32, device="cuda")
    act.act_project(h, torch.tensor(sig, dtype=torch.float32, device="cuda"), B, scores)
    torch.cuda.synchronize()
    assert act.act_grid_status(h) == act.ACT_OK
    return scores.cpu().numpy()


@pytest.mark.parametrize("name,grid", GRIDS)
def test_projection_matches_oracle(name, grid):
    B = 3
    sig = synth.random_signals(71, B, grid.n_samples)
    D, _ = oracle.dictionary(grid)
    with Templates(grid) as h:
        got = project(h, sig)
    for b in range(B):
        x = sig[b].astype(np.float32).astype(np.float64)
        err = np.max(np.abs(got[b] - D @ x))
        assert err <= SCORE_TOL * np.linalg.norm(x), (name, b, err)


@pytest.mark.parametrize("name,grid", [GRIDS[1], GRIDS[2]])
def test_every_launch_configuration_gives_the_same_bits(name, grid):
    sig = synth.random_signals(72, 2, grid.n_samples)
    with Templates(grid) as h:
        ref = project(h, sig)
        tried = 0
        for J in (8, 16, 32):
            for W in range(1, 9):
                for S in (1, 2, 3):
                    for C in (0, 1):
                        try:
                            act.act_set_shift_tuning(h, J, W, S, C)
                        except act.ActError:
                            continue
                        got = act.act_get_shift_tuning(h)
                        assert got[:3] == (J, W, S) and (C == 0 or got[3] == C)
                        assert np.array_equal(project(h, sig), ref), (J, W, S, C)
                        tried += 1
        assert tried >= 12
        for bad in ((12, 2, 2, 0), (32, 9, 2, 0), (16, 2, 4, 0), (16, 2, 0, 0), (16, 2, 2, -1), (16, 2, 2, 99)):
            with pytest.raises(act.ActError):
                act.act_set_shift_tuning(h, *bad)


@pytest.mark.parametrize("name,grid,P", [(GRIDS[0][0], GRIDS[0][1], 5), (GRIDS[1][0], GRIDS[1][1], 12),
                                         (GRIDS[2][0], GRIDS[2][1], 8), (GRIDS[3][0], GRIDS[3][1], 8)])
def test_mp_lockstep(name, grid, P):
    if name == "c1":
        s = synth.workload_c1().signals[0]
    elif name == "eeg_small":
        s, _ = synth.eeg_like_signal(2, 7)
    else:
        s = synth.random_signals(73, 1, grid.n_samples)[0]
    D, _ = oracle.dictionary(grid)
    with Templates(grid) as h:
        idx, par, coef, resid, energy = gpu_decompose(h, s[None, :], P)
        rs, cidx, ccoef = gpu_residual_chain(h, s, P)
    assert np.array_equal(cidx, idx[0]) and np.array_equal(ccoef, coef[0])
    assert np.array_equal(rs[-1], resid[0])
    check_lockstep(lambda r: D @ r, rs, idx[0], coef[0], energy[0], lambda i: D[i])
    for k in range(P):
        assert par[0, k] == pytest.approx(oracle.atom_params(grid, idx[0, k]), abs=0)


def test_mp_matches_oracle_trajectory_c1():
    w = synth.workload_c1()
    with Templates(w.grid) as h:
        idx, _, coef, _, energy = gpu_decompose(h, w.signals, w.n_atoms)
    D, _ = oracle.dictionary(w.grid)
    o_idx, o_coef, _, o_en = oracle.mp(D, w.signals[0].astype(np.float32).astype(np.float64), w.n_atoms)
    assert np.array_equal(idx[0], o_idx)
    np.testing.assert_allclose(coef[0], o_coef, rtol=1e-5)
    np.testing.assert_allclose(energy[0], o_en, rtol=1e-5)


def test_multichannel_equals_single_channel_runs():
    grid = ragged()
    sig = synth.random_signals(74, 5, grid.n_samples)
    with Templates(grid) as h:
        idx, _, coef, resid, energy = gpu_decompose(h, sig, 6)
        for b in range(5):
            i1, _, c1, r1, e1 = gpu_decompose(h, sig[b:b + 1], 6)
            assert np.array_equal(i1[0], idx[b]) and np.array_equal(c1[0], coef[b])
            assert np.array_equal(r1[0], resid[b]) and np.array_equal(e1[0], energy[b])


def test_host_buffers_and_autotune_keep_the_bits():
    grid = eeg_small()
    sig = synth.random_signals(75, 2, grid.n_samples)
    with Templates(grid) as h:
        ref = gpu_decompose(h, sig, 6)
        ms = act.act_autotune(h, torch.tensor(sig, dtype=torch.float32, device="cuda"), 2)
        assert ms > 0.0
        J, W, S, per_sm = act.act_get_shift_tuning(h)
        assert J in (8, 16, 32) and 1 <= W <= 8 and 1 <= S <= 3 and per_sm > 0
        for host in (False, True):
            got = gpu_decompose(h, sig, 6, host=host)
            for a, b in zip(ref, got):
                assert np.array_equal(a, b)


def test_zero_signal_selects_index_zero():
    grid = ragged()
    with Templates(grid) as h:
        idx, _, coef, resid, energy = gpu_decompose(h, np.zeros((1, grid.n_samples), np.float32), 3)
    assert np.all(idx == 0) and np.all(coef == 0) and not resid.any() and not energy.any()


def test_degenerate_atoms_match_oracle():
    """Atoms centred 5000 samples outside the window underflow to zero on
    both sides (scale 0) and are never selected."""
    grid = synth.Grid(64, 100.0, synth.Axis(20.0, 4980.0, 2), synth.Axis(10.0, 5.0, 2),
                      synth.Axis(-6.0, 0.5, 2), synth.Axis(0.0, 1.0, 2))
    D, deg = oracle.dictionary(grid)
    assert deg.sum() == 8
    s = synth.random_signals(33, 1, grid.n_samples)[0]
    with Templates(grid) as h:
        sc = project(h, s[None, :])[0]
        idx, _, _, _, _ = gpu_decompose(h, s[None, :], 3)
    assert not sc[deg].any()
    o_idx, _, _, _ = oracle.mp(D, s.astype(np.float32).astype(np.float64), 3)
    assert np.array_equal(idx[0], o_idx)


def test_refinement_after_template_search_equals_refinement_after_fp32_search():
    """Same grid winners -> the same BFGS starts and updates, bit for bit."""
    grid = eeg_small()
    sig = np.stack([synth.eeg_like_signal(2, 90 + b)[0] for b in range(2)]).astype(np.float32)
    with Templates(grid, refine=20) as h:
        a = gpu_decompose(h, sig, 6)
    h2 = act.act_grid_create(grid, 0)
    try:
        act.act_dictionary_build(h2, act.ACT_DICT_FP32)
        act.act_set_refinement(h2, 20)
        b = gpu_decompose(h2, sig, 6)
    finally:
        act.act_destroy(h2)
    assert np.array_equal(a[0], b[0])
    for x, y in zip(a[1:], b[1:]):
        assert np.array_equal(x, y)


def test_ragged_plan_with_template_grids():
    grids = [synth.grid_emg(256), synth.grid_emg(512)]
    grids = [synth.scaled_grid(g, fc_count=6, logdt_count=2, c_count=4) for g in grids]
    lens = [256, 512, 512, 256, 512]
    sigs = [synth.random_signals(80 + i, 1, n)[0] for i, n in enumerate(lens)]
    offsets = np.concatenate([[0], np.cumsum(lens)]).astype(np.int64)
    hs = [act.act_grid_create(g, 0) for g in grids]
    try:
        for h in hs:
            act.act_dictionary_build(h, act.ACT_DICT_RECOMPUTE)
            act.act_set_search(h, act.ACT_SEARCH_SHIFT)
        plan = act.act_ragged_plan_create(hs, offsets, 5)
        try:
            flat = torch.tensor(np.concatenate(sigs), dtype=torch.float32, device="cuda")
            C = len(lens)
            atoms = torch.empty((C, 5, act.ATOM_BYTES), dtype=torch.uint8, device="cuda")
            coef = torch.empty((C, 5), dtype=torch.float32, device="cuda")
            resid = torch.empty(int(offsets[-1]), dtype=torch.float32, device="cuda")
            energy = torch.empty((C, 6), dtype=torch.float64, device="cuda")
            act.act_ragged_decompose(plan, flat, atoms, coef, resid, energy)
            torch.cuda.synchronize()
            idx = act.atom_indices(atoms).cpu().numpy()
            coef = coef.cpu().numpy()
            resid = resid.cpu().numpy()
        finally:
            act.act_ragged_plan_destroy(plan)
        for c, n in enumerate(lens):
            h = hs[0] if n == 256 else hs[1]
            i1, _, c1, r1, _ = gpu_decompose(h, sigs[c][None, :], 5)
            assert np.array_equal(i1[0], idx[c]) and np.array_equal(c1[0], coef[c])
            assert np.array_equal(r1[0], resid[offsets[c]:offsets[c + 1]])
    finally:
        for h in hs:
            act.act_destroy(h)


def test_unsupported_and_invalid_uses():
    # time centres that are not whole samples
    with pytest.raises(act.ActError):
        with Templates(synth.grid_small_test()):
            pass
    grid = ragged()
    with Templates(grid) as h:
        out = torch.empty((1, grid.n_samples), dtype=torch.float32, device="cuda")
        with pytest.raises(act.ActError):
            act.act_dictionary_rows(h, 0, 1, out)          # no rows are stored
        act.act_set_search(h, act.ACT_SEARCH_FP32)
        with pytest.raises(act.ActError):
            gpu_decompose(h, synth.random_signals(1, 1, grid.n_samples), 1)
        act.act_set_search(h, act.ACT_SEARCH_SHIFT)
        gpu_decompose(h, synth.random_signals(1, 1, grid.n_samples), 1)
    h = act.act_grid_create(grid, 0)
    try:
        act.act_dictionary_build(h, act.ACT_DICT_FP32)
        act.act_set_search(h, act.ACT_SEARCH_SHIFT)
        with pytest.raises(act.ActError):
            gpu_decompose(h, synth.random_signals(1, 1, grid.n_samples), 1)
        with pytest.raises(act.ActError):
            act.act_set_shift_tuning(h, 32, 4, 2, 0)
    finally:
        act.act_destroy(h)


def test_full_eeg_grid():
    """The 2,097,152-atom EEG-like grid (tc step 4 samples) in the launch
    configuration the benchmark times: sampled scores against atoms the
    oracle generates one by one, the first orders in lock-step with the
    oracle scoring every atom, and the energy identity at every order."""
    w = synth.workload_c2()
    grid, s, P = w.grid, w.signals[0], w.n_atoms
    rng = np.random.default_rng(9)
    rows = np.unique(np.concatenate([rng.integers(0, grid.n_atoms, 400), [0, grid.n_atoms - 1]]))
    with Templates(grid) as h:
        sc = project(h, s[None, :])[0]
        act.act_autotune(h, torch.tensor(s[None, :], dtype=torch.float32, device="cuda"), 1)
        idx, _, coef, resid, energy = gpu_decompose(h, s[None, :], P)
        rs, cidx, ccoef = gpu_residual_chain(h, s, 3)
    x = s.astype(np.float32).astype(np.float64)
    for i in rows:
        g, _ = oracle.atom(*oracle.atom_params(grid, int(i)), grid.fs, grid.n_samples)
        assert abs(sc[i] - g @ x) <= SCORE_TOL * np.linalg.norm(x), i
    assert np.array_equal(cidx, idx[0, :3])
    check_lockstep(lambda r: oracle.scores_grid(grid, r), rs, cidx, ccoef)
    e0 = energy[0, 0]
    for k in range(P + 1):
        assert abs(e0 - (np.sum(coef[0, :k].astype(np.float64) ** 2) + energy[0, k])) <= 1e-5 * e0
    assert np.all(np.diff(energy[0]) <= 1e-7 * e0)
