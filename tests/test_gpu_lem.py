"""GPU checks of the LEM-inspired hierarchical search (no stored
dictionary) against the FP64 oracle running the same algorithm with the same
SplitMix64 draws: order by order from the GPU's own residual, the GPU picks
the oracle's candidate (bit-identical parameters) unless the oracle's scores
of the two picks differ by less than 1e-5 relative (a near-tie), and the
refined trajectories agree."""
import numpy as np
import pytest
import torch

import oracle
from paper_2607_16629_gb300 import act, synth

pytestmark = pytest.mark.gpu

STEPS = ((64, 2, 2, 5), (32, 1, 1, 2.5), (16, 0.5, 0.5, 0.5))
RADIUS = (2, 2, 1, 2)


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    act.load_library()


def box(grid):
    axes = [grid.tc, grid.fc, grid.logdt, grid.c]
    lo = np.array([min(a.lo, a.lo + (a.count - 1) * a.step) for a in axes])
    hi = np.array([max(a.lo, a.lo + (a.count - 1) * a.step) for a in axes])
    return lo, hi


def n_coarse_default(grid, steps0):
    lo, hi = box(grid)
    return int(np.prod([max(1.0, np.ceil((h - l) / s)) for l, h, s in zip(lo, hi, steps0)]))


def lem_grid(grid, top_k, levels, seed, refine):
    h = act.act_grid_create(grid, 0)
    act.act_set_search(h, act.ACT_SEARCH_LEM)
    act.act_set_lem(h, 0, top_k, levels, STEPS, RADIUS, seed)
    act.act_set_refinement(h, refine)
    return h


@pytest.mark.parametrize("top_k,levels", [(1, 0), (4, 1), (4, 2)])
def test_lem_lockstep_against_oracle(top_k, levels):
    grid = synth.grid_eeg()
    lo, hi = box(grid)
    params = oracle.lem_params(n_coarse_default(grid, STEPS[0]), top_k, levels, STEPS, RADIUS)
    B, P, seed = 3, 4, 1234
    sigs = np.stack([synth.eeg_like_signal(2, 40 + b)[0] for b in range(B)]).astype(np.float32)
    h = lem_grid(grid, top_k, levels, seed, 0)
    try:
        r = sigs.copy()
        ties = 0
        for k in range(P):
            # one order at a time with the order counter of order k: run k+1
            # orders and compare the last one (earlier orders replayed exactly)
            atoms, coef, resid, energy = act.decompose(h, torch.tensor(sigs, device="cuda"), k + 1)
            torch.cuda.synchronize()
            assert act.act_grid_status(h) == act.ACT_OK
            th_gpu = act.atom_params(atoms).cpu().numpy()[:, k]
            assert np.all(act.atom_indices(atoms).cpu().numpy() == -1)
            for b in range(B):
                th_o, s_o = oracle.lem_select(params, lo, hi, grid.fs, r[b].astype(np.float64), seed, b, k)
                if not np.array_equal(th_gpu[b], th_o):
                    g, _ = oracle.atom(*th_gpu[b], grid.fs, grid.n_samples)
                    s_g = g @ r[b].astype(np.float64)
                    assert abs(abs(s_g) - abs(s_o)) <= 1e-5 * abs(s_o), (k, b, th_gpu[b], th_o)
                    ties += 1
            r = resid.cpu().numpy().astype(np.float32)
        # measured on GB300: no near-tie in any of these configurations; one is
        # allowed (a near-tie of distinct candidates may resolve either way)
        print(f"top_k {top_k} levels {levels}: {ties} near-ties in {B * P} picks")
        assert ties <= 1, ties
    finally:
        act.act_destroy(h)


def test_lem_with_bfgs_matches_oracle_trajectory():
    grid = synth.grid_eeg()
    lo, hi = box(grid)
    w, blo, bhi = oracle.refine_box(grid)
    params = oracle.lem_params(n_coarse_default(grid, STEPS[0]), 4, 2, STEPS, RADIUS)
    B, P, seed = 2, 5, 77
    sigs = np.stack([synth.eeg_like_signal(2, 60 + b)[0] for b in range(B)]).astype(np.float32)
    h = lem_grid(grid, 4, 2, seed, 60)
    try:
        atoms, coef, resid, energy = act.decompose(h, torch.tensor(sigs, device="cuda"), P)
        torch.cuda.synchronize()
        coef = coef.cpu().numpy()
        energy = energy.cpu().numpy()
    finally:
        act.act_destroy(h)
    for b in range(B):
        th, o_coef, o_r, o_en = oracle.mp_lem(params, lo, hi, w, blo, bhi, grid.fs, sigs[b].astype(np.float64), P,
                                              60, seed, b)
        np.testing.assert_allclose(np.abs(coef[b]), np.abs(o_coef), rtol=1e-3)
        np.testing.assert_allclose(energy[b], o_en, rtol=1e-3)
        assert np.all(np.diff(energy[b]) <= 1e-7 * energy[b, 0])


def test_lem_needs_no_dictionary_and_rejects_bad_settings():
    grid = synth.grid_c1()
    h = act.act_grid_create(grid, 0)
    try:
        act.act_set_search(h, act.ACT_SEARCH_LEM)
        sig = torch.tensor(synth.workload_c1().signals, dtype=torch.float32, device="cuda")
        atoms, coef, resid, energy = act.decompose(h, sig, 3)  # no act_dictionary_build
        torch.cuda.synchronize()
        assert act.act_grid_status(h) == act.ACT_OK
        e = energy.cpu().numpy()[0]
        assert e[-1] < 0.5 * e[0]
        with pytest.raises(act.ActError):
            act.act_set_lem(h, 0, 0, 2, STEPS, RADIUS, 0)       # top_k 0
        with pytest.raises(act.ActError):
            act.act_set_lem(h, 0, 4, 3, STEPS, RADIUS, 0)       # 3 levels
        with pytest.raises(act.ActError):
            act.act_set_lem(h, 0, 4, 2, ((0, 2, 2, 5),) * 3, RADIUS, 0)  # zero step
    finally:
        act.act_destroy(h)
