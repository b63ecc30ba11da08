"""GPU checks of uneven batches (channels of different window lengths in one
plan): the plan's outputs equal the per-length act_decompose calls bit for
bit, in the caller's channel order, for FP32 and BF16 grids, with device or
host buffers; and every channel is checked order by order against the FP64
oracle of its window length."""
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


def small_emg_grid(L):
    return synth.scaled_grid(synth.grid_emg(L), tc_count=32, fc_count=12, logdt_count=4, c_count=8)


def batch(lengths, seed_base=0):
    sigs = [synth.emg_like_signal(seed_base + i, int(L))[0] for i, L in enumerate(lengths)]
    offsets = np.concatenate([[0], np.cumsum([len(s) for s in sigs])]).astype(np.int64)
    return sigs, offsets


@pytest.mark.parametrize("mode", [act.ACT_DICT_FP32, act.ACT_DICT_BF16])
@pytest.mark.parametrize("host", [False, True])
def test_ragged_equals_per_length_calls(mode, host):
    lengths = [512, 256, 1024, 256, 512, 2048, 1024, 256, 512]
    sigs, offsets = batch(lengths)
    C, P = len(lengths), 4
    grids = {L: act.act_grid_create(small_emg_grid(L), 0) for L in sorted(set(lengths))}
    try:
        for h in grids.values():
            act.act_dictionary_build(h, mode)
        plan = act.act_ragged_plan_create(list(grids.values()), offsets, P)
        try:
            groups, kernels = act.act_ragged_plan_info(plan)
            assert groups == 4 and kernels > 0
            flat = np.concatenate(sigs).astype(np.float32)
            dev = "cpu" if host else "cuda"
            mk = (lambda *a, **k: torch.empty(*a, **k).pin_memory()) if host else \
                (lambda *a, **k: torch.empty(*a, device="cuda", **k))
            sig_t = torch.tensor(flat, device=dev)
            if host:
                sig_t = sig_t.pin_memory()
            atoms = mk((C, P, act.ATOM_BYTES), dtype=torch.uint8)
            coefs = mk((C, P), dtype=torch.float32)
            resid = mk((len(flat),), dtype=torch.float32)
            energy = mk((C, P + 1), dtype=torch.float64)
            for _ in range(2):  # replays give the same result
                act.act_ragged_decompose(plan, sig_t, atoms, coefs, resid, energy)
                torch.cuda.synchronize()
                for h in grids.values():
                    assert act.act_grid_status(h) == act.ACT_OK
                for c, L in enumerate(lengths):
                    ref = act.decompose(grids[L], torch.tensor(sigs[c][None, :], dtype=torch.float32,
                                                               device="cuda"), P)
                    torch.cuda.synchronize()
                    assert torch.equal(atoms[c].cpu(), ref[0][0].cpu())
                    assert torch.equal(coefs[c].cpu(), ref[1][0].cpu())
                    assert torch.equal(resid[offsets[c]:offsets[c + 1]].cpu(), ref[2][0].cpu())
                    assert torch.equal(energy[c].cpu(), ref[3][0].cpu())
        finally:
            act.act_ragged_plan_destroy(plan)
    finally:
        for h in grids.values():
            act.act_destroy(h)


def test_ragged_plan_rejects_bad_layouts_and_goes_stale():
    lengths = [256, 512]
    sigs, offsets = batch(lengths)
    h256 = act.act_grid_create(small_emg_grid(256), 0)
    h512 = act.act_grid_create(small_emg_grid(512), 0)
    try:
        act.act_dictionary_build(h256, act.ACT_DICT_FP32)
        with pytest.raises(act.ActError) as e:
            act.act_ragged_plan_create([h256, h512], offsets, 2)
        assert e.value.status == act.ACT_ERR_NOT_BUILT
        act.act_dictionary_build(h512, act.ACT_DICT_FP32)
        with pytest.raises(act.ActError) as e:  # no grid for length 300
            act.act_ragged_plan_create([h256, h512], [0, 256, 556], 2)
        assert e.value.status == act.ACT_ERR_INVALID_ARG
        with pytest.raises(act.ActError):       # decreasing offsets
            act.act_ragged_plan_create([h256, h512], [0, 256, 100], 2)
        plan = act.act_ragged_plan_create([h256, h512], offsets, 2)
        try:
            sig_t = torch.tensor(np.concatenate(sigs).astype(np.float32), device="cuda")
            act.act_ragged_decompose(plan, sig_t)
            act.act_dictionary_build(h512, act.ACT_DICT_FP32)   # rebuild: the plan is stale
            with pytest.raises(act.ActError) as e:
                act.act_ragged_decompose(plan, sig_t)
            assert e.value.status == act.ACT_ERR_NOT_BUILT
        finally:
            act.act_ragged_plan_destroy(plan)
    finally:
        act.act_destroy(h256)
        act.act_destroy(h512)


@pytest.mark.parametrize("mode", [act.ACT_DICT_FP32, act.ACT_DICT_BF16, act.ACT_DICT_RECOMPUTE])
def test_ragged_lockstep_against_oracle(mode):
    """Every channel of an uneven batch, order by order, against the FP64
    oracle of its window length (Eq. (4)): a one-order plan is chained (its
    residuals fed back as the next signals), each order is checked from the
    plan's own residual, and a P-order plan gives the chain's selections."""
    lengths = [256, 1024, 512, 256, 2048, 512, 1024, 256]
    sigs, offsets = batch(lengths, seed_base=20)
    C, P = len(lengths), 5
    grids = {L: small_emg_grid(L) for L in sorted(set(lengths))}
    dicts = {L: oracle.dictionary(g)[0] for L, g in grids.items()}
    hs = {L: act.act_grid_create(g, 0) for L, g in grids.items()}
    try:
        for h in hs.values():
            act.act_dictionary_build(h, mode)
        plan1 = act.act_ragged_plan_create(list(hs.values()), offsets, 1)
        planP = act.act_ragged_plan_create(list(hs.values()), offsets, P)
        try:
            def run(plan, flat, p):
                atoms = torch.empty((C, p, act.ATOM_BYTES), dtype=torch.uint8, device="cuda")
                coef = torch.empty((C, p), dtype=torch.float32, device="cuda")
                res = torch.empty_like(flat)
                act.act_ragged_decompose(plan, flat, atoms, coef, res, None)
                torch.cuda.synchronize()
                for h in hs.values():
                    assert act.act_grid_status(h) == act.ACT_OK
                return act.atom_indices(atoms).cpu().numpy(), coef.cpu().numpy(), res

            flat = torch.tensor(np.concatenate(sigs).astype(np.float32), device="cuda")
            rs = [flat.cpu().numpy()]
            idx, coef = [], []
            for _ in range(P):
                i1, c1, flat = run(plan1, flat, 1)
                idx.append(i1[:, 0])
                coef.append(c1[:, 0])
                rs.append(flat.cpu().numpy())
            idx, coef = np.stack(idx, 1), np.stack(coef, 1)
            iP, cP, _ = run(planP, torch.tensor(np.concatenate(sigs).astype(np.float32), device="cuda"), P)
            assert np.array_equal(iP, idx) and np.array_equal(cP, coef)
            ties = 0
            for c, L in enumerate(lengths):
                seg = slice(offsets[c], offsets[c + 1])
                D = dicts[L]
                ties += check_lockstep(lambda r: D @ r, [r[seg] for r in rs], idx[c], coef[c])
            print(f"{ties} near-ties in {C * P} orders")
        finally:
            act.act_ragged_plan_destroy(plan1)
            act.act_ragged_plan_destroy(planP)
    finally:
        for h in hs.values():
            act.act_destroy(h)
