"""Shared pieces of the GPU parity tests: running the CUDA path through the
C ABI and checking its decomposition order by order against the FP64 oracle.

Tolerances (FP32 path): the selected atom must be the oracle's whenever the
oracle's top-two |scores| on the same residual differ by more than 1e-5
relative; coefficients and residual energies must agree within 1e-5
relative.  Near the noise floor the relative bound is measured against the
residual norm instead (absolute floor ATOL_REL * |r|)."""
import functools

import numpy as np
import torch

import oracle
from paper_2607_16629_gb300 import act

GAP = 1e-5      # near-tie threshold on the oracle's relative top-2 gap
RTOL = 1e-5     # coefficients and residual energies
ATOL_REL = 2e-6  # absolute floor, relative to |r_k|, for coefficients near 0


def gpu_decompose(h, signals: np.ndarray, P: int, host: bool = False):
    """Runs act_decompose and returns numpy outputs
    (idx [B,P], params [B,P,4], coef [B,P], resid [B,L], energy [B,P+1])."""
    sig = torch.tensor(np.asarray(signals, dtype=np.float32))
    if not host:
        sig = sig.cuda()
        atoms, coef, resid, energy = act.decompose(h, sig, P)
        torch.cuda.synchronize()
    else:
        B, L = sig.shape
        sig = sig.pin_memory()
        atoms = torch.empty((B, P, act.ATOM_BYTES), dtype=torch.uint8).pin_memory()
        coef = torch.empty((B, P), dtype=torch.float32).pin_memory()
        resid = torch.empty((B, L), dtype=torch.float32).pin_memory()
        energy = torch.empty((B, P + 1), dtype=torch.float64).pin_memory()
        act.act_decompose(h, sig, B, P, atoms, coef, resid, energy)
    st = act.act_grid_status(h)
    assert st == act.ACT_OK, act.status_name(st)
    return (act.atom_indices(atoms).cpu().numpy(), act.atom_params(atoms).cpu().numpy(),
            coef.cpu().numpy(), resid.cpu().numpy(), energy.cpu().numpy())


def gpu_residual_chain(h, signal: np.ndarray, P: int):
    """r_0 .. r_P of one channel obtained by P chained one-order calls, plus
    the per-order index and coefficient."""
    rs = [np.asarray(signal, dtype=np.float32)]
    idx, coef = [], []
    for _ in range(P):
        i, _, c, r, _ = gpu_decompose(h, rs[-1][None, :], 1)
        idx.append(int(i[0, 0]))
        coef.append(float(c[0, 0]))
        rs.append(r[0].astype(np.float32))
    return rs, np.array(idx), np.array(coef)


def check_lockstep(score_fn, rs, idx, coef, energy=None, dictionary_row=None):
    """Order-by-order check of the GPU decomposition against the oracle.

    score_fn(r) -> FP64 oracle scores of every atom against residual r.
    rs[k] is the GPU residual entering order k (float32); idx/coef are the
    GPU's choices; energy (optional) the GPU's |r_k|^2 log.  Returns the
    number of near-tie orders seen."""
    ties = 0
    for k in range(len(idx)):
        r = rs[k].astype(np.float64)
        rn = float(np.linalg.norm(r))
        sc = score_fn(r)
        best, second = oracle.select(sc)
        a = abs(sc[best])
        gap = (a - abs(sc[second])) / a if a > 0 else 0.0
        if gap > GAP:
            assert idx[k] == best, f"order {k}: gpu {idx[k]} oracle {best} gap {gap:.3e}"
        else:
            ties += 1
            assert abs(sc[idx[k]]) >= a * (1 - 2 * GAP), f"order {k}: gpu pick is not a near-tie"
        c_ref = sc[idx[k]]
        assert abs(coef[k] - c_ref) <= RTOL * abs(c_ref) + ATOL_REL * rn, \
            f"order {k}: coef {coef[k]} vs {c_ref}"
        if energy is not None and dictionary_row is not None:
            g = dictionary_row(idx[k])
            e_ref = float(np.sum((r - c_ref * g) ** 2))
            assert abs(energy[k + 1] - e_ref) <= RTOL * e_ref + 4 * ATOL_REL * rn * rn, \
                f"order {k}: energy {energy[k + 1]} vs {e_ref}"
    return ties


@functools.lru_cache(maxsize=1)
def full_dictionary(grid):
    """The oracle's FP64 dictionary of a grid, built once per test session
    (the 2,097,152-atom EEG-like grid takes 8.6 GB of host memory)."""
    D, deg = oracle.dictionary(grid)
    assert not deg.any()
    return D
