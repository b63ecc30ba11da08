"""Pins of the FP64 oracle against facts fixed outside the oracle itself.

Each test checks the oracle against something other than its own formulas:
numbers printed in the paper (Table 2), closed forms of Eq. (1), library
routines that reduce to a special case (scipy.signal.chirp, gausspulse,
numpy least squares), textbook MP properties, and brute force on tiny grids.
A plausible slip in the oracle (a dropped term, a wrong sign or unit, a
transposed operand, a wrong tie rule) fails at least one of them.
"""
import math
import os

import numpy as np
import pytest
from scipy import signal as sps

import oracle
from paper_2607_16629_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ---------------------------------------------------------------------------
# Table 2: grid sizes printed in the paper
# ---------------------------------------------------------------------------
def _table2():
    rows = {}
    with open(os.path.join(GOLDEN, "table2_ranges.txt")) as f:
        for line in f:
            if not line.strip() or line.startswith("#"):
                continue
            sig, axis, a, b, step, total = line.split()
            rows.setdefault(sig, {"total": int(total), "axes": {}})
            rows[sig]["axes"][axis] = (float(a), float(b), float(step))
    return rows


@pytest.mark.parametrize("sig", ["EEG", "EMG", "Radar"])
def test_table2_combination_counts(sig):
    """Table 2 prints 185,600 / 113,778 / 520,128 combinations."""
    row = _table2()[sig]
    total = 1
    for axis in ("tc", "fc", "logDt", "c"):
        total *= oracle.range_count(*row["axes"][axis])
    assert total == row["total"]


def test_range_count_matches_numpy_arange():
    for (a, b, s) in [(0, 256, 16), (-4, 0, 0.3), (20, 450, 10), (-10, 10, 0.75), (10, 8533, 100)]:
        assert oracle.range_count(a, b, s) == len(np.arange(a, b, s))


# ---------------------------------------------------------------------------
# Eq. (1): the complex atom and its closed forms
# ---------------------------------------------------------------------------
def test_eq1_prefactor_gives_unit_energy():
    """(sqrt(pi) Dt)^(-1/2) makes the integral of |g|^2 equal to 1; the
    sampled sum times 1/fs matches it when the atom sits well inside the
    window and spans many samples."""
    fs = 256.0
    for (tc, fc, ld, c) in [(256.0, 10.0, -2.5, 3.0), (300.0, 2.0, -2.8, -15.0),
                            (200.0, 30.0, -3.0, 0.0)]:
        g = oracle.atom_complex(tc, fc, ld, c, fs, 512)
        assert abs(np.sum(np.abs(g) ** 2) / fs - 1.0) < 1e-9


def test_eq1_envelope_falls_to_exp_minus_half_at_one_duration():
    """|g(tc + Dt)| / |g(tc)| = exp(-1/2), with Dt = exp(logDt) seconds."""
    fs = 200.0
    k = 20  # samples
    ld = math.log(k / fs)
    g = oracle.atom_complex(100.0, 17.0, ld, 40.0, fs, 256)
    assert abs(abs(g[100 + k]) / abs(g[100]) - math.exp(-0.5)) < 1e-13
    assert abs(abs(g[100 - k]) / abs(g[100]) - math.exp(-0.5)) < 1e-13


def test_eq1_instantaneous_frequency():
    """The phase of Eq. (1) advances at fc + 2 c (t - tc) cycles/s."""
    fs, tc, fc, c = 1000.0, 500.0, 50.0, 120.0
    g = oracle.atom_complex(tc, fc, -1.0, c, fs, 1000)
    ph = np.unwrap(np.angle(g))
    n = np.arange(1000)
    tau_mid = (n[:-1] + 0.5 - tc) / fs
    f_inst = np.diff(ph) * fs / (2 * math.pi)
    assert np.max(np.abs(f_inst - (fc + 2 * c * tau_mid))) < 1e-6


def test_real_atom_is_normalised_real_part_of_eq1():
    """The dictionary atom equals Re(Eq. 1) divided by its l2 norm."""
    for (tc, fc, ld, c) in [(10.0, 3.0, -2.0, 5.0), (250.0, 31.0, -3.0, -8.0), (128.5, 0.5, -0.5, 1.3)]:
        z = oracle.atom_complex(tc, fc, ld, c, 128.0, 256)
        g, deg = oracle.atom(tc, fc, ld, c, 128.0, 256)
        assert not deg
        ref = z.real / np.linalg.norm(z.real)
        assert np.max(np.abs(g - ref)) < 1e-13


def test_atom_against_scipy_chirp_and_gausspulse():
    """A Gaussian window (gausspulse's envelope) times a linear chirp
    (scipy.signal.chirp, f0 = fc, f1 = fc + 2c at t1 = 1 s), normalised,
    equals the oracle's atom: pins tc in samples, fc in Hz, c as written in
    Eq. (1) and logDt as a natural log."""
    fs, n = 256.0, 512
    for (tc, fc, ld, c) in [(100.0, 12.5, -2.2, 7.0), (400.0, 3.0, -1.0, -19.0), (0.0, 30.0, -2.9, 0.0)]:
        tau = (np.arange(n) - tc) / fs
        dt = math.exp(ld)
        bwr = -6.0
        bw = math.sqrt(-4.0 * math.log(10 ** (bwr / 20.0)) / (2 * dt * dt)) / math.pi
        _, env = sps.gausspulse(tau, fc=1.0, bw=bw, bwr=bwr, retenv=True)
        carrier = sps.chirp(tau, f0=fc, t1=1.0, f1=fc + 2 * c, method="linear")
        ref = env * carrier
        ref /= np.linalg.norm(ref)
        g, _ = oracle.atom(tc, fc, ld, c, fs, n)
        assert np.max(np.abs(g - ref)) < 1e-12


def test_atom_with_zero_chirp_is_gausspulse():
    """c = 0 reduces Eq. (1)'s real part to scipy's Gaussian-modulated cosine."""
    fs, n, tc, fc, ld = 500.0, 400, 210.0, 40.0, -3.5
    dt = math.exp(ld)
    tau = (np.arange(n) - tc) / fs
    bwr = -6.0
    bw = math.sqrt(-4.0 * math.log(10 ** (bwr / 20.0)) / (2 * dt * dt)) / (math.pi * fc)
    ref = sps.gausspulse(tau, fc=fc, bw=bw, bwr=bwr)
    ref /= np.linalg.norm(ref)
    g, _ = oracle.atom(tc, fc, ld, 0.0, fs, n)
    assert np.max(np.abs(g - ref)) < 1e-12


@pytest.mark.parametrize("fc,logdt,c", [(7.0, -1.2, 15.0), (30.0, -2.9, -20.0), (0.5, -0.5, 0.0)])
def test_eq1_depends_on_n_and_tc_only_through_their_difference(fc, logdt, c):
    """Eq. (1) sees t and tc only as t - tc: an atom centred S samples later
    is the same samples S places later (the template dictionary rests on
    this), and a normalised atom differs from its template window only by
    the window's own norm."""
    fs, L, S = 256.0, 512, 4
    a0 = oracle.atom_complex(100.0, fc, logdt, c, fs, L)
    a1 = oracle.atom_complex(100.0 + S, fc, logdt, c, fs, L)
    assert np.array_equal(a1[S:], a0[:-S])
    # template over lags -L+1 .. L-1 (tc = L - 1 puts m = n - tc in that range)
    tpl = oracle.atom_complex(float(L - 1), fc, logdt, c, fs, 2 * L - 1).real
    for tc in (0, 37, 300, 511):
        u = tpl[L - 1 - tc: 2 * L - 1 - tc]
        g, deg = oracle.atom(float(tc), fc, logdt, c, fs, L)
        assert not deg
        np.testing.assert_allclose(g, u / np.linalg.norm(u), rtol=0, atol=1e-14)


def test_every_dictionary_atom_has_unit_norm():
    grid = synth.scaled_grid(synth.grid_c1(), tc_count=8, fc_count=5)
    D, deg = oracle.dictionary(grid)
    assert not deg.any()
    assert np.max(np.abs(np.linalg.norm(D, axis=1) - 1.0)) < 1e-14


def test_dictionary_row_order_and_params():
    """Row i of D is the atom of flat index i, c fastest, tc slowest."""
    grid = synth.grid_small_test()
    D, _ = oracle.dictionary(grid)
    for i in [0, 1, 5, 17, grid.n_atoms - 1]:
        p = oracle.atom_params(grid, i)
        # the grid point at that position of numpy's row-major (C-order) layout
        axes = (grid.tc, grid.fc, grid.logdt, grid.c)
        pos = np.unravel_index(i, tuple(a.count for a in axes))
        assert p == tuple(float(a.values()[k]) for a, k in zip(axes, pos))
        g, _ = oracle.atom(*p, grid.fs, grid.n_samples)
        assert np.array_equal(D[i], g)
    assert oracle.atom_params(grid, 1)[3] == grid.c.lo + grid.c.step
    assert oracle.atom_params(grid, grid.c.count)[2] == grid.logdt.lo + grid.logdt.step


def test_degenerate_atom_is_zero():
    g, deg = oracle.atom(5000.0, 10.0, -6.0, 0.0, 100.0, 64)   # centre far outside the window
    assert deg and not np.any(g)


# ---------------------------------------------------------------------------
# Matching pursuit (Eq. 4, Fig. 1)
# ---------------------------------------------------------------------------
def test_identity_dictionary_reduces_to_sorting_by_magnitude():
    """With the canonical basis as dictionary, MP picks samples in order of
    decreasing |x| (lowest index on ties) with coefficients equal to them."""
    x = np.array([0.5, -3.0, 2.0, 0.0, 3.0, -1.0, 0.25, 2.0])
    idx, coef, r, en = oracle.mp(np.eye(8), x, 6)
    assert list(idx) == [1, 4, 2, 7, 5, 0]
    assert list(coef) == [-3.0, 3.0, 2.0, 2.0, -1.0, 0.5]
    assert list(r) == [0, 0, 0, 0, 0, 0, 0.25, 0]
    assert en[-1] == 0.25 ** 2


def test_lone_on_grid_atom_is_recovered_exactly():
    grid = synth.grid_c1()
    D, _ = oracle.dictionary(grid)
    for j, a in [(1234, 1.7), (16383, -0.6), (0, 2.0)]:
        idx, coef, r, en = oracle.mp(D, a * D[j], 1)
        assert idx[0] == j
        assert abs(coef[0] - a) <= 1e-12 * abs(a)
        assert np.linalg.norm(r) <= 1e-12 * abs(a)


def test_energy_identity_and_monotone_residual():
    """|s|^2 = sum_i c_i^2 + |r_k|^2 at every k; |r_k| never grows."""
    w = synth.workload_c1()
    grid = synth.scaled_grid(w.grid, tc_count=16, fc_count=8)
    D, _ = oracle.dictionary(grid)
    s = w.signals[0]
    idx, coef, r, en = oracle.mp(D, s, 12)
    e0 = float(s @ s)
    for k in range(13):
        assert abs(e0 - (np.sum(coef[:k] ** 2) + en[k])) <= 1e-12 * e0
    assert np.all(np.diff(en) <= 0.0)
    assert abs(en[-1] - float(r @ r)) <= 1e-14 * e0


def test_residual_orthogonal_to_chosen_atom():
    w = synth.workload_c1()
    grid = synth.scaled_grid(w.grid, tc_count=8, fc_count=8)
    D, _ = oracle.dictionary(grid)
    s = w.signals[0]
    r = s.copy()
    for _ in range(4):
        idx, coef, r, _ = oracle.mp(D, r, 1)
        assert abs(D[idx[0]] @ r) <= 1e-13 * np.linalg.norm(s)


def test_brute_force_best_one_term_approximation():
    """At every order the chosen atom and coefficient minimise |r - a g|^2
    over all atoms and all real a (least squares per atom, numpy lstsq)."""
    grid = synth.grid_small_test()
    D, _ = oracle.dictionary(grid)
    s = synth.random_signals(90, 1, grid.n_samples)[0]
    r = s.copy()
    for _ in range(6):
        errs, coefs = [], []
        for i in range(D.shape[0]):
            a, res, *_ = np.linalg.lstsq(D[i][:, None], r, rcond=None)
            coefs.append(a[0])
            errs.append(float(np.sum((r - a[0] * D[i]) ** 2)))
        best = int(np.argmin(errs))
        idx, coef, r_next, _ = oracle.mp(D, r, 1)
        assert idx[0] == best
        assert abs(coef[0] - coefs[best]) <= 1e-12 * max(1.0, abs(coefs[best]))
        r = r_next


def test_grid_mode_matches_stored_mode():
    """Regenerating atoms every order gives the same decomposition as the
    stored dictionary."""
    w = synth.workload_c1()
    grid = synth.scaled_grid(w.grid, tc_count=16, fc_count=8)
    D, _ = oracle.dictionary(grid)
    s = w.signals[0]
    a = oracle.mp(D, s, 5)
    b = oracle.mp_grid(grid, s, 5)
    assert np.array_equal(a[0], b[0])
    np.testing.assert_allclose(a[1], b[1], rtol=1e-13)
    np.testing.assert_allclose(a[2], b[2], atol=1e-13)
    assert np.all(b[4] >= 0.0) and np.all(b[4] <= 1.0)


def test_ties_go_to_lowest_index():
    sc = np.array([0.1, -0.7, 0.7, 0.3, -0.7])
    assert oracle.select(sc) == (1, 2)
    D = np.array([[1.0, 0.0], [1.0, 0.0], [0.0, 1.0]])
    idx, coef, r, _ = oracle.mp(D, np.array([2.0, 0.0]), 1)
    assert idx[0] == 0 and coef[0] == 2.0


def test_zero_signal_picks_index_zero_with_zero_coefficient():
    grid = synth.grid_small_test()
    D, _ = oracle.dictionary(grid)
    idx, coef, r, en = oracle.mp(D, np.zeros(grid.n_samples), 3)
    assert list(idx) == [0, 0, 0] and not np.any(coef) and not np.any(r) and not np.any(en)


def test_c1_recovers_planted_atoms():
    """Three on-grid atoms plus white noise (sigma 0.05): the first three
    orders find the planted atoms and leave about the noise energy."""
    w = synth.workload_c1()
    D, _ = oracle.dictionary(w.grid)
    s = w.signals[0]
    idx, coef, r, en = oracle.mp(D, s, w.n_atoms)
    planted = {w.grid.flat_of(
        round((tc - w.grid.tc.lo) / w.grid.tc.step), round((fc - w.grid.fc.lo) / w.grid.fc.step),
        round((ld - w.grid.logdt.lo) / w.grid.logdt.step), round((c - w.grid.c.lo) / w.grid.c.step))
        for (tc, fc, ld, c, a) in w.truth[0]}
    assert set(int(i) for i in idx[:3]) == planted
    noise_energy = w.grid.n_samples * 0.05 ** 2
    assert 0.5 * noise_energy < en[3] < 1.5 * noise_energy


# ---------------------------------------------------------------------------
# Off-grid refinement (Fig. 1): gradient and ascent
# ---------------------------------------------------------------------------
def _score_via_atom(theta, fs, r):
    g, _ = oracle.atom(*theta, fs, r.shape[0])
    return float(g @ r)


@pytest.mark.parametrize("theta,fs,L", [
    ((100.3, 10.2, -2.1, 3.3), 128.0, 256),
    ((600.7, 210.0, -2.9, -150.0), 1000.0, 1024),
    ((40.0, 30.5, -1.2, 12.0), 256.0, 512),
])
def test_score_gradient_matches_central_differences(theta, fs, L):
    """The analytic d<r, g(theta)>/dtheta against central differences of the
    score computed from the atom itself (normalisation term included)."""
    r = synth.random_signals(97, 1, L)[0]
    s, g = oracle.score_grad(theta, fs, r)
    assert abs(s - _score_via_atom(theta, fs, r)) <= 1e-12
    hs = [1e-4, 1e-5, 1e-6, 1e-5]
    for i, h in enumerate(hs):
        tp = list(theta)
        tm = list(theta)
        tp[i] += h
        tm[i] -= h
        fd = (_score_via_atom(tp, fs, r) - _score_via_atom(tm, fs, r)) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(g[i])), (i, fd, g[i])


def test_refinement_recovers_an_off_grid_chirplet():
    """A noiseless off-grid atom: started inside the optimum's basin (for a
    real atom |<g, x>| oscillates in tc with period about fs / (2 fc), here
    about 5 samples), the ascent climbs to |<g, x>| = 1 at the true
    parameters."""
    grid = synth.grid_c1()
    true = (61.3, 12.7, -2.23, 2.9)
    x, _ = oracle.atom(*true, grid.fs, grid.n_samples)
    start = (62.5, 12.9, -2.1, 2.3)
    w, lo, hi = oracle.refine_box(grid)
    th, J = oracle.refine(start, grid.fs, x, 40, w, lo, hi)
    assert J > 1 - 1e-8
    np.testing.assert_allclose(th, true, atol=2e-3)
    assert J > abs(_score_via_atom(start, grid.fs, x))


def test_refinement_reaches_the_bfgs_optimum():
    """On a noisy residual the refinement reaches the local optimum that
    scipy's BFGS (an independent implementation of the paper's refinement
    method) reaches from the same grid start, to within 1e-6 of the
    objective."""
    from scipy.optimize import minimize
    w0 = synth.workload_c1()
    grid = w0.grid
    r = w0.signals[0]
    D, _ = oracle.dictionary(grid)
    j = int(np.argmax(np.abs(D @ r)))
    start = oracle.atom_params(grid, j)
    w, lo, hi = oracle.refine_box(grid)
    th, J = oracle.refine(start, grid.fs, r, 60, w, lo, hi)

    def f(z):
        return -abs(_score_via_atom(tuple(z * w), grid.fs, r))

    res = minimize(f, np.array(start) / w, method="BFGS", options={"gtol": 1e-10})
    assert J >= abs(D[j] @ r)
    assert abs(J - (-res.fun)) <= 1e-6 * J


def test_refined_mp_keeps_the_mp_identities():
    """With refinement the residual stays orthogonal to the subtracted atom,
    energy is conserved and never grows, and every refined order takes at
    least as much energy as its grid winner would."""
    w0 = synth.workload_c1()
    grid = synth.scaled_grid(w0.grid, tc_count=16, fc_count=8)
    s = w0.signals[0]
    idx, coef, th, r, en = oracle.mp_refine(grid, s, 5, 20)
    e0 = float(s @ s)
    for k in range(6):
        assert abs(e0 - (np.sum(coef[:k] ** 2) + en[k])) <= 1e-12 * e0
    assert np.all(np.diff(en) <= 0)
    g, _ = oracle.atom(*th[-1], grid.fs, grid.n_samples)
    assert abs(g @ r) <= 1e-12 * np.sqrt(e0)
    D, _ = oracle.dictionary(grid)
    rr = s.copy()
    for k in range(5):
        grid_gain = (D[idx[k]] @ rr) ** 2
        assert coef[k] ** 2 >= grid_gain * (1 - 1e-12)
        gk, _ = oracle.atom(*th[k], grid.fs, grid.n_samples)
        rr = rr - coef[k] * gk


# ---------------------------------------------------------------------------
# Hierarchical (LEM-inspired) search, Sec. VII-A
# ---------------------------------------------------------------------------
def test_splitmix64_matches_published_outputs():
    with open(os.path.join(GOLDEN, "splitmix64_seed0.txt")) as f:
        rows = [l.split() for l in f if l.strip() and not l.startswith("#")]
    for n, v in rows:
        assert oracle.splitmix64_at(0, int(n)) == int(v, 16)


def test_lhs_uses_every_stratum_once_per_axis():
    lo = np.array([0.0, 0.5, -3.0, -20.0])
    hi = np.array([508.0, 32.0, -0.5, 20.0])
    n = 300
    pts = oracle.lhs(lo, hi, n, seed=123, channel=3, order=7)
    for a in range(4):
        strata = np.floor((pts[:, a] - lo[a]) / (hi[a] - lo[a]) * n).astype(int)
        assert sorted(strata) == list(range(n))
        assert np.all(pts[:, a] >= lo[a]) and np.all(pts[:, a] <= hi[a])
    other = oracle.lhs(lo, hi, n, seed=123, channel=3, order=8)
    assert not np.array_equal(pts, other)
    assert np.array_equal(pts, oracle.lhs(lo, hi, n, seed=123, channel=3, order=7))


def _lem_box(grid):
    axes = [grid.tc, grid.fc, grid.logdt, grid.c]
    lo = np.array([min(a.lo, a.lo + (a.count - 1) * a.step) for a in axes])
    hi = np.array([max(a.lo, a.lo + (a.count - 1) * a.step) for a in axes])
    return lo, hi


def test_lem_levels_never_lose_score_and_find_a_lone_atom():
    """Each refinement level contains its parents (offset 0), so the best
    |score| never drops; on a lone atom whose parameters lie on the last
    level's lattice around a coarse candidate the search recovers it."""
    grid = synth.grid_eeg()
    lo, hi = _lem_box(grid)
    true = (300.0, 12.0, -1.5, 5.0)
    x, _ = oracle.atom(*true, grid.fs, grid.n_samples)
    x = x + 0.01 * synth.random_signals(5, 1, grid.n_samples)[0]
    steps = [(64, 2, 2, 5), (32, 1, 1, 2.5), (16, 0.5, 0.5, 0.5)]
    best = []
    for levels in (0, 1, 2):
        p = oracle.lem_params(1024, 4, levels, steps, (2, 2, 1, 2))
        th, sc = oracle.lem_select(p, lo, hi, grid.fs, x, 9, 0, 0)
        best.append(abs(sc))
        g, _ = oracle.atom(*th, grid.fs, grid.n_samples)
        assert abs(sc - g @ x) <= 1e-12
    assert best[0] <= best[1] <= best[2]
    assert best[2] > 0.9


def test_lem_neighbours_are_the_clamped_offset_lattice():
    """The neighbourhood dictionary of Sec. VII-A: around every kept vector,
    each offset -R..R steps per axis (radius (2, 2, 1, 2): 375 candidates per
    parent), clamped to the box; built here independently with numpy's
    meshgrid (index order 'ij', so c runs fastest as in the oracle)."""
    grid = synth.grid_eeg()
    lo, hi = _lem_box(grid)
    step = np.array([32.0, 1.0, 1.0, 2.5])
    radius = (2, 2, 1, 2)
    kept = np.array([[300.0, 12.0, -1.5, 5.0],      # interior
                     [10.0, 0.75, -3.0, 19.0],      # clamped on tc, fc, logdt and c
                     [511.0, 31.5, -0.5, -20.0]])   # at the top corner
    got = oracle.lem_neighbours(kept, step, radius, lo, hi)
    assert got.shape == (3 * 375, 4)
    offs = np.stack(np.meshgrid(*[np.arange(-r, r + 1) for r in radius], indexing="ij"), -1).reshape(-1, 4)
    want = np.concatenate([np.clip(k + offs * step, lo, hi) for k in kept])
    assert np.array_equal(got, want)
    assert np.array_equal(got[:375][np.all(offs == 0, axis=1)][0], kept[0])  # the parent itself is a candidate


def test_lem_topk_is_a_stable_sort_without_duplicates():
    """top-k of Sec. VII-A: the k largest |score| in a stable order (lowest
    index first among equal |score|), a parameter vector equal to one already
    kept skipped; compared with numpy's stable argsort."""
    rng = np.random.default_rng(17)
    n, k = 400, 12
    cand = rng.integers(0, 6, size=(n, 4)).astype(np.float64)     # many repeated vectors
    score = rng.integers(-20, 21, size=n).astype(np.float64) / 4.0  # many equal |scores|
    kept, ks = oracle.lem_topk(cand, score, k)
    order = np.argsort(-np.abs(score), kind="stable")
    want, seen = [], set()
    for i in order:
        key = tuple(cand[i])
        if key in seen:
            continue
        seen.add(key)
        want.append(i)
        if len(want) == k:
            break
    assert np.array_equal(kept, cand[want]) and np.array_equal(ks, score[want])
    # fewer distinct vectors than k: all of them, once
    c2 = np.repeat(cand[:3], 5, axis=0)
    s2 = np.arange(15, dtype=np.float64)
    kept2, _ = oracle.lem_topk(c2, s2, 8)
    assert len(kept2) == len({tuple(v) for v in c2})
