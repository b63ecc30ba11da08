"""Seeded synthetic inputs and workload definitions.

This module is shared by the FP64 oracle's tests and by the CUDA path as the
*source of inputs only*: it draws random signals and describes parameter
grids.  It contains no step of the decomposition itself (no dictionary, no
normalisation, no projection, no selection, no residual update), and it
imports neither the oracle nor the CUDA binding.

Signals stand in for the paper's public datasets (EEG, EMG and radar
micro-Doppler windows, Sec. III-B1 and Sec. V-A), which are not available:
they are sums of Gaussian-windowed linear-FM bursts plus white or pink noise,
with the window lengths, sample rates and parameter ranges of the workloads
below.  Each burst is produced with library routines
(``scipy.signal.chirp`` for the linear-FM carrier and the Gaussian envelope
returned by ``scipy.signal.gausspulse``) and scaled to a stated l2 norm.

Conventions (the readings used throughout the project):
  * time centre ``tc`` is in samples, ``tau = (n - tc) / fs`` in seconds;
  * frequency centre ``fc`` in Hz;
  * chirp rate ``c`` in Hz/s as it multiplies ``tau**2`` inside the phase of
    Eq. (1), so the instantaneous frequency is ``fc + 2 c tau``;
  * ``logdt`` is the natural log of the duration in seconds.
"""
from __future__ import annotations

import dataclasses
import math
from typing import Dict, List, Sequence, Tuple

import numpy as np
from scipy import signal as sps

SEED_BASE = 0xAC7 * 1000


def seed_for(config: int, channel: int) -> int:
    """Seed of one synthetic channel: 0xAC7*1000 + 100*config + channel."""
    return SEED_BASE + 100 * int(config) + int(channel)


def rng_for(config: int, channel: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed_for(config, channel)))


# --------------------------------------------------------------------------
# Parameter grids (value_i = lo + i*step, i = 0..count-1)
# --------------------------------------------------------------------------
@dataclasses.dataclass(frozen=True)
class Axis:
    lo: float
    step: float
    count: int

    def values(self) -> np.ndarray:
        return self.lo + np.arange(self.count, dtype=np.float64) * self.step

    @staticmethod
    def linspace(lo: float, hi: float, count: int) -> "Axis":
        step = (hi - lo) / (count - 1) if count > 1 else 0.0
        return Axis(float(lo), float(step), int(count))


@dataclasses.dataclass(frozen=True)
class Grid:
    """A (tc, fc, logdt, c) grid on an n_samples window sampled at fs.

    Flat atom index: ((i_tc * N_fc + i_fc) * N_logdt + i_logdt) * N_c + i_c.
    """

    n_samples: int
    fs: float
    tc: Axis
    fc: Axis
    logdt: Axis
    c: Axis

    @property
    def n_atoms(self) -> int:
        return self.tc.count * self.fc.count * self.logdt.count * self.c.count

    def flat_of(self, itc: int, ifc: int, il: int, ic: int) -> int:
        return ((itc * self.fc.count + ifc) * self.logdt.count + il) * self.c.count + ic


# --------------------------------------------------------------------------
# Signal pieces
# --------------------------------------------------------------------------
def chirp_burst(n_samples: int, fs: float, tc: float, fc: float, logdt: float,
                c: float, norm: float) -> np.ndarray:
    """Gaussian-windowed linear-FM burst scaled to l2 norm ``norm``.

    The carrier is ``scipy.signal.chirp`` (linear method, f0 = fc at tau = 0,
    sweep f1 = fc + 2c at t1 = 1 s) and the window is the envelope that
    ``scipy.signal.gausspulse`` returns for a pulse whose envelope has
    standard deviation exp(logdt) seconds.
    """
    tau = (np.arange(n_samples, dtype=np.float64) - tc) / fs
    width = math.exp(logdt)
    env = _gauss_envelope(tau, width)
    carrier = sps.chirp(tau, f0=fc, t1=1.0, f1=fc + 2.0 * c, method="linear")
    burst = env * carrier
    e = float(np.sqrt(np.sum(burst * burst)))
    if e == 0.0:
        return burst
    return burst * (norm / e)


def _gauss_envelope(tau: np.ndarray, width: float) -> np.ndarray:
    # gausspulse's envelope is exp(-a t^2) with a = -(pi fc bw)^2 / (4 ln ref);
    # pick fc = 1, bwr = -6 dB and solve bw so that a = 1 / (2 width^2).
    bwr = -6.0
    ref = 10.0 ** (bwr / 20.0)
    a = 1.0 / (2.0 * width * width)
    bw = math.sqrt(-4.0 * math.log(ref) * a) / math.pi
    _, env = sps.gausspulse(tau, fc=1.0, bw=bw, bwr=bwr, retenv=True)
    return env


def white_noise(rng: np.random.Generator, n: int) -> np.ndarray:
    return rng.standard_normal(n)


def pink_noise(rng: np.random.Generator, n: int) -> np.ndarray:
    """1/f-power noise: white Gaussian shaped by f^-1/2 in the DFT domain."""
    w = rng.standard_normal(n)
    spec = np.fft.rfft(w)
    f = np.arange(spec.shape[0], dtype=np.float64)
    shape = np.zeros_like(f)
    shape[1:] = 1.0 / np.sqrt(f[1:])
    return np.fft.irfft(spec * shape, n=n)


def scale_to_snr(clean: np.ndarray, noise: np.ndarray, snr_db: float) -> np.ndarray:
    """Scale ``noise`` so that 10 log10(sum clean^2 / sum noise^2) == snr_db."""
    ps = float(np.sum(clean * clean))
    pn = float(np.sum(noise * noise))
    if pn == 0.0:
        return noise
    target = ps / (10.0 ** (snr_db / 10.0))
    return noise * math.sqrt(target / pn)


# --------------------------------------------------------------------------
# Workloads
# --------------------------------------------------------------------------
@dataclasses.dataclass
class Workload:
    name: str
    grid: Grid
    signals: np.ndarray            # [channels][n_samples] float64
    n_atoms: int                   # MP orders P
    truth: List[List[Tuple[float, float, float, float, float]]]  # per channel (tc, fc, logdt, c, coef)


def grid_small_test(n_samples: int = 32, fs: float = 32.0) -> Grid:
    """3 x 3 x 2 x 2 grid on a short window, for brute-force checks."""
    return Grid(n_samples, fs,
                Axis(4.0, float(n_samples) / 3.0, 3),
                Axis(2.0, 3.0, 3),
                Axis(-2.0, 0.5, 2),
                Axis(-4.0, 8.0, 2))


def grid_c1() -> Grid:
    """N=256, fs=128 Hz: tc 0..248 step 8 (32) x fc 1..31 Hz step 2 (16)
    x logdt {-3,-2.5,-2,-1.5} (4) x c -8..6 Hz/s step 2 (8) = 16,384 atoms."""
    return Grid(256, 128.0, Axis(0.0, 8.0, 32), Axis(1.0, 2.0, 16),
                Axis(-3.0, 0.5, 4), Axis(-8.0, 2.0, 8))


def grid_eeg(n_samples: int = 512, fs: float = 256.0) -> Grid:
    """EEG-like grid: 128 tc x 64 fc (0.5..32 Hz) x 8 logdt (-3..-0.5)
    x 32 c (-20..20 Hz/s) = 2,097,152 atoms."""
    return Grid(n_samples, fs, Axis(0.0, n_samples / 128.0, 128), Axis(0.5, 0.5, 64),
                Axis.linspace(-3.0, -0.5, 8), Axis.linspace(-20.0, 20.0, 32))


def grid_emg(n_samples: int, fs: float = 500.0) -> Grid:
    """EMG-like grid for one window length: 256 tc x 96 fc (20..200 Hz)
    x 8 logdt (-4..-1.5) x 24 c (-100..100 Hz/s) = 4,718,592 atoms."""
    return Grid(n_samples, fs, Axis(0.0, n_samples / 256.0, 256), Axis.linspace(20.0, 200.0, 96),
                Axis.linspace(-4.0, -1.5, 8), Axis.linspace(-100.0, 100.0, 24))


def grid_radar(n_samples: int = 1024, fs: float = 1000.0) -> Grid:
    """Radar-like grid: 256 tc x 128 fc (50..400 Hz) x 8 logdt (-3..-0.7)
    x 32 c (-300..300 Hz/s) = 8,388,608 atoms."""
    return Grid(n_samples, fs, Axis(0.0, n_samples / 256.0, 256), Axis.linspace(50.0, 400.0, 128),
                Axis.linspace(-3.0, -0.7, 8), Axis.linspace(-300.0, 300.0, 32))


def scaled_grid(grid: Grid, tc_count: int = None, fc_count: int = None,
                logdt_count: int = None, c_count: int = None) -> Grid:
    """Same ranges as ``grid`` with fewer points per axis (for fast tests)."""
    def shrink(ax: Axis, count):
        if count is None or count == ax.count:
            return ax
        hi = ax.lo + ax.step * (ax.count - 1)
        return Axis.linspace(ax.lo, hi, count)
    tc = grid.tc
    if tc_count is not None and tc_count != tc.count:
        tc = Axis(0.0, grid.n_samples / float(tc_count), tc_count)
    return Grid(grid.n_samples, grid.fs, tc, shrink(grid.fc, fc_count),
                shrink(grid.logdt, logdt_count), shrink(grid.c, c_count))


def _random_chirplets(rng, count, n_samples, fs, fc_rng, logdt_rng, c_rng, signed=True):
    truth = []
    for _ in range(count):
        tc = rng.uniform(0.0, float(n_samples))
        fc = rng.uniform(*fc_rng)
        ld = rng.uniform(*logdt_rng)
        c = rng.uniform(*c_rng)
        a = rng.uniform(0.5, 2.0)
        if signed and rng.random() < 0.5:
            a = -a
        truth.append((tc, fc, ld, c, a))
    return truth


def _assemble(truth, n_samples, fs):
    s = np.zeros(n_samples)
    for (tc, fc, ld, c, a) in truth:
        s += math.copysign(1.0, a) * chirp_burst(n_samples, fs, tc, fc, ld, c, abs(a))
    return s


def workload_c1(channels: int = 1) -> Workload:
    """3 on-grid chirplets (distinct grid points), coefficients U[0.5, 2]
    (positive), plus white Gaussian noise sigma = 0.05; 5 MP orders."""
    g = grid_c1()
    sigs, truths = [], []
    for ch in range(channels):
        rng = rng_for(1, ch)
        idx = rng.choice(g.n_atoms, size=3, replace=False)
        truth = []
        axes = (g.tc, g.fc, g.logdt, g.c)
        for i in idx:
            # the grid point of that position (c fastest, tc slowest)
            pos = np.unravel_index(int(i), tuple(a.count for a in axes))
            tc, fc, ld, c = (float(a.values()[k]) for a, k in zip(axes, pos))
            truth.append((tc, fc, ld, c, rng.uniform(0.5, 2.0)))
        s = _assemble(truth, g.n_samples, g.fs) + 0.05 * white_noise(rng, g.n_samples)
        sigs.append(s)
        truths.append(truth)
    return Workload("c1_plain_fp32_n256_k16384_p5", g, np.stack(sigs), 5, truths)


def eeg_like_signal(config: int, channel: int, n_samples: int = 512, fs: float = 256.0,
                    n_chirplets: int = 5, snr_db: float = 10.0):
    rng = rng_for(config, channel)
    truth = _random_chirplets(rng, n_chirplets, n_samples, fs, (1.0, 30.0), (-3.0, -0.5),
                              (-20.0, 20.0))
    clean = _assemble(truth, n_samples, fs)
    noise = scale_to_snr(clean, pink_noise(rng, n_samples), snr_db)
    return clean + noise, truth


def workload_c2() -> Workload:
    """EEG-like: N=512, fs=256 Hz, 5 random chirplets + pink noise at 10 dB,
    2,097,152-atom grid, 20 MP orders (1 channel)."""
    s, t = eeg_like_signal(2, 0)
    return Workload("c2_eeg_fp32_n512_k2097152_p20", grid_eeg(), s[None, :], 20, [t])


def workload_c3(channels: int = 64) -> Workload:
    """64 EEG-like channels with independent seeds, same grid as C2, 20 orders."""
    sigs, truths = [], []
    for ch in range(channels):
        s, t = eeg_like_signal(3, ch)
        sigs.append(s)
        truths.append(t)
    return Workload(f"c3_eeg_bf16_b{channels}_n512_k2097152_p20", grid_eeg(), np.stack(sigs), 20,
                    truths)


def emg_like_signal(channel: int, n_samples: int, fs: float = 500.0, snr_db: float = 5.0):
    rng = rng_for(4, channel)
    count = int(rng.integers(8, 16))
    truth = _random_chirplets(rng, count, n_samples, fs, (20.0, 200.0), (-4.0, -1.5),
                              (-100.0, 100.0))
    clean = _assemble(truth, n_samples, fs)
    noise = scale_to_snr(clean, white_noise(rng, n_samples), snr_db)
    return clean + noise, truth


def c4_lengths(count: int = 256) -> np.ndarray:
    rng = rng_for(4, 99)
    return rng.choice(np.array([256, 512, 1024, 2048]), size=count)


def workload_c4(count: int = 256) -> Tuple[List[np.ndarray], List[Grid], int]:
    """Uneven EMG-like batch: N uniform in {256,512,1024,2048}, fs=500 Hz,
    8-15 chirplets each, Gaussian noise at 5 dB; 30 MP orders."""
    lens = c4_lengths(count)
    sigs = []
    for ch, n in enumerate(lens):
        s, _ = emg_like_signal(ch, int(n))
        sigs.append(s)
    return sigs, [grid_emg(int(n)) for n in lens], 30


def radar_like_signal(channel: int, n_samples: int = 1024, fs: float = 1000.0,
                      snr_db: float = 15.0):
    rng = rng_for(5, channel)
    truth = _random_chirplets(rng, 4, n_samples, fs, (50.0, 400.0), (-3.0, -0.7),
                              (-300.0, 300.0))
    clean = _assemble(truth, n_samples, fs)
    noise = scale_to_snr(clean, white_noise(rng, n_samples), snr_db)
    return clean + noise, truth


def workload_c5(channels: int = 32) -> Workload:
    """Radar-like: 32 channels, N=1024, fs=1 kHz, 4 off-grid LFM chirplets each
    + white noise at 15 dB; 8,388,608-atom grid; 10 MP orders."""
    sigs, truths = [], []
    for ch in range(channels):
        s, t = radar_like_signal(ch)
        sigs.append(s)
        truths.append(t)
    return Workload(f"c5_radar_b{channels}_n1024_k8388608_p10", grid_radar(), np.stack(sigs), 10,
                    truths)


def random_signals(config: int, channels: int, n_samples: int, scale: float = 1.0) -> np.ndarray:
    """Plain white Gaussian signals (for edge-case and stress tests)."""
    if channels == 0:
        return np.zeros((0, n_samples))
    return np.stack([scale * white_noise(rng_for(config, ch), n_samples) for ch in range(channels)])
