"""Seeded synthetic inputs shared by the CUDA path's tests/bench and the CPU oracle.

This module draws data only: SFT timelines, detector velocities, PSD levels, complex
Gaussian SFT noise, Fibonacci sky grids and f1 lists.  It holds none of the method's
arithmetic (no track bins, no statistic, no candidate selection); everything here is an
*input* that both sides receive verbatim.

Conventions (readings of the paper where it is silent; all in the repository's design
notes):

* Noise (paper Sec. II.B.1, "Distribution under the noise hypothesis"): each SFT bin is a
  complex Gaussian whose real and imaginary parts have variance S_n, so the normalised
  power P = |x|^2 / S_n is chi-squared with two degrees of freedom (mean 2, variance 4).
* Timeline: SFT mid-times t_alpha = start + T_SFT/2; the reference time t0 is the start of
  the observation (first slot), where f0 is defined (paper Sec. II.A, Eq. track).
* Velocity: circular 1 AU orbit (29.8 km/s, 1 yr period, ecliptic plane rotated to the
  equatorial frame by the obliquity) plus the sidereal rotation of a site at 30 deg
  latitude (465 m/s * cos 30 deg).  Phases are zero at t = 0.
* Sky: Fibonacci sphere z_i = 1 - (2i+1)/N, phi_i = i * pi * (3 - sqrt 5).
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

MASTER_SEED = 20241127
C_LIGHT = 299_792_458.0
YEAR_S = 365.25 * 86400.0
SIDEREAL_DAY_S = 86164.0905
V_ORBIT = 29.8e3
V_ROT = 465.0 * math.cos(math.radians(30.0))
OBLIQUITY = math.radians(23.4393)

_MASK64 = (1 << 64) - 1


def splitmix64(x: int) -> int:
    """One step of the SplitMix64 mixer (Steele, Lea & Flood, OOPSLA 2014)."""
    x = (x + 0x9E3779B97F4A7C15) & _MASK64
    z = x
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _MASK64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _MASK64
    return z ^ (z >> 31)


def derive_seed(config_id: int, stream_id: int, master: int = MASTER_SEED) -> int:
    """Per-use seed = splitmix64 chain over (master, config, stream)."""
    s = splitmix64(master & _MASK64)
    s = splitmix64(s ^ (config_id & _MASK64))
    s = splitmix64(s ^ (stream_id & _MASK64))
    return s


def rng(config_id: int, stream_id: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(derive_seed(config_id, stream_id)))


# ----------------------------------------------------------------------------- sky / f1


def fibonacci_sky(n: int) -> np.ndarray:
    """Unit vectors of an n-point Fibonacci sphere, shape [n, 3], FP64."""
    i = np.arange(n, dtype=np.float64)
    z = 1.0 - (2.0 * i + 1.0) / n
    phi = i * (math.pi * (3.0 - math.sqrt(5.0)))
    r = np.sqrt(np.maximum(0.0, 1.0 - z * z))
    return np.stack([r * np.cos(phi), r * np.sin(phi), z], axis=1)


def f1_grid(n: int, lo: float, hi: float) -> np.ndarray:
    if n == 1:
        return np.array([hi], dtype=np.float64)
    return np.linspace(lo, hi, n, dtype=np.float64)


# ----------------------------------------------------------------------------- detectors


@dataclasses.dataclass(frozen=True)
class Site:
    """Synthetic interferometer: latitude/longitude (deg) and arm azimuths (deg, from north)."""

    lat_deg: float
    lon_deg: float
    arm_az_deg: tuple


SITES = (
    Site(30.0, 0.0, (0.0, 90.0)),
    Site(30.0, -90.0, (45.0, 135.0)),
)


def detector_velocity(t: np.ndarray, det: int) -> np.ndarray:
    """v/c in the equatorial frame at times t (s), shape [len(t), 3], FP64."""
    t = np.asarray(t, dtype=np.float64)
    ph = 2.0 * math.pi * t / YEAR_S
    # ecliptic-plane circular orbit, rotated about x by the obliquity
    vx = -np.sin(ph)
    vy = np.cos(ph)
    orb = V_ORBIT * np.stack(
        [vx, vy * math.cos(OBLIQUITY), vy * math.sin(OBLIQUITY)], axis=1
    )
    th = 2.0 * math.pi * t / SIDEREAL_DAY_S + math.radians(SITES[det].lon_deg)
    rot = V_ROT * np.stack([-np.sin(th), np.cos(th), np.zeros_like(th)], axis=1)
    return (orb + rot) / C_LIGHT


def detector_tensor(t: np.ndarray, det: int) -> np.ndarray:
    """Detector tensor D = (u u^T - v v^T)/2 of site `det` at times t, in the equatorial
    frame, as [len(t), 6] = (Dxx, Dxy, Dxz, Dyy, Dyz, Dzz).  u, v are the arm directions
    (azimuths from north towards east in the local horizontal plane); the site turns with
    the sidereal angle 2 pi t / T_sid + longitude (the same angle as detector_velocity)."""
    site = SITES[det]
    t = np.asarray(t, dtype=np.float64)
    th = 2.0 * math.pi * t / SIDEREAL_DAY_S + math.radians(site.lon_deg)
    lat = math.radians(site.lat_deg)
    east = np.stack([-np.sin(th), np.cos(th), np.zeros_like(th)], axis=1)
    north = np.stack([-math.sin(lat) * np.cos(th), -math.sin(lat) * np.sin(th),
                      np.full_like(th, math.cos(lat))], axis=1)
    arms = []
    for az in site.arm_az_deg:
        A = math.radians(az)
        arms.append(north * math.cos(A) + east * math.sin(A))
    u, v = arms
    D = 0.5 * (u[:, :, None] * u[:, None, :] - v[:, :, None] * v[:, None, :])
    return np.stack([D[:, 0, 0], D[:, 0, 1], D[:, 0, 2], D[:, 1, 1], D[:, 1, 2], D[:, 2, 2]], axis=1)


def max_v_over_c() -> float:
    return (V_ORBIT + V_ROT) / C_LIGHT


# ----------------------------------------------------------------------------- SFT sets


@dataclasses.dataclass
class SFTSet:
    """A narrow band of SFT power rows for one or more detectors.

    power  : [N_SFT, W] FP64 normalised power (rows ordered detector-major, time within).
    t_mid  : [N_SFT] SFT mid-times (s).
    v      : [N_SFT, 3] detector velocity / c.
    s_n    : [N_SFT] PSD level per SFT (arbitrary units).
    n_sft  : SFT count per detector.
    k_lo   : global bin index of column 0 (bin = f * T_SFT).
    """

    power: np.ndarray
    t_mid: np.ndarray
    v: np.ndarray
    s_n: np.ndarray
    n_sft: list
    k_lo: int
    t_sft: float
    t0: float
    det: np.ndarray = None
    x: np.ndarray = None  # complex SFT bins (scaled so |x|^2/S_n = power), optional

    @property
    def n_bins(self) -> int:
        return int(self.power.shape[1])

    @property
    def n_total(self) -> int:
        return int(self.power.shape[0])


def timeline(n_det: int, n_slots: int, t_sft: float, duty: float, gen: np.random.Generator):
    """Per detector, the kept slot starts (seeded Bernoulli(duty) per slot)."""
    starts = []
    for _ in range(n_det):
        keep = gen.random(n_slots) < duty if duty < 1.0 else np.ones(n_slots, bool)
        starts.append(np.nonzero(keep)[0].astype(np.float64) * t_sft)
    return starts


def complex_noise(n_rows: int, n_bins: int, s_n: np.ndarray, gen: np.random.Generator):
    """Complex SFT bins with Re, Im ~ N(0, sqrt(S_n)) per row; returns x (complex128)."""
    sd = np.sqrt(np.asarray(s_n, dtype=np.float64))[:, None]
    re = gen.standard_normal((n_rows, n_bins)) * sd
    im = gen.standard_normal((n_rows, n_bins)) * sd
    return re + 1j * im


def power_of(x: np.ndarray, s_n: np.ndarray) -> np.ndarray:
    """Normalised power |x|^2 / S_n, FP64."""
    return (x.real * x.real + x.imag * x.imag) / np.asarray(s_n, np.float64)[:, None]


def wings_for(f_hi_hz: float, f1_min: float, t_obs: float, t_sft: float):
    """Conservative (lo, hi) wing widths in bins for a band whose top is f_hi_hz.

    Sizing only: Doppler |v/c| <= max_v_over_c() and the spindown drift over t_obs.
    """
    dop = math.ceil(f_hi_hz * max_v_over_c() * t_sft)
    spin = math.ceil(abs(f1_min) * t_obs * t_sft)
    return dop + spin + 1, dop + 1


def make_sfts(
    config_id: int,
    n_det: int,
    n_slots: int,
    t_sft: float,
    duty: float,
    k_band: int,
    n_band_bins: int,
    wing_lo: int,
    wing_hi: int,
    psd_range=(1.0, 1.0),
    keep_complex: bool = False,
    stream_base: int = 0,
    slot_starts=None,
) -> SFTSet:
    """Seeded SFT set: timeline, velocities, PSD levels and chi^2_2 power rows."""
    g_time = rng(config_id, stream_base + 1)
    if slot_starts is None:
        slot_starts = timeline(n_det, n_slots, t_sft, duty, g_time)
    g_psd = rng(config_id, stream_base + 2)
    g_noise = rng(config_id, stream_base + 3)
    t_mid, v, det = [], [], []
    for X, st in enumerate(slot_starts):
        tm = st + 0.5 * t_sft
        t_mid.append(tm)
        v.append(detector_velocity(tm, X))
        det.append(np.full(len(tm), X, np.int32))
    t_mid = np.concatenate(t_mid)
    v = np.concatenate(v)
    det = np.concatenate(det)
    n = len(t_mid)
    lo, hi = psd_range
    s_n = lo + (hi - lo) * g_psd.random(n) if hi > lo else np.full(n, lo)
    W = n_band_bins + wing_lo + wing_hi
    x = complex_noise(n, W, s_n, g_noise)
    return SFTSet(
        power=power_of(x, s_n),
        t_mid=t_mid,
        v=v,
        s_n=s_n,
        n_sft=[len(s) for s in slot_starts],
        k_lo=k_band - wing_lo,
        t_sft=t_sft,
        t0=0.0,
        det=det,
        x=x if keep_complex else None,
    )


# ----------------------------------------------------------------------------- banks


@dataclasses.dataclass
class Bank:
    """Regular bank: f0_j = (k0 + j)/T_SFT for j < n_f0, a list of f1, a list of sky vectors.

    Template index t = (i_sky * n_f1 + i_f1) * n_f0 + j  (f0 fastest).
    """

    k0: int
    n_f0: int
    f1: np.ndarray
    sky: np.ndarray
    subband_bins: int

    @property
    def n_f1(self) -> int:
        return len(self.f1)

    @property
    def n_sky(self) -> int:
        return len(self.sky)

    @property
    def n_templates(self) -> int:
        return self.n_sky * self.n_f1 * self.n_f0

    @property
    def n_subbands(self) -> int:
        return (self.n_f0 + self.subband_bins - 1) // self.subband_bins

    def split(self, t):
        t = np.asarray(t, np.int64)
        j = t % self.n_f0
        r = t // self.n_f0
        return r // self.n_f1, r % self.n_f1, j


BINARY_DIMS = ("f0", "alpha", "sind", "ap", "omega", "phib")


@dataclasses.dataclass
class BinaryBank:
    """Random bank for the binary-orbit track, cut into regular boxes in the uniform
    coordinates.  lo / hi per dimension of BINARY_DIMS: f0 (Hz), right ascension alpha (turns,
    within [0, 1]), sin(declination), projected semi-major axis a_p (light-seconds), orbital
    angular frequency Omega (rad/s), orbital phase phi_b (turns, within [0, 1]).  n_div boxes
    per dimension (f0 slowest, phi_b fastest), n_per_box templates each, drawn from `seed`.
    Template i lies in box i // n_per_box."""

    lo: tuple
    hi: tuple
    n_div: tuple
    n_per_box: int
    seed: int

    @property
    def n_boxes(self) -> int:
        return int(np.prod(self.n_div))

    @property
    def n_templates(self) -> int:
        return self.n_boxes * self.n_per_box


# ----------------------------------------------------------------------------- configs

T_SFT = 1800.0


def tiny_workload(wings: str = "literal") -> tuple:
    """Plain, tiny: 1 detector, 48 SFTs 10 days, band 100.00-100.05 Hz, 4320 templates.

    wings="literal": 10 bins each side as stated; tracks near the band edges leave the
    window.  wings="auto": enough bins that every track stays inside.
    Returns (SFTSet with complex bins, Bank, injection dict).
    """
    k_band = int(round(100.0 * T_SFT))
    n_bins = 90
    if wings == "literal":
        wl = wh = 10
    else:
        wl, wh = wings_for(100.05, -1e-10, 10 * 86400.0, T_SFT)
        wl = wh = max(wl, wh)
    starts = [np.arange(48, dtype=np.float64) * (10 * 86400.0 / 48)]
    sfts = make_sfts(0, 1, 48, T_SFT, 1.0, k_band, n_bins, wl, wh, keep_complex=True,
                     slot_starts=starts)
    bank = Bank(k0=k_band, n_f0=n_bins, f1=np.array([-1e-10, -5e-11, 0.0]),
                sky=fibonacci_sky(16), subband_bins=18)
    inj = dict(j=45, i_f1=1, i_sky=7, amp=2.0, phase_seed=derive_seed(0, 9))
    return sfts, bank, inj


def search_workload(n_sky: int = 10_000, duty: float = 0.7) -> tuple:
    """Plain, search-shaped: 2 detectors, 1 yr, 70% duty, band 200.0-200.1 Hz."""
    k_band = int(round(200.0 * T_SFT))
    n_bins = 180
    n_slots = int(round(YEAR_S / T_SFT))
    wl, wh = wings_for(200.1, -1e-9, YEAR_S, T_SFT)
    sfts = make_sfts(1, 2, n_slots, T_SFT, duty, k_band, n_bins, wl, wh, psd_range=(0.8, 1.2))
    bank = Bank(k0=k_band, n_f0=n_bins, f1=f1_grid(20, -1e-9, 0.0), sky=fibonacci_sky(n_sky),
                subband_bins=18)
    return sfts, bank


def batch_bands(n_bands: int = 64, sky_scale: float = 1.0, seed_stream: int = 0):
    """The 64-band batching workload: widths log-uniform 0.05-0.5 Hz, starts U[50, 500] Hz,
    N_sky = round(1e3 (f_start/50)^2 * sky_scale) clamped to [1e3, 1e5] * sky_scale, 10 f1."""
    g = rng(3, 100 + seed_stream)
    widths = np.exp(g.uniform(math.log(0.05), math.log(0.5), n_bands))
    starts = g.uniform(50.0, 500.0, n_bands)
    out = []
    for b in range(n_bands):
        n_bins = int(round(widths[b] * T_SFT))
        k_band = int(round(starts[b] * T_SFT))
        n_sky = int(round(min(max(1e3 * (starts[b] / 50.0) ** 2, 1e3), 1e5) * sky_scale))
        out.append(dict(k_band=k_band, n_bins=n_bins, n_sky=max(n_sky, 1),
                        f_hi=(k_band + n_bins) / T_SFT))
    return out


def batch_workload(n_bands: int = 64, sky_scale: float = 1.0, n_slots: int = None, duty: float = 0.7,
            max_sky: int = None, bands=None):
    """The batching workload: bands from batch_bands() sharing one 2-detector timeline of
    1800 s SFTs (70% duty), each with its own noise, wings sized for its top frequency,
    10 f1 values in [-1e-9, 0] and N_sky Fibonacci sky points (scaled by sky_scale, capped
    by max_sky).  Returns a list of (SFTSet, Bank)."""
    if n_slots is None:
        n_slots = int(round(YEAR_S / T_SFT))
    t_obs = n_slots * T_SFT
    starts = timeline(2, n_slots, T_SFT, duty, rng(3, 1))
    specs = batch_bands(n_bands, sky_scale)
    out = []
    for b, spec in enumerate(specs if bands is None else [specs[i] for i in bands]):
        wl, wh = wings_for(spec["f_hi"], -1e-9, t_obs, T_SFT)
        sfts = make_sfts(3, 2, n_slots, T_SFT, duty, spec["k_band"], spec["n_bins"], wl, wh,
                         psd_range=(0.8, 1.2), stream_base=10 * (b + 1), slot_starts=starts)
        n_sky = spec["n_sky"] if max_sky is None else min(spec["n_sky"], max_sky)
        bank = Bank(k0=spec["k_band"], n_f0=spec["n_bins"], f1=f1_grid(10, -1e-9, 0.0),
                    sky=fibonacci_sky(max(n_sky, 1)), subband_bins=18)
        out.append((sfts, bank))
    return out


def binary_workload(days: float = 183.0, duty: float = 0.7, n_div=(2, 2, 2, 1, 1, 4),
                    n_per_box: int = 32768, seed: int = 2024):
    """Binary-orbit search slice shaped like the paper's all-sky binary search (Sec. VI.A):
    2 detectors, `days` of 1024 s SFTs at `duty`, f0 in 100-100.125 Hz (0.125 Hz, the band of
    the mismatch study in Sec. IV.A), the whole sky, a_p 5-15 light-seconds, orbital period
    7-15 days, phi_b over the full orbit; a random bank of n_per_box templates in each of
    prod(n_div) hyperboxes.  Wings cover the Doppler and orbit excursions.  Returns
    (SFTSet, BinaryBank)."""
    t_sft = 1024.0
    n_slots = int(round(days * 86400.0 / t_sft))
    f_lo, f_hi = 100.0, 100.125
    ap_hi, om_hi = 15.0, 2 * math.pi / (7 * 86400.0)
    orbit = math.ceil(f_hi * t_sft * ap_hi * om_hi * (1 + max_v_over_c()))
    wl, wh = wings_for(f_hi, 0.0, n_slots * t_sft, t_sft)
    k_band = int(round(f_lo * t_sft))
    n_bins = int(round((f_hi - f_lo) * t_sft))
    sfts = make_sfts(5, 2, n_slots, t_sft, duty, k_band, n_bins, wl + orbit + 1, wh + orbit + 1,
                     psd_range=(0.8, 1.2))
    bank = BinaryBank(lo=(f_lo, 0.0, -1.0, 5.0, 2 * math.pi / (15 * 86400.0), 0.0),
                      hi=(f_hi, 1.0, 1.0, ap_hi, om_hi, 1.0), n_div=tuple(n_div),
                      n_per_box=int(n_per_box), seed=int(seed))
    return sfts, bank


def psd_level(f_hz: float) -> float:
    """Smooth synthetic PSD shape used for the surrogate workload (arbitrary units):
    a steep low-frequency wall, a flat bucket and a rising high-frequency tail."""
    return 1.0 + (f_hz / 120.0) ** -4 + (f_hz / 600.0) ** 2


def surrogate_bands(n_bands: int = 64, sky_scale: float = 1.0, n_slots: int = None, seed_stream=0):
    """The surrogate workload's bands: the batching workload's bands, each with its own duty
    cycle U[0.5, 0.9] (SFTs dropped independently) and PSD level psd_level(f_mid) times a
    per-SFT U[0.8, 1.2] factor.  Returns dicts with the band spec, timeline, velocities,
    detector tensors and PSD levels (no power: injection runs synthesise their own data)."""
    if n_slots is None:
        n_slots = int(round(YEAR_S / T_SFT))
    g = rng(4, 200 + seed_stream)
    specs = batch_bands(n_bands, sky_scale)
    out = []
    for b, sp in enumerate(specs):
        duty = float(g.uniform(0.5, 0.9))
        starts = timeline(2, n_slots, T_SFT, duty, rng(4, 1000 + b))
        t_mid = np.concatenate([st + 0.5 * T_SFT for st in starts])
        v = np.concatenate([detector_velocity(st + 0.5 * T_SFT, X) for X, st in enumerate(starts)])
        D = np.concatenate([detector_tensor(st + 0.5 * T_SFT, X) for X, st in enumerate(starts)])
        f_mid = (sp["k_band"] + 0.5 * sp["n_bins"]) / T_SFT
        s_ref = psd_level(f_mid)
        s_n = s_ref * rng(4, 2000 + b).uniform(0.8, 1.2, len(t_mid))
        out.append(dict(spec=sp, duty=duty, t_mid=t_mid, v=v, D=D, s_n=s_n,
                        s_ref=float(np.mean(s_n)), n_sft=[len(st) for st in starts]))
    return out
