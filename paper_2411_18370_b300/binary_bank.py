"""Sizing a random binary-orbit bank (Sec. IV.A-IV.B, App. A) and sampling its mismatch.

Template count.  With the resolutions of App. A (delta f0 = 1/T, delta sky = (T v/c)^-2 f0^-2,
delta a_p = 1/(T f0 Omega), delta phi_b = 1/(T f0 a_p Omega), delta Omega =
1/(T T_obs f0 a_p Omega)) the density is rho = k f0^5 a_p^2 Omega^3, k = T^6 T_obs (v/c)^2,
and the number of templates in a region is the separable integral of Eq. (N_binary):
    N = k (f_hi^6 - f_lo^6)/6 * (Delta alpha Delta sin(delta)) * (a_hi^3 - a_lo^3)/3
          * (Omega_hi^4 - Omega_lo^4)/4 * Delta phi_b,
angles in radians.  A random bank with oversampling o holds o N templates.

Boxes (Sec. IV.B).  The uniform-coordinate box is cut into regular boxes: at least
`min_boxes` of them and none above `max_box` templates; the divisions go to the dimensions in
proportion to their extent in resolution cells.

Mismatch (Sec. IV.A).  For a signal on noise-free data (unit power on its track's bin in every
SFT, zero elsewhere) the statistic of a template counts the SFTs where its track meets the
signal's, so the best template of a bank around the signal has mismatch m = 1 - s_best / N_SFT
(Eq. (mismatch) with mu_G = 0 and no noise).  Sampling signals and banks of oversampling o gives
p(m | o).  The signal's bins follow Eq. (track) in FP64 (round to nearest).
"""
from __future__ import annotations

import math

import numpy as np

TWO_PI = 2.0 * math.pi


def density_constant(t_sft: float, t_obs: float, v_over_c: float) -> float:
    """k = T^6 T_obs (v/c)^2 of App. A."""
    return t_sft ** 6 * t_obs * v_over_c ** 2


def n_templates(lo, hi, t_sft: float, t_obs: float, v_over_c: float) -> float:
    """Eq. (N_binary) over the region lo..hi (order: f0 Hz, alpha turns, sin(delta), a_p
    light-seconds, Omega rad/s, phi_b turns)."""
    k = density_constant(t_sft, t_obs, v_over_c)
    f = (hi[0] ** 6 - lo[0] ** 6) / 6.0
    sky = (TWO_PI * (hi[1] - lo[1])) * (hi[2] - lo[2])
    a = (hi[3] ** 3 - lo[3] ** 3) / 3.0
    om = (hi[4] ** 4 - lo[4] ** 4) / 4.0
    ph = TWO_PI * (hi[5] - lo[5])
    return k * f * sky * a * om * ph


def cells_per_dim(lo, hi, t_sft: float, t_obs: float, v_over_c: float):
    """Resolution cells along each dimension: its extent over the App. A resolution evaluated
    at the region's centre (f0: T, each sky angle: T (v/c) f0, a_p: T f0 Omega, Omega:
    T T_obs f0 a_p Omega, phi_b: T f0 a_p Omega).  Their product approximates n_templates
    (exactly when the region is narrow); they set how the boxes are shared out."""
    f0 = 0.5 * (lo[0] + hi[0])
    ap = 0.5 * (lo[3] + hi[3])
    om = 0.5 * (lo[4] + hi[4])
    sky = t_sft * v_over_c * f0
    return np.array([(hi[0] - lo[0]) * t_sft,
                     TWO_PI * (hi[1] - lo[1]) * sky,
                     (hi[2] - lo[2]) * sky,
                     (hi[3] - lo[3]) * t_sft * f0 * om,
                     (hi[4] - lo[4]) * t_sft * t_obs * f0 * ap * om,
                     TWO_PI * (hi[5] - lo[5]) * t_sft * f0 * ap * om])


def plan(lo, hi, oversampling: float, t_sft: float, t_obs: float, v_over_c: float,
         min_boxes: int = 10_000, max_box: float = 1e8):
    """(n_div, n_per_box) of a random bank with o N templates in at least min_boxes boxes of at
    most max_box templates each."""
    total = oversampling * n_templates(lo, hi, t_sft, t_obs, v_over_c)
    n_boxes = max(min_boxes, math.ceil(total / max_box))
    cells = np.maximum(cells_per_dim(lo, hi, t_sft, t_obs, v_over_c), 1e-300)
    # n_div_d proportional to cells_d, scaled so that their product reaches n_boxes; a
    # dimension never gets more divisions than it has cells (nor fewer than one)
    n_div = np.ones(6, np.int64)
    free = np.ones(6, bool)
    for _ in range(6):
        if not free.any():
            break
        have = float(np.prod(n_div[~free]))
        need = n_boxes / have
        c = cells[free]
        scale = (need / np.prod(c)) ** (1.0 / free.sum())
        want = c * scale
        capped = want > cells[free]
        idx = np.nonzero(free)[0]
        if capped.any():
            for d in idx[capped]:
                n_div[d] = max(1, int(math.floor(cells[d])))
                free[d] = False
            continue
        for d, w in zip(idx, want):
            n_div[d] = max(1, int(round(w)))
        break
    while np.prod(n_div) < n_boxes:  # rounding: top up the dimension with most cells per box
        d = int(np.argmax(cells / n_div))
        n_div[d] += 1
    n_per_box = max(1, math.ceil(total / np.prod(n_div)))
    return tuple(int(x) for x in n_div), int(n_per_box)


def signal_bins(lam, t_mid, v, t0, t_sft, k_lo, n_sky_vec=None):
    """Eq. (track) bins (FP64, round half up) of a source lam = (f0, alpha turns, sin(delta),
    a_p, Omega, phi_b turns) in each SFT, as columns of a band starting at bin k_lo."""
    f0, al, sd, ap, om, ph = lam
    cd = math.sqrt(max(0.0, 1.0 - sd * sd))
    n = np.array([cd * math.cos(TWO_PI * al), cd * math.sin(TWO_PI * al), sd]) if n_sky_vec is None \
        else np.asarray(n_sky_vec, np.float64)
    t = np.asarray(t_mid, np.float64) - t0
    f = f0 * (1.0 + np.asarray(v, np.float64) @ n - ap * om * np.cos(om * t - TWO_PI * ph))
    return np.floor(f * t_sft + 0.5).astype(np.int64) - k_lo


def sample_mismatch(ctx, t_mid, v, n_sft, t0, t_sft, signals, half_cells, oversampling, seed,
                    wings=64, dtype="f32"):
    """Mismatch of the best template of a random bank around each signal (noise-free data).

    signals: [n, 6] source parameters; half_cells: the bank region around a signal spans
    +- half_cells resolution cells in each dimension (App. A resolutions at the signal);
    oversampling: templates = o x the region's Eq. (N_binary) count.  Returns m per signal."""
    from . import binary_eval, load_sfts, make_binary_bank

    N = int(np.sum(n_sft))
    vmax = float(np.max(np.linalg.norm(np.asarray(v), axis=1)))
    t_obs = float(np.max(t_mid) - np.min(t_mid)) + t_sft
    out = np.empty(len(signals))
    for i, lam in enumerate(np.asarray(signals, np.float64)):
        f0, al, sd, ap, om, ph = lam
        # resolutions at the signal (App. A), as half-widths of the region
        dfo = 1.0 / t_sft
        dsky = 1.0 / (t_sft * vmax * f0)           # per angle (sqrt of the solid-angle cell)
        cd = max(math.sqrt(max(0.0, 1 - sd * sd)), 1e-3)
        dal = dsky / cd / TWO_PI                   # right ascension, turns
        dsd = dsky * cd                            # sin(declination)
        dap = 1.0 / (t_sft * f0 * om)
        dph = 1.0 / (t_sft * f0 * ap * om) / TWO_PI
        dom = 1.0 / (t_sft * t_obs * f0 * ap * om)
        h = half_cells
        lo = [f0 - h * dfo, al - h * dal, max(-1.0, sd - h * dsd), ap - h * dap, om - h * dom, ph - h * dph]
        hi = [f0 + h * dfo, al + h * dal, min(1.0, sd + h * dsd), ap + h * dap, om + h * dom, ph + h * dph]
        # keep the angles inside one turn (the region is small)
        for d in (1, 5):
            if lo[d] < 0.0 or hi[d] > 1.0:
                shift = -lo[d] if lo[d] < 0 else 1.0 - hi[d]
                lo[d] += shift
                hi[d] += shift
        n_t = max(1, int(round(oversampling * n_templates(lo, hi, t_sft, t_obs, vmax))))
        k_sig = int(math.floor(f0 * t_sft))
        k_lo = k_sig - wings
        W = 2 * wings + 1
        P = np.zeros((N, W), np.float32)
        b = signal_bins(lam, t_mid, v, t0, t_sft, k_lo)
        if np.any((b < 0) | (b >= W)):
            raise ValueError("signal track leaves the generated window; widen wings")
        P[np.arange(N), b] = 1.0
        band = load_sfts(ctx, P, t_mid, v, n_sft, k_lo, t_sft, t0, dtype=dtype)
        bank = make_binary_bank(ctx, band, lo, hi, (1, 1, 1, 1, 1, 1), n_t, seed + i)
        s = np.empty(n_t, np.float32)
        binary_eval(ctx, band, bank, 0, n_t, s)
        out[i] = 1.0 - float(np.max(s)) / N
        bank.close()
        band.close()
    return out
