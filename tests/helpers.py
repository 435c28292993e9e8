"""Glue for the tests: hand ftsynth inputs to the C ABI (via the binding)."""
import numpy as np

import paper_2411_18370_b300 as ft


def band_from(ctx, sfts, dtype="f32", w=None, power_f32=False, on_device=False):
    P = sfts.power.astype(np.float32) if power_f32 else np.ascontiguousarray(sfts.power)
    if on_device:
        import torch

        P = torch.from_numpy(np.ascontiguousarray(P)).cuda()
    return ft.load_sfts(ctx, P, sfts.t_mid, sfts.v, sfts.n_sft, sfts.k_lo, sfts.t_sft, sfts.t0,
                        dtype=dtype, w=w, s_n=sfts.s_n)


def bank_from(ctx, band, bank):
    return ft.make_bank(ctx, band, bank.k0, bank.n_f0, bank.f1, bank.sky, bank.subband_bins)


def eval_host(ctx, band, bank, n_templates, with_z=True, with_oob=True):
    s = np.empty(n_templates, np.float32)
    z = np.empty(n_templates, np.float32) if with_z else None
    o = np.empty(n_templates, np.int32) if with_oob else None
    ft.eval_statistic(ctx, band, bank, s, z, o)
    return s, z, o


def topk_host(ctx, band, bank, n_sub, k):
    out = np.zeros((n_sub, k), dtype=ft.CANDIDATE_DTYPE)
    ft.topk_per_band(ctx, band, bank, k, out)
    return out["template_idx"].copy(), out["s"].copy(), out["z"].copy()


def inject(sfts, bins_row, amp, phase_seed):
    """Complex-domain injection: x[alpha, k_alpha] += amp e^{i phi_alpha} (phases seeded)."""
    g = np.random.default_rng(phase_seed)
    phi = g.uniform(0, 2 * np.pi, sfts.n_total)
    x = sfts.x.copy()
    for a, k in enumerate(bins_row):
        if 0 <= k < x.shape[1]:
            x[a, k] += amp * np.exp(1j * phi[a])
    return x
