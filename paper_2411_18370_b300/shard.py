"""Sharding a search over several GPUs, one process per GPU (host logic).

Templates are independent, so a search splits without any exchange on the data path:
  - by band: each rank searches whole bands (balanced by their evaluation counts);
  - by sky tile within a band: each rank searches a contiguous range of the bank's sky points.
With sky as the slowest template index (t = (i_sky n_f1 + i_f1) n_f0 + j), a rank whose bank
holds sky points [lo, hi) finds global indices by adding lo n_f1 n_f0.  The only exchange is
the per-sub-band candidate lists (k entries of 16 bytes each), merged on the host by the
same (s descending, template index ascending) key as on the device.
"""
from __future__ import annotations

import numpy as np


def shard_bands(costs, world: int, rank: int):
    """Band indices of `rank`: longest-processing-time-first assignment of the bands' costs
    (e.g. evaluations) to `world` ranks, ties by rank.  Deterministic."""
    costs = np.asarray(costs, np.float64)
    load = np.zeros(world)
    owner = np.empty(len(costs), np.int64)
    for b in np.lexsort((np.arange(len(costs)), -costs)):
        r = int(np.argmin(load))
        owner[b] = r
        load[r] += costs[b]
    return np.nonzero(owner == rank)[0]


def shard_sky(n_sky: int, world: int, rank: int):
    """[lo, hi) of the sky points searched by `rank` (contiguous, sizes differ by <= 1)."""
    base, extra = divmod(n_sky, world)
    lo = rank * base + min(rank, extra)
    return lo, lo + base + (1 if rank < extra else 0)


def globalise(cand, sky_lo: int, n_f1: int, n_f0: int):
    """Candidate records of a sky-tile bank with global template indices (empty slots stay)."""
    out = np.array(cand, copy=True)
    ok = out["template_idx"] >= 0
    out["template_idx"][ok] += sky_lo * n_f1 * n_f0
    return out


def merge(parts, k: int):
    """Merge per-sub-band candidate lists [n_sub, k] of several ranks into one [n_sub, k] by
    (s descending, template index ascending); empty slots (index -1) last."""
    parts = [np.asarray(p) for p in parts]
    allc = np.concatenate(parts, axis=1)
    out = np.empty((allc.shape[0], k), dtype=allc.dtype)
    for b in range(allc.shape[0]):
        row = allc[b]
        valid = row["template_idx"] >= 0
        key_s = np.where(valid, -row["s"].astype(np.float64), np.inf)
        key_t = np.where(valid, row["template_idx"], np.iinfo(np.int64).max)
        order = np.lexsort((key_t, key_s))[:k]
        out[b] = row[order]
        out[b]["template_idx"][~valid[order]] = -1
    return out
