"""The N > 1 path on CPU: two ranks over gloo split a band's sky points, each selects its
sub-band candidates (the oracle stands in for the GPU on this CPU-only test), the lists are
exchanged with all_gather and merged on the host; the result equals the selection over the
whole bank.  Band sharding is checked for balance and coverage."""
import os
import socket

import numpy as np
import pytest

WORLD = 2
K = 4


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _candidates(idx, val):
    import paper_2411_18370_b300 as ft

    out = np.zeros(idx.shape, dtype=ft.CANDIDATE_DTYPE)
    out["template_idx"] = idx
    out["s"] = np.where(idx >= 0, val, -np.inf).astype(np.float32)
    return out


def _worker(rank, port, result_dir):
    import torch.distributed as dist

    import ftsynth
    import oracle
    from paper_2411_18370_b300 import shard

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=WORLD)
    sfts, bank, _ = ftsynth.tiny_workload("auto")
    lo, hi = shard.shard_sky(bank.n_sky, WORLD, rank)
    per_sky = bank.n_f1 * bank.n_f0
    t = np.arange(lo * per_sky, hi * per_sky)
    s, _ = oracle.statistic(sfts, bank, t)
    s32 = s.astype(np.float32).astype(np.float64)
    # the rank's own list, as a bank of sky points [lo, hi) reports it: local indices
    idx, val = oracle.topk_per_subband(s32, bank, K, t)
    local = _candidates(np.where(idx >= 0, idx - lo * per_sky, -1), val)
    mine = shard.globalise(local, lo, bank.n_f1, bank.n_f0)
    parts = [None] * WORLD
    dist.all_gather_object(parts, mine)
    merged = shard.merge(parts, K)
    if rank == 0:
        s_all, _ = oracle.statistic(sfts, bank)
        i_all, v_all = oracle.topk_per_subband(s_all.astype(np.float32).astype(np.float64), bank, K)
        np.save(os.path.join(result_dir, "merged.npy"), merged["template_idx"])
        np.save(os.path.join(result_dir, "full.npy"), i_all)
        assert np.array_equal(merged["template_idx"], i_all)
        ok = i_all >= 0
        assert np.array_equal(merged["s"][ok].astype(np.float64), v_all[ok])
    dist.barrier()
    dist.destroy_process_group()


def test_sky_sharded_search_merges_to_the_full_selection(tmp_path):
    import torch.multiprocessing as mp

    mp.spawn(_worker, args=(_free_port(), str(tmp_path)), nprocs=WORLD, join=True)
    assert np.array_equal(np.load(tmp_path / "merged.npy"), np.load(tmp_path / "full.npy"))


def test_shard_helpers():
    from paper_2411_18370_b300 import shard

    # sky ranges tile [0, n) with sizes differing by at most one
    for n, w in [(10, 3), (1, 2), (16, 4), (7, 8)]:
        r = [shard.shard_sky(n, w, i) for i in range(w)]
        assert r[0][0] == 0 and r[-1][1] == n
        assert all(a[1] == b[0] for a, b in zip(r, r[1:]))
        sizes = [b - a for a, b in r]
        assert max(sizes) - min(sizes) <= 1
    # bands: every band owned once; the heaviest load within the largest band of the ideal
    costs = np.random.default_rng(1).uniform(1, 10, 64)
    owners = [shard.shard_bands(costs, 4, r) for r in range(4)]
    allb = np.sort(np.concatenate(owners))
    assert np.array_equal(allb, np.arange(64))
    loads = [costs[o].sum() for o in owners]
    assert max(loads) - costs.sum() / 4 <= costs.max()
    # merge: ties by the smaller index, empty slots last
    import paper_2411_18370_b300 as ft

    a = np.zeros((1, 2), ft.CANDIDATE_DTYPE)
    a["template_idx"] = [[5, -1]]
    a["s"] = [[3.0, -np.inf]]
    b = np.zeros((1, 2), ft.CANDIDATE_DTYPE)
    b["template_idx"] = [[2, 9]]
    b["s"] = [[3.0, 4.0]]
    m = shard.merge([a, b], 3)
    assert m["template_idx"].tolist() == [[9, 2, 5]]
    m = shard.merge([a, a], 3)
    assert m["template_idx"].tolist() == [[5, 5, -1]]
