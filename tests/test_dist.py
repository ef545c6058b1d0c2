"""The multi-GPU exchange (global top-k merge) on CPU ranks over gloo."""
import os

import numpy as np
import pytest

from paper_2510_20891_gb300.dist import merge_topk


def test_merge_topk_matches_global_order():
    rng = np.random.default_rng(0)
    v = rng.integers(0, 20, 1000).astype(np.float32)
    v[[5, 500]] = np.nan
    parts = np.array_split(np.arange(1000), 3)
    k = 50
    loc_v, loc_i = [], []
    for p in parts:
        key = np.lexsort((p, -v[p].astype(np.float64), np.isnan(v[p])))[:k]
        loc_i.append(p[key])
        loc_v.append(v[p][key])
    gi, gv = merge_topk(loc_v, loc_i, k)
    ref = np.lexsort((np.arange(1000), -v.astype(np.float64), np.isnan(v)))[:k]
    assert np.array_equal(gi, ref)


def _worker(rank, world, port, q):
    import torch
    import torch.distributed as dist

    from paper_2510_20891_gb300.dist import allgather_topk

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    rng = np.random.default_rng(42)
    allv = rng.integers(0, 30, 2 * 400).astype(np.float32)
    mine = allv[rank * 400:(rank + 1) * 400]
    key = np.lexsort((np.arange(400), -mine.astype(np.float64)))[: (10 if rank == 0 else 7)]
    gi, gv = allgather_topk(torch.from_numpy(key.astype(np.int64)), torch.from_numpy(mine[key]), 12, rank * 400)
    q.put((rank, gi.tolist(), gv.tolist()))
    dist.destroy_process_group()


def test_allgather_topk_two_gloo_ranks():
    torch = pytest.importorskip("torch")
    import socket

    import torch.multiprocessing as tmp

    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    ctx = tmp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    rng = np.random.default_rng(42)
    allv = rng.integers(0, 30, 800).astype(np.float32)
    # each rank contributed only its local top list: the merge is the top-12 of their union
    cand = []
    for r, kk in ((0, 10), (1, 7)):
        mine = allv[r * 400:(r + 1) * 400]
        key = np.lexsort((np.arange(400), -mine.astype(np.float64)))[:kk]
        cand.extend((r * 400 + key).tolist())
    cand = np.array(cand)
    ref = cand[np.lexsort((cand, -allv[cand].astype(np.float64)))][:12]
    for _, gi, gv in res:
        assert gi == ref.tolist()
        assert np.allclose(gv, allv[ref])
