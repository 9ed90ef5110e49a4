"""Multi-GPU sharding logic on CPU: two gloo ranks split one pencil's
eigenvectors by equal sum-c^2 work, each solves its share (the oracle stands in
for the GPU solve here), and the shares gathered on rank 0 are exactly the
full solve's columns."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import oracle
import pencilgen
from paper_2003_04776_gb300 import shard


def test_shards_cover_every_unit_once_and_balance():
    p = pencilgen.make_pencil(600, 31)
    for world in (1, 2, 3, 8):
        masks = shard.column_shards(p.block, world)
        starts, work = shard.unit_work(p.block)
        owners = np.array([sum(int(m[c] != 0) for m in masks) for c in starts])
        assert np.all(owners == 1)
        for m in masks:                     # nothing selected inside a pair's second row
            assert not np.any(m[p.block == 2])
        bal = shard.shard_balance(p.block, masks)
        assert abs(bal.sum() - work.sum()) < 1e-6 * work.sum()
        if world > 1:
            assert bal.max() - bal.min() <= work.max() + 1e-9


def test_block_pattern_matches_generator():
    p = pencilgen.make_pencil(300, 5)
    sub = np.diag(p.S, -1)
    assert np.array_equal(shard.block_pattern(sub, p.n), p.block)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, n, seed, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        p = pencilgen.make_pencil(n, seed)                     # replicated inputs
        masks = shard.column_shards(shard.block_pattern(np.diag(p.S, -1), n), world)
        st, V, sc, m = oracle.evc(p.S, p.T, select=masks[rank])
        assert st == 0
        cols = np.flatnonzero(masks[rank]).astype(np.int64)
        payload = {"cols": cols, "V": V, "scale": sc}
        gathered = [None] * world
        dist.all_gather_object(gathered, payload)             # one gather after the solve
        if rank == 0:
            out.put(gathered)
    finally:
        dist.destroy_process_group()


def test_two_rank_gloo_solve_equals_full_solve():
    n, seed, world = 180, 44, 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, world, port, n, seed, q)) for r in range(world)]
    for pr in procs:
        pr.start()
    gathered = q.get(timeout=120)
    for pr in procs:
        pr.join(timeout=120)
        assert pr.exitcode == 0
    p = pencilgen.make_pencil(n, seed)
    st, Vf, scf, mf = oracle.evc(p.S, p.T)
    parts = sorted(gathered, key=lambda d: d["cols"][0] if d["cols"].size else n)
    V = np.concatenate([d["V"] for d in parts], axis=1)
    sc = np.concatenate([d["scale"] for d in parts])
    assert V.shape == Vf.shape
    assert np.array_equal(V, Vf)
    assert np.array_equal(sc, scf)
