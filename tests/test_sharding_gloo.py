"""Multi-rank path on CPU: world_size-2 gloo ranks shard the templates, each ranks its
own block, and the merged top-k equals the single-process top-k over all templates.
The per-rank rho comes from the oracle (no GPU here); what is under test is the host
logic of sharding and merging."""
import os
import socket

import numpy as np
import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

import oracle
import synth
from paper_1712_06515_gb300 import sharding


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _hits_from_rho(rho, freqs, k, offset):
    t, b, v = oracle.topk(rho, k)
    h = np.zeros(len(t), sharding.HIT_DTYPE)
    h["tmpl"], h["bin"], h["freq"], h["rho"] = t, b, freqs[b], v
    return sharding.globalize(h, offset)


def _rank_main(rank, world, port, k, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ds = synth.tiny(seed=41, n_templates=5, injection=synth.Injection(
            h0=0.4, f0=120.1, a_p=1.44, T_asc=synth.T_ASC_O1, P=synth.SCO_X1_P))
        plan = oracle.make_plan(ds.cfg)
        s, e = sharding.shard_range(len(ds.templates), rank, world)
        rho = oracle.rho(ds, templates=ds.templates[s:e])
        local = _hits_from_rho(rho.astype(np.float32), plan.freq, k, s)
        merged = sharding.merge_topk(local, k)
        out[rank] = merged.tolist()
    finally:
        dist.destroy_process_group()


def test_shard_ranges_partition():
    for n in (0, 1, 7, 8000):
        for w in (1, 2, 3, 8):
            got = [sharding.shard_range(n, r, w) for r in range(w)]
            assert got[0][0] == 0 and got[-1][1] == n
            assert all(a[1] == b[0] for a, b in zip(got, got[1:]))
            sizes = [b - a for a, b in got]
            assert max(sizes) - min(sizes) <= 1
    with pytest.raises(ValueError):
        sharding.shard_range(5, 2, 2)


def test_order_hits_ties():
    h = np.zeros(4, sharding.HIT_DTYPE)
    h["tmpl"], h["bin"], h["rho"] = [3, 1, 1, 0], [0, 5, 2, 9], [2.0, 2.0, 2.0, 1.0]
    o = sharding.order_hits(h, 3)
    assert list(zip(o["tmpl"], o["bin"])) == [(1, 2), (1, 5), (3, 0)]


def test_two_rank_gloo_merge_equals_single_process():
    k, world = 12, 2
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    port = _free_port()
    mp.start_processes(_rank_main, args=(world, port, k, out), nprocs=world, start_method="spawn")
    ds = synth.tiny(seed=41, n_templates=5, injection=synth.Injection(
        h0=0.4, f0=120.1, a_p=1.44, T_asc=synth.T_ASC_O1, P=synth.SCO_X1_P))
    plan = oracle.make_plan(ds.cfg)
    ref = _hits_from_rho(oracle.rho(ds).astype(np.float32), plan.freq, k, 0)
    for r in range(world):
        got = np.array([tuple(x) for x in out[r]], sharding.HIT_DTYPE)
        assert list(zip(got["tmpl"], got["bin"])) == list(zip(ref["tmpl"], ref["bin"]))
        np.testing.assert_array_equal(got["rho"], ref["rho"])
