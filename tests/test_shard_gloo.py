"""Multi-rank path on CPU (gloo, world size 2): events split into contiguous
shards, each rank evaluates its shard (here with the FP64 oracle: no GPU in
this test), and merge_results reduces cut flows and histograms exactly and
concatenates the per-event outputs.  The merged result must equal the
one-rank result over all events, for any split."""
import os
import socket

import numpy as np
import pytest

import synth
from synth import analyses


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, n, q):
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    import torch.distributed as dist
    import oracle
    import synth as sy
    from synth import analyses as an_mod
    from paper_2211_14346_gb300.shard import shard_range, merge_results
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        cols = sy.gen_semilep(n, 21)
        an = an_mod.config2()
        lo, hi = shard_range(n, rank, world)
        r = oracle.run(an, cols.slice(lo, hi), seed=42, V=4, first_event_id=lo)
        m = merge_results(r)
        if rank == 0:
            q.put({k: (v.tolist() if isinstance(v, np.ndarray) else v) for k, v in m.items()})
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("n", [301, 2])
def test_two_rank_merge_equals_one_rank(n, orc):
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_worker, args=(r, 2, port, n, q)) for r in range(2)]
    for p in ps:
        p.start()
    m = q.get(timeout=120)
    for p in ps:
        p.join(timeout=60)
        assert p.exitcode == 0
    cols = synth.gen_semilep(n, 21)
    o = orc.run(analyses.config2(), cols, seed=42, V=4)
    assert np.array_equal(np.asarray(m["cutflow"], np.uint64), o["cutflow"])
    assert np.array_equal(np.asarray(m["hist"], np.uint64), o["hist"])
    assert np.array_equal(np.asarray(m["mask"], np.uint8), o["mask"])
    assert np.array_equal(np.asarray(m["n_surv"], np.uint16), o["n_surv"])
    assert np.allclose(np.asarray(m["reco"], np.float32), o["reco"].astype(np.float32), rtol=0, atol=0)


def test_shard_ranges_cover_exactly():
    from paper_2211_14346_gb300.shard import shard_range
    for n in (0, 1, 7, 1000, 10 ** 7 + 3):
        for w in (1, 2, 3, 8):
            rs = [shard_range(n, r, w) for r in range(w)]
            assert rs[0][0] == 0 and rs[-1][1] == n
            assert all(a[1] == b[0] for a, b in zip(rs, rs[1:]))
            assert max(h - l for l, h in rs) - min(h - l for l, h in rs) <= 1


def _best_worker(rank, world, port, n, q):
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    import torch.distributed as dist
    import oracle
    import synth as sy
    from synth import analyses as an_mod
    from paper_2211_14346_gb300.shard import shard_range, merge_results
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        cols = sy.gen_semilep(n, 31)
        an = an_mod.semilep(sigma_jet=0.10, sigma_met=10.0)
        lo, hi = shard_range(n, rank, world)
        b = oracle.best_of(an, cols.slice(lo, hi), seed=8, V=6, first_event_id=lo)
        r = dict(hist=b["hist"], reco=b["reco"].astype(np.float32), mask=(b["best_v"] >= 0).astype(np.uint8),
                 best_v=np.where(b["best_v"] >= 0, b["best_v"], 0xffff).astype(np.uint16))
        m = merge_results(r)
        if rank == 0:
            q.put({k: (v.tolist() if isinstance(v, np.ndarray) else v) for k, v in m.items()})
    finally:
        dist.destroy_process_group()


def test_two_rank_merge_of_best_of_variations(orc):
    """Best-of-variations over two gloo ranks (the oracle on each shard): the
    merged chosen variations, their quantities and the per-event histogram
    equal the one-rank result."""
    import multiprocessing as mp
    n = 120
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_best_worker, args=(r, 2, port, n, q)) for r in range(2)]
    for p in ps:
        p.start()
    m = q.get(timeout=180)
    for p in ps:
        p.join(timeout=60)
        assert p.exitcode == 0
    an = analyses.semilep(sigma_jet=0.10, sigma_met=10.0)
    b = orc.best_of(an, synth.gen_semilep(n, 31), seed=8, V=6)
    want = np.where(b["best_v"] >= 0, b["best_v"], 0xffff).astype(np.uint16)
    assert (want != 0xffff).sum() > 10
    assert np.array_equal(np.asarray(m["best_v"], np.uint16), want)
    assert np.array_equal(np.asarray(m["hist"], np.uint64), b["hist"])
    assert np.array_equal(np.asarray(m["reco"], np.float32), b["reco"].astype(np.float32))


def _gpu_worker(rank, world, port, n, q):
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    import torch
    import torch.distributed as dist
    import synth as sy
    from synth import analyses as an_mod
    from paper_2211_14346_gb300 import Engine, DeviceColumns
    from paper_2211_14346_gb300.shard import shard_range, merge_results
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        torch.cuda.set_device(0)
        cols = sy.gen_semilep(n, 23)
        an = an_mod.config2()
        lo, hi = shard_range(n, rank, world)
        with Engine(0) as eng:
            aid = eng.define(an)
            r = eng.run_device(aid, DeviceColumns(cols.slice(lo, hi)), V=16, seed=44, first_event_id=lo).numpy()
            assert eng.device_error() == 0
        m = merge_results(r)
        if rank == 0:
            q.put({k: (v.tolist() if isinstance(v, np.ndarray) else v) for k, v in m.items()})
    finally:
        dist.destroy_process_group()


@pytest.mark.gpu
def test_two_gpu_processes_merge_equals_oracle(orc):
    """The multi-rank path with the GPU kernels: two processes (both on
    cuda:0 here; their kernels never wait on one another), each runs its
    contiguous shard through the library, gloo merges the counts and the
    per-event outputs; the merge equals the oracle over all events."""
    import multiprocessing as mp
    from tests.parity import assert_parity
    n = 6001
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_gpu_worker, args=(r, 2, port, n, q)) for r in range(2)]
    for p in ps:
        p.start()
    m = q.get(timeout=600)
    for p in ps:
        p.join(timeout=120)
        assert p.exitcode == 0
    o = orc.run(analyses.config2(), synth.gen_semilep(n, 23), seed=44, V=16)
    g = {k: np.asarray(v) for k, v in m.items()}
    g["cutflow"] = g["cutflow"].astype(np.uint64)
    g["hist"] = g["hist"].astype(np.uint64)
    g["n_surv"] = g["n_surv"].astype(np.uint16)
    g["mask"] = g["mask"].astype(np.uint8)
    assert_parity(g, o, what="two processes")
