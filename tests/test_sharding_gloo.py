"""Sample sharding across two processes (gloo, CPU): each rank evaluates its
contiguous share of the samples, one all-reduce combines them, and the result
equals the unsharded evaluation (linearity in the samples, Eq. costHS)."""
import os
import socket

import numpy as np
import pytest

from paper_2604_20384_gb300.sharding import pack, shard_bounds, unpack


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def test_shard_bounds_cover_samples_once():
    for ns in (1, 5, 16, 63):
        for world in (1, 2, 3, 8):
            seen = []
            for r in range(world):
                lo, hi = shard_bounds(ns, r, world)
                seen.extend(range(lo, hi))
            assert seen == list(range(ns))


def _worker(rank, world, port, ret):
    import torch.distributed as dist

    from oracle import oracle
    from paper_2604_20384_gb300.inputs import make_workload
    from paper_2604_20384_gb300.sharding import allreduce

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    w = make_workload(7, 5, 11, seed=21)
    lo, hi = shard_bounds(w.n_samples, rank, world)
    sub = w.psi1q[lo:hi]
    phi = oracle.reference_states(7, 5, w.Uref, sub)
    o = oracle.evaluate(7, 5, w.G, w.V, sub, phi, threads=1)
    loss, g, h = allreduce(hi - lo, o["loss"], o["grad"], o["hvp"])
    dist.barrier()
    dist.destroy_process_group()
    if rank == 0:
        ret.put((loss, g, h))


def test_two_rank_gloo_allreduce_equals_unsharded():
    import sys

    import torch.multiprocessing as mp

    from oracle import oracle
    from paper_2604_20384_gb300.inputs import make_workload

    here = os.path.dirname(os.path.abspath(__file__))
    root = os.path.dirname(here)
    os.environ["PYTHONPATH"] = os.pathsep.join([here, root, os.environ.get("PYTHONPATH", "")])
    sys.path[:0] = [here, root]
    ctx = mp.get_context("spawn")
    ret = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, ret)) for r in range(2)]
    for p in procs:
        p.start()
    loss, g, h = ret.get(timeout=120)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    w = make_workload(7, 5, 11, seed=21)
    phi = oracle.reference_states(7, 5, w.Uref, w.psi1q)
    o = oracle.evaluate(7, 5, w.G, w.V, w.psi1q, phi, threads=1)
    assert abs(loss - o["loss"]) < 1e-14
    assert np.max(np.abs(g - o["grad"])) < 1e-14
    assert np.max(np.abs(h - o["hvp"])) < 1e-14


def test_pack_unpack_round_trip():
    rng = np.random.default_rng(0)
    g = rng.standard_normal((3, 4, 4)) + 1j * rng.standard_normal((3, 4, 4))
    h = rng.standard_normal((3, 4, 4)) + 1j * rng.standard_normal((3, 4, 4))
    loss, g2, h2 = unpack(pack(5, 0.25, g, h), 3)
    assert abs(loss - 0.25) < 1e-15 and np.allclose(g2, g) and np.allclose(h2, h)
