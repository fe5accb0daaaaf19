"""Multi-rank host logic on CPU (gloo, world size 2): disjoint vector seeds per rank,
one reduction of the moment arrays at the end, and an injected rank failure that
surfaces as an error on the surviving rank instead of a hang.  The per-rank moments
come from the oracle (no GPU here); the logic under test is the sharding and the
reduction that bench.py and users run on GPUs."""
import datetime
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

import kg_inputs as ki
from paper_1307_0288_gb300 import replicas


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, n_local, fail_rank, q):
    import torch.distributed as dist
    import oracle
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    try:
        dist.init_process_group("gloo", rank=rank, world_size=world,
                                timeout=datetime.timedelta(seconds=10))
        w = ki.sheet_cells(6, 5, vacancy_conc=0.03, lattice_seed=9,
                           vector_seed=replicas.rank_vector_seed(500, rank, n_local))
        ho = oracle.from_workload(w)
        phi = w.vectors(n_local)
        mu = np.stack([oracle.kpm_moments(ho, phi[:, r], phi[:, r], 40) for r in range(n_local)])
        if rank == fail_rank:
            raise RuntimeError("injected rank failure")
        avg = replicas.average_moments(mu, n_local)
        q.put((rank, "ok", avg))
        dist.destroy_process_group()
    except Exception as e:  # report, never hang
        q.put((rank, "error", repr(e)))


def _run(world, n_local, fail_rank=-1):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, n_local, fail_rank, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = {}
    for _ in range(world):
        rank, status, val = q.get(timeout=120)
        out[rank] = (status, val)
    for p in procs:
        p.join(timeout=60)
        if p.is_alive():
            p.kill()
    return out


def test_seeds_are_disjoint_across_ranks():
    seeds = [replicas.rank_vector_seed(1000, k, 4) for k in range(8)]
    streams = {(s + r) for s in seeds for r in range(4)}
    assert len(streams) == 32


def test_two_rank_average_equals_single_process_average():
    import oracle
    out = _run(2, 3)
    assert all(v[0] == "ok" for v in out.values()), out
    # the same six vectors in one process
    mus = []
    for rank in range(2):
        w = ki.sheet_cells(6, 5, vacancy_conc=0.03, lattice_seed=9,
                           vector_seed=replicas.rank_vector_seed(500, rank, 3))
        ho = oracle.from_workload(w)
        phi = w.vectors(3)
        mus += [oracle.kpm_moments(ho, phi[:, r], phi[:, r], 40) for r in range(3)]
    ref = np.mean(mus, axis=0)
    for rank in range(2):
        assert np.allclose(out[rank][1], ref, rtol=1e-13, atol=1e-12)


def test_failed_rank_gives_an_error_not_a_hang():
    out = _run(2, 2, fail_rank=1)
    assert out[1][0] == "error" and "injected" in out[1][1]
    assert out[0][0] == "error"      # the survivor's reduction failed (peer gone / timeout)
