"""Multi-process (world size 2, gloo on CPU) checks of the event-sharding host logic.

The GPU path shards events across ranks with no data-path collective; what crosses ranks is the
barrier, the max of the timed durations and the host-side gather of results.  These tests run
that logic on two CPU processes: each rank reconstructs its round-robin share of a small event
list with the oracle, rank 0 gathers the shares, and the union must equal the whole list
reconstructed in one process.  The weak-scaling seed ranges must be disjoint.
"""
import os
import pickle
import socket
import sys

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

from paper_2104_06573_gb300 import shard, synth  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
N_EVENTS = 7
TRACKS = 25


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _tuples(ev, P):
    import oracle
    r = oracle.reconstruct(ev.x, ev.y, ev.z, ev.layer, P)
    return sorted(tuple(int(h) for h in t) for t in r["tuples"])


def _rank_main(rank, world, port, out_dir):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        P = synth.params_barrel_quadruplets()
        mine = shard.shard(N_EVENTS, rank, world)
        res = {int(e): _tuples(synth.event_barrel(int(e), TRACKS), P) for e in mine}
        shard.barrier()
        t = shard.max_over_ranks(1.5 + rank)       # rank durations 1.5, 2.5 -> job time 2.5
        parts = shard.gather_to_rank0(res)
        if rank == 0:
            merged = {}
            for p in parts:
                assert not set(p) & set(merged), "events processed twice"
                merged.update(p)
            with open(os.path.join(out_dir, "merged.pkl"), "wb") as f:
                pickle.dump((merged, t), f)
        else:
            assert parts is None
        np.save(os.path.join(out_dir, f"max_{rank}.npy"), np.array([t]))
    finally:
        dist.destroy_process_group()


def test_shard_is_a_partition():
    for n in (0, 1, 7, 256):
        for world in (1, 2, 3, 8):
            parts = [shard.shard(n, r, world) for r in range(world)]
            allv = np.concatenate(parts) if parts else np.array([])
            assert sorted(allv.tolist()) == list(range(n))
            sizes = [len(p) for p in parts]
            assert max(sizes) - min(sizes) <= 1
    with pytest.raises(ValueError):
        shard.shard(4, 2, 2)


def test_rank_seed_ranges_disjoint():
    from paper_2104_06573_gb300 import synth as s
    n = 256
    ranges = [set(range(shard.rank_seed0(r), shard.rank_seed0(r) + n)) for r in range(8)]
    for a in range(8):
        for b in range(a + 1, 8):
            assert not ranges[a] & ranges[b]
    assert len(s.batch_track_counts(n, shard.rank_seed0(1))) == n


def test_single_process_identities():
    assert shard.max_over_ranks(3.25) == 3.25
    assert shard.gather_to_rank0({"a": 1}) == [{"a": 1}]
    shard.barrier()


def test_two_rank_gloo_shards_equal_whole(orc, tmp_path):
    world = 2
    mp.start_processes(_rank_main, args=(world, _free_port(), str(tmp_path)), nprocs=world,
                       join=True, start_method="spawn")
    with open(tmp_path / "merged.pkl", "rb") as f:
        merged, t0 = pickle.load(f)
    assert t0 == 2.5
    for r in range(world):
        assert float(np.load(tmp_path / f"max_{r}.npy")[0]) == 2.5
    P = synth.params_barrel_quadruplets()
    whole = {e: _tuples(synth.event_barrel(e, TRACKS), P) for e in range(N_EVENTS)}
    assert merged == whole
    assert sum(len(v) for v in whole.values()) > 0
