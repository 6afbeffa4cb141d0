"""The multi-GPU form is replicas with event sharding (events are independent,
no collective on the data path).  Two gloo ranks on the CPU check the host
logic: disjoint shards that together are the single-process batch, per-rank
results (oracle) that equal the single-process results, and the max-over-ranks
timing reduction."""
import os
import sys

import numpy as np
import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _rank(rank, world, port, out_dir):
    sys.path.insert(0, ROOT)
    import bench
    import oracle
    import velogen
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    first, n = bench.shard(rank, world, 3)
    b = velogen.generate(velogen.C2, n_events=n, first_event=first)
    r = oracle.reconstruct(b.offsets, b.pixels, b.geometry, oracle.Params(), n_threads=1)
    gathered = [None] * world
    dist.all_gather_object(gathered, (first, n, r["track_hits"].tolist(), r["track_offsets"].tolist()))
    slowest = bench.max_over_ranks(10.0 + rank, world, "cpu")
    if rank == 0:
        np.save(os.path.join(out_dir, "gathered.npy"), np.array(gathered, dtype=object), allow_pickle=True)
        np.save(os.path.join(out_dir, "slowest.npy"), np.array([slowest]))
    dist.destroy_process_group()


def test_two_rank_sharding_and_reduction(tmp_path):
    import socket
    with socket.socket() as s_:
        s_.bind(("127.0.0.1", 0))
        port = s_.getsockname()[1]
    mp.spawn(_rank, args=(2, port, str(tmp_path)), nprocs=2, join=True)
    gathered = np.load(tmp_path / "gathered.npy", allow_pickle=True)
    assert float(np.load(tmp_path / "slowest.npy")[0]) == 11.0
    (f0, n0, h0, o0), (f1, n1, h1, o1) = gathered
    assert (f0, n0, f1, n1) == (0, 3, 3, 3)
    import oracle
    import velogen
    whole = velogen.generate(velogen.C2, n_events=6)
    r = oracle.reconstruct(whole.offsets, whole.pixels, whole.geometry, oracle.Params(), n_threads=1)
    cut = int(r["track_offsets"][3])
    hits_cut = int(r["track_hit_offsets"][cut])
    assert h0 == r["track_hits"][:hits_cut].tolist() and h1 == r["track_hits"][hits_cut:].tolist()


def test_shard_rejects_bad_rank():
    sys.path.insert(0, ROOT)
    import bench
    with pytest.raises(ValueError):
        bench.shard(2, 2, 10)


def test_link_bound_schedules():
    """The copy bound of the end-to-end step: both directions at once while
    both have bytes left, then the rest alone -- or one after the other when
    that is shorter (worked by hand)."""
    import bench
    link = {"h2d_gbs": 50.0, "d2h_gbs": 60.0, "duplex_gbs_each": 40.0}
    # 1 GB in, 3 GB out: 1 GB each way at 40 GB/s (25 ms), then 2 GB out at 60 GB/s (33.3 ms)
    assert abs(bench.link_bound_ms(1_000_000_000, 3_000_000_000, link) - (25.0 + 2000.0 / 60.0)) < 1e-9
    # more in than out: the rest of the copy-in alone at 50 GB/s
    assert abs(bench.link_bound_ms(2_000_000_000, 1_000_000_000, link) - (25.0 + 20.0)) < 1e-9
    # a duplex rate below half of either direction: one after the other is shorter
    slow = {"h2d_gbs": 50.0, "d2h_gbs": 60.0, "duplex_gbs_each": 20.0}
    assert abs(bench.link_bound_ms(1_000_000_000, 1_000_000_000, slow) - (20.0 + 1000.0 / 60.0)) < 1e-9
    assert bench.link_bound_ms(0, 0, link) == 0.0
