"""Sharded update over two gloo ranks on the CPU: each rank updates its z-slab
of probes against the full previous state, `shard.exchange` all-gathers the
slabs, and the result equals the unsharded update.  The FP64 oracle stands
in for the device update (this checks the partition and the exchange)."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import oracle
import synth


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _as_bytes(a):
    return torch.from_numpy(a.reshape(-1).view(np.uint8))


def _rank(rank, world, port, out_path, persistent=False):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from paper_2009_10796_gb300 import shard
    sc = synth.room_scene(n_boxes=10)
    L = synth.room_lights()
    desc = synth.room_volume(counts=(4, 4, 6), spacing=(2.5, 2.5, 1.6), origin=(1.25, 1.25, 1.0),
                             hysteresis_irr=0.6, hysteresis_vis=0.6, rays_per_probe=32)
    h = oracle.SceneHandle(sc)
    st, irr, dist_ = oracle.new_state(desc)
    ranges = shard.slabs(desc.counts, world)
    P = desc.n_probes
    nb = [irr.nbytes // P, dist_.nbytes // P, 1]
    ex = shard.SlabExchange(nb, ranges, rank, "cpu") if persistent else None
    bufs = [_as_bytes(irr), _as_bytes(dist_), _as_bytes(st)]
    kept = [t.data_ptr() for t in ex.send + ex.recv] if persistent else []
    for frame in range(3):
        b, e = ranges[rank]
        oracle.update(h, L, desc, frame, st, irr, dist_, subset=np.arange(b, e))
        if persistent:
            ex(bufs)
        else:
            shard.exchange(bufs, nb, ranges, rank)
    if persistent:   # the same send and receive buffers every frame
        assert [t.data_ptr() for t in ex.send + ex.recv] == kept
    if rank == 0:
        np.savez(out_path, st=st, irr=irr, dist=dist_)
    dist.barrier()
    dist.destroy_process_group()


def test_slabs_partition_the_grid():
    from paper_2009_10796_gb300 import shard
    for counts, world in (((4, 4, 6), 2), ((32, 16, 32), 8), ((3, 2, 5), 4), ((2, 2, 2), 3)):
        r = shard.slabs(counts, world)
        assert r[0][0] == 0 and r[-1][1] == counts[0] * counts[1] * counts[2]
        assert all(r[k][1] == r[k + 1][0] for k in range(world - 1))
        assert all((e - b) % (counts[0] * counts[1]) == 0 for b, e in r)


@pytest.mark.parametrize("persistent", [False, True])
def test_two_gloo_ranks_match_unsharded_update(tmp_path, persistent):
    """Both the one-shot exchange and SlabExchange (persistent buffers, one
    all_gather_into_tensor per buffer) reproduce the unsharded update."""
    out = str(tmp_path / "sharded.npz")
    mp.start_processes(_rank, args=(2, _free_port(), out, persistent), nprocs=2, join=True, start_method="spawn")
    got = np.load(out)
    sc = synth.room_scene(n_boxes=10)
    L = synth.room_lights()
    desc = synth.room_volume(counts=(4, 4, 6), spacing=(2.5, 2.5, 1.6), origin=(1.25, 1.25, 1.0),
                             hysteresis_irr=0.6, hysteresis_vis=0.6, rays_per_probe=32)
    h = oracle.SceneHandle(sc)
    st, irr, dist_ = oracle.new_state(desc)
    for frame in range(3):
        oracle.update(h, L, desc, frame, st, irr, dist_)
    assert np.array_equal(got["st"], st)
    assert np.array_equal(got["irr"], irr)
    assert np.array_equal(got["dist"], dist_)
