"""ddgi_update_range: shards of a frame updated on copies of the same state,
their ranges exchanged, reproduce one full ddgi_update (one GPU; the
exchange is a device-to-device copy standing in for the all-gather)."""
import pytest
import torch

import synth

pytestmark = pytest.mark.gpu


def test_sequential_shards_equal_full_update():
    import paper_2009_10796_gb300 as g
    from paper_2009_10796_gb300 import shard
    torch.cuda.set_device(0)
    sc = synth.city_scene()
    L = synth.city_lights()
    desc = synth.city_volume()
    S = g.Scene.from_arrays(sc)
    full = g.Volume(desc)
    world = 3
    parts = [g.Volume(desc) for _ in range(world)]
    ranges = shard.slabs(desc.counts, world)
    P = desc.n_probes
    for frame in range(3):
        full.update(S, L, frame)
        for r, (b, e) in enumerate(ranges):
            parts[r].update_range(S, L, frame, b, e)
        # exchange: every copy receives every shard's range
        bufs = [[v.irr_raw(), v.dist_raw(), v.states()] for v in parts]
        nb = [full.info.irr_bytes // P, full.info.dist_bytes // P, 1]
        merged = []
        for k in range(3):
            m = torch.empty_like(bufs[0][k])
            for r, (b, e) in enumerate(ranges):
                m[b * nb[k]: e * nb[k]] = bufs[r][k][b * nb[k]: e * nb[k]]
            merged.append(m)
        for v in parts:
            for k in range(3):
                v.set_buffer(k, merged[k])
        torch.cuda.synchronize()
        assert torch.equal(merged[2], full.states())
        assert torch.equal(merged[0], full.irr_raw())
        assert torch.equal(merged[1], full.dist_raw())
