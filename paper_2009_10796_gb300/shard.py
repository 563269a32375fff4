"""Sharding the probe update across devices.

Within a frame every probe's update depends only on the previous frame's
atlas (hit shading may sample any probe), so a frame splits into shards of
the probe grid: each device updates a contiguous z-slab of probes
(ddgi_update_range) against its own full copy of the previous state, then
the updated slabs are exchanged so every device holds the whole new state
(one all-gather per frame).  The scene and BVH are replicated.

`slabs` partitions the grid; `SlabExchange` all-gathers the slabs of flat
per-probe buffers (atlases, states) with torch.distributed, on whatever
backend the process group uses (NCCL between GPUs: the gathered slabs land
in every device's own memory), through send and receive buffers kept
across frames; `exchange` is the one-shot form.
"""
from __future__ import annotations

import torch
import torch.distributed as dist


def slabs(counts, world: int):
    """Contiguous z-slabs of a grid with `counts` = (cx, cy, cz): per rank the
    probe index range [begin, end) (probe p = i + cx*(j + cy*k))."""
    cx, cy, cz = (int(c) for c in counts)
    plane = cx * cy
    out = []
    for r in range(world):
        k0 = (cz * r) // world
        k1 = (cz * (r + 1)) // world
        out.append((k0 * plane, k1 * plane))
    return out


def exchange(buffers, per_probe_bytes, ranges, rank: int, group=None):
    """All-gather the shards of per-probe buffers in place.

    buffers:         flat uint8 tensors [P * per_probe_bytes[b]] (one per buffer)
    per_probe_bytes: bytes of one probe's entry in each buffer
    ranges:          per-rank probe ranges (from `slabs`)
    After the call every rank's buffers hold every rank's shard."""
    world = len(ranges)
    width = max(e - b for b, e in ranges)
    for buf, nb in zip(buffers, per_probe_bytes):
        b0, e0 = ranges[rank]
        send = torch.zeros(width * nb, dtype=torch.uint8, device=buf.device)
        send[: (e0 - b0) * nb] = buf[b0 * nb: e0 * nb]
        recv = [torch.empty_like(send) for _ in range(world)]
        dist.all_gather(recv, send, group=group)
        for r, (b, e) in enumerate(ranges):
            if r != rank:
                buf[b * nb: e * nb] = recv[r][: (e - b) * nb]
    return buffers


class SlabExchange:
    """Per-frame all-gather of probe slabs with persistent buffers.

    buffers are flat uint8 tensors [P * per_probe_bytes[b]] on one device,
    the same every call (the volume's atlases and states as the caller keeps
    them); ranges the per-rank probe ranges from `slabs`.  Every slab is
    padded to the widest one, so one collective per buffer moves a
    contiguous [world][width * bytes] block; the send and receive blocks are
    allocated once here and reused every frame."""

    def __init__(self, per_probe_bytes, ranges, rank: int, device, group=None):
        self.nb = list(per_probe_bytes)
        self.ranges = list(ranges)
        self.rank = rank
        self.group = group
        self.world = len(ranges)
        self.width = max(e - b for b, e in ranges)
        self.send = [torch.zeros(self.width * nb, dtype=torch.uint8, device=device) for nb in self.nb]
        self.recv = [torch.empty(self.world * self.width * nb, dtype=torch.uint8, device=device) for nb in self.nb]

    def __call__(self, buffers):
        b0, e0 = self.ranges[self.rank]
        for buf, nb, snd, rcv in zip(buffers, self.nb, self.send, self.recv):
            snd[: (e0 - b0) * nb].copy_(buf[b0 * nb: e0 * nb])
            dist.all_gather_into_tensor(rcv, snd, group=self.group)
            blocks = rcv.view(self.world, self.width * nb)
            for r, (b, e) in enumerate(self.ranges):
                if r != self.rank:
                    buf[b * nb: e * nb].copy_(blocks[r, : (e - b) * nb])
        return buffers
