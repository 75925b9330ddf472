"""Sketch-sharded merge and restoration across ranks (one process per GPU).

Section III.C: every edge router scans its packets into a local cube; the
global server ORs the local cubes and restores the super hosts.  With one
rank per GPU, each rank is a router, and the global server's work is split
by sketch: rank k owns the sketches [k S/N, (k+1) S/N), S = 2^r.  The cube
layout keeps a sketch's words contiguous, so one all-to-all hands every
rank the N copies of its own sketches; it ORs them (cbaa_or_words -- NCCL
has no bitwise-OR reduction) and restores its sketches alone
(cbaa_detect_range_async).  Detection is independent per sketch (each has
its own eps and Zmax), so the owners' host lists together are the global
list; they are all-gathered and merged by ip -- on the host (restore), or
device to device and merged by a kernel with no host wait (enqueue), so a
window's exchange and restoration overlap the next window's update.

Orchestration only: the OR and the restoration run in libcbaa's kernels, the
exchange and the gathers are torch.distributed collectives.  The two
collective steps are plain functions so that their logic can be exercised
with any backend.
"""
from __future__ import annotations

import numpy as np

from . import cbaa as C


def owned_range(geo: dict, rank: int, world: int) -> tuple[int, int]:
    """Sketches [lo, hi) owned by ``rank``; 2^r must be a multiple of ``world``."""
    S = 1 << geo["r"]
    if world < 1 or S % world:
        raise ValueError(f"2^r = {S} sketches do not split over {world} ranks")
    per = S // world
    return rank * per, (rank + 1) * per


def exchange_slices(memory, rank: int, world: int, recv, or_fn, group=None):
    """All-to-all of the N sketch slices of ``memory`` (a flat 32-bit tensor holding a cube), then
    ``or_fn(own_slice, [the other ranks' copies of it])``.  ``recv`` is scratch of memory's size.
    Afterwards this rank's slice of ``memory`` is the OR of every rank's slice."""
    import torch.distributed as dist
    words = memory.numel()
    if words % world:
        raise ValueError("cube words do not split over the ranks")
    per = words // world
    if world > 1:
        dist.all_to_all_single(recv, memory, group=group)
        own = memory[rank * per:(rank + 1) * per]
        or_fn(own, [recv[j * per:(j + 1) * per] for j in range(world) if j != rank])
    return memory[rank * per:(rank + 1) * per]


def gather_hosts(hosts: np.ndarray, rank: int, world: int, device, group=None) -> np.ndarray:
    """All-gather every rank's host list (structured HOST_DTYPE arrays of any length) and merge them
    by ip.  The owners' sketches are disjoint, so no address appears twice."""
    import torch
    import torch.distributed as dist
    if world == 1:
        return np.sort(hosts, order="ip")
    n = torch.tensor([hosts.size], dtype=torch.int64, device=device)
    counts = [torch.zeros_like(n) for _ in range(world)]
    dist.all_gather(counts, n, group=group)
    counts = [int(c.item()) for c in counts]
    m = max(1, max(counts))
    buf = np.zeros(m, dtype=C.HOST_DTYPE)
    buf[:hosts.size] = hosts
    mine = torch.from_numpy(buf.view(np.int32).copy()).to(device)
    parts = [torch.zeros_like(mine) for _ in range(world)]
    dist.all_gather(parts, mine, group=group)
    out = np.concatenate([p.cpu().numpy().view(C.HOST_DTYPE)[:c] for p, c in zip(parts, counts)])
    return np.sort(out, order="ip")


def gather_blocks(block, info, out_blocks, out_infos, world: int, group=None):
    """All-gather, device to device, every rank's fixed-capacity block of host records and its info
    words: rank j's land in out_blocks[j] and out_infos[j] (shapes [world, ...]).  No host round trip:
    the counts travel inside the info words and are read by the merge kernel."""
    import torch.distributed as dist
    if world == 1:
        out_blocks[0].copy_(block)
        out_infos[0].copy_(info)
        return
    dist.all_gather(list(out_blocks.unbind(0)), block, group=group)
    dist.all_gather(list(out_infos.unbind(0)), info, group=group)


class ShardedDetector:
    """The global server's restoration split over the ranks of a process group."""

    def __init__(self, geo: dict, theta: int, rank: int, world: int, device="cuda", cap: int = 1 << 16,
                 max_candidates: int = 1 << 18, group=None):
        torch = C._torch()
        self.geo, self.theta, self.rank, self.world, self.group = dict(geo), theta, rank, world, group
        self.lo, self.hi = owned_range(geo, rank, world)
        self.device = device
        self.recv = torch.empty(C.cube_bytes(geo) // 4, dtype=torch.int32, device=device)
        self.ws = C.Workspace(geo, max_candidates=max_candidates, device=device)
        self.out = torch.zeros(4 * cap, dtype=torch.int32, device=device)
        self.info = torch.zeros(8, dtype=torch.int32, device=device)
        # the asynchronous path: gathered blocks, and two result slots (one window restored while the
        # previous one's list is read)
        self.gath = torch.zeros((world, 4 * cap), dtype=torch.int32, device=device)
        self.ginfo = torch.zeros((world, 8), dtype=torch.int32, device=device)
        self.res = [torch.zeros(4 * cap * world, dtype=torch.int32, device=device) for _ in range(2)]
        self.res_info = [torch.zeros(8, dtype=torch.int32, device=device) for _ in range(2)]

    def merge(self, cube: "C.Cube"):
        """After this, ``cube`` holds, in this rank's sketches, the OR of every rank's cube."""
        exchange_slices(cube.memory, self.rank, self.world, self.recv, C.or_words, self.group)

    def restore(self, cube: "C.Cube") -> tuple[np.ndarray, dict]:
        """Restore this rank's sketches and gather every rank's hosts (synchronises)."""
        cube.detect_range_async(self.lo, self.hi, self.theta, self.ws, self.out, self.info)
        hosts, info = C.hosts_from_device(self.out, self.info)
        if info["status"] != C.OK:
            raise C.CbaaError(info["status"], "sharded restore")
        return gather_hosts(hosts, self.rank, self.world, self.device, self.group), info

    def __call__(self, cube: "C.Cube") -> tuple[np.ndarray, dict]:
        self.merge(cube)
        return self.restore(cube)

    def enqueue(self, cube: "C.Cube", slot: int):
        """The whole global-server step on the current stream, with no host wait: the sketch exchange
        and OR, the restoration of this rank's sketches, the device all-gather of every rank's hosts
        and info, and their merge by ip (cbaa_merge_hosts) into result slot ``slot`` (0 or 1)."""
        self.merge(cube)
        cube.detect_range_async(self.lo, self.hi, self.theta, self.ws, self.out, self.info)
        gather_blocks(self.out, self.info, self.gath, self.ginfo, self.world, self.group)
        C.merge_hosts(self.gath, self.ginfo, self.res[slot], self.res_info[slot])

    def result(self, slot: int) -> tuple[np.ndarray, dict]:
        """The global host list of the window last enqueued into ``slot`` (synchronises)."""
        return C.hosts_from_device(self.res[slot], self.res_info[slot])
