"""Continuous-batching ingest of packet batches into per-window cubes.

Deployment model (Section III, Section IV.A): packets reach a local
server in batches; they are buffered in host memory, copied to the GPU and
scanned into the current window's cube (Alg. 1); when a window closes its
cube is restored (Alg. 2, Alg. 3) while the next window already fills.

This module serves several independent streams ("tenants": monitored
networks) at once:

* Requests (host batches of pairs) are admitted as soon as a staging
  slot is free and their window holds a cube, so the copy of one batch,
  the update of another and the detect of a closed window overlap on the
  device (copy stream, compute stream, detect stream).  Batches of the
  same window already queued behind an admitted one join it in its slot
  while they fit: one copy each, one update for all.
* Window cubes come from a pool sized by a device-memory budget; a new
  window waits (its batches stay queued) until a cube is free again.  At
  most two cubes per tenant are in use (double buffering: one filling,
  one being restored).
* Closing a window enqueues its detect behind the window's last update;
  the host list comes back through pinned memory; the latency from close
  to host list is recorded.
* Host-side waits are bounded: drain() gives up with CBAA_ERR_TIMEOUT.

Orchestration only: every step on the data runs in libcbaa's kernels.
"""
from __future__ import annotations

import collections
import dataclasses
import time

import numpy as np

from . import cbaa as C


@dataclasses.dataclass
class WindowResult:
    tenant: object
    window: int
    hosts: np.ndarray
    info: dict
    packets: int
    close_t: float
    done_t: float

    @property
    def latency_s(self) -> float:
        return self.done_t - self.close_t


@dataclasses.dataclass
class _Request:
    tenant: object
    window: int
    pairs: object          # pinned host tensor int32 [n, 2]
    n: int
    arrival_t: float


class _Slot:
    def __init__(self, geo, slot_pairs, device):
        torch = C._torch()
        self.stage = torch.empty((slot_pairs, 2), dtype=torch.int32, device=device)
        self.uws = C.UpdateWorkspace(geo, slot_pairs, device=device)
        self.done = None          # event after the update that used this slot
        self.busy = False


class _Open:
    """A tenant's window that is filling."""

    def __init__(self, window, cube):
        self.window, self.cube = window, cube
        self.last = None          # event after the latest update into this cube
        self.packets = 0


class Server:
    def __init__(self, geo: dict, theta: int, *, n_slots: int = 4, slot_pairs: int = 1 << 22,
                 mem_budget: int | None = None, n_cubes: int | None = None, max_candidates: int = 1 << 18,
                 cap: int = 1 << 14, lookahead: int = 64, device="cuda"):
        torch = C._torch()
        self.geo, self.theta, self.cap, self.device = dict(geo), theta, cap, device
        self.cube_bytes = C.cube_bytes(geo)
        slot_bytes = slot_pairs * 8 + C.update_workspace_bytes(geo, slot_pairs)
        det_bytes = C.workspace_bytes(geo, max_candidates) + 16 * cap + 64
        if n_cubes is None:
            if mem_budget is None:
                n_cubes = 4
            else:
                n_cubes = (mem_budget - n_slots * slot_bytes - det_bytes) // self.cube_bytes
        if n_cubes < 1:
            raise C.CbaaError(C.ERR_INVALID_ARG, "memory budget holds no window cube")
        self.mem_bytes = n_slots * slot_bytes + det_bytes + n_cubes * self.cube_bytes
        self.slot_pairs = slot_pairs
        self.slots = [_Slot(geo, slot_pairs, device) for _ in range(n_slots)]
        self.free_cubes = collections.deque((C.Cube(geo, device=device), None) for _ in range(n_cubes))
        self.n_cubes = n_cubes
        self.copy_s = torch.cuda.Stream(device=device)
        self.comp_s = torch.cuda.Stream(device=device)
        self.det_s = torch.cuda.Stream(device=device)
        self.dws = C.Workspace(geo, max_candidates=max_candidates, device=device)
        self.dev_out = torch.zeros(4 * cap, dtype=torch.int32, device=device)
        self.dev_info = torch.zeros(8, dtype=torch.int32, device=device)
        self.queue = collections.deque()        # requests not yet admitted (arrival order)
        self.open = {}                          # tenant -> _Open
        self.closing = collections.deque()      # (tenant, _Open, close_t) waiting for a cube-free detect slot
        self.detecting = collections.deque()    # (tenant, _Open, close_t, done_event, host_out, host_info)
        self.results = []
        self.stats = dict(admitted=0, queued_for_cube=0, queued_for_slot=0, max_cubes_in_use=0, batches=0,
                          updates=0)
        self.lookahead = lookahead
        self.opened = {}                        # tenant -> windows that got a cube (most recent last)
        self.opened_keep = 4096

    # ------------------------------------------------------------------ public API
    def submit(self, tenant, window: int, pairs, arrival_t: float | None = None, poll: bool = True):
        """Queue a batch (host int32/uint32 [n, 2] tensor, ideally pinned) for tenant's window.
        poll=False only queues it (a burst submitted at once is admitted by the next poll)."""
        n = int(pairs.shape[0])
        if n > self.slot_pairs:
            raise C.CbaaError(C.ERR_INVALID_ARG, f"batch of {n} pairs exceeds the slot size {self.slot_pairs}")
        self.queue.append(_Request(tenant, window, pairs, n, time.perf_counter() if arrival_t is None else arrival_t))
        if poll:
            self.poll()

    def close(self, tenant, window: int, poll: bool = True):
        """Mark tenant's window complete: its detect runs once its queued batches are in.  A window that
        received no batch still yields a result (the detect of an empty cube: no packets, no hosts); a
        close for a window that a newer window's batch has already closed changes nothing."""
        self.queue.append(_Request(tenant, window, None, -1, time.perf_counter()))
        if poll:
            self.poll()

    def poll(self):
        """Advance: retire finished work, admit queued requests, start detects."""
        self._retire()
        self._admit()
        self._start_detects()
        self._retire()

    def drain(self, timeout_s: float = 60.0):
        t0 = time.perf_counter()
        while self.queue or self.closing or self.detecting or any(s.busy for s in self.slots):
            self.poll()
            if time.perf_counter() - t0 > timeout_s:
                raise C.CbaaError(C.ERR_TIMEOUT, "serve drain")
            time.sleep(0)
        return self.results

    def cubes_in_use(self) -> int:
        return self.n_cubes - len(self.free_cubes)

    # ------------------------------------------------------------------ internals
    def _take_cube(self):
        if not self.free_cubes:
            return None
        cube, ready = self.free_cubes.popleft()
        if ready is not None:
            self.comp_s.wait_event(ready)        # its reset after the last detect
        self.stats["max_cubes_in_use"] = max(self.stats["max_cubes_in_use"], self.cubes_in_use())
        return cube

    def _admit(self):
        torch = C._torch()
        blocked_tenants = set()
        pending = collections.deque()
        while self.queue:
            r = self.queue.popleft()
            if r.tenant in blocked_tenants:          # keep each tenant's order
                pending.append(r)
                continue
            cur = self.open.get(r.tenant)
            if r.n < 0:                              # close marker
                if cur is not None and cur.window == r.window:
                    self.closing.append((r.tenant, cur, time.perf_counter()))
                    del self.open[r.tenant]
                elif r.window not in self.opened.get(r.tenant, ()):
                    # a window that received no batch: its result is the detect of an empty cube
                    cube = self._take_cube()
                    if cube is None:
                        self.stats["queued_for_cube"] += 1
                        blocked_tenants.add(r.tenant)
                        pending.append(r)
                        continue
                    self._mark_opened(r.tenant, r.window)
                    self.closing.append((r.tenant, _Open(r.window, cube), time.perf_counter()))
                # else: the window was closed already by a batch of a newer window; its result stands
                continue
            if cur is None or cur.window != r.window:
                if cur is not None:                  # a newer window closes the current one
                    self.closing.append((r.tenant, cur, time.perf_counter()))
                    del self.open[r.tenant]
                cube = self._take_cube()
                if cube is None:
                    self.stats["queued_for_cube"] += 1
                    blocked_tenants.add(r.tenant)
                    pending.append(r)
                    continue
                cur = self.open[r.tenant] = _Open(r.window, cube)
                self._mark_opened(r.tenant, r.window)
            slot = next((s for s in self.slots if not s.busy), None)
            if slot is None:
                self.stats["queued_for_slot"] += 1
                blocked_tenants.add(r.tenant)
                pending.append(r)
                continue
            slot.busy = True
            group = [r] + self._absorb(r)
            with torch.cuda.stream(self.copy_s):
                off = 0
                for q in group:
                    slot.stage[off:off + q.n].copy_(q.pairs, non_blocking=True)
                    off += q.n
                copied = torch.cuda.Event()
                copied.record(self.copy_s)
            self.comp_s.wait_event(copied)
            cur.cube.update_binned(slot.stage, slot.uws, n=off, stream=self.comp_s)
            slot.done = torch.cuda.Event()
            slot.done.record(self.comp_s)
            cur.last = slot.done
            cur.packets += off
            self.stats["admitted"] += len(group)
            self.stats["batches"] += len(group)
            self.stats["updates"] += 1
        self.queue = pending

    def _mark_opened(self, tenant, window):
        """Remember that tenant's window got a cube (a close marker for it then never opens an empty one);
        the most recent `opened_keep` windows per tenant are kept."""
        seen = self.opened.setdefault(tenant, collections.OrderedDict())
        seen[window] = True
        while len(seen) > self.opened_keep:
            seen.popitem(last=False)

    def _absorb(self, r):
        """Later queued batches of r's tenant and window that fill r's slot with it (one copy each, one
        update for all): the tenant's next requests in order, up to the first that is of another window,
        a close marker or too large, looking at most `lookahead` requests ahead."""
        taken, room, keep = [], self.slot_pairs - r.n, []
        for i, q in enumerate(self.queue):
            if i >= self.lookahead:
                break
            if q.tenant != r.tenant:
                continue
            if q.n < 0 or q.window != r.window or q.n > room:
                break
            taken.append(q)
            keep.append(i)
            room -= q.n
        if keep:
            drop = set(keep)
            self.queue = collections.deque(q for i, q in enumerate(self.queue) if i not in drop)
        return taken

    def _start_detects(self):
        torch = C._torch()
        # one detect at a time owns the detect workspace and output buffers
        while self.closing and not self.detecting:
            tenant, win, close_t = self.closing.popleft()
            if win.last is not None:
                self.det_s.wait_event(win.last)
            win.cube.detect_async(self.theta, self.dws, self.dev_out, self.dev_info, stream=self.det_s)
            host_out = torch.empty(4 * self.cap, dtype=torch.int32, pin_memory=True)
            host_info = torch.empty(8, dtype=torch.int32, pin_memory=True)
            with torch.cuda.stream(self.det_s):
                host_info.copy_(self.dev_info, non_blocking=True)
                host_out.copy_(self.dev_out, non_blocking=True)
                done = torch.cuda.Event()
                done.record(self.det_s)
                win.cube.reset(stream=self.det_s)
                ready = torch.cuda.Event()
                ready.record(self.det_s)
            self.detecting.append((tenant, win, close_t, done, host_out, host_info, ready))

    def _retire(self):
        for s in self.slots:
            if s.busy and s.done is not None and s.done.query():
                s.busy = False
        while self.detecting and self.detecting[0][3].query():
            tenant, win, close_t, done, host_out, host_info, ready = self.detecting.popleft()
            t = time.perf_counter()
            hosts, info = C.hosts_from_device(host_out, host_info)
            self.results.append(WindowResult(tenant, win.window, hosts, info, win.packets, close_t, t))
            self.free_cubes.append((win.cube, ready))
