"""Batched windows over simulated edge routers, replayed as one CUDA graph.

Section III.C's deployment: every edge router scans its own packets into a
local cube (Alg. 1); at the end of each time window the global server ORs
the local cubes together and restores the super hosts (Alg. 2, Alg. 3).
Here the routers are local cubes on one GPU.  For each window the
library's partitioned update feeds all router cubes in one pass (so uneven
router loads share the whole GPU) and ORs every word it flushes into a
router cube into the global cube as well (the global server's merge,
without a second pass over the router cubes), and the detect writes that
window's host list to device memory.  The global cube is double-buffered: window w's detect runs on a
side stream while window w+1's routers are reset and updated, as a global
server detects one window while the routers scan the next.  A sequence of
windows is recorded once into a CUDA graph (a fork/join over the two
streams) and replayed with a single launch.

Orchestration only: every step runs in libcbaa's kernels.
"""
from __future__ import annotations

from . import cbaa as C


class RouterWindows:
    """Device state for ``n_windows`` windows of ``n_routers`` router cubes plus a global cube."""

    def __init__(self, geo: dict, n_routers: int, theta: int, max_pairs: int, n_windows: int, cap: int = 1 << 14,
                 max_candidates: int = 1 << 18, device="cuda"):
        torch = C._torch()
        self.geo, self.theta, self.cap = dict(geo), theta, cap
        self.routers = [C.Cube(geo, device=device) for _ in range(n_routers)]
        self.globs = [C.Cube(geo, device=device) for _ in range(2)]
        self.uws = C.UpdateWorkspace(geo, max_pairs, device=device, n_cubes=n_routers)
        self.dws = [C.Workspace(geo, max_candidates=max_candidates, device=device) for _ in range(2)]
        self.side = torch.cuda.Stream(device)
        self.out = torch.zeros((n_windows, 4 * cap), dtype=torch.int32, device=device)
        self.info = torch.zeros((n_windows, 8), dtype=torch.int32, device=device)
        self.graph = None
        self._keep = None

    @property
    def glob(self):
        """The global cube of the last enqueued window."""
        return self.globs[(self._last_w if self._last_w is not None else 0) & 1]

    _last_w = None

    def enqueue_window(self, w: int, router_pairs, done=None):
        """One window on the current stream: reset router cubes and global cube w mod 2, one update
        pass over all router cubes that also ORs every bit it sets into the global cube (so global = OR
        of the router cubes without a merge pass reading them back); the detect goes to the side
        stream.  `done[b]` is the event after the last detect of global cube b (its reset waits)."""
        torch = C._torch()
        main = torch.cuda.current_stream()
        b = w & 1
        for c in self.routers:
            c.reset()
        if done is not None and done[b] is not None:
            main.wait_event(done[b])
        self.globs[b].reset()
        C.update_multi(self.routers, router_pairs, self.uws, merge_into=self.globs[b])
        merged = torch.cuda.Event()
        merged.record(main)
        self.side.wait_event(merged)
        with torch.cuda.stream(self.side):
            self.globs[b].detect_async(self.theta, self.dws[b], self.out[w], self.info[w])
            if done is not None:
                done[b] = torch.cuda.Event()
                done[b].record(self.side)
        self._last_w = w

    def enqueue(self, windows):
        """All windows on the current stream; returns after the current stream has joined the side
        stream, so everything enqueued is ordered before later work on the current stream."""
        torch = C._torch()
        main = torch.cuda.current_stream()
        self.side.wait_stream(main)
        done = [None, None]
        for w, rp in enumerate(windows):
            self.enqueue_window(w, rp, done)
        main.wait_stream(self.side)

    def tune(self, windows, reps: int = 3):
        """Pick the tiling and routing shape of the partitioned update for these router cubes by
        timing the first window (tile kinds 1-3 x routing shapes of 8 and 16 packets per thread).

        Sets the process-wide tuning; call before capture() so the graph records the choice."""
        torch = C._torch()
        stream = torch.cuda.current_stream()
        best = None
        base = C.get_tuning()
        for kind in (1, 2, 3):
            for shape in ((0,) if kind == 1 else (0, 6, 8)):      # column tiles take one shape
                C.set_tuning(**{**base, "tile_kind": kind, "scatter_shape": shape})
                times = []
                for rep in range(reps + 1):
                    for c in self.routers:
                        c.reset()
                    self.globs[0].reset()
                    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    e0.record(stream)
                    C.update_multi(self.routers, windows[0], self.uws, merge_into=self.globs[0])
                    e1.record(stream)
                    torch.cuda.synchronize()
                    if rep:
                        times.append(e0.elapsed_time(e1))
                t = sorted(times)[len(times) // 2]
                if best is None or t < best[2]:
                    best = (kind, shape, t)
        C.set_tuning(**{**base, "tile_kind": best[0], "scatter_shape": best[1]})
        return {"tile_kind": best[0], "scatter_shape": best[1], "update_ms": best[2]}

    def capture(self, windows):
        """Record every window into one CUDA graph (after one eager pass on a side stream)."""
        torch = C._torch()
        side = torch.cuda.Stream()
        side.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(side):
            self.enqueue(windows)
        torch.cuda.current_stream().wait_stream(side)
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            self.enqueue(windows)
        self.graph, self._keep = g, windows
        return g

    def replay(self):
        self.graph.replay()

    def results(self):
        """[(hosts, info)] per window (synchronises)."""
        torch = C._torch()
        torch.cuda.synchronize()
        return [C.hosts_from_device(self.out[w], self.info[w]) for w in range(self.out.shape[0])]
