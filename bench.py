#!/usr/bin/env python3
"""CBAA super-host detection benchmark on B300 (sm_103a).

One step = one time window through the whole hot path: zero the cube,
Alg. 1 over every packet of the window (already resident in HBM), then the
end-of-window pass (zero counts, eps/Zmax, Alg. 2 hot columns, Alg. 3 tuple
join + union checks, Thm. 2 estimates, sort).  The metric is packets per
second of that step (Gpps); detect latency and the update kernel's share of
its roofs are reported beside it.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl cbaa|reference]
                    [--workload window64m|window1m]

Under torchrun each rank runs its own window (weak scaling, no collective
on the data path); the step time is the maximum over ranks.
`--impl reference` times the plain CPU oracle on a bounded sample of the
same workload on this host's cores.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_1901_06207_b300 import traffic as T  # noqa: E402

METRIC = "packets/sec (Gpps) cube update + end-of-window detect ms; fraction of HBM/L2-atomic peak"


def update_kernels(partitioned: bool, tuning: dict, n: int) -> int:
    """Kernels of one single-cube update call of n packets (one pass of up to the workspace's
    packets): direct 1; partitioned count, scan, scatter, apply (with sampled run capacities the apply
    also drains the overflow list), and with the heavy-source split (on by default for row tiles and
    passes of >= 4Mi packets) sample, histogram and split (whose blocks pick the heavy sources) before
    them (the residual's counting kernel also ORs the heavy bitmaps into their columns)."""
    if not partitioned:
        return 1
    heavy = tuning.get("heavy", 0)
    split = tuning.get("tile_kind", 0) != 1 and heavy != 1 and (heavy >= 2 or n >= 4 << 20)
    return 7 if split else 4


def detect_kernels(geo: dict) -> int:
    """Kernels of one detect: zero counts (with eps and Zmax), hot lists, |RA|-1 joins, sort."""
    return 3 + (geo["n_ra"] - 1)


def workload(name: str, scale_shift: int = 0):
    from paper_1901_06207_b300.cbaa import make_params
    if name == "window64m":
        geo = make_params(5, 3, 1, 10, [12])
        spec = T.spec_window_64m(scale_shift=scale_shift)
        desc = dict(workload="window_64m_l2_cube" if scale_shift == 0 else f"window_64m_l2_cube/2^{scale_shift}",
                    packets_per_window=spec.n_packets, source_pool=spec.n_hosts,
                    planted_super_hosts=spec.n_planted, planted_peers="log-uniform [1024, 200000]",
                    background="Zipf(1.1) sources over the pool, uniform 2^32 peers", duplicate_fraction=0.3,
                    theta=1024, geometry="r=5, |RA|=3, |VA|=1, g=2^10, c=2^12 (64 MiB cube)")
    elif name == "window1m":
        geo = make_params(4, 3, 1, 12, [12])
        spec = T.spec_window_1m()
        desc = dict(workload="window_1m_paper_cube", packets_per_window=spec.n_packets, sources=10_000,
                    planted_super_hosts=20, theta=1024, geometry="r=4, |RA|=3, |VA|=1, g=2^12, c=2^12 (128 MiB)")
    else:
        raise SystemExit(f"unknown workload {name}")
    return geo, spec, 1024, desc


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return d.get("hbm_gbs", 6400.0), "measured"
    return 6400.0, "fallback"


# ----------------------------------------------------------------------------- clocks

class ClockSampler:
    """Samples SM clock and clock-event reasons of one GPU while running.

    Uses NVML through pynvml when it imports, else polls nvidia-smi."""

    NAMES = {0x1: "gpu_idle", 0x2: "applications_clocks_setting", 0x4: "sw_power_cap", 0x8: "hw_slowdown",
             0x10: "sync_boost", 0x20: "sw_thermal_slowdown", 0x40: "hw_thermal_slowdown",
             0x80: "hw_power_brake_slowdown", 0x100: "display_clock_setting"}

    def __init__(self, index: int, period_s: float = 0.005):
        self.index, self.period = index, period_s
        self.samples, self.reasons = [], 0
        self.max_mhz = None
        self._stop = threading.Event()
        self._t = self._proc = None
        self.source = "nvml"
        try:
            import pynvml
            pynvml.nvmlInit()
            self.nv = pynvml
            self.h = pynvml.nvmlDeviceGetHandleByIndex(index)
            self.max_mhz = pynvml.nvmlDeviceGetMaxClockInfo(self.h, pynvml.NVML_CLOCK_SM)
        except Exception:  # noqa: BLE001
            self.nv, self.source = None, "nvidia-smi"

    def _run(self):
        while not self._stop.is_set():
            try:
                self.samples.append(self.nv.nvmlDeviceGetClockInfo(self.h, self.nv.NVML_CLOCK_SM))
                self.reasons |= self.nv.nvmlDeviceGetCurrentClocksEventReasons(self.h)
            except Exception:  # noqa: BLE001
                pass
            time.sleep(self.period)

    def __enter__(self):
        if self.nv is not None:
            self._t = threading.Thread(target=self._run, daemon=True)
            self._t.start()
        else:
            import subprocess
            try:
                self._proc = subprocess.Popen(
                    ["nvidia-smi", "-i", str(self.index),
                     "--query-gpu=clocks.sm,clocks.max.sm,clocks_event_reasons.active",
                     "--format=csv,noheader,nounits", "-lms", "20"],
                    stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            except OSError:
                self._proc = None
        return self

    def __exit__(self, *a):
        self._stop.set()
        if self._t:
            self._t.join()
        if self._proc is not None:
            time.sleep(0.05)
            self._proc.terminate()
            out, _ = self._proc.communicate(timeout=10)
            for line in out.splitlines():
                parts = [x.strip() for x in line.split(",")]
                if len(parts) < 3:
                    continue
                try:
                    self.samples.append(float(parts[0]))
                    self.max_mhz = float(parts[1])
                    self.reasons |= int(parts[2], 16)
                except ValueError:
                    pass

    def summary(self):
        names = [n for bit, n in self.NAMES.items() if self.reasons & bit]
        return {"sm_mhz": statistics.median(self.samples) if self.samples else None, "sm_max_mhz": self.max_mhz,
                "reasons": names, "samples": len(self.samples), "source": self.source}


# ----------------------------------------------------------------------------- distributed plumbing

def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def dist_init(world: int, backend: str):
    if world > 1:
        import torch.distributed as dist
        if not dist.is_initialized():
            dist.init_process_group(backend=backend)


def barrier(world: int):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def reduce_over_ranks(x: float, world: int, op: str, device=None) -> float:
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX if op == "max" else dist.ReduceOp.SUM)
    return float(t.item())


# ----------------------------------------------------------------------------- CPU oracle leg

def sweep_split_grid(C, base_tuning: dict, run_windows, lanes: int, world: int, dev):
    """The heavy split's grid for windows in flight: time `run_windows(count)` (windows through the
    lanes loop, streams joined to the current stream) with the split on 8/8, 6/8, 4/8, 3/8, 2/8 and
    1/8 of the SMs and set the fastest (the same on every rank).  Returns {split_blocks: ms/window}."""
    import torch
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    stream = torch.cuda.current_stream(dev)
    times = {}
    for eighths in (8, 6, 4, 3, 2, 1):
        C.set_tuning(**{**base_tuning, "split_blocks": 0 if eighths == 8 else max(1, sms * eighths // 8)})
        run_windows(2 * lanes)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        run_windows(4 * lanes)
        e1.record(stream)
        torch.cuda.synchronize()
        times[C.get_tuning()["split_blocks"]] = e0.elapsed_time(e1) / (4 * lanes)
    best = reduce_over_ranks(float(min(times, key=times.get)), world, "max", dev)
    C.set_tuning(**{**base_tuning, "split_blocks": int(best)})
    return times


def oracle_sample(geo, pairs: np.ndarray, theta: int, n_sample: int):
    """Time the plain CPU oracle (single thread) on the first n_sample packets + one detect."""
    from oracle import oracle as O
    O.build()
    sample = np.ascontiguousarray(pairs[:n_sample])
    t0 = time.perf_counter()
    cube = O.build_cube(geo, sample)
    t1 = time.perf_counter()
    res = O.detect(geo, cube, theta)
    t2 = time.perf_counter()
    return {"update_s": t1 - t0, "detect_s": t2 - t1, "packets": int(n_sample), "hosts": int(res["hosts"].size)}


def _cpu_model():
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                if line.startswith("model name"):
                    return line.split(":", 1)[1].strip()
    except OSError:
        pass
    return None


def oracle_threads_sample(geo, pairs: np.ndarray, n_sample: int, threads: int):
    """Time the oracle's OpenMP build (private cubes OR-ed) on the same sample; checks it against the
    single-threaded cube so the number belongs to a correct build."""
    from oracle import oracle as O
    sample = np.ascontiguousarray(pairs[:n_sample])
    t0 = time.perf_counter()
    cube = O.update_threads(geo, O.new_cube(geo), sample, threads)
    t1 = time.perf_counter()
    same = bool(np.array_equal(cube, O.build_cube(geo, sample)))
    return {"update_s": t1 - t0, "same_cube": same}


def cpu_baseline(geo, pairs, theta, n_sample):
    r = oracle_sample(geo, pairs, theta, n_sample)
    v = r["packets"] / (r["update_s"] + r["detect_s"]) / 1e9
    out = {"value": v, "unit": "Gpps", "cores": 1, "kind": "oracle",
           "sample": f"first {r['packets']} packets of the window (Alg. 1) + one full detect of that cube; "
                     f"update {r['update_s']:.3f} s, detect {r['detect_s']:.3f} s, single-threaded C",
           "update_gpps": r["packets"] / r["update_s"] / 1e9, "detect_ms": 1e3 * r["detect_s"],
           "cpu": _cpu_model(), "host_cores": os.cpu_count()}
    threads = max(1, min(os.cpu_count() or 1, 32))
    if threads > 1:
        t = oracle_threads_sample(geo, pairs, n_sample, threads)
        out["openmp"] = {"cores": threads, "update_gpps": r["packets"] / t["update_s"] / 1e9,
                         "value": r["packets"] / (t["update_s"] + r["detect_s"]) / 1e9, "unit": "Gpps",
                         "same_cube": t["same_cube"],
                         "sample": f"same packets on {threads} OpenMP threads, one private cube each, OR-ed; "
                                   f"update {t['update_s']:.3f} s, the single-threaded detect above"}
    return out


def run_reference(args):
    rank, world, local = dist_env()
    if rank != 0:
        return 0
    geo, spec, theta, desc = workload(args.workload, args.scale_shift)
    w = T.make_window(spec)
    n_sample = min(spec.n_packets, args.reference_sample)
    for _ in range(args.warmup):
        oracle_sample(geo, w.pairs, theta, n_sample)
    t_all = time.perf_counter()
    for _ in range(args.steps):
        oracle_sample(geo, w.pairs, theta, n_sample)
    elapsed = time.perf_counter() - t_all
    v = n_sample * args.steps / elapsed / 1e9
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "Gpps", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * elapsed / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u32", "data": "synthetic",
            "config": desc,
            "cpu_baseline": {"value": v, "unit": "Gpps", "cores": 1, "kind": "oracle",
                             "sample": f"each step: first {n_sample} packets of the window + one full detect",
                             "cpu": _cpu_model()},
            "e2e": {"value": v, "unit": "Gpps", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ----------------------------------------------------------------------------- GPU leg

def source_digest(rel: str) -> str:
    import hashlib
    with open(os.path.join(ROOT, rel), "rb") as f:
        return hashlib.sha256(f.read()).hexdigest()[:16]


def load_traffic(workload_name: str, path: str):
    """DRAM bytes of one window's update from the committed ncu summary, or None when the summary is
    missing or any kernel source it lists has changed since the counters were taken."""
    p = os.path.join(ROOT, "profiles", f"update_{path}_{workload_name}.json")
    if not os.path.exists(p):
        return None
    with open(p) as f:
        d = json.load(f)
    srcs = d.get("sources")
    if not srcs:
        return None
    for rel, digest in srcs.items():
        if not os.path.exists(os.path.join(ROOT, rel)) or source_digest(rel) != digest:
            return None
    return d.get("dram_bytes_per_launch")


def detect_only(args, C, cube, ws, out, info, theta, stream, hosts):
    """The window's detect alone on its cube, the packets freed by the caller: a full-size detect
    with a device footprint of one cube and one workspace (for profiling the detect kernels)."""
    import torch
    torch.cuda.empty_cache()
    ms = []
    for _ in range(max(args.steps, 1)):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        cube.detect_async(theta, ws, out, info)
        e1.record(stream)
        torch.cuda.synchronize()
        ms.append(e0.elapsed_time(e1))
    h2, inf = C.hosts_from_device(out, info)
    assert inf["status"] == C.OK and np.array_equal(h2["ip"], hosts["ip"]), inf
    g = cube.geometry
    n_arr = g["n_ra"] + g["n_va"]
    zc_t = torch.empty((1 << g["r"]) * n_arr * max(1 << c for c in g["cbn"][:n_arr]), dtype=torch.int16,
                       device=stream.device)
    za_t = torch.empty(1 << g["r"], n_arr, dtype=torch.int64, device=stream.device)
    eps_t = torch.empty(1 << g["r"], dtype=torch.float64, device=stream.device)
    zmax_t = torch.empty(1 << g["r"], dtype=torch.int64, device=stream.device)
    zc_ms = []
    for _ in range(max(args.steps, 1)):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        st = C.lib().cbaa_column_stats(cube.handle, theta, zc_t.data_ptr(), za_t.data_ptr(), eps_t.data_ptr(),
                                       zmax_t.data_ptr(), stream.cuda_stream)
        e1.record(stream)
        assert st == 0, st
        torch.cuda.synchronize()
        zc_ms.append(e0.elapsed_time(e1))
    print(json.dumps({"detect_only": True, "hosts": int(h2.size), "detect_ms_p50": float(np.median(ms)),
                      "column_stats_ms_p50": float(np.median(zc_ms)),
                      "device_bytes": int(torch.cuda.memory_allocated())}))
    return 0


def run_cbaa(args):
    import torch
    from paper_1901_06207_b300 import cbaa as C

    rank, world, local = dist_env()
    assert torch.cuda.is_available(), "the CBAA path runs on a CUDA device only"
    torch.cuda.set_device(local)
    dist_init(world, "nccl")
    dev = torch.device("cuda", local)
    geo, spec0, theta, desc = workload(args.workload, args.scale_shift)
    spec = spec0 if rank == 0 else T.TrafficSpec(**{**spec0.__dict__, "seed": spec0.seed + 0x100 * rank})
    w = T.make_window(spec)
    n = w.pairs.shape[0]
    pairs_dev = torch.from_numpy(w.pairs.view(np.int32)).to(dev)
    pairs_pin = torch.from_numpy(w.pairs.view(np.int32)).pin_memory()
    stream = torch.cuda.current_stream(dev)

    cube = C.Cube(geo, device=dev)
    ws = C.Workspace(geo, max_candidates=1 << 18, device=dev)
    from paper_1901_06207_b300 import autotune
    if args.update == "auto":
        tuned = autotune.tune_update(geo, pairs_dev, device=dev, use_cache=False)
        path = tuned["path"]
    else:
        tuned, path = None, args.update            # library default shapes, or --tuning
        if args.tuning:
            C.set_tuning(**json.loads(args.tuning))
    uws = C.UpdateWorkspace(geo, args.workspace_packets or n, device=dev) if path == "binned" else None
    cap = 1 << 16
    out = torch.zeros(4 * cap, dtype=torch.int32, device=dev)
    info = torch.zeros(8, dtype=torch.int32, device=dev)
    # update (direct: 1 kernel; binned: count, scan, scatter, apply) | detect: zero counts, eps/zmax,
    # hot lists, |RA|-1 joins, rank sort, sort/status
    pass_n = min(n, args.workspace_packets or n) if uws is not None else n
    kernels_per_step = -(-n // pass_n) * update_kernels(uws is not None, C.get_tuning(), pass_n) + \
        detect_kernels(geo)

    def do_update(c=None, src=None, u=None, assign=False):
        """assign: the cube becomes this window's bits alone (no reset before)."""
        c = cube if c is None else c
        src = pairs_dev if src is None else src
        u = uws if u is None else u
        if u is not None:
            c.update_binned(src, u, assign=assign)
        else:
            if assign:
                c.reset()
            c.update(src)

    # Windows in flight on `lanes` lanes, as a deployed detector runs them when
    # windows close faster than one window's update and detect take: lane j
    # owns a stream, a cube, an update workspace, a detect workspace, its
    # outputs and its own resident packet buffer; window k runs on lane
    # k mod L as an assigning update (the lane's previous window discarded:
    # the split's blocks zero the cube, no reset) and a detect, in stream
    # order, so that different windows' kernels overlap (one window's heavy
    # split beside another's residual kernels and a third's detect).  Every
    # window is fully updated and detected.
    L = max(2, args.lanes)
    lane_cube = [cube] + [C.Cube(geo, device=dev) for _ in range(L - 1)]
    lane_uws = [uws] + [C.UpdateWorkspace(geo, args.workspace_packets or n, device=dev) if uws is not None else None
                        for _ in range(L - 1)]
    lane_ws = [ws] + [C.Workspace(geo, max_candidates=1 << 18, device=dev) for _ in range(L - 1)]
    lane_out = [out] + [torch.zeros(4 * cap, dtype=torch.int32, device=dev) for _ in range(L - 1)]
    lane_info = [info] + [torch.zeros(8, dtype=torch.int32, device=dev) for _ in range(L - 1)]
    lane_pairs = [pairs_dev] + [pairs_dev.clone() for _ in range(L - 1)]
    lane_stream = [torch.cuda.Stream(dev) for _ in range(L)]
    lane_fresh = [True] * L

    def piped_step(k):
        b = k % L
        lane_fresh[b] = False
        with torch.cuda.stream(lane_stream[b]):
            do_update(lane_cube[b], lane_pairs[b], lane_uws[b], assign=True)
            lane_cube[b].detect_async(theta, lane_ws[b], lane_out[b], lane_info[b])

    def join_streams():
        for su in lane_stream:
            stream.wait_stream(su)

    def step(ev=None):
        cube.reset()
        if ev is not None:
            ev[0].record(stream)
        do_update()
        if ev is not None:
            ev[1].record(stream)
        cube.detect_async(theta, ws, out, info)
        if ev is not None:
            ev[2].record(stream)

    for _ in range(max(args.warmup, 0)):
        step()
    torch.cuda.synchronize()
    hosts, inf = C.hosts_from_device(out, info)
    assert inf["status"] == C.OK, inf
    if args.detect_only:
        pairs_dev = pairs_pin = uws = None            # the packets and the second buffers freed
        lane_cube = lane_ws = lane_out = lane_info = lane_pairs = lane_uws = None
        return detect_only(args, C, cube, ws, out, info, theta, stream, hosts)

    # L2 RED.OR roof on a buffer the size of the cube (the update kernel's bound)
    red_buf = torch.empty(cube.nbytes // 4, dtype=torch.int32, device=dev)
    n_ops = 4 * n
    red_rates = []
    for rep in range(4):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        st = C.lib().cbaa_bench_red_or(red_buf.data_ptr(), red_buf.numel(), n_ops, rep, stream.cuda_stream)
        e1.record(stream)
        assert st == 0, st
        torch.cuda.synchronize()
        if rep:
            red_rates.append(n_ops / (e0.elapsed_time(e1) * 1e-3) / 1e9)
    red_peak = max(red_rates)
    del red_buf

    # the direct RED.OR update on the same window, for comparison with the chosen path
    direct_ms = []
    for rep in range(4):
        cube.reset()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        cube.update(pairs_dev)
        e1.record(stream)
        torch.cuda.synchronize()
        if rep:
            direct_ms.append(e0.elapsed_time(e1))

    # serial steps, one window at a time: the update / detect split of a window
    n_serial = max(3, min(args.steps, 50))
    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in range(n_serial)]
    s0, s1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    s0.record(stream)
    for k in range(n_serial):
        step(evs[k])
    s1.record(stream)
    torch.cuda.synchronize()
    serial_ms = s0.elapsed_time(s1) / n_serial
    upd_ms = [e[0].elapsed_time(e[1]) for e in evs]
    det_ms = [e[1].elapsed_time(e[2]) for e in evs]
    hosts, inf = C.hosts_from_device(out, info)
    assert inf["status"] == C.OK, inf

    # detect end to end on the last window's cube: window close -> sorted host list in host memory
    # through the synchronous C call (cbaa_detect: enqueue, wait, copy the list back)
    det_sync_ms = []
    for rep in range(21):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        hs = cube.detect(theta, ws=ws, cap=cap)
        if rep:
            det_sync_ms.append(1e3 * (time.perf_counter() - t0))
    assert hs.size == inf["n_hosts"], (hs.size, inf)
    # the detect's streaming pass alone (Eq. 1 zero counts, Thm. 1 eps, Zmax: reads the cube once)
    n_arr = geo["n_ra"] + geo["n_va"]
    zc_t = torch.empty((1 << geo["r"]) * n_arr * max(1 << c for c in geo["cbn"][:n_arr]), dtype=torch.int16,
                       device=dev)
    za_t = torch.empty(1 << geo["r"], n_arr, dtype=torch.int64, device=dev)
    eps_t = torch.empty(1 << geo["r"], dtype=torch.float64, device=dev)
    zmax_t = torch.empty(1 << geo["r"], dtype=torch.int64, device=dev)
    zc_ms = []
    for rep in range(11):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        st = C.lib().cbaa_column_stats(cube.handle, theta, zc_t.data_ptr(), za_t.data_ptr(), eps_t.data_ptr(),
                                       zmax_t.data_ptr(), stream.cuda_stream)
        e1.record(stream)
        assert st == 0, st
        torch.cuda.synchronize()
        if rep:
            zc_ms.append(e0.elapsed_time(e1))

    # The split's grid for windows in flight: the autotuner picks shapes for one window alone, where
    # one split block per SM is fastest; with windows in flight, a split on fewer SMs leaves the rest
    # to the other lanes' kernels.  A short sweep of the lanes loop picks the grid (results never
    # depend on it); the serial figures above keep one block per SM.
    serial_tuning = C.get_tuning()
    lanes_sweep = {}

    def run_windows(count):
        for su in lane_stream:
            su.wait_stream(stream)
        for k in range(count):
            piped_step(k)
        join_streams()

    if uws is not None and args.lanes_split_sweep:
        lanes_sweep = sweep_split_grid(C, serial_tuning, run_windows, L, world, dev)
    lanes_tuning = C.get_tuning()

    # timed region: windows in flight on the lanes
    for k in range(max(args.warmup, 0)):
        piped_step(k)
    join_streams()
    t_start, t_end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    barrier(world)
    torch.cuda.synchronize()
    with ClockSampler(local) as clocks:
        t_start.record(stream)
        for su in lane_stream:
            su.wait_stream(stream)
        for k in range(args.steps):
            piped_step(k)
        join_streams()
        t_end.record(stream)
        torch.cuda.synchronize()
    barrier(world)
    total_ms = t_start.elapsed_time(t_end)
    total_ms_max = reduce_over_ranks(total_ms, world, "max", dev)
    for b in (b for b in range(L) if not lane_fresh[b]):       # every lane that ran a window
        h2, inf2 = C.hosts_from_device(lane_out[b], lane_info[b])
        assert inf2["status"] == C.OK and inf2["n_hosts"] == inf["n_hosts"], (inf2, inf)
    packets_all = reduce_over_ranks(float(n), world, "sum", dev)
    value = packets_all * args.steps / (total_ms_max * 1e-3) / 1e9
    C.set_tuning(**serial_tuning)

    # end to end through the public API with host buffers, windows pipelined
    # on three streams: H2D of window k+1's packets from pinned memory (s_copy)
    # overlaps window k's update (s_up) and detect + D2H of its host list and
    # info into pinned host memory (s_det).  Two device packet buffers, two
    # cubes (lanes 0 and 1's).
    e2e_steps = max(3, min(args.steps, 10))
    bufs, cubes2, ws2, out2, info2 = lane_pairs[:2], lane_cube[:2], lane_ws[:2], lane_out[:2], lane_info[:2]
    host_out = [torch.empty(4 * cap, dtype=torch.int32).pin_memory() for _ in range(2)]
    host_info = [torch.empty(8, dtype=torch.int32).pin_memory() for _ in range(2)]
    s_copy, s_up, s_det = torch.cuda.Stream(dev), torch.cuda.Stream(dev), torch.cuda.Stream(dev)
    buf_free, det_done = [None, None], [None, None]
    barrier(world)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for k in range(e2e_steps):
        b = k & 1
        with torch.cuda.stream(s_copy):
            if buf_free[b] is not None:
                s_copy.wait_event(buf_free[b])
            bufs[b].copy_(pairs_pin, non_blocking=True)
            copied = torch.cuda.Event()
            copied.record(s_copy)
        with torch.cuda.stream(s_up):
            s_up.wait_event(copied)
            if det_done[b] is None:
                cubes2[b].reset()
            else:
                s_up.wait_event(det_done[b])      # detected and already reset on s_det
            do_update(cubes2[b], bufs[b])
            up = torch.cuda.Event()
            up.record(s_up)
            buf_free[b] = up
        with torch.cuda.stream(s_det):
            s_det.wait_event(up)
            cubes2[b].detect_async(theta, ws2[b], out2[b], info2[b])
            host_out[b].copy_(out2[b], non_blocking=True)
            host_info[b].copy_(info2[b], non_blocking=True)
            cubes2[b].reset()
            det_done[b] = torch.cuda.Event()
            det_done[b].record(s_det)
    torch.cuda.synchronize()
    e2e_s = reduce_over_ranks(time.perf_counter() - t0, world, "max", dev)
    e2e_value = packets_all * e2e_steps / e2e_s / 1e9
    for b in range(2):
        h2, inf2 = C.hosts_from_device(host_out[b], host_info[b])
        assert inf2["status"] == C.OK and inf2["n_hosts"] == inf["n_hosts"], (inf2, inf)
    d2h = host_out[0].numel() * 4 + host_info[0].numel() * 4
    # the e2e bound: a plain pinned host-to-device copy of one window's packets, alone
    h2d_rates = []
    for rep in range(4):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        bufs[1].copy_(pairs_pin, non_blocking=True)
        e1.record(stream)
        torch.cuda.synchronize()
        if rep:
            h2d_rates.append(8 * n / (e0.elapsed_time(e1) * 1e-3) / 1e9)
    h2d_peak = max(h2d_rates)

    hbm_peak, hbm_src = measured_peaks()
    upd_s = statistics.mean(upd_ms) * 1e-3
    # the committed counters describe one pass over a whole default window
    traffic = None if (args.workspace_packets or args.scale_shift) else load_traffic(args.workload, path)
    line = {
        "metric": METRIC, "value": value, "unit": "Gpps", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms_max / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "u32", "data": "synthetic",
        "config": {**desc, "l2": f"inputs larger than L2: each step streams a {8 * n >> 20} MiB packet buffer (one per lane); "
                                 "each lane's 64 MiB cube fits L2 (the lanes' cubes together do not) and is re-zeroed every window",
                   "pipelining": f"{L} windows in flight: window k's assigning update (the lane's previous "
                                 "window discarded inside the update, no reset) and detect run in order on "
                                 f"lane k mod {L} (its own stream, cube, workspaces and resident packet buffer), "
                                 "overlapping the other lanes' windows",
                   "lanes": L,
                   "parallelism": "one window per rank" if world > 1 else "single GPU",
                   **({"update_workspace_packets": args.workspace_packets} if args.workspace_packets else {})},
        "serial": {"ms_per_window": serial_ms, "value": n / (serial_ms * 1e-3) / 1e9, "unit": "Gpps",
                   "steps": n_serial, "note": "one window at a time on one stream (reset, update, detect)"},
        "update_ms": statistics.mean(upd_ms), "update_gpps": n / upd_s / 1e9,
        "detect_ms": statistics.mean(det_ms), "detect_ms_p50": statistics.median(det_ms),
        "detect_sync_ms": {"p50": statistics.median(det_sync_ms), "max": max(det_sync_ms),
                           "what": "window close -> sorted host list in host memory (cbaa_detect, synchronous, "
                                   "through the Python binding)"},
        "detect_roofline": {"bound": "hbm", "kernel": "zero counts, eps and Zmax (cbaa_column_stats: memset, "
                                                      "k_zero_counts, k_eps_zmax)",
                            "achieved": cube.nbytes / (statistics.median(zc_ms) * 1e-3) / 1e9, "peak": hbm_peak,
                            "unit": "GB/s",
                            "frac": cube.nbytes / (statistics.median(zc_ms) * 1e-3) / 1e9 / hbm_peak,
                            "ms": statistics.median(zc_ms),
                            "note": "reads the cube once (M bytes); the cube is L2-resident after its update"},
        "hosts_detected": int(inf["n_hosts"]), "hot_columns": int(inf["n_hot"]),
        "update_path": path,
        "autotune": None if tuned is None else {
            "pick": tuned["path"], "tuning": tuned["tuning"], "best_ms": tuned["ms"],
            "worst_ms": tuned["worst_ms"], "candidates": tuned["candidates"]},
        "tuning": serial_tuning,
        "lanes_tuning": {"tuning": lanes_tuning,
                         "split_sweep_ms_per_window": {str(k): v for k, v in lanes_sweep.items()},
                         "note": "the timed region's shapes: the autotuner's pick with the split grid "
                                 "(split_blocks, 0 = one block per SM) chosen by timing the lanes loop"},
        "roofline": {"bound": "hbm", "kernel": f"update ({path}: " +
                     ({7: "heavy sample+hist+split (selection in each split block), residual count (with the "
                         "heavy bitmaps' expansion)+scan+scatter+apply",
                       4: "count+scan+scatter+apply", 1: "k_update"}[
                         update_kernels(uws is not None, C.get_tuning(), pass_n)]) + ")",
                     "achieved": 8 * n / upd_s / 1e9, "peak": hbm_peak, "unit": "GB/s",
                     "frac": 8 * n / upd_s / 1e9 / hbm_peak,
                     "peak_source": f"MEASURED_PEAKS.json hbm_gbs ({hbm_src})",
                     "units_per_launch": f"{n} packets x 8 B (the packet stream Alg. 1 must read)",
                     "traffic": traffic},
        "roofline_l2_atomic": {"bound": "l2_atomic", "kernel": "k_update (direct RED.OR design)",
                               "achieved": 4 * n / (statistics.mean(direct_ms) * 1e-3) / 1e9, "peak": red_peak,
                               "unit": "Gop/s",
                               "frac": 4 * n / (statistics.mean(direct_ms) * 1e-3) / 1e9 / red_peak,
                               "peak_source": "RED.OR microbenchmark on a cube-sized buffer, measured in this run",
                               "update_ms": statistics.mean(direct_ms),
                               "chosen_path": {
                                   "update_gpps": n / upd_s / 1e9, "roof_gpps": red_peak / 4,
                                   "ratio": n / upd_s / 1e9 / (red_peak / 4),
                                   "note": "the chosen update against the roof of one L2 RED.OR per bit "
                                           "(4 per packet); it issues about one reduction per cube word "
                                           "instead"}},
        "gpu_launches": kernels_per_step * args.steps,
        "clocks": clocks.summary(),
        "e2e": {"value": e2e_value, "unit": "Gpps", "h2d_bytes_per_step": 8 * n,
                "d2h_bytes_per_step": int(d2h), "steps": e2e_steps,
                "path": "pinned host packets -> H2D (stream 0) -> " +
                        ("cbaa_cube_update_binned" if uws is not None else "cbaa_cube_update") +
                        " (stream 1) -> cbaa_detect_async + D2H of the host list and info (stream 2), "
                        "windows pipelined",
                "roofline": {"bound": "h2d", "achieved": e2e_value * 8, "peak": h2d_peak, "unit": "GB/s",
                             "frac": e2e_value * 8 / h2d_peak,
                             "peak_source": "pinned host-to-device copy of one window's packets alone, "
                                            "measured in this run"}},
    }
    if rank == 0 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(geo, w.pairs, theta, min(n, args.cpu_sample or n))
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


def run_sharded(args):
    """Every rank is an edge router with its own 64M-packet window.  Window k's assigning update (its
    lane's previous window discarded inside the update) runs on lane k mod L (stream, cube, update
    workspace and packet buffer each) and overlaps the other lanes' updates and the earlier windows'
    global-server steps, which run on one stream in window order -- the
    all-to-all of sketch slices, the OR of the owned ones, their restoration, the device all-gather of
    every rank's host block and the merge by ip (ShardedDetector.enqueue: no host wait).  Timed with
    CUDA events, max over ranks; value = packets of all ranks / step time."""
    import torch
    from paper_1901_06207_b300 import cbaa as C
    from paper_1901_06207_b300.shard import ShardedDetector

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dist_init(world, "nccl")
    dev = torch.device("cuda", local)
    geo, spec0, theta, desc = workload("window64m")
    spec = T.TrafficSpec(**{**spec0.__dict__, "seed": spec0.seed + 0x100 * rank})
    w = T.make_window(spec)
    n = w.pairs.shape[0]
    pairs = torch.from_numpy(w.pairs.view(np.int32)).to(dev)
    if args.tuning:
        C.set_tuning(**json.loads(args.tuning))
    # Updates on `lanes` lanes (stream, cube, update workspace, packet buffer each), as in the plain
    # step; the exchange and restoration of every window stay on one stream, in window order (the
    # collectives of all ranks must be issued in one order), in the detector's two slots.
    L = max(2, args.lanes)
    cubes = [C.Cube(geo, device=dev) for _ in range(L)]
    uwss = [C.UpdateWorkspace(geo, n, device=dev) for _ in range(L)]
    lane_pairs = [pairs] + [pairs.clone() for _ in range(L - 1)]
    det = ShardedDetector(geo, theta, rank, world, device=dev)
    stream = torch.cuda.current_stream(dev)
    s_ups, s_det = [torch.cuda.Stream(dev) for _ in range(L)], torch.cuda.Stream(dev)
    done = [None] * L

    def step(k):
        b = k % L
        su = s_ups[b]
        with torch.cuda.stream(su):
            if done[b] is not None:
                su.wait_event(done[b])            # its previous window's exchange has read the cube
            cubes[b].update_binned(lane_pairs[b], uwss[b], assign=True)     # no reset: the update replaces it
            up = torch.cuda.Event()
            up.record(su)
        with torch.cuda.stream(s_det):
            s_det.wait_event(up)
            det.enqueue(cubes[b], k & 1)
            done[b] = torch.cuda.Event()
            done[b].record(s_det)

    def join():
        for su in s_ups:
            stream.wait_stream(su)
        stream.wait_stream(s_det)

    for su in s_ups:
        su.wait_stream(stream)
    s_det.wait_stream(stream)
    for k in range(max(args.warmup, 3)):
        step(k)
    join()
    torch.cuda.synchronize()

    def run_windows(count):
        for su in s_ups:
            su.wait_stream(stream)
        s_det.wait_stream(stream)
        for k in range(count):
            step(k)
        join()

    split_sweep = sweep_split_grid(C, C.get_tuning(), run_windows, L, world, dev) if args.lanes_split_sweep else {}
    steps = max(1, min(args.steps, 200))
    t_start, t_end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    barrier(world)
    torch.cuda.synchronize()
    with ClockSampler(local) as clocks:
        t_start.record(stream)
        for su in s_ups:
            su.wait_stream(stream)
        s_det.wait_stream(stream)
        for k in range(steps):
            step(k)
        join()
        t_end.record(stream)
        torch.cuda.synchronize()
    barrier(world)
    ms = reduce_over_ranks(t_start.elapsed_time(t_end), world, "max", dev)
    hosts, info = det.result((steps - 1) & 1)
    assert info["status"] == C.OK, info
    packets_all = reduce_over_ranks(float(n), world, "sum", dev)
    value = packets_all * steps / (ms * 1e-3) / 1e9
    words = C.cube_bytes(geo) // 4
    line = {"metric": METRIC, "value": value, "unit": "Gpps", "n_gpus": world, "steps": steps,
            "warmup": args.warmup, "ms_per_step": ms / steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u32", "data": "synthetic",
            "config": {**desc, "workload": "sharded_64m_per_rank",
                       "step": f"window k's assigning update on lane k mod {L} (its own stream, cube, update "
                               "workspace and packet buffer; the split's grid from a timed sweep) overlap the "
                               "other lanes' updates and the earlier "
                               "windows' all-to-all of sketch slices, OR of the owned ones, restoration, device "
                               "all-gather of the host blocks and merge by ip (one exchange stream, window "
                               "order); no host wait",
                       "lanes": L,
                       "parallelism": f"{world} ranks, sketches split {1 << geo['r']} / {world}"},
            "tuning": C.get_tuning(),
            "split_sweep_ms_per_window": {str(k): v for k, v in split_sweep.items()},
            "all_to_all_bytes_per_rank": {"sent": 4 * words * (world - 1) // world,
                                          "received": 4 * words * (world - 1) // world},
            "hosts_detected": int(hosts.size),
            "gpu_launches": steps * (update_kernels(True, C.get_tuning(), n) + detect_kernels(geo) + 2 +
                                     (1 if world > 1 else 0)),
            "clocks": clocks.summary()}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


def eq2_eq3(detected, ips, cnt, theta):
    """FNR and FPR of Section V.B (Eq. 2, Eq. 3): H = hosts with >= theta peers; false positives are
    detected addresses with fewer than theta peers (0 for addresses never seen); both over |H|."""
    card = dict(zip(ips.tolist(), cnt.tolist()))
    H = {ip for ip, c in card.items() if c >= theta}
    D = set(np.asarray(detected).tolist())
    fp = sum(1 for ip in D if card.get(ip, 0) < theta)
    return len(H - D) / max(1, len(H)), fp / max(1, len(H)), len(H)


def run_learned(args):
    """The learned estimator at its workload: windows of the 64M shape at 256M packets (2^24-host pool) in
    a cube 4x undersized in columns (r=6, 3+1, g=2^10, c=2^11: about 1.3 flows per row of a column, eps
    about 0.3), theta = 1024, candidates restored at the looser bound 0.8 theta.  Trained on 10^6 samples
    of one training window (seed 0xC0FFEE41): its candidates plus present sources stratified by octave of
    cardinality; scored on the held-out window 0xC0FFEE40 by Eq. 2 / Eq. 3 for Thm. 2 alone and for the
    learned decision, without and with a threshold margin chosen on the training window's candidates.
    `--learned-size scaled` keeps theta and the column load at a quarter of the traffic (64M packets,
    r=4).  Exact cardinalities are counted on the device (torch.unique of the pairs): measurement, not the
    detector's path."""
    import torch
    from paper_1901_06207_b300 import cbaa as C
    from paper_1901_06207_b300 import learned as L
    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dist_init(world, "nccl")
    dev = torch.device("cuda", local)
    full = args.learned_size == "full"
    geo = C.make_params(6 if full else 4, 3, 1, 10, [11])
    spec = T.spec_window_256m if full else (lambda seed: T.spec_window_64m(seed=seed))
    theta = 1024
    cand_theta = int(0.8 * theta)
    n_samples = 10 ** 6

    def exact(pairs):
        key = ((pairs[:, 0].to(torch.int64) & 0xFFFFFFFF) << 32) | (pairs[:, 1].to(torch.int64) & 0xFFFFFFFF)
        src = (torch.unique(key) >> 32) & 0xFFFFFFFF
        del key
        ips, cnt = torch.unique_consecutive(src, return_counts=True)
        ips, cnt = ips.cpu().numpy().astype(np.uint32), cnt.cpu().numpy().astype(np.int64)
        order = np.argsort(ips, kind="stable")      # int64 keys of sources >= 2^31 sort first: unsigned order
        return ips[order], cnt[order]

    def window(seed):
        t0 = time.perf_counter()
        w = T.make_window(spec(seed))
        gen_s = time.perf_counter() - t0
        pairs = torch.from_numpy(w.pairs.view(np.int32)).to(dev)
        n = int(pairs.shape[0])
        del w
        cube = C.Cube(geo, device=dev)
        ws = C.UpdateWorkspace(geo, n, device=dev)
        cube.update_binned(pairs, ws)
        del ws
        ips, cnt = exact(pairs)
        del pairs
        torch.cuda.empty_cache()
        cand = cube.detect(cand_theta, ws=C.Workspace(geo, max_candidates=1 << 20, device=dev), cap=1 << 20)
        cand = cand["ip"].astype(np.uint32)
        pos = np.minimum(np.searchsorted(ips, cand), ips.size - 1)
        truth = np.where(ips[pos] == cand, cnt[pos], 0)
        return dict(cube=cube, cand=cand, truth=truth, ips=ips, cnt=cnt, n=n, gen_s=gen_s)

    def as_dev(ips):
        return torch.from_numpy(np.ascontiguousarray(ips, dtype=np.uint32).view(np.int32)).to(dev)

    tr = window(0xC0FFEE41)
    sel_ips, sel_cnt = L.LearnedEstimator.training_set(tr["cand"], tr["truth"], tr["ips"], tr["cnt"], n_samples)
    X = L.features(tr["cube"], theta, as_dev(sel_ips))
    t = L.LearnedEstimator.target(X, torch.from_numpy(sel_cnt.astype(np.float32)).to(dev))
    net = L.LearnedEstimator(device=dev, seed=7)
    epochs, batch = 30, 1 << 14
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    losses = net.train(X, t, epochs=epochs, batch=batch, lr=3e-3)
    torch.cuda.synchronize()
    train_s = time.perf_counter() - t0
    # the threshold margin, chosen on the training window's candidates (the population it decides on)
    Xc = L.features(tr["cube"], theta, as_dev(tr["cand"]))
    card_tr, _ = net.decide(net.predict(Xc), Xc, geo["log2_g"], theta)
    card_tr = card_tr.cpu().numpy()
    factor = L.LearnedEstimator.choose_threshold(card_tr, tr["truth"], theta)
    fnr_cap = 0.02
    factor_cap = L.LearnedEstimator.choose_threshold(card_tr, tr["truth"], theta, max_fnr=fnr_cap)
    train_info = {"window_packets": tr["n"], "candidates": int(tr["cand"].size),
                  "phantom_candidates": int((tr["truth"] == 0).sum()), "samples": int(sel_ips.size),
                  "present_sources": int(tr["ips"].size), "generation_s": tr["gen_s"]}
    del tr, X, t, Xc, card_tr
    torch.cuda.empty_cache()
    te = window(0xC0FFEE40)
    # the gradient + Adam kernels alone, on one batch, CUDA events
    xb = L.features(te["cube"], theta, as_dev(te["ips"][:batch]))
    tb = L.LearnedEstimator.target(xb, torch.from_numpy(te["cnt"][:batch].astype(np.float32)).to(dev))
    probe = L.LearnedEstimator(device=dev, seed=8)
    stream = torch.cuda.current_stream(dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    for _ in range(3):
        probe.loss_grad(xb, tb, scale=1.0 / batch)
        probe.adam(lr=1e-6)
    reps = 200
    e0.record(stream)
    for _ in range(reps):
        probe.loss_grad(xb, tb, scale=1.0 / batch)
        probe.adam(lr=1e-6)
    e1.record(stream)
    torch.cuda.synchronize()
    step_ms = e0.elapsed_time(e1) / reps
    # inference on the held-out candidates: features, forward, decision
    cand_dev = as_dev(te["cand"])
    for _ in range(3):
        Xte = L.features(te["cube"], theta, cand_dev)
        card, dec = net.decide(net.predict(Xte), Xte, geo["log2_g"], theta)
    e0.record(stream)
    for _ in range(20):
        Xte = L.features(te["cube"], theta, cand_dev)
        card, dec = net.decide(net.predict(Xte), Xte, geo["log2_g"], theta)
    e1.record(stream)
    torch.cuda.synchronize()
    infer_ms = e0.elapsed_time(e1) / 20
    card = card.cpu().numpy().astype(np.float64)
    plain = te["cube"].detect(theta)["ip"]
    fnr_p, fpr_p, nH = eq2_eq3(plain, te["ips"], te["cnt"], theta)
    fnr_l, fpr_l, _ = eq2_eq3(te["cand"][card >= theta], te["ips"], te["cnt"], theta)
    fnr_m, fpr_m, _ = eq2_eq3(te["cand"][card >= factor * theta], te["ips"], te["cnt"], theta)
    fnr_c, fpr_c, _ = eq2_eq3(te["cand"][card >= factor_cap * theta], te["ips"], te["cnt"], theta)
    flop_per_sample = 3 * 2 * (16 * 64 + 64 * 64 + 64)          # forward + backward multiply-adds, x2 flops
    achieved = flop_per_sample * batch / (step_ms * 1e-3)
    peak_fp32 = 148 * 128 * 2 * 2.032e9                          # SMs x FP32 lanes x FMA x max clock
    work = ("learned_undersized_256m", "r=6, |RA|=3, |VA|=1, g=2^10, c=2^11 (64 MiB, 4x undersized)") if full else \
        ("learned_undersized_64m", "r=4, |RA|=3, |VA|=1, g=2^10, c=2^11 (16 MiB, the same column load)")
    line = {"metric": "learned estimator: FNR + FPR (Eq. 2, Eq. 3) on a held-out window of the undersized cube",
            "value": fnr_m + fpr_m, "unit": "fraction of |H|", "n_gpus": world, "steps": epochs, "warmup": 0,
            "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "bf16 weights, fp32",
            "data": "synthetic",
            "config": {"workload": work[0], "geometry": work[1], "packets_per_window": te["n"], "theta": theta,
                       "candidates": "restored at 0.8 theta", "train_seed": "0xC0FFEE41", "test_seed": "0xC0FFEE40",
                       "network": "16-64-64-1, residual on ln(1 + Thm. 2 estimate)",
                       "training_set": "the training window's candidates + present sources stratified by octave"},
            "hosts_H": nH, "thm2": {"fnr": fnr_p, "fpr": fpr_p},
            "learned": {"fnr": fnr_l, "fpr": fpr_l},
            "learned_margin": {"fnr": fnr_m, "fpr": fpr_m, "threshold_factor": factor,
                               "chosen": "min FNR + FPR on the training window's candidates"},
            "learned_fnr_cap": {"fnr": fnr_c, "fpr": fpr_c, "threshold_factor": factor_cap,
                                "chosen": f"largest factor with FNR <= {fnr_cap} on the training window's candidates"},
            "train": {**train_info, "epochs": epochs, "batch": batch, "seconds_api": train_s,
                      "loss_first_last": [losses[0], losses[-1]]},
            "candidates_test": int(te["cand"].size), "phantom_candidates_test": int((te["truth"] == 0).sum()),
            "step_ms_batch": step_ms, "train_samples_per_s": batch / (step_ms * 1e-3),
            "inference_ms_all_candidates": infer_ms,
            "inference_ns_per_candidate": infer_ms * 1e6 / max(1, te["cand"].size),
            "roofline": {"bound": "alu", "kernel": "cbaa_mlp_grad + cbaa_mlp_adam (one batch)",
                         "achieved": achieved / 1e12, "peak": peak_fp32 / 1e12, "unit": "TFLOP/s",
                         "frac": achieved / peak_fp32,
                         "peak_source": "148 SMs x 128 FP32 lanes x 2 x 2032 MHz (nominal, CUDA cores)"},
            "gpu_launches": reps * 2}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


def _router_window_job(args):
    seed, n_routers = args
    spec = T.spec_window_64m(seed=seed, scale_shift=2)
    pairs, counts, _ = T.router_window(spec, n_routers)
    return pairs, counts


def make_router_windows(n_windows: int, n_routers: int, seed0: int = 0xC0FFEE20):
    """16M-packet windows (the 64M window's shape scaled by 1/4) split over routers, in a spawn pool."""
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    with ctx.Pool(min(n_windows, max(1, (os.cpu_count() or 2) // 2))) as pool:
        return pool.map(_router_window_job, [(seed0 + w, n_routers) for w in range(n_windows)])


def run_batched(args):
    """Batched router windows: one CUDA graph replays every window (update pass over all router cubes,
    OR-merge, detect); the plain single-cube path on the same windows is timed beside it."""
    rank, world, local = dist_env()
    wins = make_router_windows(args.windows, args.routers, 0xC0FFEE20 + 0x1000 * rank)   # before CUDA init
    import torch
    from paper_1901_06207_b300 import cbaa as C
    from paper_1901_06207_b300.batch import RouterWindows
    torch.cuda.set_device(local)
    dist_init(world, "nccl")
    dev = torch.device("cuda", local)
    geo = C.make_params(5, 3, 1, 10, [12])
    theta, R = 1024, args.routers
    n_per = [int(c.sum()) for _, c in wins]
    dev_w, flat = [], []
    for pairs, counts in wins:
        p = torch.from_numpy(pairs.view(np.int32)).to(dev)
        flat.append(p)
        b = np.concatenate([[0], np.cumsum(counts)])
        dev_w.append([p[b[j]:b[j + 1]] if counts[j] else None for j in range(R)])
    rw = RouterWindows(geo, R, theta, max_pairs=max(n_per), n_windows=len(wins), device=dev)
    tiling = rw.tune(dev_w)
    rw.capture(dev_w)
    stream = torch.cuda.current_stream(dev)
    for _ in range(max(args.warmup, 1)):
        rw.replay()
    torch.cuda.synchronize()
    res = rw.results()
    assert all(inf["status"] == C.OK for _, inf in res), [inf for _, inf in res]

    def timed(fn, k):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        barrier(world)
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(k):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return reduce_over_ranks(e0.elapsed_time(e1), world, "max", dev)

    steps = max(1, args.steps)
    with ClockSampler(local) as clocks:
        ms = timed(rw.replay, steps)
    total_packets = reduce_over_ranks(float(sum(n_per)), world, "sum", dev)
    value = total_packets * steps / (ms * 1e-3) / 1e9

    # the plain single-cube path on the same windows: one cube, partitioned update of the whole
    # window, detect; eager launches, no routers, no graph
    cube = C.Cube(geo, device=dev)
    ws = C.Workspace(geo, device=dev)
    uws = C.UpdateWorkspace(geo, max(n_per), device=dev)
    out = torch.zeros(4 * rw.cap, dtype=torch.int32, device=dev)
    info = torch.zeros(8, dtype=torch.int32, device=dev)

    def plain():
        for p in flat:
            cube.reset()
            cube.update_binned(p, uws)
            cube.detect_async(theta, ws, out, info)

    plain()
    plain_ms = timed(plain, steps)
    hosts_last, _ = C.hosts_from_device(out, info)
    assert np.array_equal(hosts_last, res[-1][0]), "plain and batched host lists differ"
    plain_value = total_packets * steps / (plain_ms * 1e-3) / 1e9

    # the OR merge of Section III.C alone (a6): the 8 router cubes of the last window into a global cube,
    # as the graph does it (global = OR of the routers: every router cube read, the global cube written);
    # beside it the merge into a global cube that keeps its bits (dst |= ..., dst read as well)
    merge_reps = 20
    merge_ms = timed(lambda: rw.globs[0].merge(rw.routers, assign=True), merge_reps) / merge_reps
    merge_bytes = (R + 1) * C.cube_bytes(geo)
    merge_or_ms = timed(lambda: rw.globs[0].merge(rw.routers), merge_reps) / merge_reps
    merge_or_bytes = (R + 2) * C.cube_bytes(geo)
    hbm_peak, hbm_src = measured_peaks()
    merge_gbs = merge_bytes / (merge_ms * 1e-3) / 1e9
    line = {"metric": METRIC, "value": value, "unit": "Gpps", "n_gpus": world, "steps": steps,
            "warmup": args.warmup, "ms_per_step": ms / steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "u32", "data": "synthetic",
            "config": {"workload": f"batched_{len(wins)}x16m_{R}_routers",
                       "windows": len(wins), "routers": R, "packets_per_window": n_per[0],
                       "router_loads": "lognormal(sigma=0.8) weights over a 5-tuple hash",
                       "geometry": "r=5, |RA|=3, |VA|=1, g=2^10, c=2^12 (64 MiB per cube)", "theta": theta,
                       "step": "one CUDA graph replay: per window reset the router cubes and global cube w mod 2, "
                               "one partitioned update pass over all routers that also ORs every word it flushes "
                               "into the global cube (the merge of Section III.C in the same pass), detect on a "
                               "side stream (overlapping the next window's router update)",
                       "l2": "inputs larger than L2 (2 GiB of packets per step)"},
            "window_ms": ms / steps / len(wins), "router_update_tiling": tiling,
            "plain_single_cube": {"value": plain_value, "unit": "Gpps", "window_ms": plain_ms / steps / len(wins),
                                  "path": "one cube, partitioned update of the whole window, detect, no graph"},
            "merge": {"ms": merge_ms, "sources": R, "bytes": merge_bytes, "call": "cbaa_cube_merge_assign",
                      "roofline": {"bound": "hbm", "kernel": "k_merge", "achieved": merge_gbs, "peak": hbm_peak,
                                   "unit": "GB/s", "frac": merge_gbs / hbm_peak,
                                   "peak_source": f"MEASURED_PEAKS.json hbm_gbs ({hbm_src})"},
                      "or_into": {"call": "cbaa_cube_merge", "ms": merge_or_ms, "bytes": merge_or_bytes,
                                  "frac": merge_or_bytes / (merge_or_ms * 1e-3) / 1e9 / hbm_peak}},
            "hosts_per_window": [int(i["n_hosts"]) for _, i in res],
            # a pass over several router cubes takes no heavy split; the merge is inside it
            "gpu_launches": steps * len(wins) * (update_kernels(True, {**C.get_tuning(), "heavy": 1}, 0) +
                                                 detect_kernels(geo)),
            "clocks": clocks.summary()}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


def serve_schedule(n_pool: int, rate_pps: float, horizon_s: float, seed: int = 0xC0FFEE30):
    """Batches (offset into the packet pool, size) and Poisson arrival times at rate_pps for horizon_s."""
    out, t, off, i = [], 0.0, 0, 0
    while t < horizon_s:
        u = T.rand_unit(seed, 11, 2, 2 * i)
        size = int(np.exp(np.log(1 << 16) + u[0] * (np.log(4 << 20) - np.log(1 << 16))))
        t += -np.log(max(u[1], 1e-12)) * size / rate_pps
        if off + size > n_pool:
            off = 0
        out.append((off, size, t))
        off += size
        i += 1
    return out


def run_serve(args):
    """Serving: uneven batches through the continuous-batching server into 1 s windows.  A paced run
    at the target rate gives window latency; an unpaced run gives the server's capacity."""
    rank, world, local = dist_env()
    import torch
    from paper_1901_06207_b300 import cbaa as C
    from paper_1901_06207_b300.serve import Server
    torch.cuda.set_device(local)
    dist_init(world, "nccl")
    dev = torch.device("cuda", local)
    geo = C.make_params(6, 3, 1, 10, [13])                        # 256 MiB cubes for ~200M-packet windows
    theta = 1024
    w = T.make_window(T.spec_window_64m(seed=0xC0FFEE30 + 0x100 * rank))
    pool = torch.from_numpy(w.pairs.view(np.int32)).pin_memory()
    n_pool = pool.shape[0]
    rate = args.serve_rate
    srv = Server(geo, theta, n_slots=4, slot_pairs=4 << 20, n_cubes=4, device=dev)

    def run(schedule, paced: bool):
        srv.results.clear()
        t0 = time.perf_counter()
        cur = 0
        for off, size, t_arr in schedule:
            win = int(t_arr // args.serve_window_s)
            if paced:
                while time.perf_counter() - t0 < t_arr:
                    srv.poll()
            if win != cur:
                srv.close(0, cur)
                cur = win
            srv.submit(0, win, pool[off:off + size], arrival_t=t0 + t_arr)
        srv.close(0, cur)
        res = srv.drain(timeout_s=300)
        torch.cuda.synchronize()
        return res, time.perf_counter() - t0

    warm = serve_schedule(n_pool, rate, 0.2 * args.serve_window_s, seed=0xC0FFEE31)
    run(warm, paced=False)
    paced_sched = serve_schedule(n_pool, rate, args.serve_windows * args.serve_window_s)
    with ClockSampler(local) as clocks:
        res_p, el_p = run(paced_sched, paced=True)
    lat = sorted(r.latency_s * 1e3 for r in res_p)
    cap_sched = serve_schedule(n_pool, rate, args.serve_windows * args.serve_window_s, seed=0xC0FFEE32)
    res_c, el_c = run(cap_sched, paced=False)
    pk_p = sum(r.packets for r in res_p)
    pk_c = sum(r.packets for r in res_c)
    cap_gpps = reduce_over_ranks(pk_c, world, "sum", dev) / reduce_over_ranks(el_c, world, "max", dev) / 1e9
    # the capacity's bound on this host: a plain pinned host-to-device copy of a slot's worth of pairs
    dst = torch.empty((4 << 20, 2), dtype=torch.int32, device=dev)
    stream = torch.cuda.current_stream(dev)
    h2d = []
    for rep in range(6):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        dst.copy_(pool[:4 << 20], non_blocking=True)
        e1.record(stream)
        torch.cuda.synchronize()
        if rep:
            h2d.append(dst.numel() * 4 / (e0.elapsed_time(e1) * 1e-3) / 1e9)
    h2d_gbs = max(h2d)
    line = {"metric": METRIC, "value": cap_gpps, "unit": "Gpps", "n_gpus": world, "steps": len(res_c),
            "warmup": 1, "ms_per_step": 1e3 * el_c / max(1, len(res_c)), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u32", "data": "synthetic",
            "config": {"workload": "serve_200mpps_1s_windows",
                       "batches": "log-uniform sizes in [64Ki, 4Mi] pairs cut from a 64M-packet window",
                       "arrivals": f"Poisson at {rate / 1e6:.0f} Mpps", "window_s": args.serve_window_s,
                       "geometry": "r=6, |RA|=3, |VA|=1, g=2^10, c=2^13 (256 MiB cubes)", "theta": theta,
                       "server": "4 staging slots of 4Mi pairs, 4 cube buffers, copy/compute/detect streams",
                       "value": "unpaced capacity: host batches -> H2D -> update -> windows -> host lists"},
            "paced": {"offered_mpps": rate / 1e6, "sustained_gpps": pk_p / el_p / 1e9, "windows": len(res_p),
                      "latency_ms_p50": lat[len(lat) // 2] if lat else None,
                      "latency_ms_p99": lat[min(len(lat) - 1, int(0.99 * len(lat)))] if lat else None,
                      "latency": "window close -> host list on the host"},
            "capacity": {"packets": pk_c, "seconds": el_c, "windows": len(res_c),
                         "roofline": {"bound": "h2d", "achieved": 8 * pk_c / el_c / 1e9, "peak": h2d_gbs,
                                      "unit": "GB/s", "frac": 8 * pk_c / el_c / 1e9 / h2d_gbs,
                                      "peak_source": "pinned host-to-device copy of 4Mi pairs alone, "
                                                     "measured in this run"}},
            "server_stats": dict(srv.stats),
            "hosts_per_window": [int(r.info["n_hosts"]) for r in res_p],
            "clocks": clocks.summary()}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=None,
                    help="timed steps (default 1000 windows for the window workloads on the GPU, 200 otherwise)")
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", choices=["cbaa", "reference"], default="cbaa")
    ap.add_argument("--workload", default="window64m",
                    choices=["window64m", "window1m", "batched", "serve", "sharded", "learned"])
    ap.add_argument("--serve-rate", type=float, default=2e8, help="serve workload: offered packets/s")
    ap.add_argument("--serve-window-s", type=float, default=1.0, help="serve workload: window length")
    ap.add_argument("--serve-windows", type=int, default=3, help="serve workload: windows per run")
    ap.add_argument("--update", default="auto", choices=["auto", "binned", "direct"],
                    help="Alg. 1 path: partitioned by cube tile (binned), RED.OR into the cube (direct), "
                         "or the autotuner's pick (auto)")
    ap.add_argument("--tuning", default="", help="with --update binned/direct: launch shapes as JSON, e.g. "
                                                 "'{\"scatter_shape\": 6, \"tile_kind\": 3}'")
    ap.add_argument("--windows", type=int, default=16, help="batched workload: windows per batch")
    ap.add_argument("--routers", type=int, default=8, help="batched workload: simulated edge routers")
    ap.add_argument("--reference-sample", type=int, default=4 << 20,
                    help="packets per CPU-oracle step (bounded sample of the window)")
    ap.add_argument("--cpu-sample", type=int, default=0,
                    help="packets of the window the cpu_baseline oracle run takes (0: the whole window)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--lanes", type=int, default=6,
                    help="cbaa workload: windows in flight in the timed loop (at least 2), each on its own stream "
                         "with its own cube, workspaces and packet buffer")
    ap.add_argument("--no-lanes-split-sweep", dest="lanes_split_sweep", action="store_false",
                    help="cbaa workload: keep the tuning's split grid in the timed region instead of timing "
                         "the lanes loop at 8/8 .. 1/8 of the SMs")
    ap.add_argument("--workspace-packets", type=int, default=0,
                    help="window workloads: size the update workspace for this many packets (0: the window); "
                         "fewer than a window makes the update run in several passes")
    ap.add_argument("--scale-shift", type=int, default=0,
                    help="window64m: the same window shape at 2^-k the packets and pool (small profiling cases)")
    ap.add_argument("--detect-only", action="store_true",
                    help="window workloads: after the warm-up, free the packets and time the detect alone "
                         "(a full-size detect in a small device footprint, for profiling)")
    ap.add_argument("--learned-size", default="full", choices=["full", "scaled"],
                    help="learned workload: 256M-packet windows (full) or 64M with the same column load")
    args = ap.parse_args()
    if args.steps is None:
        args.steps = 1000 if args.impl == "cbaa" and args.workload in ("window64m", "window1m") else 200
    if args.warmup < 3 and args.impl == "cbaa":
        print("warning: fewer than 3 warm-up steps", file=sys.stderr)
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "batched":
        return run_batched(args)
    if args.workload == "serve":
        return run_serve(args)
    if args.workload == "sharded":
        return run_sharded(args)
    if args.workload == "learned":
        return run_learned(args)
    return run_cbaa(args)


if __name__ == "__main__":
    sys.exit(main())
