"""Benchmark of the fused sea-ice labeler on GB300.

Default workload (one step = one pass of the whole labeling path over one
input): a full 10980 x 10980 uint8 RGB Sentinel-2-sized scene (seeded
synthetic: 200 Voronoi floes, 5-15 thin-cloud blobs, 3-8 shadow ellipses),
labelled into uint8 label codes with per-256x256-chip and per-scene class
counts.  The input (362 MB) is larger than L2 (129 MB).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl sil|reference]

Prints ONE JSON line.  ``value`` is Gpixel/s labelled (bit-exact with the
oracle), device-resident input, whole job over all ranks; ``e2e`` is the same
metric through the host-buffer entry point (pinned host image in, labels and
counts back, copies inside the timed region).  Under torchrun every rank
labels its own scene (weak scaling, no collective on the data path).
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

SIDE = 10980
CHIP = 256
# DRAM bytes (read + write) of one labeler launch on this workload, from an
# ncu capture of the current kernel (dram__bytes_read.sum +
# dram__bytes_write.sum); None whenever the kernel has changed since.
TRAFFIC_BYTES_PER_LAUNCH = (366.439424 + 91.333376) * 1e6
METRIC = "Gpixel/s labeled (bit-exact)"
UNIT = "Gpixel/s"


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clock / throttle samples taken while the timed region runs."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.samples = []
        self._stop = threading.Event()
        self._th = None
        self._t0 = self._t1 = None
        self._regions = {}

    def _run(self):
        while not self._stop.is_set():
            try:
                out = subprocess.run(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                      "--format=csv,noheader,nounits"], capture_output=True,
                                     text=True, timeout=5).stdout.strip()
                self.samples.append((time.monotonic(), out))
            except Exception:
                return
            self._stop.wait(0.05)

    def start(self):
        self._th = threading.Thread(target=self._run, daemon=True)
        self._th.start()

    def mark(self, t0, t1, name="timed"):
        self._regions[name] = (t0, t1)
        if name == "timed":
            self._t0, self._t1 = t0, t1

    def stop(self):
        self._stop.set()
        if self._th:
            self._th.join(timeout=10)

    def _rows(self):
        rows = []
        for t, line in self.samples:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9:
                rows.append((t, parts))
        return rows

    @staticmethod
    def _stats(inside):
        sm = sorted(float(r[1][1]) for r in inside)
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for _, p in inside:
            for n, v in zip(names, p[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        pw = [float(r[1][3]) for r in inside if r[1][3] not in ("", "[N/A]")]
        return {"sm_mhz": sm[len(sm) // 2], "sm_max_mhz": float(inside[0][1][2]),
                "power_w_max": max(pw) if pw else None, "samples": len(inside),
                "reasons": sorted(reasons)}

    def summary(self, name="timed"):
        """Clock statistics of the samples taken inside the named region
        (the nearest two, with a note, when the region is shorter than the
        sampling interval)."""
        rows = self._rows()
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no nvidia-smi samples"]}
        t0, t1 = self._regions.get(name, (None, None))
        inside = [r for r in rows if t0 is not None and t0 <= r[0] <= t1]
        note = []
        if not inside:
            mid = 0.5 * (t0 + t1) if t0 is not None else rows[-1][0]
            inside = sorted(rows, key=lambda r: abs(r[0] - mid))[:2]
            note.append("region shorter than the sampling interval; nearest samples")
        out = self._stats(inside)
        out["reasons"] = out["reasons"] + note
        return out


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def aggregate(elapsed_s: float, units: float, world: int, backend_group=None):
    """Max of elapsed over ranks, sum of units: the whole-job rate."""
    if world > 1:
        import torch
        import torch.distributed as dist
        dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
        t = torch.tensor([elapsed_s, units], dtype=torch.float64, device=dev)
        mx = t.clone()
        dist.all_reduce(mx, op=dist.ReduceOp.MAX)
        sm = t.clone()
        dist.all_reduce(sm, op=dist.ReduceOp.SUM)
        return float(mx[0]), float(sm[1])
    return elapsed_s, units


def cpu_baseline(img: np.ndarray, budget_s: float = 12.0, seed: int = 0):
    """The oracle as it stands, single thread, on whole chips of the scene
    (at least one) until budget_s of CPU time is spent; returns Gpixel/s and
    the sample."""
    import oracle
    gy, gx = -(-img.shape[0] // CHIP), -(-img.shape[1] // CHIP)
    rng = np.random.default_rng(seed)
    order = rng.permutation(gy * gx)
    px = 0
    n = 0
    t0 = time.perf_counter()
    for k in order:
        cy, cx = divmod(int(k), gx)
        crop = np.ascontiguousarray(img[cy * CHIP:(cy + 1) * CHIP, cx * CHIP:(cx + 1) * CHIP])
        oracle.label(crop)
        px += crop.shape[0] * crop.shape[1]
        n += 1
        if time.perf_counter() - t0 > budget_s:
            break
    dt = time.perf_counter() - t0
    return px / dt / 1e9, f"{n} random 256x256 chips of the scene ({px} px) in {dt:.1f} s"


def _chip_worker(task):
    """Pool worker: the oracle on whole chips of the shared scene until the
    budget is spent; returns (pixels, chips)."""
    name, shape, dtype, chips, budget_s = task
    from multiprocessing import shared_memory
    import oracle
    shm = shared_memory.SharedMemory(name=name)
    try:
        img = np.ndarray(shape, dtype=np.dtype(dtype), buffer=shm.buf)
        px, n = 0, 0
        t0 = time.perf_counter()
        for cy, cx in chips:
            crop = np.ascontiguousarray(img[cy * CHIP:(cy + 1) * CHIP, cx * CHIP:(cx + 1) * CHIP])
            oracle.label(crop)
            px += crop.shape[0] * crop.shape[1]
            n += 1
            if time.perf_counter() - t0 > budget_s:
                break
        del img, crop
    finally:
        shm.close()
    return px, n


def _worker_ready(_):
    import oracle  # noqa: F401  (load the library once per worker)
    return os.getpid()


class OraclePool:
    """The oracle, unchanged, run on every host core: one single-threaded
    worker process per core, each labelling its own random whole chips of the
    scene (shared memory, no copies).  Workers are spawned, never forked, so
    a CUDA context in the parent is not inherited."""

    def __init__(self, img: np.ndarray, cores: int | None = None):
        import multiprocessing as mp
        from multiprocessing import shared_memory
        self.cores = int(cores or len(os.sched_getaffinity(0)))
        self.shape = img.shape
        self.dtype = img.dtype.str  # uint8 RGB or uint16 reflectance
        self.shm = shared_memory.SharedMemory(create=True, size=img.nbytes)
        np.ndarray(img.shape, dtype=img.dtype, buffer=self.shm.buf)[...] = img
        self.pool = mp.get_context("spawn").Pool(self.cores)
        self.pool.map(_worker_ready, range(self.cores), chunksize=1)

    def run(self, budget_s: float, seed: int = 0):
        gy, gx = -(-self.shape[0] // CHIP), -(-self.shape[1] // CHIP)
        order = np.random.default_rng(seed).permutation(gy * gx)
        chips = [divmod(int(k), gx) for k in order]
        tasks = [(self.shm.name, self.shape, self.dtype, chips[i::self.cores], budget_s)
                 for i in range(self.cores)]
        t0 = time.perf_counter()
        res = self.pool.map(_chip_worker, tasks, chunksize=1)
        dt = time.perf_counter() - t0
        px, n = sum(r[0] for r in res), sum(r[1] for r in res)
        return px / dt / 1e9, (f"{n} random 256x256 chips of the scene ({px} px) on {self.cores} "
                               f"worker processes in {dt:.3f} s wall")

    def close(self):
        self.pool.close()
        self.pool.join()
        self.shm.close()
        self.shm.unlink()


def run_reference(args):
    """The oracle on the host cores (rank 0 only), same metric and workload."""
    ws, rank, local = _dist()
    if rank != 0:
        return 0
    import synth
    u16 = args.dtype == "u16"
    img, _ = synth.full_scene(1, SIDE, dtype=np.uint16 if u16 else np.uint8)
    times = []
    sample = ""
    per_step = args.ref_budget / max(1, args.steps + args.warmup)
    pool = OraclePool(img, args.cpu_cores or None)
    try:
        for i in range(args.warmup + args.steps):
            v, sample = pool.run(per_step, seed=i)
            if i >= args.warmup:
                times.append(v)
    finally:
        pool.close()
    value = float(len(times) / np.sum(1.0 / np.array(times))) if times else 0.0
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": (SIDE * SIDE / (value * 1e9) * 1e3) if value else None,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": args.dtype,
        "data": "synthetic",
        "config": {"workload": f"one {SIDE}x{SIDE} " + ("uint16 reflectance" if u16 else "uint8")
                               + f" RGB scene, chip {CHIP}, seed 1",
                   "l2": "input larger than L2"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": pool.cores, "kind": "oracle",
                         "sample": f"per step: {sample}"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))
    return 0


def run_sil(args):
    import torch
    ws, rank, local = _dist()
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    import paper_2403_13135_gb300 as sil
    import synth

    u16 = args.dtype == "u16"
    img, _ = synth.full_scene(1 + rank, SIDE, dtype=np.uint16 if u16 else np.uint8)
    H, W, _ = img.shape
    bpp = 6 if u16 else 3  # bytes per input pixel
    # uint16 images travel as int16 tensors (the same bytes)
    dev = torch.from_numpy(img.view(np.int16) if u16 else img).cuda()
    lab = torch.empty((H, W), dtype=torch.uint8, device="cuda")
    cnt = torch.empty(4, dtype=torch.int64, device="cuda")
    cc = torch.empty((-(-H // CHIP), -(-W // CHIP), 4), dtype=torch.int32, device="cuda")
    p = sil.params()
    stream = torch.cuda.current_stream()

    def step():
        sil.label(dev, p, out_labels=lab, out_counts=cnt, out_chip_counts=cc, chip_counts=True,
                  stream=stream)

    for _ in range(max(3, args.warmup)):
        step()
    torch.cuda.synchronize()

    sampler = ClockSampler(local)
    sampler.start()
    time.sleep(0.3)
    n_ev = args.steps
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(n_ev)]
    if ws > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    t0 = time.monotonic()
    start = torch.cuda.Event(enable_timing=True)
    end = torch.cuda.Event(enable_timing=True)
    start.record(stream)
    for i in range(args.steps):
        evs[i][0].record(stream)
        step()
        evs[i][1].record(stream)
    end.record(stream)
    torch.cuda.synchronize()
    t1 = time.monotonic()
    if ws > 1:
        torch.distributed.barrier()
    sampler.mark(t0, t1)
    # clock soak: the same step for at least args.soak seconds right after
    # the timed region, so that the clocks the timed steps ran at are
    # sampled many times even when the timed region is short
    ts0 = time.monotonic()
    n_soak = 0
    while time.monotonic() - ts0 < args.soak:
        for _ in range(200):
            step()
        n_soak += 200
        torch.cuda.synchronize()
    sampler.mark(ts0, time.monotonic(), "soak")
    time.sleep(0.2)
    sampler.stop()
    elapsed = start.elapsed_time(end) / 1e3
    per_launch = np.array([a.elapsed_time(b) for a, b in evs]) / 1e3
    el_max, units = aggregate(elapsed, float(H * W * args.steps), ws)
    value = units / el_max / 1e9

    # end to end through the host-buffer entry point (pinned host memory)
    himg = torch.from_numpy(img.view(np.uint8).reshape(H, W * bpp)).pin_memory()
    hlab = torch.empty((H, W), dtype=torch.uint8).pin_memory()
    hcnt = np.zeros(4, np.uint64)
    hcc = np.zeros(cc.shape, np.uint32)
    import ctypes
    e2e_steps = max(3, min(args.steps, args.e2e_steps))

    def e2e_step():
        sil.check(sil.sil_label_host(himg.data_ptr(), H, W, bpp * W, sil.SIL_U16 if u16 else sil.SIL_U8,
                                     ctypes.byref(p),
                                     hlab.data_ptr(), W, hcnt.ctypes.data, hcc.ctypes.data,
                                     ctypes.c_void_p(stream.cuda_stream)))

    for _ in range(2):
        e2e_step()
    if ws > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    te0 = time.perf_counter()
    for _ in range(e2e_steps):
        e2e_step()
    torch.cuda.synchronize()
    te = time.perf_counter() - te0
    te_max, e2e_units = aggregate(te, float(H * W * e2e_steps), ws)
    e2e_value = e2e_units / te_max / 1e9
    # result of the last device step agrees with the host-path result
    assert np.array_equal(cnt.cpu().numpy().astype(np.uint64), hcnt)

    peak, peak_kind = _peaks()
    alg_bytes = float(bpp + 1) * H * W + cc.numel() * 4 + 32
    avg_launch = float(per_launch.mean())
    achieved = alg_bytes / avg_launch / 1e9
    clocks = sampler.summary()
    soak = sampler.summary("soak")
    soak["steps"] = n_soak
    clocks["soak"] = soak
    if clocks.get("sm_mhz") and soak.get("sm_mhz"):
        # time x clock: the step's cycle count, comparable across clock states
        clocks["ms_per_step_x_soak_mhz"] = el_max / args.steps * 1e3 * soak["sm_mhz"]
    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": max(3, args.warmup), "ms_per_step": el_max / args.steps * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": args.dtype,
            "data": "synthetic",
            "config": {"workload": f"{SIDE}x{SIDE} " + ("uint16 reflectance" if u16 else "uint8")
                                   + f" RGB scene per GPU, chip {CHIP}, labels + per-chip + per-scene counts",
                       "l2": f"input ({H * W * bpp / 1e6:.0f} MB) larger than L2, no flush",
                       "parallelism": f"replicas{ws}"},
            "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": int(bpp * H * W),
                    "d2h_bytes_per_step": int(H * W + 32 + cc.numel() * 4)},
            "gpu_launches": int(args.steps),
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak,
                         # the committed DRAM figure is the uint8 scene's
                         "traffic": None if (u16 and args.traffic == TRAFFIC_BYTES_PER_LAUNCH) else args.traffic,
                         "peak_source": f"{peak_kind} hbm_gbs",
                         "alg_bytes_per_launch": alg_bytes,
                         "avg_launch_us": avg_launch * 1e6},
            "clocks": clocks,
        }
        if not args.no_cpu_baseline and ws == 1:  # rank 0 at N = 1 only
            pool = OraclePool(img, args.cpu_cores or None)
            try:
                v, sample = pool.run(args.cpu_budget)
            finally:
                pool.close()
            v1, sample1 = cpu_baseline(img, args.cpu_budget / 2)
            line["cpu_baseline"] = {"value": v, "unit": UNIT, "cores": pool.cores, "kind": "oracle",
                                    "sample": sample,
                                    "single_core": {"value": v1, "cores": 1, "sample": sample1}}
        print(json.dumps(line))
    if ws > 1:
        torch.distributed.destroy_process_group()
    return 0


def _time_cuda(fn, reps, stream):
    import torch
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(reps):
        fn()
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / 1e3 / reps


def run_batch(args):
    """512 uneven tiles (side in {128..2048}, aspect 1:1-1:2): one persistent
    launch through a captured graph (default and autotuned schedule) vs one
    sil_label launch per tile."""
    import torch
    import paper_2403_13135_gb300 as sil
    import synth
    scene, _ = synth.full_scene(1, SIDE)
    shapes = synth.uneven_tile_shapes(args.tiles)
    tiles, _ = synth.crop_tiles(scene, shapes, seed=0)
    npx = sum(t.shape[0] * t.shape[1] for t in tiles)
    dev = [torch.from_numpy(t).cuda() for t in tiles]
    labs = [torch.empty(t.shape[:2], dtype=torch.uint8, device="cuda") for t in tiles]
    cnts = [torch.empty(4, dtype=torch.int64, device="cuda") for _ in tiles]
    ccs = [torch.empty((-(-t.shape[0] // CHIP), -(-t.shape[1] // CHIP), 4), dtype=torch.int32,
                       device="cuda") for t in tiles]
    p = sil.params()
    stream = torch.cuda.current_stream()

    def per_tile():
        for d, l, c, cc in zip(dev, labs, cnts, ccs):
            sil.label(d, p, out_labels=l, out_counts=c, out_chip_counts=cc, chip_counts=True, stream=stream)

    ctx = sil.Context()
    arr = sil.make_tiles(dev, labs, cnts, ccs)
    batch = lambda: sil.label_batch(ctx, arr, len(tiles), sil.SIL_U8, p, stream)
    for _ in range(args.warmup):
        per_tile()
    t_tile = _time_cuda(per_tile, args.steps, stream)
    ref = [c.clone() for c in cnts]
    for _ in range(args.warmup):
        batch()
    t_batch = _time_cuda(batch, args.steps, stream)
    same = all(torch.equal(a, b) for a, b in zip(ref, cnts))
    best = sil.autotune(ctx, arr, len(tiles), sil.SIL_U8, p, stream)
    for _ in range(args.warmup):
        batch()
    t_tuned = _time_cuda(batch, args.steps, stream)
    print(json.dumps({
        "metric": METRIC, "config": {"workload": f"{len(tiles)} uneven tiles, {npx} px, chip {CHIP}"},
        "per_tile_launches": {"value": npx / t_tile / 1e9, "unit": UNIT, "ms": t_tile * 1e3},
        "batched_graph": {"value": npx / t_batch / 1e9, "unit": UNIT, "ms": t_batch * 1e3},
        "batched_autotuned": {"value": npx / t_tuned / 1e9, "unit": UNIT, "ms": t_tuned * 1e3,
                              "tuning": best},
        "speedup_vs_per_tile": t_tile / min(t_batch, t_tuned), "counts_identical": bool(same)}))
    ctx.close()
    return 0


def run_served(args):
    """Poisson stream of requests (90% square tiles, side U{256..4096}; 10%
    full scenes) from pinned host memory through the continuous-batching
    server; throughput and p50/p99 latency per arrival rate.  Label buffers
    come from a pinned pool; when the pool is empty the client waits for a
    completion before it submits (back-pressure), which the report counts."""
    import queue
    import torch
    import paper_2403_13135_gb300 as sil
    import synth
    scene, _ = synth.full_scene(1, SIDE)
    rng = np.random.default_rng(4)
    pool = []
    for i in range(24):
        s = int(rng.integers(256, 4097))
        y, x = (int(v) for v in rng.integers(0, SIDE - s + 1, 2))
        pool.append(torch.from_numpy(np.ascontiguousarray(scene[y:y + s, x:x + s])).pin_memory().numpy())
    big = torch.from_numpy(scene).pin_memory().numpy()
    lab_tiles = queue.Queue()
    for _ in range(args.label_pool):
        lab_tiles.put(torch.empty((4096, 4096), dtype=torch.uint8).pin_memory().numpy())
    lab_scenes = queue.Queue()
    for _ in range(max(2, args.label_pool // 16)):
        lab_scenes.put(torch.empty((SIDE, SIDE), dtype=torch.uint8).pin_memory().numpy())
    results = []
    for rate in [float(r) for r in args.rates.split(",")]:
        lat, svc, px = [], [], [0]
        stalls = 0
        pending = queue.Queue()
        with sil.Server(max_inflight=128, want_labels=True) as srv:
            def collector():
                while True:
                    item = pending.get()
                    if item is None:
                        return
                    rid, n, buf, q = item
                    r = srv.wait(rid, 600000)
                    lat.append(r["t_done_ms"] - r["t_submit_ms"])
                    svc.append(r["t_done_ms"] - r["t_admit_ms"])
                    px[0] += n
                    q.put(buf)
            th = threading.Thread(target=collector, daemon=True)
            th.start()
            arr = np.random.default_rng(int(rate)).exponential(1.0 / rate, 10 ** 7)
            t0 = time.perf_counter()
            t_next, k, n_sub = t0, 0, 0
            while True:
                now = time.perf_counter()
                if now - t0 >= args.served_seconds:
                    break
                if t_next > now:
                    time.sleep(min(t_next - now, 0.001))
                    continue
                is_scene = rng.random() < 0.1
                img = big if is_scene else pool[int(rng.integers(0, len(pool)))]
                q = lab_scenes if is_scene else lab_tiles
                if q.empty():
                    stalls += 1
                buf = q.get()
                h, w = img.shape[:2]
                lab = buf if is_scene else buf.reshape(-1)[:h * w].reshape(h, w)
                rid = srv.submit(img, lab)
                pending.put((rid, h * w, buf, q))
                n_sub += 1
                t_next += arr[k]
                k += 1
            pending.put(None)
            th.join()
            t_all = time.perf_counter() - t0
            stats = srv.stats()
        lat = np.array(lat)
        results.append({"rate_req_s": rate, "requests": int(len(lat)), "seconds": t_all,
                        "throughput_gpx_s": px[0] / t_all / 1e9, "req_s": len(lat) / t_all,
                        "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
                        "service_p50_ms": float(np.percentile(svc, 50)),
                        "service_p99_ms": float(np.percentile(svc, 99)),
                        "backpressure_waits": stalls, "kernel_launches": stats["kernel_launches"]})
        print(json.dumps({"served": results[-1]}), flush=True)
    print(json.dumps({"metric": "served labelling: throughput and p50/p99 latency",
                      "config": {"workload": "Poisson arrivals; 90% square tiles side U{256..4096}, "
                                             f"10% {SIDE}^2 scenes; pinned host uint8 RGB and labels; "
                                             f"{args.served_seconds} s per rate"},
                      "served": results}))
    return 0


def run_sweep(args):
    """Many full scenes back to back: device-resident batched labelling, and
    end to end with the host-to-device copy of scene i+1 overlapped with the
    labelling of scene i; uint8 and uint16 reflectance."""
    import ctypes
    import torch
    import paper_2403_13135_gb300 as sil
    import synth
    out = {}
    for dtname, dtype in (("u8", np.uint8), ("u16", np.uint16)):
        scenes = [synth.full_scene(2000 + i, SIDE, dtype=dtype)[0] for i in range(args.distinct)]
        n = args.scenes
        host = [torch.from_numpy(scenes[i % len(scenes)].view(np.uint8).reshape(SIDE, -1)).pin_memory()
                for i in range(len(scenes))]
        bpp = 3 if dtype == np.uint8 else 6
        dt = sil.SIL_U8 if dtype == np.uint8 else sil.SIL_U16
        p = sil.params()
        dbuf = [torch.empty((SIDE, SIDE * bpp), dtype=torch.uint8, device="cuda") for _ in range(2)]
        lab = [torch.empty((SIDE, SIDE), dtype=torch.uint8, device="cuda") for _ in range(2)]
        cnt = [torch.empty(4, dtype=torch.int64, device="cuda") for _ in range(n)]
        s_copy, s_comp = torch.cuda.Stream(), torch.cuda.Stream()
        ev_copy = [torch.cuda.Event() for _ in range(2)]
        ev_used = [torch.cuda.Event() for _ in range(2)]
        # device resident: all distinct scenes on device, labelled n times in one batch
        dres = [h.cuda() for h in host]
        labs = [torch.empty((SIDE, SIDE), dtype=torch.uint8, device="cuda") for _ in range(n)]
        imgs = [dres[i % len(dres)] for i in range(n)]
        tiles = (sil.sil_tile * n)()
        for i in range(n):
            t = tiles[i]
            t.img = imgs[i].data_ptr(); t.H = SIDE; t.W = SIDE; t.pitch_bytes = SIDE * bpp
            t.labels = labs[i].data_ptr(); t.label_pitch = SIDE; t.counts = cnt[i].data_ptr(); t.chip_counts = None
        ctx = sil.Context()
        st = torch.cuda.current_stream()
        sil.label_batch(ctx, tiles, n, dt, p, st)
        t_dev = _time_cuda(lambda: sil.label_batch(ctx, tiles, n, dt, p, st), 3, st)
        del dres, labs
        # end to end: double-buffered copy-in / label / labels back
        hl = [torch.empty((SIDE, SIDE), dtype=torch.uint8).pin_memory() for _ in range(2)]
        for b in range(2):  # warm the copy paths
            dbuf[b].copy_(host[b % len(host)], non_blocking=True)
            hl[b].copy_(lab[b], non_blocking=True)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for i in range(n):
            b = i % 2
            with torch.cuda.stream(s_copy):
                s_copy.wait_event(ev_used[b])
                dbuf[b].copy_(host[i % len(host)], non_blocking=True)
                ev_copy[b].record(s_copy)
            with torch.cuda.stream(s_comp):
                s_comp.wait_event(ev_copy[b])
                sil.check(sil.sil_label(dbuf[b].data_ptr(), SIDE, SIDE, SIDE * bpp, dt, ctypes.byref(p),
                                        lab[b].data_ptr(), SIDE, cnt[i].data_ptr(), None,
                                        ctypes.c_void_p(s_comp.cuda_stream)))
                hl[b].copy_(lab[b], non_blocking=True)
                ev_used[b].record(s_comp)
        torch.cuda.synchronize()
        t_e2e = time.perf_counter() - t0
        px = n * SIDE * SIDE
        out[dtname] = {"scenes": n, "distinct_scenes": len(scenes),
                       "device_resident_gpx_s": px / t_dev / 1e9,
                       "e2e_gpx_s": px / t_e2e / 1e9,
                       "h2d_gb_s": px * bpp / t_e2e / 1e9,
                       "alg_bytes_per_px": bpp + 1,
                       "device_hbm_gb_s": px * (bpp + 1) / t_dev / 1e9}
        ctx.close()
        del dbuf, lab, host
        torch.cuda.empty_cache()
    print(json.dumps({"metric": METRIC, "config": {"workload": f"throughput sweep of {SIDE}^2 scenes"},
                      "sweep": out}))
    return 0


def run_unet(args):
    """U-Net inference on filtered 256 x 256 chips of the scene (random weights,
    throughput only), as the paper's inferencing workflow: the scene is labelled
    with the filter's V' kept (sil_label_v), chips are cut with their V', and the
    timed step is the forward pass on the filtered chips (device-resident;
    tensor-core roofline); end to end with chips and V' copied in and the labels
    copied out."""
    import torch
    import paper_2403_13135_gb300 as sil
    import synth
    F, D, B = args.unet_width, args.unet_depth, args.unet_batch
    img, _ = synth.full_scene(1, SIDE)
    chips_h = synth.chips_from_scene(img, B, seed=3)
    # the filter's V' of the scene (on the GPU), cut at the same chip positions
    scene_dev = torch.from_numpy(img).cuda()
    _, vp_dev, _ = sil.label_v(scene_dev, None, labels=False)
    vp_h = synth.chips_from_scene(vp_dev.cpu().numpy()[..., None], B, seed=3)[..., 0].copy()
    del img
    wts = synth.unet_weights(F, D, seed=0)
    net = sil.UNet(sil.unet_config(F, D, B), list(wts.values()))
    chips = torch.from_numpy(chips_h).cuda()
    vps = torch.from_numpy(vp_h).cuda()
    lab = torch.empty((B, 256, 256), dtype=torch.uint8, device="cuda")
    st = torch.cuda.current_stream()
    for _ in range(max(3, args.warmup if args.warmup < 50 else 5)):
        net.forward(chips, lab, vprime=vps)
    torch.cuda.synchronize()
    steps = args.unet_steps
    clk = ClockSampler(0)
    clk.start()
    time.sleep(0.15)
    t0 = time.monotonic()
    dt = _time_cuda(lambda: net.forward(chips, lab, stream=st, vprime=vps), steps, st)
    t1 = time.monotonic()
    clk.mark(t0, t1)
    time.sleep(0.1)
    clk.stop()
    flops = net.flops_per_chip() * B
    achieved = flops / dt / 1e12
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            pk = json.load(f)
        peak, peak_src = float(pk["bf16_tflops_sustained"]), "measured bf16_tflops_sustained"
        burst = float(pk["bf16_tflops"])
    except Exception:
        peak, peak_src, burst = 1700.0, "fallback (sustained)", 1900.0
    # end to end: pinned chips in, forward, labels out, every step
    host = torch.from_numpy(chips_h).pin_memory()
    host_vp = torch.from_numpy(vp_h).pin_memory()
    hl = torch.empty((B, 256, 256), dtype=torch.uint8).pin_memory()
    e2e_steps = max(3, min(args.e2e_steps, steps))
    torch.cuda.synchronize()
    te0 = time.perf_counter()
    for _ in range(e2e_steps):
        chips.copy_(host, non_blocking=True)
        vps.copy_(host_vp, non_blocking=True)
        net.forward(chips, lab, vprime=vps)
        hl.copy_(lab, non_blocking=True)
    torch.cuda.synchronize()
    te = (time.perf_counter() - te0) / e2e_steps
    # the whole scene through the workflow: its 1849 chips filtered, batched,
    # labels written back into the scene's map
    scene_lab = torch.empty((SIDE, SIDE), dtype=torch.uint8, device="cuda")
    net.label_scene(scene_dev, vprime=vp_dev, labels=scene_lab)
    t_scene = _time_cuda(lambda: net.label_scene(scene_dev, vprime=vp_dev, labels=scene_lab), 3, st)
    del scene_dev, vp_dev, scene_lab
    errors = net.error_count()
    line = {
        "metric": "U-Net chips/s (F=%d, depth %d, bf16 tensor cores)" % (F, D),
        "value": B / dt, "unit": "chips/s", "n_gpus": 1, "steps": steps,
        "warmup": max(3, args.warmup if args.warmup < 50 else 5), "ms_per_step": dt * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "bf16",
        "data": "synthetic filtered chips of the seeded scene, seeded random weights",
        "config": {"workload": f"U-Net inference on filtered chips, {B} chips of 256x256 per step, "
                               f"base width {F}, depth {D}",
                   "l2": "activations (~1 GB per step) larger than L2",
                   "gpx_per_s": B * 65536 / dt / 1e9},
        "e2e": {"value": B / te, "unit": "chips/s",
                "h2d_bytes_per_step": int(chips_h.nbytes + vp_h.nbytes),
                "d2h_bytes_per_step": int(B * 65536)},
        "gpu_launches": int(steps * (1 + sil._lib.sil_unet_num_layers(D) - 1)),
        "roofline": {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                     "frac": achieved / peak, "traffic": None, "peak_source": peak_src,
                     "frac_of_burst": achieved / burst, "flops_per_step": flops},
        "clocks": clk.summary(),
        "wait_errors": errors,
        "scene": {"workload": f"one {SIDE}x{SIDE} scene: {(-(-SIDE // 256)) ** 2} filtered chips through "
                              f"sil_unet_label_scene", "ms": t_scene * 1e3,
                  "gpx_per_s": SIDE * SIDE / t_scene / 1e9},
    }
    if not args.no_cpu_baseline:
        import oracle.unet as U
        n, t_c = 0, time.perf_counter()
        while True:
            U.forward(chips_h[n % B:n % B + 1], wts, depth=D, vprime_u8=vp_h[n % B:n % B + 1])
            n += 1
            if time.perf_counter() - t_c > args.cpu_budget / 2:
                break
        tc = time.perf_counter() - t_c
        line["cpu_baseline"] = {"value": n / tc, "unit": "chips/s", "cores": 1, "kind": "oracle",
                                "sample": f"{n} chips through the float64 numpy oracle in {tc:.1f} s"}
    print(json.dumps(line))
    return 0


def _train_launches(shapes, D, F, B):
    """This library's kernel launches in one training step (forward,
    loss, backward, Adam and re-packing; the cuBLAS weight-gradient GEMMs
    are library kernels and not counted)."""
    nl = len(shapes)
    res = [256 >> l for l in range(D)] + [256 >> D]
    col_need, convs = 0, []
    for i, (shape, kind) in enumerate(shapes):
        if kind == 0:
            if i < 2 * D:
                H = res[i // 2]
            elif i < 2 * D + 2:
                H = res[D]
            else:
                H = res[D - 1 - (i - 2 * D - 2) // 3]
            cp = max(8, shape[1])
            convs.append(B * H * H * 9 * cp)
            col_need = max(col_need, B * H * H * 9 * cp)
    cap = min(col_need, 1 << 29)
    n = 1 + (nl - 1)                       # forward: input preparation + every layer
    n += 5                                 # count, loss, its sum, head backward, its sum
    n += sum(-(-c // cap) for c in convs)  # im2col chunks
    n += nl - 1                            # weight gradients to PyTorch layout
    n += (nl - 1) - 1                      # dgrad of every layer but the first
    n += 2 * D                             # space-to-depth and pool backward per level
    n += 1 + (nl - 1) + (nl - 2)           # Adam, forward and dgrad weight packing
    return n


def run_train(args):
    """One data-parallel training step of the U-Net (Sec. III-C: Adam,
    categorical cross-entropy, batch 32 per GPU) on auto-labelled chips of
    the seeded scene: forward, loss, backward, gradient averaging (none on
    one GPU), Adam, weight re-packing.  Device-resident timing (tensor-core
    roofline on 3x the forward FLOPs); end to end with the chips and labels
    copied in and the loss copied out every step."""
    import torch
    import paper_2403_13135_gb300 as sil
    import synth
    F, D, B = args.unet_width, args.unet_depth, args.train_batch
    img, _ = synth.full_scene(1, SIDE)
    scene_dev = torch.from_numpy(img).cuda()
    lab_scene, _, _ = sil.label(scene_dev)              # the auto-labels
    chips_h = synth.chips_from_scene(img, B, seed=3)
    lab_h = synth.chips_from_scene(lab_scene.cpu().numpy()[..., None], B, seed=3)[..., 0].copy()
    del img, scene_dev, lab_scene
    wts = synth.unet_weights(F, D, seed=0)
    tr = sil.Trainer(sil.unet_config(F, D, B), list(wts.values()))
    chips = torch.from_numpy(chips_h).cuda()
    labs = torch.from_numpy(lab_h).cuda()
    grads = torch.empty(tr.num_params, dtype=torch.float32, device="cuda")
    loss = torch.empty(1, dtype=torch.float32, device="cuda")
    st = torch.cuda.current_stream()
    warm = max(3, args.warmup if args.warmup < 50 else 5)
    losses = []
    for _ in range(warm):
        tr.step(chips, labs, lr=1e-4, grads=grads, loss=loss)
        losses.append(float(loss.item()))
    torch.cuda.synchronize()
    steps = args.train_steps
    clk = ClockSampler(0)
    clk.start()
    time.sleep(0.15)
    t0 = time.monotonic()
    dt = _time_cuda(lambda: tr.step(chips, labs, lr=1e-4, grads=grads, loss=loss, stream=st), steps, st)
    t1 = time.monotonic()
    clk.mark(t0, t1)
    time.sleep(0.1)
    clk.stop()
    losses.append(float(loss.item()))
    fwd = tr.net.flops_per_chip() * B
    flops = 3 * fwd
    achieved = flops / dt / 1e12
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            pk = json.load(f)
        peak, peak_src = float(pk["bf16_tflops_sustained"]), "measured bf16_tflops_sustained"
        burst = float(pk["bf16_tflops"])
    except Exception:
        peak, peak_src, burst = 1700.0, "fallback (sustained)", 1900.0
    host = torch.from_numpy(chips_h).pin_memory()
    host_lab = torch.from_numpy(lab_h).pin_memory()
    hloss = torch.empty(1, dtype=torch.float32).pin_memory()
    e2e_steps = max(3, min(args.e2e_steps, steps))
    torch.cuda.synchronize()
    te0 = time.perf_counter()
    for _ in range(e2e_steps):
        chips.copy_(host, non_blocking=True)
        labs.copy_(host_lab, non_blocking=True)
        tr.step(chips, labs, lr=1e-4, grads=grads, loss=loss)
        hloss.copy_(loss, non_blocking=True)
    torch.cuda.synchronize()
    te = (time.perf_counter() - te0) / e2e_steps
    errors = tr.net.error_count()
    line = {
        "metric": "U-Net training images/s (F=%d, depth %d, Adam, bf16 tensor cores)" % (F, D),
        "value": B / dt, "unit": "images/s", "n_gpus": 1, "steps": steps, "warmup": warm,
        "ms_per_step": dt * 1e3, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "bf16", "data": "synthetic chips of the seeded scene with the labeler's auto-labels, "
                                 "seeded random initial weights",
        "config": {"workload": f"U-Net training step, {B} chips of 256x256 per GPU, base width {F}, "
                               f"depth {D} ({sil._lib.sil_unet_num_layers(D)} layers, "
                               f"{tr.num_params} parameters)",
                   "l2": "activations and their gradients (several GB per step) larger than L2"},
        "e2e": {"value": B / te, "unit": "images/s",
                "h2d_bytes_per_step": int(chips_h.nbytes + lab_h.nbytes), "d2h_bytes_per_step": 4},
        "gpu_launches": int(steps * _train_launches(tr.shapes, D, F, B)),
        "roofline": {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                     "frac": achieved / peak, "traffic": None, "peak_source": peak_src,
                     "frac_of_burst": achieved / burst, "flops_per_step": flops,
                     "flops_note": "3x the forward pass (forward, input gradients, weight gradients)"},
        "loss": {"first": losses[0], "last": losses[-1]},
        "clocks": clk.summary(),
        "wait_errors": errors,
        "paper_context": "585.88 images/s on one A100 (Table III; TensorFlow, its own U-Net widths)",
    }
    if not args.no_cpu_baseline:
        import oracle.unet_train as T
        import oracle.unet as U
        n, t_c = 0, time.perf_counter()
        w64 = {k: (U.bf16(w), b) for k, (w, b) in wts.items()}
        while True:
            x = U.prep(chips_h[n % B:n % B + 1])
            acts, logits = T.forward_saved(x, w64, D)
            T.backward_network(acts, logits, lab_h[n % B:n % B + 1], w64, D)
            n += 1
            if time.perf_counter() - t_c > args.cpu_budget:
                break
        tc = time.perf_counter() - t_c
        line["cpu_baseline"] = {"value": n / tc, "unit": "images/s", "cores": 1, "kind": "oracle",
                                "sample": f"{n} chips through the float64 numpy training oracle "
                                          f"(forward + backward) in {tc:.1f} s"}
    print(json.dumps(line))
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="sil", choices=["sil", "reference"])
    ap.add_argument("--e2e-steps", type=int, default=20)
    ap.add_argument("--soak", type=float, default=1.5,
                    help="seconds of extra steps after the timed region, for clock samples")
    ap.add_argument("--cpu-budget", type=float, default=12.0)
    ap.add_argument("--ref-budget", type=float, default=60.0)
    ap.add_argument("--traffic", type=float, default=TRAFFIC_BYTES_PER_LAUNCH,
                    help="ncu DRAM bytes per launch of the labeler")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-cores", type=int, default=0,
                    help="oracle worker processes for the CPU baseline (0 = every host core)")
    ap.add_argument("--dtype", default="u8", choices=["u8", "u16"],
                    help="scene workload: uint8 RGB (the headline) or uint16 reflectance")
    ap.add_argument("--config", default="scene",
                    choices=["scene", "batch", "served", "sweep", "unet", "train"],
                    help="scene: the headline line; batch/served/sweep/unet/train: the other workloads")
    ap.add_argument("--unet-width", type=int, default=32)
    ap.add_argument("--unet-depth", type=int, default=5)
    ap.add_argument("--unet-batch", type=int, default=64)
    ap.add_argument("--unet-steps", type=int, default=50)
    ap.add_argument("--train-batch", type=int, default=32)
    ap.add_argument("--train-steps", type=int, default=20)
    ap.add_argument("--tiles", type=int, default=512)
    ap.add_argument("--rates", default="50,200,1000,2000")
    ap.add_argument("--served-seconds", type=float, default=60.0)
    ap.add_argument("--label-pool", type=int, default=96)
    ap.add_argument("--scenes", type=int, default=32)
    ap.add_argument("--distinct", type=int, default=4)
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    if args.config == "batch":
        return run_batch(args)
    if args.config == "served":
        return run_served(args)
    if args.config == "sweep":
        return run_sweep(args)
    if args.config == "unet":
        return run_unet(args)
    if args.config == "train":
        return run_train(args)
    return run_sil(args)


if __name__ == "__main__":
    sys.exit(main())
