#!/usr/bin/env python3
"""Throughput of grayscale morphological reconstruction on GB300.

One step = the whole reconstruction of one batch of synthetic tiles through
the C ABI (marker reset from its pristine copy, the learned schedule's
planning pass, validation, scan pairs, queue propagation, neighbour
notification, persistent launch replayed from a CUDA graph). Default workload
"uneven1000": 1000 tiles whose heights and widths are drawn from
{256, 512, ..., 4096} (4.7 Gpx, h-dome and fill-holes markers 50/50,
8-connectivity), reconstructed in one persistent launch. Metric:
reconstructed Mpix/s. "single4096" is one 4096 x 4096 mask reconstructed four
times (4-/8-connectivity x both markers); "batch64" is 64 tiles of 4096 x 4096.

--op selects the operation: "dilate" (the default, reconstruction by
dilation), "erode" (reconstruction by erosion of the complemented pairs, the
same propagation work as the dilation tiles) or "fill_holes" (FillHoles of
every distinct (mask, connectivity) of the workload; the output needs no
reset, so a step is the library call alone) or "dt" (the distance transform of
the workload's masks: objects I >= 100 and the space between them).
The line's "compare" block (skip it with --no-compare) times the plain
schedule, the per-tile launch loop, the learned schedule with and without its
planning pass, and the sweep-only and queue-first halves of the method with
their own rooflines. "cpu_baseline" is the CPU oracle on a bounded sample of
the workload, on all host cores and on one core. --microbench runs the
random-access and atomic micro-benchmarks instead; --tile T reconstructs one
tile alone (a small fixed case for profilers); --subset n keeps every n-th
tile; --impl reference times the CPU oracle on the same workload (the
reference arm).

Timing: CUDA events on the library's stream around each step; L2 is flushed
(a 512 MiB write) before every timed step, outside the events. Under torchrun
the job is the workload's family with N times its tiles, split across the N
ranks by longest-processing-time-first (weak scaling, no collective on the
data path), and the slowest rank's time counts.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

PEAKS_FALLBACK = {"hbm_gbs": 6800.0}
# compulsory traffic per pixel: read I, read J, write R (reconstruction by
# dilation or erosion); read I, write the result (FillHoles)
ALG_BYTES_PER_PX = {"dilate": 3, "erode": 3, "fill_holes": 2, "dt": 5}
OP_CODE = {"dilate": 0, "erode": 1, "fill_holes": 2}
OPS = sorted(list(OP_CODE) + ["dt"])


def code_of(text):
    """Source text without comments and blank space: what the compiler sees of it."""
    import re
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    text = re.sub(r"//[^\n]*", "", text)
    return "\n".join(l.strip() for l in text.splitlines() if l.strip())


def kernel_hash(read=None):
    """Hash of the reconstruction kernel's code (comments excluded), to tell
    whether committed ncu counters still describe it."""
    import hashlib
    h = hashlib.sha256()
    for f in ("paper_1311_0378_gb300/csrc/recon_kernels.cu", "paper_1311_0378_gb300/csrc/recon_internal.h"):
        if read:
            text = read(f)
        else:
            with open(os.path.join(ROOT, f)) as fh:
                text = fh.read()
        h.update(code_of(text).encode())
    return h.hexdigest()[:16]


def measured_traffic(workload):
    """DRAM bytes per launch from the committed ncu capture, or None when the
    kernel source changed since the counters were taken."""
    try:
        with open(os.path.join(ROOT, "profiles", "traffic.json")) as f:
            t = json.load(f)
    except OSError:
        return None
    if t.get("kernel_source_sha256_16") != kernel_hash():
        return None
    w = t.get("workloads", {}).get(workload)
    return w.get("dram_bytes_per_launch") if w else None


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except OSError:
        return PEAKS_FALLBACK, "fallback"


class Clocks:
    """Samples SM clock and throttle reasons with nvidia-smi during the timed
    region: the sampler is started, and its first sample awaited, before the
    region begins, so the samples taken inside it are counted from there."""

    INTERVAL_MS = 50

    def __init__(self, index=0):
        self.index = index
        self.rows = []
        self.proc = None
        self.start = 0
        self.end = None

    def __enter__(self):
        q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
             "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
             "clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + q,
                                          "--format=csv,noheader,nounits", "-lms", str(self.INTERVAL_MS)],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
            t0 = time.time()
            while not self.rows and time.time() - t0 < 5.0:   # sampler live before the region starts
                time.sleep(0.01)
        except OSError:
            self.proc = None
        self.start = len(self.rows)
        return self

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) == 7:
                self.rows.append(parts)

    def __exit__(self, *a):
        self.end = len(self.rows)
        if self.proc:
            if self.end == self.start:   # a region shorter than the interval: take the next sample
                t0 = time.time()
                while len(self.rows) == self.start and time.time() - t0 < 1.0:
                    time.sleep(0.005)
                self.end = len(self.rows)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        rows = self.rows[self.start:self.end]
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm = [float(r[0]) for r in rows if r[0].replace(".", "").isdigit()]
        mx = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[3 + i] == "Active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows), "interval_ms": self.INTERVAL_MS}


def workload_tiles(name, op="dilate", copies=1):
    import synth
    w = synth.scaled_workload(name, copies)
    tiles = w.tiles
    if op == "fill_holes" and name == "single4096":
        # one shared mask: the marker kinds collapse, one tile per connectivity
        seen, tiles = set(), []
        for t in w.tiles:
            if t.conn not in seen:
                seen.add(t.conn)
                tiles.append(t)
    return w, tiles, name == "single4096"


def job_tiles(name, op, world, rank, subset=1):
    """The whole job's tiles and this rank's share. With N ranks the job is
    the workload's family with N times its tiles (weak scaling: the same work
    per GPU), split across ranks by longest-processing-time-first on the pixel
    count; tiles are independent, so no data crosses ranks. subset > 1 keeps
    every subset-th tile of the job (a stated smaller case, e.g. for a
    profiler capture)."""
    from paper_1311_0378_gb300.shard import lpt_shards
    w, tiles, shared = workload_tiles(name, op, world)
    tiles = list(tiles)[::max(1, subset)]
    shards = lpt_shards([t.H * t.W for t in tiles], world)
    mine = [tiles[i] for i in sorted(shards[rank])]
    return w, tiles, mine, shared


def complement_(t):
    """In place: v -> 255 - v (turns a dilation pair into an erosion pair)."""
    t.bitwise_not_()
    return t


def gen_host(w, tiles, shared_mask, op="dilate"):
    """Pinned host tensors: masks and pristine markers for every tile (for
    erosion, the complemented pairs)."""
    import torch
    import synth
    if shared_mask:
        pairs = synth.generate(tiles, w.seed)
        I = torch.from_numpy(pairs[0][0]).pin_memory()
        Is = [I] * len(tiles)
        Js = [torch.from_numpy(J).pin_memory() for _, J in pairs]
    else:
        Is = [torch.empty((t.H, t.W), dtype=torch.uint8).pin_memory() for t in tiles]
        Js = [torch.empty((t.H, t.W), dtype=torch.uint8).pin_memory() for t in tiles]
        synth.generate_into(tiles, w.seed, [x.data_ptr() for x in Is], [x.data_ptr() for x in Js])
    if op == "erode":
        for x in ({id(x): x for x in Is}.values()):
            complement_(x)
        for x in Js:
            complement_(x)
    return Is, Js


def oracle_op(pairs, conns, op, nthreads):
    """The CPU oracle for one operation over independent tiles on host
    threads; erosion pairs come already complemented."""
    import oracle
    if op == "fill_holes":
        from concurrent.futures import ThreadPoolExecutor   # the C oracle releases the GIL
        with ThreadPoolExecutor(max_workers=max(1, nthreads)) as ex:
            list(ex.map(lambda a: oracle.fill_holes(a[0][0], a[1]), zip(pairs, conns)))
        return max(1, min(nthreads, len(pairs)))
    _, used = oracle.recon_tiles(pairs, conns, "erode" if op == "erode" else "sweep", nthreads=nthreads)
    return used


def baseline_samples(name, tiles):
    """Bounded samples of the workload for the CPU oracle: (all-cores sample,
    one-core sample), each a list of tile indices."""
    n = len(tiles)
    if n <= 8:
        return list(range(n)), list(range(min(2, n)))
    ncores = os.cpu_count() or 1
    stride = max(1, n // max(ncores, 16))
    many = list(range(0, n, stride))[:max(ncores, 16)]
    one = many[::max(1, len(many) // 4)][:4] if n > 64 else many[:1]
    return many, one


def cpu_baseline(w, tiles, shared_mask, op="dilate"):
    """The CPU oracle (sweeps to stability), as it stands, on a bounded sample
    of the workload: once with one tile per host thread on all cores, once on
    a single core. Returns the JSON object of the bench line."""
    import synth
    many, one = baseline_samples(w.name, tiles)
    out = {}
    for key, idx, threads in (("all_cores", many, os.cpu_count() or 1), ("one_core", one, 1)):
        sample = [tiles[i] for i in idx]
        pairs = synth.generate(sample, w.seed)
        if op == "erode":   # input preparation, outside the timing
            pairs = [(255 - I, 255 - J) for I, J in pairs]
        t0 = time.perf_counter()
        used = oracle_op(pairs, [t.conn for t in sample], op, min(threads, len(sample)))
        dt = time.perf_counter() - t0
        px = sum(t.H * t.W for t in sample)
        out[key] = {"value": round(px / dt / 1e6, 3), "cores": used, "seconds": round(dt, 2),
                    "sample": "tiles %s of %d (%s), full size, op %s" % (
                        idx if len(idx) <= 8 else "%d..%d step %d (%d tiles)" % (idx[0], idx[-1], idx[1] - idx[0],
                                                                              len(idx)),
                        len(tiles), w.name, op)}
    return {"value": out["all_cores"]["value"], "unit": "Mpix/s", "cores": out["all_cores"]["cores"],
            "kind": "oracle", "sample": out["all_cores"]["sample"], "seconds": out["all_cores"]["seconds"],
            "host_cores": os.cpu_count(), "one_core": out["one_core"]}


def run_reference(args):
    """--impl reference: the CPU oracle timed as the reference arm."""
    import numpy as np
    import oracle
    import synth
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    w, tiles, shared = workload_tiles(args.workload, args.op)
    # one step = one tile of the workload, rotating through the tiles, each
    # reconstructed in full by the oracle on one host thread
    pairs = synth.generate(tiles, w.seed) if len(tiles) <= 8 else None
    def step(i):
        t = tiles[i % len(tiles)]
        I, J = pairs[i % len(tiles)] if pairs else synth.tile_pair(t, w.seed)
        if args.op == "erode":
            I, J = 255 - I, 255 - J
        t0 = time.perf_counter()
        if args.op == "dt":
            B = np.ascontiguousarray((I >= 100) if i % 2 == 0 else (I < 100), dtype=np.uint8)
            t0 = time.perf_counter()
            oracle.distance_transform(B)
            return time.perf_counter() - t0, t.H * t.W
        if args.op == "erode":
            oracle.recon_erode(I, J, t.conn)
        elif args.op == "fill_holes":
            oracle.fill_holes(I, t.conn)
        else:
            oracle.recon(I, J, t.conn)
        return time.perf_counter() - t0, t.H * t.W
    for i in range(args.warmup):
        step(i)
    tot_t, tot_px = 0.0, 0
    for i in range(args.steps):
        dt, px = step(args.warmup + i)
        tot_t += dt
        tot_px += px
    v = tot_px / tot_t / 1e6
    metric = "distance-transformed Mpix/s" if args.op == "dt" else "reconstructed Mpix/s"
    line = {"impl": "reference", "metric": metric, "value": round(v, 3),
            "unit": "Mpix/s", "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": round(1000 * tot_t / max(args.steps, 1), 3), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u8", "data": "synthetic",
            "config": {"workload": w.name, "op": args.op, "step": "one tile per step, rotating",
                       "conn": "per tile"},
            "cpu_baseline": {"value": round(v, 3), "unit": "Mpix/s", "cores": 1, "kind": "oracle",
                             "sample": "one full tile per step, rotating through the %d tiles" % len(tiles)},
            "e2e": {"value": round(v, 3), "unit": "Mpix/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def time_fn(fn, stream, J, J0, flush, reps=3):
    """Median device time (ms) of fn() over reps runs, J reset before each."""
    import torch
    out = []
    for i in range(reps + 1):
        with torch.cuda.stream(stream):
            for a, b in zip(J, J0):
                a.copy_(b, non_blocking=True)
        flush.fill_(i & 0xFF)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        fn()
        e1.record(stream)
        stream.synchronize()
        if i > 0:
            out.append(e0.elapsed_time(e1))
    return statistics.median(out)


def compare_schedules(rc, ctx, stream, Is, Js, J0, tiles, desc, px, flush, args):
    """Batched persistent launch vs a per-tile launch loop, and the learned
    schedule vs the plain one, on the same tiles and GPU (outputs identical:
    R is unique; the tests check it)."""
    res = {}
    k_default = rc.recon_get_param(ctx, rc.RECON_P_SWEEPS)
    g_default = rc.recon_get_param(ctx, rc.RECON_P_SCAN_GAIN)
    plain_var = [k_default + 256 * (g_default // 64) if k_default >= 0 else -1] * len(desc)
    plain_order = sorted(range(len(desc)), key=lambda i: -desc[i][2] * desc[i][3])
    def batched():   # the plain schedule: context defaults, largest tiles first
        rc.check(rc.recon_batch_ex(ctx, desc, plain_var, plain_order), "batch")
    def loop():      # the plain per-tile path: one launch per tile, context defaults
        for d in desc:
            st = rc.recon_batch_ex(ctx, [d], plain_var[:1], [0])
            if st != rc.RECON_OK:
                raise rc.ReconError(st, "per-tile launch")
    res["batched_plain_mpix_s"] = round(px / time_fn(batched, stream, Js, J0, flush) / 1e3, 1)
    res["per_tile_loop_mpix_s"] = round(px / time_fn(loop, stream, Js, J0, flush, reps=2) / 1e3, 1)
    try:
        from paper_1311_0378_gb300 import cost_model
        meta = cost_model.install(ctx)
        import torch
        with torch.cuda.stream(stream):   # plan on the pristine markers
            for a, b in zip(Js, J0):
                a.copy_(b, non_blocking=True)
        torch.cuda.synchronize()
        st, var, order, pred = rc.recon_sched_plan_batch(ctx, desc)
        rc.check(st, "plan")
        def learned():
            rc.check(rc.recon_batch_ex(ctx, desc, var, order), "learned batch")
        def learned_full():   # planning (features + MLP) inside the timed region
            st2, v2, o2, _ = rc.recon_sched_plan_batch(ctx, desc)
            rc.check(st2, "plan")
            rc.check(rc.recon_batch_ex(ctx, desc, v2, o2), "learned batch")
        res["batched_learned_mpix_s"] = round(px / time_fn(learned, stream, Js, J0, flush) / 1e3, 1)
        res["batched_learned_with_planning_mpix_s"] = round(px / time_fn(learned_full, stream, Js, J0, flush) / 1e3, 1)
        vb = cost_model.load()[2][1]
        res["learned_queue_variant_fraction"] = round(sum(1 for v in var if v == vb) / len(var), 3)
        res["model_tiles"] = meta.get("tiles")
    except (OSError, ValueError) as e:
        res["batched_learned_mpix_s"] = None
        res["learned_note"] = "no trained model: %s" % e
    return res


def run_microbench(args):
    """--microbench: the GB300 versions of Tables III and IV (random 32-bit
    reads / writes in a matrix; atomic adds on one variable or an array), in
    the paper's configuration (4K x 4K matrix, 10 million operations) and in
    an HBM-sized one (2^30 elements, 4 GiB). One JSON line."""
    import torch
    import paper_1311_0378_gb300 as rc
    from paper_1311_0378_gb300 import build as rbuild
    rbuild.build()
    torch.cuda.set_device(0)
    reps = max(args.steps, 3)
    res = {}
    for name, log2n, ops in (("paper_4Kx4K", 24, 10_000_000), ("hbm_4GiB", 30, 100_000_000)):
        M = torch.zeros(1 << log2n, dtype=torch.int32, device="cuda")
        torch.cuda.synchronize()
        for write in (False, True):
            times = []
            for r in range(reps + 1):
                st, _, ms = rc.recon_mb_random(M.data_ptr(), log2n, ops, write, 1000 + r)
                rc.check(st, "recon_mb_random")
                if r:
                    times.append(ms)
            ms = statistics.median(times)
            res["%s_random_%s_MBps" % (name, "write" if write else "read")] = round(ops * 4 / (ms / 1e3) / 1e6, 1)
            res["%s_random_%s_Mops" % (name, "write" if write else "read")] = round(ops / (ms / 1e3) / 1e6, 1)
        del M
    threads = rc.recon_mb_threads(0)
    C = torch.zeros(threads, dtype=torch.int32, device="cuda")
    for mode, label, iters in ((0, "global_single_variable", 64), (1, "global_array", 256),
                               (2, "shared_single_word_per_cta", 256), (3, "shared_array", 1024)):
        times = []
        for r in range(reps + 1):
            C.zero_()
            torch.cuda.synchronize()
            st, ms = rc.recon_mb_atomic(C.data_ptr(), mode, iters)
            rc.check(st, "recon_mb_atomic")
            if r:
                times.append(ms)
        res["atomic_add_%s_Mops" % label] = round(threads * iters / (statistics.median(times) / 1e3) / 1e6, 1)
    line = {"metric": "device micro-benchmarks (Tables III-IV)", "unit": "MB/s and Mops/s", "n_gpus": 1,
            "steps": reps, "data": "synthetic", "config": {"threads": threads, "timing": "CUDA events, median"},
            "results": res,
            "paper_gpu": {"random_read_MBps": 895, "random_write_MBps": 126,
                          "atomic_single_variable_Mops": 693, "atomic_array_Mops": 38630}}
    print(json.dumps(line), flush=True)
    return 0


def dt_masks(w, tiles):
    """Distance-transform inputs: the objects (blob pixels, I >= 100) of each
    distinct mask of the workload, and the space between them (I < 100)."""
    import numpy as np
    import synth
    masks, seen = [], set()
    for t in tiles:
        I, _ = synth.tile_pair(t, w.seed)
        h = hash(I[::97, ::89].tobytes())
        if h in seen:
            continue
        seen.add(h)
        masks.append(np.ascontiguousarray(I >= 100, dtype=np.uint8))
        masks.append(np.ascontiguousarray(I < 100, dtype=np.uint8))
    return masks


def run_dt(args):
    """--op dt: the distance transform (Table II) on the workload's masks."""
    import numpy as np
    import torch
    import paper_1311_0378_gb300 as rc
    from paper_1311_0378_gb300 import build as rbuild
    rbuild.build()
    torch.cuda.set_device(0)
    w, tiles, _ = workload_tiles(args.workload)
    masks = dt_masks(w, tiles[:8])
    px = sum(m.size for m in masks)
    # the transform runs on torch's current stream, where the timing events are recorded
    ctx = rc.recon_init(0, torch.cuda.current_stream().cuda_stream, 0)
    dB = [torch.from_numpy(m).cuda() for m in masks]
    d2 = [torch.empty(m.shape, dtype=torch.int32, device="cuda") for m in masks]
    flush = torch.empty(512 << 20, dtype=torch.uint8, device="cuda")
    torch.cuda.synchronize()

    def step():
        for b, d in zip(dB, d2):
            rc.check(rc.recon_dt(ctx, b.data_ptr(), d.data_ptr(), 0, b.shape[0], b.shape[1]), "recon_dt")
    launches = 0
    for b, d in zip(dB, d2):   # per mask: init, the level launches (batches of 16), final
        rc.check(rc.recon_dt(ctx, b.data_ptr(), d.data_ptr(), 0, b.shape[0], b.shape[1]), "recon_dt")
        launches += 2 + rc.recon_dt_levels(ctx)
    for _ in range(max(args.warmup, 3)):
        step()
    times = []
    with Clocks(0) as clk:
        for i in range(args.steps):
            flush.fill_(i & 0xFF)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            step()
            e1.record()
            torch.cuda.synchronize()
            times.append(e0.elapsed_time(e1))
    levels = rc.recon_dt_levels(ctx)
    # end to end: host mask in, host distances out
    hd2 = [torch.empty(m.shape, dtype=torch.int32).pin_memory() for m in masks]
    hB = [torch.from_numpy(m).pin_memory() for m in masks]
    e2e = []
    for i in range(3):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for b, hb, d, hd in zip(dB, hB, d2, hd2):
            b.copy_(hb, non_blocking=True)
            torch.cuda.synchronize()
            rc.check(rc.recon_dt(ctx, b.data_ptr(), d.data_ptr(), 0, b.shape[0], b.shape[1]), "recon_dt")
            hd.copy_(d)
        e2e.append(time.perf_counter() - t0)
    rc.recon_free(ctx)
    ms = statistics.mean(times)
    pk, src = peaks()
    achieved = ALG_BYTES_PER_PX["dt"] * px / (ms / 1e3) / 1e9
    line = {"metric": "distance-transformed Mpix/s", "value": round(px / (ms / 1e3) / 1e6, 2), "unit": "Mpix/s",
            "n_gpus": 1, "steps": args.steps, "warmup": max(args.warmup, 3), "ms_per_step": round(ms, 4),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int32",
            "data": "synthetic",
            "config": {"workload": w.name, "op": "dt", "masks": len(masks), "pixels_per_step": px,
                       "objects": "blob pixels (I >= 100) and the space between them (I < 100)",
                       "l2": "flushed before each timed step (512 MiB write)", "levels_last_mask": levels},
            "roofline": {"bound": "hbm", "achieved": round(achieved, 2), "peak": pk["hbm_gbs"], "unit": "GB/s",
                         "frac": round(achieved / pk["hbm_gbs"], 5), "traffic": None,
                         "alg_bytes_per_px": ALG_BYTES_PER_PX["dt"], "peak_source": src,
                         "note": "step time includes the host reads of the level counters"},
            "e2e": {"value": round(px / statistics.median(e2e) / 1e6, 2), "unit": "Mpix/s",
                    "h2d_bytes_per_step": px, "d2h_bytes_per_step": 4 * px},
            "gpu_launches": launches * args.steps, "clocks": clk.summary()}
    if not args.no_cpu_baseline:
        import oracle
        from concurrent.futures import ThreadPoolExecutor
        t0 = time.perf_counter()
        with ThreadPoolExecutor(max_workers=len(masks)) as ex:
            list(ex.map(oracle.distance_transform, masks))
        dt = time.perf_counter() - t0
        line["cpu_baseline"] = {"value": round(px / dt / 1e6, 3), "unit": "Mpix/s", "cores": len(masks),
                                "kind": "oracle", "sample": "all %d masks, full size" % len(masks),
                                "seconds": round(dt, 2)}
    print(json.dumps(line), flush=True)
    return 0


def phase_rooflines(rc, ctx, stream, Js, J0, desc, tiles, px, flush):
    """The scan (sweep) and queue halves of the method, each timed on its own
    over the same batch, with its own roofline: the sweeps-only variant moves
    3 bytes per pixel per directional pass (read I and J, write J; 128-pixel
    block rows counted by the kernel) against the measured HBM copy bandwidth;
    the queue-first variant (no scan pairs) checks |N| neighbours per wavefront
    entry, each a shared-memory test and, for a candidate, one claim (an
    atomic OR), against the shared-memory atomic-add rate measured here by the
    micro-benchmark."""
    import torch
    n = len(desc)
    order = sorted(range(n), key=lambda i: -desc[i][2] * desc[i][3])
    pk, src = peaks()
    out = {}
    for name, var in (("sweeps_only", -1), ("queue_first", 0)):
        def run(v=var):
            rc.check(rc.recon_batch_ex(ctx, desc, [v] * n, order), name)
        ms = time_fn(run, stream, Js, J0, flush)
        kms = rc.recon_last_kernel_ms(ctx)
        w = rc.recon_get_work(ctx, n)
        rows = sum(x["scan_rows"] for x in w)
        pops = sum(x["pops"] for x in w)
        res = {"mpix_s": round(px / ms / 1e3, 1), "kernel_ms": round(kms, 3), "scan_rows": rows, "pops": pops}
        if name == "sweeps_only":
            gbs = rows * 128 * 3 / (kms / 1e3) / 1e9
            res.update({"bound": "hbm", "achieved_GBps": round(gbs, 1), "peak_GBps": pk["hbm_gbs"],
                        "frac": round(gbs / pk["hbm_gbs"], 4), "bytes_per_row_px": 3})
        else:
            checks = sum(x["pops"] * t.conn for x, t in zip(w, tiles))
            threads = rc.recon_mb_threads(0)
            C = torch.zeros(threads, dtype=torch.int32, device=Js[0].device)
            torch.cuda.synchronize()
            for _ in range(2):   # the first launch is a warm-up
                st, mb_ms = rc.recon_mb_atomic(C.data_ptr(), 3, 1024)
                rc.check(st, "recon_mb_atomic")
            peak = threads * 1024 / (mb_ms / 1e3)
            rate = checks / (kms / 1e3)
            res.update({"bound": "shared-memory atomics", "achieved_Gops": round(rate / 1e9, 2),
                        "peak_Gops": round(peak / 1e9, 1), "frac": round(rate / peak, 5),
                        "unit_op": "one neighbour test (and claim, for a candidate) per neighbour of a popped entry"})
        out[name] = res
    return out


def run_tile_mode(args):
    """--tile T: reconstructs tile T of the workload alone through recon_run_op,
    --steps times after --warmup runs, and prints one JSON line per run with
    its device time and work counters (a small, fixed case for profilers)."""
    import torch
    import paper_1311_0378_gb300 as rc
    from paper_1311_0378_gb300 import build as rbuild
    import synth
    rbuild.build()
    w = synth.workload(args.workload)
    spec = w.tiles[args.tile]
    I, J = synth.tile_pair(spec, w.seed)
    if args.op == "erode":
        I, J = 255 - I, 255 - J
    ctx = rc.recon_init(0, 0, 0)
    for kv in args.param:
        k, v = kv.split("=")
        rc.check(rc.recon_set_param(ctx, getattr(rc, "RECON_P_" + k.upper()), int(v)), kv)
    dI = torch.from_numpy(I).cuda()
    J0 = torch.from_numpy(J).cuda()
    dJ = J0.clone()
    torch.cuda.synchronize()
    for r in range(args.warmup + args.steps):
        dJ.copy_(J0)
        torch.cuda.synchronize()
        rc.check(rc.recon_run_op(ctx, dI.data_ptr(), dJ.data_ptr(), spec.H, spec.W, spec.conn, OP_CODE[args.op]),
                 "recon_run_op")
        rc.check(rc.recon_sync_for(ctx, 120000), "sync")
        if r >= args.warmup:
            print(json.dumps({"tile": args.tile, "workload": w.name, "H": spec.H, "W": spec.W, "conn": spec.conn,
                              "marker": spec.marker, "op": args.op, "run": r - args.warmup,
                              "kernel_ms": round(rc.recon_last_kernel_ms(ctx), 4),
                              **rc.recon_get_work(ctx, 1)[0]}), flush=True)
    rc.recon_free(ctx)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--workload", default="uneven1000",
                    choices=["uneven1000", "batch64", "single4096", "single512"],
                    help="uneven1000 (default): 1000 tiles of uneven sizes, 4.7 Gpx, one persistent launch")
    ap.add_argument("--op", default="dilate", choices=OPS,
                    help="dilate: reconstruction by dilation; erode: by erosion (complemented pairs); "
                         "fill_holes: FillHoles of the masks")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--e2e-steps", type=int, default=3)
    ap.add_argument("--block-h", type=int, default=0)
    ap.add_argument("--sweeps", type=int, default=-99)
    ap.add_argument("--bands", type=int, default=0)
    ap.add_argument("--no-compare", action="store_true",
                    help="skip the plain schedule, per-tile launch loop and the two halves of the method")
    ap.add_argument("--subset", type=int, default=1,
                    help="keep every n-th tile of the job (a stated smaller case, e.g. for ncu captures)")
    ap.add_argument("--tile", type=int, default=-1,
                    help="reconstruct this one tile of the workload alone and print its time and work")
    ap.add_argument("--param", action="append", default=[],
                    help="with --tile: KEY=VALUE context parameter, KEY a RECON_P_* suffix")
    ap.add_argument("--autotune", action="store_true")
    ap.add_argument("--schedule", default="learned", choices=["learned", "plain"],
                    help="learned: the cost model picks each tile's variant and the packing order "
                         "(planning runs inside every timed step); plain: context defaults")
    ap.add_argument("--microbench", action="store_true",
                    help="run the random-access and atomic micro-benchmarks (Tables III-IV) instead")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    if args.microbench:
        return run_microbench(args)
    if args.tile >= 0:
        return run_tile_mode(args)
    if args.op == "dt":
        return run_dt(args)

    import torch
    import paper_1311_0378_gb300 as rc
    from paper_1311_0378_gb300 import build as rbuild

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    if rank == 0 or world == 1:
        rbuild.build()
    if dist:
        dist.barrier()

    w, job, tiles, shared = job_tiles(args.workload, args.op, world, rank, args.subset)
    Is_h, Js_h = gen_host(w, tiles, shared, args.op)
    opc = OP_CODE[args.op]
    reset_j = args.op != "fill_holes"   # a FillHoles output needs no reset
    dev = torch.device("cuda", local)
    if shared:
        Id = Is_h[0].to(dev)
        Is = [Id] * len(tiles)
    else:
        Is = [x.to(dev) for x in Is_h]
    J0 = [x.to(dev) for x in Js_h]
    Js = [x.clone() for x in J0]
    torch.cuda.synchronize()

    stream = torch.cuda.Stream(device=dev)
    learned = args.schedule == "learned"
    ctx = rc.recon_init(local, stream.cuda_stream, rc.RECON_FLAG_LEARNED if learned else 0)
    model_meta = None
    if learned:
        from paper_1311_0378_gb300 import cost_model
        model_meta = cost_model.install(ctx)
    for key, val in ((rc.RECON_P_BLOCK_H, args.block_h), (rc.RECON_P_BANDS, args.bands)):
        if val:
            rc.check(rc.recon_set_param(ctx, key, val))
    if args.sweeps != -99:
        rc.check(rc.recon_set_param(ctx, rc.RECON_P_SWEEPS, args.sweeps))
    desc = [(I.data_ptr(), J.data_ptr(), t.H, t.W, t.W, t.conn, opc) for I, J, t in zip(Is, Js, tiles)]
    tuned = None
    if args.autotune:
        st, tuned = rc.recon_autotune(ctx, desc, 2)
        rc.check(st, "recon_autotune")
    params = {"block_h": rc.recon_get_param(ctx, rc.RECON_P_BLOCK_H),
              "bands": rc.recon_get_param(ctx, rc.RECON_P_BANDS),
              "scan_pairs": rc.recon_get_param(ctx, rc.RECON_P_SWEEPS),
              "grid": rc.recon_get_param(ctx, rc.RECON_P_GRID), "autotuned": tuned is not None,
              "schedule": args.schedule,
              "cost_model": ({"tiles": model_meta.get("tiles"), "variants": model_meta.get("variants")}
                             if model_meta else None)}
    px = sum(t.H * t.W for t in tiles)          # this rank's pixels per step
    job_px = sum(t.H * t.W for t in job)        # every rank's pixels per step
    flush = torch.empty(512 << 20, dtype=torch.uint8, device=dev)

    def step():
        if reset_j:
            with torch.cuda.stream(stream):
                for J, J0_ in zip(Js, J0):
                    J.copy_(J0_, non_blocking=True)
        st = rc.recon_batch(ctx, desc)
        if st != rc.RECON_OK:
            raise rc.ReconError(st, "recon_batch")

    for _ in range(max(args.warmup, 3)):
        step()
    rc.check(rc.recon_sync(ctx), "warmup")

    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    kern_ms = []
    with Clocks(local) as clk:
        for i in range(args.steps):
            flush.fill_(i & 0xFF)
            torch.cuda.synchronize()
            if dist:
                dist.barrier()
            ev[i][0].record(stream)
            step()
            ev[i][1].record(stream)
            stream.synchronize()
            kern_ms.append(rc.recon_last_kernel_ms(ctx))
        torch.cuda.synchronize()
    rc.check(rc.recon_sync(ctx), "timed steps")
    step_ms = [a.elapsed_time(b) for a, b in ev]
    ms = sum(step_ms) / len(step_ms)
    if dist:
        t = torch.tensor([ms], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
    value = job_px / (ms / 1e3) / 1e6

    compare = None
    if not args.no_compare and len(tiles) > 1:
        compare = compare_schedules(rc, ctx, stream, Is, Js, J0, tiles, desc, px, flush, args)
        compare["learned_with_planning_vs_plain"] = (
            round(compare["batched_learned_with_planning_mpix_s"] / compare["batched_plain_mpix_s"], 3)
            if compare.get("batched_learned_with_planning_mpix_s") else None)
        compare["batched_plain_vs_per_tile_loop"] = round(
            compare["batched_plain_mpix_s"] / compare["per_tile_loop_mpix_s"], 3)
        if args.op == "dilate":
            compare["phases"] = phase_rooflines(rc, ctx, stream, Js, J0, desc, tiles, px, flush)

    # end to end: host (pinned) buffers through recon_batch_host
    Jh = [x.clone().pin_memory() for x in Js_h]
    htiles = [(I.data_ptr(), J.data_ptr(), t.H, t.W, t.W, t.conn, opc) for I, J, t in zip(Is_h, Jh, tiles)]
    e2e_ms = []
    for i in range(args.e2e_steps + 1):
        for a, b in zip(Jh, Js_h):
            a.copy_(b)
        flush.fill_(i & 0xFF)
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        t0 = time.perf_counter()
        rc.check(rc.recon_batch_host(ctx, htiles), "recon_batch_host")
        if i > 0:
            e2e_ms.append(1e3 * (time.perf_counter() - t0))
    e2e_t = statistics.median(e2e_ms)
    if dist:
        t = torch.tensor([e2e_t], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        e2e_t = float(t.item())
    e2e = job_px / (e2e_t / 1e3) / 1e6
    h2d = sum((2 if reset_j else 1) * t.H * t.W for t in tiles)
    d2h = px
    rc.recon_free(ctx)

    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return 0
    pk, src = peaks()
    kms = statistics.mean(kern_ms)
    alg = ALG_BYTES_PER_PX[args.op]
    achieved = alg * px / (kms / 1e3) / 1e9
    traffic_key = w.name if args.op == "dilate" else "%s:%s" % (w.name, args.op)
    traffic = measured_traffic(traffic_key) if args.subset == 1 and world == 1 else None
    roof = {"bound": "hbm", "achieved": round(achieved, 2), "peak": pk["hbm_gbs"], "unit": "GB/s",
            "frac": round(achieved / pk["hbm_gbs"], 5), "traffic": traffic,
            "kernel": "recon_persistent", "kernel_ms": round(kms, 4),
            "alg_bytes_per_px": alg, "alg_bytes_per_launch": alg * px, "peak_source": src,
            "limiter": "propagation depth and shared-memory latency of thin wavefronts (not DRAM)"}
    if traffic:
        roof["dram_GBps"] = round(traffic / (kms / 1e3) / 1e9, 2)
        roof["dram_frac"] = round(traffic / (kms / 1e3) / 1e9 / pk["hbm_gbs"], 5)
    line = {
        "metric": "reconstructed Mpix/s", "value": round(value, 2), "unit": "Mpix/s",
        "n_gpus": world, "steps": args.steps, "warmup": max(args.warmup, 3),
        "ms_per_step": round(ms, 4), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "u8", "data": "synthetic",
        "config": {"workload": w.name, "op": args.op, "tiles": len(job), "pixels_per_step": job_px,
                   "tiles_per_rank": len(tiles), "subset": args.subset,
                   "sharding": "LPT on pixel count, no collective on the data path" if world > 1 else None,
                   "conn": sorted({t.conn for t in tiles}),
                   "markers": "h-dome + fill-holes" if reset_j else "border (FillHoles)",
                   "l2": "flushed before each timed step (512 MiB write)", "bit_exact": "see tests -m gpu",
                   **params},
        "roofline": roof,
        "e2e": {"value": round(e2e, 2), "unit": "Mpix/s", "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
        # per step: init + persistent kernel, plus features, finalize and MLP forward
        # when learned, plus the marker kernel for FillHoles
        "gpu_launches": ((5 if learned else 2) + (0 if reset_j else 1)) * args.steps,
        "compare": compare,
        "clocks": clk.summary(),
    }
    if not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(w, tiles, shared, args.op)
    print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
