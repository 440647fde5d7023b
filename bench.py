#!/usr/bin/env python
"""Benchmark of the sliding-window-analysis hot path on GB300.

One step = one pass of the whole path over one image: build S and Q
(swa_build_sat), evaluate every window size of the workload on them
(swa_window_stats_multi) and release the tables (swa_free).

Default workload: the 70,000 x 85,000 uint8 synthetic microscopy image
(5.95e9 px, 95 GB of tables) with windows 256 and 1024 at stride 16.
``--workload 1`` runs the 20,000 x 20,000 image with windows 50/100/200 at
stride 1; 3 the batched engine on 256 uneven images; 4 the served request
stream; 5 the out-of-core banded path on a 70,000 x 85,000 uint16 image
(host to host).

Prints one JSON line.  ``value`` is image pixels per second of the whole step
(Gpx/s) with the image resident in HBM; ``e2e`` is the same metric through
``swa_analyze`` with the image in pinned host memory and the results copied
back to host memory inside the timed region.  ``--impl reference`` times the
CPU oracle on a bounded sample of the same workload instead.
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "SAT build Gpx/s + window outputs/s, % HBM peak; served p50/p99 vs plain path"
# Thread instructions per window (sum, mean, std; 2 windows per thread) of
# the window kernel, from ncu on the 12,288^2 stride-1 case
# (profiles/window_stats_dense_12288x12288.md): 1.8691e9 warp instructions x
# 31.99 active threads / 148.57 M windows.
INSTR_PER_WINDOW = 402.4
# The same for windows served from the corner lattice of the default
# workload (window areas 256^2 and 1024^2, powers of two: the divisions are
# exact shifts), from ncu on the 8,192 x 16,384 case with windows 256/1024 at
# stride 16 (profiles/window_stats_lattice_8192x16384.md): 8.8121e6 warp
# instructions x 31.43 active threads / 932,962 windows.
INSTR_PER_WINDOW_LATTICE_POW2 = 296.9
# The same for the batched engine's query kernel over the batched workload's
# mix (uint8 and uint16 images, windows 16-512 at strides 1-8, a quarter of
# them on the 128-bit path), from ncu on its first 8 images
# (profiles/batch_8images.md): 1.5378e9 warp instructions x 31.79 active
# threads / 112.6 M windows.
INSTR_PER_WINDOW_BATCH = 434.0
FALLBACK_HBM_GBS = 6800.0
NOMINAL_HBM_GBS = 7900.0   # GB300 HBM3e datasheet bandwidth, for context beside the measured peak


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=30)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", type=int, default=2, choices=[1, 2, 3, 4, 5])
    ap.add_argument("--band-rows", type=int, default=5000,
                    help="workload 5: rows per band (0: automatic)")
    ap.add_argument("--requests", type=int, default=200, help="workload 4: requests")
    ap.add_argument("--budget-gb", type=float, default=120.0, help="workload 4: HBM budget")
    ap.add_argument("--plain-steps", type=int, default=2,
                    help="passes of the plain per-request path (workload 3)")
    ap.add_argument("--no-tune", action="store_true", help="workload 3: default batch config")
    ap.add_argument("--e2e-steps", type=int, default=40)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-lattice", action="store_true",
                    help="build without the corner lattice the windows could use")
    ap.add_argument("--no-sub", action="store_true",
                    help="default workload: skip the batched and served sub-records")
    ap.add_argument("--cpu-rows", type=int, default=0,
                    help="rows of the CPU sample (0: CPU_SAMPLE_ROWS)")
    ap.add_argument("--twopass", action="store_true", help="force the two-pass SAT build")
    ap.add_argument("--shape", default="",
                    help="custom image RxC (profiling cases), e.g. 8192x8192")
    ap.add_argument("--dtype", default="u8", choices=["u8", "u16"],
                    help="pixel type of a --shape image")
    ap.add_argument("--threshold", type=int, default=None,
                    help="build the count table of pixels > THRESHOLD instead of S and Q "
                         "(windows then give count / fraction / indicator std)")
    ap.add_argument("--batch-images", type=int, default=0,
                    help="workload 3: use only the first N images (0: all 256)")
    ap.add_argument("--windows", default="",
                    help="custom windows w/stride list, e.g. 100/1,256/16")
    return ap.parse_args()


# ------------------------------------------------------------------ helpers --

def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return FALLBACK_HBM_GBS, "fallback"


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons while running."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id):
        self.gpu_id = gpu_id
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu_id), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        time.sleep(0.3)

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.2)
        self.proc.terminate()
        self.proc.wait()
        rows = []
        with open(self.path) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}

        def num(v):
            try:
                return float(v)
            except ValueError:
                return None
        sm = [num(r[1]) for r in rows if num(r[1]) is not None]
        mx = [num(r[2]) for r in rows if num(r[2]) is not None]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k] == "Active"})
        power = [num(r[3]) for r in rows if num(r[3]) is not None]
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons,
                "samples": len(rows), "power_w_max": max(power) if power else None}


def gpu_id_for_smi(local_rank):
    vis = os.environ.get("CUDA_VISIBLE_DEVICES")
    if vis:
        ids = [v.strip() for v in vis.split(",") if v.strip()]
        if local_rank < len(ids):
            return ids[local_rank]
    return local_rank


def max_over_ranks(value: float, device=None) -> float:
    """The maximum of `value` over all ranks (the slowest rank's time): the
    job's time under weak scaling.  Without a process group it is `value`."""
    import torch
    import torch.distributed as td
    if not (td.is_available() and td.is_initialized()) or td.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    td.all_reduce(t, op=td.ReduceOp.MAX)
    return float(t.item())


def job_throughput(units_per_rank: float, seconds: float, world: int) -> float:
    """Whole-job throughput: the units all ranks processed over the slowest
    rank's time."""
    return world * units_per_rank / seconds


def distinct_corner_bytes(rows, cols, wh, ww, sy, sx, tables):
    """Bytes of the distinct table entries a window query reads: rows
    {i*sy - 1, i*sy + wh - 1} x columns {j*sx - 1, j*sx + ww - 1} (index -1
    excluded), 8 bytes per entry per table."""
    R = (rows - wh) // sy + 1
    C = (cols - ww) // sx + 1
    i = np.arange(R, dtype=np.int64)
    j = np.arange(C, dtype=np.int64)
    ry = np.unique(np.concatenate([i * sy - 1, i * sy + wh - 1]))
    cx = np.unique(np.concatenate([j * sx - 1, j * sx + ww - 1]))
    return int((ry >= 0).sum()) * int((cx >= 0).sum()) * 8 * tables


def distinct_corner_bytes_all(rows, cols, windows, tables):
    """Bytes of the distinct table entries a set of window queries reads
    together: each query's corners are the product of its corner rows and
    corner columns, and the union of the products is counted by
    inclusion-exclusion over subsets of the queries."""
    import itertools
    sets = []
    for wh, ww, sy, sx in windows:
        i = np.arange((rows - wh) // sy + 1, dtype=np.int64)
        j = np.arange((cols - ww) // sx + 1, dtype=np.int64)
        ry = np.unique(np.concatenate([i * sy - 1, i * sy + wh - 1]))
        cx = np.unique(np.concatenate([j * sx - 1, j * sx + ww - 1]))
        sets.append((ry[ry >= 0], cx[cx >= 0]))
    total = 0
    for k in range(1, len(sets) + 1):
        for sub in itertools.combinations(sets, k):
            ry, cx = sub[0]
            for r2, c2 in sub[1:]:
                ry = np.intersect1d(ry, r2, assume_unique=True)
                cx = np.intersect1d(cx, c2, assume_unique=True)
            total += (-1) ** (k + 1) * len(ry) * len(cx)
    return total * 8 * tables


def traffic_record(kernel, case=None):
    """ncu DRAM bytes per launch for `kernel` on the workload `case` (e.g.
    "70000x85000 u8 S+Q lattice 16"), if a committed capture of that case is
    of the current source; else None.  A kernel's entry is one record or a
    list of them, one per captured case."""
    p = os.path.join(ROOT, "profiles", "dram_traffic.json")
    if not os.path.exists(p):
        return None
    import hashlib
    with open(p) as f:
        d = json.load(f)
    recs = d.get(kernel)
    if isinstance(recs, dict):
        recs = [recs]
    for e in recs or []:
        if e.get("full_case") != case:
            continue
        names = e["source"] if isinstance(e["source"], list) else [e["source"]]
        h = hashlib.sha256()
        for name in names:                   # the kernel's sources, in order
            src = os.path.join(ROOT, "paper_2410_16291_gb300", "csrc", name)
            if not os.path.exists(src):
                return None
            h.update(open(src, "rb").read())
        if h.hexdigest()[:16] != e["source_sha"]:
            return None
        return e["bytes_per_launch_full"]
    return None


# --------------------------------------------------------------- CPU legs --

# The CPU legs time the oracle on one fixed sample of the workload: its first
# CPU_SAMPLE_ROWS full-width rows (fewer if host memory is short), so the
# cpu_baseline record and the reference arm measure the same work.
CPU_SAMPLE_ROWS = 16384


def oracle_sample(sample, windows, par):
    """Time the CPU oracle on `sample` (full-width rows of the image): tables,
    then every window of the workload that fits.  par: the row-parallel
    variants on all threads, else the serial oracle."""
    import oracle
    sat = oracle.sat_par if par else oracle.sat
    win = oracle.window_sat_par if par else oracle.window_sat
    rows = sample.shape[0]
    t0 = time.perf_counter()
    S, Q = sat(sample)
    outs = 0
    for (wh, ww, sy, sx) in windows:
        if wh <= rows:
            outs += win(S, Q, wh, ww, sy, sx)["sum"].size
    dt = time.perf_counter() - t0
    return sample.size, outs, dt


def cpu_sample(im, windows, rows=0):
    """The fixed CPU sample of workload image `im` (numpy): its first `rows`
    (default CPU_SAMPLE_ROWS) full-width rows."""
    import synth
    free = None
    try:
        with open("/proc/meminfo") as f:
            for line in f:
                if line.startswith("MemAvailable:"):
                    free = int(line.split()[1]) * 1024
    except OSError:
        pass
    rows = rows or CPU_SAMPLE_ROWS
    if free:
        rows = min(rows, int(free * 0.3 / (18 * im.cols)))
    rows = max(rows, max(w[0] for w in windows))
    rows = min(rows, im.rows)
    gen = synth.intensity_u16 if im.dtype == "u16" else synth.intensity_u8
    return gen(rows, im.cols, im.seed, synth.cluster_count(rows, im.cols))


def cpu_baseline(im, windows, rows=0):
    """Both CPU legs on the same sample: the serial oracle on one core and
    its row-parallel variant on every host core."""
    import oracle
    sample = cpu_sample(im, windows, rows)
    cores = oracle.par_threads(os.cpu_count() or 1)
    oracle_sample(sample, windows, True)                 # warm-up (page faults, threads)
    par = [oracle_sample(sample, windows, True) for _ in range(3)]
    ser = [oracle_sample(sample, windows, False) for _ in range(2)]
    px = sample.size
    v_par = px * len(par) / sum(p[2] for p in par) / 1e9
    v_ser = px * len(ser) / sum(p[2] for p in ser) / 1e9
    return {"value": v_par, "unit": "Gpx/s", "cores": cores, "kind": "oracle",
            "sample": "%d x %d rows of the workload's generator (%.2e px): tables + the "
                      "workload's windows that fit (%d outputs); row-parallel oracle on %d "
                      "threads, %d runs, %.2f s each" % (
                          sample.shape[0], im.cols, px, par[0][1], cores, len(par),
                          sum(p[2] for p in par) / len(par)),
            "serial": {"value": v_ser, "unit": "Gpx/s", "cores": 1,
                       "sample": "the same sample, serial oracle, %d runs, %.2f s each" % (
                           len(ser), sum(p[2] for p in ser) / len(ser))}}


def workload_of(args):
    """The benchmark image: a standard workload, or a custom image for
    profiling cases (--shape / --dtype / --windows)."""
    import synth
    if args.shape:
        r, c = (int(v) for v in args.shape.lower().split("x"))
        wins = [synth.Window(int(w), int(w), int(s), int(s)) for w, s in
                (x.split("/") for x in (args.windows or "100/1").split(","))]
        return synth.Image(r, c, args.dtype, "intensity", synth.DEFAULT_SEED + 17,
                           synth.cluster_count(r, c), wins)
    (im,) = synth.workload(args.workload)
    if args.windows:
        im.windows = [synth.Window(int(w), int(w), int(s), int(s)) for w, s in
                      (x.split("/") for x in args.windows.split(","))]
    return im


def run_reference(args, rank, world):
    """The oracle on the host cores as the reference arm: each step is the
    CPU baseline's fixed sample, through the row-parallel oracle on every
    host core."""
    import oracle
    if rank != 0:
        return
    im = workload_of(args)
    windows = [(w.wh, w.ww, w.sy, w.sx) for w in im.windows]
    sample = cpu_sample(im, windows, args.cpu_rows)
    cores = oracle.par_threads(os.cpu_count() or 1)
    for _ in range(args.warmup):
        oracle_sample(sample, windows, True)
    tot_px, tot_out, tot_t = 0, 0, 0.0
    for _ in range(args.steps):
        px, outs, dt = oracle_sample(sample, windows, True)
        tot_px += px
        tot_out += outs
        tot_t += dt
    v = tot_px / tot_t / 1e9
    line = {"metric": METRIC, "value": v, "unit": "Gpx/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": tot_t / args.steps * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u64", "data": "synthetic",
            "impl": "reference",
            "config": config_of(im, windows),
            "window_outputs_per_s": tot_out / tot_t,
            "cpu_baseline": {"value": v, "unit": "Gpx/s", "cores": cores, "kind": "oracle",
                             "sample": "%d x %d rows per step (the CPU baseline's sample), "
                                       "row-parallel oracle on %d threads" % (
                                           sample.shape[0], im.cols, cores)},
            "e2e": {"value": v, "unit": "Gpx/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def config_of(im, windows, threshold=None):
    return {"workload": "%dx%d %s synthetic microscopy image, %d clusters" % (
        im.rows, im.cols, im.dtype, im.n_clusters),
        "windows": ["%dx%d/s%d" % (w[0], w[1], w[2]) for w in windows],
        "outputs": ("count,fraction,std of pixels > %d" % threshold if threshold is not None
                    else "sum,mean,std"),
        "tables": ("count table of pixels > %d, uint64" % threshold if threshold is not None
                   else "S and Q, uint64"),
        "l2": "inputs larger than L2 (image %.2f GB, tables %.1f GB)" % (
            im.pixels * (2 if im.dtype == "u16" else 1) / 1e9, 16 * im.pixels / 1e9)}


# ---------------------------------------------------------------- GPU legs --

def run_ours(args, rank, world, local_rank):
    import torch

    import paper_2410_16291_gb300 as swa
    import synth
    from paper_2410_16291_gb300 import build as swa_build
    swa_build.build()
    torch.cuda.set_device(local_rank)
    dist = world > 1
    if dist:
        import torch.distributed as td

    im = workload_of(args)
    windows = [(w.wh, w.ww, w.sy, w.sx) for w in im.windows]
    px = im.pixels
    u16 = im.dtype == "u16"
    host = torch.empty((im.rows, im.cols), dtype=torch.int16 if u16 else torch.uint8,
                       pin_memory=True)
    im.generate(out=host.numpy().view(np.uint16) if u16 else host.numpy())
    dev = host.to("cuda", non_blocking=True)
    stream = torch.cuda.current_stream()
    torch.cuda.synchronize()

    # Outputs, preallocated once.
    shapes = [swa.window_shape(im.rows, im.cols, *w) for w in windows]
    outs = [{"sum": torch.empty(s, dtype=torch.int64, device="cuda"),
             "mean": torch.empty(s, dtype=torch.float64, device="cuda"),
             "std": torch.empty(s, dtype=torch.float64, device="cuda")} for s in shapes]
    n_out = sum(R * C for R, C in shapes)

    # The corner lattice of the windows' common stride, when every window
    # can use it (strides (s, s), sides multiples of s, 8 <= s <= 255).
    lat = 0
    strides = {(w[2], w[3]) for w in windows}
    if len(strides) == 1 and not args.twopass and not args.no_lattice and args.threshold is None:
        sy, sx = strides.pop()
        if sy == sx and 8 <= sy <= 255 and all(w[0] % sy == 0 and w[1] % sy == 0
                                               for w in windows):
            lat = sy

    def step():
        if args.threshold is not None:
            sat = swa.build_count_sat(dev, args.threshold)
        else:
            sat = swa.build_sat(dev, with_sq=True, twopass=args.twopass, lattice=lat)
        sat.window_stats(windows, out=outs)
        sat.free()

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()

    clocks = Clocks(gpu_id_for_smi(local_rank))
    if rank == 0:
        clocks.start()
    if dist:
        td.barrier()
    torch.cuda.synchronize()
    l0 = swa.lib().swa_launch_count()
    swa.profile_begin()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        step()
    e1.record(stream)
    torch.cuda.synchronize()
    prof = swa.profile_end()
    launches = swa.lib().swa_launch_count() - l0
    if dist:
        td.barrier()
    ms = max_over_ranks(e0.elapsed_time(e1) / args.steps, device="cuda")
    clk = clocks.stop() if rank == 0 else None

    # Per-kernel averages and the dominant kernel's roofline.
    hbm, hbm_kind = peaks()
    tables = 2
    if args.threshold is not None:
        tables = 1                     # the count table serves as S and Q
    build_bytes = px * ((2 if u16 else 1) + 8 * tables)
    if lat:                  # the build also writes the two lattice arrays
        build_bytes += 2 * (im.rows // lat) * (im.cols // lat) * 8
    kernels = {}
    for name, (n, tot, mx) in prof.items():
        kernels[name] = {"launches": n, "avg_ms": tot / n, "share": 0.0}
    total_ms = sum(tot for (_, tot, _) in prof.values()) or 1.0
    for name, (n, tot, mx) in prof.items():
        kernels[name]["share"] = tot / total_ms
    dom = max(prof.items(), key=lambda kv: kv[1][1])[0] if prof else None
    bytes_per_launch = {"sat_build": build_bytes, "sat_scan": build_bytes,
                        "sat_reduce": px * 1}
    win_bytes = (distinct_corner_bytes_all(im.rows, im.cols, windows, tables) +
                 sum(24 * R * C for R, C in shapes))
    win_launches = kernels.get("window_stats", {}).get("launches", 0)
    bytes_per_launch["window_stats"] = win_bytes * args.steps / max(1, win_launches)
    roof = None
    if dom == "window_stats" and all(w[3] < 3 for w in windows):
        # Dense column strides: the exact mean/std arithmetic bounds the
        # kernel by instruction issue.  Peak = SMs x 4 schedulers x 32 lanes x
        # the SM clock sampled during the run; achieved = windows/s x the
        # instructions per window ncu measured for this kernel (sum, mean and
        # std at stride 1, profiles/window_stats_dense_12288x12288.md).
        n_win = sum(R * C for R, C in shapes)
        sms = torch.cuda.get_device_properties(local_rank).multi_processor_count
        mhz = (clk or {}).get("sm_mhz") or 2070.0
        peak_t = sms * 4 * 32 * mhz * 1e6 / 1e12
        ach_t = n_win / (kernels[dom]["avg_ms"] * win_launches / args.steps / 1e3) * \
            INSTR_PER_WINDOW / 1e12
        roof = {"bound": "alu", "kernel": dom, "achieved": ach_t, "peak": peak_t,
                "unit": "Tinst/s", "frac": ach_t / peak_t, "peak_kind": "issue rate at the "
                "sampled SM clock", "instructions_per_window": INSTR_PER_WINDOW,
                "traffic": None, "avg_ms": kernels[dom]["avg_ms"]}
    elif dom is not None and dom in bytes_per_launch:
        avg = kernels[dom]["avg_ms"]
        ach = bytes_per_launch[dom] / (avg / 1e3) / 1e9
        roof = {"bound": "hbm", "kernel": dom, "achieved": ach, "peak": hbm, "unit": "GB/s",
                "frac": ach / hbm, "peak_kind": hbm_kind,
                "frac_of_nominal": ach / NOMINAL_HBM_GBS, "nominal_peak": NOMINAL_HBM_GBS,
                "algorithmic_bytes_per_launch": bytes_per_launch[dom],
                "traffic": traffic_record(dom, "%dx%d %s %s" % (
                    im.rows, im.cols, im.dtype,
                    "count" if args.threshold is not None else
                    ("two-pass S+Q" if args.twopass else
                     "S+Q" + (" lattice %d" % lat if lat else "")))), "avg_ms": avg}
    # The window step beside the build: algorithmic bytes (outputs and the
    # distinct table entries the corners read, once) against HBM, and the
    # issue rate its exact arithmetic needs.
    win_roof = None
    if "window_stats" in kernels and kernels.get("window_stats", {}).get("launches"):
        w_ms = kernels["window_stats"]["avg_ms"] * win_launches / args.steps
        n_win = sum(R * C for R, C in shapes)
        mhz = (clk or {}).get("sm_mhz") or 2070.0
        sms = torch.cuda.get_device_properties(local_rank).multi_processor_count
        pow2 = all((w[0] * w[1]) & (w[0] * w[1] - 1) == 0 for w in windows)
        ipw = INSTR_PER_WINDOW_LATTICE_POW2 if (lat and pow2) else INSTR_PER_WINDOW
        win_roof = {"ms_per_step": w_ms, "windows": n_win,
                    "algorithmic_bytes": win_bytes, "bytes_per_window": win_bytes / n_win,
                    "hbm_achieved_gbs": win_bytes / (w_ms / 1e3) / 1e9,
                    "hbm_frac": win_bytes / (w_ms / 1e3) / 1e9 / hbm,
                    "instructions_per_window": ipw,
                    "issue_frac": n_win * ipw / (w_ms / 1e3) / (sms * 4 * 32 * mhz * 1e6),
                    "source": "corner lattice" if lat else "tables"}
    build_ms = sum(kernels[k]["avg_ms"] * kernels[k]["launches"] for k in kernels
                   if k.startswith("sat_")) / args.steps
    win_ms = sum(kernels[k]["avg_ms"] * kernels[k]["launches"] for k in kernels
                 if k.startswith("window")) / args.steps

    # End to end through swa_analyze with host buffers.
    e2e = None
    if not args.no_e2e and args.threshold is None:   # swa_analyze builds S and Q
        hout = [{"sum": torch.empty(s, dtype=torch.int64, pin_memory=True),
                 "mean": torch.empty(s, dtype=torch.float64, pin_memory=True),
                 "std": torch.empty(s, dtype=torch.float64, pin_memory=True)} for s in shapes]
        for _ in range(max(3, args.warmup)):        # first calls map pool memory
            swa.analyze(host, windows, out=hout)
        torch.cuda.synchronize()
        if dist:
            td.barrier()
        # Each call returns with its results on the host.  The pinned host
        # link's rate swings from call to call on a shared machine, so the
        # median, min and max call are reported beside the mean.
        times = []
        for _ in range(args.e2e_steps):
            t0 = time.perf_counter()
            swa.analyze(host, windows, out=hout)
            torch.cuda.synchronize()
            times.append(time.perf_counter() - t0)
        et = max_over_ranks(sum(times) / len(times), device="cuda")
        # The host link alone, for comparison: plain uploads of the same
        # pinned image (its bytes are most of what a call moves).
        link = []
        for _ in range(5):
            t0 = time.perf_counter()
            dev.copy_(host, non_blocking=True)
            torch.cuda.synchronize()
            link.append(time.perf_counter() - t0)
        med = statistics.median(times)
        e2e = {"value": job_throughput(px, et, world) / 1e9, "unit": "Gpx/s",
               "h2d_bytes_per_step": px, "d2h_bytes_per_step": 24 * n_out,
               "ms_per_step": et * 1e3, "steps": args.e2e_steps,
               "ms_median": 1e3 * med, "ms_min": 1e3 * min(times),
               "ms_max": 1e3 * max(times),
               "calls_over_1_5x_median": sum(1 for t in times if t > 1.5 * med),
               "link_upload_ms_median": 1e3 * statistics.median(link),
               "api": "swa_analyze (pinned host image in, pinned host results out; "
                      "host images of 256 MiB or more stream in bands)"}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(im, windows, args.cpu_rows)

    # The batched and served workloads, measured in the same run (one GPU,
    # default workload only) after this workload's memory is released.
    sub = {}
    if world == 1 and not args.no_sub and not args.shape and args.workload == 2 and \
            args.threshold is None:
        del dev, host, outs
        if e2e is not None:
            del hout
        torch.cuda.synchronize()
        torch.cuda.empty_cache()
        swa.lib().swa_trim(0)
        sub["batched"] = batch_measure(args, local_rank, steps=5, plain_steps=2)
        sub["served"] = serve_measure(args, local_rank, args.requests, args.budget_gb)

    if rank != 0:
        return
    value = job_throughput(px, ms / 1e3, world) / 1e9
    line = {"metric": METRIC, "value": value, "unit": "Gpx/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "u64", "data": "synthetic",
            "config": dict(config_of(im, windows, args.threshold), **(
                {"tables": "S and Q, uint64, with their corner lattice of stride %d" % lat}
                if lat else {})),
            "sat_build_gpx_s": px / (build_ms / 1e3) / 1e9 if build_ms else None,
            "sat_build_ms": build_ms, "window_ms": win_ms,
            "window_outputs_per_s": world * n_out / (ms / 1e3),
            "window_outputs_per_step": n_out,
            "roofline": roof, "window_roofline": win_roof, "kernels": kernels,
            "cpu_baseline": cpu, "e2e": e2e,
            "clocks": clk, "gpu_launches": launches, **sub,
            "build_path": "twopass" if args.twopass else "default",
            "lattice_stride": lat}
    print(json.dumps(line), flush=True)


def batch_measure(args, local_rank, steps, plain_steps, n_images=0, dist=False):
    """Workload 3: 256 uneven uint8/uint16 images with 1-4 queries each, all
    built and queried by one persistent launch replayed from a CUDA graph,
    against the plain per-request path (build, query, free per image, in
    order on one stream) on the same device-resident images and outputs.
    Returns the measurements as a dict (the batch pass's ms under ``ms``)."""
    import torch

    import paper_2410_16291_gb300 as swa
    import synth
    from paper_2410_16291_gb300 import tune
    if dist:
        import torch.distributed as td
    imgs = synth.workload(3)
    if n_images:
        imgs = imgs[:n_images]                    # a smaller batch (profiling)
    t0 = time.perf_counter()
    devs, wins = [], []
    for im in imgs:
        a = im.generate()
        t = torch.from_numpy(a.view(np.int16) if im.dtype == "u16" else a).cuda()
        devs.append(t)
        wins.append([(w.wh, w.ww, w.sy, w.sx) for w in im.windows])
    gen_s = time.perf_counter() - t0
    px = sum(im.pixels for im in imgs)
    n_out = sum(((im.rows - w.wh) // w.sy + 1) * ((im.cols - w.ww) // w.sx + 1)
                for im in imgs for w in im.windows)
    cfg = {"u8_tile_rows": 64, "order": 0} if args.no_tune else tune.tune(devs, wins)
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        b = swa.Batch(devs, wins, stream=stream, **cfg)
        for _ in range(max(3, args.warmup)):
            b.run(stream)
    stream.synchronize()
    b.sync()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=stream):
        b.run(stream)
    torch.cuda.synchronize()
    g.replay()
    torch.cuda.synchronize()

    clocks = Clocks(gpu_id_for_smi(local_rank))
    clocks.start()
    if dist:
        td.barrier()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with torch.cuda.stream(stream):
        e0.record(stream)
        for _ in range(steps):
            g.replay()
        e1.record(stream)
    torch.cuda.synchronize()
    b.sync()
    if dist:
        td.barrier()
    ms = max_over_ranks(e0.elapsed_time(e1) / steps, device="cuda")

    # Plain per-request path on the same images and output buffers.
    def plain_pass():
        for dev, wl, outs in zip(devs, wins, b.outputs):
            sat = swa.build_sat(dev, with_sq=True)
            sat.window_stats(wl, out=outs)
            sat.free()
    plain_pass()
    torch.cuda.synchronize()
    l0 = swa.lib().swa_launch_count()
    p0, p1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    p0.record()
    for _ in range(plain_steps):
        plain_pass()
    p1.record()
    torch.cuda.synchronize()
    plain_ms = p0.elapsed_time(p1) / plain_steps
    plain_launches = (swa.lib().swa_launch_count() - l0) // plain_steps
    clk = clocks.stop()

    # Per-kernel device time of both paths (event-bracketed launches, outside
    # the graph): where each path spends its step.
    def per_kernel(fn, reps):
        swa.profile_begin()
        for _ in range(reps):
            fn()
        torch.cuda.synchronize()
        return {k: {"launches": n // reps, "ms_per_pass": tot / reps}
                for k, (n, tot, _) in swa.profile_end().items()}

    def batch_pass():
        with torch.cuda.stream(stream):
            b.run(stream)
    batch_kernels = per_kernel(batch_pass, max(1, plain_steps))
    b.sync()
    plain_kernels = per_kernel(plain_pass, max(1, plain_steps))
    hbm, hbm_kind = peaks()
    build_algo = sum(im.pixels * ((2 if im.dtype == "u16" else 1) + 16) for im in imgs)
    build = batch_kernels.get("batch_build", {}).get("ms_per_pass")
    query = batch_kernels.get("batch_windows", {}).get("ms_per_pass")
    # The query kernel is bound by instruction issue: thread instructions it
    # needs per second against 152 SMs x 4 schedulers x 32 lanes x the
    # sampled SM clock.
    sms = torch.cuda.get_device_properties(local_rank).multi_processor_count
    issue_peak = sms * 4 * 32 * ((clk or {}).get("sm_mhz") or 2070.0) * 1e6
    q_rate = n_out * INSTR_PER_WINDOW_BATCH / (query / 1e3) if query else None
    rec = {"ms": ms, "gpx_s": px / (ms / 1e3) / 1e9,
           "window_outputs_per_s": n_out / (ms / 1e3),
           "images": len(imgs), "pixels": px, "window_outputs": n_out, "batch_config": cfg,
           "launch": "one persistent build launch + one query launch per pass, replayed as "
                     "one CUDA graph", "steps": steps,
           "build_ms": build, "query_ms": query,
           "build_hbm_frac": (build_algo / (build / 1e3) / 1e9 / hbm) if build else None,
           "build_algorithmic_bytes": build_algo, "peak_kind": hbm_kind,
           "query_issue_frac": q_rate / issue_peak if q_rate else None,
           "query_instructions_per_window": INSTR_PER_WINDOW_BATCH,
           "issue_peak_tinst_s": issue_peak / 1e12,
           "kernels": batch_kernels,
           "plain_path": {"ms_per_pass": plain_ms, "gpx_s": px / (plain_ms / 1e3) / 1e9,
                          "launches_per_pass": plain_launches, "kernels": plain_kernels,
                          "passes": plain_steps},
           "speedup_vs_plain": plain_ms / ms, "plan_bytes": b.nbytes(),
           "gpu_launches_per_pass": sum(v["launches"] for v in batch_kernels.values()),
           "host_generation_s": gen_s, "clocks": clk}
    b.free()
    del g, b, devs
    torch.cuda.synchronize()
    torch.cuda.empty_cache()
    swa.lib().swa_trim(0)
    return rec


def run_batch(args, rank, world, local_rank):
    """Workload 3 as the bench line (see batch_measure)."""
    import torch

    from paper_2410_16291_gb300 import build as swa_build
    swa_build.build()
    torch.cuda.set_device(local_rank)
    rec = batch_measure(args, local_rank, args.steps, args.plain_steps, args.batch_images,
                        dist=world > 1)
    if rank != 0:
        return
    ms = rec["ms"]
    hbm, hbm_kind = peaks()
    # The roofline of the pass's dominant kernel: the query kernel (bound by
    # instruction issue) or the build (bound by HBM), each on its own
    # event-timed duration; the other one's fraction stays beside it.
    build_roof = {"bound": "hbm", "kernel": "k_batch",
                  "achieved": rec["build_algorithmic_bytes"] / (rec["build_ms"] / 1e3) / 1e9,
                  "peak": hbm, "unit": "GB/s", "frac": rec["build_hbm_frac"],
                  "peak_kind": hbm_kind,
                  "algorithmic_bytes_per_launch": rec["build_algorithmic_bytes"],
                  "traffic": traffic_record("k_batch")}
    if rec["query_ms"] and rec["query_ms"] > rec["build_ms"]:
        peak_t = rec["issue_peak_tinst_s"]
        roof = {"bound": "alu", "kernel": "k_batch_windows",
                "achieved": rec["query_issue_frac"] * peak_t, "peak": peak_t,
                "unit": "Tinst/s", "frac": rec["query_issue_frac"],
                "peak_kind": "152 SMs x 4 schedulers x 32 lanes x sampled SM clock",
                "instructions_per_window": rec["query_instructions_per_window"],
                "traffic": None}
    else:
        roof = build_roof
    line = {"metric": METRIC, "value": world * rec["pixels"] / (ms / 1e3) / 1e9,
            "unit": "Gpx/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "u64", "data": "synthetic",
            "config": {"workload": "256 uneven synthetic images (sides 512-8192, aspect 0.5-2, "
                                   "uint8/uint16 50/50), 1-4 windows 16-512 px stride 1-8",
                       "images": rec["images"], "pixels": rec["pixels"],
                       "window_outputs": rec["window_outputs"],
                       "batch_config": rec["batch_config"], "launch": rec["launch"],
                       "l2": "inputs larger than L2 (%.1f GB of tables)" % (
                           16 * rec["pixels"] / 1e9)},
            "window_outputs_per_s": world * rec["window_outputs"] / (ms / 1e3),
            "kernels": rec["kernels"], "plain_path": rec["plain_path"],
            "speedup_vs_plain": rec["speedup_vs_plain"],
            "roofline": roof, "build_roofline": build_roof,
            "build_ms": rec["build_ms"], "query_ms": rec["query_ms"],
            "build_hbm_frac": rec["build_hbm_frac"], "plan_bytes": rec["plan_bytes"],
            "gpu_launches": args.steps * rec["gpu_launches_per_pass"],
            "host_generation_s": rec["host_generation_s"], "clocks": rec["clocks"],
            "cpu_baseline": None, "e2e": None}
    print(json.dumps(line), flush=True)


def serve_measure(args, local_rank, n_requests, budget_gb):
    """Workload 4: a Poisson request stream (200 req/s) over a pool of 64
    images (sides 1,000-40,000, uint8/uint16), each request 1-8 windows with
    sum/mean/std, served by the continuous-batching server under an HBM
    budget with resident tables, against the plain per-request path on the
    same trace.  Returns the measurements as a dict."""
    import torch

    import synth
    import paper_2410_16291_gb300 as swa
    from paper_2410_16291_gb300 import serve
    pool, trace = synth.serve_requests(n_requests, synth.DEFAULT_SEED + 4)
    t0 = time.perf_counter()
    host = {}
    for _, idx, _ in trace:                   # generated straight into pinned memory
        if idx in host:
            continue
        im = pool[idx]
        if im.dtype == "u16":
            t = torch.empty((im.rows, im.cols), dtype=torch.int16, pin_memory=True)
            im.generate(out=t.numpy().view(np.uint16))
        else:
            t = torch.empty((im.rows, im.cols), dtype=torch.uint8, pin_memory=True)
            im.generate(out=t.numpy())
        host[idx] = t
    gen_s = time.perf_counter() - t0

    def requests():
        return [serve.Request(k, idx, host[idx], [(w.wh, w.ww, w.sy, w.sx) for w in wl],
                              arrival=t) for k, (t, idx, wl) in enumerate(trace)]
    px = sum(pool[idx].pixels for _, idx, _ in trace)
    n_out = sum(((pool[idx].rows - w.wh) // w.sy + 1) * ((pool[idx].cols - w.ww) // w.sx + 1)
                for _, idx, wl in trace for w in wl)
    # Both paths run on streams created once, as a long-lived server's would
    # be; one untimed closed-loop pass of each first, so that PyTorch's
    # caching allocator (which keeps freed device blocks per stream) and the
    # library's memory pool already hold blocks for the staged images and
    # tables, as they do in steady state.
    streams = [torch.cuda.Stream() for _ in range(4)]
    plain_stream = torch.cuda.Stream()

    def served(realtime):
        srv = serve.Server(int(budget_gb * 1e9), streams=streams, slots=8,
                           keep_results=False)
        reqs = requests()
        l0 = swa.lib().swa_launch_count()
        t = srv.run(reqs, realtime=realtime)
        out = dict(serve.latency_summary(reqs), seconds=t, requests_per_s=len(reqs) / t,
                   window_outputs_per_s=n_out / t, cache_hits=srv.hits,
                   cache_misses=srv.misses, evictions=srv.evictions,
                   gpu_launches=swa.lib().swa_launch_count() - l0)
        srv.close()
        torch.cuda.synchronize()
        return t, out

    def plain(realtime):
        reqs = requests()
        t = serve.plain_path(reqs, realtime=realtime, stream=plain_stream, keep_results=False)
        torch.cuda.synchronize()
        return t, dict(serve.latency_summary(reqs), seconds=t, requests_per_s=len(reqs) / t,
                       window_outputs_per_s=n_out / t)
    served(False)
    plain(False)
    clocks = Clocks(gpu_id_for_smi(local_rank))
    clocks.start()
    # closed loop (every request submitted at t=0): throughput
    t_srv_c, srv_c = served(False)
    t_plain_c, plain_c = plain(False)
    # open loop (Poisson arrivals in real time): latency
    t_srv, srv = served(True)
    t_plain, plain_rt = plain(True)
    clk = clocks.stop()
    rec = {"requests": len(trace), "budget_gb": budget_gb, "streams": 4, "slots": 8,
           "image_pixels_requested": px, "window_outputs": n_out,
           "gpx_s": px / t_srv_c / 1e9,
           "served_closed_loop": srv_c, "plain_closed_loop": plain_c,
           "served_realtime": srv, "plain_realtime": plain_rt,
           "throughput_vs_plain": t_plain_c / t_srv_c,
           "p99_vs_plain_realtime": (plain_rt.get("p99_ms", 0) / srv["p99_ms"]
                                     if srv.get("p99_ms") else None),
           "host_generation_s": gen_s, "clocks": clk}
    del host
    torch.cuda.synchronize()
    torch.cuda.empty_cache()
    swa.lib().swa_trim(0)
    return rec


def run_serve(args, rank, world, local_rank):
    """Workload 4 as the bench line (see serve_measure)."""
    import torch

    from paper_2410_16291_gb300 import build as swa_build
    swa_build.build()
    torch.cuda.set_device(local_rank)
    if rank != 0:
        return
    rec = serve_measure(args, local_rank, args.requests, args.budget_gb)
    n = rec["requests"]
    t_srv_c = rec["served_closed_loop"]["seconds"]
    line = {"metric": METRIC, "value": rec["gpx_s"], "unit": "Gpx/s", "n_gpus": 1,
            "steps": n, "warmup": 1, "ms_per_step": t_srv_c / n * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u64",
            "data": "synthetic",
            "config": {"workload": "served: Poisson 200 req/s over 64 images (sides "
                                   "1,000-40,000, uint8/uint16), 1-8 windows 16-1024 px, "
                                   "stride 4-16, sum/mean/std",
                       "requests": n, "budget_gb": rec["budget_gb"], "streams": 4, "slots": 8,
                       "image_pixels_requested": rec["image_pixels_requested"],
                       "window_outputs": rec["window_outputs"],
                       "value": "closed loop: requested image pixels / makespan with "
                                "every request submitted at once"},
            "served_closed_loop": rec["served_closed_loop"],
            "plain_closed_loop": rec["plain_closed_loop"],
            "served_realtime": rec["served_realtime"], "plain_realtime": rec["plain_realtime"],
            "throughput_vs_plain": rec["throughput_vs_plain"],
            "p99_vs_plain_realtime": rec["p99_vs_plain_realtime"],
            "host_generation_s": rec["host_generation_s"],
            "window_outputs_per_s": rec["window_outputs"] / t_srv_c,
            "gpu_launches": rec["served_closed_loop"]["gpu_launches"], "clocks": rec["clocks"],
            "cpu_baseline": None, "e2e": None}
    print(json.dumps(line), flush=True)


def run_banded(args, rank, world, local_rank):
    """Workload 5: the 70,000 x 85,000 uint16 image (whose whole squared
    table could overflow uint64) through swa_analyze_banded, pinned host
    image in and host outputs out, windows 256 and 1024 at stride 16.  Every
    step moves the image over the host link, so value and e2e coincide; the
    link's bound is a plain pinned host-to-device copy of the image timed in
    the same run."""
    import torch

    import paper_2410_16291_gb300 as swa
    import synth
    from paper_2410_16291_gb300 import build as swa_build
    swa_build.build()
    torch.cuda.set_device(local_rank)
    dist = world > 1
    if dist:
        import torch.distributed as td
    r, c = 70000, 85000
    t0 = time.perf_counter()
    host = torch.empty((r, c), dtype=torch.int16, pin_memory=True)
    synth.intensity_u16(r, c, synth.DEFAULT_SEED + 5, 50000, out=host.numpy().view(np.uint16))
    gen_s = time.perf_counter() - t0
    windows = [(256, 256, 16, 16), (1024, 1024, 16, 16)]
    shapes = [swa.window_shape(r, c, *w) for w in windows]
    outs = [{"sum": torch.empty(sh, dtype=torch.int64, pin_memory=True),
             "mean": torch.empty(sh, dtype=torch.float64, pin_memory=True),
             "std": torch.empty(sh, dtype=torch.float64, pin_memory=True)} for sh in shapes]
    n_out = sum(R * C for R, C in shapes)
    px = r * c
    stream = torch.cuda.current_stream()

    def step():
        swa.analyze(host, windows, out=outs, stream=stream, band_rows=args.band_rows)
    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    clocks = Clocks(gpu_id_for_smi(local_rank))
    if rank == 0:
        clocks.start()
    if dist:
        td.barrier()
    l0 = swa.lib().swa_launch_count()
    swa.profile_begin()
    # Every step returns with its results on the host.  The pinned host
    # link's rate swings from step to step on a shared machine, so the
    # median, min and max step are reported beside the mean.
    times = []
    for _ in range(args.steps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        step()
        e1.record(stream)
        torch.cuda.synchronize()
        times.append(e0.elapsed_time(e1))
    prof = swa.profile_end()
    launches = swa.lib().swa_launch_count() - l0
    if dist:
        td.barrier()
    ms = max_over_ranks(sum(times) / len(times), device="cuda")
    clk = clocks.stop() if rank == 0 else None
    # The host link alone: the best of three pinned copies of the whole
    # image, device-timed.
    dev = torch.empty((r, c), dtype=torch.int16, device="cuda")
    dev.copy_(host, non_blocking=True)
    torch.cuda.synchronize()
    best = float("inf")
    for _ in range(3):
        c0, c1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        c0.record(stream)
        dev.copy_(host, non_blocking=True)
        c1.record(stream)
        torch.cuda.synchronize()
        best = min(best, c0.elapsed_time(c1))
    h2d_gbs = host.numel() * 2 / (best / 1e3) / 1e9
    del dev
    # Bytes over the link per step: the image once (a band's halo rows are
    # copied from the previous band on the device), every output out.  The
    # builds still process the halo rows.
    B = args.band_rows
    halo_rows = 0 if B else None       # the library picks B itself when 0
    if B:
        for b in range(1, -(-r // B)):
            tops = []
            for wh, _, sy, _ in windows:
                ib, ie = swa.band_range(r, wh, sy, B, b)
                if ib < ie:
                    tops.append(ib * sy)
            halo_rows += b * B - min(tops) if tops else 0
    h2d = r * c * 2
    d2h = 24 * n_out
    hbm, hbm_kind = peaks()
    kernels = {k: {"launches": n, "avg_ms": tot / n, "share": tot / max(1e-9, sum(
        t for _, t, _ in prof.values()))} for k, (n, tot, _) in prof.items()}
    build = kernels.get("sat_build", {"avg_ms": float("nan"), "launches": 0})
    band_px = (r + (halo_rows or 0)) * c / max(1, build["launches"] // args.steps)
    build_bytes = band_px * (2 + 16)
    if rank != 0:
        return
    value = job_throughput(px, ms / 1e3, world) / 1e9
    line = {"metric": METRIC, "value": value, "unit": "Gpx/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u64",
            "data": "synthetic",
            "config": {"workload": "70000x85000 u16 synthetic microscopy image, 50000 clusters, "
                                   "out-of-core banded analysis, pinned host image in, host "
                                   "outputs out",
                       "windows": ["256x256/s16", "1024x1024/s16"], "outputs": "sum,mean,std",
                       "band_rows": B, "halo_rows_per_step": halo_rows,
                       "l2": "inputs larger than L2 (image 11.9 GB)"},
            "window_outputs_per_s": world * n_out / (ms / 1e3),
            "step_ms": {"median": statistics.median(times), "min": min(times),
                        "max": max(times)},
            "kernels": kernels,
            "host_link": {"h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                          "achieved_gbs": (h2d + d2h) / (ms / 1e3) / 1e9,
                          "pinned_h2d_copy_gbs": h2d_gbs,
                          "frac": (h2d + d2h) / (ms / 1e3) / 1e9 / h2d_gbs},
            "roofline": {"bound": "hbm", "kernel": "sat_build",
                         "achieved": build_bytes / (build["avg_ms"] / 1e3) / 1e9,
                         "peak": hbm, "unit": "GB/s",
                         "frac": build_bytes / (build["avg_ms"] / 1e3) / 1e9 / hbm,
                         "peak_kind": hbm_kind, "algorithmic_bytes_per_launch": build_bytes,
                         "traffic": None},
            "cpu_baseline": None,
            "e2e": {"value": value, "unit": "Gpx/s", "h2d_bytes_per_step": h2d,
                    "d2h_bytes_per_step": d2h},
            "gpu_launches": launches, "host_generation_s": gen_s, "clocks": clk}
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    if world > 1:
        import torch
        import torch.distributed as td
        torch.cuda.set_device(local_rank)
        td.init_process_group("nccl", device_id=torch.device("cuda", local_rank))
    if args.workload == 3:
        run_batch(args, rank, world, local_rank)
    elif args.workload == 4:
        run_serve(args, rank, world, local_rank)
    elif args.workload == 5:
        run_banded(args, rank, world, local_rank)
    else:
        run_ours(args, rank, world, local_rank)
    if world > 1:
        import torch.distributed as td
        td.destroy_process_group()


if __name__ == "__main__":
    main()
