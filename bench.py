"""AIR benchmark: 512 x 512 split-Bregman AIR reconstructions per second on GB300.

Workload (the 512^2 configuration): 512 x 512 images of 0.8 mm pixels,
equiangular fan beam (source-isocentre 850 mm, source-detector 1450 mm),
738 bins, 800 views (full) and 200 views (25 %), seeded ellipse + disk
phantoms with Poisson noise at 2e4 photons/ray, lambda = 3e-4, mu = 1,
30 split-Bregman x 8 CG iterations.  One step = one batch of B slices (half
800-view, half 200-view) solved by air_solve_batch (grouped per-phase
launches captured in a CUDA graph, split-BF16 tensor-core filter).
value = slices/s on the device with inputs resident; e2e = the same through
the host-buffer call air_solve_batch_host, pinned sinograms copied in and
images copied out inside the timed region.  The batch's working set (~60 MB
per slice) exceeds L2 and L2 is also flushed between timed steps.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl air|reference]

Under torchrun each rank solves its own batches (no collective on the data
path: slices are independent) and rank 0 prints the JSON line with the max
time over ranks.
"""
from __future__ import annotations

import argparse
import dataclasses
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_1310_1434_gb300 import inputs  # noqa: E402

METRIC = "512^2 AIR slices/s (split-Bregman TF, 30x8, fan beam 738 bins, 800/200 views)"
UNIT = "slices/s"
PEAKS_PATH = os.path.join(ROOT, "MEASURED_PEAKS.json")


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="air", choices=["air", "reference"])
    ap.add_argument("--batch", type=int, default=8, help="slices per step (even: half 800, half 200 views)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--kernel", default=None,
                    choices=["fwd", "bwd", "ramp", "ramp_tc", "shrink", "solve", "plain", "batch"],
                    help="profiling mode: run one operator on the 512^2/800-view slice --reps times")
    ap.add_argument("--reps", type=int, default=3)
    ap.add_argument("--batch64", type=int, default=1,
                    help="also time the 64-slice batch of uneven geometry (0 skips it)")
    ap.add_argument("--serve-requests", type=int, default=500,
                    help="requests in each serving trace (0 skips the serving measurement)")
    return ap.parse_args()


def serve_trace(air, n_req: int, rate_hz: float, cache: dict, seed: int = 7):
    """Replays a bounded prefix of the serving trace (Poisson arrivals, sizes
    256/512/1024 x 200/400/800 views, 30x8 each, 120 GB budget) and returns
    latency percentiles and throughput.  Sinograms are generated before the
    clock starts, one per distinct geometry."""
    trace = inputs.serving_trace(count=n_req, rate_hz=rate_hz, seed=seed)
    data = []
    for t_arr, w in trace:
        key = (w.geom.n, w.geom.n_views)
        if key not in cache:
            cache[key] = inputs.make_case(w)[2].astype(np.float32).ravel()
        data.append((t_arr, w, cache[key]))
    srv = cache.setdefault("server", air.Server(120 * (1 << 30), max_slots=64))
    t0 = time.perf_counter()
    ids = []
    for t_arr, w, Y in data:
        dt = t0 + t_arr - time.perf_counter()
        if dt > 0:
            time.sleep(dt)
        ids.append((srv.submit(w.geom, Y, w.lam, w.mu, w.n_outer, w.n_cg), w))
    lat, lat512, ends, starts = [], [], [], []
    for rid, w in ids:
        while True:
            try:
                tm = srv.times(rid)
                break
            except air.AirError:
                time.sleep(0.0005)
        srv.poll(rid, w.geom.n)
        lat.append(tm[2] - tm[0])
        if w.geom.n == 512:
            lat512.append(tm[2] - tm[0])
        starts.append(tm[0])
        ends.append(tm[2])
    makespan = max(ends) - min(starts)
    return {"requests": n_req, "arrival_rate_hz": rate_hz,
            "requests_per_s": n_req / makespan, "makespan_s": makespan,
            "p50_ms": 1000 * float(np.percentile(lat, 50)), "p99_ms": 1000 * float(np.percentile(lat, 99)),
            "p50_ms_512": 1000 * float(np.percentile(lat512, 50)) if lat512 else None,
            "p99_ms_512": 1000 * float(np.percentile(lat512, 99)) if lat512 else None}


def serve_512(air, ws, Yh, rounds: int = 2):
    """The served form on the 512^2 slices alone: the benchmark's 8 slices
    (4 x 800, 4 x 200 views, split-BF16 filter) submitted together, `rounds`
    times, to one continuous-batching server (plans pooled by a first,
    untimed round).  Returns slices/s over the makespan, per-request latency
    percentiles, and the served images of the first timed round."""
    srv = air.Server(120 * (1 << 30), max_slots=64)
    geoms = [dataclasses.replace(w.geom, precision=1) for w in ws]
    for g, w, Y in zip(geoms, ws, Yh):                   # warm the plan pool
        srv.wait(srv.submit(g, Y, w.lam, w.mu, w.n_outer, w.n_cg), g.n)
    ids = []
    for _ in range(rounds):
        ids += [(srv.submit(g, Y, w.lam, w.mu, w.n_outer, w.n_cg), g) for g, w, Y in zip(geoms, ws, Yh)]
    lat, starts, ends, images = [], [], [], []
    for rid, g in ids:
        while True:
            try:
                tm = srv.times(rid)
                break
            except air.AirError:
                time.sleep(0.0005)
        images.append(srv.poll(rid, g.n))
        lat.append(tm[2] - tm[0])
        starts.append(tm[0])
        ends.append(tm[2])
    srv.close()
    makespan = max(ends) - min(starts)
    return {"requests": len(ids), "slices_per_s": len(ids) / makespan, "makespan_s": makespan,
            "p50_ms": 1000 * float(np.percentile(lat, 50)), "p99_ms": 1000 * float(np.percentile(lat, 99)),
            "precision": "split-BF16 filter (BF16X3)",
            "arrivals": f"{rounds} waves of the 8 benchmark slices submitted at once"}, images[:len(ws)]


def segment_count(geom) -> int:
    """nnz(A): ray-pixel intersections of every ray of the geometry.

    A line crossing a grid visits one cell more than the grid lines it
    crosses, so each ray clipped to the image square contributes
    |ix_out - ix_in| + |iy_out - iy_in| + 1 pixels (exact for rays through
    no grid vertex; a measure of the algorithmic work, not a step of A).
    """
    src, u = inputs.ray_lines(geom)
    half = 0.5 * geom.n * geom.pixel_mm
    sx, sy = np.broadcast_to(src[..., 0], u.shape[:2]), np.broadcast_to(src[..., 1], u.shape[:2])
    ux, uy = u[..., 0], u[..., 1]
    with np.errstate(divide="ignore", invalid="ignore"):
        tx0, tx1 = (-half - sx) / ux, (half - sx) / ux
        ty0, ty1 = (-half - sy) / uy, (half - sy) / uy
    t_in = np.maximum(np.minimum(tx0, tx1), np.minimum(ty0, ty1))
    t_out = np.minimum(np.maximum(tx0, tx1), np.maximum(ty0, ty1))
    hit = t_out > t_in
    to_px = lambda c: np.clip(np.floor((c + half) / geom.pixel_mm), 0, geom.n - 1)
    ix0, ix1 = to_px(sx + t_in * ux), to_px(sx + t_out * ux)
    iy0, iy1 = to_px(sy + t_in * uy), to_px(sy + t_out * uy)
    cells = np.abs(ix1 - ix0) + np.abs(iy1 - iy0) + 1
    return int(np.sum(np.where(hit, cells, 0)))


def run_kernel(args):
    """Runs one operator of the hot path --reps times (for ncu captures)."""
    import torch
    from paper_1310_1434_gb300 import air
    air.load()
    w = inputs.AIR512_V800
    g = w.geom
    ell, _, Y = inputs.make_case(w)
    X = inputs.rasterize(g, ell)
    plan = air.Plan(g)
    if args.kernel == "bwd":   # the view split bench.py's roofline times
        vpb, _, s_max = air.air_plan_config(plan)
        air.air_plan_tune(plan, vpb, min(BWD_PARTS, s_max))
    Yd = torch.as_tensor(Y.astype(np.float32).ravel(), device="cuda")
    Xd = torch.as_tensor(X.astype(np.float32).ravel(), device="cuda")
    Zd = torch.empty_like(Yd)
    X2 = torch.empty_like(Xd)
    b = torch.zeros(9 * g.n * g.n, device="cuda")
    gg = torch.empty_like(Xd)
    ops = {"fwd": lambda: air.air_project(plan, Xd, Zd),
           "bwd": lambda: air.air_backproject(plan, Yd, X2),
           "ramp": lambda: air.air_filter(plan, Yd, Zd),
           "shrink": lambda: air.air_shrink(plan, Xd, b, gg, w.lam / w.mu),
           "solve": lambda: air.air_solve(plan, Yd, w.lam, w.mu, w.n_outer, w.n_cg, X2),
           "plain": lambda: air.air_solve(plan, Yd, w.lam, w.mu, 1, 2, X2)}
    if args.kernel == "ramp_tc":   # the split-BF16 tensor-core filter
        plan_tc = air.Plan(dataclasses.replace(g, precision=1))
        ops["ramp_tc"] = lambda: air.air_filter(plan_tc, Yd, Zd)
    if args.kernel == "batch":   # the timed step: one batch as bench times it
        ws = workloads(max(2, args.batch), 0)
        Ys = [torch.as_tensor(inputs.make_case(v)[2].astype(np.float32).ravel(), device="cuda") for v in ws]
        Xs = [torch.empty(v.geom.n ** 2, device="cuda") for v in ws]
        bplans = [air.Plan(dataclasses.replace(v.geom, precision=1)) for v in ws]
        ops["batch"] = lambda: air.air_solve_batch(bplans, Ys, [v.lam for v in ws], [v.mu for v in ws],
                                                   [v.n_outer for v in ws], [v.n_cg for v in ws], Xs)
    for _ in range(args.reps):
        ops[args.kernel]()
    torch.cuda.synchronize()
    print(f"ran {args.kernel} x{args.reps}")


def max_over_ranks(values, dist, device):
    """Element-wise maximum of per-rank times over all ranks (a no-op alone)."""
    import torch
    t = torch.tensor([float(v) for v in values], dtype=torch.float64, device=device)
    if dist is not None:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return [float(x) for x in t]


def workloads(batch: int, rank: int):
    out = []
    for i in range(batch):
        base = inputs.AIR512_V800 if i % 2 == 0 else inputs.AIR512_V200
        seed = 1 + i // 2 + 1000 * rank
        out.append(inputs.Workload(f"{base.name}_s{seed}", base.geom, seed, base.n_ellipses, base.n_disks,
                                   base.photons, base.lam, base.mu, base.n_outer, base.n_cg))
    return out


def load_peaks():
    try:
        with open(PEAKS_PATH) as f:
            p = json.load(f)
        return {"hbm_gbs": float(p["hbm_gbs"]), "bf16_tflops": float(p["bf16_tflops"]),
                "sm_max_mhz": float(p.get("sm_max_mhz", 2070.0)), "src": "measured"}
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0, "src": "fallback"}


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""
    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.thread.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 7:
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
            except ValueError:
                continue
            for nm, val in zip(names, parts[3:7]):
                if val.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": float(max(smax)) if smax else None,
                "samples": len(sm), "reasons": sorted(reasons)}


def events_time(torch, stream, fn, reps: int) -> float:
    """Average ms of fn() over reps launches on `stream`, CUDA events on that stream."""
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    a.record(stream)
    for _ in range(reps):
        fn()
    b.record(stream)
    b.synchronize()
    return a.elapsed_time(b) / reps


def oracle_outer_step_seconds(oracle, w):
    """Measured seconds of the oracle's split-Bregman solve of workload w:
    its A'^T Y (once) and ONE outer step (the CG of n_cg steps with its
    true-residual restart, i.e. n_cg + 1 operator pairs, and the shrink),
    timed on this host's cores.  Every outer step of the oracle does the same
    work, so a full solve takes rhs + n_outer * outer."""
    og = oracle.Geometry(**{k: getattr(w.geom, k) for k in oracle.Geometry.__dataclass_fields__})
    Y = inputs.make_case(w)[2].astype(np.float32).astype(np.float64)
    t = time.perf_counter()
    rhs0 = oracle.filtered_backproject(og, Y)
    t_rhs = time.perf_counter() - t
    t = time.perf_counter()
    X = oracle.cg(og, rhs0, w.mu, w.n_cg, X0=np.zeros((w.geom.n, w.geom.n)))
    oracle.shrink(X, np.zeros((9, w.geom.n, w.geom.n)), w.lam / w.mu)
    t_outer = time.perf_counter() - t
    return t_rhs, t_outer


_ONE_THREAD_SOLVE = """
import sys, time
sys.path.insert(0, sys.argv[1])
import numpy as np, oracle
from paper_1310_1434_gb300 import inputs
w = inputs.AIR128
og = oracle.Geometry(**{k: getattr(w.geom, k) for k in oracle.Geometry.__dataclass_fields__})
Y = inputs.make_case(w)[2].astype(np.float32).astype(np.float64)
t = time.perf_counter()
oracle.solve(og, Y, w.lam, w.mu, w.n_outer, w.n_cg)
print(oracle.threads(), time.perf_counter() - t)
"""


def oracle_one_thread_seconds():
    """The oracle's full 128^2 solve on one host thread (OpenMP limited to one
    thread in a child process), or None if the child fails."""
    env = dict(os.environ, OMP_NUM_THREADS="1")
    try:
        out = subprocess.run([sys.executable, "-c", _ONE_THREAD_SOLVE, ROOT], env=env, capture_output=True,
                             text=True, timeout=300, check=True).stdout.split()
        return {"threads": int(out[0]), "air128_v90_full_solve_s": float(out[1])}
    except (subprocess.SubprocessError, OSError, ValueError, IndexError):
        return None


def cpu_baseline(gpu):
    """The FP64 oracle (as it stands) on this host's cores.  Measured: one
    full split-Bregman solve of the 128^2 configuration (20 x 5), and for
    each 512^2 slice (800 and 200 views, 30 x 8) its A'^T Y and one whole
    outer step, which give the full solve exactly (every outer step does the
    same work).  value = slices/s of the benchmark's 50/50 mix of 800- and
    200-view slices.  The oracle's recorded full solves of the same slices
    (tests/golden, written by the oracle) are quoted with their thread count.
    The oracle's outputs also give the GPU's single-application errors, and
    the stored reconstructions the final-image errors."""
    import oracle
    oracle.build()
    w0 = inputs.AIR128
    og0 = oracle.Geometry(**{k: getattr(w0.geom, k) for k in oracle.Geometry.__dataclass_fields__})
    Y0 = inputs.make_case(w0)[2].astype(np.float32).astype(np.float64)
    t = time.perf_counter()
    oracle.solve(og0, Y0, w0.lam, w0.mu, w0.n_outer, w0.n_cg)
    t_c0 = time.perf_counter() - t
    one = oracle_one_thread_seconds()
    if one is not None:
        one["speedup_of_all_threads"] = one["air128_v90_full_solve_s"] / t_c0
    per = {}
    for w in (inputs.AIR512_V800, inputs.AIR512_V200):
        t_rhs, t_outer = oracle_outer_step_seconds(oracle, w)
        per[w.name] = {"rhs_s": t_rhs, "outer_step_s": t_outer, "solve_s": t_rhs + w.n_outer * t_outer}
    t_mix = 0.5 * (per["air512_v800"]["solve_s"] + per["air512_v200"]["solve_s"])
    recorded = {}
    for name in ("air512_v800", "air512_v200"):
        path = os.path.join(ROOT, "tests", "golden", f"{name}_oracle.npz")
        if os.path.exists(path):
            d = np.load(path)
            recorded[name] = {"solve_s": float(d["seconds"]), "threads": int(d["threads"])}

    w = inputs.AIR512_V800
    og = oracle.Geometry(**{k: getattr(w.geom, k) for k in oracle.Geometry.__dataclass_fields__})
    ell, _, Y = inputs.make_case(w)
    Y = Y.astype(np.float32).astype(np.float64)
    X = inputs.rasterize(w.geom, ell).astype(np.float32).astype(np.float64)
    A_o = oracle.project(og, X)
    ATC_o = oracle.filtered_backproject(og, Y)

    def rel(a, b):
        return float(np.linalg.norm(np.asarray(a, np.float64).ravel() - b.ravel()) / np.linalg.norm(b))

    prec = {"A_fp32": rel(gpu["A"], A_o), "ATC_fp32": rel(gpu["ATC_fp32"], ATC_o),
            "ATC_bf16x3": rel(gpu["ATC_bf16x3"], ATC_o)}
    for key, name in (("X_v800", "air512_v800"), ("X_v200", "air512_v200")):
        path = os.path.join(ROOT, "tests", "golden", f"{name}_oracle.npz")
        if key in gpu and os.path.exists(path):
            prec[f"final_{name}_bf16x3_batched"] = rel(gpu[key], np.load(path)["X"].astype(np.float64))
        skey = f"served_{key}"
        if skey in gpu and os.path.exists(path):
            prec[f"final_{name}_bf16x3_served"] = rel(gpu[skey], np.load(path)["X"].astype(np.float64))
    return {"value": 1.0 / t_mix, "unit": UNIT, "cores": oracle.threads(), "kind": "oracle (measured)",
            "sample": (f"FP64 oracle, measured on {oracle.threads()} threads: the 128^2 solve in full "
                       f"({t_c0:.2f} s); per 512^2 slice A'^T Y and one outer step of 30 "
                       f"(800 views {per['air512_v800']['outer_step_s']:.2f} s, 200 views "
                       f"{per['air512_v200']['outer_step_s']:.2f} s), x 30 for the full solve, "
                       "weighted 50/50 over 800 and 200 views as the benchmark's batch"),
            "seconds_per_slice": t_mix,
            "per_config_s": {"air128_v90_full_solve": t_c0,
                             **{k: v["solve_s"] for k, v in per.items()}},
            "per_config_detail": per,
            "one_thread": one,
            "recorded_full_solves": recorded}, prec


def run_reference(args, rank, world):
    """The reference arm: the FP64 CPU oracle, timed on this host's cores on
    the benchmark's workload.  One step = one outer split-Bregman step (its
    CG with the true-residual restart, n_cg + 1 operator pairs, and the
    shrink) of a 512^2 slice, alternately of 800 and of 200 views (both in a
    run of one step).  A full solve is A'^T Y (timed once) plus 30 such outer
    steps, and value = slices/s of the 50/50 mix."""
    if rank != 0:
        return
    import oracle
    oracle.build()
    ws = (inputs.AIR512_V800, inputs.AIR512_V200)
    prep = []
    for w in ws:
        og = oracle.Geometry(**{k: getattr(w.geom, k) for k in oracle.Geometry.__dataclass_fields__})
        Y = inputs.make_case(w)[2].astype(np.float32).astype(np.float64)
        t = time.perf_counter()
        rhs0 = oracle.filtered_backproject(og, Y)
        prep.append((w, og, rhs0, time.perf_counter() - t))

    def outer(kind):
        w, og, rhs0, _ = prep[kind]
        t = time.perf_counter()
        X = oracle.cg(og, rhs0, w.mu, w.n_cg, X0=np.zeros((w.geom.n, w.geom.n)))
        oracle.shrink(X, np.zeros((9, w.geom.n, w.geom.n)), w.lam / w.mu)
        return time.perf_counter() - t

    for i in range(args.warmup):
        outer(i % 2)
    times = {0: [], 1: []}
    step_s = []
    for i in range(args.steps):
        kinds = (0, 1) if args.steps == 1 else (i % 2,)
        t = 0.0
        for k in kinds:
            dt = outer(k)
            times[k].append(dt)
            t += dt
        step_s.append(t)
    if not times[1]:
        times[1].append(outer(1))
    solve = [p[3] + w.n_outer * float(np.mean(times[k])) for k, (p, w) in enumerate(zip(prep, ws))]
    value = 2.0 / float(sum(solve))
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000 * float(np.mean(step_s)),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": "air512: 512x512 0.8 mm, 738 bins, 800 and 200 views, 30x8 split-Bregman",
                       "views_mix": "half 800, half 200"},
            "cpu_baseline": {"kind": "oracle (measured)", "cores": oracle.threads(), "value": value, "unit": UNIT,
                             "sample": ("per step one outer split-Bregman step of a 512^2 slice, alternately with "
                                        "800 and 200 views; full solve = A'^T Y + 30 outer steps: "
                                        f"{solve[0]:.1f} s (800 views), {solve[1]:.1f} s (200 views)")},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    if args.kernel:
        run_kernel(args)
        return
    import torch
    from paper_1310_1434_gb300 import air

    assert torch.cuda.is_available(), "bench.py needs a CUDA device"
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    air.load()
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream(dev)
    B = max(2, args.batch)

    # ---- inputs: seeded synthetic sinograms, resident on the device ----
    ws = workloads(B, rank)
    Yh = [inputs.make_case(w)[2].astype(np.float32).ravel() for w in ws]
    Yd = [torch.as_tensor(y, device=dev) for y in Yh]
    Xd = [torch.empty(w.geom.n ** 2, device=dev) for w in ws]
    # the served/batched mixed-precision form: split-BF16 tensor-core filter
    plans = [air.Plan(dataclasses.replace(w.geom, precision=1)) for w in ws]
    plans32 = [air.Plan(w.geom) for w in ws]
    lam = [w.lam for w in ws]
    mu = [w.mu for w in ws]
    no = [w.n_outer for w in ws]
    ncg = [w.n_cg for w in ws]
    flush = torch.empty(256 * 1024 * 1024 // 4, device=dev)   # > L2 (129 MB)

    def step():
        air.air_solve_batch(plans, Yd, lam, mu, no, ncg, Xd)

    for _ in range(max(3, args.warmup)):
        step()
    torch.cuda.synchronize()
    # kernels per step, as the library counted them in the graph it chose
    # (one per grouped phase launch of each chain, two per tensor-core filter
    # application)
    graph_chains, launches_per_step = air.air_batch_graph_info()

    # ---- timed region: device-resident inputs ----
    clocks = ClockSampler(local)
    clocks.start()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    ms = []
    for _ in range(args.steps):
        flush.zero_()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        step()
        b.record(stream)
        b.synchronize()
        ms.append(a.elapsed_time(b))
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    total_ms = float(sum(ms))

    final_images = {"X_v800": Xd[0].cpu().numpy(), "X_v200": Xd[1].cpu().numpy()}

    # ---- e2e: the host-buffer C-ABI call (air_solve_batch_host), pinned host
    # sinograms in and images out inside the timed region ----
    Yp = [torch.from_numpy(y).pin_memory() for y in Yh]
    Xp = [torch.empty(w.geom.n ** 2, pin_memory=True) for w in ws]
    air.air_solve_batch_host(plans, Yp, lam, mu, no, ncg, Xp)     # captures the host-buffer graph
    host_chains = air.air_batch_graph_info()[0]
    e2e_ms = []
    for _ in range(args.steps):
        flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        air.air_solve_batch_host(plans, Yp, lam, mu, no, ncg, Xp)
        e2e_ms.append(1000 * (time.perf_counter() - t0))
    clk = clocks.stop()
    h2d = sum(y.nbytes for y in Yh)
    d2h = sum(x.numel() * 4 for x in Xp)

    # ---- the other forms on the same batch (device-resident, L2 flushed) ----
    def form_rate(fn, reps=2):
        fn()
        t = []
        for _ in range(reps):
            flush.zero_()
            t.append(events_time(torch, stream, fn, 1))
        return B * 1000.0 / float(np.mean(t))

    forms = {
        "batched_bf16x3_graph": None,
        "batched_fp32_graph": form_rate(lambda: air.air_solve_batch(plans32, Yd, lam, mu, no, ncg, Xd)),
        "batched_fp32_persistent": form_rate(
            lambda: air.air_solve_batch_persistent(plans32, Yd, lam, mu, no, ncg, Xd)),
    }

    # ---- the 64-slice batch of uneven geometry (256^2/200 views, 512^2/400,
    # 512^2/800, 768^2/800 bins 384/738/738/1024; seeds 100..163), FP32 ----
    config64 = None
    if args.batch64:
        w64 = inputs.batch_workloads(64, first_seed=100 + 1000 * rank)
        Y64 = [torch.as_tensor(inputs.make_case(w)[2].astype(np.float32).ravel(), device=dev) for w in w64]
        t0 = time.perf_counter()
        p64 = [air.Plan(w.geom) for w in w64]
        t_plans = time.perf_counter() - t0
        X64 = [torch.empty(w.geom.n ** 2, device=dev) for w in w64]
        args64 = ([w.lam for w in w64], [w.mu for w in w64], [w.n_outer for w in w64], [w.n_cg for w in w64])
        config64 = {"slices": 64, "shapes": "16 each of 256^2/200, 512^2/400, 512^2/800, 768^2/800",
                    "plan_create_s": t_plans}
        for form, fn in (("grouped_graph", air.air_solve_batch), ("persistent", air.air_solve_batch_persistent)):
            fn(p64, Y64, *args64[:2], *args64[2:], X64)          # first call builds and captures the graph
            flush.zero_()
            t = events_time(torch, stream, lambda: fn(p64, Y64, *args64[:2], *args64[2:], X64), 1)
            config64[f"{form}_slices_per_s"] = 64 * 1000.0 / t
            config64[f"{form}_ms"] = t
        del p64, X64, Y64

    # ---- serving: continuous batching of the Poisson trace (sizes
    # 256/512/1024 x 200/400/800 views), and the 512^2 slices alone ----
    serving = None
    served_images = {}
    if args.serve_requests > 0:
        cache = {}
        serve_trace(air, 9, 1000.0, cache, seed=11)              # warm-up: fills the plan pool
        stated = serve_trace(air, args.serve_requests, 200.0, cache)
        sustain = serve_trace(air, args.serve_requests, 0.7 * stated["requests_per_s"], cache, seed=8)
        cache["server"].close()
        s512, imgs = serve_512(air, ws, Yh)
        served_images = {"served_X_v800": imgs[0], "served_X_v200": imgs[1]}
        serving = {"stated_rate_200_per_s": stated, "sustainable_rate": sustain, "served_512": s512,
                   "note": (f"first {args.serve_requests} requests of the 2000-request trace (seed 7) at the "
                            "stated 200/s, which exceeds capacity (latency there is mostly queueing), and at "
                            "0.7 x the throughput that run reached (seed 8); served_512: the benchmark's "
                            "512^2 slices through the server, compared with the oracle in "
                            "precision_vs_fp64_oracle")}

    # ---- the 128^2 configuration (90 views, 192 bins, lambda 0.01, mu 1,
    # 20 x 5): plain single-slice solves and a grouped batch of 16 slices ----
    w0 = inputs.AIR128
    p0 = air.Plan(w0.geom)
    Y0 = torch.as_tensor(inputs.make_case(w0)[2].astype(np.float32).ravel(), device=dev)
    X0 = torch.empty(w0.geom.n ** 2, device=dev)
    air.air_solve(p0, Y0, w0.lam, w0.mu, w0.n_outer, w0.n_cg, X0)
    t0_plain = events_time(torch, stream, lambda: air.air_solve(p0, Y0, w0.lam, w0.mu, w0.n_outer, w0.n_cg, X0), 5)
    w16 = [dataclasses.replace(w0, seed=w0.seed + k) for k in range(16)]
    Y16 = [torch.as_tensor(inputs.make_case(w)[2].astype(np.float32).ravel(), device=dev) for w in w16]
    p16 = [air.Plan(w.geom) for w in w16]
    X16 = [torch.empty(w0.geom.n ** 2, device=dev) for _ in w16]
    a16 = ([w.lam for w in w16], [w.mu for w in w16], [w.n_outer for w in w16], [w.n_cg for w in w16])
    air.air_solve_batch(p16, Y16, *a16, X16)
    t0_batch = events_time(torch, stream, lambda: air.air_solve_batch(p16, Y16, *a16, X16), 3)
    config0 = {"workload": "air128_v90: 128x128 1 mm, 192 bins, 90 views, lambda 0.01, mu 1, 20x5",
               "plain_ms_per_slice": t0_plain, "plain_slices_per_s": 1000.0 / t0_plain,
               "batch16_ms": t0_batch, "batch16_slices_per_s": 16 * 1000.0 / t0_batch}
    del p16, X16, Y16

    # ---- plain single-slice path: one air_solve per slice, per-slice latency ----
    lat = {800: [], 200: []}
    for i in range(min(B, 4)):
        w = ws[i]
        for _ in range(2):
            flush.zero_()
            t = events_time(torch, stream, lambda: air.air_solve(plans32[i], Yd[i], w.lam, w.mu, w.n_outer,
                                                                  w.n_cg, Xd[i]), 1)
            lat[w.geom.n_views].append(t)
    plain_ms = [t for v in lat.values() for t in v]

    # ---- the next rows: L2-regularised AIR (Eq. 5) and forward-backward
    # splitting AIR (Eq. 6), single slice, 240 operator pairs each (as the
    # 30 x 8 split-Bregman solve) ----
    n_pairs = ws[0].n_outer * ws[0].n_cg
    xl = torch.randn(ws[0].geom.n ** 2, device=dev)
    xl /= xl.norm()
    xl2 = torch.empty_like(xl)
    yl = torch.empty(ws[0].geom.n_views * ws[0].geom.n_bins, device=dev)
    lip = 1.0
    for _ in range(10):   # power iteration for ||A'^T A||; the forward-backward step is its inverse
        air.air_project(plans32[0], xl, yl)
        air.air_filtered_backproject(plans32[0], yl, xl2)
        lip = float(xl2.norm())
        xl = xl2 / lip
    step = 1.0 / lip
    next_rows = {"slice": "512^2 / 800 views", "operator_pairs": n_pairs, "fbs_step": step}
    for tag, pl in (("fp32", plans32[0]), ("bf16x3", plans[0])):
        t_l2 = events_time(torch, stream, lambda: air.air_solve_l2(pl, Yd[0], ws[0].lam * 100, n_pairs, Xd[0]), 2)
        t_fbs = events_time(torch, stream, lambda: air.air_solve_fbs(pl, Yd[0], ws[0].lam, step, n_pairs, Xd[0]), 2)
        next_rows[f"l2_air_ms_{tag}"] = t_l2
        next_rows[f"fbs_air_ms_{tag}"] = t_fbs
    xf = torch.empty_like(Xd[0])
    air.air_fbp(plans32[0], Yd[0], xf)
    next_rows["fbp_ms"] = events_time(torch, stream, lambda: air.air_fbp(plans32[0], Yd[0], xf), 5)
    next_rows["l2_lambda"] = ws[0].lam * 100
    next_rows["fbs_lambda"] = ws[0].lam

    # ---- dominant kernel: the backprojector on a 512^2/800 slice ----
    p800 = plans32[0]
    g8 = ws[0].geom
    zin = Yd[0]
    xout = torch.empty(g8.n ** 2, device=dev)
    air.air_backproject(p800, zin, xout)
    t_bwd_tuned = events_time(torch, stream, lambda: air.air_backproject(p800, zin, xout), 20)
    # the roofline's configuration: BWD_PARTS view parts in one k_op<OP_BWD>
    # launch plus their sum (k_op<OP_BWD_FIN>), as `--kernel bwd` runs it for
    # the ncu capture
    vpb, s_tuned, s_max = air.air_plan_config(p800)
    s_rf = min(BWD_PARTS, s_max)
    air.air_plan_tune(p800, vpb, s_rf)
    air.air_backproject(p800, zin, xout)
    t_bwd = events_time(torch, stream, lambda: air.air_backproject(p800, zin, xout), 20)
    air.air_plan_tune(p800, vpb, s_tuned)
    yout = torch.empty(g8.n_views * g8.n_bins, device=dev)
    air.air_project(p800, Xd[0], yout)
    t_fwd = events_time(torch, stream, lambda: air.air_project(p800, Xd[0], yout), 20)
    alg_bytes = 4 * (g8.n ** 2 + g8.n_views * g8.n_bins)       # read Z + write X (fwd: read X + write Y)
    # single applications on the phantom and the measured sinogram, for the
    # precision report (compared with the oracle in the CPU-baseline leg)
    ell0 = inputs.random_phantom(g8, ws[0].seed, ws[0].n_ellipses, ws[0].n_disks)
    Xph = torch.as_tensor(inputs.rasterize(g8, ell0).astype(np.float32).ravel(), device=dev)
    A_g = torch.empty(g8.n_views * g8.n_bins, device=dev)
    air.air_project(p800, Xph, A_g)
    atc32 = torch.empty(g8.n ** 2, device=dev)
    atc16 = torch.empty(g8.n ** 2, device=dev)
    air.air_filtered_backproject(p800, Yd[0], atc32)
    air.air_filtered_backproject(plans[0], Yd[0], atc16)
    torch.cuda.synchronize()
    gpu_out = {"A": A_g.cpu().numpy(), "ATC_fp32": atc32.cpu().numpy(), "ATC_bf16x3": atc16.cpu().numpy(),
               **final_images, **served_images}
    peaks = load_peaks()
    # issue-limited roofline of the backprojector: algorithmic work = nnz(A)
    # segment evaluations per application; peak = SMs x 4 warp issues/clk x
    # 32 lanes x max SM clock / SEG_INST thread-instructions per segment
    nnz = segment_count(g8)
    seg_peak = 152 * 4 * 32 * peaks["sm_max_mhz"] * 1e6 / SEG_INST / 1e9     # Gsegment/s
    sm_mhz = clk.get("sm_mhz") or peaks["sm_max_mhz"]

    # ---- reduce over ranks (max time) ----
    total_ms, e2e_total = max_over_ranks([total_ms, float(np.sum(e2e_ms))], dist, dev)
    slices = B * args.steps * world
    value = slices / (total_ms / 1000.0)
    e2e_value = slices / (e2e_total / 1000.0)
    forms["batched_bf16x3_graph"] = B * args.steps / (float(sum(ms)) / 1000.0)

    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return
    cpu, prec = None, None
    if not args.no_cpu_baseline and world == 1:
        cpu, prec = cpu_baseline(gpu_out)
    line = {
        "metric": METRIC,
        "value": value,
        "unit": UNIT,
        "n_gpus": world,
        "steps": args.steps,
        "warmup": max(3, args.warmup),
        "ms_per_step": total_ms / args.steps,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f32, filter split-bf16x6 -> fp32",
        "data": "synthetic",
        "config": {"workload": "air512: 512x512 0.8 mm, 738 bins, 800 and 200 views, 30x8 split-Bregman",
                   "slices_per_step": B, "views_mix": "half 800, half 200",
                   "form": "air_solve_batch: grouped per-phase launches in a CUDA graph, BF16X3 filter",
                   "l2": "flushed between timed steps (256 MB write); working set > L2",
                   "parallelism": f"slices sharded over {world} GPU(s), no collective"},
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                "ms_per_step": [round(t, 2) for t in e2e_ms]},
        "gpu_launches": args.steps * launches_per_step,
        "batch_graph": {"chains": graph_chains, "kernels_per_step": launches_per_step,
                        "host_buffer_chains": host_chains},
        "forms_slices_per_s": forms,
        "clocks": clk,
        "plain_gpu": {"path": "air_solve, one slice at a time",
                      "slices_per_s": 1000.0 * len(plain_ms) / sum(plain_ms),
                      "p50_ms": float(np.percentile(plain_ms, 50)), "p99_ms": float(np.percentile(plain_ms, 99)),
                      "ms_800_views": float(np.mean(lat[800])) if lat[800] else None,
                      "ms_200_views": float(np.mean(lat[200])) if lat[200] else None},
        "serving": serving,
        "config0_128": config0,
        "batch64_uneven": config64,
        "next_rows": next_rows,
        "latency_batch": {"p50_ms": float(np.percentile(ms, 50)), "p99_ms": float(np.percentile(ms, 99)),
                          "plain_p99_ms": float(np.percentile(plain_ms, 99)),
                          "note": "every slice of a batch completes with the batch: the batched form "
                                  "trades per-slice latency for throughput"},
        "projector": {"fwd_ms": t_fwd, "bwd_ms": t_bwd, "bwd_ms_tuned": t_bwd_tuned, "bwd_parts_tuned": s_tuned,
                      "alg_bytes": alg_bytes,
                      "fwd_hbm_gbs": alg_bytes / (t_fwd * 1e-3) / 1e9,
                      "bwd_hbm_gbs": alg_bytes / (t_bwd * 1e-3) / 1e9,
                      "hbm_frac_of_measured": alg_bytes / (t_bwd * 1e-3) / 1e9 / peaks["hbm_gbs"]},
        "roofline": {"kernel": f"backprojector (strip sweep, k_op<OP_BWD> over {s_rf} view parts "
                               "+ k_op<OP_BWD_FIN>), 512^2 / 800 views / 738 bins",
                     "bound": "alu",
                     "achieved": nnz / (t_bwd * 1e-3) / 1e9,
                     "peak": seg_peak, "unit": "Gsegment/s",
                     "frac": nnz / (t_bwd * 1e-3) / 1e9 / seg_peak,
                     "traffic": BWD_DRAM_BYTES_512_V800,
                     "segments_per_launch": nnz,
                     "peak_src": f"152 SMs x 4 issue/clk x 32 lanes x {peaks['sm_max_mhz']:.0f} MHz (max SM clock)"
                                 f" / {SEG_INST} instructions per segment",
                     "fwd_frac": nnz / (t_fwd * 1e-3) / 1e9 / seg_peak,
                     "sm_mhz_under_load": sm_mhz,
                     # the unit that binds both operators: the L1 data pipe
                     # (one wavefront per SM per clock), the wavefronts per
                     # launch counted by ncu, the time live
                     "binding_unit": {
                         "unit": "L1 data-pipe wavefronts (shared-memory and global loads and stores)",
                         "bwd_wavefronts_per_launch": BWD_L1_WAVEFRONTS_512_V800,
                         "fwd_wavefronts_per_launch": FWD_L1_WAVEFRONTS_512_V800,
                         "peak_per_s": 152 * sm_mhz * 1e6,
                         "bwd_frac": BWD_L1_WAVEFRONTS_512_V800 / (t_bwd * 1e-3) / (152 * sm_mhz * 1e6),
                         "fwd_frac": FWD_L1_WAVEFRONTS_512_V800 / (t_fwd * 1e-3) / (152 * sm_mhz * 1e6),
                         "note": "bwd time includes the part sum k_op<OP_BWD_FIN>; peak at the SM clock "
                                 "sampled under load"}},
        "cpu_baseline": cpu,
        "precision_vs_fp64_oracle": prec,
    }
    print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


# View parts of the backprojector launch the roofline times (2048 blocks of
# 32 x 32 pixels at 512^2: 2.7 waves at 5 blocks per SM).
BWD_PARTS = 8
# Thread-instructions of the least a segment evaluation takes (overlap
# compare, intersection length, gather, FMA, loop step): the divisor of the
# issue-limited peak.
SEG_INST = 8
# DRAM bytes (read + write) of one backprojector launch on the 512^2 / 800-view
# slice, from the committed ncu capture of the current kernel (None when the
# kernel has changed since).
BWD_DRAM_BYTES_512_V800 = 11_852_288
# L1 data-pipe wavefronts of one launch of each operator on the 512^2 /
# 800-view slice (l1tex__data_pipe_lsu_wavefronts: percent of peak x cycles x
# 152 SMs) from the committed ncu captures of the current kernels: the
# backprojector's shared-memory strip updates, the projector's gathers.
BWD_L1_WAVEFRONTS_512_V800 = 58_059_172
FWD_L1_WAVEFRONTS_512_V800 = 36_488_677


if __name__ == "__main__":
    main()
