"""Benchmark of the damped acoustic FD time step on GB300 (one JSON line).

Default workload: the paper-shaped sweep, a 256^3 interior + 10-cell absorbing
layer (276^3 points), 4-layer velocity model, space orders 2/4/8/12/16, each in
the factored and the expanded stencil form, 500 time steps per shot. One bench
step = the whole sweep (10 shots: reset, 500 steps each). Metric: Gpts/s
(computational-domain points updated per second) and the fraction of the
measured HBM roofline of the step kernel.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--workload sweep|plain] [--n 256] [--nt 500]

With N > 1 (torchrun) every rank runs its own replica of the workload on its
own GPU (independent shots, no data-path collective; weak scaling).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

ORDERS = (2, 4, 8, 12, 16)
FORMS = ("factored", "expanded")


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def _kernel_hash() -> str:
    """Hash of the step kernels' code (comments and whitespace left out): a
    committed ncu traffic figure is used only while it was measured on this code."""
    import re
    h = hashlib.sha256()
    for name in ("fd_stencil.cuh", "fd_tma.cuh", "fd_tma2.cuh", "fd_flow.cuh", "fd_flow.h", "fd_internal.h"):
        with open(os.path.join(ROOT, "paper_1912_00695_gb300", "csrc", name), encoding="utf-8") as f:
            src = f.read()
        src = re.sub(r"/\*.*?\*/", " ", src, flags=re.S)
        src = re.sub(r"//[^\n]*", " ", src)
        h.update(" ".join(src.split()).encode())
    return h.hexdigest()[:16]


def _ncu_traffic(kernel_hash: str, key: str):
    """Per-launch DRAM bytes from a committed ncu summary, if it was taken on
    the current kernel source; else None."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(path) as f:
            rec = json.load(f)
        if rec.get("kernel_hash") != kernel_hash:
            return None
        return rec.get("per_launch_bytes", {}).get(key)
    except Exception:
        return None


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []
        self.t = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        if self.t:
            self.t.join(timeout=2)
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
            for nm, v in zip(names, parts[3:7]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def clocks_ok(clk: dict) -> bool:
    """False for a timed region that saw a hardware or thermal slowdown, or SM
    clocks well below their maximum with no reason reported (a clock lock left by
    another user); a power cap alone is kept (normal on this part)."""
    bad = {"hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown"}
    reasons = set(clk.get("reasons") or [])
    if reasons & bad:
        return False
    sm, smax = clk.get("sm_mhz"), clk.get("sm_max_mhz")
    if sm and smax and sm < 0.85 * smax and not (reasons - {"nvidia-smi unavailable"}):
        return False
    return True


def max_over_ranks(value: float) -> float:
    """Largest value over the ranks of the default process group (the timing
    rule: a multi-GPU step takes as long as its slowest replica); the value
    itself when not distributed."""
    import torch
    import torch.distributed as tdist
    if not (tdist.is_available() and tdist.is_initialized()):
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64)
    tdist.all_reduce(t, op=tdist.ReduceOp.MAX)
    return float(t.item())


# ---- workload -----------------------------------------------------------------

def build_workload(name: str, n: int, nt: int, orders=ORDERS, forms=FORMS):
    from paper_1912_00695_gb300 import inputs
    if name == "plain":
        spec = inputs.plain_shot()
        desc = "plain 64^3+10, space order 4, 1.5 km/s, 10 Hz Ricker at the centre, 100 steps"
        cfg = {"workload": desc, "interior": 64, "nbl": 10, "space_orders": [4],
               "forms": ["factored"], "nt": spec.nt}
        return [(spec, "factored")], desc, cfg
    runs = []
    for k in orders:
        spec = inputs.sweep_shot(k, n=n, nt=nt)
        for form in forms:
            runs.append((spec, form))
    desc = (f"sweep {n}^3+10 (4-layer model 1.5-4.5 km/s), space orders "
            f"{'/'.join(map(str, orders))} x {'/'.join(forms)}, {nt} steps, 15 Hz Ricker")
    cfg = {"workload": desc, "interior": n, "nbl": 10, "space_orders": list(orders),
           "forms": list(forms), "nt": nt}
    return runs, desc, cfg


def layer_points(spec) -> int:
    N = spec.shape
    inner = [max(a - 2 * spec.nbl, 0) for a in N]
    return int(np.prod(N) - np.prod(inner))


def algorithmic_bytes_per_step(spec, storage="f32") -> int:
    """Read u^n, u^{n-1} and the per-point coefficient, write u^{n+1}; read the
    damping field only in the layer (it vanishes in the interior)."""
    e = 4 if storage == "f32" else 2
    return int(spec.points * (3 * e + 4) + layer_points(spec) * 4)


def algorithmic_bytes_two_steps(spec) -> int:
    """One launch of the two-step kernel (FP32): read u^n, u^{n-1} and the
    coefficient, write u^{n+1} and u^{n+2}; the damping field in the layer."""
    return int(spec.points * 20 + layer_points(spec) * 4)


def run_ours(args, rank: int, world: int):
    import torch

    import paper_1912_00695_gb300 as fd
    from paper_1912_00695_gb300 import inputs

    dev = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(dev)
    stream = torch.cuda.Stream()
    runs, desc, wcfg = build_workload(args.workload, args.n, args.nt, args.orders, args.forms)
    shots = []
    for spec, form in runs:
        dt = 0.9 * fd.fd_dt_max(spec.space_order, inputs.H, spec.vmax)
        shape = {}
        if args.rows:
            shape["rows"] = args.rows
        if args.tile[0]:
            shape.update(tile_z=args.tile[0], tile_y=args.tile[1])
        if args.xblock:
            shape["x_block"] = args.xblock
        shot = fd.Shot(spec.interior, spec.space_order, inputs.H, dt, spec.nbl, form=form, **shape)
        m = spec.m
        shot.set_model(m)
        wav = inputs.ricker(spec.f0, dt, spec.nt)
        shot.inject(*spec.source, wav)
        shot.set_stream(stream.cuda_stream)
        shots.append((spec, form, shot, m, wav))

    def bench_step(record=None):
        for spec, form, shot, _, _ in shots:
            shot.reset()
            n0 = fd.fd_kernel_launches()
            shot.forward(spec.nt)
            if record is not None:
                record.append((shot.last_forward_ms(), fd.fd_kernel_launches() - n0))

    # the job's shots one after another on one stream (the headline), and the same
    # shots each on its own stream (reported beside it), and each shot alone
    shot_streams = [torch.cuda.Stream() for _ in shots]

    def set_streams(concurrent):
        for (*_, shot, _, _), st in zip(shots, shot_streams):
            shot.set_stream((st if concurrent else stream).cuda_stream)

    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)

    def timed_pass(concurrent):
        set_streams(concurrent)
        torch.cuda.synchronize()
        n0 = fd.fd_kernel_launches()
        ev0.record(stream)
        if concurrent:
            for st in shot_streams:
                st.wait_event(ev0)
        for _ in range(args.steps):
            for spec, form, shot, _, _ in shots:
                shot.reset()
                shot.forward(spec.nt)
        if concurrent:
            for st in shot_streams:
                stream.wait_stream(st)
        ev1.record(stream)
        torch.cuda.synchronize()
        return ev0.elapsed_time(ev1), fd.fd_kernel_launches() - n0

    for concurrent in (False, True):
        set_streams(concurrent)
        for _ in range(args.warmup):
            bench_step()
        torch.cuda.synchronize()

    dist = world > 1
    if dist:
        import torch.distributed as tdist
        tdist.barrier()
    clocks = ClockSampler(dev)
    clocks.start()
    total_ms, gpu_launches = timed_pass(False)
    clk = clocks.stop()
    if max_over_ranks(0.0 if clocks_ok(clk) else 1.0) > 0:
        # a slowed-down or clock-locked region is measured once more (every rank)
        if dist:
            tdist.barrier()
        clocks = ClockSampler(dev)
        clocks.start()
        total_ms, gpu_launches = timed_pass(False)
        clk = dict(clocks.stop(), remeasured_after=clk)
    conc_ms, _ = timed_pass(True)
    # per-shot kernel time alone (events around each graph replay on the launching stream)
    kernel_ms = []
    set_streams(False)
    bench_step(kernel_ms)
    torch.cuda.synchronize()
    total_ms = max_over_ranks(total_ms)
    conc_ms = max_over_ranks(conc_ms)

    pts_per_step = sum(spec.points * spec.nt for spec, *_ in shots)
    value = pts_per_step * args.steps * world / (total_ms * 1e-3) / 1e9
    conc_value = pts_per_step * args.steps * world / (conc_ms * 1e-3) / 1e9
    # schedule of each shot, from its launch count: one flow launch for the nt steps
    # (fd_tma_flow_kernel), one launch per step (fd_tma_kernel), or two steps per
    # launch (space order 2, factored: fd_tma2_kernel, its own algorithmic bytes)
    def schedule(spec, nl):
        return "flow" if nl == 1 else "step" if nl == spec.nt else "two_step"

    # roofline of the dominant kernel (the single-step arithmetic: flow or per-step
    # launches, most of the device time): algorithmic bytes / kernel time over its shots
    peak, peak_kind = _peaks()
    one = [(spec, ms, nl) for (spec, *_), (ms, nl) in zip(shots, kernel_ms) if schedule(spec, nl) != "two_step"]
    alg_bytes = sum(algorithmic_bytes_per_step(spec) * spec.nt for spec, _, _ in one)
    kern_s = sum(ms for _, ms, _ in one) * 1e-3
    launches = sum(nl for _, _, nl in one)
    achieved = alg_bytes / kern_s / 1e9 if one else 0.0
    dominant = "fd_tma_flow_kernel" if all(schedule(sp, nl) == "flow" for sp, _, nl in one) else "fd_tma_kernel"
    khash = _kernel_hash()
    # per-step DRAM bytes from the committed ncu record; a flow launch covers nt steps
    traffic = _ncu_traffic(khash, f"{args.workload}_n{args.n}")
    if traffic is not None and launches:
        traffic = int(traffic * sum(spec.nt for spec, _, _ in one) / launches)
    breakdown = {}
    for (spec, form, shot, _, _), (ms, nl) in zip(shots, kernel_ms):
        key = f"so{spec.space_order}_{form}"
        entry = {"gpts": round(spec.points * spec.nt / (ms * 1e-3) / 1e9, 2),
                 "us_per_step": round(ms * 1e3 / spec.nt, 2), "launches": nl}
        sched = schedule(spec, nl)
        if sched != "two_step":
            gbs = algorithmic_bytes_per_step(spec) * spec.nt / (ms * 1e-3) / 1e9
            entry.update(kernel="fd_tma_flow_kernel (one launch for the nt steps)" if sched == "flow"
                         else "fd_tma_kernel", hbm_frac=round(gbs / peak, 4),
                         kernel_tz_ty_xb=list(shot.config), rows_schedule_flowxb=list(shot.schedule))
        else:
            pairs = spec.nt // 2
            gbs = (algorithmic_bytes_two_steps(spec) * pairs
                   + algorithmic_bytes_per_step(spec) * (spec.nt - 2 * pairs)) / (ms * 1e-3) / 1e9
            eff = algorithmic_bytes_per_step(spec) * spec.nt / (ms * 1e-3) / 1e9
            entry.update(kernel="fd_tma2_kernel (two steps per launch)", hbm_frac=round(gbs / peak, 4),
                         hbm_frac_of_single_step_bytes=round(eff / peak, 4),
                         algorithmic_bytes_per_launch=algorithmic_bytes_two_steps(spec),
                         traffic=_ncu_traffic(khash, f"{args.workload}_n{args.n}_two_step"))
        breakdown[key] = entry

    # end to end through the public API with host buffers
    e2e = run_e2e(args, shots, stream, world)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(args)

    line = {
        "metric": "Gpts/s (computational-domain points updated per second) and fraction of "
                  "measured HBM roofline, 256^3+10 sweep, space orders 2-16",
        "value": round(value, 3), "unit": "Gpts/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(total_ms / args.steps, 3),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic (seeded layered velocity model, Ricker source)",
        "config": dict(wcfg, shots_per_step=len(shots), points_per_shot=shots[0][0].points,
                       l2=("inputs larger than L2 (4 fields per shot, "
                           f"{4 * shots[0][0].points * 4 / 1e6:.0f} MB per shot, {len(shots)} shots)"),
                       parallelism=f"replicas x{world}",
                       streams="one: the shots run one after another (one stream per shot reported beside)"),
        "roofline": {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak,
                     "unit": "GB/s", "frac": round(achieved / peak, 4), "traffic": traffic,
                     "kernel": dominant, "peak_source": peak_kind,
                     "algorithmic_bytes_per_launch_avg": int(alg_bytes / launches) if launches else 0},
        "concurrent": {"value": round(conc_value, 3), "unit": "Gpts/s", "ms_per_step": round(conc_ms / args.steps, 3),
                       "what": "the same shots, each on its own stream"},
        "breakdown": breakdown,
        "e2e": e2e,
        "gpu_launches": gpu_launches,
        "clocks": clk,
        "cpu_baseline": cpu,
        "kernel_hash": khash,
    }
    for *_, shot, _, _ in shots:
        shot.close()
    # the metric's other half: batched, reduced-precision and served forms on the same GPU
    legs = [x for x in args.legs.split(",") if x and x != "none"] if args.workload == "sweep" else []
    for leg in legs:
        torch.cuda.synchronize()
        torch.cuda.empty_cache()
        t0 = time.perf_counter()
        if leg == "batched":
            rec = leg_batched(args, world)
        elif leg == "precision":
            rec = leg_precision(args, world)
        elif leg == "serving":
            rec = leg_serving(args, world, args.leg_requests)
        else:
            raise SystemExit(f"unknown leg {leg!r}")
        rec["leg_wall_s"] = round(time.perf_counter() - t0, 1)
        line[leg] = rec
    if rank == 0:
        print(json.dumps(line), flush=True)


def run_receivers(args, rank: int, world: int):
    """Off-grid source and a surface receiver array on the sweep shot: 256^3 + 10,
    space order 8 (factored), 4-layer model, 500 steps, the source at
    (127.3, 128.6, 20.25) spread onto its 8 nodes and (n-1)^2 receivers at
    (i + 1/2, j + 1/2, 10.5) sampled every step, against the same shot with the
    integer-node source and no receivers."""
    import torch

    import paper_1912_00695_gb300 as fd
    from paper_1912_00695_gb300 import inputs

    dev = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(dev)
    stream = torch.cuda.Stream()
    spec = inputs.sweep_shot(args.rec_order, n=args.n, nt=args.nt)
    dt = 0.9 * fd.fd_dt_max(spec.space_order, inputs.H, spec.vmax)
    m = spec.m
    wav = inputs.ricker(spec.f0, dt, spec.nt)
    n = args.n
    g = np.arange(n - 1, dtype=np.float64) + 0.5
    rx, ry = np.meshgrid(g, g, indexing="ij")
    recs = np.stack([rx.ravel(), ry.ravel(), np.full(rx.size, 10.5)], axis=1)
    src_at = (n / 2 - 0.7, n / 2 + 0.6, 20.25)

    plain = fd.Shot(spec.interior, spec.space_order, inputs.H, dt, spec.nbl)
    plain.set_model(m)
    plain.inject(*spec.source, wav)
    plain.set_stream(stream.cuda_stream)
    rshot = fd.Shot(spec.interior, spec.space_order, inputs.H, dt, spec.nbl)
    rshot.set_model(m)
    rshot.inject_at(*src_at, wav)
    rshot.set_receivers(recs, spec.nt)
    rshot.set_stream(stream.cuda_stream)

    def timed(shot):
        for _ in range(args.warmup):
            shot.reset()
            shot.forward(spec.nt)
        torch.cuda.synchronize()
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        n0 = fd.fd_kernel_launches()
        ev0.record(stream)
        for _ in range(args.steps):
            shot.reset()
            shot.forward(spec.nt)
        ev1.record(stream)
        torch.cuda.synchronize()
        return ev0.elapsed_time(ev1), fd.fd_kernel_launches() - n0

    ms_plain = max_over_ranks(timed(plain)[0])
    clocks = ClockSampler(dev)
    clocks.start()
    ms_rec, rec_launches = timed(rshot)
    ms_rec = max_over_ranks(ms_rec)
    clk = clocks.stop()
    pts = spec.points * spec.nt * args.steps * world
    gpts, gpts_plain = pts / (ms_rec * 1e-3) / 1e9, pts / (ms_plain * 1e-3) / 1e9
    tr = rshot.traces()
    sched = rshot.schedule[1]
    rec_kernel = ("fd_tma_flow_kernel (receivers sampled and extra sources added per work item) "
                  "+ sample_receivers_kernel (last level)" if sched == 1 else
                  "fd_tma_kernel (receivers sampled) + inject_extra_kernel + sample_receivers_kernel (last level)")
    # end to end through the public API with host buffers: model upload, source,
    # receivers, the run, read-back of the traces and the final field
    h2d = m.nbytes + wav.nbytes + recs.nbytes
    d2h = tr.nbytes + m.nbytes
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        s = fd.Shot(spec.interior, spec.space_order, inputs.H, dt, spec.nbl)
        s.set_model(m)
        s.inject_at(*src_at, wav)
        s.set_receivers(recs, spec.nt)
        s.forward(spec.nt)
        s.traces()
        s.wavefield(0)
        s.close()
    e2e_s = max_over_ranks((time.perf_counter() - t0) * 1e3) * 1e-3
    peak, peak_kind = _peaks()
    alg = algorithmic_bytes_per_step(spec) * spec.nt * args.steps
    line = {
        "metric": "Gpts/s with an off-grid source and a surface receiver array sampled every step "
                  "(256^3+10, space order 8) vs the integer-node source alone",
        "value": round(gpts, 3), "unit": "Gpts/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(ms_rec / args.steps, 3), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic (seeded layered velocity model, Ricker source)",
        "config": {"workload": f"receivers: {n}^3+10, space order {spec.space_order}, {spec.nt} steps, "
                               f"{len(recs)} receivers at depth 10.5, off-grid source {src_at}",
                   "receivers": len(recs), "l2": "inputs larger than L2", "parallelism": f"replicas x{world}"},
        "plain_gpts": round(gpts_plain, 3),
        "receiver_cost_frac": round(ms_rec / ms_plain - 1.0, 4),
        "schedule": {0: "per-step", 1: "flow", 2: "two-step"}.get(sched, str(sched)),
        "plain_schedule": {0: "per-step", 1: "flow", 2: "two-step"}.get(plain.schedule[1], "?"),
        "roofline": {"bound": "hbm", "achieved": round(alg / (ms_rec * 1e-3) / 1e9, 1), "peak": peak,
                     "unit": "GB/s", "frac": round(alg / (ms_rec * 1e-3) / 1e9 / peak, 4), "traffic": None,
                     "kernel": rec_kernel, "peak_source": peak_kind},
        "e2e": {"value": round(spec.points * spec.nt * args.steps * world / e2e_s / 1e9, 3), "unit": "Gpts/s",
                "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h)},
        "gpu_launches": rec_launches,
        "clocks": clk,
    }
    if rank == 0:
        print(json.dumps(line), flush=True)
    plain.close()
    rshot.close()


def run_gradient(args, rank: int, world: int):
    """FWI gradient of one shot (forward pass storing the second time difference
    of every step, adjoint pass backward in time with the residuals injected at
    the receivers and the gradient accumulated in its step kernel): the sweep
    shot (256^3 + 10, 4-layer model, 15 Hz Ricker at (128,128,20)), space order 8,
    500 steps, (n-1)^2 receivers at (i + 1/2, j + 1/2, 10.5), d_obs = 0 (the
    residual is the synthetic data; the cost does not depend on it)."""
    import torch

    import paper_1912_00695_gb300 as fd
    from paper_1912_00695_gb300 import inputs

    dev = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(dev)
    spec = inputs.sweep_shot(args.rec_order, n=args.n, nt=args.nt)
    dt = 0.9 * fd.fd_dt_max(spec.space_order, inputs.H, spec.vmax)
    m = spec.m
    wav = inputs.ricker(spec.f0, dt, spec.nt)
    n = args.n
    g = np.arange(n - 1, dtype=np.float64) + 0.5
    rx, ry = np.meshgrid(g, g, indexing="ij")
    recs = np.stack([rx.ravel(), ry.ravel(), np.full(rx.size, 10.5)], axis=1)
    obs = np.zeros((len(recs), spec.nt), np.float32)
    shot = fd.Shot(spec.interior, spec.space_order, inputs.H, dt, spec.nbl)
    shot.set_model(m)
    shot.inject(*spec.source, wav)
    for _ in range(args.warmup):
        shot.fwi_gradient(recs, obs)
    clocks = ClockSampler(dev)
    clocks.start()
    dev_ms, wall = [], []
    launches0 = fd.fd_kernel_launches()
    for _ in range(args.steps):
        t0 = time.perf_counter()
        shot.fwi_gradient(recs, obs)
        wall.append(time.perf_counter() - t0)
        dev_ms.append(shot.last_forward_ms())
    clk = clocks.stop()
    grad_launches = fd.fd_kernel_launches() - launches0
    ms = max_over_ranks(sum(dev_ms))
    wall_s = max_over_ranks(sum(wall) * 1e3) * 1e-3
    updates = 2 * spec.points * spec.nt * args.steps * world
    peak, peak_kind = _peaks()
    layer = layer_points(spec)
    # forward: u^n, u^{n-1}, w read, u^{n+1} and D written (16 + 4 B); adjoint: the same
    # step (16 B) plus D read and the gradient read and written (12 B); g in the layer
    alg = (spec.points * (20 + 28) + 2 * layer * 4) * spec.nt * args.steps
    line = {
        "metric": "FWI gradient Gpts/s (forward + adjoint point updates per second), 256^3+10, space order 8",
        "value": round(updates / (ms * 1e-3) / 1e9, 3), "unit": "Gpts/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms / args.steps, 3),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic (seeded layered velocity model, Ricker source, zero observed data)",
        "config": {"workload": f"fwi gradient: {n}^3+10, space order {spec.space_order}, {spec.nt} steps, "
                               f"{len(recs)} receivers at depth 10.5, history {spec.nt} x "
                               f"{spec.points * 4 / 1e6:.0f} MB in HBM",
                   "receivers": len(recs), "l2": "inputs larger than L2", "parallelism": f"replicas x{world}"},
        "roofline": {"bound": "hbm", "achieved": round(alg / (ms * 1e-3) / 1e9, 1), "peak": peak, "unit": "GB/s",
                     "frac": round(alg / (ms * 1e-3) / 1e9 / peak, 4), "traffic": None,
                     "kernel": "fd_tma_grad_kernel (forward D / adjoint gradient)", "peak_source": peak_kind},
        "e2e": {"value": round(updates / wall_s / 1e9, 3), "unit": "Gpts/s",
                "h2d_bytes_per_step": int(obs.nbytes), "d2h_bytes_per_step": int(m.nbytes + obs.nbytes)},
        "gpu_launches": grad_launches,
        "clocks": clk,
    }
    if rank == 0:
        print(json.dumps(line), flush=True)
    shot.close()


def leg_batched(args, world: int) -> dict:
    """64 uneven shots (each axis U{96..256} + 10, smooth random velocity, k=8,
    300 steps): the batch (one launch per step over all shots) against the same
    shots run one after another through the single-shot path. Returns the
    leg's record (its own clocks, roofline and launch count)."""
    import torch

    import paper_1912_00695_gb300 as fd
    from paper_1912_00695_gb300 import inputs

    dev = torch.cuda.current_device()
    stream = torch.cuda.Stream()
    specs = inputs.batched_shots(count=args.shots, nt=args.nt_batched, lo=args.shot_range[0],
                                 hi=args.shot_range[1])
    k = specs[0].space_order
    batch = fd.Batch(k, inputs.H, tile_z=args.batch_tile[0], tile_y=args.batch_tile[1],
                     x_block=args.batch_xb)
    batch.set_stream(stream.cuda_stream)
    singles = []
    for spec in specs:
        spec.dt = 0.9 * fd.fd_dt_max(k, inputs.H, spec.vmax)
        m = spec.m
        wav = inputs.ricker(spec.f0, spec.dt, spec.nt)
        s = batch.add(spec.interior, spec.nbl, spec.dt, m)
        batch.inject(s, *spec.source, wav)
        shot = fd.Shot(spec.interior, k, inputs.H, spec.dt, spec.nbl)
        shot.set_model(m)
        shot.inject(*spec.source, wav)
        shot.set_stream(stream.cuda_stream)
        singles.append(shot)
    nt = args.nt_batched
    pts = sum(spec.points for spec in specs) * nt

    def plain_step():
        for shot in singles:
            shot.reset()
            shot.forward(nt)

    def batch_step():
        batch.reset()
        if args.batch_schedule == "flow":
            batch.forward_flow(nt)
        else:
            batch.forward(nt)

    def timed(fn, steps):
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        ev0.record(stream)
        for _ in range(steps):
            fn()
        ev1.record(stream)
        torch.cuda.synchronize()
        return ev0.elapsed_time(ev1)

    steps = max(1, args.leg_steps)
    for _ in range(args.warmup):
        plain_step()
        batch_step()
    torch.cuda.synchronize()
    plain_ms = max_over_ranks(timed(plain_step, steps))
    if world > 1:
        import torch.distributed as tdist
        tdist.barrier()
    clocks = ClockSampler(dev)
    clocks.start()
    launches0 = fd.fd_kernel_launches()
    batch_ms = timed(batch_step, steps)
    batch_launches = fd.fd_kernel_launches() - launches0
    batch_ms = max_over_ranks(batch_ms)
    clk = clocks.stop()
    value = pts * steps * world / (batch_ms * 1e-3) / 1e9
    plain = pts * steps * world / (plain_ms * 1e-3) / 1e9
    peak, peak_kind = _peaks()
    alg = sum(algorithmic_bytes_per_step(spec) for spec in specs) * nt * steps
    achieved = alg / (batch_ms * 1e-3) / 1e9
    active, items = batch.size()
    cfg = batch.config() if hasattr(batch, "config") else (args.batch_tile[0], args.batch_tile[1], args.batch_xb)
    flow_sched = bool(batch.schedule()) or args.batch_schedule == "flow"
    schedule = "one persistent launch per forward" if flow_sched else "one launch per step"
    field_gb = 4 * 4 * sum(spec.points for spec in specs) / 1e9  # u, u^{n-1}, and two coefficient fields
    rec = {
        "metric": f"Gpts/s, {len(specs)} uneven shots advanced as one batch vs the same shots one by one",
        "value": round(value, 3), "unit": "Gpts/s", "steps": steps, "warmup": args.warmup,
        "ms_per_step": round(batch_ms / steps, 3),
        "config": {"workload": f"batched: {len(specs)} shots, interiors U{{{args.shot_range[0]}.."
                               f"{args.shot_range[1]}}} per axis + 10, space order {k}, {nt} steps, "
                               "factored, FP32, smooth random velocity (sigma 8 cells)",
                   "batch_tile_z_y_x_block": list(cfg), "schedule": schedule, "points": sum(spec.points for spec in specs),
                   "work_items_per_step": items, "l2": f"inputs larger than L2 ({field_gb:.1f} GB of fields per copy)"},
        "plain_one_by_one": {"value": round(plain, 3), "unit": "Gpts/s",
                             "ms_per_step": round(plain_ms / steps, 3),
                             "what": "the same shots one after another through fd_forward (device-timed)"},
        "speedup_vs_plain": round(value / plain, 3),
        "roofline": {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                     "frac": round(achieved / peak, 4), "traffic": None,
                     "kernel": "fd_tma_batch_flow_kernel" if flow_sched else "fd_tma_batch_kernel",
                     "peak_source": peak_kind,
                     "algorithmic_bytes_per_step": int(alg / steps)},
        "gpu_launches": batch_launches,
        "clocks": clk,
    }
    batch.close()
    for shot in singles:
        shot.close()
    return rec


def run_batched(args, rank: int, world: int):
    rec = leg_batched(args, world)
    line = dict(rec, n_gpus=world, higher_is_better=True, scaling="weak", vs_baseline=None, dtype="f32",
                data="synthetic (seeded smooth random velocity models, Ricker sources)")
    line["config"] = dict(rec["config"], parallelism=f"replicas x{world}")
    if rank == 0:
        print(json.dumps(line), flush=True)


def leg_precision(args, world: int) -> dict:
    """384^3 + 20 (424^3 points), space order 12, 4-layer model, 1000 steps: the
    same shot with FP32, BF16 and FP16 wavefield storage (per-level
    power-of-two scales, FP32 arithmetic), and the three storages on the
    256^3 + 10 sweep shot at the requested space orders. The error of each
    storage against the FP64 oracle at this configuration is measured by the
    precision_error workload."""
    import torch

    import paper_1912_00695_gb300 as fd
    from paper_1912_00695_gb300 import inputs

    dev = torch.cuda.current_device()
    stream = torch.cuda.Stream()
    peak, peak_kind = _peaks()
    clk = None
    steps = max(1, args.leg_steps)

    def measure(spec, sample_clocks):
        nonlocal clk
        dt = 0.9 * fd.fd_dt_max(spec.space_order, inputs.H, spec.vmax)
        m = spec.m
        wav = inputs.ricker(spec.f0, dt, spec.nt)
        res = {}
        for st in ("f32", "bf16", "f16"):
            shot = fd.Shot(spec.interior, spec.space_order, inputs.H, dt, spec.nbl, storage=st)
            shot.set_model(m)
            shot.inject(*spec.source, wav)
            shot.set_stream(stream.cuda_stream)
            for _ in range(args.warmup):
                shot.reset()
                shot.forward(spec.nt)
            torch.cuda.synchronize()
            clocks = ClockSampler(dev)
            if sample_clocks and st == "bf16":
                clocks.start()
            ev0 = torch.cuda.Event(enable_timing=True)
            ev1 = torch.cuda.Event(enable_timing=True)
            n0 = fd.fd_kernel_launches()
            ev0.record(stream)
            for _ in range(steps):
                shot.reset()
                shot.forward(spec.nt)
            ev1.record(stream)
            torch.cuda.synchronize()
            n_launch = fd.fd_kernel_launches() - n0
            if sample_clocks and st == "bf16":
                clk = clocks.stop()
            ms = max_over_ranks(ev0.elapsed_time(ev1))
            gpts = spec.points * spec.nt * steps * world / (ms * 1e-3) / 1e9
            alg = algorithmic_bytes_per_step(spec, st) * spec.nt * steps
            res[st] = {"gpts": round(gpts, 2), "ms_per_step": round(ms / steps, 3),
                       "hbm_frac": round(alg / (ms * 1e-3) / 1e9 / peak, 4), "config": list(shot.config),
                       "rows_schedule_flowxb": list(shot.schedule), "launches": n_launch}
            shot.close()
        return res

    spec = inputs.precision_shot(n=args.n_precision, nt=args.nt_precision)
    res = measure(spec, True)
    by_order = {}
    for k in args.precision_orders:
        sp = inputs.sweep_shot(k, n=args.n, nt=min(args.nt, args.nt_precision))
        r = measure(sp, False)
        by_order[f"so{k}"] = {st: {"gpts": v["gpts"], "hbm_frac": v["hbm_frac"],
                                   "rows_schedule_flowxb": v["rows_schedule_flowxb"]} for st, v in r.items()}
        by_order[f"so{k}"]["bf16_vs_f32"] = round(r["bf16"]["gpts"] / r["f32"]["gpts"], 3)
        by_order[f"so{k}"]["f16_vs_f32"] = round(r["f16"]["gpts"] / r["f32"]["gpts"], 3)
    return {
        "metric": "Gpts/s with BF16 / FP16 wavefield storage (per-level scale, FP32 arithmetic) vs FP32 "
                  "storage, 384^3+20, space order 12",
        "value": round(res["bf16"]["gpts"], 3), "unit": "Gpts/s", "steps": steps, "warmup": args.warmup,
        "ms_per_step": res["bf16"]["ms_per_step"],
        "config": {"workload": f"precision: {args.n_precision}^3+20, space order 12, 4-layer model, "
                               f"{spec.nt} steps", "points": spec.points, "l2": "inputs larger than L2"},
        "by_storage": res,
        "speedup_bf16_vs_f32": round(res["bf16"]["gpts"] / res["f32"]["gpts"], 3),
        "speedup_f16_vs_f32": round(res["f16"]["gpts"] / res["f32"]["gpts"], 3),
        "sweep_shot_by_order": by_order,
        "sweep_shot_steps": min(args.nt, args.nt_precision),
        "roofline": {"bound": "hbm", "achieved": round(res["bf16"]["hbm_frac"] * peak, 1), "peak": peak,
                     "unit": "GB/s", "frac": res["bf16"]["hbm_frac"], "traffic": None,
                     "kernel": "fd_tma_kernel (bf16)", "peak_source": peak_kind,
                     "algorithmic_bytes_per_point": "10 + 4 in the layer (three 2-byte levels, FP32 coefficient)"},
        "gpu_launches": res["bf16"]["launches"],
        "clocks": clk,
    }


def run_precision(args, rank: int, world: int):
    rec = leg_precision(args, world)
    line = dict(rec, n_gpus=world, higher_is_better=True, scaling="weak", vs_baseline=None,
                dtype="bf16 storage, f32 math",
                data="synthetic (seeded layered velocity model, Ricker source)")
    line["config"] = dict(rec["config"], parallelism=f"replicas x{world}")
    if rank == 0:
        print(json.dumps(line), flush=True)


class ModelSource:
    """Velocity models (as squared slowness) of a serving trace, made on demand:
    a thread pool generates the models of the next `ahead` requests in
    arrival order while the current ones are served, and keeps them in host
    memory up to `keep_bytes` (the rest is regenerated when asked for again),
    so that a trace of hundreds of large requests neither waits for all its
    models up front nor holds them all."""

    def __init__(self, trace, ahead: int = 12, workers: int = 8, keep_bytes: int = 0):
        import concurrent.futures as cf
        self.trace = trace
        self.ahead = ahead
        self.keep_bytes = keep_bytes
        self.pool = cf.ThreadPoolExecutor(max_workers=workers)
        self.futs = {}
        self.kept = {}
        self.kept_bytes = 0

    def _make(self, i):
        from paper_1912_00695_gb300 import inputs
        return inputs.slowness2(inputs.velocity_for(self.trace[i]))

    def _submit(self, i):
        if 0 <= i < len(self.trace) and i not in self.kept and i not in self.futs:
            self.futs[i] = self.pool.submit(self._make, i)

    def get(self, i):
        for j in range(i, i + self.ahead):
            self._submit(j)
        if i in self.kept:
            return self.kept[i]
        m = self.futs.pop(i).result()
        if self.kept_bytes + m.nbytes <= self.keep_bytes:
            self.kept[i] = m
            self.kept_bytes += m.nbytes
        return m

    def close(self):
        self.pool.shutdown(wait=True, cancel_futures=True)
        self.futs.clear()
        self.kept.clear()


def leg_serving(args, world: int, requests: int) -> dict:
    """Continuous-batching server (paper_1912_00695_gb300.serve) on the Poisson
    trace of shot requests: cubic interiors U{lo..hi} + 10, space order 8 or
    16, FP32 or BF16 storage (50/50), steps U{steps}, smooth random velocity,
    the first `requests` requests of the seeded trace. Passes over the same
    requests: offline (all present at t=0: the capacity), at the trace's
    Poisson rate, at 70 % of the measured capacity (arrival times rescaled, so
    that latency percentiles are also reported below saturation), and the
    plain form (each request alone through a single-shot handle: set-up, run,
    read-back), all on the wall clock."""
    import torch

    import paper_1912_00695_gb300 as fd
    from paper_1912_00695_gb300 import inputs
    from paper_1912_00695_gb300.serve import Request, Server

    dev = torch.cuda.current_device()
    trace = inputs.serving_trace(count=requests, rate=args.rate, lo=args.serve_range[0],
                                 hi=args.serve_range[1], steps=args.serve_steps)
    try:
        import psutil
        avail = int(psutil.virtual_memory().available)
    except Exception:
        avail = 16 << 30
    models = ModelSource(trace, keep_bytes=max(0, int(0.4 * avail) - (8 << 30)))
    vmax = 4500.0  # the smooth models are min-max rescaled to [1.5, 4.5] km/s

    def make_requests(rate_scale=1.0):
        reqs = []
        for i, spec in enumerate(trace):
            dt = 0.9 * fd.fd_dt_max(spec.space_order, inputs.H, vmax)
            reqs.append(Request(i, spec.arrival * rate_scale, spec.interior, spec.nbl, spec.space_order,
                                spec.storage, dt, None, spec.source,
                                inputs.ricker(spec.f0, dt, spec.nt), spec.nt,
                                m_fn=(lambda i=i: models.get(i))))
        return reqs

    free, _ = torch.cuda.mem_get_info()
    budget = int(args.serve_budget * free)

    def serve(reqs, realtime):
        srv = Server(inputs.H, budget, chunk=args.chunk, keep_results=False)
        stats = srv.run(reqs, realtime=realtime)
        srv.close()
        return stats

    serve(make_requests()[: min(4, len(trace))], realtime=False)  # warm-up: graphs, classes
    offline = serve(make_requests(), realtime=False)
    capacity = offline["gpts"]
    mean_work = np.mean([spec.points * spec.nt for spec in trace])
    offered = args.rate * mean_work / 1e9
    clocks = ClockSampler(dev)
    clocks.start()
    launches0 = fd.fd_kernel_launches()
    at_rate = serve(make_requests(), realtime=True)
    serve_launches = fd.fd_kernel_launches() - launches0
    clk = clocks.stop()
    scale70 = offered / (0.7 * capacity) if capacity > 0 else 1.0
    at70 = serve(make_requests(scale70), realtime=True)

    def plain():
        pts = 0
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for r in make_requests():
            with fd.Shot(r.interior, r.space_order, inputs.H, r.dt, r.nbl, storage=r.storage) as shot:
                shot.set_model(r.model())
                shot.inject(*r.source, r.wavelet)
                shot.forward(r.nt)
                shot.wavefield(0)
            pts += r.points * r.nt
        torch.cuda.synchronize()
        return pts / (time.perf_counter() - t0) / 1e9

    plain_gpts = plain()
    models.close()
    rnd = (lambda d: {k: round(v, 4) if isinstance(v, float) else v for k, v in d.items()})
    return {
        "metric": "served Gpts/s and p50/p99 request latency, continuous batching of shot requests",
        "value": round(at_rate["gpts"] * world, 3), "unit": "Gpts/s",
        "config": {"workload": f"serving: first {len(trace)} requests of the seeded Poisson trace "
                               f"({args.rate}/s), cubic interiors U{{{args.serve_range[0]}..{args.serve_range[1]}}}"
                               f" + 10, space order 8/16, FP32/BF16, steps U{{{args.serve_steps[0]}.."
                               f"{args.serve_steps[1]}}}, smooth random velocity per request",
                   "requests": len(trace), "chunk": args.chunk, "budget_bytes": budget,
                   "models": "generated per request from its seed by a host thread pool ahead of admission"},
        "offered_gpts": round(offered, 2),
        "offered_vs_capacity": round(offered / capacity, 3) if capacity > 0 else None,
        "capacity_offline_gpts": round(capacity, 2),
        "plain_one_by_one": {"value": round(plain_gpts, 3), "unit": "Gpts/s",
                             "what": "the same requests one after another through single-shot handles "
                                     "(set-up, run, read-back each), wall clock"},
        "capacity_vs_plain": round(capacity / plain_gpts, 3) if plain_gpts > 0 else None,
        "served_at_rate_vs_plain": round(at_rate["gpts"] / plain_gpts, 3) if plain_gpts > 0 else None,
        "at_trace_rate": rnd(at_rate),
        "at_70pct_capacity": dict(rnd(at70), rate_per_s=round(args.rate / scale70, 3)),
        "offline": rnd(offline),
        "gpu_launches": serve_launches,
        "clocks": clk,
    }


def run_serving(args, rank: int, world: int):
    rec = leg_serving(args, world, args.requests)
    line = dict(rec, n_gpus=world, steps=1, warmup=1, ms_per_step=round(rec["at_trace_rate"]["makespan_s"] * 1e3, 1),
                higher_is_better=True, scaling="weak", vs_baseline=None, dtype="f32 / bf16 storage per request",
                data="synthetic (seeded smooth random velocity models, Ricker sources, Poisson arrivals)")
    line["config"] = dict(rec["config"], parallelism=f"replicas x{world}")
    if rank == 0:
        print(json.dumps(line), flush=True)


def run_e2e(args, shots, stream, world):
    """Same metric through the public C-ABI calls with host buffers: per shot,
    set the model from pinned host memory, inject the host wavelet, reset, run,
    and read the final wavefield back into pinned host memory. Each shot has its
    own stream, so one shot's model upload and read-back overlap another's time
    steps; the time steps of consecutive shots are ordered by events (one shot
    computes at a time, as in the device-timed pass). Wall clock, synchronised."""
    import torch

    from paper_1912_00695_gb300 import fd_clear_sources

    e2e_steps = max(1, min(args.steps, 2))
    streams = [torch.cuda.Stream() for _ in shots]
    pinned_m, pinned_out = [], []
    for spec, form, shot, m, wav in shots:
        pm = torch.empty(spec.shape, dtype=torch.float32, pin_memory=True).numpy()
        pm[...] = m  # the step's input, already in pinned host memory when the clock starts
        pinned_m.append(pm)
        pinned_out.append(torch.empty(spec.shape, dtype=torch.float32, pin_memory=True).numpy())
    for (*_, shot, _, _), st in zip(shots, streams):
        shot.set_stream(st.cuda_stream)
    h2d = d2h = 0
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    prev = None
    for _ in range(e2e_steps):
        for (spec, form, shot, m, wav), pm, st in zip(shots, pinned_m, streams):
            shot.set_model(pm)
            fd_clear_sources(shot.handle)
            shot.inject(*spec.source, wav)
            shot.reset()
            if prev is not None:
                st.wait_event(prev)  # the previous shot's steps first
            shot.forward(spec.nt)
            prev = torch.cuda.Event()
            prev.record(st)
            h2d += pm.nbytes + wav.nbytes
        for (spec, form, shot, m, wav), out in zip(shots, pinned_out):
            shot.wavefield(0, out)
            d2h += out.nbytes
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    for *_, shot, _, _ in shots:
        shot.set_stream(stream.cuda_stream)
    pts = sum(spec.points * spec.nt for spec, *_ in shots) * e2e_steps * world
    return {"value": round(pts / dt / 1e9, 3), "unit": "Gpts/s",
            "h2d_bytes_per_step": int(h2d // e2e_steps), "d2h_bytes_per_step": int(d2h // e2e_steps),
            "steps": e2e_steps, "host_buffers": "pinned",
            "streams": "one per shot; transfers overlap, time steps one shot at a time"}


def cpu_baseline(args, target_s: float = 10.0):
    """The FP64 oracle (as it stands) on the host cores, on a bounded sample of
    the workload: the space-order-8 shot of the sweep for a few steps."""
    import oracle
    from paper_1912_00695_gb300 import inputs
    spec = inputs.sweep_shot(8, n=args.n, nt=args.nt)
    m = spec.m.astype(np.float64)
    eta = oracle.default_damping(m, spec.nbl, inputs.H)
    dt = 0.9 * oracle.dt_max(8, inputs.H, spec.vmax)
    wav = inputs.ricker(spec.f0, dt, spec.nt).astype(np.float64)[None, :]
    src = [tuple(c + spec.nbl for c in spec.source)]
    t0 = time.perf_counter()
    u, up = oracle.forward(m, eta, 8, inputs.H, dt, 1, src, wav)
    one = time.perf_counter() - t0
    steps = int(max(1, min(20, target_s / max(one, 1e-3))))
    t0 = time.perf_counter()
    oracle.forward(m, eta, 8, inputs.H, dt, steps, src, wav, u0=u, u_prev0=up, step0=1)
    el = time.perf_counter() - t0
    return {"value": round(spec.points * steps / el / 1e9, 5), "unit": "Gpts/s",
            "cores": oracle.num_threads(), "kind": "oracle",
            "sample": f"space order 8 shot of the sweep ({spec.shape[0]}^3 points), {steps} steps, FP64"}


def run_reference(args, rank: int, world: int):
    """The oracle timed as the reference arm: each step is a bounded sample of
    the sweep workload (the space-order-8 shot, 2 time steps) on host cores."""
    if rank != 0:
        return
    import oracle
    from paper_1912_00695_gb300 import inputs
    spec = inputs.sweep_shot(8, n=args.n, nt=args.nt)
    m = spec.m.astype(np.float64)
    eta = oracle.default_damping(m, spec.nbl, inputs.H)
    dt = 0.9 * oracle.dt_max(8, inputs.H, spec.vmax)
    wav = inputs.ricker(spec.f0, dt, spec.nt).astype(np.float64)[None, :]
    src = [tuple(c + spec.nbl for c in spec.source)]
    per = 2
    u = up = None
    step = 0
    for _ in range(args.warmup):
        u, up = oracle.forward(m, eta, 8, inputs.H, dt, per, src, wav, u0=u, u_prev0=up, step0=step)
        step += per
    t0 = time.perf_counter()
    for _ in range(args.steps):
        u, up = oracle.forward(m, eta, 8, inputs.H, dt, per, src, wav, u0=u, u_prev0=up, step0=step)
        step += per
    el = time.perf_counter() - t0
    value = spec.points * per * args.steps / el / 1e9
    _, desc, wcfg = build_workload(args.workload, args.n, args.nt, args.orders, args.forms)
    sample = f"space order 8 shot of the sweep ({spec.shape[0]}^3 points), {per} steps per bench step, FP64"
    line = {"impl": "reference",
            "metric": "Gpts/s (computational-domain points updated per second) and fraction of "
                      "measured HBM roofline, 256^3+10 sweep, space orders 2-16",
            "value": round(value, 5), "unit": "Gpts/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": round(el * 1e3 / args.steps, 3),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic (seeded layered velocity model, Ricker source)",
            "config": wcfg,
            "cpu_baseline": {"value": round(value, 5), "unit": "Gpts/s", "kind": "oracle",
                             "cores": oracle.num_threads(), "sample": sample},
            "e2e": {"value": round(value, 5), "unit": "Gpts/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="sweep",
                    choices=["sweep", "plain", "batched", "precision", "serving", "receivers", "gradient"])
    ap.add_argument("--legs", default="batched,precision,serving",
                    help="sweep workload: legs added to the line (batched, precision, serving; 'none')")
    ap.add_argument("--leg-steps", type=int, default=2, help="timed repetitions of the batched/precision legs")
    ap.add_argument("--leg-requests", type=int, default=60,
                    help="serving leg of the default line: the first N requests of the trace")
    ap.add_argument("--requests", type=int, default=200, help="serving workload: requests in the trace")
    ap.add_argument("--rate", type=float, default=20.0, help="serving: Poisson arrivals per second")
    ap.add_argument("--serve-range", type=lambda v: tuple(int(x) for x in v.split(",")), default=(128, 512),
                    help="serving: cubic interior size range lo,hi")
    ap.add_argument("--serve-steps", type=lambda v: tuple(int(x) for x in v.split(",")), default=(200, 2000),
                    help="serving: steps range lo,hi")
    ap.add_argument("--serve-budget", type=float, default=0.8, help="serving: fraction of free HBM to admit into")
    ap.add_argument("--chunk", type=int, default=50, help="serving: steps per scheduling chunk")
    ap.add_argument("--n-precision", type=int, default=384, help="precision workload: interior size")
    ap.add_argument("--nt-precision", type=int, default=1000, help="precision workload: steps")
    ap.add_argument("--precision-orders", type=lambda v: tuple(int(x) for x in v.split(",") if x),
                    default=(2, 4, 8, 12, 16),
                    help="precision workload: also compare the storages on the sweep shot at these orders")
    ap.add_argument("--shots", type=int, default=64, help="batched workload: number of shots")
    ap.add_argument("--nt-batched", type=int, default=300, help="batched workload: steps per shot")
    ap.add_argument("--batch-xb", type=int, default=0, help="batched workload: x_block (0 = the library default)")
    ap.add_argument("--batch-schedule", default="auto", choices=["auto", "flow"],
                    help="batched workload: the autotuned schedule, or one persistent launch per forward")
    ap.add_argument("--batch-tile", type=lambda v: tuple(int(x) for x in v.split("x")), default=(0, 0),
                    help="batched workload: tile as ZxY (32x16 or 64x8; default 32x16)")
    ap.add_argument("--shot-range", type=lambda v: tuple(int(x) for x in v.split(",")), default=(96, 256),
                    help="batched workload: interior size range lo,hi per axis")
    ap.add_argument("--rec-order", type=int, default=8, help="receivers/gradient workloads: space order")
    ap.add_argument("--n", type=int, default=256)
    ap.add_argument("--nt", type=int, default=500)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--rows", type=int, default=0, help="sweep: y rows per thread of the step kernel (0 = autotuned)")
    ap.add_argument("--tile", type=lambda v: tuple(int(x) for x in v.split("x")), default=(0, 0),
                    help="sweep: step kernel tile as ZxY (default autotuned)")
    ap.add_argument("--xblock", type=int, default=0,
                    help="sweep: planes per CTA / flow x-chunk of the step kernel (0 = tuned)")
    ap.add_argument("--orders", type=lambda v: tuple(int(x) for x in v.split(",")), default=ORDERS,
                    help="comma-separated space orders of the sweep (default 2,4,8,12,16)")
    ap.add_argument("--forms", type=lambda v: tuple(v.split(",")), default=FORMS,
                    help="comma-separated stencil forms (default factored,expanded)")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if world > 1:
        import torch.distributed as tdist
        tdist.init_process_group("gloo")
    if args.impl == "reference":
        run_reference(args, rank, world)
    elif args.workload == "batched":
        run_batched(args, rank, world)
    elif args.workload == "precision":
        run_precision(args, rank, world)
    elif args.workload == "serving":
        run_serving(args, rank, world)
    elif args.workload == "receivers":
        run_receivers(args, rank, world)
    elif args.workload == "gradient":
        run_gradient(args, rank, world)
    else:
        run_ours(args, rank, world)
    if world > 1:
        import torch.distributed as tdist
        tdist.barrier()
        tdist.destroy_process_group()


if __name__ == "__main__":
    main()
