"""Throughput of the fused D2Q13 time step on GB300.

Workload (one bench step = one time step of the whole lattice): the periodic
transverse shear wave u_x = 0.01 sin(2 pi y / n) of the throughput sweep, at
n x n = 8192 x 8192 by default, parameters nu = 0.05, Pr = 0.71, in
FP32-deviation storage.  A lattice this size, periodic in x and y, takes two
time steps per launch (52 algorithmic bytes per lattice update; 104 with one
step per launch).  The FP64 path (208 B/LU) is measured on the same lattice
and reported beside it.

Prints one JSON line (rank 0).  `--impl reference` times the FP64 CPU oracle
instead, on a bounded sample of the same workload.
"""
import argparse
import json
import os
import statistics
import subprocess
import tempfile
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "MLUPS and % of HBM roofline per GB300; p50/p99 time-to-steady-state vs plain FP64"
UNIT = "MLUPS"
NU, PR = 0.05, 0.71


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--size", type=int, default=8192)
    ap.add_argument("--precision", default="fp32", choices=["fp32", "fp64"])
    ap.add_argument("--fp64-steps", type=int, default=60)
    ap.add_argument("--no-fp64", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-batched", action="store_true")
    ap.add_argument("--no-serving", action="store_true")
    ap.add_argument("--batched-steps", type=int, default=200)
    ap.add_argument("--serving-requests", type=int, default=16)
    ap.add_argument("--batched-count", type=int, default=256)
    ap.add_argument("--batched-config", default="",
                    help="R,BY,ctas_per_sm,order for the batched plan instead of autotuning")
    ap.add_argument("--no-sweep", action="store_true")
    ap.add_argument("--no-pairs", action="store_true",
                    help="one time step per launch on the main lattice (the single-step kernel)")
    return ap.parse_args()


def dist_env():
    return int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("LOCAL_RANK", "0"))


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during a region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = os.path.join(tempfile.gettempdir(), f"lbm13_clocks_{os.getpid()}.csv")

    def __enter__(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=self.fh, stderr=subprocess.DEVNULL)
            time.sleep(0.3)
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            time.sleep(0.15)
            self.proc.terminate()
            try:
                self.proc.wait(5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            self.fh.close()

    def summary(self):
        if self.proc is None:
            return None
        rows = []
        try:
            for line in open(self.path):
                parts = [p.strip() for p in line.split(",")]
                if len(parts) >= 9 and parts[1].replace(".", "").isdigit():
                    rows.append(parts)
        except OSError:
            return None
        if not rows:
            return None
        sm = [float(r[1]) for r in rows]
        mx = float(rows[0][2])
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        reasons = sorted({n for r in rows for n, v in zip(names, r[5:9]) if v.lower() == "active"})
        loaded = [s for s in sm if s > 0.5 * mx] or sm
        return {"sm_mhz": statistics.median(loaded), "sm_max_mhz": mx, "reasons": reasons,
                "samples": len(rows), "power_w_max": max(float(r[3]) for r in rows if r[3].replace(".", "").isdigit())}


STEP_SOURCES = ("lbm13_internal.h", "lbm13_math.cuh", "lbm13_stepdev.cuh", "lbm13_step.cu")
PAIR_SOURCES = STEP_SOURCES + ("lbm13_pair.h", "lbm13_mbar.cuh", "lbm13_step2.cu")


def code_only(text):
    """C/C++ source without its comments and blank lines, trailing blanks
    dropped (string and character literals are kept as they are)."""
    out, i, n = [], 0, len(text)
    while i < n:
        c = text[i]
        if c in "\"'":
            j = i + 1
            while j < n and text[j] != c:
                j += 2 if text[j] == "\\" else 1
            out.append(text[i:j + 1])
            i = j + 1
        elif text.startswith("//", i):
            j = text.find("\n", i)
            i = n if j < 0 else j
        elif text.startswith("/*", i):
            j = text.find("*/", i + 2)
            i = n if j < 0 else j + 2
            out.append(" ")
        else:
            out.append(c)
            i += 1
    lines = (line.rstrip() for line in "".join(out).splitlines())
    return "\n".join(line for line in lines if line)


def kernel_hash(sources=STEP_SOURCES):
    """Hash of the code of the sources that define a kernel (its launch, body
    and arguments; the single-step kernel by default, PAIR_SOURCES for the
    paired one), comments left out: a profile record only applies to the
    kernel it was taken on, whatever its comments say since."""
    import hashlib
    src = os.path.join(ROOT, "paper_1401_0188_gb300", "csrc")
    h = hashlib.sha256()
    for name in sources:
        with open(os.path.join(src, name), encoding="utf-8") as f:
            h.update(code_only(f.read()).encode("utf-8"))
    return h.hexdigest()[:16]


def profile_record(fname, tag, sources=STEP_SOURCES):
    """The value recorded under `tag` in profiles/<fname> ("tag hash value"
    lines) if it was taken on the current source of its kernel; else None."""
    digest = kernel_hash(sources)
    try:
        for line in open(os.path.join(ROOT, "profiles", fname)):
            parts = line.split()
            if len(parts) == 3 and parts[0] == tag and parts[1] == digest:
                return float(parts[2])
    except OSError:
        pass
    return None


def traffic_record(tag):
    """Per-launch DRAM bytes of the step kernel from the committed ncu summary."""
    return profile_record("step_kernel_traffic.txt", tag)


def pair_record(tag):
    """Per-launch figures of the paired-step kernel (DRAM bytes, warp
    instructions per update) from its committed ncu summary."""
    return profile_record("pair_step_kernel_records.txt", tag, PAIR_SOURCES)


# Nominal FP64 rate of a GB300 (1.25 TFLOP/s at its 2070 MHz maximum SM
# clock: 2 FMA per SM per clock over 152 SMs), reported beside the measured
# rate as context only.
FP64_NOMINAL_FMA_PER_S = 2 * 152 * 2070e6


def oracle_served_check(served, budget_lu=1.5e9):
    """The oracle run on the served cavity with the fewest lattice updates to
    its stop (under budget_lu), for exactly the steps it was served: its FP64
    Nusselt number against the served FP32 one (same stopping point)."""
    from oracle import oracle as O
    from paper_1401_0188_gb300 import serving as S
    cav = [r for r in served if r.kind == "cavity" and r.converged]
    if not cav:
        return None
    r = min(cav, key=lambda r: r.nx * r.ny * r.steps)
    if r.nx * r.ny * r.steps > budget_lu:
        return {"skipped": f"cheapest served cavity needs {r.nx * r.ny * r.steps:.3g} updates"}
    req = S.Request(r.rid, "cavity", r.nx, r.Ra, r.Pr)
    nx, ny, p, bnd = S.request_setup(req)
    o = O.Lattice(nx, ny, p, bnd, nthreads=os.cpu_count() or 1)
    o.set_equilibrium(1.0, 0.0, 0.0, (p["E0"] + 28.0) / 26.0)
    t = time.perf_counter()
    o.step(r.steps)
    dt = time.perf_counter() - t
    nu = float(o.residual()[8])
    return {"rid": r.rid, "side": nx, "Ra": r.Ra, "Pr": r.Pr, "steps": r.steps, "Nu_oracle_fp64": nu,
            "Nu_served_fp32": r.Nu, "abs_err": abs(r.Nu - nu), "oracle_s": dt}


def cpu_baseline(steps_target_s=12.0, n=512):
    """The FP64 oracle as it stands, on the host cores: n x n shear wave."""
    import numpy as np
    from oracle import oracle as O
    from paper_1401_0188_gb300 import workloads as W
    cores = os.cpu_count() or 1
    p = O.pstar(NU, PR)
    lat = O.Lattice(n, n, p, nthreads=cores)
    ux, uy = W.shear_wave(n, n, 0.01)
    lat.set_equilibrium(1.0, ux, uy, (p["E0"] + 28) / 26)
    t = time.perf_counter()
    lat.step(2)
    per = (time.perf_counter() - t) / 2
    steps = max(2, int(steps_target_s / max(per, 1e-6)))
    t = time.perf_counter()
    lat.step(steps)
    dt = time.perf_counter() - t
    # the same oracle on one thread, for a bounded few seconds
    one = O.Lattice(n, n, p, nthreads=1)
    one.set_equilibrium(1.0, ux, uy, (p["E0"] + 28) / 26)
    t = time.perf_counter()
    one.step(1)
    per1 = time.perf_counter() - t
    steps1 = max(1, int(0.33 * steps_target_s / max(per1, 1e-6)))
    t = time.perf_counter()
    one.step(steps1)
    dt1 = time.perf_counter() - t
    return {"value": n * n * steps / dt / 1e6, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{n}x{n} periodic shear wave, {steps} steps, FP64 oracle, {cores} OpenMP threads",
            "one_thread": {"value": n * n * steps1 / dt1 / 1e6, "unit": UNIT, "cores": 1,
                           "sample": f"{n}x{n}, {steps1} steps, 1 thread"}}


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    import numpy as np
    from oracle import build as ob, oracle as O
    from paper_1401_0188_gb300 import workloads as W
    ob.build()
    n = 512
    cores = os.cpu_count() or 1
    p = O.pstar(NU, PR)
    lat = O.Lattice(n, n, p, nthreads=cores)
    ux, uy = W.shear_wave(n, n, 0.01)
    lat.set_equilibrium(1.0, ux, uy, (p["E0"] + 28) / 26)
    lat.step(args.warmup)
    t = time.perf_counter()
    lat.step(args.steps)
    dt = time.perf_counter() - t
    v = n * n * args.steps / dt / 1e6
    out = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": f"periodic shear wave u_x=0.01 sin(2 pi y/n), bounded sample {n}x{n} of the "
                                  f"{args.size}x{args.size} lattice (MLUPS is per node)", "nu": NU, "Pr": PR,
                      "precision": "fp64", "l2": "n/a (CPU)"},
           "cpu_baseline": {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle",
                            "sample": f"{n}x{n}, {args.steps} timed steps after {args.warmup}"},
           "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out))


def max_over_ranks(x, device, world):
    """Largest value of x over all ranks (the slowest replica sets the time)."""
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    if world > 1:
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return float(t.item())


def aggregate_mlups(nodes_per_rank, steps, seconds_max, world):
    """Whole-job throughput of N independent replicas: all ranks' lattice
    updates over the slowest rank's time (weak scaling)."""
    return world * nodes_per_rank * steps / seconds_max / 1e6


def time_steps(lat, steps, torch):
    stream = lat.stream
    start = torch.cuda.Event(enable_timing=True)
    end = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    start.record(stream)
    lat.step(steps)
    end.record(stream)
    end.synchronize()
    torch.cuda.synchronize()
    return start.elapsed_time(end)  # ms


def run_batched(args, torch):
    """256 uneven cavities (sides 64..512, Ra 1e3..1e6, Pr 0.5..1.0) stepped in
    one launch per step by an autotuned plan, FP32-deviation; against the same
    lattices in FP64, each with its own launches."""
    from paper_1401_0188_gb300 import lbm13, serving as S
    reqs = S.batch_workload(args.batched_count)
    out = {"workload": f"{args.batched_count} cavities, side uniform in {{64,96,128,192,256,384,512}}, "
                       "Ra log-uniform [1e3,1e6], Pr uniform [0.5,1.0], seed 4242, from rest"}

    def make(prec):
        lats = []
        for r in reqs:
            nx, ny, p, bnd = S.request_setup(r)
            g = lbm13.Lattice(nx, ny, p, bnd, precision=prec)
            g.set_state(1.0, 0.0, 0.0, (p["E0"] + 28) / 26)
            lats.append(g)
        return lats

    nodes = None
    for prec, name in ((lbm13.FP32_DEVIATION, "fp32_plan"), (lbm13.FP64, "fp64_per_lattice")):
        lats = make(prec)
        nodes = sum(g.nx * g.ny for g in lats)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        if name == "fp32_plan":
            plan = lbm13.Plan(lats)
            if args.batched_config:
                plan.set_config(*[int(v) for v in args.batched_config.split(",")])
            else:
                plan.tune(4)
            plan.step(8)
            torch.cuda.synchronize()
            e0.record()
            plan.step(args.batched_steps)
            e1.record()
            e1.synchronize()
            ms = e0.elapsed_time(e1) / args.batched_steps
            out["tune"] = plan.config()
            out["gpu_launches_per_step"] = 1
            plan.close()
        else:
            steps = max(4, args.batched_steps // 20)
            for g in lats:
                g.step(2)
            torch.cuda.synchronize()
            e0.record()
            for _ in range(steps):
                for g in lats:
                    g.step(1)
            e1.record()
            e1.synchronize()
            ms = e0.elapsed_time(e1) / steps
        out[name] = {"MLUPS": nodes / (ms / 1e3) / 1e6, "ms_per_step": ms}
        for g in lats:
            g.close()
        del lats
        torch.cuda.empty_cache()
    out["nodes_per_step"] = nodes
    out["speedup_vs_fp64_per_lattice"] = out["fp32_plan"]["MLUPS"] / out["fp64_per_lattice"]["MLUPS"]
    return out


def run_sweep(args, torch, peak):
    """The periodic shear wave at 512^2 .. 8192^2 in both precisions: MLUPS and
    the fraction of the HBM roofline (at 512^2 and 1024^2 the populations fit
    in the 129 MB L2, so that fraction is not an HBM measurement)."""
    from paper_1401_0188_gb300 import lbm13, pstar, rest_temperature, workloads as W
    p = pstar(NU, PR)
    T0 = rest_temperature(p)
    out = []
    for n in (512, 1024, 2048, 4096, 8192):
        for prec, name, bl in ((lbm13.FP32_DEVIATION, "fp32", 104), (lbm13.FP64, "fp64", 208)):
            lat = lbm13.Lattice(n, n, p, W.boundary(), precision=prec)
            ux, uy = W.shear_wave(n, n, 0.01)
            lat.set_state(1.0, ux, uy, T0)
            steps = 256 if name == "fp32" else 32
            lat.step(8)
            ms = time_steps(lat, steps, torch) / steps
            mlups = n * n / (ms / 1e3) / 1e6
            paired = lat.step_launches(steps) < steps  # two steps per launch: half the bytes per update
            out.append({"n": n, "precision": name, "MLUPS": mlups, "ms_per_step": ms, "paired": paired,
                        "hbm_frac": mlups * 1e6 * (bl // 2 if paired else bl) / 1e9 / peak,
                        "state_MB": 2 * 13 * bl // 26 * n * n / 1e6})
            lat.close()
            del lat
            torch.cuda.empty_cache()
    return out


def run_serving(args):
    """The fifth configuration as a bounded prefix: the first
    args.serving_requests requests of its Poisson stream (200 requests/s, seed
    5151, cavities and channels alternating, side log-uniform 64..1024, Ra
    log-uniform 1e3..1e6, Pr uniform 0.5..1.0, residual 1e-7, 120 GB budget),
    served in FP32-deviation storage with continuous batching; then the
    requests of side <= 128 of that prefix on both paths, FP32 served and plain
    FP64 one lattice per launch, for a like-for-like latency ratio."""
    from paper_1401_0188_gb300 import lbm13, serving as S
    reqs = S.poisson_trace(args.serving_requests, rate=200.0, seed=5151, side_range=(64, 1024),
                           ra_range=(1e3, 1e6), pr_range=(0.5, 1.0), tol=1e-7)
    res32, sum32 = S.Server(lbm13.FP32_DEVIATION, hbm_budget=120e9, check_every=1000).run(reqs)
    small = [r for r in reqs if r.L <= 128]
    s32, ssum32 = S.Server(lbm13.FP32_DEVIATION, hbm_budget=120e9, check_every=1000).run(small)
    s64, ssum64 = S.Server(lbm13.FP64, hbm_budget=120e9, check_every=1000, batched=False).run(small)
    nu_err = max((abs(a.Nu - b.Nu) for a, b in zip(s32, s64) if a.kind == "cavity"), default=0.0)
    served = [{"rid": r.rid, "kind": r.kind, "nx": r.nx, "ny": r.ny, "Ra": r.Ra, "Pr": r.Pr, "steps": r.steps,
               "tts_s": r.tts, "Nu": r.Nu, "converged": r.converged} for r in res32]
    return {"trace": f"first {len(reqs)} requests of the fifth configuration's stream: Poisson 200/s (seed 5151), "
                     "alternating cavity/channel, side log-uniform 64..1024, Ra log-uniform 1e3..1e6, Pr uniform "
                     "0.5..1.0, residual 1e-7, budget 120 GB, FP32-deviation, continuous batching",
            "fp32_batched": sum32, "requests_served": served,
            "small_subset": {"requests": [r.rid for r in small],
                             "fp32_batched": ssum32, "fp64_per_lattice": ssum64,
                             "p99_speedup": ssum64["p99_tts_s"] / ssum32["p99_tts_s"],
                             "nusselt_max_abs_err_fp32_vs_fp64": nu_err},
            "_results": res32}


def run_ours(args):
    import torch
    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    from paper_1401_0188_gb300 import build as lb
    if rank == 0 or world == 1:
        lb.build()
    if world > 1:
        torch.distributed.barrier()
    from paper_1401_0188_gb300 import lbm13, pstar, rest_temperature, workloads as W

    n = args.size
    p = pstar(NU, PR)
    T0 = rest_temperature(p)
    prec = lbm13.FP32_DEVIATION if args.precision == "fp32" else lbm13.FP64
    elem = 4 if prec == lbm13.FP32_DEVIATION else 8
    bytes_lu = 26 * elem
    dev = torch.device("cuda", local)

    def device_fields():
        y = torch.arange(n, device=dev, dtype=torch.float64)[:, None].expand(n, n)
        ux = (0.01 * torch.sin(2 * torch.pi * y / n)).contiguous()
        return (torch.ones(n, n, device=dev, dtype=torch.float64), ux,
                torch.zeros(n, n, device=dev, dtype=torch.float64),
                torch.full((n, n), T0, device=dev, dtype=torch.float64))

    lat = lbm13.Lattice(n, n, p, W.boundary(), precision=prec)
    if args.no_pairs:
        lat.set_pair_steps(lbm13.PAIR_OFF)
    f = device_fields()
    lat.set_state_device(*f)
    del f
    lat.step(args.warmup)
    lat.synchronize()
    if world > 1:
        torch.distributed.barrier()
    with Clocks(local) as clk:
        ms = time_steps(lat, args.steps, torch)
    if world > 1:
        torch.distributed.barrier()
    ms_max = max_over_ranks(ms, dev, world)
    per_step_s = ms / 1e3 / args.steps
    value = aggregate_mlups(n * n, args.steps, ms_max / 1e3, world)
    peak, peak_kind = measured_peaks()
    launches = lat.step_launches(args.steps)
    paired = launches < args.steps
    if paired:
        # two steps per launch: one read and one write of every population per
        # two updates (52 B per update); the kernel is bound by instruction
        # issue, so its roofline is the issue rate: 4 warp instructions per SM
        # per clock at the SM clock sampled during the timed region
        bytes_lu = 13 * elem
        clocks = clk.summary() or {}
        sm_mhz = clocks.get("sm_mhz") or 2070.0
        sms = torch.cuda.get_device_properties(dev).multi_processor_count
        issue_peak = 4 * sms * sm_mhz * 1e6 / 1e9
        ipl = pair_record(f"pair_{args.precision}_warp_instr_per_lu")
        traffic = pair_record(f"pair_{args.precision}_{n}")
        achieved_hbm = bytes_lu * n * n / per_step_s / 1e9
        roofline = {
            "bound": "alu", "unit": "G warp instr/s", "peak": issue_peak, "peak_kind": "derived",
            "peak_basis": f"4 warp instructions per SM per clock x {sms} SMs x {sm_mhz:.0f} MHz (sampled)",
            "achieved": None if ipl is None else ipl * n * n / per_step_s / 1e9,
            "frac": None if ipl is None else ipl * n * n / per_step_s / 1e9 / issue_peak,
            "instr_per_lu": ipl, "traffic": traffic,
            "hbm": {"achieved": achieved_hbm, "peak": peak, "unit": "GB/s", "frac": achieved_hbm / peak,
                    "bytes_per_lu": bytes_lu, "peak_kind": peak_kind},
            "kernel": "pair_step_kernel (two fused steps per launch: 28x28 tiles, intermediate state in "
                      "shared memory, persistent blocks, next tile by tensor copy)"}
    else:
        achieved = bytes_lu * n * n / per_step_s / 1e9
        roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                    "frac": achieved / peak, "traffic": traffic_record(f"step_{args.precision}_{n}"),
                    "peak_kind": peak_kind,
                    "kernel": "step_kernel (fused pull-stream + walls + MRT collision)"}

    # end to end through the C ABI with host buffers: upload fields, step, read back
    e2e = None
    if not args.no_e2e:
        y = torch.arange(n, dtype=torch.float64)[:, None].expand(n, n)
        host = [torch.ones(n, n, dtype=torch.float64).pin_memory(),
                (0.01 * torch.sin(2 * torch.pi * y / n)).contiguous().pin_memory(),
                torch.zeros(n, n, dtype=torch.float64).pin_memory(),
                torch.full((n, n), T0, dtype=torch.float64).pin_memory()]
        out = torch.empty(4, n, n, dtype=torch.float64).pin_memory()
        mask = 1 | lbm13.FIELD_UX | lbm13.FIELD_UY | lbm13.FIELD_T
        import ctypes
        dp = ctypes.POINTER(ctypes.c_double)
        ptrs = [ctypes.cast(h.data_ptr(), dp) for h in host]
        outp = ctypes.cast(out.data_ptr(), dp)
        L = lbm13.lib()
        # one untimed job first (staging buffers come from the caching allocator)
        lbm13._check(L.lbm13_set_state(lat.handle, *ptrs), lat.handle)
        lat.step(1)
        lbm13._check(L.lbm13_moments(lat.handle, outp, mask), lat.handle)
        torch.cuda.synchronize()
        if world > 1:
            torch.distributed.barrier()
        t0 = time.perf_counter()
        lbm13._check(L.lbm13_set_state(lat.handle, *ptrs), lat.handle)  # returns after the upload
        t1 = time.perf_counter()
        lat.step(args.steps)
        lat.synchronize()
        t2 = time.perf_counter()
        lbm13._check(L.lbm13_moments(lat.handle, outp, mask), lat.handle)  # returns after the download
        t3 = time.perf_counter()
        dt = t3 - t0
        e2e = {"value": aggregate_mlups(n * n, args.steps, max_over_ranks(dt, dev, world), world), "unit": UNIT,
               "h2d_bytes_per_step": 4 * 8 * n * n / args.steps, "d2h_bytes_per_step": 4 * 8 * n * n / args.steps,
               "split_ms": {"upload_and_init": 1e3 * (t1 - t0), "steps": 1e3 * (t2 - t1),
                            "readout_and_download": 1e3 * (t3 - t2)},
               "copy_fraction": ((t1 - t0) + (t3 - t2)) / dt,
               "note": f"per job: upload (rho,ux,uy,T) from pinned host, {args.steps} steps, download the same 4 fields"}
        del host, out
    lat.close()
    del lat
    torch.cuda.empty_cache()

    fp64 = None
    if not args.no_fp64 and prec != lbm13.FP64:
        lat = lbm13.Lattice(n, n, p, W.boundary(), precision=lbm13.FP64)
        f = device_fields()
        lat.set_state_device(*f)
        del f
        lat.step(3)
        ms64 = time_steps(lat, args.fp64_steps, torch)
        s64 = ms64 / 1e3 / args.fp64_steps
        fp64 = {"value": n * n / s64 / 1e6, "unit": UNIT, "ms_per_step": 1e3 * s64, "steps": args.fp64_steps,
                "bytes_per_lu": 208, "hbm_gbs": 208 * n * n / s64 / 1e9,
                "hbm_frac": 208 * n * n / s64 / 1e9 / peak}
        # bound by the FP64 pipe: FP64 instructions per node (DADD + DMUL +
        # DFMA, counted by ncu on this kernel source) against the FP64
        # instruction rate measured on this GPU by the library's FMA-chain
        # probe, right after the step's timing (clocks sampled during both)
        ops = profile_record("step_kernel_fp64_ops.txt", "fp64_instr_per_node")
        with Clocks(local) as clk64:
            rate, probe_s = lbm13.fp64_fma_rate(1 << 16)
        peak_alu = rate / 1e9
        fp64["roofline"] = {
            "bound": "alu", "unit": "G FP64 instr/s", "peak": peak_alu, "peak_kind": "measured",
            "achieved": None if ops is None else ops * n * n / s64 / 1e9,
            "frac": None if ops is None else ops * n * n / s64 / 1e9 / peak_alu,
            "instr_per_node": ops,
            "peak_basis": f"lbm13_fp64_fma_rate: 8 independent FMA chains per thread, 8 blocks of 256 per SM, "
                          f"{probe_s * 1e3:.1f} ms timed with CUDA events",
            "peak_clocks": clk64.summary(),
            "nominal_peak": FP64_NOMINAL_FMA_PER_S / 1e9}
        lat.close()
        del lat
        torch.cuda.empty_cache()

    sweep = None
    if not args.no_sweep:
        sweep = run_sweep(args, torch, peak)
    batched = None
    if not args.no_batched:
        batched = run_batched(args, torch)
    serving = None
    if not args.no_serving:
        serving = run_serving(args)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        from oracle import build as ob
        ob.build()
        cpu = cpu_baseline()
        if serving is not None:
            serving["nusselt_vs_oracle"] = oracle_served_check(serving["_results"])
    if serving is not None:
        serving.pop("_results", None)

    if rank == 0:
        res = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32" if elem == 4 else "f64", "data": "synthetic",
            "config": {"workload": f"periodic shear wave {n}x{n} (throughput sweep), u_x = 0.01 sin(2 pi y/n)",
                       "nu": NU, "Pr": PR, "precision": "fp32-deviation" if elem == 4 else "fp64",
                       "bytes_per_lu": bytes_lu, "steps_per_launch": 2 if paired else 1, "parallelism": f"replicas x{world}" if world > 1 else "single GPU",
                       "l2": f"inputs larger than L2 ({2 * 13 * elem * n * n / 1e9:.1f} GB of populations)"},
            "roofline": roofline,
            "gpu_launches": launches,
            "clocks": clk.summary(),
            "e2e": e2e,
            "fp64": fp64,
            "sweep": sweep,
            "batched": batched,
            "serving": serving,
            "cpu_baseline": cpu,
        }
        print(json.dumps(res))
    if world > 1:
        torch.distributed.destroy_process_group()


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
