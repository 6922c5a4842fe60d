"""Benchmark of the explicit hyperbolic-SGN step on one GB300 (or N replicas).

Workload: the second configuration -- 4096 x 4096 cells, dx = 10 m, 1:50 beach
from 200 m depth to dry land plus a Gaussian seamount, landslide-like Gaussian
depression (-5 m, radius 1 km), wet/dry shoreline with the SWE switch (h* = 20 m),
HSGN with alpha = 3, 64 gauges.  A step is one time step of the whole method over
the grid.  Prints one JSON line (driver contract).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--precision mixed|fp64] [--model hsgn|mbhsgn] [--nx 4096]

Under torchrun every rank runs an independent replica on its own GPU (the method
needs no exchange between replicas); rank 0 prints the aggregate.
"""
import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "cell-updates/s and % of HBM roofline; FP64 plain vs mixed/batched/learned"
UNIT = "cell-updates/s"
HBM_FALLBACK_GBS = 6800.0
# FP64 CUDA-core peak: 152 SMs x 2 DFMA/clk/SM x 2 flop x 2.07 GHz (the nominal
# 1.25 TFLOP/s of the part; 1.19 TFLOP/s measured with a DFMA loop at 1.99 GHz)
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.07e9 / 1e12
# FP32 CUDA-core peak: 152 SMs x 128 FFMA/clk/SM x 2 flop x 2.07 GHz
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12
# Instruction issue peak: 152 SMs x 4 schedulers x 1 warp instruction/clk x 32
# threads x 2.07 GHz, in thread instructions per second (the bound of a kernel
# whose time goes to issuing FP32/integer/select work, not to HBM)
ISSUE_PEAK_TINST = 152 * 4 * 32 * 2.07e9 / 1e12

# Counters per cell-update of each kernel, keyed by (model, precision, kernel,
# block shape) -- the shape the launch used, since the halo work of a face
# block depends on it; profiles/step_kernels_2048_counters.md (2048^2 is above
# L2, so per-cell figures carry over to 4096^2).  A kernel launched with a shape
# or code that these captures did not see reports null.
# FP64 flops (dadd + dmul + 2 dfma thread instructions / cells), FP64 path:
FLOPS_PER_CELL = {
    ("hsgn", "fp64", "k_prep", "32x8"): 133.2, ("hsgn", "fp64", "k_face_x", "64x4"): 312.9,
    ("hsgn", "fp64", "k_face_y", "16x16"): 326.3, ("hsgn", "fp64", "k_theta", "32x8"): 29.4,
    ("hsgn", "fp64", "k_update", "32x8"): 217.4,
}
# Issue slots per cell-update (ncu smsp__inst_executed x 32: thread instructions
# issued, predicated-off lanes included) of the one-pass kernel, HSGN mixed,
# 2048^2 (profiles/k_step_fused_2048_counters.md); the block key is 128 columns
# x the rows of its long chunks:
INSTR_PER_CELL = {
    ("hsgn", "mixed", "k_step_fused", "128x128"): 2126.4,
    ("hsgn", "mixed", "k_step_fused", "128x64"): 2228.7,
    ("hsgn", "mixed", "k_step_fused", "128x256"): 2075.0,
}
# DRAM bytes (read + write):
TRAFFIC_PER_CELL = {
    ("hsgn", "mixed", "k_step_fused", "128x128"): 67.4,
    ("hsgn", "mixed", "k_step_fused", "128x64"): 68.3,
    ("hsgn", "mixed", "k_step_fused", "128x256"): 66.5,
    **{("hsgn", "mixed", "k_prep", sh): 58 for sh in ("32x8", "32x4", "64x4")},
    ("hsgn", "mixed", "k_face_x", "128x2"): 128, ("hsgn", "mixed", "k_face_x", "256x1"): 128,
    ("hsgn", "mixed", "k_face_x", "64x4"): 129,
    **{("hsgn", "mixed", "k_face_y", sh): 129 for sh in ("32x8", "32x16", "64x4")},
    **{("hsgn", "mixed", "k_trans_x", sh): 106 for sh in ("32x4", "32x8", "64x4")},
    **{("hsgn", "mixed", "k_trans_y", sh): 107 for sh in ("32x4", "32x8", "64x4")},
    **{("hsgn", "mixed", "k_theta", sh): 17 for sh in ("32x8", "32x4", "64x4")},
    **{("hsgn", "mixed", "k_update", sh): 221 for sh in ("32x8", "32x4", "64x4")},
    ("hsgn", "fp64", "k_prep", "32x8"): 183, ("hsgn", "fp64", "k_face_x", "64x4"): 293,
    ("hsgn", "fp64", "k_face_y", "16x16"): 279, ("hsgn", "fp64", "k_theta", "32x8"): 37,
    ("hsgn", "fp64", "k_update", "32x8"): 441,
}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="mixed", choices=["mixed", "fp64"])
    ap.add_argument("--model", default="hsgn", choices=["hsgn", "mbhsgn", "swe"])
    ap.add_argument("--nx", type=int, default=4096)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-fp64-line", action="store_true")
    ap.add_argument("--no-batched", action="store_true", help="skip the refined-hierarchy (config 4) line")
    ap.add_argument("--batched-n0", type=int, default=1024, help="level-0 size of the config-4 hierarchy")
    ap.add_argument("--no-learned", action="store_true", help="skip the learned-corrector (config 5) line")
    ap.add_argument("--no-config3", action="store_true", help="skip the 8192^2 (config 3) mixed and FP64 rows")
    ap.add_argument("--config3-steps", type=int, default=30, help="timed mixed steps of the config-3 row")
    ap.add_argument("--tuning", default=None,
                    help="force a launch tuning (8 comma-separated option indices of sgn_set_tuning) instead of "
                         "autotuning")
    ap.add_argument("--fp64-check-steps", type=int, default=25,
                    help="fixed steps of the mixed-vs-FP64 error check beside the FP64 line")
    ap.add_argument("--no-regrid", action="store_true", help="skip the flag-driven regrid after the config-4 timing")
    ap.add_argument("--no-tune", action="store_true",
                    help="keep the default launch shapes (no sgn_autotune before timing)")
    ap.add_argument("--table-configs", default="1,2,3", help="configurations of --only table")
    ap.add_argument("--table-c2-steps", type=int, default=1000)
    ap.add_argument("--table-c3-steps", type=int, default=2000)
    ap.add_argument("--only", default=None, choices=["batched", "learned", "table"],
                    help="run only that line (for profiling); prints its object alone")
    return ap.parse_args()


def model_id(name):
    return {"swe": 0, "mbhsgn": 1, "hsgn": 2}[name]


def workload(args):
    from paper_2606_12162_gb300 import workloads as W
    m = model_id(args.model)
    dx = 10.0 * 4096 / args.nx
    c = W.config2(model=m, nx=args.nx, ny=args.nx, dx=dx)
    return c


def cfg_kwargs(c):
    return dict(dx=c["dx"], model=c["model"], bc=c["bc"], h_star=c["h_star"], alpha=c["alpha"],
                cfl=c["cfl"], dry_tol=c["dry_tol"])


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d.get("hbm_gbs", HBM_FALLBACK_GBS)), "measured"
    return HBM_FALLBACK_GBS, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu):
        self.gpu = gpu
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.Q, "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.th = threading.Thread(target=self._read, daemon=True)
            self.th.start()
        except (OSError, FileNotFoundError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.th.join(timeout=2)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(mx)), "reasons": sorted(reasons),
                "samples": len(sm)}


def dist_setup():
    import torch
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if ws > 1:
        import torch.distributed as dist
        backend = "nccl" if torch.cuda.is_available() else "gloo"
        if torch.cuda.is_available():
            torch.cuda.set_device(local)
        dist.init_process_group(backend=backend)
    elif torch.cuda.is_available():
        torch.cuda.set_device(0)
    return ws, rank, local


def reduce_max(x, ws):
    """Max over ranks (the slowest replica sets the time)."""
    if ws <= 1:
        return float(x)
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([float(x)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def barrier(ws):
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()


# Compulsory bytes per cell-update of each kernel of the step: every plane it
# reads or writes, once, for element size s, nvar fields nv (the depth plane and
# the positivity factors are FP64 in both precisions).
def kernel_bytes(name, nv, s):
    p = nv + 1 if s == 8 else 0            # primitive planes: FP64 path only
    if name == "k_prep":        # q, b, c2 -> W, P, depth
        return (nv + 2) * s + (nv + p) * s + 8
    if name in ("k_face_x", "k_face_y"):   # W, P, b, c2, psi, depth -> face planes
        return (nv + p + 3) * s + 8 + (2 * nv + 9) * s
    if name in ("k_trans_x", "k_trans_y"):  # other direction's Lv, Rv; Roe data, M -> T
        return (2 * nv + 9) * s + nv * s
    if name == "k_theta":       # two mass fluxes, eta, b -> theta
        return 4 * s + 8
    if name == "k_update":      # W, 4 face vectors, transverse fluxes, theta, b, c2 -> q
        return (nv + 4 * (nv - 1) + 2 * nv + 2 + nv) * s + 8
    if name == "k_step_fused":  # q, b, c2, psi_x, psi_y -> q
        return (2 * nv + 4) * s
    return 0


SLOT = {"k_prep": "prep", "k_face_x": "face_x", "k_face_y": "face_y", "k_trans_x": "trans_x",
        "k_trans_y": "trans_y", "k_theta": "theta", "k_update": "update",
        "k_step_fused": "update"}       # the one-pass kernel's block: 128 columns x rows per chunk


def roofline(model, prec, kt, cells, b_alg, nv, esize, hbm, hbm_src, shapes=None):
    """Roofline of the kernel with the largest time in kt (name -> (ms, launches)).
    FP64 path: bound by the FP64 pipe (flops counted by ncu per cell).  Mixed path:
    HBM; achieved = the step's algorithmic bytes per cell-update x cells of one
    launch / that kernel's average launch time; the kernel's own compulsory bytes
    and the ncu-measured traffic are reported beside it."""
    if not kt:
        return None
    name, (kms, kn) = max(kt.items(), key=lambda kv: kv[1][0])
    per = kms / 1e3 / max(kn, 1)
    shape = (shapes or {}).get(SLOT.get(name, ""), "")
    tr = TRAFFIC_PER_CELL.get((model, prec, name, shape))
    out = {"kernel": name, "block": shape, "launch_ms": per * 1e3, "share": kms / sum(v[0] for v in kt.values()),
           "traffic": tr * cells if tr else None}
    fl = FLOPS_PER_CELL.get((model, prec, name, shape))
    ins = INSTR_PER_CELL.get((model, prec, name, shape))
    if ins:
        # one-pass kernel: HBM roof (the step's algorithmic bytes) and issue roof
        # (ncu-counted thread instructions per cell); the lower one bounds it
        ach_b = b_alg * cells / per / 1e9
        ach_i = ins * cells / per / 1e12
        roof_b = hbm * 1e9 / b_alg
        roof_i = ISSUE_PEAK_TINST * 1e12 / ins
        alu = {"achieved": ach_i, "peak": ISSUE_PEAK_TINST, "unit": "Tinst/s", "frac": ach_i / ISSUE_PEAK_TINST,
               "inst_per_cell": ins, "roof_cell_updates_per_s": roof_i,
               "peak_source": "152 SMs x 4 schedulers x 32 threads x 2.07 GHz"}
        hb = {"achieved": ach_b, "peak": hbm, "unit": "GB/s", "frac": ach_b / hbm, "bytes_per_cell": b_alg,
              "roof_cell_updates_per_s": roof_b, "peak_source": hbm_src}
        main = alu if roof_i < roof_b else hb
        out.update({"bound": "alu" if roof_i < roof_b else "hbm", "achieved": main["achieved"],
                    "peak": main["peak"], "unit": main["unit"], "frac": main["frac"],
                    "hbm_frac": hb["frac"], "alu_frac": alu["frac"], "hbm": hb, "alu": alu})
    elif prec == "fp64" and fl:
        ach = fl * cells / per / 1e12
        ach_b = b_alg * cells / per / 1e9
        out.update({"bound": "alu", "achieved": ach, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                    "frac": ach / FP64_PEAK_TFLOPS, "flops_per_cell": fl, "alu_frac": ach / FP64_PEAK_TFLOPS,
                    "hbm_frac": ach_b / hbm,
                    "peak_source": "152 SMs x 2 DFMA/clk x 2 flop x 2.07 GHz (1.19 measured)"})
    else:
        ach = b_alg * cells / per / 1e9
        kb = kernel_bytes(name, nv, esize)
        out.update({"bound": "hbm", "achieved": ach, "peak": hbm, "unit": "GB/s", "frac": ach / hbm,
                    "bytes_per_cell": b_alg, "kernel_bytes_per_cell": kb,
                    "kernel_frac": kb * cells / per / 1e9 / hbm, "peak_source": hbm_src})
    return out


def cpu_baseline(args, budget_s=15.0):
    """The FP64 oracle as it stands, on the host cores, on a bounded crop of the
    same workload (a 384 x 384 window around the source, as many steps as fit)."""
    from oracle import oracle as O
    from paper_2606_12162_gb300 import workloads as W
    c = workload(args)
    cx, cy = c["source"]
    n = min(384, args.nx)
    i0 = int(min(max(cx / c["dx"] - n // 2, 0), args.nx - n))
    j0 = int(min(max(cy / c["dx"] - n // 2, 0), args.nx - n))
    sl = (slice(j0, j0 + n), slice(i0, i0 + n))
    b = c["b"][sl]
    q = c["q"][(slice(None),) + sl]
    o = O.Oracle(b, **cfg_kwargs(c))
    o.set_state(q)
    t0 = time.perf_counter()
    o.step(1)
    t1 = time.perf_counter()
    per = max(t1 - t0, 1e-6)
    k = max(1, int(budget_s / per))
    t0 = time.perf_counter()
    o.step(k)
    el = time.perf_counter() - t0
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    return {"value": n * n * k / el, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": "%dx%d crop of the 4096^2 workload around the source, %d steps, FP64 oracle" % (n, n, k),
            "seconds": el}


def run_reference(args):
    """Reference arm: the FP64 CPU oracle on the host cores, on the same workload,
    metric and unit (a bounded 256 x 256 crop per step)."""
    ws, rank, _ = int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("RANK", "0")), 0
    if rank != 0:
        return
    from oracle import oracle as O
    c = workload(args)
    cx, cy = c["source"]
    n = 256
    i0 = int(min(max(cx / c["dx"] - n // 2, 0), args.nx - n))
    j0 = int(min(max(cy / c["dx"] - n // 2, 0), args.nx - n))
    sl = (slice(j0, j0 + n), slice(i0, i0 + n))
    o = O.Oracle(c["b"][sl], **cfg_kwargs(c))
    o.set_state(c["q"][(slice(None),) + sl])
    o.step(args.warmup)
    t0 = time.perf_counter()
    o.step(args.steps)
    el = time.perf_counter() - t0
    v = n * n * args.steps / el
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": el / args.steps * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": "config2 %dx%d beach+seamount landslide, %s (oracle: %dx%d crop per step)"
                       % (args.nx, args.nx, args.model.upper(), n, n)},
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": "%dx%d crop around the source, %d steps" % (n, n, args.steps)},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def time_path(S, c, args, precision, prof_steps=None):
    """Warm-up, then exactly K steps between CUDA events on the solver stream:
    the product path (each step one CUDA-graph replay of the tuned schedule,
    no per-kernel events).  A separate pass of prof_steps steps afterwards
    (outside the timed region) launches the same kernels without the graph,
    each between two CUDA events, for the per-kernel times."""
    import torch
    s = S.Solver(c["b"], precision=precision, **cfg_kwargs(c))
    s.set_state(c["q"])
    kp = args.steps if prof_steps is None else prof_steps
    s.add_gauges(c["gauges"], args.steps + args.warmup + kp + 8)
    s.step(args.warmup)
    tuning = None
    if args.tuning:
        s.set_tuning([int(v) for v in args.tuning.split(",")])
        tuning = {"s": 0.0, "forced": args.tuning,
                  "shapes": {k: ("%dx%d" % v[1]) if k != "schedule" else v[0] for k, v in s.tuning().items()}}
    elif not args.no_tune:
        # autotuner (setup, outside the timed region): launch shapes per kernel
        t0 = time.perf_counter()
        s.autotune(reps=10)
        tuning = {"s": time.perf_counter() - t0,
                  "shapes": {k: ("%dx%d" % v[1]) if k != "schedule" else v[0] for k, v in s.tuning().items()}}
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    s.step(args.steps)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    f, dt, cr = s.status()
    kt = {}
    if kp > 0:
        s.set_profiling(True)
        s.step(kp)
        kt = s.kernel_times()
        s.set_profiling(False)
    s.tuning_report = tuning
    s.shapes = {k: "%dx%d" % v[1] for k, v in s.tuning().items() if k != "schedule"}
    s.schedule = s.tuning()["schedule"][0]
    return s, ms, kt, f


def mixed_error(S, c, steps):
    """Error of the mixed path against the FP64 path (itself equal to the FP64
    oracle to 1e-12 on the parity cases) on the full workload: both take the
    same `steps` fixed steps of 0.9 x the FP64 path's first CFL step from the
    same state; relative L2 of eta, hu, hv over wet cells and the largest
    surface error relative to the largest initial surface displacement."""
    out = {}
    for prec in (0, 1):
        s = S.Solver(c["b"], precision=prec, **cfg_kwargs(c))
        s.set_state(c["q"])
        if prec == 0:
            dt = 0.9 * s.next_dt()
        for _ in range(steps):
            s.step_dt(dt)
        out[prec] = s.get_state(0b111)[0]
        del s
    ref, got = out[0], out[1]
    b = c["b"]
    wet = ref[0] - b > 1e-3
    rel = [float(np.linalg.norm((got[k] - ref[k])[wet]) / max(np.linalg.norm(ref[k][wet]), 1e-300))
           for k in range(3)]
    eta0 = np.where(np.asarray(c["q"][0]) - b > 0, np.asarray(c["q"][0]), 0.0)
    return {"steps": steps, "dt_s": dt, "rel_l2": {"eta": rel[0], "hu": rel[1], "hv": rel[2]},
            "max_eta_err_rel": float(np.abs(got[0] - ref[0]).max() / max(np.abs(eta0).max(), 1e-300)),
            "tolerance": {"rel_l2": 1e-4, "max_eta_err_rel": 1e-3}}


def _oracle_rate(c, threads, budget_s, crop=384):
    """Oracle cell-updates/s on a crop (whole grid if smaller) around the
    source, in a fresh process with OMP_NUM_THREADS = threads."""
    code = r"""
import json, os, sys, time
import numpy as np
sys.path.insert(0, %r)
from oracle import oracle as O
d = np.load(sys.argv[1])
kw = json.loads(sys.argv[2])
o = O.Oracle(d["b"], **kw)
o.set_state(d["q"])
t0 = time.perf_counter(); o.step(1); per = max(time.perf_counter() - t0, 1e-6)
k = max(1, int(%f / per))
t0 = time.perf_counter(); o.step(k); el = time.perf_counter() - t0
print(json.dumps({"rate": d["b"].size * k / el, "steps": k, "seconds": el}))
""" % (ROOT, budget_s)
    import tempfile
    ny, nx = c["b"].shape
    n = min(crop, nx, ny)
    cx, cy = c.get("source", (0.5 * nx * c["dx"], 0.5 * ny * c["dx"]))
    i0 = int(min(max((cx - c.get("x0", 0.0)) / c["dx"] - n // 2, 0), nx - n))
    j0 = int(min(max((cy - c.get("y0", 0.0)) / c["dx"] - n // 2, 0), ny - n))
    sl = (slice(j0, j0 + n), slice(i0, i0 + n))
    with tempfile.TemporaryDirectory() as td:
        f = os.path.join(td, "crop.npz")
        np.savez(f, b=c["b"][sl], q=c["q"][(slice(None),) + sl])
        env = dict(os.environ, OMP_NUM_THREADS=str(threads))
        r = subprocess.run([sys.executable, "-c", code, f, json.dumps(cfg_kwargs(c))], env=env,
                           capture_output=True, text=True)
    if r.returncode:
        return {"error": r.stderr[-300:]}
    out = json.loads(r.stdout.strip().splitlines()[-1])
    out.update(threads=threads, crop=n)
    return out


def _arrivals(rec, frac):
    """First record time per gauge where |eta - eta(first record)| exceeds frac
    (NaN where it never does)."""
    eta = rec[:, :, 1]
    hit = np.abs(eta - eta[0][None, :]) > frac
    out = np.full(eta.shape[1], np.nan)
    for g in range(eta.shape[1]):
        k = np.nonzero(hit[:, g])[0]
        if len(k):
            out[g] = rec[k[0], g, 0]
    return out


def config_row(S, name, c, steps, rate_steps, warmup=3):
    """One row of the results table: FP64 and mixed cell-updates/s (CFL steps,
    graph replay, CUDA events), and the mixed path's error against the FP64
    path after `steps` steps, both driven by the same dt (the smaller of their
    two CFL steps; the FP64 path equals the oracle to 1e-12 on the parity
    cases): relative L2 over wet cells, largest surface error relative to the
    largest initial displacement, gauge arrival times (1 % of that
    displacement) in units of the mean step."""
    import torch
    kw = dict(cfg_kwargs(c), x0=c.get("x0", 0.0), y0=c.get("y0", 0.0))
    cells = c["b"].size
    row = {"config": name, "cells": cells}
    for prec, key in ((0, "fp64"), (1, "mixed")):
        s = S.Solver(c["b"], precision=prec, **kw)
        s.set_state(c["q"])
        s.step(warmup)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        st = torch.cuda.current_stream()
        torch.cuda.synchronize()
        e0.record(st)
        s.step(rate_steps)
        e1.record(st)
        torch.cuda.synchronize()
        row[key] = cells * rate_steps / (e0.elapsed_time(e1) / 1e3)
        del s
    eta0 = np.where(c["q"][0] - c["b"] > 0, c["q"][0], 0.0)
    amp = float(np.abs(eta0).max())
    sv = {}
    for prec in (0, 1):
        sv[prec] = S.Solver(c["b"], precision=prec, **kw)
        sv[prec].set_state(c["q"])
        if c.get("gauges") is not None:
            sv[prec].add_gauges(c["gauges"], steps + 2)
    t = 0.0
    for _ in range(steps):
        # the smaller of the two CFL steps, so that neither path exceeds its own
        dt = min(sv[0].next_dt(), sv[1].next_dt())
        sv[0].step_dt(dt)
        sv[1].step_dt(dt)
        t += dt
    ref, got = sv[0].get_state(0b111)[0], sv[1].get_state(0b111)[0]
    wet = ref[0] - c["b"] > 1e-3
    rel = [float(np.linalg.norm((got[k] - ref[k])[wet]) / max(np.linalg.norm(ref[k][wet]), 1e-300))
           for k in range(3)]
    err = {"steps": steps, "t_s": t, "rel_l2": {"eta": rel[0], "hu": rel[1], "hv": rel[2]},
           "max_eta_err_rel": float(np.abs(got[0] - ref[0]).max() / amp)}
    if c.get("gauges") is not None:
        ga, gb = _arrivals(sv[0].gauges(), 0.01 * amp), _arrivals(sv[1].gauges(), 0.01 * amp)
        seen = ~np.isnan(ga) & ~np.isnan(gb)
        err["gauges_with_arrival"] = int(seen.sum())
        err["arrival_diff_max_in_dt"] = float(np.abs(ga - gb)[seen].max() / (t / steps)) if seen.any() else None
        err["arrival_mismatch"] = int((np.isnan(ga) != np.isnan(gb)).sum())
    row["mixed_vs_fp64"] = err
    del sv
    return row


def results_table(args):
    """Rows of the results table for configurations 1-3 (HSGN): GPU FP64 and
    mixed throughput, the mixed error against FP64 over the configuration's
    step count, and the oracle on the host cores, one thread and all."""
    from paper_2606_12162_gb300 import sgn as S, workloads as W
    rows = []
    for k, (name, make, steps, rate_steps) in enumerate((
            ("config1 256^2 dx=0.05 m soliton", lambda: W.config1(model=W.HSGN), 200, 200),
            ("config2 4096^2 dx=10 m beach + landslide", lambda: W.config2(model=W.HSGN), args.table_c2_steps, 100),
            ("config3 8192^2 dx=500 m fractal + uplift", lambda: W.config3(model=W.HSGN), args.table_c3_steps, 50))):
        if str(k + 1) not in args.table_configs.split(","):
            continue
        c = make()
        row = config_row(S, name, c, steps, rate_steps)
        row["oracle_1_thread"] = _oracle_rate(c, 1, 8.0)
        row["oracle_all_cores"] = _oracle_rate(c, os.cpu_count() or 1, 8.0)
        rows.append(row)
        print(json.dumps(row), flush=True)
        del c
    return rows


def time_config3(S, args, hbm, hbm_src, ws):
    """Configuration 3 (8192^2, dx = 500 m, fractal bathymetry, 2 m uplift, HSGN):
    mixed (autotuned; one graph replay per step) and FP64 cell-updates/s between
    CUDA events with the clocks sampled over each timed region, then a profiled
    pass of each for the dominant kernel's roofline (outside the timed regions)."""
    import copy
    import torch
    from paper_2606_12162_gb300 import workloads as W
    t0 = time.perf_counter()
    c = W.config3(model=W.HSGN)
    c["gauges"] = c.get("gauges")
    if c["gauges"] is None:
        c["gauges"] = np.zeros((0, 2))
    setup = time.perf_counter() - t0
    cells = c["b"].size
    nv = S.NVAR[W.HSGN]
    out = {"workload": "config3: 8192x8192, dx=500 m, fractal bathymetry (|k|^-2, ~20 % land, to -6000 m), "
                       "2 m Gaussian uplift (r=30 km), HSGN alpha=3, 64 gauges", "setup_s": setup}
    local = int(os.environ.get("LOCAL_RANK", "0"))
    for prec, key, steps in ((1, "mixed", args.config3_steps), (0, "fp64", max(3, args.config3_steps // 6))):
        a2 = copy.copy(args)
        a2.steps, a2.warmup = steps, 3
        if prec == 0:
            a2.no_tune, a2.tuning = True, None
        clk = ClockSampler(local)
        clk.start()
        s, ms, kt, f = time_path(S, c, a2, prec, prof_steps=min(steps, 5))
        clocks = clk.stop()
        ms = reduce_max(ms, ws)
        b_alg = nv * 2 * (4 if prec else 8) + (4 if prec else 8) + 1
        v = cells * steps * ws / (ms / 1e3)
        out[key] = {"value": v, "unit": UNIT, "steps": steps, "ms_per_step": ms / steps, "status_flags": f,
                    "dtype": "f32+f64" if prec else "f64", "clocks": clocks, "tuning": s.tuning_report,
                    "hbm_fraction_step": v / ws * b_alg / (hbm * 1e9),
                    "roofline": roofline("hsgn", key, kt, cells, b_alg, nv, 4 if prec else 8, hbm, hbm_src,
                                         s.shapes),
                    "kernels_ms_per_step": {k: v2[0] / max(v2[1], 1) for k, v2 in kt.items() if v2[1]},
                    "gpu_launches": s.launches_per_step() * steps}
        del s
        torch.cuda.empty_cache()
    del c
    return out


def time_batched(args):
    """Config 4 (three levels, ratio 4, ~2000 patches along a wave front), mixed
    precision: W level-0 steps of warm-up, then K level-0 steps (each with all
    finer substeps, one CUDA graph) between CUDA events on the stream."""
    import torch
    from paper_2606_12162_gb300 import amr, workloads as W
    t0 = time.perf_counter()
    c = W.config4(n0=args.batched_n0)
    g = amr.Hierarchy(c["b"], c["n0"], c["n0"], c["dx0"], c["r"], c["boxes"], model=c["model"], bc=c["bc"],
                      precision=1, alpha=c["alpha"], h_star=c["h_star"], cfl=c["cfl"], dry_tol=c["dry_tol"])
    for l, lv in enumerate(c["states"]):
        for k, q in enumerate(lv):
            g.set_patch(l, k, q)
    setup = time.perf_counter() - t0
    b_finest = c.pop("b")
    rc0 = g.step_rc(max(1, args.warmup))
    tune = None
    if rc0 == 0 and not args.no_tune:
        t1 = time.perf_counter()
        ch, _ = g.autotune(reps=5)
        tune = {"s": time.perf_counter() - t1, "choice_per_level": ch.tolist()}
    k = max(3, min(args.steps, 20))
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    rc = g.step_rc(k) if rc0 == 0 else rc0
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    cells, atlas = g.info()
    r = c["r"]
    per_step = sum(n * r ** l for l, n in enumerate(cells))           # interior cell-updates per level-0 step
    atlas_per_step = sum(n * r ** l for l, n in enumerate(atlas))
    nf = c["n0"] * r ** (len(cells) - 1)
    fine_equiv = float(nf) * nf * r ** (len(cells) - 1)                # uniform finest grid, same span
    m, clipped = g.mass()
    launches = g.launches_per_step() * k
    # one flag-driven regrid after the timed region (outside it): the patches
    # move from the ring onto the cells whose surface jump exceeds 5 cm, then
    # three more level-0 steps, with retaking of steps over the CFL limit (the
    # new patches start from interpolated states), check the new hierarchy
    regrid = None
    if rc == 0 and not args.no_regrid:
        try:
            torch.cuda.synchronize()
            t1 = time.perf_counter()
            nb = g.regrid_flagged(b_finest, 0.05, 16, 2)
            torch.cuda.synchronize()
            regrid = {"s": time.perf_counter() - t1, "tol_m": 0.05, "tile": 16, "buffer": 2,
                      "patches_per_level": [1] + nb}
            g.set_retake(4)
            regrid["status_after_3_steps"] = g.step_rc(3)
            regrid["steps_retaken"] = g.retakes()
        except Exception as ex:          # reported, not fatal to the line
            regrid = {"error": str(ex)[:200]}
    del b_finest
    return {"value": per_step * k / (ms / 1e3), "unit": UNIT, "steps": k, "ms_per_step": ms / k,
            "dtype": "f32+f64", "status": rc,
            "workload": "config4: 3 levels, ratio 4, level 0 %dx%d at 2 km, fractal bathymetry + coast strip, "
                        "%d patches (16..128 cells) along a ring front, 2 m Gaussian uplift, HSGN"
                        % (c["n0"], c["n0"], sum(len(b) for b in c["boxes"])),
            "patches_per_level": [1] + [len(b) for b in c["boxes"]],
            "interior_cells_per_level": cells, "atlas_cells_per_level": atlas,
            "cell_updates_per_step": per_step, "atlas_cell_updates_per_step": atlas_per_step,
            "fine_equivalent_cell_updates_per_s": fine_equiv * k / (ms / 1e3),
            "gpu_launches": launches, "setup_s": setup, "tuning": tune, "regrid": regrid,
            "mass": m, "clipped": clipped}


def time_learned(args, nc=1024, r=4, dxc=2000.0, n_train=8, held=(8, 9), iters=3000, thr=0.02,
                 times=(60.0, 120.0, 180.0, 240.0, 300.0)):
    """Config 5 (coarse 1024^2 at 2 km, fine 4096^2 at 500 m, ratio 4): the
    learned form measured end to end.  The library generates the coarse/fine
    pairs of n_train scenarios and trains the corrector on them (setup, outside
    the measurement); on each held-out scenario it then runs the learned form
    with its runtime fallback (corrector.hybrid_run: a plain coarse solve, the
    network's corrected prolongation at the output times, and patches of the
    plain fine solve where the a-priori surface-jump flag fires on the coarse
    state) and compares the fine-level surface at the output times with the
    plain fine solve of the same scenario.  Rate = fine-level cell-updates the
    plain fine solve makes over the same simulated time / the learned form's
    wall time (stepping, regrids, network and assembly included)."""
    import torch
    from paper_2606_12162_gb300 import corrector as C
    t0 = time.perf_counter()
    stats = {}
    pairs, meta = C.generate_pairs(nc, r, dxc, list(range(n_train)) + list(held), times,
                                   keep_fine=lambda s: s in held, gauges=64, stats=stats)
    gen_s = time.perf_counter() - t0
    trn = [p for p in pairs if p["scenario"] < n_train]
    hp = [p for p in pairs if p["scenario"] in held]
    net = C.Net(cin=5, width=32, depth=5, r=r, max_hw=nc * nc, seed=5000)
    t0 = time.perf_counter()
    losses = C.train(net, trn, iters, 128, 1e-3)
    train_s = time.perf_counter() - t0
    ocean_f, ocean_c = C.ocean_masks(meta)
    ev = {(q["scenario"], q["time"]): q for q in C.evaluate(net, hp, 16, 0.1, ocean_f=ocean_f, ocean_c=ocean_c)}
    m = ocean_f.to(torch.float64)
    nt = len(times)
    ok = stats["ok"]
    fine_s = dict(zip(ok, np.array(stats["fine_s"]).reshape(len(ok), nt).sum(axis=1)))
    fine_steps = dict(zip(ok, np.array(stats["fine_steps"]).reshape(len(ok), nt).sum(axis=1)))
    nf2 = float(nc * r) ** 2
    rows, wall, fine_updates, fine_wall = [], 0.0, 0.0, 0.0
    for s in [h for h in held if h in ok]:
        ref = {q["time"]: q["qf"] for q in hp if q["scenario"] == s}
        errs = {}

        def cb(T, fine):
            d = fine[0] - ref[T][0]
            errs[T] = ((torch.linalg.norm(d * m) / torch.linalg.norm(ref[T][0] * m)).item(),
                       ((d * m).abs().max() / (ref[T][0] * m).abs().max()).item())

        res = C.hybrid_run(net, meta, s, times, cb, thr=thr, regrid_every=16, buffer=6)
        w = res["step_s"] + res["regrid_s"] + res["snapshot_s"]
        wall += w
        fine_updates += nf2 * fine_steps[s]
        fine_wall += fine_s[s]
        g = stats["gauges"][s]
        ta, tb = C.arrival_times(g["coarse"]), C.arrival_times(g["fine"])
        keep = np.isfinite(ta) & np.isfinite(tb)
        rows.append({"scenario": s, "wall_s": w, "fine_solve_s": float(fine_s[s]),
                     "step_s": res["step_s"], "regrid_s": res["regrid_s"], "snapshot_s": res["snapshot_s"],
                     "regrids": res["regrids"], "patch_frac": res["patch_frac"],
                     "eta_rel_l2": [errs[T][0] for T in times], "eta_max_err_rel": [errs[T][1] for T in times],
                     "eta_rel_l2_network_alone": [ev[(s, T)]["rel_net"] for T in times],
                     "eta_rel_l2_prolongation": [ev[(s, T)]["rel_prolong"] for T in times],
                     "gauge_arrival_abs_diff_s": {"median": float(np.median(np.abs(ta[keep] - tb[keep])))
                                                  if keep.any() else None,
                                                  "max": float(np.abs(ta[keep] - tb[keep]).max()) if keep.any()
                                                  else None, "gauges": int(keep.sum())}})
    el = [e for rr in rows for e in rr["eta_rel_l2"]]
    return {"value": fine_updates / wall if wall > 0 else None, "unit": UNIT, "dtype": "f32+f64 solve, bf16 network",
            "fine_cell_updates": fine_updates, "wall_s": wall,
            "workload": "config5: coarse %dx%d at %.0f m + corrector to %dx%d (ratio %d), fractal bathymetry (seed "
                        "5001), %d training scenarios (%d iterations, in-bench), held-out scenarios %s, output at "
                        "%s s" % (nc, nc, dxc, nc * r, nc * r, r, n_train, iters, list(held), list(times)),
            "fine_mixed_cell_updates_per_s": fine_updates / fine_wall if fine_wall > 0 else None,
            "speedup_vs_fine_mixed": fine_wall / wall if wall > 0 else None,
            "eta_rel_l2_max": max(el) if el else None, "eta_rel_l2_median": float(np.median(el)) if el else None,
            "fallback_flag_m": thr, "rows": rows, "setup": {"pairs_s": gen_s, "train_s": train_s,
                                                          "loss_first_last": [float(losses[:50].mean()),
                                                                              float(losses[-50:].mean())]},
            "gauges_note": "arrival times of the coarse solve (the learned form's time series between output "
                           "times) against the fine solve"}


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
        return
    import torch
    from paper_2606_12162_gb300 import build, sgn as S
    ws, rank, local = dist_setup()
    build.build()
    S.load()
    if args.only == "table":
        if rank == 0:
            print(json.dumps({"table": results_table(args)}), flush=True)
        return
    if args.only:
        res = time_batched(args) if args.only == "batched" else time_learned(args)
        if rank == 0:
            print(json.dumps({args.only: res}), flush=True)
        return
    c = workload(args)
    prec = 1 if args.precision == "mixed" else 0
    nv = S.NVAR[c["model"]]
    cells = args.nx * args.nx
    esize = 4 if prec == 1 else 8
    hbm, hbm_src = peaks()

    clk = ClockSampler(local)
    barrier(ws)
    clk.start()
    s, ms, kt, flags = time_path(S, c, args, prec, prof_steps=min(args.steps, 20))
    clocks = clk.stop()
    ms = reduce_max(ms, ws)
    value = cells * args.steps * ws / (ms / 1e3)
    launches = s.launches_per_step() * args.steps

    # dominant kernel and its roofline
    b_alg = (nv * 2 * esize + esize + 1)   # algorithmic bytes per cell-update of the step
    roof = roofline(args.model, args.precision, kt, cells, b_alg, nv, esize, hbm, hbm_src, s.shapes)
    step_hbm_frac = value / ws * b_alg / (hbm * 1e9)

    # end to end through the C ABI with pinned host buffers
    e2e = None
    if not args.no_e2e:
        ke = max(1, min(args.steps, 10))
        hq = torch.from_numpy(np.ascontiguousarray(c["q"])).pin_memory()
        out = torch.empty_like(hq).pin_memory()
        s.set_state_ptr(hq.data_ptr())
        s.step(1)
        s.get_state_ptr(out.data_ptr(), out.numel())
        torch.cuda.synchronize()
        barrier(ws)
        t0 = time.perf_counter()
        for _ in range(ke):
            s.set_state_ptr(hq.data_ptr())
            s.step(1)
            s.get_state_ptr(out.data_ptr(), out.numel())
        torch.cuda.synchronize()
        el = reduce_max(time.perf_counter() - t0, ws)
        nb = nv * cells * 8
        e2e = {"value": cells * ke * ws / el, "unit": UNIT, "h2d_bytes_per_step": nb, "d2h_bytes_per_step": nb,
               "steps": ke}

    # FP64 plain path beside the mixed one (same workload, fewer steps)
    extra = None
    if prec == 1 and not args.no_fp64_line:
        import copy
        a2 = copy.copy(args)
        a2.steps = max(3, min(args.steps, 20))
        # default launch shapes (the FP64 counters' shapes); tuning gains nothing
        # measurable on this FP64-pipe-bound path (33.0 vs 33.1 ms per step)
        a2.no_tune, a2.tuning = True, None
        s2, ms2, kt2, f2 = time_path(S, c, a2, 0, prof_steps=a2.steps)
        ms2 = reduce_max(ms2, ws)
        v2 = cells * a2.steps * ws / (ms2 / 1e3)
        extra = {"value": v2, "unit": UNIT, "steps": a2.steps, "ms_per_step": ms2 / a2.steps,
                 "dtype": "f64", "tuning": s2.tuning_report,
                 "roofline": roofline(args.model, "fp64", kt2, cells, nv * 16 + 9, nv, 8, hbm, hbm_src,
                                      s2.shapes),
                 "hbm_fraction_step": v2 / ws * (nv * 16 + 9) / (hbm * 1e9),
                 "kernels_ms_per_step": {k: v[0] / max(v[1], 1) for k, v in kt2.items() if v[1]}}
        del s2
        extra["mixed_vs_fp64"] = mixed_error(S, c, args.fp64_check_steps)

    config3 = None
    if not args.no_config3:
        config3 = time_config3(S, args, hbm, hbm_src, ws)

    batched = None
    if not args.no_batched:
        batched = time_batched(args)
        bms = reduce_max(batched["ms_per_step"], ws)          # replicas: slowest rank
        batched["value"] = batched["cell_updates_per_step"] * ws / (bms / 1e3)
        batched["fine_equivalent_cell_updates_per_s"] *= ws * batched["ms_per_step"] / bms
        batched["ms_per_step"] = bms
        if extra:
            batched["vs_fp64_uniform"] = batched["value"] / extra["value"]

    learned = None
    if not args.no_learned:
        learned = time_learned(args)
        if learned["value"]:
            # replicas: the slowest rank's wall time for every rank's work
            learned["value"] = learned["fine_cell_updates"] * ws / reduce_max(learned["wall_s"], ws)
        if extra and learned["value"]:
            learned["vs_fp64_uniform"] = learned["value"] / extra["value"]

    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu:
        cpu = cpu_baseline(args)

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None,
            "dtype": "f32+f64" if prec == 1 else "f64", "data": "synthetic",
            "config": {"workload": "config2: %dx%d, dx=%.1f m, 1:50 beach + seamount, -5 m landslide "
                                   "depression, wet/dry + SWE switch (h*=20 m), 64 gauges"
                                   % (args.nx, args.nx, c["dx"]),
                       "model": args.model.upper(), "precision": args.precision, "alpha": 3.0,
                       "parallelism": "replicas" if ws > 1 else "single",
                       "l2": "inputs larger than L2 (state %.0f MB per buffer)" % (nv * cells * esize / 1e6),
                       "tuning": s.tuning_report},
            "roofline": roof,
            "hbm_fraction_step": step_hbm_frac,
            "algorithmic_bytes_per_cell": b_alg,
            "kernels_ms_per_step": {k: v[0] / max(v[1], 1) for k, v in kt.items() if v[1]},
            "status_flags": flags,
            "gpu_launches": launches,
            "clocks": clocks,
            "e2e": e2e,
            "cpu_baseline": cpu,
            "fp64": extra,
            "config3": config3,
            "batched": batched,
            "learned": learned,
        }
        print(json.dumps(line), flush=True)
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
