#!/usr/bin/env python
"""Throughput of the fused relativistic lattice Boltzmann step on GB300.

One step = one launch of the fused kernel (pull-streaming with bounce-back, moments,
Landau matching, equilibrium, Anderson-Witting relaxation, projected stirring force,
store) over the whole lattice, plus the stirring table the same launch prepares for
the next step.  Default workload: 1024 x 1024 periodic lattice, FP32, eps0 = 1 at
rest, stirring shell 8 <= |k| <= 10 with amplitude 1e-4 redrawn every step, eta/s =
0.05, dt = 0.05, a = 0.1.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference] [--no-forms]

With N > 1 (torchrun), every rank advances its own independently seeded lattice
(replicas: the update has no cross-lattice exchange), and `value` counts the cell
updates of all ranks over the slowest rank's time.  L2 is flushed (a 256 MiB write)
before every timed step; only the step launches are inside the CUDA-event windows.

The line also carries `forms` (rank 0 of a one-GPU run): the same workload as it runs
(chained 500-step blocks between spectra), a 4096^2 lattice, the graphene-like sample in
FP16 and FP32, the 64-member ensemble batched in FP16 and BF16 against the plain FP32
form run member by member, and the time per gradient of the adjoint, each with its
roofline and its velocity error on a 200-step slice against the FP64 path.
"""
import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "MLUPS & HBM GB/s fraction of peak, plain vs mixed/batched at stated error"
ALG_BYTES = {"f64": 272, "f32": 136, "f16": 68, "bf16": 68}  # 2 x 17 planes x storage bytes per cell update
FALLBACK_HBM_GBS = 6800.0
TRAFFIC_FILE = os.path.join(ROOT, "profiles", "ncu_step_kernel_stirred1024_f32.txt")
CHAINED_TRAFFIC_FILE = os.path.join(ROOT, "profiles", "ncu_step_kernel_stirred1024_f32_chained.txt")


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=20000)
    p.add_argument("--warmup", type=int, default=20)
    p.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    p.add_argument("--nx", type=int, default=1024)
    p.add_argument("--ny", type=int, default=1024)
    p.add_argument("--precision", default=None, choices=["f64", "f32", "f16", "bf16"],
                   help="storage type (default: f32; f16 for the graphene and ensemble workloads)")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-forms", action="store_true", help="skip the other forms (C2 chained, C2', C3, C4, C5)")
    p.add_argument("--shape", default=None,
                   help="ctas,stages,stir_rows: use this launch shape instead of tuning (profiling runs)")
    p.add_argument("--members", type=int, default=64,
                   help="ensemble64: number of members (64; fewer only for profiling runs)")
    p.add_argument("--adjoint-steps", type=int, default=2000,
                   help="adjoint512: steps of the differentiated run (2000; fewer only for profiling runs)")
    p.add_argument("--workload", default="stirred",
                   choices=["stirred", "chained", "ensemble64", "adjoint512", "graphene", "channel"],
                   help="stirred: one lattice (default); chained: the same in 500-step chained blocks, as the "
                        "workload runs; ensemble64: 64 stirred members of uneven sizes "
                        "advanced by one persistent launch per step; adjoint512: gradient of the kinetic "
                        "energy of a 512^2 stirred run (2000 steps) by the checkpointed adjoint")
    a = p.parse_args()
    if a.precision is None:
        a.precision = "f16" if a.workload in ("graphene", "ensemble64") else "f32"
    return a


# the stirred workload's job: 20 000 steps, energy spectrum every 500 steps
E2E_JOB_STEPS, E2E_SPECTRUM_EVERY = 20000, 500


def slowest(duration, world, device):
    """The job time of N replicas: the largest of the ranks' durations (all-reduce max over
    the process group; `device` is where the group's tensors live: "cuda" for NCCL, "cpu"
    for gloo).  One rank: the duration itself."""
    if world <= 1:
        return float(duration)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(duration)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_mlups(world, cells, steps, seconds):
    """Whole-job throughput of N replicas of `cells` cells each, `steps` steps in `seconds`."""
    return world * cells * steps / seconds / 1e6


def workload(args, rank):
    return dict(eta_over_s=0.05, kmin=8, kmax=10, force_amp=1e-4, seed=2 + rank)


def workload_name(args):
    return ("stirred %dx%d %s, shell 8<=|k|<=10, amp 1e-4 (Philox per step and mode), eta/s 0.05, "
            "dt 0.05, a 0.1, eps0 1 at rest" % (args.nx, args.ny, args.precision.upper()))


STEP_KERNEL_SOURCES = ("rlbm_device.cuh", "rlbm_kernels.cuh", "rlbm_tma.cuh", "rlbm_launch.h", "rlbm_kernels_f32.cu")


def csrc_digest():
    """Digest of the sources the FP32 step kernel is compiled from (the kernel whose ncu
    counters profiles/ holds); a change there invalidates the committed traffic figure."""
    h = hashlib.sha256()
    d = os.path.join(ROOT, "paper_2205_04658_gb300", "csrc")
    for f in STEP_KERNEL_SOURCES:
        h.update(open(os.path.join(d, f), "rb").read())
    return h.hexdigest()[:16]


def measured_peak():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback"


def traffic_from(path, workload):
    """DRAM bytes per launch from a committed ncu summary, if it was taken on the current
    step-kernel sources and on `workload`; else None."""
    try:
        kv = {}
        for line in open(path):
            if ":" in line and not line.startswith("#"):
                k, v = line.split(":", 1)
                kv[k.strip()] = v.strip()
        if kv.get("source_digest") != csrc_digest():
            return None
        if kv.get("workload") != workload:
            return None
        return float(kv["dram_bytes_per_launch"])
    except Exception:
        return None


def committed_traffic(args):
    """DRAM bytes per launch of the timed kernel from the committed ncu summary, if it was
    taken on the current kernel source and this workload; else None."""
    return traffic_from(TRAFFIC_FILE, "%dx%d %s" % (args.nx, args.ny, args.precision))


class Clocks:
    """nvidia-smi samples (200 ms) of the SM clock and throttle reasons while running."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device):
        self.device = device  # index or "GPU-<uuid>"
        self.lines = []
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "--id=%s" % self.device, "--query-gpu=" + self.FIELDS,
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
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.lines:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm)}


class NvmlClocks:
    """The SM clock and the active clock-event reasons of one GPU, read through NVML (the
    driver's libnvidia-ml) every `period` seconds by a host thread: dense enough to sample a
    timed region of a few milliseconds.  Only reads; nothing on the GPU changes."""

    REASONS = {0x4: "sw_power_cap", 0x8: "hw_slowdown", 0x40: "sw_thermal_slowdown",
               0x80: "hw_thermal_slowdown", 0x100: "hw_power_brake_slowdown"}
    NVML_CLOCK_SM = 1

    def __init__(self, uuid=None, index=0, period=0.0005):
        import ctypes
        self.period = period
        self.samples = []
        self.ok = False
        self.thread = None
        try:
            L = ctypes.CDLL("libnvidia-ml.so.1")
            if L.nvmlInit_v2() != 0:
                return
            h = ctypes.c_void_p()
            r = L.nvmlDeviceGetHandleByUUID(uuid.encode(), ctypes.byref(h)) if uuid else -1
            if r != 0:
                r = L.nvmlDeviceGetHandleByIndex_v2(ctypes.c_uint(index), ctypes.byref(h))
            if r != 0:
                return
            self.reasons_fn = getattr(L, "nvmlDeviceGetCurrentClocksEventReasons", None) or \
                L.nvmlDeviceGetCurrentClocksThrottleReasons
            mx = ctypes.c_uint(0)
            self.max_mhz = float(mx.value) if L.nvmlDeviceGetMaxClockInfo(h, self.NVML_CLOCK_SM, ctypes.byref(mx)) == 0 \
                and mx.value else None
            self.L, self.h = L, h
            self.ok = True
        except Exception:
            self.ok = False

    def _run(self):
        import ctypes
        c, r = ctypes.c_uint(0), ctypes.c_ulonglong(0)
        while not self._stop.is_set():
            t = time.perf_counter()
            if self.L.nvmlDeviceGetClockInfo(self.h, self.NVML_CLOCK_SM, ctypes.byref(c)) == 0 and \
                    self.reasons_fn(self.h, ctypes.byref(r)) == 0:
                self.samples.append((t, float(c.value), int(r.value)))
            time.sleep(self.period)

    def start(self):
        if self.ok:
            self._stop = threading.Event()
            self.thread = threading.Thread(target=self._run, daemon=True)
            self.thread.start()

    def stop(self):
        if self.thread is not None:
            self._stop.set()
            self.thread.join(timeout=5)
            self.thread = None

    def summary(self, t0=None, t1=None):
        """Median SM clock, max clock and the reasons seen in the samples taken between host
        times t0 and t1 (all samples when no window is given or none falls in it)."""
        return summarise_clock_samples(self.samples, getattr(self, "max_mhz", None), t0, t1, self.period)


def summarise_clock_samples(samples, max_mhz, t0=None, t1=None, period=0.0005):
    """samples: [(host time, SM MHz, NVML clock-event reason bits)]."""
    inside = [s for s in samples if t0 is not None and t0 <= s[0] <= t1]
    use = inside or samples
    if not use:
        return None
    reasons = set()
    for _, _, bits in use:
        for b, name in NvmlClocks.REASONS.items():
            if bits & b:
                reasons.add(name)
    return {"sm_mhz": statistics.median(s[1] for s in use), "sm_max_mhz": max_mhz, "reasons": sorted(reasons),
            "samples": len(use), "in_timed_region": bool(inside),
            "source": "NVML every %.1f ms" % (1e3 * period)}


def oracle_mlups(nx, ny, rows, steps, kw, cols=None):
    """Time the FP64 oracle on a periodic window of `cols` x `rows` cells of the lattice
    (cols = nx: a band of whole rows) for `steps` steps."""
    import numpy as np
    from oracle import rlbm_oracle as O
    cols = nx if cols is None else cols
    cfg = dict(nx=nx, ny=ny, **kw)
    o = O.Oracle(cfg, xs=np.arange(cols), ys=np.arange(rows))
    t0 = time.perf_counter()
    o.run(steps)
    dt = time.perf_counter() - t0
    return cols * rows * steps / dt / 1e6, dt


def _oracle_band_worker(a):
    """One host core: the oracle on a periodic window of cols x rows cells, `warm` untimed
    then `steps` timed steps; returns the timed seconds."""
    nx, ny, cols, rows, steps, kw, warm = a
    import numpy as np
    from oracle import rlbm_oracle as O
    o = O.Oracle(dict(nx=nx, ny=ny, **kw), xs=np.arange(cols), ys=np.arange(rows))
    o.run(warm)
    t0 = time.perf_counter()
    o.run(steps)
    return time.perf_counter() - t0


def oracle_mlups_all_cores(nx, ny, rows, steps, kw, warm=0, cols=None):
    """The oracle as it stands on every host core at once: one process per core (spawned,
    one BLAS thread each), each on its own window of cols x rows cells (cols = nx: a band
    of whole rows).  Returns (MLUPS over the slowest process's time, cores, seconds)."""
    import multiprocessing as mp
    cols = nx if cols is None else cols
    n = os.cpu_count() or 1
    for v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ[v] = "1"
    with mp.get_context("spawn").Pool(n) as pool:
        times = pool.map(_oracle_band_worker, [(nx, ny, cols, rows, steps, kw, warm)] * n)
    t = max(times)
    return n * cols * rows * steps / t / 1e6, n, t


REFERENCE_SECONDS = 120.0  # host time the reference arm aims at for its warm-up + timed steps


def reference_window(nx, ny, nsteps, kw, seconds=REFERENCE_SECONDS):
    """Window (cols, rows) of the lattice that one host core steps nsteps times in about
    `seconds`: whole rows (at least 8) while they fit, else a square periodic window, at
    least 8 x 8, the smallest lattice.  A step of the oracle has a fixed cost besides its
    per-cell cost, so the window is sized from probes of both."""
    _, t_band = oracle_mlups(nx, ny, 8, 1, kw)             # 8 whole rows, one step
    per_step = seconds / max(1, nsteps)
    if per_step >= t_band:
        return nx, int(min(ny, 8 * per_step / t_band))
    _, t_min = oracle_mlups(nx, ny, 8, 2, kw, cols=8)       # fixed cost: an 8 x 8 window
    t_min /= 2
    per_cell = max(1e-12, (t_band - t_min) / (8 * nx - 64))
    side = int((max(0.0, per_step - t_min) / per_cell + 64) ** 0.5)
    side = max(8, min(side, nx, ny))
    return side, side


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    kw = workload(args, 0)
    # each step a bounded sample: warm-up + timed steps take about two minutes on every core
    cols, rows = reference_window(args.nx, args.ny, args.steps + args.warmup, kw)
    value, cores, dt = oracle_mlups_all_cores(args.nx, args.ny, rows, args.steps, kw, warm=args.warmup, cols=cols)
    sample = ("%d host cores, each a %d x %d periodic window of the %dx%d lattice, %d steps after %d warm-up"
              % (cores, cols, rows, args.nx, args.ny, args.steps, args.warmup))
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "MLUPS", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt * 1e3 / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": workload_name(args), "lattice": [args.nx, args.ny], "sample_window": [cols, rows]},
            "cpu_baseline": {"value": value, "unit": "MLUPS", "cores": cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": "MLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def tune_flushed(lat, flush, torch, reps=12):
    """Pick the step kernel's launch shape (persistent CTAs x pipeline depth x stirring
    rows staged or from global memory) by timing `reps` steps of each with the L2 flushed
    before every step, as in the timed region.  Advances the lattice by 16 x (reps + 1)
    steps (part of the warm-up)."""
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    best = None
    for rows in (1, 2):
        for stages in (2, 1):
            for ctas in (0, 2 * sms, 3 * sms, 4 * sms):
                lat.set_launch(ctas, stages, rows)
                t = statistics.median(time_flushed(lat, flush, torch, reps))
                if best is None or t < best[0]:
                    best = (t, ctas, stages, rows)
    lat.set_launch(best[1], best[2], best[3])
    return {"ctas": best[1], "stages": best[2], "stir_rows": best[3], "ms": best[0]}


def time_flushed(lat, flush, torch, steps, warm=1):
    """Per-step times (ms) of `steps` single-step launches, each after an L2 flush (a write
    of a buffer larger than L2), CUDA events on the lattice's stream around the launch only."""
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    with torch.cuda.stream(lat.stream):
        for _ in range(warm):
            flush.zero_()
            lat.step(1)
        for a, b in ev:
            flush.zero_()
            a.record(lat.stream)
            lat.step(1)
            b.record(lat.stream)
    torch.cuda.synchronize()
    return [a.elapsed_time(b) for a, b in ev]


def time_chained(lat, torch, steps):
    """ms per step of one rlbm_step(steps) call (consecutive launches chained), CUDA events
    on the lattice's stream around the call."""
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with torch.cuda.stream(lat.stream):
        a.record(lat.stream)
        lat.step(steps)
        b.record(lat.stream)
    torch.cuda.synchronize()
    return a.elapsed_time(b) / steps


def roofline_entry(alg_bytes_per_cell, cells, ms, traffic=None):
    peak, kind = measured_peak()
    achieved = alg_bytes_per_cell * cells / (ms / 1e3) / 1e9
    return {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
            "traffic": traffic, "peak_kind": kind, "alg_bytes_per_cell": alg_bytes_per_cell}


def common_16bit(h):
    """h rounded (to nearest) until FP16, BF16 and FP32 all hold it exactly: a start that
    every storage type takes without rounding."""
    import numpy as np
    import torch
    x = torch.from_numpy(np.ascontiguousarray(h, dtype=np.float64))
    for _ in range(8):
        y = x.to(torch.float32).to(torch.bfloat16).to(torch.float32).to(torch.float16).to(torch.float64)
        if torch.equal(x, y):
            return x.numpy()
        x = y
    raise RuntimeError("no common 16-bit representation reached")


def slice_errors(rlbm, nx, ny, phys, fields, precisions, dev_steps=24, steps=200, stream=None):
    """Velocity error of each storage type on a 200-step slice against the FP64 path of the
    library (pinned to the FP64 oracle at 1e-10 by the parity tests): the FP64 path develops
    the seeded fields for dev_steps steps, the state is rounded to a common 16-bit start,
    and every type runs `steps` more steps from it.  Error = max |u - u_64| / max |u_64|
    (and eps relative per cell) over all cells."""
    import numpy as np
    ref = rlbm.Lattice(nx, ny, stream=stream, precision="f64", **phys, **fields)
    ref.step(dev_steps)
    h, step = ref.get_state()
    h = common_16bit(h)
    ref.set_state(h, step)
    ref.step(steps)
    Er, UXr, UYr, _ = ref.moments()
    ref.close()
    fluid = Er > 0.0
    umax = max(np.abs(UXr).max(), np.abs(UYr).max())
    out = {}
    for p in precisions:
        lat = rlbm.Lattice(nx, ny, stream=stream, precision=p, **phys)
        lat.set_state(h, step)
        lat.step(steps)
        E, UX, UY, _ = lat.moments()
        lat.close()
        out[p] = {"value": float(max(np.abs(UX - UXr).max(), np.abs(UY - UYr).max()) / umax), "unit": "max|u|",
                  "eps_rel": float(np.max(np.abs(E[fluid] - Er[fluid]) / Er[fluid])),
                  "vs": "FP64 library path (parity with the FP64 oracle 1e-10), %dx%d, %d-step slice from a common "
                        "16-bit start developed %d FP64 steps" % (nx, ny, steps, dev_steps),
                  "bar": 1e-5 if p == "f32" else 1e-3}
        out[p]["meets_bar"] = out[p]["value"] <= out[p]["bar"]
    return out


# --------------------------------------------------------------------------------------
# The forms: each returns a dict with its value, roofline and error
# --------------------------------------------------------------------------------------
def stirred_fields(nx, ny, seed):
    """Seeded smooth fields at the stirred workload's velocity scale (|u| up to 3e-3 on
    |k| <= 10): the start of its error slices."""
    from paper_2205_04658_gb300 import inputs
    e, ux, uy = inputs.smooth_random_fields(nx, ny, seed=seed, eps_amp=1e-3, u_amp=3e-3, kmax=10)
    return dict(init_eps=e, init_ux=ux, init_uy=uy)


def form_stirred_chained(args, torch, rlbm):
    """The stirred 1024^2 workload as it runs: blocks of 500 chained steps (one rlbm_step
    call each), an energy spectrum between blocks, outside the event windows.  The state
    (2 x 71 MB) is near L2's 129 MB, so consecutive steps reuse some of it from L2: the
    committed ncu summary of chained steps gives the DRAM bytes per step beside it."""
    nx = ny = 1024
    lat = rlbm.Lattice(nx, ny, precision="f32", **workload(args, 0))
    if args.shape:  # a fixed launch shape (profiling runs, where timing the candidates means nothing)
        lat.set_launch(*(int(v) for v in args.shape.split(",")))
    else:
        lat.autotune(20)
    lat.step(50)
    blocks = []
    for _ in range(4):
        blocks.append(time_chained(lat, torch, 500))
        lat.spectrum(512)
    lat.close()
    ms = statistics.median(blocks)
    return {"value": nx * ny / (ms / 1e3) / 1e6, "unit": "MLUPS", "ms_per_step": ms, "dtype": "f32",
            "workload": "stirred 1024x1024 FP32, 4 blocks of 500 chained steps (median block), spectrum between",
            "roofline": roofline_entry(ALG_BYTES["f32"], nx * ny, ms,
                                       traffic_from(CHAINED_TRAFFIC_FILE, "1024x1024 f32 chained")),
            "l2": "not flushed between chained steps (the workload's own pattern)"}


def form_stirred_4096(args, torch, rlbm):
    """The stirred workload on 4096^2 (2 x 1.1 GB, far above L2): 200 chained steps."""
    nx = ny = 4096
    lat = rlbm.Lattice(nx, ny, precision="f32", **workload(args, 0))
    lat.autotune(5)
    lat.step(10)
    ms = time_chained(lat, torch, 200)
    lat.close()
    return {"value": nx * ny / (ms / 1e3) / 1e6, "unit": "MLUPS", "ms_per_step": ms, "dtype": "f32",
            "workload": "stirred 4096x4096 FP32, 200 chained steps", "l2": "state 2.3 GB > L2, no flush",
            "roofline": roofline_entry(ALG_BYTES["f32"], nx * ny, ms)}


def graphene_setup(frac=0.15, gseed=315):
    from paper_2205_04658_gb300 import inputs
    nx, ny = 2048, 512
    mask, _ = inputs.disc_mask(nx, ny, radius=6, fraction=frac, seed=gseed, walls_y=True)
    phys = dict(walls_y=1, solid=mask, body_force=(1e-6, 0.0), eta_over_s=0.05)
    return nx, ny, mask, phys


def form_graphene(args, torch, rlbm, flush, prec, steps=40, frac=0.15, gseed=315):
    """The graphene-like sample (2048 x 512, walls, body force 1e-6, discs r = 6): single
    steps after an L2 flush (the FP16 state, 2 x 36 MB, fits in L2)."""
    import numpy as np
    nx, ny, mask, phys = graphene_setup(frac, gseed)
    lat = rlbm.Lattice(nx, ny, precision=prec, **phys)
    lat.autotune(10)
    times = time_flushed(lat, flush, torch, steps, warm=max(3, args.warmup))
    lat.close()
    ms = float(np.mean(times))
    cells = nx * ny
    alg = ALG_BYTES[prec] + 2  # populations + the 16-bit neighbour mask
    return {"value": cells / (ms / 1e3) / 1e6, "unit": "MLUPS", "ms_per_step": ms, "dtype": prec,
            "workload": "graphene-like 2048x512, walls, body force 1e-6, discs r=6 at %d %% (%d fluid cells), %s "
                        "storage, %d flushed single steps" % (round(100 * frac), int((mask == 0).sum()),
                                                              prec.upper(), steps),
            "l2": "flushed before every timed step (256 MiB write)", "roofline": roofline_entry(alg, cells, ms)}


def graphene_errors(rlbm, precisions):
    from paper_2205_04658_gb300 import inputs
    nx, ny, _, phys = graphene_setup()
    e, ux, uy = inputs.smooth_random_fields(nx, ny, seed=31, eps_amp=1e-4, u_amp=1e-4, kmax=6)
    ux = ux + 2e-3  # the plug flow the 50 000-step run reaches under its body force
    return slice_errors(rlbm, nx, ny, phys, dict(init_eps=e, init_ux=ux, init_uy=uy), precisions)


ENSEMBLE_KW = dict(eta_over_s=0.05, kmin=8, kmax=10, force_amp=1e-4)


def form_ensemble(args, torch, rlbm, prec, steps, members=64):
    """The 64-member ensemble (sides uniform over 256..1024 by seed 4, member seeds 1000 + m)
    advanced by one persistent launch per step, chunks of steps replayed from CUDA graphs.
    The state (> 2 GB) is far larger than L2, so no flush is needed between steps."""
    from paper_2205_04658_gb300 import inputs
    sides = inputs.ensemble_sides(members, 4)
    stream = torch.cuda.Stream()
    lats = [rlbm.Lattice(n, n, stream=stream, precision=prec, seed=1000 + m, **ENSEMBLE_KW) for m, n in enumerate(sides)]
    cells = sum(n * n for n in sides)
    batch = rlbm.Batch(lats, stream=stream)
    tuned_ms = batch.autotune(5)
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with torch.cuda.stream(stream):
        batch.step(max(args.warmup, 3))
        torch.cuda.synchronize()
        a.record(stream)
        batch.step(steps)
        b.record(stream)
    torch.cuda.synchronize()
    ms = a.elapsed_time(b) / steps
    for lat in lats:
        lat.sync()
    batch.close()
    for lat in lats:
        lat.close()
    mix = "/".join(str(sides.count(v)) + "x" + str(v) for v in (256, 512, 768, 1024))
    return {"value": cells / (ms / 1e3) / 1e6, "unit": "MLUPS", "ms_per_step": ms, "dtype": prec,
            "workload": "ensemble of %d stirred lattices (%s, %d cells), %s storage, one persistent launch per step, "
                        "CUDA-graph replay, %d steps" % (len(sides), mix, cells, prec.upper(), steps),
            "l2": "state %.1f GB > L2, no flush" % (cells * ALG_BYTES[prec] / 1e9), "autotuned_ms": tuned_ms,
            "roofline": roofline_entry(ALG_BYTES[prec], cells, ms), "cells": cells, "sides": sides}


def form_plain_members(args, torch, rlbm, sides, steps=50):
    """The plain FP32 form run member by member: each distinct side timed alone (chained
    steps), summed over the members."""
    stream = torch.cuda.Stream()
    per_side = {}
    for n in sorted(set(sides)):
        lat = rlbm.Lattice(n, n, stream=stream, precision="f32", seed=1000, **ENSEMBLE_KW)
        lat.autotune(10)
        lat.step(5)
        per_side[n] = time_chained(lat, torch, steps)
        lat.close()
    ms = sum(per_side[n] for n in sides)
    cells = sum(n * n for n in sides)
    return {"value": cells / (ms / 1e3) / 1e6, "unit": "MLUPS", "ms_per_step": ms, "dtype": "f32",
            "workload": "the same %d lattices, plain FP32 step kernel, one lattice at a time (%d chained steps per "
                        "side)" % (len(sides), steps),
            "roofline": roofline_entry(ALG_BYTES["f32"], cells, ms),
            "ms_per_side": {str(k): v for k, v in per_side.items()}}


def ensemble_errors(rlbm, precisions):
    """A 256^2 member of the ensemble's physics (seed 1000) from seeded fields at the stirred
    velocity scale."""
    phys = dict(ENSEMBLE_KW, seed=1000)
    return slice_errors(rlbm, 256, 256, phys, stirred_fields(256, 256, 1000), precisions)


def form_adjoint(args, torch, rlbm, nsteps=2000, reps=3):
    """Time per gradient of J = time-averaged mean |v|^2 / 2 of the 512^2 stirred run (shell
    4 <= |k| <= 6, 34 modes, amplitude 1e-4, seed 5, eta/s 0.05) with respect to the 34
    mode multipliers, eta/s and the body force: the forward (keeping every state and each
    step's Landau solution and force when they fit in a third of the free memory, else
    sqrt(N) checkpoints and a recomputation per segment) and the reverse sweep, all inside
    the timed call; compared with the forward alone."""
    import numpy as np
    nx = ny = 512
    kw = dict(eta_over_s=0.05, kmin=4, kmax=6, force_amp=1e-4, seed=5)
    stream = torch.cuda.Stream()
    lat = rlbm.Lattice(nx, ny, stream=stream, precision="f32", **kw)
    tuned_ms = lat.autotune(20)
    # every state kept when it fits in a third of the free memory (the forward runs once),
    # else checkpoints every ceil(sqrt(N)) steps and each segment recomputed
    segment = nsteps
    nbytes = rlbm.rlbm_gradient_query_workspace(lat.ctx, nsteps, segment)
    if nbytes > torch.cuda.mem_get_info()[0] // 3:
        segment = 0
        nbytes = rlbm.rlbm_gradient_query_workspace(lat.ctx, nsteps, segment)
    ws = torch.empty(nbytes + 256, dtype=torch.uint8, device="cuda")
    ptr = (ws.data_ptr() + 255) // 256 * 256
    with torch.cuda.stream(stream):
        rlbm.rlbm_gradient(lat.ctx, nsteps, segment, ptr, nbytes)  # warm-up
        times = []
        for _ in range(reps):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            J, gs, ge, gb = rlbm.rlbm_gradient(lat.ctx, nsteps, segment, ptr, nbytes)  # returns after a stream sync
            times.append(time.perf_counter() - t0)
    fwd = [time_chained(lat, torch, nsteps) * nsteps / 1e3 for _ in range(reps)]
    lat.close()
    del ws
    # accuracy (untimed): each timed call above continued the run, so the FP32 gradient of the
    # first nsteps steps is taken again on a fresh lattice and set against the FP64 adjoint of
    # the same steps (sqrt(N) checkpoints), which the tests hold to 1e-4 of central
    # differences on every component
    grads = {}
    for prec in ("f32", "f64"):
        fresh = rlbm.Lattice(nx, ny, stream=stream, precision=prec, **kw)
        with torch.cuda.stream(stream):
            grads[prec] = fresh.gradient(nsteps, 0)
        fresh.close()
    J, gs, ge, gb = grads["f32"]
    _, gs64, ge64, gb64 = grads["f64"]
    t, tf = statistics.median(times), statistics.median(fwd)
    return {"value": t, "unit": "s per gradient", "higher_is_better": False, "dtype": "f32",
            "workload": "gradient of the 512x512 stirred run (shell 4<=|k|<=6, 34 modes, amp 1e-4, seed 5, "
                        "eta/s 0.05), %d steps, wrt 34 mode multipliers, eta/s, body force" % nsteps,
            "checkpoint_segment": segment if segment else int(round(nsteps ** 0.5 + 0.4999)),
            "workspace_bytes": nbytes,
            "forward_only_s": tf, "gradient_over_forward": t / tf, "gradient_mlups": nx * ny * nsteps / t / 1e6,
            "J": J, "grad_eta_over_s": ge, "step_launch_tuned_ms": tuned_ms,
            "error": {"vs": "FP64 adjoint of the same run (itself within 1e-4 of central differences of the FP64 "
                            "forward on every component: tests/test_gpu_adjoint.py)",
                      "modes_max_over_largest": float(np.abs(gs - gs64).max() / np.abs(gs64).max()),
                      "eta_over_s": float(abs(ge - ge64) / abs(ge64)),
                      "body_force_x": float(abs(gb[0] - gb64[0]) / abs(gb64[0])),
                      "bars": {"modes_max_over_largest": 1e-4, "eta_over_s": 1e-4, "body_force_x": 2e-3}}}


def run_forms(args, torch, rlbm, flush):
    """Every form of the metric on this GPU (a few tens of seconds)."""
    forms = {}
    forms["c2_stirred1024_f32_chained"] = form_stirred_chained(args, torch, rlbm)
    forms["c2prime_stirred4096_f32"] = form_stirred_4096(args, torch, rlbm)
    errs = graphene_errors(rlbm, ["f32", "f16", "bf16"])
    for p in ("f16", "f32", "bf16"):
        forms["c3_graphene2048x512_%s" % p] = dict(form_graphene(args, torch, rlbm, flush, p), error=errs[p])
    # the config's other impurity fractions (geometry seeds 31, 35), timed in FP16 and FP32
    # (their errors are those of the same storage forms on the 15 % sample above)
    for frac, gseed in ((0.01, 31), (0.05, 35)):
        for p in ("f16", "f32"):
            forms["c3_graphene2048x512_%dpct_%s" % (round(100 * frac), p)] = form_graphene(
                args, torch, rlbm, flush, p, frac=frac, gseed=gseed)
    errs = ensemble_errors(rlbm, ["f32", "f16", "bf16"])
    plain = form_plain_members(args, torch, rlbm, form_sides())
    plain["error"] = errs["f32"]
    for p in ("f16", "bf16", "f32"):
        f = form_ensemble(args, torch, rlbm, p, 100)
        f.pop("sides")
        f["speedup_vs_plain_f32_member_by_member"] = plain["ms_per_step"] / f["ms_per_step"]
        f["error"] = errs[p]
        forms["c4_ensemble64_%s_batched" % p] = f
    forms["c4_ensemble64_f32_member_by_member"] = plain
    forms["c5_adjoint512_f32"] = form_adjoint(args, torch, rlbm)
    return forms


def form_sides():
    from paper_2205_04658_gb300 import inputs
    return inputs.ensemble_sides(64, 4)


def run_gb300(args):
    import numpy as np
    import torch
    import torch.distributed as dist
    from paper_2205_04658_gb300 import rlbm, inputs  # noqa: F401

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    else:
        torch.cuda.set_device(0)
    dev = torch.cuda.current_device()
    rlbm.lib()  # fails loudly when the library is missing
    uuid = getattr(torch.cuda.get_device_properties(dev), "uuid", None)
    uuid = "GPU-%s" % uuid if uuid is not None else None
    run_clocks = Clocks(uuid or dev)  # nvidia-smi every 200 ms over the whole run
    run_clocks.start()
    nvml = NvmlClocks(uuid=uuid, index=dev)  # dense samples around the timed region

    def barrier():
        if world > 1:
            dist.barrier()

    nx, ny, prec = args.nx, args.ny, args.precision
    cells = nx * ny
    kw = workload(args, rank)
    lat = rlbm.Lattice(nx, ny, precision=prec, **kw)
    stream = lat.stream
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    if args.shape:
        tuned_ms = None
        c_, s_, r_ = (int(v) for v in args.shape.split(","))
        lat.set_launch(c_, s_, r_)
        shape = {"ctas": c_, "stages": s_, "stir_rows": r_, "ms": None}
    else:
        tuned_ms = lat.autotune(20)  # launch shape (pipeline depth, CTA count); the state is not advanced
        shape = tune_flushed(lat, flush, torch)  # the same candidates, timed under the timed region's L2 flush
    nvml.start()
    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            flush.zero_()
            lat.step(1)
    torch.cuda.synchronize()
    barrier()
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    t_on = time.perf_counter()
    with torch.cuda.stream(stream):
        for a, b in ev:
            flush.zero_()
            a.record(stream)
            lat.step(1)
            b.record(stream)
    torch.cuda.synchronize()
    t_off = time.perf_counter()
    nvml.stop()
    barrier()
    torch.cuda.synchronize()
    lat.sync()
    clk = nvml.summary(t_on, t_off)
    times = [a.elapsed_time(b) for a, b in ev]
    total_ms = slowest(sum(times), world, "cuda")
    ms_per_step = total_ms / args.steps
    value = replica_mlups(world, cells, args.steps, total_ms / 1e3)
    peak, peak_kind = measured_peak()
    achieved = ALG_BYTES[prec] * cells / (statistics.mean(times) / 1e3) / 1e9
    traffic = committed_traffic(args)
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                "traffic": traffic, "peak_kind": peak_kind,
                "kernel": "step_kernel (fused stream+collide)", "alg_bytes_per_cell": ALG_BYTES[prec],
                "autotuned_ms": tuned_ms, "launch_shape": shape}
    lat.close()

    # end to end through the C ABI with host buffers, the workload's whole job: initial
    # fields H2D (rlbm_init), launch-shape tuning, 20 000 steps with the energy spectrum read
    # back to pinned host memory every 500 steps, then eps/u^x/u^y/totals D2H (rlbm_moments)
    e2e = None
    if not args.no_e2e:
        e, ux, uy = inputs.smooth_random_fields(nx, ny, seed=rank, eps_amp=0.0, u_amp=0.0)
        pin = [torch.empty((ny, nx), dtype=torch.float64).pin_memory() for _ in range(6)]
        pin[0].numpy()[:] = e
        pin[1].numpy()[:] = ux
        pin[2].numpy()[:] = uy
        tot = torch.empty(4, dtype=torch.float64).pin_memory()
        cfg, keep = rlbm.make_config(nx, ny, precision=prec, init_eps=pin[0].numpy(), init_ux=pin[1].numpy(),
                                     init_uy=pin[2].numpy(), **kw)
        # make_config copies non-contiguous input; these are contiguous, so it points at pinned memory
        nbytes = rlbm.rlbm_query_workspace(cfg)
        ws = torch.empty(nbytes + 256, dtype=torch.uint8, device="cuda")
        ptr = (ws.data_ptr() + 255) // 256 * 256
        job, every, nbins = E2E_JOB_STEPS, E2E_SPECTRUM_EVERY, min(nx, ny) // 2
        spec = torch.empty((job // every, nbins), dtype=torch.float64).pin_memory()
        torch.cuda.synchronize()
        barrier()
        t0 = time.perf_counter()
        ctx = rlbm.rlbm_init(cfg, ptr, nbytes, torch.cuda.current_stream().cuda_stream)
        rlbm.rlbm_autotune(ctx, 20)
        for i in range(job // every):
            rlbm.rlbm_step(ctx, every)
            rlbm.rlbm_spectrum(ctx, nbins, spec[i].numpy())
        rlbm.rlbm_moments(ctx, pin[3].numpy(), pin[4].numpy(), pin[5].numpy(), tot.numpy())
        t1 = time.perf_counter()
        rlbm.rlbm_free(ctx)
        dt = slowest(t1 - t0, world, "cuda")
        e2e = {"value": replica_mlups(world, cells, job, dt), "unit": "MLUPS",
               "h2d_bytes_per_step": 3 * 8 * cells / job,
               "d2h_bytes_per_step": (spec.numel() * 8 + 3 * 8 * cells + 32) / job,
               "job_steps": job, "seconds": dt,
               "note": "rlbm_init from pinned host fields + rlbm_autotune + %d steps with rlbm_spectrum (%d bins) "
                       "to pinned host every %d steps + rlbm_moments to pinned host" % (job, nbins, every)}
        del ws

    # the error of this form on a 200-step slice of the workload's own shape
    error = None
    forms = None
    if rank == 0 and world == 1 and not args.no_forms:
        error = slice_errors(rlbm, nx, ny, dict(kw), stirred_fields(nx, ny, 21), [prec])[prec] \
            if prec != "f64" else None
        forms = run_forms(args, torch, rlbm, flush)
    del flush

    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        rows, csteps = 512, 3  # about 10 s of oracle work per host core
        v1, dt1 = oracle_mlups(nx, ny, rows, csteps, kw)
        v, cores, dt = oracle_mlups_all_cores(nx, ny, rows, csteps, kw)
        cpu = {"value": v, "unit": "MLUPS", "cores": cores, "kind": "oracle",
               "sample": "FP64 oracle, %d steps of a %d x %d periodic band of the %dx%d workload per host core, "
                         "%d cores at once (%.1f s)" % (csteps, nx, rows, nx, ny, cores, dt),
               "single_core": {"value": v1, "cores": 1, "seconds": dt1}}

    if world > 1:
        dist.barrier()
    run_clk = run_clocks.stop()
    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": "MLUPS", "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": prec, "data": "synthetic",
                "config": {"workload": workload_name(args), "lattice": [nx, ny], "precision": prec,
                           "l2": "flushed before every timed step (256 MiB write)",
                           "parallelism": "replicas" if world > 1 else "single"},
                "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": args.steps,
                "clocks": clk if clk is not None else run_clk, "clocks_whole_run": run_clk,
                "error": error, "forms": forms}
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def standalone_line(f, args):
    """One JSON line of a single form (the --workload runs)."""
    line = {"metric": METRIC if f.get("unit") == "MLUPS" else "time per gradient (adjoint)",
            "value": f["value"], "unit": "MLUPS" if f.get("unit") == "MLUPS" else "s", "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": f.get("ms_per_step"),
            "higher_is_better": f.get("higher_is_better", True), "scaling": "weak", "vs_baseline": None,
            "dtype": f["dtype"], "data": "synthetic", "config": {"workload": f["workload"], "l2": f.get("l2")}}
    line.update({k: v for k, v in f.items() if k not in line and k not in ("workload", "l2")})
    return line


def run_ensemble(args):
    """The 64-member ensemble in the requested storage type against the plain FP32 form
    run member by member, with the velocity error of the storage type on a member slice."""
    import torch
    from paper_2205_04658_gb300 import rlbm
    torch.cuda.set_device(0)
    rlbm.lib()
    f = form_ensemble(args, torch, rlbm, args.precision, args.steps, args.members)
    plain = form_plain_members(args, torch, rlbm, f.pop("sides"))
    f["plain_f32_member_by_member"] = plain
    f["speedup_vs_plain_f32"] = plain["ms_per_step"] / f["ms_per_step"]
    if args.precision != "f64":
        f["error"] = ensemble_errors(rlbm, [args.precision])[args.precision]
    print(json.dumps(standalone_line(f, args)), flush=True)


def run_chained(args):
    import torch
    from paper_2205_04658_gb300 import rlbm
    torch.cuda.set_device(0)
    rlbm.lib()
    print(json.dumps(standalone_line(form_stirred_chained(args, torch, rlbm), args)), flush=True)


def run_adjoint(args):
    import torch
    from paper_2205_04658_gb300 import rlbm
    torch.cuda.set_device(0)
    rlbm.lib()
    f = form_adjoint(args, torch, rlbm, args.adjoint_steps, max(1, min(args.steps, 5)))
    print(json.dumps(standalone_line(f, args)), flush=True)


def run_graphene(args):
    """One line per area fraction (1 %, 5 %, 15 %; geometry seeds 31, 35, 315)."""
    import torch
    from paper_2205_04658_gb300 import rlbm
    torch.cuda.set_device(0)
    rlbm.lib()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    for frac, gseed in ((0.01, 31), (0.05, 35), (0.15, 315)):
        f = form_graphene(args, torch, rlbm, flush, args.precision, args.steps, frac, gseed)
        print(json.dumps(standalone_line(f, args)), flush=True)


def run_channel(args):
    """Part II's sample as an open channel: 1024 x 256 nodes, inflow u^x = 0.1 at x = 0,
    zero-gradient outflow, periodic sides, one or two impurities of 13 nodes (0.5 um at
    0.038 um per node), eta/s set for Re = 6.37 (one impurity; the two-impurity run keeps
    it).  Starts from the uniform inflow state.  The state (2 x 36 MB in FP32) fits in L2,
    so L2 is flushed (a 256 MiB write) before every timed step."""
    import numpy as np
    import torch
    from paper_2205_04658_gb300 import rlbm, inputs, units
    torch.cuda.set_device(0)
    rlbm.lib()
    w = inputs.CHANNEL_1024x256
    nx, ny = w["nx"], w["ny"]
    es = units.eta_over_s_for_reynolds(w["reynolds"], w["diameter_nodes"], w["inflow_ux"])
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    for count in (1, 2):
        mask = inputs.channel_impurities(nx, ny, w["diameter_nodes"], count=count)
        lat = rlbm.Lattice(nx, ny, precision=args.precision, open_x=1, inflow_ux=w["inflow_ux"], solid=mask,
                           eta_over_s=es, init_ux=np.full((ny, nx), w["inflow_ux"]))
        lat.autotune(10)
        times = time_flushed(lat, flush, torch, args.steps, warm=args.warmup)
        jx, _ = lat.column_means()
        lat.close()
        ms = float(np.mean(times))
        cells = nx * ny
        f = {"value": cells / (ms / 1e3) / 1e6, "unit": "MLUPS", "ms_per_step": ms, "dtype": args.precision,
             "workload": "open channel 1024x256 (Part II sample), inflow 0.1, %d impurit%s of 13 nodes, "
                         "eta/s %.4f (Re 6.37)" % (count, "y" if count == 1 else "ies", es),
             "l2": "flushed before every timed step (256 MiB write)",
             "roofline": roofline_entry(ALG_BYTES[args.precision] + 2, cells, ms), "j_outflow": float(jx[-1])}
        print(json.dumps(standalone_line(f, args)), flush=True)


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "chained":
        run_chained(args)
    elif args.workload == "ensemble64":
        run_ensemble(args)
    elif args.workload == "adjoint512":
        run_adjoint(args)
    elif args.workload == "graphene":
        run_graphene(args)
    elif args.workload == "channel":
        run_channel(args)
    else:
        run_gb300(args)


if __name__ == "__main__":
    main()
