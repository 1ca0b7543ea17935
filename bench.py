#!/usr/bin/env python
"""Throughput of the fused relativistic lattice Boltzmann step on GB300.

One step = one launch of the fused kernel (pull-streaming with bounce-back, moments,
Landau matching, equilibrium, Anderson-Witting relaxation, projected stirring force,
store) over the whole lattice, plus the stirring table the same launch prepares for
the next step.  Default workload: 1024 x 1024 periodic lattice, FP32, eps0 = 1 at
rest, stirring shell 8 <= |k| <= 10 with amplitude 1e-4 redrawn every step, eta/s =
0.05, dt = 0.05, a = 0.1.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

With N > 1 (torchrun), every rank advances its own independently seeded lattice
(replicas: the update has no cross-lattice exchange), and `value` counts the cell
updates of all ranks over the slowest rank's time.  L2 is flushed (a 256 MiB write)
before every timed step; only the step launches are inside the CUDA-event windows.
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
    p.add_argument("--shape", default=None,
                   help="ctas,stages,stir_rows: use this launch shape instead of tuning (profiling runs)")
    p.add_argument("--members", type=int, default=64,
                   help="ensemble64: number of members (64; fewer only for profiling runs)")
    p.add_argument("--adjoint-steps", type=int, default=2000,
                   help="adjoint512: steps of the differentiated run (2000; fewer only for profiling runs)")
    p.add_argument("--workload", default="stirred", choices=["stirred", "ensemble64", "adjoint512", "graphene", "channel"],
                   help="stirred: one lattice (default); ensemble64: 64 stirred members of uneven sizes "
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


def committed_traffic(args):
    """DRAM bytes per launch from the committed ncu summary, if it was taken on the
    current kernel source and this workload; else None."""
    try:
        kv = {}
        for line in open(TRAFFIC_FILE):
            if ":" in line and not line.startswith("#"):
                k, v = line.split(":", 1)
                kv[k.strip()] = v.strip()
        if kv.get("source_digest") != csrc_digest():
            return None
        if kv.get("workload") != "%dx%d %s" % (args.nx, args.ny, args.precision):
            return None
        return float(kv["dram_bytes_per_launch"])
    except Exception:
        return None


class Clocks:
    """nvidia-smi samples (200 ms) of the SM clock and throttle reasons while running."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device):
        self.device = device
        self.lines = []
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "--id=%d" % self.device, "--query-gpu=" + self.FIELDS,
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
                ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(reps)]
                with torch.cuda.stream(lat.stream):
                    flush.zero_()
                    lat.step(1)
                    for a, b in ev:
                        flush.zero_()
                        a.record(lat.stream)
                        lat.step(1)
                        b.record(lat.stream)
                torch.cuda.synchronize()
                t = statistics.median(a.elapsed_time(b) for a, b in ev)
                if best is None or t < best[0]:
                    best = (t, ctas, stages, rows)
    lat.set_launch(best[1], best[2], best[3])
    return {"ctas": best[1], "stages": best[2], "stir_rows": best[3], "ms": best[0]}


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
    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            flush.zero_()
            lat.step(1)
    torch.cuda.synchronize()
    barrier()
    torch.cuda.synchronize()
    clocks = Clocks(dev)
    clocks.start()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    with torch.cuda.stream(stream):
        for a, b in ev:
            flush.zero_()
            a.record(stream)
            lat.step(1)
            b.record(stream)
    torch.cuda.synchronize()
    barrier()
    torch.cuda.synchronize()
    clk = clocks.stop()
    lat.sync()
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
    del flush

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
    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": "MLUPS", "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": prec, "data": "synthetic",
                "config": {"workload": workload_name(args), "lattice": [nx, ny], "precision": prec,
                           "l2": "flushed before every timed step (256 MiB write)",
                           "parallelism": "replicas" if world > 1 else "single"},
                "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": args.steps,
                "clocks": clk}
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def run_ensemble(args):
    """64 stirred realisations, sides uniform over {256, 512, 768, 1024} (seed 4), member
    seeds 1000 + m, advanced together (one launch per step, CUDA-graph replay) in the
    requested storage type; compared with the plain FP32 form stepped member by member.
    The state (> 2 GB) is far larger than L2, so no flush is needed between steps."""
    import numpy as np
    import torch
    from paper_2205_04658_gb300 import rlbm, inputs
    torch.cuda.set_device(0)
    rlbm.lib()
    sides = inputs.ensemble_sides(args.members, 4)
    prec = args.precision
    kw = dict(eta_over_s=0.05, kmin=8, kmax=10, force_amp=1e-4)
    stream = torch.cuda.Stream()
    lats = [rlbm.Lattice(n, n, stream=stream, precision=prec, seed=1000 + m, **kw) for m, n in enumerate(sides)]
    cells = sum(n * n for n in sides)
    batch = rlbm.Batch(lats, stream=stream)
    tuned_ms = batch.autotune(5)  # launch shape of the batched kernel; the members are not advanced
    with torch.cuda.stream(stream):
        batch.step(args.warmup)
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        batch.step(args.steps)
        b.record(stream)
    torch.cuda.synchronize()
    ms = a.elapsed_time(b) / args.steps
    for lat in lats:
        lat.sync()
    batch.close()
    for lat in lats:
        lat.close()
    # plain FP32, one member at a time (one launch per member and step)
    per_side = {}
    for n in sorted(set(sides)):
        lat = rlbm.Lattice(n, n, stream=stream, precision="f32", seed=1000, **kw)
        lat.autotune(10)
        with torch.cuda.stream(stream):
            lat.step(5)
            torch.cuda.synchronize()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            lat.step(50)
            b.record(stream)
        torch.cuda.synchronize()
        per_side[n] = a.elapsed_time(b) / 50
        lat.close()
    ms_plain = sum(per_side[n] for n in sides)
    value = cells / (ms / 1e3) / 1e6
    # velocity error of the storage type: a 256^2 member developed for 400 steps in FP64,
    # then 200 more steps from that (representable) state in both types
    err = None
    if prec != "f64":
        ref = rlbm.Lattice(256, 256, stream=stream, precision="f64", seed=1000, **dict(kw, force_amp=2e-3, kmin=4, kmax=6))
        ref.step(400)
        h, step = ref.get_state()
        h = h.astype({"f32": np.float32, "f16": np.float16, "bf16": np.float32}[prec]).astype(np.float64)
        if prec == "bf16":
            h = (np.frombuffer(h.astype(np.float32).tobytes(), np.uint32) & 0xFFFF0000).view(np.float32).reshape(h.shape).astype(np.float64)
        ref.set_state(h, step)
        ref.step(200)
        r = ref.moments()
        ref.close()
        lat = rlbm.Lattice(256, 256, stream=stream, precision=prec, seed=1000, **dict(kw, force_amp=2e-3, kmin=4, kmax=6))
        lat.set_state(h, step)
        lat.step(200)
        g = lat.moments()
        lat.close()
        umax = max(np.abs(r[1]).max(), np.abs(r[2]).max())
        err = max(np.abs(g[1] - r[1]).max(), np.abs(g[2] - r[2]).max()) / umax
    line = {"metric": METRIC, "value": value, "unit": "MLUPS", "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": prec, "data": "synthetic",
            "config": {"workload": "ensemble of %d stirred lattices, sides %s (%d cells), %s storage, "
                                   "one persistent launch per step, CUDA-graph replay" % (
                                       len(sides),
                                       "/".join(str(sides.count(v)) + "x" + str(v) for v in (256, 512, 768, 1024)),
                                       cells, prec.upper()),
                       "l2": "state %.1f GB > L2, no flush" % (cells * ALG_BYTES[prec] / 1e9)},
            "roofline": {"bound": "hbm", "achieved": ALG_BYTES[prec] * cells / (ms / 1e3) / 1e9,
                         "peak": measured_peak()[0], "unit": "GB/s",
                         "frac": ALG_BYTES[prec] * cells / (ms / 1e3) / 1e9 / measured_peak()[0]},
            "plain_f32_member_by_member": {"value": cells / (ms_plain / 1e3) / 1e6, "unit": "MLUPS",
                                           "ms_per_step": ms_plain},
            "speedup_vs_plain_f32": ms_plain / ms, "autotuned_ms": tuned_ms,
            "velocity_error": {"value": err, "vs": "FP64 path, 256x256 developed stirred flow, 200 steps",
                               "measure": "max |u - u_ref| / max |u_ref|"}}
    print(json.dumps(line), flush=True)


def run_adjoint(args):
    """Time per gradient of J = time-averaged mean |v|^2 / 2 of the 512^2 stirred run
    (shell 4 <= |k| <= 6, 34 modes, amplitude 1e-4, seed 5, eta/s 0.05, 2000 steps) with
    respect to the 34 mode multipliers, eta/s and the body force: forward with sqrt(N)
    checkpoints, segment recomputation and the reverse sweep, all inside the timed call.
    Compared with the forward alone (2000 steps)."""
    import torch
    from paper_2205_04658_gb300 import rlbm
    torch.cuda.set_device(0)
    rlbm.lib()
    nx = ny = 512
    N = args.adjoint_steps
    prec = args.precision
    kw = dict(eta_over_s=0.05, kmin=4, kmax=6, force_amp=1e-4, seed=5)
    stream = torch.cuda.Stream()
    lat = rlbm.Lattice(nx, ny, stream=stream, precision=prec, **kw)
    # launch shape of the step kernel that the gradient's forward and recomputation use
    # (timed on the current state, which it does not advance)
    tuned_ms = lat.autotune(20)
    nbytes = rlbm.rlbm_gradient_query_workspace(lat.ctx, N, 0)
    ws = torch.empty(nbytes + 256, dtype=torch.uint8, device="cuda")
    ptr = (ws.data_ptr() + 255) // 256 * 256
    for _ in range(max(1, args.warmup // 10)):
        rlbm.rlbm_gradient(lat.ctx, N, 0, ptr, nbytes)
    reps = max(1, min(args.steps, 5))
    times = []
    for _ in range(reps):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        J, gs, ge, gb = rlbm.rlbm_gradient(lat.ctx, N, 0, ptr, nbytes)  # returns after a stream sync
        times.append(time.perf_counter() - t0)
    fwd = []
    for _ in range(reps):
        with torch.cuda.stream(stream):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            lat.step(N)
            b.record(stream)
        torch.cuda.synchronize()
        fwd.append(a.elapsed_time(b) / 1e3)
    lat.close()
    t = statistics.median(times)
    tf = statistics.median(fwd)
    line = {"metric": "time per gradient (adjoint, sqrt(N) checkpoints)", "value": t, "unit": "s",
            "n_gpus": 1, "steps": reps, "warmup": max(1, args.warmup // 10), "higher_is_better": False,
            "scaling": "weak", "vs_baseline": None, "dtype": prec, "data": "synthetic",
            "config": {"workload": "gradient of the 512x512 stirred run (shell 4<=|k|<=6, 34 modes, amp 1e-4, "
                                   "seed 5, eta/s 0.05), %d steps, wrt 34 mode multipliers, eta/s, body force" % N,
                       "checkpoint_segment": int(round(N ** 0.5 + 0.4999)), "workspace_bytes": nbytes,
                       "step_launch_tuned_ms": tuned_ms},
            "forward_only_s": tf, "gradient_over_forward": t / tf,
            "gradient_mlups": nx * ny * N / t / 1e6, "J": J, "grad_eta_over_s": ge}
    print(json.dumps(line), flush=True)


def run_graphene(args):
    """The graphene-like sample: 2048 x 512, x periodic, bounce-back walls in y, uniform
    body force 1e-6 along x, discs of radius 6 at 1 %, 5 % and 15 % area (geometry seeds
    31, 35, 315), eta/s 0.05, in the requested storage type (default FP16 with stochastic
    rounding).  One line per area fraction.  The two population buffers (2 x 71 MB in
    FP16) fit in L2, so L2 is flushed (a 256 MiB write) before every timed step."""
    import numpy as np
    import torch
    from paper_2205_04658_gb300 import rlbm, inputs
    torch.cuda.set_device(0)
    rlbm.lib()
    prec = args.precision
    nx, ny = 2048, 512
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    for frac, gseed in ((0.01, 31), (0.05, 35), (0.15, 315)):
        mask, _ = inputs.disc_mask(nx, ny, radius=6, fraction=frac, seed=gseed, walls_y=True)
        lat = rlbm.Lattice(nx, ny, precision=prec, walls_y=1, solid=mask, body_force=(1e-6, 0.0), eta_over_s=0.05)
        lat.autotune(10)
        stream = lat.stream
        with torch.cuda.stream(stream):
            for _ in range(args.warmup):
                flush.zero_()
                lat.step(1)
            ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
            for a, b in ev:
                flush.zero_()
                a.record(stream)
                lat.step(1)
                b.record(stream)
        torch.cuda.synchronize()
        lat.sync()
        times = [a.elapsed_time(b) for a, b in ev]
        lat.close()
        ms = float(np.mean(times))
        cells = nx * ny
        fluid = int((mask == 0).sum())
        alg = ALG_BYTES[prec] * cells + 2 * cells  # populations + the 16-bit neighbour mask
        line = {"metric": METRIC, "value": cells / (ms / 1e3) / 1e6, "unit": "MLUPS", "n_gpus": 1,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": prec, "data": "synthetic",
                "config": {"workload": "graphene-like 2048x512, walls in y, body force 1e-6, discs r=6 at %d %% "
                                       "(%d fluid cells), %s storage" % (round(100 * frac), fluid, prec.upper()),
                           "l2": "flushed before every timed step (256 MiB write)"},
                "roofline": {"bound": "hbm", "achieved": alg / (ms / 1e3) / 1e9, "peak": measured_peak()[0],
                             "unit": "GB/s", "frac": alg / (ms / 1e3) / 1e9 / measured_peak()[0],
                             "alg_bytes_per_cell": alg / cells}}
        print(json.dumps(line), flush=True)


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
        stream = lat.stream
        with torch.cuda.stream(stream):
            for _ in range(args.warmup):
                flush.zero_()
                lat.step(1)
            ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
            for a, b in ev:
                flush.zero_()
                a.record(stream)
                lat.step(1)
                b.record(stream)
        torch.cuda.synchronize()
        times = [a.elapsed_time(b) for a, b in ev]
        jx, _ = lat.column_means()
        lat.close()
        ms = float(np.mean(times))
        cells = nx * ny
        alg = ALG_BYTES[args.precision] * cells + 2 * cells
        line = {"metric": METRIC, "value": cells / (ms / 1e3) / 1e6, "unit": "MLUPS", "n_gpus": 1,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": args.precision, "data": "synthetic",
                "config": {"workload": "open channel 1024x256 (Part II sample), inflow 0.1, %d impurit%s of 13 nodes, "
                                       "eta/s %.4f (Re 6.37)" % (count, "y" if count == 1 else "ies", es),
                           "l2": "flushed before every timed step (256 MiB write)"},
                "roofline": {"bound": "hbm", "achieved": alg / (ms / 1e3) / 1e9, "peak": measured_peak()[0],
                             "unit": "GB/s", "frac": alg / (ms / 1e3) / 1e9 / measured_peak()[0]},
                "j_outflow": float(jx[-1])}
        print(json.dumps(line), flush=True)


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
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
