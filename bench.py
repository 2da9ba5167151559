"""Throughput of the fused two-colour D2Q9 chromodynamic MRT step on GB300.

Workload: 8192 x 8192 periodic lattice, 64 seeded drops (radii uniform in
[8, 64]), Lambda = 10, sigma = 0.005, beta = 0.67, nu = 1/6 (both fluids).
One step = one lattice update of every node (all rows of the hot path, one
fused kernel launch).  The state (2 x 4.8 GB of FP32 populations) is far
larger than L2, so no flush is needed between steps.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl cmrt|reference]

Under torchrun (N > 1) every rank runs an independent replica of the
workload on its own GPU (weak scaling, no collective on the data path); the
time is the maximum over ranks.  ``--impl reference`` times the FP64 CPU
oracle on the host cores instead, on a bounded crop of the same workload.
Rank 0 prints one JSON line.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

METRIC = "2-colour D2Q9 MRT MLUPS, % HBM roofline; low-prec/batched/adjoint vs plain FP32"
UNIT = "MLUPS"
BYTES_PER_CELL = 144  # 18 FP32 populations read + 18 written per node update
N_SIDE = 8192
NOMINAL_HBM_GBS = 7900.0  # GB300 HBM3e, nominal (the roofline uses the measured copy bandwidth)
WORKLOAD = "drops_8192x8192_periodic_64drops_Lambda10"
KERNEL_SOURCES = ["paper_2005_04642_gb300/csrc/cmrt_step.cu", "paper_2005_04642_gb300/csrc/cmrt_device.cuh",
                  "paper_2005_04642_gb300/csrc/cmrt_internal.h"]


def workload_config(side=N_SIDE):
    ndrops = max(1, round(64 * (side / N_SIDE) ** 2))
    name = WORKLOAD if side == N_SIDE else f"drops_{side}x{side}_periodic_{ndrops}drops_Lambda10"
    return {"workload": name, "nx": side, "ny": side, "ndrops": ndrops, "radii": [8, 64], "seed": 3,
            "Lambda": 10.0, "sigma": 0.005, "beta": 0.67, "nu": 1.0 / 6.0, "storage": "fp32",
            "l2": f"no flush: state {2 * 72 * side * side / 1e9:.2f} GB (two population buffers) >> 129 MB L2"}


def make_workload(side):
    from paper_2005_04642_gb300 import inputs as I
    if side == N_SIDE:
        return I.drops_8192()
    return I.random_drops(side, side, workload_config(side)["ndrops"], 8.0, 64.0, 3, Lambda=10.0)


def kernel_source_sha():
    h = hashlib.sha256()
    for rel in KERNEL_SOURCES:
        with open(os.path.join(ROOT, rel), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def measured_peak_hbm():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def recorded_traffic(cells):
    """DRAM bytes per launch of the step kernel from a committed ncu summary,
    scaled to `cells`, if the summary was taken on the current kernel source."""
    path = os.path.join(ROOT, "profiles", "step_kernel_traffic.json")
    try:
        with open(path) as fh:
            d = json.load(fh)
    except Exception:
        return None
    if d.get("source_sha") != kernel_source_sha():
        return None
    return float(d["dram_bytes_per_cell"]) * cells


# ---------------------------------------------------------------- clocks
class NvmlClockSampler:
    """SM clock and clock-event reasons of the GPU in use, read through NVML
    (read-only queries) every few milliseconds in a background thread during
    the timed region; the device is found by its PCI bus id, so that the
    sample is of the GPU the process runs on whatever the device numbering."""

    # clock-event reason bits of NVML's public API
    REASONS = {0x4: "sw_power_cap", 0x8: "hw_slowdown", 0x20: "sw_thermal_slowdown", 0x40: "hw_thermal_slowdown",
               0x80: "hw_power_brake_slowdown"}

    def __init__(self, cuda_index, period_s=0.005):
        self.cuda_index = cuda_index
        self.period = period_s
        self.samples = []
        self.max_mhz = None
        self.ok = False

    def __enter__(self):
        import ctypes
        import threading
        import torch
        try:
            self.nvml = ctypes.CDLL("libnvidia-ml.so.1")
            if self.nvml.nvmlInit_v2() != 0:
                return self
            props = torch.cuda.get_device_properties(self.cuda_index)
            bus = f"{props.pci_domain_id:08X}:{props.pci_bus_id:02X}:{props.pci_device_id:02X}.0".encode()
            self.dev = ctypes.c_void_p()
            if self.nvml.nvmlDeviceGetHandleByPciBusId_v2(bus, ctypes.byref(self.dev)) != 0:
                return self
            mx = ctypes.c_uint()
            if self.nvml.nvmlDeviceGetMaxClockInfo(self.dev, 1, ctypes.byref(mx)) == 0:  # 1: SM clock
                self.max_mhz = float(mx.value)
            self.reasons_fn = getattr(self.nvml, "nvmlDeviceGetCurrentClocksEventReasons", None) or \
                self.nvml.nvmlDeviceGetCurrentClocksThrottleReasons
            self.stop = threading.Event()
            self.thread = threading.Thread(target=self._run, daemon=True)
            self.ok = True
            self.thread.start()
        except Exception:
            self.ok = False
        return self

    def _run(self):
        import ctypes
        clk, rs = ctypes.c_uint(), ctypes.c_ulonglong()
        while not self.stop.is_set():
            if (self.nvml.nvmlDeviceGetClockInfo(self.dev, 1, ctypes.byref(clk)) == 0 and
                    self.reasons_fn(self.dev, ctypes.byref(rs)) == 0):
                self.samples.append((float(clk.value), int(rs.value)))
            time.sleep(self.period)

    def __exit__(self, *exc):
        if self.ok:
            self.stop.set()
            self.thread.join(timeout=2)

    def summary(self):
        if not self.ok or not self.samples:
            return None
        reasons = set()
        for _, r in self.samples:
            for bit, name in self.REASONS.items():
                if r & bit:
                    reasons.add(name)
        return {"sm_mhz": statistics.median(c for c, _ in self.samples), "sm_max_mhz": self.max_mhz,
                "reasons": sorted(reasons), "samples": len(self.samples), "source": "nvml"}


class Clocks:
    """NVML sampling where the library loads, else nvidia-smi."""

    def __init__(self, gpu_index):
        self.nvml = NvmlClockSampler(gpu_index)
        self.smi = ClockSampler(gpu_index)

    def __enter__(self):
        self.nvml.__enter__()
        if not self.nvml.ok:
            self.smi.__enter__()
        return self

    def __exit__(self, *exc):
        self.nvml.__exit__(*exc)
        if not self.nvml.ok:
            self.smi.__exit__(*exc)

    def summary(self):
        return self.nvml.summary() or self.smi.summary()


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def __enter__(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.fh, stderr=subprocess.DEVNULL)
            time.sleep(0.3)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.fh.close()

    def summary(self):
        if self.proc is None or not self.path:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        sms, maxs, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as fh:
            for line in fh:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    sms.append(float(parts[1]))
                    maxs.append(float(parts[2]))
                except ValueError:
                    continue
                for n, v in zip(names, parts[5:9]):
                    if v.lower() == "active":
                        reasons.add(n)
        os.unlink(self.path)
        if not sms:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": statistics.median(sms), "sm_max_mhz": max(maxs), "reasons": sorted(reasons),
                "samples": len(sms)}


# ---------------------------------------------------------------- oracle timing (CPU)
def oracle_rate(side, steps, warmup, procs=1):
    """MLUPS of the FP64 NumPy oracle on a side x side crop of the workload:
    `procs` child processes, each with BLAS pinned to one thread and its own
    replica of the crop, started together; the rate counts every replica's
    cell updates over the slowest one's time."""
    code = f"""
import json, sys, time
sys.path.insert(0, {ROOT!r})
import numpy as np
from oracle import cmrt_oracle as O
from paper_2005_04642_gb300 import inputs as I
d, rn, u = I.drops_8192()
s = {side}
d = dict(d, nx=s, ny=s)
p = O.Params(**d)
R, B = O.init_state(np.ascontiguousarray(rn[:s, :s]), u[0][:s, :s], u[1][:s, :s], p)
R, B = O.run(R, B, p, {warmup})
t0 = time.perf_counter()
R, B = O.run(R, B, p, {steps})
dt = time.perf_counter() - t0
print(json.dumps({{"mlups": s * s * {steps} / dt / 1e6, "seconds": dt}}))
"""
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")
    children = [subprocess.Popen([sys.executable, "-c", code], stdout=subprocess.PIPE, stderr=subprocess.PIPE,
                                 text=True, env=env) for _ in range(procs)]
    seconds = []
    for ch in children:
        out, err = ch.communicate(timeout=1800)
        if ch.returncode != 0:
            raise RuntimeError("oracle timing failed: " + err[-2000:])
        seconds.append(json.loads(out.strip().splitlines()[-1])["seconds"])
    slowest = max(seconds)
    return {"mlups": procs * side * side * steps / slowest / 1e6, "seconds": slowest, "procs": procs}


def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def cpu_model():
    try:
        r = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10)
        for line in r.stdout.splitlines():
            if line.strip().lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    try:
        with open("/proc/cpuinfo") as fh:
            for line in fh:
                if line.lower().startswith("model name"):
                    return line.split(":", 1)[1].strip()
    except Exception:
        pass
    import platform
    return platform.machine()


def oracle_baseline(side, steps, warmup):
    """The oracle on one core and as one replica per host core."""
    one = oracle_rate(side, steps, warmup, 1)
    n = host_cores()
    all_ = oracle_rate(side, steps, warmup, n) if n > 1 else one
    sample = (f"{side}x{side} crop of the {N_SIDE}^2 drops field, {warmup} untimed + {steps} timed FP64 NumPy "
              f"oracle steps, one replica per process")
    return {"value": all_["mlups"], "unit": UNIT, "cores": n, "kind": "oracle", "sample": sample,
            "seconds": all_["seconds"], "single_core": {"value": one["mlups"], "cores": 1, "seconds": one["seconds"]},
            "cpu_model": cpu_model()}


def crop_side(steps, warmup, budget_cell_updates=2.0e7):
    side = int((budget_cell_updates / max(1, steps + warmup)) ** 0.5)
    return max(64, min(1024, side - side % 8))


def run_reference(args, rank):
    if rank != 0:
        return
    side = crop_side(args.steps, args.warmup)
    cb = oracle_baseline(side, args.steps, args.warmup)
    line = {"impl": "reference", "metric": METRIC, "value": cb["value"], "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * cb["seconds"] / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic", "config": workload_config(),
            "cpu_baseline": cb,
            "e2e": {"value": cb["value"], "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------- ranks
def max_over_ranks(value, dist=None, device="cpu"):
    """The largest `value` over all ranks (the slowest rank's time): an
    all-reduce with MAX when a process group is up, else the value itself."""
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    if dist is not None:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_mlups(cells, steps, world, seconds):
    """Whole-job throughput: every rank steps its own replica of `cells`
    nodes `steps` times, all within `seconds` (the max over ranks)."""
    return world * cells * steps / seconds / 1e6


# ---------------------------------------------------------------- GPU arm
def run_cmrt(args, rank, world, local_rank):
    import torch

    from paper_2005_04642_gb300 import cmrt as cm
    from paper_2005_04642_gb300 import inputs as I

    torch.cuda.set_device(local_rank)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    d, rn, u = make_workload(args.side)
    cells = d["nx"] * d["ny"]
    rn32 = np.ascontiguousarray(rn, dtype=np.float32)
    u32 = np.ascontiguousarray(u, dtype=np.float32)
    stream = torch.cuda.current_stream()

    # ---- device-resident throughput
    lat = cm.Lattice(d, torch.from_numpy(rn32).cuda(), torch.from_numpy(u32).cuda(), stream=stream)
    lat.step(args.warmup)
    barrier()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    n_launch0 = lat.launches
    with Clocks(local_rank) as clk:
        barrier()
        ev0.record(stream)
        lat.step(args.steps)
        ev1.record(stream)
        barrier()
    launches = lat.launches - n_launch0
    ms = ev0.elapsed_time(ev1)
    diag = lat.diagnostics()
    lat.close()
    del lat
    torch.cuda.empty_cache()
    ms_max = max_over_ranks(ms, dist, "cuda")
    value = whole_job_mlups(cells, args.steps, world, ms_max * 1e-3)
    per_launch_s = (ms / args.steps) * 1e-3

    # ---- end to end through the C ABI with pinned host buffers
    h_rn = torch.from_numpy(rn32).pin_memory()
    h_u = torch.from_numpy(u32).pin_memory()
    h_out = [torch.empty((d["ny"], d["nx"]), dtype=torch.float32).pin_memory() for _ in range(5)]
    barrier()
    t0 = time.perf_counter()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
    th = [0.0] * 4
    ev[0].record(stream)
    pr = cm.make_params(d)
    ctx = cm.cmrt_init(pr, h_rn.data_ptr(), h_u.data_ptr(), stream.cuda_stream)
    ev[1].record(stream)
    th[1] = time.perf_counter()
    cm.cmrt_step(ctx, args.steps)
    ev[2].record(stream)
    th[2] = time.perf_counter()
    cm.cmrt_fields(ctx, *(o.data_ptr() for o in h_out))
    ev[3].record(stream)
    th[3] = time.perf_counter()
    barrier()
    e2e_s = time.perf_counter() - t0
    torch.cuda.synchronize()
    # where the end-to-end time went: device time between the calls' events,
    # and host time to each call's return (cmrt_init allocates the lattice)
    e2e_phases = {"init_device_ms": ev[0].elapsed_time(ev[1]), "steps_device_ms": ev[1].elapsed_time(ev[2]),
                  "fields_device_ms": ev[2].elapsed_time(ev[3]), "init_host_ms": (th[1] - t0) * 1e3,
                  "steps_enqueue_host_ms": (th[2] - th[1]) * 1e3, "fields_host_ms": (th[3] - th[2]) * 1e3,
                  "wall_ms": e2e_s * 1e3}
    cm.cmrt_destroy(ctx)
    e2e_value = whole_job_mlups(cells, args.steps, world, max_over_ranks(e2e_s, dist, "cuda"))
    h2d = (h_rn.numel() + h_u.numel()) * 4
    d2h = sum(o.numel() for o in h_out) * 4

    variants = run_variants(args, cm, I, stream, ms / args.steps) if (args.variants and rank == 0) else None

    if rank != 0:
        if dist is not None:
            dist.barrier()
            dist.destroy_process_group()
        return

    peak, peak_kind = measured_peak_hbm()
    achieved = BYTES_PER_CELL * cells / per_launch_s / 1e9
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                "peak_source": peak_kind, "nominal_peak": NOMINAL_HBM_GBS, "frac_of_nominal": achieved / NOMINAL_HBM_GBS,
                "traffic": recorded_traffic(cells),
                "algorithmic_bytes_per_launch": BYTES_PER_CELL * cells, "kernel": "k_chain<Step>",
                "source_sha": kernel_source_sha()}
    cpu = None
    if world == 1 and not args.no_cpu_baseline:
        cpu = oracle_baseline(crop_side(10, 2), 10, 2)
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": workload_config(args.side), "clocks": clk.summary(),
            "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d / args.steps,
                    "d2h_bytes_per_step": d2h / args.steps, "phases": e2e_phases,
                    "what": "cmrt_init from pinned host rho^N_0, u_0 + K steps + cmrt_fields into pinned host buffers"},
            "gpu_launches": launches, "roofline": roofline, "cpu_baseline": cpu, "variants": variants,
            "check": {"mass_r": diag["mass_r"], "mass_b": diag["mass_b"], "nonfinite": diag["nonfinite"]}}
    print(json.dumps(line), flush=True)
    if dist is not None:
        dist.barrier()
        dist.destroy_process_group()


def time_steps(cm, d, rn, u, steps, warmup, stream):
    """ms per step (CUDA events on the launching stream) of a device-resident lattice."""
    import torch
    lat = cm.Lattice(d, torch.from_numpy(np.ascontiguousarray(rn, dtype=np.float32)).cuda(),
                     torch.from_numpy(np.ascontiguousarray(u, dtype=np.float32)).cuda(), stream=stream)
    lat.step(warmup)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    lat.step(steps)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / steps
    diag = lat.diagnostics()
    lat.close()
    torch.cuda.empty_cache()
    return ms, diag


def run_variants(args, cm, I, stream, fp32_ms):
    """The reduced-precision storage forms on the same workload and on the
    16384 x 8192 buoyant-drops field (walls, gravity), each against FP32 there."""
    peak, _ = measured_peak_hbm()
    out = {}
    d, rn, u = make_workload(args.side)
    cells = d["nx"] * d["ny"]
    steps = max(20, args.steps // 4)
    for name, prec, nbytes in (("fp16", 2, 128), ("bf16", 1, 128)):
        ms, _ = time_steps(cm, dict(d, precision=prec), rn, u, steps, 5, stream)
        out[f"{name}_{WORKLOAD if args.side == N_SIDE else args.side}"] = {
            "value": cells / (ms * 1e-3) / 1e6, "unit": UNIT, "ms_per_step": ms, "speedup_vs_fp32": fp32_ms / ms,
            "bytes_per_cell": nbytes, "achieved_GBs": nbytes * cells / (ms * 1e-3) / 1e9,
            "frac_of_hbm_peak": nbytes * cells / (ms * 1e-3) / 1e9 / peak, "steps": steps}
    if args.side == N_SIDE:
        d, rn, u = I.buoyant_drops()
        cells = d["nx"] * d["ny"]
        base = None
        for name, prec, nbytes in (("fp32", 0, 144), ("fp16", 2, 128), ("bf16", 1, 128)):
            ms, diag = time_steps(cm, dict(d, precision=prec), rn, u, steps, 5, stream)
            base = base or ms
            out[f"{name}_buoyant_16384x8192_walls_256drops"] = {
                "value": cells / (ms * 1e-3) / 1e6, "unit": UNIT, "ms_per_step": ms, "speedup_vs_fp32": base / ms,
                "bytes_per_cell": nbytes, "achieved_GBs": nbytes * cells / (ms * 1e-3) / 1e9,
                "frac_of_hbm_peak": nbytes * cells / (ms * 1e-3) / 1e9 / peak, "steps": steps,
                "nonfinite": diag["nonfinite"]}
        out.update(run_layered(cm, I, stream, steps, fp32_ms, peak))
        out.update(run_batch(cm, I, stream, steps, fp32_ms, peak))
        out.update(run_adjoint(cm, I, stream))
    return out


def run_layered(cm, I, stream, steps, fp32_ms, peak):
    """Layered two-fluid flow (App. C): heavy fluid below a flat interface at
    mid-height, Lambda = 100, viscosity ratio 1, walls in y, body force 1e-6
    along x.  At 8192 x 8192 the step is bandwidth-bound like the drops
    workload; the 1024 x 128 channel of the parity tests fills a fifth of the
    GPU and shows the latency-bound small-lattice rate."""
    out = {}
    for name, nx, ny, nsteps in (("fp32_layered_8192x8192_walls_Lambda100", 8192, 8192, steps),
                                 ("fp32_layered_1024x128_walls_Lambda100", 1024, 128, 2000)):
        d, rn, u = I.layered_channel(nx=nx, ny=ny)
        ms, diag = time_steps(cm, d, rn, u, nsteps, 20, stream)
        cells = nx * ny
        gbs = 144 * cells / (ms * 1e-3) / 1e9
        out[name] = {"value": cells / (ms * 1e-3) / 1e6, "unit": UNIT, "ms_per_step": ms,
                     "vs_drops_8192_per_cell": (fp32_ms / (N_SIDE * N_SIDE)) / (ms / cells),
                     "bytes_per_cell": 144, "achieved_GBs": gbs, "frac_of_hbm_peak": gbs / peak, "steps": nsteps,
                     "nonfinite": diag["nonfinite"]}
    return out


def run_adjoint(cm, I, stream):
    """Cost of the discrete adjoint (cmrt_adjoint: forward with checkpoints,
    segment recomputation, reverse sweep) against plain forward steps: the
    256^2 drop of radius 32 (Lambda 10, gravity 1e-5 along -y) over 4000 steps
    with checkpoints every 200, and a 2048^2 lattice of the same drops field
    over 200 steps (checkpoints every 20) where launch latency no longer
    dominates; each also with every state kept (ckpt_every = 1: 19 GB and
    60 GB of HBM, no recomputation).  The objective's target is the final
    colour field of a run with sigma 5 % larger."""
    import torch
    res = {}
    for name, n, nsteps, K, drops in (("adjoint_256x256_drop_4000steps", 256, 4000, 200, 1),
                                      ("adjoint_256x256_drop_4000steps_every_state_kept", 256, 4000, 1, 1),
                                      ("adjoint_2048x2048_drops_200steps", 2048, 200, 20, 16),
                                      ("adjoint_2048x2048_drops_200steps_every_state_kept", 2048, 200, 1, 16)):
        if drops == 1:
            d = I.base_params(n, n, rho0_r=1.0, rho0_b=0.1, g_acc=(0.0, -1e-5))
            rn0 = I.drops_field(n, n, [(n / 2.0, n / 2.0)], [32.0], dtype=np.float32)
        else:
            d, rn0, _ = I.random_drops(n, n, drops, 8.0, 64.0, 3, Lambda=10.0, g_acc=(0.0, -1e-5))
            rn0 = rn0.astype(np.float32)
        rn_dev = torch.from_numpy(rn0).cuda()
        lt = cm.Lattice(dict(d, sigma=1.05 * d["sigma"]), rn_dev, None, stream=stream)
        lt.step(nsteps)
        f = lt.fields()
        a, b = f["rho_r"] / d["rho0_r"], f["rho_b"] / d["rho0_b"]
        target = ((a - b) / (a + b)).contiguous()
        lt.close()

        def timed(fn):
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            out = fn()
            e1.record(stream)
            torch.cuda.synchronize()
            return e0.elapsed_time(e1), out

        lat = cm.Lattice(d, rn_dev, None, stream=stream)
        lat.step(10)  # warm-up
        lat.close()
        lat = cm.Lattice(d, rn_dev, None, stream=stream)
        t_fwd, _ = timed(lambda: lat.step(nsteps))
        lat.close()
        lat = cm.Lattice(d, rn_dev, None, stream=stream)
        l0 = lat.launches
        t_adj, (J, g, _) = timed(lambda: lat.adjoint(nsteps, target, ckpt_every=K, want_rho_n0=True))
        launches = lat.launches - l0
        dev_bytes = cm.cmrt_device_bytes(lat.ctx)
        lat.close()
        torch.cuda.empty_cache()
        # one reverse step against one forward step: the call minus its forward
        # run and its segment replay (nsteps - ceil(nsteps / K) recomputed steps,
        # the same kernel as the forward steps), per step
        replayed = nsteps - (nsteps + K - 1) // K
        f = t_fwd / nsteps
        reverse_step = (t_adj - f * (nsteps + replayed)) / nsteps
        res[name] = {"forward_ms_per_step": f, "adjoint_ms_per_step": t_adj / nsteps,
                     "adjoint_vs_forward": t_adj / t_fwd, "reverse_vs_forward": (t_adj - t_fwd) / t_fwd,
                     "reverse_step_vs_forward_step": reverse_step / f, "replayed_steps": replayed,
                     "launches_per_step": launches / nsteps, "ckpt_every": K, "steps": nsteps,
                     "device_bytes": dev_bytes, "J": J, "dJ_dsigma": g["sigma"]}
    return res


def run_batch(cm, I, stream, steps, fp32_ms, peak):
    """The 512-lattice ensemble (sides 64..512, one drop each, sigma and
    Lambda per member) in one persistent launch per step, replayed from CUDA
    graphs: untuned rows (min(64, ny) per size class) against the autotuned
    ones, each against the plain FP32 step of the 8192^2 lattice per cell."""
    import torch
    members = I.batch_ensemble(512, seed=5)
    cells = sum(m[0]["nx"] * m[0]["ny"] for m in members)
    b = cm.Batch(members, stream=stream)
    graph = 32
    steps = max(graph, (steps + graph - 1) // graph * graph)

    def timed():
        b.step(2 * graph)  # warm-up; records the graph of each parity
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        launches0 = b.launches
        b.step(steps)
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / steps, b.launches - launches0

    ms_untuned, _ = timed()
    tuned_us = b.tune()
    ms, launches = timed()
    diag = b.diagnostics()
    sides = sorted({m[0]["nx"] for m in members})
    single = N_SIDE * N_SIDE / (fp32_ms * 1e-3) / 1e6
    value = cells / (ms * 1e-3) / 1e6
    res = {"batch_512_lattices_sides64-512_fp32": {
        "value": value, "unit": UNIT, "ms_per_step": ms, "members": len(members), "cells": cells,
        "work_items_per_step": b.work_items, "launches_per_step": launches / steps, "graph_steps": graph,
        "rows_per_class": {f"{s}x{s}": b.get_rows(s, s, 0) for s in sides},
        "untuned_ms_per_step": ms_untuned, "tuner_speedup": ms_untuned / ms, "tuner_us_per_step": tuned_us,
        "vs_fp32_single_lattice": value / single, "bytes_per_cell": 144,
        "achieved_GBs": 144 * cells / (ms * 1e-3) / 1e9, "frac_of_hbm_peak": 144 * cells / (ms * 1e-3) / 1e9 / peak,
        "steps": steps, "nonfinite": float(diag[:, 5].sum())}}
    b.close()
    torch.cuda.empty_cache()
    return res


def run_adjoint_only(args):
    """Only the discrete adjoint (cmrt_adjoint) on the drops field of
    args.side (16 drops per 2048^2, gravity 1e-5 along -y): args.steps steps
    with checkpoints every args.ckpt_every, against as many forward steps.
    A short run for kernel launch lists of the reverse passes."""
    import torch

    from paper_2005_04642_gb300 import cmrt as cm
    from paper_2005_04642_gb300 import inputs as I
    n, T, K = args.side, args.steps, args.ckpt_every
    ndrops = max(1, round(16 * (n / 2048.0) ** 2))
    d, rn0, _ = I.random_drops(n, n, ndrops, 8.0, 64.0, 3, Lambda=10.0, g_acc=(0.0, -1e-5))
    rn = torch.from_numpy(rn0.astype(np.float32)).cuda()
    stream = torch.cuda.current_stream()
    lt = cm.Lattice(dict(d, sigma=1.05 * d["sigma"]), rn, None, stream=stream)
    lt.step(T)
    f = lt.fields()
    a, b = f["rho_r"] / d["rho0_r"], f["rho_b"] / d["rho0_b"]
    target = ((a - b) / (a + b)).contiguous()
    lt.close()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    lat = cm.Lattice(d, rn, None, stream=stream)
    torch.cuda.synchronize()
    e0.record(stream)
    lat.step(T)
    e1.record(stream)
    torch.cuda.synchronize()
    fwd = e0.elapsed_time(e1) / T
    lat.close()
    lat = cm.Lattice(d, rn, None, stream=stream)
    torch.cuda.synchronize()
    e0.record(stream)
    J, g, _ = lat.adjoint(T, target, ckpt_every=K)
    e1.record(stream)
    torch.cuda.synchronize()
    adj = e0.elapsed_time(e1) / T
    lat.close()
    print(json.dumps({"adjoint_only": True, "side": n, "drops": ndrops, "steps": T, "ckpt_every": K,
                      "forward_ms_per_step": fwd, "adjoint_ms_per_step": adj, "adjoint_vs_forward": adj / fwd,
                      "J": J}), flush=True)


def run_profile_step(args):
    """Only the device-resident steps of the drops field of --side in storage
    form --precision (init, --warmup steps, --steps steps): a short command
    for ncu captures of the step kernel.  Prints one JSON line."""
    import torch
    from paper_2005_04642_gb300 import cmrt as cm
    cm.load()
    d, rn, u = make_workload(args.side)
    d = dict(d, precision=args.precision)
    stream = torch.cuda.current_stream()
    ms, diag = time_steps(cm, d, rn, u, args.steps, args.warmup, stream)
    cells = d["nx"] * d["ny"]
    nbytes = 144 if args.precision == 0 else 128
    print(json.dumps({"side": args.side, "precision": args.precision, "ms_per_step": ms,
                      "MLUPS": cells / (ms * 1e-3) / 1e6, "GBs": nbytes * cells / (ms * 1e-3) / 1e9,
                      "nonfinite": diag["nonfinite"]}), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", default="cmrt", choices=["cmrt", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-variants", dest="variants", action="store_false",
                    help="skip the reduced-precision timings reported under 'variants'")
    ap.add_argument("--side", type=int, default=N_SIDE,
                    help="lattice side; smaller sides (same drop density) are for profiling captures")
    ap.add_argument("--adjoint-only", action="store_true",
                    help="time only cmrt_adjoint on the drops field of --side (--steps steps, checkpoints every "
                         "--ckpt-every); a short run for launch lists of the reverse passes")
    ap.add_argument("--ckpt-every", type=int, default=10)
    ap.add_argument("--profile-step", action="store_true",
                    help="time only the steps of the drops field of --side in storage form --precision "
                         "(a short run for ncu captures of the step kernel)")
    ap.add_argument("--precision", type=int, default=0, choices=[0, 1, 2],
                    help="storage form for --profile-step: 0 FP32, 1 BF16, 2 FP16")
    args = ap.parse_args()
    if args.adjoint_only:
        run_adjoint_only(args)
        return
    if args.profile_step:
        args.warmup = max(args.warmup, 3)
        run_profile_step(args)
        return
    args.warmup = max(args.warmup, 3)
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank)
    else:
        run_cmrt(args, rank, world, local_rank)


if __name__ == "__main__":
    main()
