#!/usr/bin/env python
"""Benchmark of the B300 LDG hot path.

Default workload (`--workload jv`): the exact Jacobian-vector product of 3-D steady
convection-diffusion div(beta u - kappa grad u) = f on [0,1]^3 with 48^3 affine
hexahedra, p = 4 (Gauss-Lobatto nodes, 5^3 Gauss points), beta = (1, 0.5, 0.25),
kappa = 1e-2, manufactured u = exp(x+y+z) sin(pi xyz): 13,824,000 DOF. One *step*
is one FP64 J.v application on the full state (the q-stage of Eq. 1a on the
direction, then the residual stage of Eq. 1b), with v drawn N(0, 1). The inputs
and scratch of one J.v (v 110.6 MB, q(v) 331.8 MB, J.v 110.6 MB) exceed the 126 MB
L2, so no flush is needed between steps.

Metric: J.v GDOF/s = DOF x steps / time of the K timed steps (CUDA events on the
launching stream), with the %HBM roofline of the algorithmic bytes per DOF and the
FP64-ALU fraction. The same line reports the FP32-arithmetic J.v (with its error
against the FP64 oracle on sampled elements), the J.v end to end through the
host-buffer C-ABI call, the Newton-GMRES time to 1e-8 of the 2-D vortex BDF2 step
(FP32 Krylov + block-Jacobi against plain FP64 block-Jacobi, and through the
host-buffer solve call), and the FP64 oracle timed on the host cores.

Other workloads: vortex (the 64x64 p=3 Euler BDF2 step), batch (256 parametrised
solves in one graph launch), hex (the 48^3 J.v sweep p = 1..6), tri, tet (Table 3's
problem), cylinder (Navier-Stokes past a cylinder, learned + mixed against plain
FP64 block-Jacobi).

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
With N > 1 (torchrun), every rank runs its own instance (weak scaling, no collective
on the data path); rank 0 prints one JSON line.
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

METRIC = "J·v GDOF/s (%HBM roofline); Newton-GMRES time-to-1e-8, learned+mixed vs plain FP64"
UNIT = "GDOF/s"
WORKLOAD = ("2D compressible Euler isentropic vortex (gamma 1.4, strength 5, centre (5,5)), periodic "
            "[0,10]^2, 64x64 quads, p=3, Lax-Friedrichs flux, BDF2 dt=0.05, matrix-free Newton-GMRES(30) "
            "to 1e-8 (FP64 residual)")
N_SIDE, P, DT = 64, 3, 0.05
LAGGED_PC_REUSE = 4    # implicit steps per block-Jacobi build in the lagged form
# FLOPs per element of one J.v launch (dual-number Euler kernel, p = 3, 5 x 5 Gauss points),
# counted by ncu as 2*FMA + ADD + MUL thread instructions: FP64 instance (index 0) and
# FP32 instance (index 1).
JV_FLOP_PER_ELEM = (18449.0, 17027.0)
# ALU peaks derived from the unit counts and the maximum SM clock (2.032 GHz):
# FP64 148 SMs x 2 FMA/clk x 2 FLOP; FP32 148 SMs x 128 FMA/clk x 2 FLOP.
FP64_PEAK_TFLOPS = 148 * 2 * 2 * 2.032e9 / 1e12
FP32_PEAK_TFLOPS = 148 * 128 * 2 * 2.032e9 / 1e12
# Per-DOF FP64 FLOPs and DRAM bytes of one J.v of the default workload, by kernel
# variant (ncu thread-instruction counts and dram__bytes_read.sum + dram__bytes_write.sum
# of one capture); a variant not listed reports the HBM roofline only.
JV_FLOP_PER_DOF = {
    # 820 + 1655 MFLOP per J.v of 13,824,000 DOF (k_lin_q, k_lin_r; general affine elements)
    "k_lin_q + k_lin_r [hex p=4 nq=5 convdiff fp64, q scratch fp64]": 179.07,
    # 266 + 1472 MFLOP (the trace form for axis-aligned boxes, the 48^3 box mesh)
    "k_lin_qt + k_lin_rt [hex p=4 nq=5 convdiff fp64 cartesian, q scratch fp64]": 125.72,
}
JV_TRAFFIC_PER_DOF = {
    # (154.6 + 274.9) + (486.4 + 99.7) MB of DRAM reads + writes per J.v (k_lin_q, k_lin_r)
    "k_lin_q + k_lin_r [hex p=4 nq=5 convdiff fp64, q scratch fp64]": 73.47,
    # (135.2 + 96.1) + (287.4 + 92.3) MB
    "k_lin_qt + k_lin_rt [hex p=4 nq=5 convdiff fp64 cartesian, q scratch fp64]": 44.20,
}


# Default workload: the FP64 J.v of 3-D convection-diffusion on 48^3 hexahedra, p = 4.
JV_N, JV_P = 48, 4
JV_MU = (1e-2, 1.0, 1.0, 0.5, 0.25)          # kappa, tau, beta
JV_WORKLOAD = ("3D steady convection-diffusion div(beta u - kappa grad u) = f on [0,1]^3, 48^3 hexahedra, p=4 "
               "(GLL nodes, 5^3 Gauss points), beta=(1,0.5,0.25), kappa=1e-2, tau=1, u=exp(x+y+z) sin(pi xyz); "
               "one exact J.v application on the full 13,824,000-DOF state per step")
# Algorithmic HBM bytes per DOF of one linear 3-D J.v with FP64 storage: v read, q(v)
# written and read (3 components), J.v written: (1 + 2 x 3 + 1) x 8.
JV_BYTES_PER_DOF = 64.0


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


class ClockSampler:
    """SM clock and clock-event (throttle) reasons during the timed region: read through
    NVML every 5 ms in a thread (a timed region can be a few tens of milliseconds), or from
    `nvidia-smi -lms 200` when NVML cannot be loaded."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
    NAMES = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")

    def __init__(self, index: int, period_s: float = 0.005):
        # NVML numbers the GPUs of the machine; CUDA_VISIBLE_DEVICES may renumber them
        vis = os.environ.get("CUDA_VISIBLE_DEVICES", "")
        ids = [x.strip() for x in vis.split(",") if x.strip()]
        self.index = int(ids[index]) if index < len(ids) and ids[index].isdigit() else index
        self.period = period_s
        self.proc = None
        self.lines = []
        self.samples = []
        self.thread = None
        self.halt = threading.Event()
        self.nvml = None
        self.nvml_error = None

    # NVML's clock-event reason bits (nvml.h) and its SM clock domain
    BITS = (0x8, 0x40, 0x20, 0x4)   # hw_slowdown, hw_thermal_slowdown, sw_thermal_slowdown, sw_power_cap
    CLOCK_SM = 1

    def _open_nvml(self):
        import ctypes
        lib = ctypes.CDLL("libnvidia-ml.so.1")
        if lib.nvmlInit_v2() != 0:
            raise OSError("nvmlInit_v2 failed")
        h = ctypes.c_void_p()
        if lib.nvmlDeviceGetHandleByIndex_v2(ctypes.c_uint(self.index), ctypes.byref(h)) != 0 and \
                lib.nvmlDeviceGetHandleByIndex_v2(ctypes.c_uint(0), ctypes.byref(h)) != 0:
            raise OSError("nvmlDeviceGetHandleByIndex_v2 failed")
        reasons = getattr(lib, "nvmlDeviceGetCurrentClocksEventReasons", None) or \
            lib.nvmlDeviceGetCurrentClocksThrottleReasons
        return lib, h, reasons

    def start(self):
        try:
            self.nvml = self._open_nvml()
        except Exception as exc:
            self.nvml = None
            self.nvml_error = repr(exc)[:200]
        if self.nvml is not None:
            self.thread = threading.Thread(target=self._poll, daemon=True)
            self.thread.start()
            while not self.samples and self.thread.is_alive():
                time.sleep(0.001)
            return
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _poll(self):
        import ctypes
        lib, h, get_reasons = self.nvml
        sm, smax, r = ctypes.c_uint(), ctypes.c_uint(), ctypes.c_ulonglong()
        while not self.halt.is_set():
            if (lib.nvmlDeviceGetClockInfo(h, self.CLOCK_SM, ctypes.byref(sm)) != 0 or
                    lib.nvmlDeviceGetMaxClockInfo(h, self.CLOCK_SM, ctypes.byref(smax)) != 0 or
                    get_reasons(h, ctypes.byref(r)) != 0):
                self.nvml_error = "an NVML query failed"
                return
            self.samples.append((float(sm.value), float(smax.value),
                                 [nm for nm, b in zip(self.NAMES, self.BITS) if r.value & b]))
            self.halt.wait(self.period)

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.nvml is not None:
            self.halt.set()
            self.thread.join(timeout=5)
            # the first sample is taken before the work starts: keep the ones under load
            loaded = self.samples[1:] or self.samples
            sm = [x[0] for x in loaded]
            smax = [x[1] for x in loaded]
            reasons = {nm for x in loaded for nm in x[2]}
            try:
                self.nvml[0].nvmlShutdown()
            except Exception:
                pass
            out = {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                   "reasons": sorted(reasons), "samples": len(sm), "source": "NVML, every 5 ms"}
            if self.nvml_error:
                out["nvml_error"] = self.nvml_error
            return out
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
            except ValueError:
                continue
            for nm, val in zip(self.NAMES, parts[4:8]):
                if val.lower().startswith("active"):
                    reasons.add(nm)
        out = {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
               "reasons": sorted(reasons), "samples": len(sm), "source": "nvidia-smi, every 200 ms"}
        if self.nvml_error:
            out["nvml_error"] = self.nvml_error
        return out


def aggregate(local_times_ms, local_jv_dofs, world, rank):
    """Whole-job numbers: work summed over ranks, time = max over ranks (weak scaling)."""
    import torch
    import torch.distributed as dist
    t = torch.tensor([sum(local_times_ms)], dtype=torch.float64)
    w = torch.tensor([float(local_jv_dofs)], dtype=torch.float64)
    if world > 1:
        if dist.get_backend() == "nccl":
            t, w = t.cuda(), w.cuda()
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        dist.all_reduce(w, op=dist.ReduceOp.SUM)
    total_ms = float(t.item())
    gdofs = float(w.item()) / (total_ms * 1e-3) / 1e9
    return total_ms, gdofs


def cpu_baseline_jv(u0, v, seconds=12.0):
    """The FP64 oracle's J.v on the same workload, single-threaded, on the host cores."""
    import oracle
    from paper_2205_07824_b300 import synth
    mesh = synth.quad_box(N_SIDE, hi=(10.0, 10.0), periodic=(True, True))
    o = oracle.Oracle(mesh, P, oracle.EULER, oracle.CASE_VORTEX, (1.4,))
    un, unm1 = o.interpolate(0.0), o.interpolate(-DT)
    o.set_time(2, DT, DT, un, unm1)
    calls, t0 = 0, time.perf_counter()
    while True:
        o.jvp(u0, v)
        calls += 1
        el = time.perf_counter() - t0
        if el > seconds or calls >= 40:
            break
    return {"value": o.ndof * calls / el / 1e9, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"{calls} oracle J.v applications on the full 64x64 p=3 vortex state (BDF2 term on), "
                      f"{el:.1f} s single-threaded"}


def run_reference(args):
    """The oracle, as it stands, timed on the host cores on the default workload (the J.v of
    48^3 hexahedra, p = 4): each step is the FP64 oracle's J.v on a bounded sample of that
    workload, every 1103rd element (offset by the step) with the q-neighbourhood it needs;
    value = DOF of the sampled elements / time."""
    import numpy as np
    import oracle
    from paper_2205_07824_b300 import synth
    ws, rank, _ = _dist()
    if rank != 0:
        return
    mesh = synth.hex_box(JV_N)
    o = oracle.Oracle(mesh, JV_P, oracle.CONVDIFF, oracle.CASE_EXPSIN, JV_MU)
    u = synth.random_vector(o.ndof, 0)
    v = synth.random_vector(o.ndof, 1)
    stride = 1103
    for w in range(args.warmup):
        o.jvp_some(u, v, np.arange(w % stride, mesh.n_elem, stride, dtype=np.int64))
    times, dofs = [], 0
    for k in range(args.steps):
        el = np.arange((args.warmup + k) % stride, mesh.n_elem, stride, dtype=np.int64)
        t0 = time.perf_counter()
        o.jvp_some(u, v, el)
        times.append(time.perf_counter() - t0)
        dofs += len(el) * o.npe
    tot = sum(times)
    val = dofs / tot / 1e9
    ms = tot / args.steps * 1e3
    sample = (f"each step: the FP64 oracle's J.v on one element in {stride} of the {mesh.n_elem} (about "
              f"{dofs // max(args.steps, 1) // o.npe} elements, offset by the step, each with the q-stage of its face "
              f"neighbours), single-threaded; value = DOF of the sampled elements / time")
    line = {"metric": METRIC, "value": val, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
            "config": {"workload": JV_WORKLOAD, "n_dof": int(o.ndof), "sample": sample},
            "cpu_baseline": {"value": val, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample},
            "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def graph_time_ms(g, fn, reps):
    """Device time of one call of fn (launches on context g, no allocation): `reps` calls
    captured back to back in a CUDA graph, one replay timed with CUDA events, so that
    the host's per-call overhead does not hide the kernels' own duration."""
    import torch
    reps = max(int(reps), 20)     # one replay of a short graph carries launch overhead
    old = g.stream
    s = torch.cuda.Stream()
    g.set_stream(s)
    try:
        with torch.cuda.stream(s):
            for _ in range(3):
                fn()
        torch.cuda.synchronize()
        cg = torch.cuda.CUDAGraph()
        with torch.cuda.graph(cg, stream=s):
            for _ in range(reps):
                fn()
        for _ in range(2):
            cg.replay()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        cur = torch.cuda.current_stream()
        e0.record(cur)
        cg.replay()
        e1.record(cur)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps
    finally:
        g.set_stream(old)


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def jv_oracle_sample(mesh, u_h, v_h, stride, seconds=None):
    """The FP64 oracle's J.v on every `stride`-th element (with the q-neighbourhood it
    needs); returns (element ids, oracle J.v rows [n][n_pe], seconds)."""
    import numpy as np
    import oracle
    o = oracle.Oracle(mesh, JV_P, oracle.CONVDIFF, oracle.CASE_EXPSIN, JV_MU)
    el = np.arange(0, mesh.n_elem, stride, dtype=np.int64)
    t0 = time.perf_counter()
    ref = o.jvp_some(u_h, v_h, el)
    return el, ref.reshape(len(el), -1), time.perf_counter() - t0


def run_jv(args):
    """The default workload: FP64 J.v GDOF/s on 48^3 hexahedra, p = 4."""
    import numpy as np
    import torch
    import torch.distributed as dist
    from paper_2205_07824_b300 import synth
    from paper_2205_07824_b300.ldg import LDG, CONVDIFF, CASE_EXPSIN, kernel_launches

    world, rank, local = _dist()
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl")
    mesh = synth.hex_box(JV_N)
    stream = torch.cuda.current_stream()
    g = LDG(mesh, JV_P, CONVDIFF, CASE_EXPSIN, JV_MU, krylov_precision=0)
    tile, _ = g.autotune()
    n = g.n_dof
    u = g.interpolate(0.0)
    v = torch.randn(n, dtype=torch.float64, device="cuda", generator=torch.Generator("cuda").manual_seed(1 + rank))
    out = torch.empty_like(v)

    def timed(prec, steps, warmup):
        for _ in range(warmup):
            g.jvp_prec(prec, u, v, out)
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        l0 = kernel_launches()
        e0.record(stream)
        for _ in range(steps):
            g.jvp_prec(prec, u, v, out)
        e1.record(stream)
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
        return e0.elapsed_time(e1), kernel_launches() - l0

    clocks = ClockSampler(local)
    clocks.start()
    t64, launches = timed(0, args.steps, args.warmup)
    clk = clocks.stop()
    jv64 = out.clone()
    total_ms, gdofs = aggregate([t64], n * args.steps, world, rank)
    ms = t64 / args.steps

    # the FP32-arithmetic J.v (FP64 storage) on the same inputs
    t32, _ = timed(1, args.steps, args.warmup)
    jv32 = out.clone()
    ms32 = t32 / args.steps
    # the (hi, lo) float-pair J.v (emulated FP64 on the FP32 pipes) on the same inputs
    tff, _ = timed(2, args.steps, args.warmup)
    jvff = out.clone()
    msff = tff / args.steps

    peaks = _peaks()
    hbm = float(peaks.get("hbm_gbs", 6400.0))
    hbm64 = JV_BYTES_PER_DOF * n / (ms * 1e-3) / 1e9
    hbm32 = JV_BYTES_PER_DOF * n / (ms32 * 1e-3) / 1e9
    kname = g.jv_kernels(0)
    fpd = JV_FLOP_PER_DOF.get(kname)
    roofline = {"bound": "alu" if fpd else "hbm",
                "unit": "TFLOP/s" if fpd else "GB/s",
                "achieved": (fpd * n / (ms * 1e-3) / 1e12) if fpd else hbm64,
                "peak": FP64_PEAK_TFLOPS if fpd else hbm,
                "traffic": JV_TRAFFIC_PER_DOF.get(kname, 0) * n or None,
                "kernel": kname + " (one J.v: all its launches)",
                "timing": "CUDA events on the launching stream around the K timed J.v applications",
                "flop_per_dof": fpd,
                "flop_source": "ncu thread-instruction counts of the kernels (DFMA x2 + DADD + DMUL)" if fpd else None,
                "peak_source": "FP64 ALU: 148 SMs x 2 FMA/clk x 2 FLOP x 2.032 GHz (derived)" if fpd else
                               ("measured copy bandwidth" if "hbm_gbs" in peaks else "fallback 6.4 TB/s"),
                "hbm": {"bytes_per_dof": JV_BYTES_PER_DOF, "achieved_gbs": hbm64, "peak_gbs": hbm,
                        "frac": hbm64 / hbm,
                        "peak_source": "measured copy bandwidth" if "hbm_gbs" in peaks else "fallback 6.4 TB/s"}}
    roofline["frac"] = roofline["achieved"] / roofline["peak"]

    # FP32 and FP64 J.v against the FP64 oracle on sampled elements (rank 0)
    samp = None
    cpu = None
    if rank == 0:
        uh, vh = u.cpu().numpy(), v.cpu().numpy()
        el, ref, _ = jv_oracle_sample(mesh, uh, vh, 1103)
        npe = g.n_pe
        r64 = jv64.view(-1, npe).cpu().numpy()[el]
        r32 = jv32.view(-1, npe).cpu().numpy()[el]
        rff = jvff.view(-1, npe).cpu().numpy()[el]
        nr = np.linalg.norm(ref)
        samp = {"elements": int(len(el)), "stride": 1103,
                "fp64_rel_err_vs_oracle": float(np.linalg.norm(r64 - ref) / nr),
                "fp32_rel_err_vs_oracle": float(np.linalg.norm(r32 - ref) / nr),
                "f32x2_rel_err_vs_oracle": float(np.linalg.norm(rff - ref) / nr)}
        if not args.no_cpu_baseline:
            el_c, _, sec = jv_oracle_sample(mesh, uh, vh, 251)
            cpu = {"value": len(el_c) * npe / sec / 1e9, "unit": UNIT, "cores": 1, "kind": "oracle",
                   "sample": f"the FP64 oracle's J.v on every 251st element ({len(el_c)} elements, each with "
                             f"the q-stage of its face neighbours), {sec:.1f} s single-threaded; "
                             "DOF of the sampled elements / time"}

    # end to end through the host-buffer C-ABI calls: every step copies its direction in from
    # pinned host memory and its J.v back. ldg_jvp_host_many overlaps the copies of one step
    # with the J.v of its neighbours (the headline e2e); ldg_jvp_host does the three in turn.
    e2e = None
    if not args.no_e2e:
        hv = [torch.empty(n, dtype=torch.float64, pin_memory=True) for _ in range(2)]
        hv[0].copy_(v)
        hv[1].copy_(v)
        hv[1].mul_(-0.5)
        ho = [torch.empty(n, dtype=torch.float64, pin_memory=True) for _ in range(2)]
        k2 = max(3, args.steps)
        g.jvp_host_many(0, None, hv, ho)             # staging buffers and streams allocated once
        if world > 1:
            dist.barrier()
        t0 = time.perf_counter()
        g.jvp_host_many(0, None, [hv[i % 2] for i in range(k2)], [ho[i % 2] for i in range(k2)])
        te = time.perf_counter() - t0
        tmax, e2e_gdofs = aggregate([te * 1e3], n * k2, world, rank)
        k1 = max(3, min(args.steps, 10))
        g.jvp_host(0, None, hv[0], ho[0])
        t0 = time.perf_counter()
        for _ in range(k1):
            g.jvp_host(0, None, hv[0], ho[0])
        t1 = time.perf_counter() - t0
        tmax1, e2e1 = aggregate([t1 * 1e3], n * k1, world, rank)
        # the host link's own time for one step's copies: 8 n bytes in and 8 n out, on two
        # streams at once (what bounds the overlapped calls)
        sa, sb = torch.cuda.Stream(), torch.cuda.Stream()
        da = torch.empty(n, dtype=torch.float64, device="cuda")
        link = []
        for rep in range(6):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            with torch.cuda.stream(sa):
                da.copy_(hv[0], non_blocking=True)
            with torch.cuda.stream(sb):
                ho[1].copy_(v, non_blocking=True)
            torch.cuda.synchronize()
            if rep >= 2:
                link.append((time.perf_counter() - t0) * 1e3)
        del da
        link_ms = statistics.median(link)
        e2e = {"value": e2e_gdofs, "unit": UNIT, "h2d_bytes_per_step": 8 * n, "d2h_bytes_per_step": 8 * n,
               "steps": k2, "ms_per_step": tmax / k2,
               "host_link": {"copies_ms": link_ms, "frac": link_ms / (tmax / k2),
                             "what": "one step's copies alone (8 n bytes in, 8 n out, two streams at once), "
                                     "median of 4; frac = that time / ms_per_step"},
               "call": "ldg_jvp_host_many (FP64): one call over the K step directions, each copied in from "
                       "pinned host memory and its J.v copied back, the copies of a step overlapped with the J.v "
                       "of its neighbours (two device slots, copy-in and copy-out streams); host wall clock "
                       "around the call (a linear model's J.v does not read u)",
               "single_call": {"value": e2e1, "ms_per_step": tmax1 / k1, "steps": k1,
                               "call": "ldg_jvp_host per step: copy in, J.v, copy back, synchronise"}}

    solve = c5 = None
    if not args.no_solve:
        solve = vortex_solve_summary(args, stream)
        c5 = cylinder_solve_summary(args, stream)

    if rank == 0:
        line = {"metric": METRIC, "value": gdofs, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
                "config": {"workload": JV_WORKLOAD, "n_dof": int(n), "n_elem": int(mesh.n_elem),
                           "step": "one FP64 J.v application (q-stage of the direction, then the residual stage)",
                           "tile": tile,
                           "l2": "not flushed: the inputs and scratch of each J.v (553 MB) exceed the 126 MB L2",
                           "parallelism": f"{world} independent instance(s), one per GPU",
                           "fp32_jv": {"ms": ms32, "gdofs": n / (ms32 * 1e-3) / 1e9, "hbm_gbs": hbm32,
                                       "hbm_frac": hbm32 / hbm, "kernel": g.jv_kernels(1),
                                       "arithmetic": "FP32 (inputs and output FP64 in memory, q scratch FP32)"},
                           "f32x2_jv": {"ms": msff, "gdofs": n / (msff * 1e-3) / 1e9,
                                        "hbm_gbs": JV_BYTES_PER_DOF * n / (msff * 1e-3) / 1e9,
                                        "hbm_frac": JV_BYTES_PER_DOF * n / (msff * 1e-3) / 1e9 / hbm,
                                        "kernel": g.jv_kernels(2),
                                        "arithmetic": "(hi, lo) float pairs on the FP32 pipes, about 48 significand "
                                                      "bits (emulated FP64); inputs and output FP64 in memory, q "
                                                      "scratch float pairs"},
                           "oracle_sample": samp,
                           "solve_time_to_1e-8": solve,
                           "c5_time_to_1e-8_scaled16": c5},
                "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": int(launches),
                "clocks": clk}
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def run_mlp_probe(args):
    """The learned preconditioner's tensor-core inference for profilers and timing: the
    network of a 256 x 256 quadrilateral Euler mesh at p = 3 (65,536 element rows, n = 64,
    hidden width 128; three tcgen05 GEMMs per apply), `warmup` untimed and `steps` timed
    applications (CUDA events on the launching stream); prints the time per apply."""
    import torch
    from paper_2205_07824_b300 import synth
    from paper_2205_07824_b300.ldg import LDG, EULER, CASE_VORTEX
    mesh = synth.quad_box(256, hi=(10.0, 10.0), periodic=(True, True))
    g = LDG(mesh, 3, EULER, CASE_VORTEX, (1.4,), gmres_m=1)
    g.mlp_init(seed=1)
    u = g.interpolate(0.0)
    x = torch.randn(g.n_dof, dtype=torch.float64, device="cuda", generator=torch.Generator("cuda").manual_seed(2))
    out = torch.empty_like(x)
    stream = torch.cuda.current_stream()
    for _ in range(max(args.warmup, 1)):
        g.mlp_apply(u, x, out)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        g.mlp_apply(u, x, out)
    e1.record(stream)
    torch.cuda.synchronize()
    print(json.dumps({"probe": "learned preconditioner inference, 65,536 element rows (256 x 256 quadrilaterals, "
                               "Euler p = 3), three tcgen05 GEMMs per apply",
                      "ms_per_apply": e0.elapsed_time(e1) / max(args.steps, 1), "applies": args.steps,
                      "finite": bool(torch.isfinite(out).all().item())}))


def run_jv_probe(args):
    """The default workload's J.v for profilers: the same context with a one-column Krylov
    space (about 1.5 GB on the device), no autotuning, `warmup + steps` FP64 J.v applications
    then as many FP32 ones and as many float-pair ones; prints the kernels it ran."""
    import torch
    from paper_2205_07824_b300 import synth
    from paper_2205_07824_b300.ldg import LDG, CONVDIFF, CASE_EXPSIN
    g = LDG(synth.hex_box(JV_N), JV_P, CONVDIFF, CASE_EXPSIN, JV_MU, gmres_m=1)
    u = g.interpolate(0.0)
    v = torch.randn(g.n_dof, dtype=torch.float64, device="cuda", generator=torch.Generator("cuda").manual_seed(1))
    out = torch.empty_like(v)
    for prec in (0, 1, 2):
        for _ in range(args.warmup + args.steps):
            g.jvp_prec(prec, u, v, out)
    torch.cuda.synchronize()
    print(json.dumps({"probe": JV_WORKLOAD, "fp64": g.jv_kernels(0), "fp32": g.jv_kernels(1),
                      "f32x2": g.jv_kernels(2), "applications_each": args.warmup + args.steps}))


def vortex_solve_summary(args, stream):
    """Newton-GMRES time to 1e-8 of the 64x64 p=3 vortex BDF2 step: FP32 Krylov J.v +
    block-Jacobi against plain FP64 block-Jacobi (same steps, same forcing rule), and the
    same step end to end through the host-buffer solve call."""
    import torch
    from paper_2205_07824_b300 import synth
    from paper_2205_07824_b300.ldg import LDG, BDF2, kernel_launches
    mesh = synth.quad_box(N_SIDE, hi=(10.0, 10.0), periodic=(True, True))
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")
    steps = max(3, min(args.steps, 10))
    prob = vortex_problem(LDG, mesh, forcing_of(args), 1)
    forms = {}
    sol = {}
    for name, kp in (("fp32_krylov_bjacobi", 1), ("fp64_bjacobi", 0), ("tc_bf16x3_krylov_bjacobi", 3),
                     ("tc_bf16_krylov_bjacobi", 4)):
        g, u, times, tot, _, t_end, _ = run_mode(prob, kp, 1, steps, 3, flush, stream, kernel_launches)
        forms[name] = {"ms_per_step": sum(times) / steps, "gmres_iters_per_step": tot["gmres"] / steps,
                       "newton_iters_per_step": tot["newton"] / steps}
        sol[name] = u.clone()
        if kp == 1:
            # the same step end to end: u^n from host memory through ldg_newton_gmres_host
            import numpy as np
            un = u.cpu().numpy()
            g.set_time(BDF2, t_end + DT, DT, u, u)
            hu = np.array(un)
            g.newton_gmres_host(hu)                       # untimed first call
            k2 = 3
            t0 = time.perf_counter()
            for _ in range(k2):
                hu[:] = un
                rep = g.newton_gmres_host(hu)
            te = (time.perf_counter() - t0) / k2
            forms[name]["e2e_host_call_ms"] = te * 1e3
            forms[name]["e2e_note"] = ("ldg_newton_gmres_host: u^n copied in from host memory, solved to 1e-8, "
                                       "solution copied back; host wall clock")
        del g
    forms["speedup_fp32_vs_fp64"] = forms["fp64_bjacobi"]["ms_per_step"] / forms["fp32_krylov_bjacobi"]["ms_per_step"]
    forms["solution_rel_diff"] = float(torch.linalg.norm(sol["fp32_krylov_bjacobi"] - sol["fp64_bjacobi"]) /
                                       torch.linalg.norm(sol["fp64_bjacobi"]))
    for name in ("tc_bf16x3_krylov_bjacobi", "tc_bf16_krylov_bjacobi"):
        forms[name]["speedup_vs_fp64_bjacobi"] = forms["fp64_bjacobi"]["ms_per_step"] / forms[name]["ms_per_step"]
        forms[name]["solution_rel_diff_vs_fp64_bjacobi"] = float(
            torch.linalg.norm(sol[name] - sol["fp64_bjacobi"]) / torch.linalg.norm(sol["fp64_bjacobi"]))
    forms["workload"] = WORKLOAD
    forms["jv_kernels"] = vortex_jv_kernels(mesh, sol["fp64_bjacobi"], args)
    return forms


# tensor-core MMA flops per element of the Euler J.v at p = 3 (padded GEMM extents, 32
# elements per CTA): interpolation of u and v (2 x 128 x 32 x 16 x 2), own and neighbour
# face traces (4 x 128 x 32 x 16 x 2), mass (128 x 16 x 16 x 2), volume integration
# (128 x 16 x 64 x 2) and lift (128 x 16 x 32 x 2), per CTA / 32, times the passes
TC_MMA_FLOP_PER_ELEM_P3 = (2 * 128 * 32 * 16 * 2 + 4 * 128 * 32 * 16 * 2 + 128 * 16 * 16 * 2 + 128 * 16 * 64 * 2 +
                           128 * 16 * 32 * 2) / 32


def vortex_jv_kernels(mesh, u, args):
    """The c2 J.v (64 x 64 quadrilaterals, p = 3, Euler) in every arithmetic: graph-timed
    kernel time at the state u and a random direction, and each form's error against the
    FP64 oracle's J.v on the same inputs."""
    import numpy as np
    import torch
    from paper_2205_07824_b300.ldg import LDG, EULER, CASE_VORTEX
    g = LDG(mesh, P, EULER, CASE_VORTEX, (1.4,), gmres_m=2)
    g.autotune()
    v = torch.randn(g.n_dof, dtype=torch.float64, device="cuda", generator=torch.Generator("cuda").manual_seed(3))
    out = torch.empty_like(v)
    peaks = _peaks()
    bf16 = float(peaks.get("bf16_tflops", 1800.0))
    rows = {}
    res = {}
    for name, kp in (("fp64", 0), ("fp32", 1), ("tc_bf16x3", 3), ("tc_bf16", 4)):
        ms = graph_time_ms(g, lambda: g.jvp_prec(kp, u, v, out), args.jv_reps)
        g.jvp_prec(kp, u, v, out)
        res[name] = out.cpu().numpy().copy()
        rows[name] = {"us": ms * 1e3, "gdofs": g.n_dof / (ms * 1e-3) / 1e9, "kernel": g.jv_kernels(kp)}
        if kp >= 3:
            passes = 3 if kp == 3 else 1
            tf = TC_MMA_FLOP_PER_ELEM_P3 * passes * mesh.n_elem / (ms * 1e-3) / 1e12
            rows[name]["tensor_tflops"] = tf
            rows[name]["tensor_frac_of_bf16_peak"] = tf / bf16
    if not args.no_cpu_baseline:
        # the FP64 oracle's J.v on the same inputs (rank 0, after the timed regions)
        import oracle
        o = oracle.Oracle(mesh, P, oracle.EULER, oracle.CASE_VORTEX, (1.4,))
        ref = o.jvp(u.cpu().numpy(), v.cpu().numpy())
        for name in rows:
            rows[name]["rel_err_vs_fp64_oracle"] = float(np.linalg.norm(res[name] - ref) / np.linalg.norm(ref))
    rows["timing"] = "CUDA graph of jv_reps back-to-back J.v launches, one replay timed with CUDA events"
    rows["bf16_peak_source"] = "measured cuBLAS bf16 (burst)" if "bf16_tflops" in peaks else "fallback 1.8 PFLOP/s"
    del g
    return rows


def run_tc_probe(args):
    """The Euler J.v (periodic vortex box, p = 3) in FP64, FP32 and with the tensor-core
    contractions (BF16 hi/lo splits and one BF16 product) on square meshes of the given
    sides: graph-timed kernel time per launch, one JSON line; also the command a profiler
    captures the tensor-core kernel under (--tc-sides 256)."""
    import torch
    from paper_2205_07824_b300 import synth
    from paper_2205_07824_b300.ldg import LDG, EULER, CASE_VORTEX
    torch.cuda.set_device(0)
    peaks = _peaks()
    bf16 = float(peaks.get("bf16_tflops", 1800.0))
    table = {}
    for side in (int(x) for x in args.tc_sides.split(",")):
        mesh = synth.quad_box(side, hi=(10.0, 10.0), periodic=(True, True))
        g = LDG(mesh, P, EULER, CASE_VORTEX, (1.4,), gmres_m=2, krylov_precision=1)
        g.autotune()
        u = g.interpolate(0.0)
        v = torch.randn(g.n_dof, dtype=torch.float64, device="cuda", generator=torch.Generator("cuda").manual_seed(5))
        out = torch.empty_like(v)
        row = {"n_dof": int(g.n_dof)}
        for name, kp in (("fp64", 0), ("fp32", 1), ("tc_bf16x3", 3), ("tc_bf16", 4)):
            ms = graph_time_ms(g, lambda: g.jvp_prec(kp, u, v, out), args.jv_reps)
            row[name] = {"us": ms * 1e3, "gdofs": g.n_dof / (ms * 1e-3) / 1e9}
            if kp >= 3:
                tf = TC_MMA_FLOP_PER_ELEM_P3 * (3 if kp == 3 else 1) * mesh.n_elem / (ms * 1e-3) / 1e12
                row[name]["tensor_frac_of_bf16_peak"] = tf / bf16
        table[f"{side}x{side}"] = row
        del g
    print(json.dumps({"workload": "Euler J.v, periodic isentropic-vortex box [0,10]^2, p=3, 5 Gauss points per "
                                  "direction", "timing": "CUDA graph of jv_reps back-to-back J.v launches, one "
                                  "replay timed with CUDA events", "table": table}), flush=True)


def cylinder_solve_summary(args, stream):
    """Time to 1e-8 per BDF2 step of the Navier-Stokes cylinder on 1/16 of c5's mesh (25
    layers x 100 around, 2,500 curved quadrilaterals, p = 3, Re from seed 0): plain FP64
    block-Jacobi, FP32 Krylov J.v + block-Jacobi, and FP32 Krylov J.v + the learned
    correction of block-Jacobi trained on the warm-up steps' block-Jacobi solves."""
    import numpy as np
    import torch
    from paper_2205_07824_b300 import synth
    from paper_2205_07824_b300.ldg import LDG, kernel_launches
    mesh = synth.cylinder_mesh(25, 100, 3, seed=7)
    re = float(np.random.default_rng(0).uniform(100.0, 1000.0))
    prob = cylinder_problem(LDG, mesh, re, forcing_of(args))
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")
    steps = 2
    forms, sol = {}, {}
    for name, kp, pc in (("fp64_bjacobi", 0, 1), ("fp32_bjacobi", 1, 1), ("fp32_learned", 1, 3)):
        g, u, times, tot, _, _, train = run_mode(prob, kp, pc, steps, 3, flush, stream, kernel_launches)
        forms[name] = {"ms_per_step": sum(times) / steps, "gmres_iters_per_step": tot["gmres"] / steps,
                       "newton_iters_per_step": tot["newton"] / steps, "pc_fallbacks": tot["pc_fallbacks"]}
        if train:
            forms[name]["learned_pc_training"] = {k: train[k] for k in ("pairs", "vectors") if k in train}
        sol[name] = u.clone()
        del g
    base = forms["fp64_bjacobi"]["ms_per_step"]
    for name in ("fp32_bjacobi", "fp32_learned"):
        forms[name]["speedup_vs_fp64_bjacobi"] = base / forms[name]["ms_per_step"]
        forms[name]["solution_rel_diff_vs_fp64_bjacobi"] = float(
            torch.linalg.norm(sol[name] - sol["fp64_bjacobi"]) / torch.linalg.norm(sol["fp64_bjacobi"]))
    forms["workload"] = (f"2D compressible Navier-Stokes past a cylinder, 1/16 of the c5 mesh: 2,500 curved "
                         f"quadrilaterals (25 layers x 100 around, seed 7), p=3, Re={re:.1f}, Mach 0.2, BDF2 "
                         f"dt=0.1, Newton-GMRES(30) to 1e-8 (FP64 residual); {steps} timed steps after 3 warm-up "
                         f"steps per form; the full 40,000-element case is bench.py --workload cylinder")
    return forms


def forcing_of(args):
    """ldg newton_forcing value of the --forcing choice."""
    return 1 if args.forcing == "last" else 0


def linear_tolerance(args):
    """The linear-solve tolerance rule of the --forcing choice, for the JSON config."""
    return ("max(1e-3, 0.5e-8 ||R0|| / ||Rk||) per Newton step k (every form)" if args.forcing == "last"
            else "1e-3 per Newton step")


def vortex_problem(LDG, mesh, forcing=0, pc_reuse=1, basis=0):
    """The vortex: context factory (preconditioner, Krylov precision), initial states, dt."""
    from paper_2205_07824_b300.ldg import EULER, CASE_VORTEX

    def make(p, kprec):
        return LDG(mesh, P, EULER, CASE_VORTEX, (1.4,), gmres_m=30, newton_rtol=1e-8, gmres_rtol=1e-3,
                   krylov_precision=kprec, precond=p, newton_forcing=forcing, pc_reuse=pc_reuse, krylov_basis=basis)
    return dict(make=make, init=lambda g: (g.interpolate(0.0), g.interpolate(-DT)), dt=DT, n_elem=mesh.n_elem)


def run_mode(prob, kprec, pc, steps, warmup, flush, stream, launches):
    """Advance the problem `warmup` + `steps` BDF2 steps; time the last `steps`.

    pc = 2 (learned, distilled block-Jacobi): the warm-up steps run the block-Jacobi
    solver and collect its (v, M^{-1} v, u) triples; pc = 3 (learned correction of
    block-Jacobi): they collect the solver's (residual, update) pairs, its Newton steps
    (R(u_k), delta_k) and its Arnoldi steps (J z_j, z_j), as block-Jacobi features. The
    network is trained on them once (reported, not in the timed steps), one more untimed
    step runs with the learned preconditioner, then the timed steps."""
    import torch
    from paper_2205_07824_b300.ldg import BDF2
    DT = prob["dt"]
    mk = lambda p: prob["make"](p, kprec)
    g = mk(1 if pc in (2, 3) else pc)
    g.autotune()                       # tile of the kernels (cached per shape in the process)
    un, unm1 = prob["init"](g)
    u = torch.empty_like(un)
    state = {"t": 0.0, "g": g}
    nloc = g.n_cu * g.n_pe
    train = None
    cap = 160 if pc in (2, 3) else 0
    if cap:
        bufs = [torch.empty(cap * g.n_dof, dtype=torch.float64, device="cuda") for _ in range(3)]
        state["used"] = 0

    def step(collect=False):
        gg = state["g"]
        t1 = state["t"] + DT
        gg.set_time(BDF2, t1, DT, un, unm1)
        u.copy_(un)
        if collect and state["used"] < cap:
            o = state["used"] * gg.n_dof
            if pc == 3:
                c, rep = gg.newton_collect_updates(u, bufs[0][o:], bufs[1][o:], bufs[2][o:], cap - state["used"], 3)
            else:
                c, rep = gg.newton_gmres_collect(u, bufs[0][o:], bufs[1][o:], bufs[2][o:], cap - state["used"])
            state["used"] += c
        else:
            rep = gg.newton_gmres(u)
        unm1.copy_(un)
        un.copy_(u)
        state["t"] = t1
        return rep

    # the learned form spends its last warm-up step on the learned preconditioner (after
    # training), so every form ends its timed steps at the same time level
    for _ in range(max(1, warmup - 1) if cap else warmup):
        step(collect=bool(cap))
    if cap:
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        nd = state["used"] * g.n_dof
        g.mlp_init(seed=1)
        rep_t = g.mlp_train(bufs[0][:nd], bufs[1][:nd], bufs[2][:nd], epochs=8, batch=4096, lr=1e-3)
        torch.cuda.synchronize()
        train = {"pairs": state["used"] * prob["n_elem"], "vectors": state["used"],
                 "seconds": time.perf_counter() - t0,
                 "adam_steps": rep_t["steps"], "loss_first": rep_t["loss_first"], "loss_last": rep_t["loss_last"],
                 "data": ("(residual, update) pairs of the block-Jacobi warm-up solves: Newton steps (R(u_k), delta_k) "
                          "and Arnoldi steps (J z_j, z_j), as block-Jacobi images with neighbour traces" if pc == 3 else
                          "Arnoldi vectors of the block-Jacobi warm-up steps with their block corrections")}
        gm = mk(pc)
        gm.autotune()
        gm.mlp_init(seed=1)
        gm.mlp_params(g.mlp_params())
        state["g"] = gm
        del bufs
        step()
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    tot = {"jv": 0, "newton": 0, "gmres": 0, "pc": 0}
    l0 = launches()
    for k in range(steps):
        flush.zero_()
        ev[k][0].record(stream)
        rep = step()
        ev[k][1].record(stream)
        assert rep["rfinal"] <= 1e-8 * rep["r0"], rep
        tot["jv"] += rep["jv_calls"] + rep["pc_setups"] * nloc   # block extraction: one J.v per block column
        tot["newton"] += rep["newton_iters"]
        tot["gmres"] += rep["gmres_iters"]
        tot["pc"] += rep["pc_setups"]
        tot["pc_fallbacks"] = tot.get("pc_fallbacks", 0) + rep["pc_fallbacks"]
    torch.cuda.synchronize()
    n_launch = launches() - l0
    times = [a.elapsed_time(b) for a, b in ev]
    tot["pc_fallbacks"] = tot.get("pc_fallbacks", 0)
    return state["g"], u, times, tot, n_launch, state["t"], train


BATCH_WORKLOAD = ("256 steady 2D convection-diffusion instances, kappa log-uniform on [1e-3,1e-1], beta = "
                  "(cos a, sin a) with a uniform on [0,2pi), quad meshes of [0,1]^2 with side uniform in "
                  "{8,16,32,64}, p uniform in {2,3,4} (seed 20221), manufactured u = sin(pi x) sin(pi y) with "
                  "Dirichlet data, Newton-GMRES(30) to 1e-8 per instance, one CUDA graph launch")
# Algorithmic HBM bytes per DOF of the linear J.v (q-stage then residual, FP64 storage):
# read v twice (8 + 8), write and read q(v) (2 x 16), write J.v (8).
BATCH_JV_BYTES_PER_DOF = 56.0


def run_batch(args):
    """The batched parametrised workload: every step solves all instances from u = 0."""
    import numpy as np
    import torch
    import torch.distributed as dist
    from paper_2205_07824_b300 import synth
    from paper_2205_07824_b300.ldg import Batch, CONVDIFF, CASE_SINSIN, kernel_launches

    world, rank, local = _dist()
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl")
    insts = synth.batch_instances(256, 20221 + rank)
    meshes = [synth.quad_box(d["side"]) for d in insts]
    ps = [d["p"] for d in insts]
    mus = [(d["kappa"], 1.0, d["beta"][0], d["beta"][1]) for d in insts]
    kprec = 1 if args.krylov == "fp32" else 0
    pc = 1 if args.precond == "bjacobi" else 0
    stream = torch.cuda.current_stream()
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")   # 256 MiB > L2

    def make(kp):
        return Batch(meshes, ps, CONVDIFF, CASE_SINSIN, mus, gmres_m=30, newton_rtol=1e-8, gmres_rtol=1e-3,
                     krylov_precision=kp, precond=pc, newton_forcing=forcing_of(args))

    def timed(b, steps, warmup, use_graph=True):
        u = b.empty()
        for _ in range(warmup):
            u.zero_()
            b.solve(u, use_graph=use_graph and not args.host_loops)
        times, reps = [], None
        for _ in range(steps):
            u.zero_()
            flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            reps, _ = b.solve(u, use_graph=use_graph and not args.host_loops)
            e1.record(stream)
            torch.cuda.synchronize()
            times.append(e0.elapsed_time(e1))
        return u, times, reps

    b = make(kprec)
    # default tile first, then the autotuned tiles (the headline)
    _, t_def, _ = timed(b, max(1, args.steps // 2), 1)
    tiles = b.autotune(force=True)
    if world > 1:
        dist.barrier()
    clocks = ClockSampler(local)
    clocks.start()
    l0 = kernel_launches()
    u, times, reps = timed(b, args.steps, args.warmup)
    launches = kernel_launches() - l0
    clk = clocks.stop()
    if world > 1:
        dist.barrier()
    bad = [i for i, r in enumerate(reps) if r["status"] != 0 or r["rfinal"] > 1e-8 * r["r0"]]
    assert not bad, [reps[i] for i in bad[:3]]
    jv_dofs = sum(b.n_dof[i] * reps[i]["jv_calls"] for i in range(b.n_inst))
    total_ms, gdofs = aggregate(times, jv_dofs * args.steps, world, rank)
    ms_per_step = total_ms / args.steps
    _, t_eager, _ = timed(b, 1, 0, use_graph=False)

    # plain FP64 block-Jacobi form on the same batch
    base = None
    if not args.no_fp64_baseline and kprec == 1:
        b64 = make(0)
        b64.autotune()
        u64, t64, r64 = timed(b64, max(1, args.steps // 2), 1)
        base = {"form": "FP64 Krylov J.v" + (" + block-Jacobi" if pc else ""), "ms_per_step": sum(t64) / len(t64),
                "gmres_iters_total": int(sum(r["gmres_iters"] for r in r64)),
                "solution_rel_diff_vs_headline": float(torch.linalg.norm(u64 - u) / torch.linalg.norm(u64))}
        base["speedup_headline_vs_fp64"] = base["ms_per_step"] / ms_per_step
        del b64

    # the batched J.v alone (all groups), CUDA events
    v = torch.randn(b.n_total, dtype=torch.float64, device="cuda", generator=torch.Generator("cuda").manual_seed(1))
    jv = torch.empty_like(v)
    for _ in range(5):
        b.jvp(u, v, kprec, jv)
    flush.zero_()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.jv_reps):
        b.jvp(u, v, kprec, jv)
    e1.record(stream)
    torch.cuda.synchronize()
    jv_ms = e0.elapsed_time(e1) / args.jv_reps
    achieved = BATCH_JV_BYTES_PER_DOF * b.n_total / (jv_ms * 1e-3) / 1e9
    peaks = {}
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            peaks = json.load(f)
    except (OSError, ValueError):
        pass
    hbm = float(peaks.get("hbm_gbs", 6400.0))
    roofline = {"bound": "hbm", "unit": "GB/s", "achieved": achieved, "peak": hbm, "frac": achieved / hbm,
                "traffic": None, "kernel": "batched J.v (k_lin_q + k_lin_r over the quadrilateral order groups)",
                "launch_ms": jv_ms, "bytes_per_dof": BATCH_JV_BYTES_PER_DOF,
                "peak_source": "measured copy bandwidth" if "hbm_gbs" in peaks else "fallback 6.4 TB/s"}

    # end to end: host state in, solution out, per step
    h_u = torch.zeros(b.n_total, dtype=torch.float64, pin_memory=True)
    d_u = b.empty()
    k2 = min(args.steps, 3)
    t0 = time.perf_counter()
    jv_e2e = 0
    for _ in range(k2):
        h_u.zero_()
        d_u.copy_(h_u, non_blocking=True)
        r_e, _ = b.solve(d_u, use_graph=not args.host_loops)
        h_u.copy_(d_u)
        jv_e2e += sum(b.n_dof[i] * r_e[i]["jv_calls"] for i in range(b.n_inst))
    t_e2e = time.perf_counter() - t0
    e2e = {"value": jv_e2e / t_e2e / 1e9, "unit": UNIT, "h2d_bytes_per_step": 8 * b.n_total,
           "d2h_bytes_per_step": 8 * b.n_total, "steps": k2, "ms_per_step": t_e2e / k2 * 1e3}

    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        import oracle
        t0, calls, dofs = time.perf_counter(), 0, 0
        for i in range(b.n_inst):
            o = oracle.Oracle(meshes[i], ps[i], oracle.CONVDIFF, oracle.CASE_SINSIN, mus[i])
            x = synth.random_vector(o.ndof, i)
            o.jvp(x, x)
            calls += 1
            dofs += o.ndof
            if time.perf_counter() - t0 > 10.0:
                break
        el = time.perf_counter() - t0
        cpu = {"value": dofs / el / 1e9, "unit": UNIT, "cores": 1, "kind": "oracle",
               "sample": f"one oracle J.v on each of the first {calls} instances ({dofs} DOF, set-up included), "
                         f"{el:.1f} s single-threaded"}
    if rank == 0:
        its = [r["gmres_iters"] for r in reps]
        line = {"metric": METRIC, "value": gdofs, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f64" if kprec == 0 else "f64+f32", "data": "synthetic",
                "config": {"linear_tolerance": linear_tolerance(args), "workload": BATCH_WORKLOAD, "n_inst": b.n_inst, "n_dof_total": int(b.n_total),
                           "order_groups": b.n_groups, "tiles_autotuned": tiles,
                           "value_definition": "sum over instances of DOF x J.v applications (Arnoldi and true "
                                               "residual; block probing excluded) / timed batched solve time",
                           "time_to_1e-8_ms_per_step": ms_per_step,
                           "ms_per_step_default_tile": sum(t_def) / len(t_def),
                           "ms_per_step_host_driven_loops": t_eager[0],
                           "graph_kernel_executions_per_step": b.kernel_executions(),
                           "gmres_iters_min_median_max": [min(its), int(np.median(its)), max(its)],
                           "newton_iters_max": max(r["newton_iters"] for r in reps),
                           "preconditioner": "block-Jacobi (exact element blocks, built in every step)" if pc
                           else "none",
                           "precision": "FP64 throughout" if kprec == 0 else
                           "Krylov J.v and preconditioner in FP32 arithmetic; Newton residual, Arnoldi, Givens, "
                           "vectors FP64",
                           "l2": "flushed (256 MiB write) before each timed step, outside its event window",
                           "parallelism": f"{world} independent 256-instance batch(es), one per GPU",
                           "fp64_baseline": base},
                "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": int(launches),
                "clocks": clk}
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


HEX_WORKLOAD = ("3D steady convection-diffusion on [0,1]^3, 48^3 affine hexahedra, beta = (1, 0.5, 0.25), "
                "kappa = 1e-2, manufactured u = exp(x+y+z) sin(pi xyz); J.v throughput sweep p = 1..6 in FP64 and "
                "FP32 arithmetic (FP64 storage)")
# Algorithmic HBM bytes per DOF of the 3-D linear J.v: v read twice (8 + 8), q(v) written
# and read (2 x 24), J.v written (8).
HEX_JV_BYTES_PER_DOF = 72.0
TRI_WORKLOAD = ("2D steady convection-diffusion on [0,1]^2, 256 x 256 squares split into 131,072 affine "
                "triangles, beta = (1, 0.5), kappa = 1e-2, manufactured u = exp(x+y) sin(pi xy); equispaced nodes, "
                "p + 2 collapsed Gauss points per direction; J.v throughput sweep p = 1..6 in FP64 and FP32 "
                "arithmetic (FP64 storage)")
# Algorithmic HBM bytes per DOF of the 2-D linear J.v: v read twice (8 + 8), q(v) written
# and read (2 x 16), J.v written (8).
TRI_JV_BYTES_PER_DOF = 56.0


def run_hex(args):
    """J.v throughput of the 3-D convection-diffusion operator, p = 1..6 (p = 4 is the headline)."""
    from paper_2205_07824_b300 import synth
    jv_sweep(args, lambda: synth.hex_box(48), (1e-2, 1.0, 1.0, 0.5, 0.25), 4, HEX_JV_BYTES_PER_DOF, HEX_WORKLOAD,
             "FP32 J.v, hex p = 4")


def run_tri(args):
    """J.v throughput of the 2-D convection-diffusion operator on triangles, p = 1..6
    (p = 6 is the headline)."""
    from paper_2205_07824_b300 import synth
    jv_sweep(args, lambda: synth.tri_square(256), (1e-2, 1.0, 1.0, 0.5), 6, TRI_JV_BYTES_PER_DOF, TRI_WORKLOAD,
             "FP32 J.v, triangles p = 6")


def jv_sweep(args, make_mesh, mu, head_p, bytes_per_dof, workload, kernel_label):
    """Median J.v time (L2 flushed before each) of the linear convection-diffusion operator
    on one mesh for p = 1..6 in FP64, FP32 and (hi, lo) float-pair arithmetic; the FP32
    p = head_p row is the headline."""
    import torch
    from paper_2205_07824_b300.ldg import LDG, CONVDIFF, CASE_EXPSIN, kernel_launches
    world, rank, local = _dist()
    torch.cuda.set_device(local)
    mesh = make_mesh()
    stream = torch.cuda.current_stream()
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")
    peaks = {}
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            peaks = json.load(f)
    except (OSError, ValueError):
        pass
    hbm = float(peaks.get("hbm_gbs", 6400.0))
    sweep = []
    head = None
    clocks = ClockSampler(local)
    clocks.start()
    l0 = kernel_launches()
    for p in range(1, 7):
        row = {"p": p}
        for prec in (0, 1, 2):
            g = LDG(mesh, p, CONVDIFF, CASE_EXPSIN, mu, krylov_precision=prec)
            tile, _ = g.autotune()
            u = g.interpolate(0.0)
            v = torch.randn(g.n_dof, dtype=torch.float64, device="cuda",
                            generator=torch.Generator("cuda").manual_seed(p))
            out = torch.empty_like(v)
            for _ in range(args.warmup):
                g.jvp_prec(prec, u, v, out)
            times = []
            for _ in range(args.steps):
                flush.zero_()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                g.jvp_prec(prec, u, v, out)
                e1.record(stream)
                torch.cuda.synchronize()
                times.append(e0.elapsed_time(e1))
            ms = sorted(times)[len(times) // 2]
            key = ("fp64", "fp32", "f32x2")[prec]
            row[key] = {"ms": ms, "gdofs": g.n_dof / (ms * 1e-3) / 1e9, "tile": tile,
                        "hbm_frac": bytes_per_dof * g.n_dof / (ms * 1e-3) / 1e9 / hbm}
            row[key]["kernels"] = g.jv_kernels(prec)
            row["n_dof"] = g.n_dof
            if p == head_p and prec == 1:
                head = (g.n_dof, ms, tile)
                kernel_label = g.jv_kernels(prec)
            del g, u, v, out
            torch.cuda.empty_cache()
        sweep.append(row)
    launches = kernel_launches() - l0
    clk = clocks.stop()
    n, ms, tile = head
    achieved = bytes_per_dof * n / (ms * 1e-3) / 1e9
    line = {"metric": METRIC, "value": n / (ms * 1e-3) / 1e9, "unit": UNIT, "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64+f32", "data": "synthetic",
            "config": {"workload": workload, f"n_dof_p{head_p}": n,
                       "step": "one J.v application (median of the timed ones)",
                       "headline": f"p = {head_p}, FP32 arithmetic", "sweep": sweep,
                       "l2": "flushed (256 MiB write) before each timed J.v"},
            "roofline": {"bound": "hbm", "unit": "GB/s", "achieved": achieved, "peak": hbm, "frac": achieved / hbm,
                         "traffic": None, "bytes_per_dof": bytes_per_dof,
                         "kernel": kernel_label,
                         "peak_source": "measured copy bandwidth" if "hbm_gbs" in peaks else "fallback 6.4 TB/s"},
            "cpu_baseline": None, "e2e": None, "gpu_launches": int(launches), "clocks": clk}
    print(json.dumps(line), flush=True)


TET_WORKLOAD = ("Section 4.1 / Table 3: 3D Poisson -lap u = f on the unit cube, u = sin(pi x) sin(pi y) sin(pi z), "
                "structured tetrahedral mesh 1/n = {n} (6 n^3 = {E} tetrahedra), p = {p}, Dirichlet data; one "
                "Newton-GMRES(30) solve from u = 0 to 1e-8 (linear solves to 1e-3) with block-Jacobi")
# Algorithmic HBM bytes per DOF of the 3-D linear J.v (FP64 storage): v read twice,
# q(v) written and read (3 components), J.v written: (2 + 2 x 3 + 1) x 8
TET_JV_BYTES_PER_DOF = 72.0


def run_tet(args):
    """Table 3's finest mesh on the GPU: the J.v (FP64, FP32 and float-pair arithmetic)
    against the HBM roofline, and the time of the whole Newton-GMRES solve."""
    import torch
    from paper_2205_07824_b300 import synth
    from paper_2205_07824_b300.ldg import LDG, POISSON, CASE_SINSIN, kernel_launches
    world, rank, local = _dist()
    torch.cuda.set_device(local)
    n_side, p = args.tet_n, args.tet_p
    mesh = synth.tet_cube(n_side)
    peaks = {}
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            peaks = json.load(f)
    except (OSError, ValueError):
        pass
    hbm = float(peaks.get("hbm_gbs", 6400.0))
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream()
    clocks = ClockSampler(local)
    clocks.start()
    l0 = kernel_launches()
    jv = {}
    for prec in (1, 0, 2):
        g = LDG(mesh, p, POISSON, CASE_SINSIN, (1.0, 1.0), krylov_precision=prec, precond=1, newton_rtol=1e-8,
                gmres_rtol=1e-3, max_restarts=400)
        tile, _ = g.autotune()
        u = g.interpolate(0.0)
        v = torch.randn(g.n_dof, dtype=torch.float64, device="cuda", generator=torch.Generator("cuda").manual_seed(1))
        out = torch.empty_like(v)
        ms = graph_time_ms(g, lambda: g.jvp_prec(prec, u, v, out), args.jv_reps)
        key = ("fp64", "fp32", "f32x2")[prec]
        jv[key] = {"ms": ms, "gdofs": g.n_dof / (ms * 1e-3) / 1e9, "tile": tile,
                   "hbm_frac": TET_JV_BYTES_PER_DOF * g.n_dof / (ms * 1e-3) / 1e9 / hbm}
        jv[key]["kernels"] = g.jv_kernels(prec)
        if prec == 1:
            g32 = g
    # the solve: FP32 Krylov + block-Jacobi from u = 0, timed steps (each a full solve)
    n = g32.n_dof
    times, reps = [], []
    for k in range(args.warmup + args.steps):
        u = torch.zeros(n, dtype=torch.float64, device="cuda")
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        rep = g32.newton_gmres(u)
        e1.record(stream)
        torch.cuda.synchronize()
        if k >= args.warmup:
            times.append(e0.elapsed_time(e1))
            reps.append(rep)
    launches = kernel_launches() - l0
    clk = clocks.stop()
    assert all(r["status"] == 0 for r in reps), reps
    ms_step = sum(times) / len(times)
    jv_calls = sum(r["jv_calls"] for r in reps) / len(reps)
    head = jv["fp32"]
    achieved = TET_JV_BYTES_PER_DOF * n / (head["ms"] * 1e-3) / 1e9
    line = {"metric": METRIC, "value": head["gdofs"], "unit": UNIT, "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64+f32", "data": "synthetic",
            "config": {"workload": TET_WORKLOAD.format(n=n_side, E=mesh.n_elem, p=p), "n_dof": n,
                       "value_definition": "FP32-arithmetic J.v of the solve, DOF / kernel time (graph-timed)",
                       "jv": jv, "solve_ms": ms_step, "newton_iters": reps[-1]["newton_iters"],
                       "gmres_iters": reps[-1]["gmres_iters"], "jv_calls_per_solve": jv_calls,
                       "l2": "flushed (256 MiB write) before each timed solve; J.v graph-timed"},
            "roofline": {"bound": "hbm", "unit": "GB/s", "achieved": achieved, "peak": hbm, "frac": achieved / hbm,
                         "traffic": None, "bytes_per_dof": TET_JV_BYTES_PER_DOF,
                         "kernel": g32.jv_kernels(1),
                         "peak_source": "measured copy bandwidth" if "hbm_gbs" in peaks else "fallback 6.4 TB/s"},
            "cpu_baseline": None, "e2e": None, "gpu_launches": int(launches), "clocks": clk}
    print(json.dumps(line), flush=True)


WAVE_WORKLOAD = ("Section 2.1's wave model: w_tt = c^2 lap w as u = w_t, dq/dt + grad u = 0, du/dt + "
                 "div(c^2 q) = 0 and the ODE dw/dt = u, on [0,1]^3 with 48^3 hexahedra, p = 4 (13,824,000 DOF "
                 "of u, 41,472,000 of q), c = 1, tau = 1, homogeneous Dirichlet; from w = sin(pi x) sin(pi y) "
                 "sin(pi z), u = 0, q = Q(w); DIRK34 steps of dt = h / 2, each stage a Newton-GMRES(30) "
                 "solve to 1e-8 (linear solves to 1e-6, no preconditioner)")


def run_wave(args):
    """DIRK34 steps of the scalar wave equation (the wave model with the displacement ODE)
    on 48^3 hexahedra, p = 4: time per step, the Krylov J.v count, and the displacement's
    nodal error against the exact standing wave at the end."""
    import math
    import torch
    from paper_2205_07824_b300 import synth
    from paper_2205_07824_b300.ldg import LDG, CONVDIFF, CASE_ZERO, CASE_SINSIN, DIRK34, kernel_launches
    world, rank, local = _dist()
    torch.cuda.set_device(local)
    n_side, p, c = 48, 4, 1.0
    mesh = synth.hex_box(n_side)
    # the diffusion operator with beta = 0 (the compiled hexahedral set of p = 4)
    kprec = {"fp64": 0, "fp32": 1, "f32x2": 2}[args.krylov]
    pc = {"none": 0, "bjacobi": 1, "mlp": 0}[args.precond]
    g = LDG(mesh, p, CONVDIFF, CASE_ZERO, (c * c, 1.0, 0.0, 0.0, 0.0), gmres_m=30, newton_rtol=1e-8,
            gmres_rtol=1e-6, max_newton=10, max_restarts=50, precond=pc, krylov_precision=kprec)
    w0 = LDG(mesh, p, CONVDIFF, CASE_SINSIN, (1.0, 1.0, 0.0, 0.0, 0.0), gmres_m=1).interpolate(0.0)
    u = torch.zeros_like(w0)
    q = g.q(w0)
    w = w0.clone()
    dt = 0.5 / n_side / c
    stream = torch.cuda.current_stream()
    clocks = ClockSampler(local)
    clocks.start()
    t = 0.0
    for _ in range(args.warmup):
        g.wave_step(u, q, w, t=t, dt=dt, scheme=DIRK34)
        t += dt
    torch.cuda.synchronize()
    l0 = kernel_launches()
    reps = []
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        reps.append(g.wave_step(u, q, w, t=t, dt=dt, scheme=DIRK34))
        t += dt
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / args.steps
    launches = kernel_launches() - l0
    clk = clocks.stop()
    omega = c * math.pi * math.sqrt(3.0)
    err = float(torch.linalg.norm(w - w0 * math.cos(omega * t)) / torch.linalg.norm(w0 * math.cos(omega * t)))
    jv = sum(r["jv_calls"] for r in reps) / len(reps)
    n = g.n_dof
    line = {"metric": METRIC, "value": n / (ms * 1e-3) / 1e9, "unit": UNIT, "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WAVE_WORKLOAD, "n_dof": n, "dt": dt, "t_end": t,
                       "value_definition": "DOF of u x DIRK34 steps / time (each step three stage solves)",
                       "krylov_precision": args.krylov, "precond": ("none", "bjacobi")[pc],
                       "jv_calls_per_step": jv,
                       "gmres_iters_per_step": sum(r["gmres_iters"] for r in reps) / len(reps),
                       "w_rel_err_vs_standing_wave": err,
                       "l2": "not flushed: the state and the Krylov space (about 7 GB) exceed the 126 MB L2"},
            "roofline": None, "cpu_baseline": None, "e2e": None, "gpu_launches": int(launches), "clocks": clk}
    print(json.dumps(line), flush=True)


CYL_WORKLOAD = ("2D compressible Navier-Stokes flow past a cylinder (radius 0.5 at the origin, domain "
                "[-10,30]x[-10,10]), {E} curved quadrilaterals ({nr} advancing layers x {nt} around, first layer "
                "0.01, map degree 3, seeded node jitter, seed 7), p=3, Re={re:.1f} (uniform [100,1000], seed {rs}), "
                "Mach 0.2 free stream, no-slip adiabatic wall, BDF2 dt=0.1 from the free stream blended to rest "
                "at the wall (velocity x tanh((r-0.5)/0.1)), Newton-GMRES(30) to 1e-8 (FP64 residual)")


def cylinder_problem(LDG, mesh, re, forcing=0):
    """Far-field data: the uniform Mach 0.2 free stream. Initial state (both BDF2 levels):
    the free stream with its velocity scaled by tanh((r - 0.5) / 0.1), which meets the
    no-slip wall (an impulsive start, free stream up to the wall, is not a state the
    full-step Newton iteration reaches 1e-8 from in one dt = 0.1 step)."""
    from paper_2205_07824_b300.ldg import NS, CASE_CYLINDER, CASE_CYLINDER_START

    def make(p, kprec):
        return LDG(mesh, 3, NS, CASE_CYLINDER, (1.4, re, 0.72), gmres_m=30, newton_rtol=1e-8, gmres_rtol=1e-3,
                   krylov_precision=kprec, precond=p, newton_forcing=forcing)

    def init(g):
        g0 = LDG(mesh, 3, NS, CASE_CYLINDER_START, (1.4, re, 0.72))
        u0 = g0.interpolate(0.0)
        return u0, u0.clone()
    return dict(make=make, init=init, dt=0.1, n_elem=mesh.n_elem)


def run_cylinder_sweep(args):
    """Reynolds-number sweep: K cylinder instances (Re from seeds 0 .. K-1) on the same
    mesh, solved together per BDF2 step by the batched engine in one CUDA graph launch
    (FP32 Krylov J.v and block-Jacobi)."""
    import numpy as np
    import torch
    from paper_2205_07824_b300 import synth
    from paper_2205_07824_b300.ldg import LDG, Batch, NS, CASE_CYLINDER, CASE_CYLINDER_START, BDF2, kernel_launches

    world, rank, local = _dist()
    torch.cuda.set_device(local)
    K = args.cyl_sweep
    mesh = synth.cylinder_mesh(args.cyl_layers, args.cyl_around, 3, seed=7)
    res = [float(np.random.default_rng(args.re_seed + k).uniform(100.0, 1000.0)) for k in range(K)]
    mus = [(1.4, re, 0.72) for re in res]
    b = Batch([mesh] * K, [3] * K, NS, CASE_CYLINDER, mus, gmres_m=30, newton_rtol=1e-8, gmres_rtol=1e-3,
              krylov_precision=1, precond=1, newton_forcing=forcing_of(args))
    g0 = LDG(mesh, 3, NS, CASE_CYLINDER_START, mus[0])
    u0 = g0.interpolate(0.0)
    del g0
    un = u0.repeat(K)
    unm1 = un.clone()
    u = torch.empty_like(un)
    stream = torch.cuda.current_stream()
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")
    dt, t = 0.1, 0.0
    clocks = ClockSampler(local)
    times, reps_all = [], []
    l0 = None
    for k in range(args.warmup + args.steps):
        if k == args.warmup:
            clocks.start()
            l0 = kernel_launches()
        b.set_time(BDF2, t + dt, dt, un, unm1)
        u.copy_(un)
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        reps, _ = b.solve(u)
        e1.record(stream)
        torch.cuda.synchronize()
        unm1.copy_(un)
        un.copy_(u)
        t += dt
        if k >= args.warmup:
            times.append(e0.elapsed_time(e1))
            reps_all.append(reps)
    launches = kernel_launches() - l0
    clk = clocks.stop()
    bad = [r for reps in reps_all for r in reps if r["status"] != 0 or r["rfinal"] > 1e-8 * r["r0"]]
    assert not bad, bad[:2]
    jv_dofs = sum(b.n_dof[i] * reps[i]["jv_calls"] for reps in reps_all for i in range(K))
    total_ms, gdofs = aggregate(times, jv_dofs, world, rank)
    if rank == 0:
        per = [{"re": round(res[i], 1),
                "gmres_iters_per_step": sum(r[i]["gmres_iters"] for r in reps_all) / len(reps_all),
                "newton_iters_per_step": sum(r[i]["newton_iters"] for r in reps_all) / len(reps_all)}
               for i in range(K)]
        line = {"metric": METRIC, "value": gdofs, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f64+f32", "data": "synthetic",
                "config": {"linear_tolerance": linear_tolerance(args), "workload": f"Reynolds-number sweep of the cylinder flow: {K} instances (Re from seeds "
                                       f"{args.re_seed}..{args.re_seed + K - 1}) on the {mesh.n_elem}-element mesh, "
                                       "p=3, one batched Newton-GMRES per BDF2 step (dt=0.1) in one CUDA graph launch, "
                                       "FP32 Krylov J.v + block-Jacobi, each instance to 1e-8",
                           "n_dof_total": int(b.n_total), "instances": per,
                           "value_definition": "J.v applications of all instances x their DOF / timed step time",
                           "l2": "flushed (256 MiB write) before each timed step"},
                "roofline": None, "cpu_baseline": None, "e2e": None, "gpu_launches": int(launches), "clocks": clk}
        print(json.dumps(line), flush=True)


def run_cylinder(args):
    """The cylinder workload: time-to-1e-8 per BDF2 step for the plain FP64 block-Jacobi
    form, the mixed form with block-Jacobi, and the learned + mixed form (the MLP
    trained on the warm-up steps' block-Jacobi data), on the same seeds; the Krylov J.v
    kernel pair timed alone against its HBM roofline."""
    import numpy as np
    import torch
    from paper_2205_07824_b300 import synth
    from paper_2205_07824_b300.ldg import LDG, kernel_launches

    world, rank, local = _dist()
    torch.cuda.set_device(local)
    nr, nt = args.cyl_layers, args.cyl_around
    mesh = synth.cylinder_mesh(nr, nt, 3, seed=7)
    re = float(np.random.default_rng(args.re_seed + rank).uniform(100.0, 1000.0))
    prob = cylinder_problem(LDG, mesh, re, forcing_of(args))
    stream = torch.cuda.current_stream()
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")
    clocks = ClockSampler(local)
    clocks.start()
    forms = {}
    sols = {}
    headline = None
    all_forms = (("fp64_bjacobi", 0, 1), ("fp32_bjacobi", 1, 1), ("fp32_learned_distilled", 1, 2),
                 ("fp32_learned", 1, 3))
    want = args.cyl_forms.split(",")
    for name, kp, pc in [f for f in all_forms if f[0] in want]:
        g, u, times, tot, launches, t_end, train = run_mode(prob, kp, pc, args.steps, args.warmup, flush, stream,
                                                            kernel_launches)
        ms = sum(times) / args.steps
        forms[name] = {"ms_per_step": ms, "newton_iters_per_step": tot["newton"] / args.steps,
                       "gmres_iters_per_step": tot["gmres"] / args.steps,
                       "jv_applications_per_step": tot["jv"] / args.steps, "pc_fallbacks": tot["pc_fallbacks"],
                       "jv_gdofs": g.n_dof * tot["jv"] / (sum(times) * 1e-3) / 1e9, "gpu_launches": int(launches)}
        if train:
            forms[name]["learned_pc_training"] = train
        sols[name] = u.clone()
        headline = (g, u, times, tot, launches)   # the last form run is the headline
    clk = clocks.stop()
    ref = sols.get("fp64_bjacobi", next(iter(sols.values())))
    base_ms = forms.get("fp64_bjacobi", next(iter(forms.values())))["ms_per_step"]
    for name in forms:
        forms[name]["solution_rel_diff_vs_fp64_bjacobi"] = float(torch.linalg.norm(sols[name] - ref) /
                                                                 torch.linalg.norm(ref))
        forms[name]["speedup_vs_fp64_bjacobi"] = base_ms / forms[name]["ms_per_step"]
    g, u, times, tot, launches = headline
    n = g.n_dof
    # the Krylov J.v as the solver runs it (q(u) of the step's residual reused), FP32 arithmetic
    v = torch.randn(n, dtype=torch.float64, device="cuda", generator=torch.Generator("cuda").manual_seed(1))
    jv = torch.empty_like(v)
    g.residual(u)
    jvt = {}
    for kp in (1, 0):
        jvt[kp] = graph_time_ms(g, lambda: g.jvp_after_residual(kp, u, v, jv), args.jv_reps)
    jv32 = g.jvp_after_residual(1, u, v)
    jv64 = g.jvp_after_residual(0, u, v)
    jv_err = float(torch.linalg.norm(jv32 - jv64) / torch.linalg.norm(jv64))
    # algorithmic bytes per FP32 J.v: the FP32 copies of u and q(u) (1 + 2 per DOF, 4 B),
    # the FP64 direction v (8 B), Q v written and read in FP32 (2 + 2, 4 B) and J.v written
    # in FP64 (8 B): 44 B per DOF; plus the curved-geometry records the two kernels read in
    # FP32: per-point metrics twice and the element mass inverse once
    npe = g.n_pe
    nq1, nf = 5, 4
    geo_rec = nq1 * nq1 * 5 + nf * nq1 * 3
    geo_bytes = (2 * geo_rec + npe * npe) * 4 * mesh.n_elem
    b_alg = 44.0 * n + geo_bytes
    hbm = None
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            hbm = float(json.load(f)["hbm_gbs"])
        peak_src = "MEASURED_PEAKS.json hbm_gbs (of measured)"
    except Exception:
        hbm, peak_src = 6400.0, "fallback 6.4 TB/s (of fallback)"
    achieved = b_alg / (jvt[1] * 1e-3) / 1e9
    # DRAM traffic of the pair per DOF from one ncu capture of the same kernels on the
    # 1/16-scaled cylinder mesh (2,500 elements, 160,000 DOF), scaled by the DOF count
    # (traffic grows with the elements)
    traffic = (6.491392e6 + 1280 + 5.785088e6) / 160000.0 * n
    roofline = {"bound": "hbm", "unit": "GB/s", "achieved": achieved, "peak": hbm, "frac": achieved / hbm,
                "traffic": traffic, "traffic_source": "ncu dram__bytes_read.sum + dram__bytes_write.sum of the pair "
                                                      "on the 2,500-element mesh, scaled by DOF (its writes stay in "
                                                      "L2 in that capture)",
                "peak_source": peak_src,
                "kernel": "k_qstage_curved<CurvedQuadEl<3,5>, NSModel, MODE_HOM, float> + "
                          "k_residual<CurvedQuadEl<3,5>, NSModel, MODE_JV, float>",
                "launch_pair_ms": jvt[1], "fp64_pair_ms": jvt[0], "bytes_per_jv": b_alg,
                "bytes_definition": "44 B/DOF state traffic (FP32 u and q(u), FP64 v, FP32 Q v written and read, "
                                    "FP64 J.v) + FP32 curved metrics (read by both kernels) and element mass "
                                    "inverses",
                "jv_gdofs_kernel_fp32": n / (jvt[1] * 1e-3) / 1e9, "jv_gdofs_kernel_fp64": n / (jvt[0] * 1e-3) / 1e9,
                "jv_fp32_rel_err_vs_fp64": jv_err}
    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        import oracle
        o = oracle.Oracle(mesh, 3, oracle.NS, oracle.CASE_CYLINDER, (1.4, re, 0.72))
        un = o.interpolate()
        o.set_time(2, 0.1, 0.1, un, un)
        uh, vh = u.cpu().numpy(), v.cpu().numpy()
        elems = np.arange(0, mesh.n_elem, 40)
        calls, t0 = 0, time.perf_counter()
        while True:
            o.jvp_some(uh, vh, elems)
            calls += 1
            el = time.perf_counter() - t0
            if el > 12.0 or calls >= 20:
                break
        dofs = len(elems) * o.npe * o.ncu * calls
        cpu = {"value": dofs / el / 1e9, "unit": UNIT, "cores": 1, "kind": "oracle",
               "sample": f"{calls} oracle J.v evaluations on every 40th element ({len(elems)} elements, their q "
                         f"neighbourhoods included), {el:.1f} s single-threaded"}
    total_ms, gdofs = aggregate(times, n * tot["jv"], world, rank)
    if rank == 0:
        line = {"metric": METRIC, "value": gdofs, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f64+f32", "data": "synthetic",
                "config": {"linear_tolerance": linear_tolerance(args), "workload": CYL_WORKLOAD.format(E=mesh.n_elem, nr=nr, nt=nt, re=re, rs=args.re_seed),
                           "n_dof": int(n), "n_elem": int(mesh.n_elem),
                           "value_definition": "learned + mixed form: J.v applications of the whole solve x DOF / "
                                               "timed step time",
                           "forms": forms, "headline_form": list(forms)[-1],
                           "l2": "flushed (256 MiB write) before each timed step, outside its event window",
                           "parallelism": f"{world} independent instance(s), one per GPU"},
                "roofline": roofline, "cpu_baseline": cpu, "e2e": None, "gpu_launches": int(launches),
                "clocks": clk}
        print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-fp64-baseline", action="store_true")
    ap.add_argument("--jv-reps", type=int, default=50)
    ap.add_argument("--precond", default="bjacobi", choices=["none", "bjacobi", "mlp"],
                    help="block-Jacobi: exact element-diagonal blocks, rebuilt once per implicit step; "
                         "mlp: the learned per-element preconditioner trained on the warm-up steps")
    ap.add_argument("--krylov", default="fp32", choices=["fp64", "fp32", "f32x2", "tc_bf16x3", "tc_bf16"],
                    help="arithmetic of the J.v inside GMRES (Newton residual and Arnoldi stay FP64)")
    ap.add_argument("--forcing", default="last", choices=["fixed", "last"],
                    help="Newton-GMRES workloads (vortex, batch, cylinder): linear tolerance of each Newton "
                         "step, gmres_rtol throughout (fixed) or max(gmres_rtol, 1/2 newton_rtol ||R0|| / ||Rk||) "
                         "(last; every form compared)")
    ap.add_argument("--no-lagged-pc", action="store_true")
    ap.add_argument("--no-pair-basis", action="store_true")
    ap.add_argument("--pc-reuse", type=int, default=1,
                    help="vortex: build the block-Jacobi blocks every K implicit steps (every form compared)")
    ap.add_argument("--host-loops", action="store_true",
                    help="run the solver's Newton / restart / Arnoldi loops from the host instead of the CUDA "
                         "graph's WHILE nodes (same kernels; for profilers that do not follow graph nodes)")
    ap.add_argument("--no-solve", action="store_true", help="jv: skip the vortex time-to-1e-8 comparison")
    ap.add_argument("--workload", default="jv",
                    choices=["jv", "jvprobe", "vortex", "batch", "hex", "tri", "cylinder", "tet", "wave", "tcprobe",
                             "mlpprobe"],
                    help="jv (default): the FP64 J.v of 48^3 p=4 convection-diffusion; jvprobe: its J.v "
                         "applications alone, for profilers; "
                         "vortex: the 64x64 p=3 Euler BDF2 step; batch: 256 parametrised convection-diffusion "
                         "solves in one graph launch; hex: the 48^3 convection-diffusion J.v sweep p=1..6; "
                         "tri: the same sweep on 131,072 triangles; "
                         "cylinder: Navier-Stokes past a cylinder on 40,000 curved quads, learned + mixed vs "
                         "plain FP64 block-Jacobi; tet: Table 3's Poisson problem on tetrahedra, 1/n = 32, p = 3; "
                         "mlpprobe: the learned preconditioner's tensor-core inference on 65,536 rows; "
                         "wave: DIRK34 steps of the wave model on 48^3 hexahedra, p = 4; tcprobe: the Euler J.v "
                         "in FP64, FP32 and with tensor-core contractions on square vortex meshes")
    ap.add_argument("--tc-sides", default="64,128,256,512", help="tcprobe: square mesh sides")
    ap.add_argument("--tet-n", type=int, default=32, help="tet: cubes per side (Table 3's 1/n)")
    ap.add_argument("--tet-p", type=int, default=3, help="tet: polynomial order")
    ap.add_argument("--cyl-layers", type=int, default=100, help="cylinder mesh: layers across the domain")
    ap.add_argument("--cyl-around", type=int, default=400, help="cylinder mesh: elements around the cylinder")
    ap.add_argument("--re-seed", type=int, default=0, help="cylinder: seed of the Reynolds-number draw")
    ap.add_argument("--cyl-sweep", type=int, default=1,
                    help="cylinder: K > 1 solves K Reynolds numbers together in one batched graph launch per step")
    ap.add_argument("--cyl-forms", default="fp64_bjacobi,fp32_bjacobi,fp32_learned",
                    help="cylinder: forms to run (the last one is the headline)")
    args = ap.parse_args()
    if args.host_loops:
        os.environ["LDG_SOLVER_HOST_LOOPS"] = "1"
    if args.impl == "reference":
        run_reference(args)
        return
    if args.workload == "jv":
        run_jv(args)
        return
    if args.workload == "jvprobe":
        run_jv_probe(args)
        return
    if args.workload == "batch":
        run_batch(args)
        return
    if args.workload == "hex":
        run_hex(args)
        return
    if args.workload == "tri":
        run_tri(args)
        return
    if args.workload == "cylinder":
        if args.cyl_sweep > 1:
            run_cylinder_sweep(args)
        else:
            run_cylinder(args)
        return
    if args.workload == "tet":
        run_tet(args)
        return
    if args.workload == "wave":
        run_wave(args)
        return
    if args.workload == "tcprobe":
        run_tc_probe(args)
        return
    if args.workload == "mlpprobe":
        run_mlp_probe(args)
        return

    import numpy as np
    import torch
    import torch.distributed as dist
    from paper_2205_07824_b300 import synth
    from paper_2205_07824_b300.ldg import LDG, kernel_launches, BDF2

    world, rank, local = _dist()
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl")
    mesh = synth.quad_box(N_SIDE, hi=(10.0, 10.0), periodic=(True, True))
    stream = torch.cuda.current_stream()
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")   # 256 MiB > L2
    kprec = {"fp64": 0, "fp32": 1, "f32x2": 2, "tc_bf16x3": 3, "tc_bf16": 4}[args.krylov]
    pc = {"none": 0, "bjacobi": 1, "mlp": 2}[args.precond]

    if world > 1:
        dist.barrier()
    clocks = ClockSampler(local)
    clocks.start()
    forcing = forcing_of(args)
    prob = vortex_problem(LDG, mesh, forcing, max(1, args.pc_reuse))
    g, u, times, tot, launches, t_end, train = run_mode(prob, kprec, pc, args.steps, args.warmup, flush, stream,
                                                        kernel_launches)
    if world > 1:
        dist.barrier()
    clk = clocks.stop()
    n = g.n_dof
    total_ms, gdofs = aggregate(times, n * tot["jv"], world, rank)
    ms_per_step = total_ms / args.steps

    # the plain FP64 block-Jacobi form on the same box, same steps
    base = None
    if not args.no_fp64_baseline and (kprec, pc) != (0, 1):
        gb, ub, tb, totb, _, _, _ = run_mode(prob, 0, 1, args.steps, args.warmup, flush, stream, kernel_launches)
        base = {"form": "FP64 Krylov J.v + block-Jacobi", "ms_per_step": sum(tb) / args.steps,
                "gmres_iters_per_step": totb["gmres"] / args.steps,
                "solution_rel_diff_vs_headline": float(torch.linalg.norm(ub - u) / torch.linalg.norm(ub))}
        base["speedup_headline_vs_fp64_bjacobi"] = base["ms_per_step"] / ms_per_step
        del gb

    # the same form with the block-Jacobi blocks lagged over LAGGED_PC_REUSE implicit steps:
    # faster steps with fewer J.v applications (block extraction), so it is reported beside
    # the headline instead of in it
    lagged = None
    if not args.no_lagged_pc and pc == 1 and args.pc_reuse <= 1:
        prob_lag = vortex_problem(LDG, mesh, forcing, LAGGED_PC_REUSE)
        gl, ul, tl, totl, _, _, _ = run_mode(prob_lag, kprec, 1, args.steps, args.warmup, flush, stream,
                                             kernel_launches)
        lagged = {"form": f"the headline form with the blocks built every {LAGGED_PC_REUSE} implicit steps "
                          f"(pc_reuse = {LAGGED_PC_REUSE})",
                  "ms_per_step": sum(tl) / args.steps, "gmres_iters_per_step": totl["gmres"] / args.steps,
                  "solution_rel_diff_vs_headline": float(torch.linalg.norm(ul - u) / torch.linalg.norm(u))}
        lagged["speedup_vs_headline"] = ms_per_step / lagged["ms_per_step"]
        del gl

    # the same form with Gram-Schmidt on (hi, lo) float pairs (emulated FP64, krylov_basis
    # = F32X2), reported beside the FP64-basis headline
    pair_basis = None
    if not args.no_pair_basis and args.pc_reuse <= 1:
        prob_ff = vortex_problem(LDG, mesh, forcing, 1, 1)
        gf, uf, tf, totf, _, _, _ = run_mode(prob_ff, kprec, pc, args.steps, args.warmup, flush, stream,
                                             kernel_launches)
        pair_basis = {"form": "the headline form with the Krylov basis and Gram-Schmidt sweeps on (hi, lo) float "
                              "pairs (about 48 significand bits, emulated FP64)",
                      "ms_per_step": sum(tf) / args.steps, "gmres_iters_per_step": totf["gmres"] / args.steps,
                      "solution_rel_diff_vs_headline": float(torch.linalg.norm(uf - u) / torch.linalg.norm(u))}
        pair_basis["speedup_vs_headline"] = ms_per_step / pair_basis["ms_per_step"]
        del gf

    # the Krylov J.v kernel alone (the dominant kernel), CUDA events on the launching stream
    v = torch.randn(n, dtype=torch.float64, device="cuda", generator=torch.Generator("cuda").manual_seed(1))
    jv = torch.empty_like(v)
    jv_ms = graph_time_ms(g, lambda: g.jvp_prec(kprec, u, v, jv), args.jv_reps)
    jv64 = g.jvp_prec(0, u, v)
    jv_err = float(torch.linalg.norm(jv - jv64) / torch.linalg.norm(jv64)) if kprec else 0.0
    if kprec >= 3:
        # tensor-core J.v: its MMA flops against the measured bf16 peak (the pointwise
        # fluxes between the MMA phases run on the CUDA cores and bound it)
        peaks = _peaks()
        passes = 3 if kprec == 3 else 1
        bf16 = float(peaks.get("bf16_tflops", 1800.0))
        achieved = TC_MMA_FLOP_PER_ELEM_P3 * passes * mesh.n_elem / (jv_ms * 1e-3) / 1e12
        roofline = {"bound": "tensor", "unit": "TFLOP/s", "achieved": achieved, "peak": bf16,
                    "frac": achieved / bf16, "traffic": None, "kernel": g.jv_kernels(kprec),
                    "timing": "CUDA graph of jv_reps back-to-back J.v launches, one replay timed with CUDA events",
                    "launch_ms": jv_ms, "jv_gdofs_kernel": n / (jv_ms * 1e-3) / 1e9,
                    "mma_flop_per_elem": TC_MMA_FLOP_PER_ELEM_P3 * passes,
                    "peak_source": "measured cuBLAS bf16 (burst)" if "bf16_tflops" in peaks else "fallback 1.8 PFLOP/s",
                    "jv_rel_err_vs_fp64": jv_err}
    fpe = JV_FLOP_PER_ELEM[min(kprec, 1)]
    achieved = fpe * mesh.n_elem / (jv_ms * 1e-3) / 1e12
    peak = FP32_PEAK_TFLOPS if kprec else FP64_PEAK_TFLOPS
    # DRAM bytes per launch of the FP32 kernel (tile 8) from one ncu capture inside the step:
    # the state is L2-resident
    traffic = (1.792e3 + 1.024e3) if kprec else None
    roofline = roofline if kprec >= 3 else {"bound": "alu", "unit": "TFLOP/s", "achieved": achieved, "peak": peak, "frac": achieved / peak,
                "traffic": traffic,
                "traffic_source": "ncu dram__bytes_read.sum + dram__bytes_write.sum of one launch (Tile<8>) inside "
                                  "the step; the 6.3 MB of state per launch come from L2" if kprec else None,
                "kernel": (f"k_residual<TensorEl<2,3,5>, EulerModel, MODE_JV, {'float' if kprec else 'double'}, "
                           f"Tile{g.get_tile()[0]}>"),
                "timing": "CUDA graph of jv_reps back-to-back J.v launches, one replay timed with CUDA events",
                "launch_ms": jv_ms, "jv_gdofs_kernel": n / (jv_ms * 1e-3) / 1e9,
                "flop_per_elem": fpe, "flop_source": "ncu thread-instruction counts (FMA x2 + ADD + MUL)",
                "peak_source": ("FP32 ALU: 148 SMs x 128 FMA/clk x 2 FLOP x 2.032 GHz (derived)" if kprec else
                                "FP64 ALU: 148 SMs x 2 FMA/clk x 2 FLOP x 2.032 GHz (derived)"),
                "jv_fp32_rel_err_vs_fp64": jv_err}

    # end to end through the public API with host buffers
    e2e = None
    if not args.no_e2e:
        h_un = torch.empty(n, dtype=torch.float64, pin_memory=True)
        h_unm1 = torch.empty(n, dtype=torch.float64, pin_memory=True)
        h_un.copy_(u)
        h_unm1.copy_(u)
        # the solution read back to pinned memory, like the inputs
        h_u_t = torch.empty(n, dtype=torch.float64, pin_memory=True)
        d_un, d_unm1, d_u = torch.empty_like(u), torch.empty_like(u), torch.empty_like(u)
        k2 = min(args.steps, 5)
        t_e2e, jv_e2e = 0.0, 0
        tt = t_end
        nloc = g.n_cu * g.n_pe
        for it in range(k2 + 1):          # the first (untimed) step takes the one-time costs
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            d_un.copy_(h_un, non_blocking=True)
            d_unm1.copy_(h_unm1, non_blocking=True)
            g.set_time(BDF2, tt + DT, DT, d_un, d_unm1)
            d_u.copy_(d_un)               # the initial guess is u^n, already on the device
            rep = g.newton_gmres(d_u)
            h_u_t.copy_(d_u)              # the solution back to the host (synchronous)
            if it > 0:
                t_e2e += time.perf_counter() - t0
                jv_e2e += rep["jv_calls"] + rep["pc_setups"] * nloc
            h_unm1.copy_(h_un)
            h_un.copy_(h_u_t)
            tt += DT
        e2e = {"value": n * jv_e2e / t_e2e / 1e9, "unit": UNIT, "h2d_bytes_per_step": 2 * 8 * n,
               "d2h_bytes_per_step": 8 * n, "steps": k2, "ms_per_step": t_e2e / k2 * 1e3,
               "note": "host u^n and u^{n-1} copied in (the initial guess is u^n on the device), "
                       "ldg_newton_gmres, the solution copied out, per step; host wall clock"}

    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        cpu = cpu_baseline_jv(u.cpu().numpy(), v.cpu().numpy())

    if rank == 0:
        line = {"metric": METRIC, "value": gdofs, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": {0: "f64", 1: "f64+f32", 3: "f64+bf16x3", 4: "f64+bf16"}[kprec],
                "data": "synthetic",
                "config": {"workload": WORKLOAD, "n_dof": int(n), "n_elem": int(mesh.n_elem),
                           "value_definition": "J.v applications of the whole solve (Arnoldi, true residual, "
                                               "block extraction) x DOF / timed step time",
                           "time_to_1e-8_ms_per_step": ms_per_step,
                           "newton_iters_per_step": tot["newton"] / args.steps,
                           "gmres_iters_per_step": tot["gmres"] / args.steps,
                           "jv_applications_per_step": tot["jv"] / args.steps,
                           "preconditioner": {0: "none",
                                              1: "block-Jacobi (exact element-diagonal blocks, built once per "
                                                 + ("implicit step)" if args.pc_reuse <= 1 else
                                                    f"{args.pc_reuse} implicit steps, at the first one's initial "
                                                    "guess)"),
                                              2: "learned per-element MLP (BF16 weights), block-Jacobi fallback"}[pc],
                           "pc_fallbacks": tot["pc_fallbacks"], "learned_pc_training": train,
                           "precision": "FP64 throughout" if kprec == 0 else
                           "Krylov J.v and preconditioner in FP32 arithmetic; Newton residual, Arnoldi, Givens, "
                           "vectors FP64",
                           "linear_tolerance": linear_tolerance(args),
                           "l2": "flushed (256 MiB write) before each timed step, outside its event window",
                           "parallelism": f"{world} independent instance(s), one per GPU",
                           "fp64_bjacobi_baseline": base, "lagged_block_jacobi": lagged,
                           "pair_basis_gram_schmidt": pair_basis},
                "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": int(launches),
                "clocks": clk}
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
