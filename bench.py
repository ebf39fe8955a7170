#!/usr/bin/env python3
"""Benchmark of the GB300 hypercube convolution (arXiv 1608.00206).

Metric: 3^D outputs per second (whole job, all ranks), with the dominant
kernel's achieved HBM bandwidth against the measured peak.  One step is one
pass of the whole method over the workload's inputs, which are resident in
HBM before the timed region starts.

Workloads (--workload):
  d20_int64  (default) D = 20 int64 exact, x, y iid uniform integers in
             [-1000, 1000]; z has 3^20 = 3.49e9 int64 outputs (27.9 GB)
  d16_fp64   D = 16 float64 probability hypercubes (Exponential(1) / sum)
  d16_mixed  the same inputs in float32, float-float interpolation
  d16_ff     the same inputs in float32, every value in float-float
  d10_int64  D = 10 int64, values in [-100, 100]
  batched    4096 float32 instances, D ~ U{6..14}, U[0,1) inputs; fused
             persistent launch + per-D grouped passes at the autotuned fusion
             depth, replayed from one CUDA graph
  fwdbwd     D = 18 float32, x, y, w iid N(0,1), loss = sum(w * z), forward
             plus the hand-written adjoint through torch.autograd

--impl reference times the CPU oracle (the plain C++ recurrence, all host
cores) on bounded samples of the same workload and prints the same JSON line
with "impl": "reference".
"""
from __future__ import annotations

import argparse
import hashlib
import glob
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "3^D outputs/s"
UNIT = "outputs/s"

WORKLOADS = {
    "d20_int64": "D=20 int64 exact single instance: x,y 2^20 iid uniform integers in "
                 "[-1000,1000]; z 3^20 int64 (27.9 GB)",
    "d16_fp64": "D=16 float64 probability hypercubes: x,y 2^16 iid Exponential(1) normalised "
                "to sum 1; z 3^16 float64",
    "d16_mixed": "D=16 float32 probability hypercubes, float32 evaluation and products, "
                 "float-float interpolation",
    "d16_ff": "D=16 float32 probability hypercubes, every value in float-float (two-sum "
              "evaluation, FMA two-product, two-sum interpolation)",
    "d10_int64": "D=10 int64 exact: x,y 1024 iid uniform integers in [-100,100]",
    "d18_fp32": "D=18 float32: x,y 2^18 iid U[0,1); z 3^18 float32",
    "batched": "4096 float32 instances, D iid uniform in 6..14, x,y iid U[0,1); fused "
               "persistent launch and per-D grouped passes at the autotuned fusion depth, "
               "replayed from one CUDA graph",
    "fwdbwd": "D=18 float32, x,y,w iid N(0,1), loss = sum(w*z) (torch.dot), forward + "
              "hand-written adjoint via torch.autograd",
    "maxconv": "D=14 max-convolution of bounded non-negative integers: x,y 2^14 iid uniform "
               "integers in [0,3]; p-norm ring (sums of p-th powers in limbs on 4 extra "
               "carry-free axes, one 18-axis int64 convolution, nearest-integer roots); z 3^14 "
               "int64",
}
DEFAULT_STEPS = {"d20_int64": 30, "d16_fp64": 30, "d16_mixed": 50, "d16_ff": 50, "d10_int64": 200,
                 "d18_fp32": 50, "batched": 20, "fwdbwd": 30, "maxconv": 30}
SINGLE = ("d20_int64", "d16_fp64", "d16_mixed", "d16_ff", "d10_int64", "d18_fp32")


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


# FP64 throughput of GB300 from the nominal dense FP64 rate (1.25 TFLOP/s,
# counting a fused multiply-add as two): 0.625e12 FP64 add, subtract or
# multiply instructions per second -- context only; the roofline's FP64 peak
# is measured on the device by hc_probe_alu_rate (see _fp64_peak).
FP64_OPS_NOMINAL = 0.625e12
_FP64_MEASURED = []


def _fp64_peak():
    """(ops/s, source): FP64 add/multiply rate measured on this device by the
    library's probe kernel (independent add/multiply chains, CUDA events),
    once per process; the nominal rate if the probe fails."""
    if not _FP64_MEASURED:
        import ctypes

        import torch

        from paper_1608_00206_gb300 import _lib
        v = ctypes.c_double()
        rc = _lib.lib().hc_probe_alu_rate(_lib.HC_FP64, ctypes.byref(v),
                                          torch.cuda.current_stream().cuda_stream)
        _FP64_MEASURED.append(float(v.value) if rc == 0 and v.value > 0 else None)
    m = _FP64_MEASURED[0]
    if m is None:
        return FP64_OPS_NOMINAL, "nominal GB300 FP64 rate (1.25 TFLOP/s with FMA = 2)"
    return m, ("measured FP64 add/multiply rate of this device (hc_probe_alu_rate: "
               "independent __dadd_rn/__dmul_rn chains, CUDA events)")
_FP32_MEASURED = []
FP32_OPS_NOMINAL = 2070e6 * 152 * 128  # 128 binary32 add/multiply lanes per SM at 2070 MHz


def _fp32_peak():
    """(ops/s, source): binary32 add/multiply rate measured by the library's
    probe kernel, once per process (the roof of the float-float kernels)."""
    if not _FP32_MEASURED:
        import ctypes

        import torch

        from paper_1608_00206_gb300 import _lib
        v = ctypes.c_double()
        rc = _lib.lib().hc_probe_alu_rate(_lib.HC_FP32, ctypes.byref(v),
                                          torch.cuda.current_stream().cuda_stream)
        _FP32_MEASURED.append(float(v.value) if rc == 0 and v.value > 0 else None)
    m = _FP32_MEASURED[0]
    if m is None:
        return FP32_OPS_NOMINAL, "nominal GB300 binary32 add/multiply rate"
    return m, ("measured binary32 add/multiply rate of this device (hc_probe_alu_rate: "
               "independent __fadd_rn/__fmul_rn chains, CUDA events)")


L2_BYTES = 129 << 20  # GB300 L2 (rounded up)
L2_FLUSH_BYTES = 256 << 20


def _src_hash():
    h = hashlib.sha256()
    for f in sorted(glob.glob(os.path.join(ROOT, "paper_1608_00206_gb300", "csrc", "*"))):
        with open(f, "rb") as fh:
            h.update(os.path.basename(f).encode())
            h.update(fh.read())
    return h.hexdigest()[:12]


def _traffic_from_profiles(workload, kernel):
    """dram bytes per launch from profiles/traffic.txt when captured on the
    current kernel sources (same source hash); None otherwise."""
    path = os.path.join(ROOT, "profiles", "traffic.txt")
    if not os.path.exists(path):
        return None
    src = _src_hash()
    with open(path) as f:
        for line in f:
            parts = line.split()
            if len(parts) >= 4 and not line.startswith("#"):
                if parts[0] == workload and parts[1] == kernel and parts[3] == src:
                    return float(parts[2])
    return None


# ------------------------------------------------------------------ clocks


class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index):
        self.proc = None
        self.out = None
        try:
            import torch
            uuid = str(torch.cuda.get_device_properties(device_index).uuid)
            self.sel = uuid if uuid.startswith("GPU-") else "GPU-" + uuid
        except Exception:
            self.sel = None

    def start(self):
        try:
            cmd = ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                   "-lms", "100"]
            if self.sel:
                cmd += ["-i", self.sel]
            self.proc = subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.DEVNULL,
                                         text=True)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except Exception:
            self.proc.kill()
            out, _ = self.proc.communicate()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.splitlines():
            p = [v.strip() for v in line.split(",")]
            if len(p) < 7:
                continue
            try:
                sm.append(float(p[0]))
                mx.append(float(p[1]))
            except ValueError:
                continue
            for n, v in zip(names, p[3:7]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx),
                "reasons": sorted(reasons), "samples": len(sm)}


# --------------------------------------------------------------- workloads


class Workload:
    """Device-resident inputs, a step function and the bookkeeping for one
    workload."""

    def __init__(self, name, dev, rank=0, D_override=None, instances=4096):
        import numpy as np
        import torch

        import paper_1608_00206_gb300 as hc
        from paper_1608_00206_gb300 import inputs

        self.name = name
        self.dev = dev
        self.D_override = D_override
        self.sched = {}
        self.hc = hc
        self.torch = torch
        seed = 1000 + rank
        self.graph = None
        if name in ("d20_int64", "d10_int64"):
            D = D_override or (20 if name == "d20_int64" else 10)
            r = 1000 if name == "d20_int64" else 100
            x, y = inputs.uniform_int_pair(D, -r, r, seed)
            self._single(D, x, y, torch.int64, mixed=False)
            self.dtype = "int64"
        elif name == "d18_fp32":
            D = D_override or 18
            x, y = inputs.uniform01_pair(D, seed)
            self._single(D, x, y, torch.float32, mixed=False)
            self.dtype = "f32"
        elif name in ("d16_fp64", "d16_mixed", "d16_ff"):
            D = D_override or 16
            x, y = inputs.prob_exponential_pair(D, seed)
            if name != "d16_fp64":
                x, y = x.astype(np.float32), y.astype(np.float32)
            self._single(D, x, y, torch.float64 if name == "d16_fp64" else torch.float32,
                         mixed={"d16_mixed": True, "d16_ff": "ff"}.get(name, False))
            self.dtype = _dtype_name(name)
        elif name == "batched":
            dims = inputs.batched_dims(instances, 6, 14, seed)
            pairs = inputs.batched_uniform01(dims, seed + 1)
            self.dims = [int(d) for d in dims]
            self.host_pairs = pairs
            self.xs = [torch.from_numpy(x).to(dev) for x, _ in pairs]
            self.ys = [torch.from_numpy(y).to(dev) for _, y in pairs]
            # fusion depth (fused persistent launch vs per-D grouped passes)
            # picked by the batched autotuner, outside the timed region
            self.batch = hc.BatchedConv(self.xs, self.ys, fused_max_d="tune")
            self.batch.capture()
            self.outputs = sum(3 ** d for d in self.dims)
            self.alg_bytes = sum(4 * (3 ** d + 2 * 2 ** d) for d in self.dims)
            self.dtype = "f32"
            self.D = None
        elif name == "maxconv":
            D = D_override or 14
            vmax = 3
            x, y = inputs.uniform_int_pair(D, 0, vmax, seed)
            self.D = D
            self.vmax = vmax
            self.plan = hc.maxconv_plan(D, vmax)
            self.conv_D = D + self.plan["e"]
            self.host = (x, y)
            self.x = torch.from_numpy(x).to(dev)
            self.y = torch.from_numpy(y).to(dev)
            self.z = torch.empty(3 ** D, dtype=torch.int64, device=dev)
            nb = hc.maxconv_workspace_size(D, vmax)
            self.ws = torch.empty(nb, dtype=torch.uint8, device=dev)
            self.outputs = 3 ** D
            # the result needs x, y read and z written once
            self.alg_bytes = 8 * (3 ** D + 2 * 2 ** D)
            self.dtype = "int64"
        elif name == "fwdbwd":
            D = D_override or 18
            self.D = D
            x = inputs.normal(1 << D, seed, np.float32)
            y = inputs.normal(1 << D, seed + 1, np.float32)
            w = inputs.normal(3 ** D, seed + 2, np.float32)
            self.host = (x, y, w)
            self.x = torch.from_numpy(x).to(dev).requires_grad_()
            self.y = torch.from_numpy(y).to(dev).requires_grad_()
            self.w = torch.from_numpy(w).to(dev)
            self.outputs = 3 ** D
            # forward writes z (3^D), backward reads dz (3^D); inputs and grads 2^D each
            self.alg_bytes = 4 * (2 * 3 ** D + 4 * 2 ** D)
            self.dtype = "f32"
        else:
            raise ValueError(name)

    def _single(self, D, x, y, tdtype, mixed):
        torch = self.torch
        self.D = D
        self.mixed = mixed
        self.host = (x, y)
        self.x = torch.from_numpy(x).to(self.dev)
        self.y = torch.from_numpy(y).to(self.dev)
        self.z = torch.empty(3 ** D, dtype=tdtype, device=self.dev)
        nb = self.hc.workspace_size(D, tdtype, mixed)
        self.ws = torch.empty(max(nb, 256), dtype=torch.uint8, device=self.dev)
        self.outputs = 3 ** D
        s = x.itemsize
        self.alg_bytes = 3 ** D * s + 2 * 2 ** D * s

    def use_graph(self):
        """Capture one convolution in a CUDA graph (for a launch-bound small
        problem: the host's per-call overhead would otherwise dominate)."""
        torch = self.torch
        self.eager_step()
        torch.cuda.synchronize(self.dev)
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, capture_error_mode="thread_local"):
            self.eager_step()
        self.graph = g

    def eager_step(self):
        self.hc.convolve(self.x, self.y, out=self.z, mixed=self.mixed, workspace=self.ws,
                         **self.sched)

    def step(self):
        if self.name == "batched":
            self.batch.replay()
        elif self.graph is not None:
            self.graph.replay()
        elif self.name == "maxconv":
            self.hc.maxconv(self.x, self.y, self.vmax, out=self.z, workspace=self.ws)
        elif self.name == "fwdbwd":
            self.x.grad = None
            self.y.grad = None
            # sum(w * z) as one fused reduction (no 3^D temporary)
            loss = self.torch.dot(self.w, self.hc.hypercube_conv(self.x, self.y))
            loss.backward()
        else:
            self.hc.convolve(self.x, self.y, out=self.z, mixed=self.mixed, workspace=self.ws,
                             **self.sched)

    def schedule_geometry(self):
        """(kind, C, m, ap, ev) of the schedule the single-instance step runs."""
        import ctypes

        from paper_1608_00206_gb300 import _lib
        code = {"d20_int64": 0, "d10_int64": 0, "d16_fp64": 1, "d18_fp32": 2,
                "d16_mixed": 3, "d16_ff": 4, "maxconv": 0}[self.name]
        # the max-convolution's own convolution has D + e axes
        Dc = getattr(self, "conv_D", self.D)
        cmax = 9 if code == 2 else 8
        if self.sched.get("lowmem"):
            # leaves of D - top axes on the whole-array-pass plan
            C = min(self.sched.get("c") or 8, Dc - self.sched["top"])
            return 1, C, 0, Dc - C, Dc - C
        if self.sched.get("top"):
            C = min(self.sched.get("c") or 8, Dc - self.sched["top"])
            return 4, C, self.sched["top"], Dc - self.sched["top"] - C, 0
        if self.sched:
            kind = (3 if self.sched.get("bulk") else 2) if "m" in self.sched else 1
            c, k = self.sched.get("c", 0), self.sched.get("m", self.sched.get("kmax", 0))
        else:
            s = _lib.hc_schedule()
            _lib.lib().hc_get_default_schedule(Dc, code, ctypes.byref(s))
            kind, c, k = s.kind, s.c, s.k
            if kind == 6:
                kind = 1  # padded whole-array passes: the same geometry
            if kind in (4, 5):  # hybrid / low-workspace defaults (int64)
                C = min(c or 8, Dc - s.top)
                if kind == 5:
                    return 1, C, 0, Dc - C, Dc - C
                return 4, C, s.top, Dc - s.top - C, 0
        C = min(c or cmax, Dc)
        if kind == 1:
            return kind, C, 0, Dc - C, Dc - C
        m = min(Dc - C, k or 6)
        ap = Dc - C - m
        return kind, C, m, ap, ap + (m if kind == 3 else max(m - 3, 0))

    # per-kernel algorithmic bytes (or FP64 operations) per launch
    def kernel_alg(self, kname, launches_per_step):
        D = getattr(self, "conv_D", self.D)
        if self.name == "batched":
            return self._batched_bytes(kname) / max(launches_per_step, 1), "hbm"
        if kname == "maxconv_root":
            # read the 3^(D+e) convolution once, write the 3^D maxima
            return 8 * (3 ** D + 3 ** self.D), "hbm"
        if kname == "maxconv_spread":
            # read x, y; write the two limb cubes of 2^(D+e) each
            return 8 * (2 * 2 ** self.D + 2 * 2 ** D), "hbm"
        s = 8 if self.name in ("d20_int64", "d10_int64", "d16_fp64", "d16_ff", "maxconv") else 4
        sw = 8 if self.name in ("d16_mixed", "d16_ff") else s
        if kname in ("chunk", "slab"):
            kind, C, m, ap, ev = self.schedule_geometry()
            if self.name in ("d16_mixed", "d16_ff") and kname == "slab":
                # binary32 operations: per tile the evaluation of both
                # operands on C axes (3^C - 2^C additions each: 1 operation
                # binary32, 11 float-float), 3^C products (1, or 9 for the
                # float-float product), per unit the interpolation of its
                # C + m axes (a third of the elements per axis are middles,
                # each two float-float subtractions of 11 operations)
                ea, mu = (1, 1) if self.name == "d16_mixed" else (11, 9)
                tile = 2 * (3 ** C - 2 ** C) * ea + 3 ** C * mu
                interp = (C + m) * 3 ** (C + m - 1) * 22
                return 3 ** ap * (3 ** m * tile + interp), "alu32"
            if self.name == "d16_fp64":
                tile = 2 * (3 ** C - 2 ** C) + 3 ** C + 2 * C * 3 ** (C - 1)
                return 3 ** ap * (3 ** m * tile + 2 * m * 3 ** (C + m - 1)), "alu"
            # read the operands evaluated on ev axes, write the 3^D intermediate once
            return 2 * 3 ** ev * 2 ** (D - ev) * s + 3 ** D * sw, "hbm"
        if kname == "eval_pass" and self.name != "fwdbwd":
            # whole-array evaluation passes of <= 3 axes over the ev outer
            # axes: each reads and writes both operands
            _, _, _, _, ev = self.schedule_geometry()
            total, d0 = 0, 0
            while d0 < ev:
                k = min(3, ev - d0)
                total += 2 * s * (3 ** d0 * 2 ** (D - d0) + 3 ** (d0 + k) * 2 ** (D - d0 - k))
                d0 += k
            return total / max(launches_per_step, 1), "hbm"
        if self.name == "d16_fp64":
            return self._fp64_ops(kname, launches_per_step), "alu"
        if kname in ("interp_pass", "interp_t_pass"):
            return 2 * 3 ** D * sw, "hbm"  # read and write the whole 3^D array
        if kname == "hybrid_tile":
            # write the 3^D outputs; read a pair of rows per sub-cube pair:
            # 4^top pairs of top strings x 3^a middle rows of 2^C elements
            _, C, top, a, _ = self.schedule_geometry()
            return 3 ** D * sw + 2 * 4 ** top * 3 ** a * 2 ** C * s, "hbm"
        if kname in ("tile_conv", "tile_adj"):
            C = min(D, 9 if (s == 4 and sw == 4 and kname == "tile_conv") else 8)
            a = D - C
            return 3 ** D * sw + 2 * 3 ** a * 2 ** C * s, "hbm"
        return None, "hbm"

    def _batched_bytes(self, kname):
        """Algorithmic bytes per step of one kind of batched kernel: the fused
        launch reads x, y and writes z of its instances; the grouped tile
        launches write each grouped instance's 3^D outputs and read its
        operands evaluated on the a outer axes; the grouped interpolation
        passes read and write the 3^D array of every instance with a > 0."""
        fm = max(self.batch.fused_max_d, 0)

        def tile_axes(d):
            return d if d <= 8 else (8 if d <= 14 else 9)
        fused = [d for d in self.dims if d <= fm]
        grouped = [d for d in self.dims if d > fm]
        if kname == "batched":
            return sum(4 * (3 ** d + 2 * 2 ** d) for d in fused)
        if kname == "batched_tile":
            return sum(4 * 3 ** d + 2 * 4 * 3 ** (d - tile_axes(d)) * 2 ** tile_axes(d)
                       for d in grouped)
        if kname == "batched_interp":
            return sum(2 * 4 * 3 ** d for d in grouped if d > tile_axes(d))
        if kname in ("batched_eval", "eval_pass"):
            return sum(4 * 2 * (2 ** d + 3 ** (d - tile_axes(d)) * 2 ** tile_axes(d))
                       for d in grouped if d > tile_axes(d))
        return 0

    def _fp64_ops(self, kname, lps):
        D = self.D
        C = min(D, 8)
        a = D - C
        if kname == "tile_conv":
            # per tile: evaluation of both operands on C axes, 3^C products,
            # interpolation of C axes (2 subtractions per 3 outputs per axis)
            per_tile = 2 * (3 ** C - 2 ** C) + 3 ** C + 2 * C * 3 ** (C - 1)
            return 3 ** a * per_tile
        if kname == "interp_pass":
            k = a / max(1, lps)
            return 2 * k * 3 ** (D - 1)
        return None


def _time_steps(wl, steps, warmup, dist):
    import torch

    from paper_1608_00206_gb300 import _lib

    for _ in range(warmup):
        wl.step()
    torch.cuda.synchronize()
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    _lib.profile_collect()  # drop anything recorded so far
    _lib.lib().hc_profile_enable(1)
    clocks = ClockSampler(wl.dev.index or 0)
    clocks.start()
    time.sleep(0.3)  # let the sampler start before the timed region
    stream = torch.cuda.current_stream(wl.dev)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    graph_events = []
    # A working set below L2 would stay resident from one step to the next:
    # flush L2 between steps (outside the per-step events) and time the steps
    # by their own events.
    flush = (torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=wl.dev)
             if wl.alg_bytes < L2_BYTES else None)
    e0.record(stream)
    for _ in range(steps):
        if flush is not None:
            flush.fill_(1)
        if wl.name == "batched" or wl.graph is not None or flush is not None:
            # the tracer does not see inside graph replays, so time each replay
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            wl.step()
            b.record(stream)
            graph_events.append((a, b))
        else:
            wl.step()
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    if flush is not None:
        ms = sum(a.elapsed_time(b) for a, b in graph_events)
    _lib.lib().hc_profile_enable(0)
    clk = clocks.stop()
    prof = _lib.profile_collect()
    if graph_events and (wl.name == "batched" or wl.graph is not None):
        # The tracer does not see inside graph replays: the per-kernel split
        # comes from one eager launch of the same batch after the timed
        # region, scaled to the timed steps (the step time itself is the
        # replays' own, measured above).
        eager = None
        if wl.name != "batched":
            # a single convolution: capture it once more with the tracer's
            # event pairs inside the graph and replay that graph once, so
            # that each kernel's time is its own, without the host's launch
            # gaps of an eager call (which dominate steps of tens of us)
            try:
                _lib.lib().hc_profile_enable(1)
                g2 = torch.cuda.CUDAGraph()
                with torch.cuda.graph(g2, capture_error_mode="thread_local"):
                    wl.eager_step()
                _lib.lib().hc_profile_enable(0)
                g2.replay()
                torch.cuda.synchronize()
                eager = _lib.profile_collect()
                del g2
                if not eager or min(v[1] for v in eager.values()) <= 0.0:
                    eager = None  # no event timings from the replay: use an eager call
            except Exception:  # capture refused: fall back to one eager call
                _lib.lib().hc_profile_enable(0)
                _lib.profile_collect()
                eager = None
        if eager is None:
            _lib.lib().hc_profile_enable(1)
            if wl.name == "batched":
                wl.batch.launch()
            else:
                wl.eager_step()
            torch.cuda.synchronize()
            _lib.lib().hc_profile_enable(0)
            eager = _lib.profile_collect()
        prof = {k: (v[0] * steps, v[1] * steps) for k, v in eager.items()}
    ms = _max_over_ranks(ms, dist, wl.dev)
    torch.cuda.synchronize()
    return ms, prof, clk


def _max_over_ranks(ms, dist, device):
    """The slowest rank's time (every rank gets it), then a barrier; ms itself
    with one rank.  Replicas run the same work, so the whole job's throughput
    is world x per-rank work / this time."""
    if dist is None:
        return ms
    import torch
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.barrier()
    return float(t.item())


def _whole_job_value(world, outputs_per_step, steps, ms):
    """Outputs per second over all ranks for `steps` steps in `ms`."""
    return world * outputs_per_step * steps / (ms / 1e3)


def _comparisons(wl, ms_per_step):
    """The forms against the plain GPU method, timed after the main timed
    region with CUDA events (device-resident inputs): the batched launch
    against a per-instance loop of hc_convolve, forward+backward against the
    forward alone, mixed precision against plain float32."""
    import torch

    hc = wl.hc

    def timed(fn, reps=3):
        fn()
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        for _ in range(reps):
            fn()
        b.record()
        torch.cuda.synchronize()
        return a.elapsed_time(b) / reps

    if wl.name == "batched":
        outs = wl.batch.outs
        wss = {}
        for d in set(wl.dims):
            nb = hc.workspace_size(d, torch.float32)
            wss[d] = torch.empty(max(nb, 256), dtype=torch.uint8, device=wl.dev)

        def loop():
            for x, y, z, d in zip(wl.xs, wl.ys, outs, wl.dims):
                hc.convolve(x, y, out=z, workspace=wss[d])
        t = timed(loop)
        return {"per_instance_loop_ms": t, "batched_speedup_vs_loop": t / ms_per_step}
    if wl.name == "fwdbwd":
        x, y = wl.x.detach(), wl.y.detach()
        t = timed(lambda: hc.convolve(x, y), reps=5)
        return {"forward_only_ms": t, "fwdbwd_over_forward": ms_per_step / t}
    if wl.name == "d18_fp32" and wl.D == 18:
        # the hybrid schedule: 4 direct-form top axes leave one
        # 6-axis middle pass; its own rounding, so never a default
        nb = hc.workspace_size(wl.D, torch.float32, top=4, c=8, kmax=6, cols=32)
        ws = torch.empty(max(nb, 256), dtype=torch.uint8, device=wl.dev)
        z = torch.empty(3 ** wl.D, dtype=torch.float32, device=wl.dev)
        t = timed(lambda: hc.convolve(wl.x, wl.y, out=z, workspace=ws, top=4, c=8, kmax=6,
                                      cols=32), reps=10)
        return {"hybrid_top4_ms": t, "hybrid_over_default": t / ms_per_step}
    if wl.name == "maxconv":
        # the (sum) convolution of the same inputs, and of the D + e axes the
        # p-norm ring convolves
        z = torch.empty(3 ** wl.D, dtype=torch.int64, device=wl.dev)
        nb = hc.workspace_size(wl.D, torch.int64)
        ws = torch.empty(max(nb, 256), dtype=torch.uint8, device=wl.dev)
        t = timed(lambda: hc.convolve(wl.x, wl.y, out=z, workspace=ws), reps=10)
        return {"plain_int64_ms": t, "maxconv_over_plain_int64": ms_per_step / t,
                "p": wl.plan["p"], "limb_bits": wl.plan["b"], "limb_axes": wl.plan["e"],
                "limbs": wl.plan["L"], "convolution_axes": wl.conv_D}
    if wl.name in ("d16_mixed", "d16_ff"):
        z = torch.empty(3 ** wl.D, dtype=torch.float32, device=wl.dev)
        nb = hc.workspace_size(wl.D, torch.float32)
        ws = torch.empty(max(nb, 256), dtype=torch.uint8, device=wl.dev)
        t = timed(lambda: hc.convolve(wl.x, wl.y, out=z, workspace=ws), reps=10)
        key = "mixed" if wl.name == "d16_mixed" else "ff"
        out = {"plain_fp32_ms": t, f"{key}_over_plain_fp32": ms_per_step / t}
        if wl.name == "d16_ff":
            nbm = hc.workspace_size(wl.D, torch.float32, True)
            wsm = torch.empty(max(nbm, 256), dtype=torch.uint8, device=wl.dev)
            tm = timed(lambda: hc.convolve(wl.x, wl.y, out=z, mixed=True, workspace=wsm), reps=10)
            out.update({"mixed_ms": tm, "ff_over_mixed": ms_per_step / tm})
        return out
    return None


def _timed_host_steps(one, min_steps, warmup, min_seconds=1.0, max_steps=100):
    """Host wall-clock time of repeated synchronous end-to-end steps: at least
    min_steps and about min_seconds (one untimed step sizes the count)."""
    for _ in range(warmup):
        one()
    t0 = time.perf_counter()
    one()
    t1 = time.perf_counter() - t0
    steps = max(min_steps, min(max_steps, int(min_seconds / max(t1, 1e-6)) + 1))
    per = []
    for _ in range(steps):
        t0 = time.perf_counter()
        one()
        per.append(time.perf_counter() - t0)
    per.sort()
    _timed_host_steps.last = {"step_ms_median": 1e3 * per[len(per) // 2], "step_ms_min": 1e3 * per[0]}
    return steps, sum(per)


def _e2e(wl, steps=3, warmup=1):
    """Same metric through the public API with host (pinned) buffers: every
    step copies x, y to the device, convolves, and copies z back."""
    import torch

    hc = wl.hc
    if wl.name in ("batched", "fwdbwd", "maxconv"):
        return _e2e_other(wl, steps, warmup)
    x, y = wl.host
    xh = torch.from_numpy(x).pin_memory()
    yh = torch.from_numpy(y).pin_memory()
    zh = torch.empty(3 ** wl.D, dtype=xh.dtype, pin_memory=True)
    # the device-resident output is not needed here
    wl.z = None
    torch.cuda.empty_cache()
    def one():
        hc.convolve(xh, yh, out=zh, mixed=wl.mixed, workspace=wl.ws)

    steps, dt = _timed_host_steps(one, steps, warmup)
    return {"value": wl.outputs * steps / dt, "unit": UNIT, "steps": steps,
            **_timed_host_steps.last,
            "h2d_bytes_per_step": int(2 * x.nbytes), "d2h_bytes_per_step": int(zh.numel() * zh.element_size())}


def _e2e_other(wl, steps, warmup):
    import torch

    hc = wl.hc
    if wl.name == "batched":
        # the packed layout: all instances back to back in one page-locked
        # array per operand, one copy each way (BatchedConv.from_packed)
        import numpy as np

        xo, nx = hc.packed_offsets(wl.dims, torch.float32, 2)
        _, nz = hc.packed_offsets(wl.dims, torch.float32, 3)
        xa = np.zeros(nx, np.float32)
        ya = np.zeros(nx, np.float32)
        for o, (x, y) in zip(xo, wl.host_pairs):
            xa[o:o + x.size] = x
            ya[o:o + y.size] = y
        xh = torch.from_numpy(xa).pin_memory()
        yh = torch.from_numpy(ya).pin_memory()
        zh = torch.empty(nz, dtype=torch.float32, pin_memory=True)
        b = hc.BatchedConv.from_packed(torch.empty(nx, dtype=torch.float32, device=wl.dev),
                                       torch.empty(nx, dtype=torch.float32, device=wl.dev),
                                       wl.dims, fused_max_d=wl.batch.fused_max_d)
        b.capture()
        h2d = 2 * 4 * nx
        d2h = 4 * nz

        def one():
            b.run_host(xh, yh, zh)
    elif wl.name == "maxconv":
        x, y = wl.host
        xh, yh = (torch.from_numpy(a).pin_memory() for a in (x, y))
        zh = torch.empty(3 ** wl.D, dtype=torch.int64, pin_memory=True)
        h2d = x.nbytes + y.nbytes
        d2h = zh.numel() * 8

        def one():
            xd = xh.to(wl.dev, non_blocking=True)
            yd = yh.to(wl.dev, non_blocking=True)
            hc.maxconv(xd, yd, wl.vmax, out=wl.z, workspace=wl.ws)
            zh.copy_(wl.z, non_blocking=True)
            torch.cuda.synchronize(wl.dev)
    else:
        x, y, w = wl.host
        xh, yh, wh = (torch.from_numpy(a).pin_memory() for a in (x, y, w))
        gxh = torch.empty_like(xh).pin_memory()
        gyh = torch.empty_like(yh).pin_memory()
        h2d = x.nbytes + y.nbytes + w.nbytes
        d2h = x.nbytes + y.nbytes + 4

        def one():
            xd = xh.to(wl.dev, non_blocking=True).requires_grad_()
            yd = yh.to(wl.dev, non_blocking=True).requires_grad_()
            wd = wh.to(wl.dev, non_blocking=True)
            loss = torch.dot(wd, hc.hypercube_conv(xd, yd))
            loss.backward()
            gxh.copy_(xd.grad, non_blocking=True)
            gyh.copy_(yd.grad, non_blocking=True)
            loss.item()
    steps, dt = _timed_host_steps(one, steps, warmup)
    return {"value": wl.outputs * steps / dt, "unit": UNIT, "steps": steps, **_timed_host_steps.last,
            "h2d_bytes_per_step": int(h2d),
            "d2h_bytes_per_step": int(d2h)}


# ------------------------------------------------------------ CPU oracle


def _oracle_samples(name):
    """Bounded samples of the workload for the CPU oracle: a list of
    (description, callable returning the number of outputs computed)."""
    import numpy as np

    import oracle
    from paper_1608_00206_gb300 import inputs

    thr = os.cpu_count() or 1
    seed = 1000
    if name == "d20_int64":
        x, y = inputs.uniform_int_pair(20, -1000, 1000, seed)
        samples = []
        for d1 in (0, 2):
            for d2 in (0, 2):
                sel = ((d1 // 2) * 2 + (d2 // 2)) << 18
                xs, ys = x[sel:sel + (1 << 18)].copy(), y[sel:sel + (1 << 18)].copy()
                samples.append((lambda xs=xs, ys=ys: oracle.convolve(xs, ys, threads=thr).size))
        return ("slices z[d1,d2,:] (d1,d2 in {0,2}) of the D=20 problem: the 18-D recurrence on "
                "the matching sub-cubes, 3^18 outputs each", samples, thr)
    if name in ("d16_fp64", "d16_mixed", "d16_ff"):
        x, y = inputs.prob_exponential_pair(16, seed)
        if name != "d16_fp64":
            x32, y32 = x.astype(np.float32), y.astype(np.float32)
            fn = oracle.convolve_mixed if name == "d16_mixed" else oracle.convolve_ff
            f = lambda: fn(x32, y32).size  # noqa: E731
            return "the full D=16 problem (single thread)", [f], 1
        return "the full D=16 problem", [lambda: oracle.convolve(x, y, threads=thr).size], thr
    if name == "d18_fp32":
        x, y = inputs.uniform01_pair(18, seed)
        return "the full D=18 problem", [lambda: oracle.convolve(x, y, threads=thr).size], thr
    if name == "d10_int64":
        x, y = inputs.uniform_int_pair(10, -100, 100, seed)
        return "the full D=10 problem (single thread)", [lambda: oracle.convolve(x, y).size], 1
    if name == "batched":
        dims = inputs.batched_dims(4096, 6, 14, seed)
        pairs = inputs.batched_uniform01(dims, seed + 1)
        samples = []
        for lo in range(0, 4096, 256):
            chunk = pairs[lo:lo + 256]
            samples.append(lambda chunk=chunk: sum(oracle.convolve(a, b, threads=thr).size
                                                   for a, b in chunk))
        return "consecutive blocks of 256 of the 4096 instances", samples, thr
    if name == "fwdbwd":
        D = 18
        x = inputs.normal(1 << D, seed, np.float32)
        y = inputs.normal(1 << D, seed + 1, np.float32)
        w = inputs.normal(3 ** D, seed + 2, np.float32)

        def f():
            z = oracle.convolve(x, y, threads=thr)
            oracle.adjoint(w, x, y)
            return z.size
        return "the full D=18 forward (all cores) and adjoint (single thread)", [f], thr
    if name == "maxconv":
        x, y = inputs.uniform_int_pair(14, 0, 3, seed)
        return ("the full D=14 max-convolution from its definition (the oracle's pair loop, "
                "single thread)", [lambda: oracle.maxconv_brute(x, y).size], 1)
    raise ValueError(name)


def _cpu_baseline(name, budget_s=12.0):
    desc, samples, thr = _oracle_samples(name)
    outs, t = 0, 0.0
    i = 0
    while i < len(samples) and (t < budget_s or i == 0):
        t0 = time.perf_counter()
        outs += samples[i]()
        t += time.perf_counter() - t0
        i += 1
    return {"value": outs / t, "unit": UNIT, "cores": thr, "kind": "oracle",
            "sample": f"{i} of: {desc}; {t:.1f} s"}


def _reference_arm(args, rank, world):
    if rank != 0:
        return 0
    desc, samples, thr = _oracle_samples(args.workload)
    for i in range(args.warmup):
        samples[i % len(samples)]()
    outs, t = 0, 0.0
    for i in range(args.steps):
        t0 = time.perf_counter()
        outs += samples[i % len(samples)]()
        t += time.perf_counter() - t0
    v = outs / t
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": _dtype_name(args.workload), "data": "synthetic",
            "config": {"workload": WORKLOADS[args.workload], "name": args.workload},
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": thr, "kind": "oracle",
                             "sample": desc},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def _dtype_name(w):
    return {"d20_int64": "int64", "d10_int64": "int64", "d16_fp64": "f64", "d16_mixed": "f32+ff",
            "d16_ff": "ff", "d18_fp32": "f32", "batched": "f32", "fwdbwd": "f32",
            "maxconv": "int64"}[w]


# ------------------------------------------------------------------- main


def _roofline(wl, prof, steps):
    """Roofline of the kernel with the largest traced device time: its
    algorithmic bytes (or FP64 operations) per launch over its mean launch
    time, against the measured HBM peak (or the FP64 roof)."""
    peak_hbm, peak_kind = _peaks()
    if not prof:
        return None
    kname, (launches, kms) = max(prof.items(), key=lambda kv: kv[1][1])
    lps = launches / steps
    alg, bound = wl.kernel_alg(kname, lps)
    per_launch_ms = kms / launches
    if alg is None:
        return {"bound": "hbm", "kernel": kname, "achieved": None, "peak": peak_hbm,
                "unit": "GB/s", "frac": None, "traffic": None}
    if bound == "alu32":
        achieved = alg / (per_launch_ms / 1e3) / 1e12
        peak, source = _fp32_peak()
        return {"bound": "alu", "kernel": kname, "achieved": achieved,
                "peak": peak / 1e12, "unit": "TFLOP/s",
                "frac": achieved / (peak / 1e12), "traffic": None,
                "ms_per_launch": per_launch_ms, "peak_source": source,
                "frac_of_nominal": achieved / (FP32_OPS_NOMINAL / 1e12)}
    if bound == "alu":
        achieved = alg / (per_launch_ms / 1e3) / 1e12
        peak, source = _fp64_peak()
        return {"bound": "alu", "kernel": kname, "achieved": achieved,
                "peak": peak / 1e12, "unit": "TFLOP/s",
                "frac": achieved / (peak / 1e12), "traffic": None,
                "ms_per_launch": per_launch_ms, "peak_source": source,
                "frac_of_nominal": achieved / (FP64_OPS_NOMINAL / 1e12)}
    achieved = alg / (per_launch_ms / 1e3) / 1e9
    return {"bound": "hbm", "kernel": kname, "achieved": achieved, "peak": peak_hbm,
            "unit": "GB/s", "frac": achieved / peak_hbm,
            "traffic": _traffic_from_profiles(wl.name if wl.D_override is None else
                                              f"{wl.name}@D{wl.D}", kname),
            "ms_per_launch": per_launch_ms,
            "peak_source": f"{peak_kind} (MEASURED_PEAKS.json hbm_gbs)"}


def _measure(wl, steps, warmup, dist, world):
    """Time `steps` steps of a prepared workload; the per-workload part of the
    JSON line (time, value, roofline, kernels, clocks)."""
    ms, prof, clk = _time_steps(wl, steps, warmup, dist)
    peak_hbm, _ = _peaks()
    return {
        "ms_per_step": ms / steps,
        "value": _whole_job_value(world, wl.outputs, steps, ms),
        "steps": steps,
        "roofline": _roofline(wl, prof, steps),
        "alg_hbm_frac": (wl.alg_bytes * steps / (ms / 1e3) / 1e9) / peak_hbm,
        "kernels": {k: {"launches": v[0], "ms": round(v[1], 4)} for k, v in prof.items()},
        "gpu_launches": sum(v[0] for v in prof.values()),
        "clocks": clk,
    }


# D = 14..19 of the D = 20 int64 workload (same value distribution, tuned
# schedules): steps per D so that each point takes a fraction of a second.
SWEEP_STEPS = {14: 200, 15: 100, 16: 60, 17: 40, 18: 30, 19: 20}
# Sweep points up to this D replay their convolution from a CUDA graph (one
# launch per step), so that the host's per-call work does not leave the GPU
# idle inside the timed steps.
SWEEP_GRAPH_MAX_D = 16
# The training-system forms beside the plain method, each timed after the
# headline: (workload, steps).
FORMS = (("batched", 20), ("fwdbwd", 30), ("d16_fp64", 30), ("d16_mixed", 50),
         ("d16_ff", 50), ("d18_fp32", 50), ("maxconv", 30))


def _brief(res):
    r = res.get("roofline") or {}
    out = {"ms_per_step": round(res["ms_per_step"], 5), "value": res["value"],
           "alg_hbm_frac": round(res["alg_hbm_frac"], 4),
           "dominant": {k: (round(v, 4) if isinstance(v, float) else v)
                        for k, v in r.items() if k in ("kernel", "bound", "achieved", "frac",
                                                       "peak", "unit", "ms_per_launch",
                                                       "traffic")},
           "kernels": res["kernels"], "gpu_launches": res["gpu_launches"],
           "clocks": res["clocks"]}
    return out


def _sweep(dev, main_res, main_D, warmup):
    """D = 14..20 int64 (the D = 20 workload's distribution, tuned schedules):
    per D the step time, outputs/s, the whole-method algorithmic fraction and
    the dominant kernel's roofline."""
    import torch
    out = {}
    for D in sorted(SWEEP_STEPS):
        if D == main_D:
            continue
        wl = Workload("d20_int64", dev, 0, D)
        if D <= SWEEP_GRAPH_MAX_D:
            wl.use_graph()  # steps of a few launches and < 0.4 ms: replay one graph
        res = _measure(wl, SWEEP_STEPS[D], warmup, None, 1)
        out[str(D)] = {"outputs": 3 ** D, **_brief(res),
                       **({"cuda_graph": True} if wl.graph is not None else {})}
        del wl
        torch.cuda.empty_cache()
    out[str(main_D)] = {"outputs": 3 ** main_D, **_brief(main_res)}
    return dict(sorted(out.items(), key=lambda kv: int(kv[0])))


def _forms(dev, warmup):
    """The batched, differentiation and precision forms, each timed on its
    own after the headline, with its comparison against the plain method."""
    import torch
    out = {}
    for name, steps in FORMS:
        wl = Workload(name, dev, 0, None)
        res = _measure(wl, steps, warmup, None, 1)
        entry = {"workload": WORKLOADS[name], "dtype": _dtype_name(name),
                 "outputs_per_step": wl.outputs, **_brief(res)}
        if name == "batched":
            entry["fused_max_d"] = wl.batch.fused_max_d
        cmp = _comparisons(wl, res["ms_per_step"])
        if cmp is not None:
            entry["comparisons"] = cmp
        out[name] = entry
        del wl
        torch.cuda.empty_cache()
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=None)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--workload", default="d20_int64", choices=sorted(WORKLOADS))
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-sweep", action="store_true",
                    help="skip the D=14..19 sweep and the forms after the D=20 headline")
    ap.add_argument("--instances", type=int, default=4096,
                    help="instances of the batched workload (4096; smaller batches are for "
                         "profiling captures)")
    ap.add_argument("--D", type=int, default=None,
                    help="override D of a single-instance workload (same distribution)")
    ap.add_argument("--schedule", default=None,
                    help="force a schedule kind:c:k:cols[:cols_outer] (kind passes|padded|chunked|bulk; "
                         "hybrid|lowmem:c:k:cols:cols_outer:top) "
                         "instead of the tuned default, e.g. passes:6:6:32")
    args = ap.parse_args()
    if args.D is not None and args.workload not in SINGLE + ("fwdbwd",):
        ap.error("--D applies to single-instance workloads only")
    if args.steps is None:
        args.steps = DEFAULT_STEPS[args.workload]
    args.warmup = max(args.warmup, 3) if args.impl == "ours" else args.warmup

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        return _reference_arm(args, rank, world)

    import torch

    from paper_1608_00206_gb300.build import build

    if rank == 0 or world == 1:
        build()
    dist = None
    if world > 1:
        import torch.distributed as dist_mod
        dist_mod.init_process_group("nccl", device_id=torch.device("cuda", local))
        dist = dist_mod
        if rank != 0:
            build()  # the library is in-tree; the build is a no-op once rank 0 made it
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)

    if args.instances != 4096 and args.workload != "batched":
        ap.error("--instances applies to the batched workload only")
    wl = Workload(args.workload, dev, rank, args.D, args.instances)
    if args.schedule:
        if args.workload not in SINGLE:
            ap.error("--schedule applies to single-instance workloads only")
        kind, c, k, cols, *outer = args.schedule.split(":")
        if kind not in ("passes", "padded", "chunked", "bulk", "hybrid", "lowmem"):
            ap.error("schedule kind is passes, padded, chunked, bulk, hybrid or lowmem")
        wl.sched = {"c": int(c), "cols": int(cols),
                    ("kmax" if kind in ("passes", "padded", "hybrid", "lowmem") else "m"): int(k)}
        if kind == "padded":
            wl.sched["padded"] = True
        if kind == "bulk":
            wl.sched["bulk"] = True
        if kind in ("hybrid", "lowmem"):
            if len(outer) != 2:
                ap.error(f"{kind} schedules are {kind}:c:k:cols:cols_outer:top")
            wl.sched["top"] = int(outer[1])
            wl.sched["lowmem"] = kind == "lowmem"
        if outer:
            wl.sched["cols_outer"] = int(outer[0])
        nb = wl.hc.workspace_size(wl.D, wl.z.dtype, wl.mixed, **wl.sched)
        wl.ws = torch.empty(max(nb, 256), dtype=torch.uint8, device=dev)
    if args.workload == "d10_int64":
        wl.use_graph()  # launch-bound: replay the convolution from a CUDA graph
    res = _measure(wl, args.steps, args.warmup, dist, world)
    ms = res["ms_per_step"] * args.steps

    line = {
        "metric": METRIC, "value": res["value"], "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": res["ms_per_step"],
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": _dtype_name(args.workload), "data": "synthetic",
        "config": {"workload": WORKLOADS[args.workload] if args.D is None else
                   f"{WORKLOADS[args.workload]} with D overridden to {args.D}",
                   "schedule": args.schedule or "tuned default",
                   "name": args.workload, "D": wl.D,
                   "outputs_per_step": wl.outputs, "parallelism": f"replicas{world}",
                   **({"fused_max_d": wl.batch.fused_max_d} if args.workload == "batched" else {}),
                   **({"cuda_graph": True,
                       "kernel_times": "per-kernel split from one replay of the step "
                                       "captured with the tracer's event pairs (batched: one "
                                       "eager launch) after the timed graph replays, scaled by "
                                       "steps"}
                      if args.workload == "batched" or wl.graph is not None else {}),
                   "l2": "working set larger than L2 (129 MB); no flush"
                   if wl.alg_bytes >= L2_BYTES else
                   "working set below L2: L2 flushed between steps (256 MB write, "
                   "outside the per-step CUDA events; time = sum of the steps' events)"},
        "roofline": res["roofline"],
        "alg_hbm_frac": res["alg_hbm_frac"],
        "kernels": res["kernels"],
        "gpu_launches": res["gpu_launches"],
        "clocks": res["clocks"],
    }
    if world == 1:
        cmp = _comparisons(wl, ms / args.steps)
        if cmp is not None:
            line["comparisons"] = cmp
    if world == 1 and not args.no_e2e:
        line["e2e"] = _e2e(wl)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = _cpu_baseline(args.workload)
    if args.instances != 4096:
        line["config"]["workload"] += f" with {args.instances} instances"
    headline_default = (args.workload == "d20_int64" and args.D is None and not args.schedule)
    if world == 1 and headline_default and not args.no_sweep:
        del wl
        torch.cuda.empty_cache()
        line["sweep"] = _sweep(dev, res, 20, args.warmup)
        line["forms"] = _forms(dev, args.warmup)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
