"""Benchmark: HVPs/s (loss + gradient + HVP per call) of the brickwall workload
n = 20, L = 16 (K = 152 gates), N_s = 64 Haar product states, complex64 states
with FP64 accumulation, on synthetic seeded inputs.

One step = one full evaluation of the whole workload (every pass plus the FP64
post-processing) in the schedule the library's autotuner picks at set-up: the
fused 5-qubit blocks on the tensor cores or the SIMT window passes; the other
schedule is timed on a line of its own. `value` is measured with the inputs
resident in HBM (stream-ordered device-pointer call replaying the captured
CUDA graph, CUDA events on the library's stream); `e2e` times the host-memory
C ABI call (G, V uploaded and every result downloaded each step).

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
Under torchrun each rank runs an independent replica of the workload on its
own GPU, and rank 0 prints one JSON line.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import re
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD = dict(n=20, n_layers=16, n_samples=64, seed=0)
METRIC = "HVPs/sec (loss+grad+HVP) at n=20,L=16,N_s=64; fraction of HBM roofline"
MEASURED_FFMA_TFLOPS = 74.6   # FP32 FFMA throughput measured on a GB300 by a register-only loop
FP32_LANES_PER_SM, N_SM = 128, 152


# Per schedule: the sources of its dominant (backward) kernel, whose committed
# DRAM traffic record counts only while they are unchanged, the record, and
# the plan fields a record must match.
KERNEL_SOURCES = {
    "window": ["paper_2604_20384_gb300/csrc/tiled.cu", "paper_2604_20384_gb300/csrc/tiled_common.cuh"],
    "tensor": ["paper_2604_20384_gb300/csrc/tcblock.cu", "paper_2604_20384_gb300/csrc/internal.h"],
}
TRAFFIC_FILES = {"window": os.path.join(ROOT, "profiles", "traffic_n20_L16_Ns64.json"),
                 "tensor": os.path.join(ROOT, "profiles", "traffic_tcb_n20_L16_Ns64.json")}
PLAN_KEYS = {"window": ("window", "threads", "variant", "passes", "checkpoint_stride"),
             "tensor": ("window", "passes", "variant")}


def strip_comments(src: str) -> str:
    """C/C++ source without comments and blank lines (string literals in the
    kernel sources hold no comment markers)."""
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    src = re.sub(r"//[^\n]*", "", src)
    return "\n".join(line.rstrip() for line in src.splitlines() if line.strip())


def kernel_source_hash(schedule: str = "window") -> str:
    """Hash of the code (comments stripped) of a schedule's kernel sources."""
    h = hashlib.sha256()
    for rel in KERNEL_SOURCES[schedule]:
        with open(os.path.join(ROOT, rel)) as f:
            h.update(strip_comments(f.read()).encode())
    return h.hexdigest()


def recorded_traffic(info, schedule: str = "window"):
    """DRAM bytes per backward-kernel launch from the committed ncu capture, if
    it was taken on the current kernel sources and the same plan, else None."""
    try:
        with open(TRAFFIC_FILES[schedule]) as f:
            doc = json.load(f)
    except (OSError, ValueError):
        return None
    if doc.get("source_sha256") != kernel_source_hash(schedule):
        return None
    for rec in doc.get("records", []):
        plan = rec.get("plan", {})
        if all(plan.get(k) == info[k] for k in PLAN_KEYS[schedule]):
            return rec.get("bwd_kernel_bytes_per_launch")
    return None


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device: int):
        self.device = device
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.device), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except OSError:
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
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.thread.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for name, val in zip(names, parts[5:9]):
                if val.lower() == "active":
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "samples": len(sm), "reasons": sorted(reasons)}


def cpu_model() -> str:
    """Host CPU model as lscpu reports it (x86 and Arm), else /proc/cpuinfo."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.strip().startswith("Model name:"):
                return line.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                if line.lower().startswith("model name"):
                    return line.split(":", 1)[1].strip()
    except OSError:
        pass
    return "unknown"


def cpu_baseline(w, steps=1, warmup=0, max_seconds=150.0):
    """The FP64 oracle, as it stands, on a bounded sample of the workload:
    as many of the N_s samples as the host has cores, one thread each. Cost is
    exactly linear in N_s (samples are independent), so HVPs/s = (sample /
    N_s) / seconds."""
    from oracle import oracle

    cores = os.cpu_count() or 1
    m = max(1, min(w.n_samples, cores))
    sub = w.psi1q[:m]
    phi = oracle.reference_states(w.n, w.n_layers, w.Uref, sub)
    stride = max(1, int(round(w.K ** 0.5)))
    times = []
    out = None
    for i in range(warmup + steps):
        t0 = time.perf_counter()
        out = oracle.evaluate(w.n, w.n_layers, w.G, w.V, sub, phi, threads=m, ckpt_stride=stride, want_env=True)
        dt = time.perf_counter() - t0
        if i >= warmup:
            times.append(dt)
        if sum(times) > max_seconds:
            break
    sec = statistics.median(times)
    return dict(value=(m / w.n_samples) / sec, unit="HVPs/s", cores=m, kind="oracle", cpu=cpu_model(),
                sample=f"{m} of {w.n_samples} samples (n={w.n}, L={w.n_layers}), {m} threads, "
                       f"checkpoint stride {stride}; {sec:.2f} s per sample batch, scaled by {m}/{w.n_samples}",
                seconds_per_step=sec, steps=len(times), oracle_out=out)


def run_reference(args, rank, world):
    """--impl reference: the FP64 CPU oracle on the host cores (rank 0 only).

    Every step (warm-up and timed alike) is one oracle run over a bounded
    sample of the workload: as many of the N_s samples as the host has cores,
    one thread each. `ms_per_step` is the wall time of such a step; `value`
    scales it to the whole workload by N_s / sample (samples are independent,
    so the cost is exactly linear in N_s), stated in `ns_scaling`."""
    if rank != 0:
        return 0
    from oracle import oracle
    from paper_2604_20384_gb300.inputs import make_workload

    w = make_workload(**WORKLOAD)
    cores = os.cpu_count() or 1
    m = max(1, min(w.n_samples, cores))
    sub = w.psi1q[:m]
    phi = oracle.reference_states(w.n, w.n_layers, w.Uref, sub)
    stride = max(1, int(round(w.K ** 0.5)))
    steps, warmup = max(1, args.steps), max(0, args.warmup)
    for _ in range(warmup):
        oracle.evaluate(w.n, w.n_layers, w.G, w.V, sub, phi, threads=m, ckpt_stride=stride)
    t0 = time.perf_counter()
    for _ in range(steps):
        oracle.evaluate(w.n, w.n_layers, w.G, w.V, sub, phi, threads=m, ckpt_stride=stride)
    sec = (time.perf_counter() - t0) / steps
    value = (m / w.n_samples) / sec
    sample = (f"{m} of {w.n_samples} samples (n={w.n}, L={w.n_layers}) per step, {m} threads, checkpoint stride "
              f"{stride}; {sec:.2f} s per step, HVPs/s scaled by {m}/{w.n_samples}")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "HVPs/s", "n_gpus": world,
            "steps": steps, "warmup": warmup, "ms_per_step": 1000.0 * sec,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": "brickwall HVP n=20 L=16 N_s=64 (K=152)", "n": 20, "L": 16, "N_s": 64},
            "ns_scaling": {"samples_per_step": m, "n_samples": w.n_samples, "factor": m / w.n_samples},
            "cpu_baseline": {"value": value, "unit": "HVPs/s", "cores": m, "kind": "oracle", "sample": sample,
                             "cpu": cpu_model()},
            "e2e": {"value": value, "unit": "HVPs/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def batch_line(native, make_workload, torch, dev, local, n_circuits: int, reps: int) -> dict:
    """Batched uneven circuits (n ~ U{8..16}, L ~ U{4..20}, N_s log-uniform in
    32..512, seed 0; the first n_circuits of the 64): one persistent launch per
    call, window width autotuned at set-up."""
    import numpy as np
    from paper_2604_20384_gb300.inputs import uneven_batch_shapes

    shapes = uneven_batch_shapes(64, seed=0)[:n_circuits]
    bws = [make_workload(n, L, ns, sd) for (n, L, ns, sd) in shapes]
    bstream = torch.cuda.Stream(device=dev)
    with native.BatchContext([(x.n, x.n_layers, x.psi1q, x.Uref) for x in bws], device=local,
                             stream=bstream.cuda_stream, autotune=True) as bctx:
        Gb = torch.from_numpy(np.concatenate([x.G for x in bws]).view(np.float64).reshape(-1).copy()).to(dev)
        Vb = torch.from_numpy(np.concatenate([x.V for x in bws]).view(np.float64).reshape(-1).copy()).to(dev)
        for _ in range(3):
            bctx.hvp_dev(Gb.data_ptr(), Vb.data_ptr(), None, None, None)
        torch.cuda.synchronize(dev)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(bstream)
        for _ in range(reps):
            bctx.hvp_dev(Gb.data_ptr(), Vb.data_ptr(), None, None, None)
        e1.record(bstream)
        torch.cuda.synchronize(dev)
        b_ms = e0.elapsed_time(e1) / reps
        binfo = bctx.plan_info()
    amp_gates = sum((1 << x.n) * x.n_samples * x.K for x in bws)
    return {"workload": f"{n_circuits} circuits, n~U{{8..16}}, L~U{{4..20}}, N_s log-uniform 32..512 (seed 0)",
            "value": 1000.0 / b_ms, "unit": "batch HVP evaluations/s", "ms_per_step": b_ms,
            "circuit_hvps_per_s": n_circuits * 1000.0 / b_ms, "work_items": binfo["items"],
            "persistent_ctas": binfo["ctas"], "launches_per_step": binfo["launches_per_hvp"],
            "window": binfo["window"], "window_choice": "autotuned among 12, 11, 10 at set-up",
            "achieved_tflops": amp_gates * 384 / (b_ms / 1e3) / 1e12}


def _time_calls(torch, stream, dev, fn, reps: int, warm: int = 2) -> float:
    for _ in range(warm):
        fn()
    torch.cuda.synchronize(dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(reps):
        fn()
    e1.record(stream)
    torch.cuda.synchronize(dev)
    return e0.elapsed_time(e1) / reps


def n12_precision_line(native, make_workload, torch, dev, local) -> dict:
    """n = 12, L = 8, N_s = 256: complex64 window passes with FP64 accumulation
    next to the complex128 per-gate sweep, each timed and compared with the
    other (the oracle comparison of both is in the GPU tests)."""
    import numpy as np

    w = make_workload(12, 8, 256, seed=0)
    st = torch.cuda.Stream(device=dev)
    G = torch.from_numpy(w.G.view(np.float64).reshape(-1).copy()).to(dev)
    V = torch.from_numpy(w.V.view(np.float64).reshape(-1).copy()).to(dev)
    out = {}
    res = {}
    for prec in ("c64", "c128"):
        with native.Context(w.n, w.n_layers, w.psi1q, w.Uref, precision=prec, device=local,
                            stream=st.cuda_stream) as c:
            ms = _time_calls(torch, st, dev, lambda: c.hvp_dev(G.data_ptr(), V.data_ptr(), None, None, None), 20)
            res[prec] = c.hvp(w.G, w.V)
            out[prec] = {"value": 1000.0 / ms, "unit": "HVPs/s", "ms_per_step": ms}
    g64, h64 = res["c64"][1], res["c64"][2]
    g128, h128 = res["c128"][1], res["c128"][2]
    out["c64_vs_c128"] = {"grad_rel": float(np.linalg.norm(g64 - g128) / np.linalg.norm(g128)),
                          "hvp_rel": float(np.linalg.norm(h64 - h128) / np.linalg.norm(h128)),
                          "loss_abs": abs(res["c64"][0] - res["c128"][0])}
    out["workload"] = "n=12 L=8 N_s=256 (K=44), 8 MiB per state set (L2-resident)"
    return out


def n26_autograd_line(make_workload, torch, dev, local) -> dict:
    """n = 26, L = 24, N_s = 8 through the torch.autograd layer: loss and
    gradient by the adjoint sweep (HSLoss backward) and the HVP by forward-
    over-reverse (jvp of HSGrad); the forward cache does not fit at this
    size, so forward states are recomputed from boundary checkpoints."""
    from paper_2604_20384_gb300 import autograd as hsa

    w = make_workload(26, 24, 8, seed=0)
    cost = hsa.HSCost(w.n, w.n_layers, w.psi1q, w.Uref, device=local)
    try:
        G = torch.from_numpy(w.G).to(dev)
        V = torch.from_numpy(w.V).to(dev)
        cur = torch.cuda.current_stream(dev)

        def grad_step():
            Gr = G.clone().requires_grad_(True)
            hsa.loss(Gr, cost).backward()

        ms_g = _time_calls(torch, cur, dev, grad_step, 3, warm=1)
        ms_h = _time_calls(torch, cur, dev, lambda: hsa.hvp(G, V, cost), 3, warm=1)
        info = cost.ctx.plan_info()
    finally:
        cost.close()
    return {"workload": "n=26 L=24 N_s=8 (K=300, 8 GiB per state set), torch.autograd layer",
            "loss_grad_backward": {"value": 1000.0 / ms_g, "unit": "evaluations/s", "ms_per_step": ms_g},
            "hvp_forward_over_reverse": {"value": 1000.0 / ms_h, "unit": "HVPs/s", "ms_per_step": ms_h},
            "passes": info["passes"], "checkpoint_stride": info["checkpoint_stride"],
            "device_mib": info["device_mib"]}


def kinds_summary(native, prof) -> dict:
    """Per launch kind of one profiled call: launches, device ms, flops and
    algorithmic bytes."""
    kinds = prof["kind"]
    out = {}
    for k in sorted(set(kinds.tolist())):
        sel = kinds == k
        out[native.KINDS[k]] = dict(launches=int(sel.sum()), ms=float(prof["ms"][sel].sum()),
                                    flops=float(prof["flops"][sel].sum()), bytes=float(prof["bytes"][sel].sum()))
    return out


def window_roofline(by_kind, info, total_ms, peaks, src):
    """Roofline of the window-pass schedule's dominant kernel, the backward
    window-pass kernel (backward passes and, when forward states are
    recomputed, the turnaround pass). Its arithmetic is FP32 SIMT, so the
    bound is the FP32 lane rate at the maximum SM clock; with the forward cache
    it also streams 16 B per amplitude per gate from HBM (the HBM fraction is
    reported beside it). Also returns the step's HBM fraction: every window
    pass's algorithmic bytes over their time."""
    cached = info["checkpoint_stride"] == 0
    bwd_kinds = [k for k in ("pass_bwd", "pass_turnaround") if k in by_kind]
    p_ms = sum(by_kind[k]["ms"] for k in bwd_kinds)
    p_fl = sum(by_kind[k]["flops"] for k in bwd_kinds)
    p_by = sum(by_kind[k]["bytes"] for k in bwd_kinds)
    p_n = sum(by_kind[k]["launches"] for k in bwd_kinds)
    sm_mhz = peaks.get("sm_max_mhz", 2070.0)
    alu_peak = N_SM * FP32_LANES_PER_SM * 2 * sm_mhz * 1e6 / 1e12       # TFLOP/s
    achieved = (p_fl / p_n) / (p_ms / p_n / 1e3) / 1e12
    fwd = by_kind.get("pass_fwd", {"ms": 0.0, "flops": 0.0, "launches": 0})
    all_ms = sum(by_kind[k]["ms"] for k in by_kind if k.startswith("pass_"))
    all_fl = sum(by_kind[k]["flops"] for k in by_kind if k.startswith("pass_"))
    all_by = sum(by_kind[k]["bytes"] for k in by_kind if k.startswith("pass_"))
    hbm_peak = peaks.get("hbm_gbs", 6800.0)
    roofline = {"bound": "alu", "achieved": achieved, "peak": alu_peak, "unit": "TFLOP/s",
                "frac": achieved / alu_peak, "traffic": recorded_traffic(info, "window"),
                "kernel": (f"tiled_bwdc_kernel<tangent, {info['threads']} threads> (backward window passes "
                           f"reading the forward cache, window {info['window']})" if cached else
                           f"tiled_bwd_kernel<tangent, {'packed' if info['variant'] == 2 else 'scalar'}, "
                           f"{info['threads']} threads> (backward and turnaround window passes, "
                           f"window {info['window']})"),
                "launches_per_step": p_n, "share_of_step": p_ms / total_ms,
                "algorithmic_bytes_per_launch": p_by / p_n,
                "peak_note": f"152 SMs x 128 FP32 lanes x 2 flop x {sm_mhz:.0f} MHz (unit counts and max clock)",
                # measured beside it: a register-only FFMA loop on every SM of this GPU model
                "peak_measured": MEASURED_FFMA_TFLOPS, "frac_of_measured": achieved / MEASURED_FFMA_TFLOPS,
                "peak_measured_note": "register-only FFMA loop, 152 SMs, CUDA events (packed fma.rn.f32x2: 75.5)",
                "forward_kernel": {"achieved": fwd["flops"] / max(fwd["ms"], 1e-9) / 1e9,
                                   "frac": fwd["flops"] / max(fwd["ms"], 1e-9) / 1e9 / alu_peak,
                                   "share_of_step": fwd["ms"] / total_ms},
                "all_window_passes": {"achieved": all_fl / (all_ms / 1e3) / 1e12,
                                      "frac": all_fl / (all_ms / 1e3) / 1e12 / alu_peak},
                "hbm": {"achieved_gbs": p_by / (p_ms / 1e3) / 1e9, "peak_gbs": hbm_peak,
                        "frac": (p_by / (p_ms / 1e3) / 1e9) / hbm_peak, "peak_source": src}}
    gbs = all_by / (all_ms / 1e3) / 1e9
    # every window pass of the step: the schedule's algorithmic bytes (state I/O and, with the
    # forward cache, 16 B per amplitude per gate written and read back) over their time
    hbm = {"frac": gbs / hbm_peak, "achieved_gbs": gbs, "peak_gbs": hbm_peak, "peak_source": src,
           "bytes_per_step": all_by, "over": "window passes"}
    return roofline, hbm


def tensor_roofline(by_kind, info, total_ms, peaks, src):
    """Roofline of the fused-block tensor-core schedule's dominant kernel, the
    backward block pass: algorithmic HBM bytes per launch (co-states read and
    written, forward states read: 48 B per amplitude, 32 B in the last pass)
    over its event-timed duration against the measured copy bandwidth, with
    its tensor-pipe rate beside it. Also returns the step's HBM fraction: every
    block pass's algorithmic bytes over their time."""
    hbm_peak = peaks.get("hbm_gbs", 6800.0)
    bf16 = peaks.get("bf16_tflops_sustained", peaks.get("bf16_tflops", 1900.0))
    bw = by_kind.get("block_bwd", {"ms": 0.0, "flops": 0.0, "bytes": 0.0, "launches": 1})
    fw = by_kind.get("block_fwd", {"ms": 0.0, "flops": 0.0, "bytes": 0.0, "launches": 1})

    def _rate(d):
        n = max(d["launches"], 1)
        per_ms = max(d["ms"], 1e-9) / n
        gbs = d["bytes"] / n / per_ms / 1e6
        tfl = d["flops"] / n / per_ms / 1e9
        return {"achieved": gbs, "peak": hbm_peak, "unit": "GB/s", "frac": gbs / hbm_peak,
                "algorithmic_bytes_per_launch": d["bytes"] / n, "ms_per_launch": per_ms, "launches_per_step": n,
                "share_of_step": d["ms"] / total_ms, "tensor_pipe": {
                    "achieved_tflops": tfl, "peak_tflops": bf16, "frac": tfl / bf16,
                    "note": "bf16 slice products and TF32 environment products issued, against the measured "
                            "sustained bf16 cuBLAS rate"}}

    roofline = dict(_rate(bw), bound="hbm", traffic=recorded_traffic(info, "tensor"), peak_source=src,
                    kernel="tcb_kernel<1, 1> (backward fused 5-qubit block with tangents: exact-integer bf16 "
                           "slice GEMM and TF32 environment GEMM on tcgen05, TMA tile loads)")
    roofline["forward_kernel"] = _rate(fw)
    all_by = bw["bytes"] + fw["bytes"]
    all_ms = bw["ms"] + fw["ms"]
    gbs = all_by / max(all_ms, 1e-9) / 1e6
    hbm = {"frac": gbs / hbm_peak, "achieved_gbs": gbs, "peak_gbs": hbm_peak, "peak_source": src,
           "bytes_per_step": all_by, "over": "block passes"}
    return roofline, hbm


def parity_outputs(native, ctx, w, m: int, local: int, stream, tensor: bool) -> dict:
    """What the parity check compares with the oracle's run on the first m
    samples, read after a full (tangent) call of ctx: the per-sample overlaps
    T and Omega and, for the window-pass schedule, the per-sample
    environments E and DE; the tensor schedule keeps no per-sample
    environments, so a context on the first m samples gives the gradient and
    HVP instead (sums over those samples)."""
    d = {"T": ctx.get("T"), "Omega": ctx.get("Omega")}
    if tensor:
        with native.Context(w.n, w.n_layers, w.psi1q[:m], w.Uref, device=local, stream=stream, tensor=True) as sub:
            _, d["grad"], d["hvp"] = sub.hvp(w.G, w.V)
    else:
        d["E"], d["DE"] = ctx.get("env")
    return d


def parity_check(d: dict, o: dict, m: int, tol: float = 1e-5) -> dict:
    """Relative errors of parity_outputs against the oracle's outputs."""
    import numpy as np

    def _rel(a, b):
        return float(np.linalg.norm(np.ravel(a - b)) / np.linalg.norm(np.ravel(b)))

    per_sample = ("T", "Omega", "E", "DE")
    res = {"samples": m, "tolerance": tol}
    for k in ("T", "Omega", "E", "DE", "grad", "hvp"):
        if k in d:
            res[k + "_rel"] = _rel(d[k][:m] if k in per_sample else d[k], o[k])
    res["pass"] = all(v < tol for k, v in res.items() if k.endswith("_rel"))
    return res


def schedule_line(native, torch, dev, local, w, steps: int, m: int, tensor: bool):
    """The same workload on the schedule the autotuner did not pick: the
    fused-block tensor-core schedule (HVP_TENSOR), or the window passes with
    the forward cache (12-qubit windows, 256 threads, scalar arithmetic).
    Device-resident HVPs/s, per-kind device time, the roofline of its dominant
    kernel, and what its parity check needs."""
    import numpy as np

    ts = torch.cuda.Stream(device=dev)
    G = torch.from_numpy(w.G.view(np.float64).reshape(-1).copy()).to(dev)
    V = torch.from_numpy(w.V.view(np.float64).reshape(-1).copy()).to(dev)
    kw = dict(tensor=True) if tensor else dict(precision="c64", window=12, threads=256, variant=1)
    with native.Context(w.n, w.n_layers, w.psi1q, w.Uref, device=local, stream=ts.cuda_stream, **kw) as c:
        for _ in range(3):
            c.hvp_dev(G.data_ptr(), V.data_ptr(), None, None, None)
        torch.cuda.synchronize(dev)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(ts)
        for _ in range(steps):
            c.hvp_dev(G.data_ptr(), V.data_ptr(), None, None, None)
        e1.record(ts)
        torch.cuda.synchronize(dev)
        t_ms = e0.elapsed_time(e1) / steps
        info = c.plan_info()
        prof = c.profile(G.data_ptr(), V.data_ptr())
        c.hvp(w.G, w.V)
        par = parity_outputs(native, c, w, m, local, ts.cuda_stream, tensor)
    by_kind = kinds_summary(native, prof)
    total = float(prof["ms"].sum())
    peaks, src = _peaks()
    roof, hbm = (tensor_roofline if tensor else window_roofline)(by_kind, info, total, peaks, src)
    line = {"workload": ("brickwall HVP n=20 L=16 N_s=64 (K=152), " +
                         ("fused 5-qubit blocks on the tensor cores (HVP_TENSOR): exact-integer bf16 slice GEMMs, "
                          "TF32 environment GEMM, FP64 reductions" if tensor else
                          "complex64 window passes with the forward cache, FP64 accumulation")),
            "value": 1000.0 / t_ms, "unit": "HVPs/s", "ms_per_step": t_ms, "plan": info,
            "per_kind": by_kind, "roofline": roof, "hbm_roofline": hbm}
    return line, par


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=40)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-fp64", action="store_true", help="skip the unfused FP64 comparison sweep")
    ap.add_argument("--no-batch", action="store_true", help="skip the batched uneven-circuit measurement")
    ap.add_argument("--no-multi", action="store_true", help="skip the two-directions-per-sweep measurement")
    ap.add_argument("--no-configs", action="store_true", help="skip the n=12 precision and n=26 autograd lines")
    ap.add_argument("--no-other", "--no-tensor", dest="no_other", action="store_true",
                    help="skip the line of the schedule the autotuner did not pick")
    ap.add_argument("--samples", type=int, default=64,
                    help="N_s of the workload (64 is the benchmark; smaller only for profiler captures)")
    ap.add_argument("--threads", type=int, default=0, help="window-pass kernel threads (0 = library default)")
    ap.add_argument("--variant", type=int, default=0, help="1 scalar FMA, 2 packed FMA (0 = library default)")
    ap.add_argument("--window", type=int, default=0, help="window qubits (0 = library default)")
    ap.add_argument("--recompute", action="store_true",
                    help="recompute forward states inside window passes instead of caching every gate's")
    ap.add_argument("--no-autotune", action="store_true",
                    help="use the library defaults (or --threads/--variant/--window) instead of autotuning at set-up")
    ap.add_argument("--multi", action="store_true",
                    help="with --quick: time two directions per call in a two-direction (HVP_MULTI_DIR) context")
    ap.add_argument("--quick-batch", type=int, default=0, metavar="C",
                    help="only time the batched line on its first C circuits (for profiler captures)")
    ap.add_argument("--quick-fp64", action="store_true",
                    help="only time the unfused complex128 sweep at --samples (for profiler captures)")
    ap.add_argument("--quick", action="store_true",
                    help="only the device-resident timing (for profiler captures)")
    ap.add_argument("--tensor", action="store_true",
                    help="with --quick: time the fused-block tensor-core schedule (HVP_TENSOR)")
    args = ap.parse_args()
    if args.warmup < 3 and args.impl == "ours":
        args.warmup = 3

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))

    if args.impl == "reference":
        return run_reference(args, rank, world)

    import numpy as np
    import torch

    from paper_2604_20384_gb300 import native
    from paper_2604_20384_gb300.inputs import make_workload

    dist = None
    if world > 1:
        import torch.distributed as dist

        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if args.quick_batch:
        if rank == 0:
            print(json.dumps(dict(batch_line(native, make_workload, torch, dev, local, args.quick_batch,
                                             max(args.steps, 1)), quick=True)), flush=True)
        return 0

    w = make_workload(**dict(WORKLOAD, n_samples=args.samples))
    if args.quick_fp64:
        fstream = torch.cuda.Stream(device=dev)
        Gf = torch.from_numpy(w.G.view(np.float64).reshape(-1).copy()).to(dev)
        Vf = torch.from_numpy(w.V.view(np.float64).reshape(-1).copy()).to(dev)
        with native.Context(w.n, w.n_layers, w.psi1q, w.Uref, precision="c128", device=local,
                            stream=fstream.cuda_stream) as c2:
            for _ in range(args.warmup):
                c2.hvp_dev(Gf.data_ptr(), Vf.data_ptr(), None, None, None)
            torch.cuda.synchronize(dev)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(fstream)
            for _ in range(max(args.steps, 1)):
                c2.hvp_dev(Gf.data_ptr(), Vf.data_ptr(), None, None, None)
            e1.record(fstream)
            torch.cuda.synchronize(dev)
            f_ms = e0.elapsed_time(e1) / max(args.steps, 1)
        if rank == 0:
            print(json.dumps({"fp64_unfused": True, "n_samples": args.samples, "ms_per_step": f_ms,
                              "value": 1000.0 / f_ms, "unit": "HVPs/s", "quick": True}), flush=True)
        return 0
    multi = args.multi and args.quick
    tensor = args.tensor and args.quick
    autotune = not (args.no_autotune or args.threads or args.variant or args.window or multi or tensor)
    stream = torch.cuda.Stream(device=dev)
    if tensor:
        ctx = native.Context(w.n, w.n_layers, w.psi1q, w.Uref, device=local, stream=stream.cuda_stream,
                             tensor=True)
    else:
        ctx = native.Context(w.n, w.n_layers, w.psi1q, w.Uref, precision="c64", device=local,
                             stream=stream.cuda_stream, threads=args.threads, variant=args.variant,
                             window=args.window, autotune=autotune, recompute=args.recompute, multi_dir=multi)
    K = w.K
    G_dev = torch.from_numpy(w.G.view(np.float64).reshape(-1).copy()).to(dev)
    if multi:
        from paper_2604_20384_gb300.inputs import random_direction

        Vs = np.stack([w.V, random_direction(K, w.G, seed=5)])
        V_dev = torch.from_numpy(Vs.view(np.float64).reshape(-1).copy()).to(dev)
    else:
        V_dev = torch.from_numpy(w.V.view(np.float64).reshape(-1).copy()).to(dev)
    loss_dev = torch.zeros(1, dtype=torch.float64, device=dev)
    grad_dev = torch.zeros(32 * K, dtype=torch.float64, device=dev)
    hvp_dev = torch.zeros(32 * K * (2 if multi else 1), dtype=torch.float64, device=dev)
    torch.cuda.synchronize(dev)

    def step():
        if multi:
            ctx.hvp_multi_dev(G_dev.data_ptr(), 2, V_dev.data_ptr(), loss_dev.data_ptr(), grad_dev.data_ptr(),
                              hvp_dev.data_ptr())
            return
        ctx.hvp_dev(G_dev.data_ptr(), V_dev.data_ptr(), loss_dev.data_ptr(), grad_dev.data_ptr(),
                    hvp_dev.data_ptr())

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize(dev)
    info = ctx.plan_info()

    # ---------------------------------------------------------- timed region
    if dist:
        dist.barrier()
    torch.cuda.synchronize(dev)
    sampler = ClockSampler(local)
    sampler.start()
    time.sleep(0.3)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for _ in range(args.steps):
        step()
    ev1.record(stream)
    torch.cuda.synchronize(dev)
    if dist:
        dist.barrier()
    torch.cuda.synchronize(dev)
    clocks = sampler.stop()
    ms = ev0.elapsed_time(ev1) / args.steps
    if dist:
        t = torch.tensor([ms], device=dev, dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
    value = world * 1000.0 / ms
    if args.quick:
        if rank == 0:
            print(json.dumps({"metric": METRIC, "value": value * (2 if multi else 1), "unit": "HVPs/s",
                              "ms_per_step": ms, "n_samples": args.samples, "quick": True,
                              "directions_per_step": 2 if multi else 1, "tensor": tensor, "plan": info,
                              "clocks": clocks}),
                  flush=True)
        ctx.close()
        if dist:
            dist.destroy_process_group()
        return 0

    # ------------------------------------------------ end to end (host API)
    Gh = w.G.view(np.float64).reshape(-1).copy()
    Vh = w.V.view(np.float64).reshape(-1).copy()
    for _ in range(2):
        ctx.hvp(Gh, Vh)
    e2e_steps = max(3, min(args.steps, 20))
    if dist:
        dist.barrier()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        ctx.hvp(Gh, Vh)
    e2e_ms = (time.perf_counter() - t0) * 1000.0 / e2e_steps
    if dist:
        t = torch.tensor([e2e_ms], device=dev, dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        e2e_ms = float(t.item())
    res_doubles = 2 + 4 * w.n_samples + 4 * 32 * K
    e2e = {"value": world * 1000.0 / e2e_ms, "unit": "HVPs/s", "h2d_bytes_per_step": 2 * 32 * K * 8,
           "d2h_bytes_per_step": res_doubles * 8 + 4, "ms_per_step": e2e_ms}

    # hvp_plan_info marks the fused-block tensor-core schedule with arithmetic variant 0
    tensor_plan = info["variant"] == 0
    schedule = "tensor" if tensor_plan else "window"
    # per-sample outputs of the last (host-array) call, for the parity check
    m_or = max(1, min(w.n_samples, os.cpu_count() or 1))
    par = parity_outputs(native, ctx, w, m_or, local, stream.cuda_stream, tensor_plan) if rank == 0 else None

    # ------------------------------- loss and gradient only (no tangent sweep; after the
    # per-sample outputs of the last HVP call were read)
    for _ in range(3):
        ctx.hvp_dev(G_dev.data_ptr(), None, loss_dev.data_ptr(), grad_dev.data_ptr(), None)
    torch.cuda.synchronize(dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(10):
        ctx.hvp_dev(G_dev.data_ptr(), None, loss_dev.data_ptr(), grad_dev.data_ptr(), None)
    e1.record(stream)
    torch.cuda.synchronize(dev)
    lg_ms = e0.elapsed_time(e1) / 10
    loss_grad_line = {"workload": "n=20 L=16 N_s=64, loss and gradient only (Alg. 1 without tangents)",
                      "value": world * 1000.0 / lg_ms, "unit": "evaluations/s", "ms_per_step": lg_ms}

    # ------------------------------------------- per-launch roofline (events)
    prof = ctx.profile(G_dev.data_ptr(), V_dev.data_ptr())
    by_kind = kinds_summary(native, prof)
    total_ms = float(prof["ms"].sum())
    peaks, src = _peaks()
    roofline, hbm_roofline = (tensor_roofline if tensor_plan else window_roofline)(by_kind, info, total_ms, peaks,
                                                                                   src)
    cached = info["checkpoint_stride"] == 0
    if tensor_plan:
        workload = ("brickwall HVP n=20 L=16 N_s=64 (K=152), fused 5-qubit blocks on the tensor cores "
                    "(exact-integer bf16 slice GEMMs, TF32 environment GEMM), complex64 states, FP64 accumulation")
        sched_text = ("fused 5-qubit blocks (App. D): the forward states at every block boundary kept, "
                      "block operators applied on tcgen05 tensor cores, per-gate environments by FP64 cuts")
    else:
        workload = "brickwall HVP n=20 L=16 N_s=64 (K=152), complex64 window passes, FP64 accumulation"
        sched_text = ("forward states of every gate cached (Alg. 1), read back by bulk copies"
                      if cached else "forward states recomputed inside each window pass")

    line = {"metric": METRIC, "value": value, "unit": "HVPs/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "c64",
            "data": "synthetic (seeded Haar brickwall, Haar product states)",
            "config": {"workload": workload, "n": 20, "L": 16, "N_s": 64, "K": K,
                       "schedule_kind": schedule,
                       "window": info["window"], "passes": info["passes"], "threads": info["threads"],
                       "variant": info["variant"], "autotuned": autotune,
                       "checkpoint_stride": info["checkpoint_stride"], "tiles_per_cta": info["tiles_per_cta"],
                       "schedule": sched_text, "device_mib": info["device_mib"],
                       "l2": "inputs larger than L2 (512 MiB per state set, 129 MB L2)",
                       "parallelism": f"replicas x{world}"},
            "roofline": roofline,
            # the metric's HBM-roofline fraction: the step's algorithmic bytes over the time of the
            # passes that move them, against the measured copy bandwidth
            "hbm_roofline": hbm_roofline,
            "e2e": e2e, "gpu_launches": info["launches_per_hvp"] * args.steps,
            "clocks": clocks, "per_kind": by_kind, "loss_grad_only": loss_grad_line}

    # ------------------------------------------ unfused FP64 sweep, same GPU
    if not args.no_fp64 and rank == 0:
        ctx.close()
        with native.Context(w.n, w.n_layers, w.psi1q, w.Uref, precision="c128", device=local,
                            stream=stream.cuda_stream) as c2:
            c2.hvp_dev(G_dev.data_ptr(), V_dev.data_ptr(), None, None, None)
            torch.cuda.synchronize(dev)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(2):
                c2.hvp_dev(G_dev.data_ptr(), V_dev.data_ptr(), None, None, None)
            e1.record(stream)
            torch.cuda.synchronize(dev)
            f_ms = e0.elapsed_time(e1) / 2
        line["fp64_unfused"] = {"value": 1000.0 / f_ms, "unit": "HVPs/s", "ms_per_step": f_ms,
                                "speedup_of_value": value / world / (1000.0 / f_ms)}

    # ------------------------------- batched uneven circuits (secondary line)
    if not args.no_batch and rank == 0:
        line["batched_uneven"] = batch_line(native, make_workload, torch, dev, local, 64, 10)

    # ------------------- two directions at the same gates per sweep (f1 line)
    if not args.no_multi and rank == 0:
        from paper_2604_20384_gb300.inputs import random_direction

        wm = make_workload(20, 16, 32, seed=0)
        Vs = np.stack([wm.V, random_direction(wm.K, wm.G, seed=5)])
        mstream = torch.cuda.Stream(device=dev)
        Gm = torch.from_numpy(wm.G.view(np.float64).reshape(-1).copy()).to(dev)
        Vm = torch.from_numpy(Vs.view(np.float64).reshape(-1).copy()).to(dev)
        hm = torch.zeros(2 * 32 * wm.K, dtype=torch.float64, device=dev)

        def _time_two(**kw):
            with native.Context(wm.n, wm.n_layers, wm.psi1q, wm.Uref, device=local, stream=mstream.cuda_stream,
                                **kw) as cm:
                for _ in range(3):
                    cm.hvp_multi_dev(Gm.data_ptr(), 2, Vm.data_ptr(), None, None, hm.data_ptr())
                torch.cuda.synchronize(dev)
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(mstream)
                for _ in range(10):
                    cm.hvp_multi_dev(Gm.data_ptr(), 2, Vm.data_ptr(), None, None, hm.data_ptr())
                e1.record(mstream)
                torch.cuda.synchronize(dev)
                return e0.elapsed_time(e1) / 10, cm.plan_info()

        pair_ms, pinfo = _time_two(window=11, multi_dir=True)
        same_ms, _ = _time_two(window=11)
        best_ms, binfo = _time_two()
        line["two_directions"] = {
            "workload": "n=20 L=16 N_s=32 (K=152), two directions at the same gates per call",
            "value": 2000.0 / pair_ms, "unit": "HVPs/s", "ms_per_call": pair_ms,
            "window": pinfo["window"], "device_mib": pinfo["device_mib"],
            "one_direction_sweeps_same_window": {"value": 2000.0 / same_ms, "ms_per_call": same_ms},
            "one_direction_sweeps_default_plan": {"value": 2000.0 / best_ms, "ms_per_call": best_ms,
                                                  "window": binfo["window"]}}

    # -------------- the schedule the autotuner did not pick, same workload
    other = None
    if not args.no_other and rank == 0:
        key = "window_passes" if tensor_plan else "tensor_blocks"
        line[key], other = schedule_line(native, torch, dev, local, w, max(3, min(args.steps, 10)), m_or,
                                         not tensor_plan)

    # --------------- n = 12 precision comparison and n = 26 autograd form
    if not args.no_configs and rank == 0:
        line["n12_precision"] = n12_precision_line(native, make_workload, torch, dev, local)
        line["n26_autograd"] = n26_autograd_line(make_workload, torch, dev, local)

    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cb = cpu_baseline(w)
        line["cpu_baseline"] = {k: v for k, v in cb.items() if k not in ("seconds_per_step", "steps", "oracle_out")}
        # Parity of the timed configuration (and of the other schedule's line)
        # against the same oracle run, on the samples it covered.
        o, m = cb["oracle_out"], cb["cores"]
        pv = line["parity_vs_oracle"] = parity_check(par, o, m)
        if other is not None:
            tp = line[key]["parity_vs_oracle"] = parity_check(other, o, m)
            pv["pass"] = pv["pass"] and tp["pass"]
    if rank == 0:
        print(json.dumps(line), flush=True)
        if not line.get("parity_vs_oracle", {}).get("pass", True):
            print("bench: timed configuration disagrees with the oracle", file=sys.stderr, flush=True)
            return 1
    if dist:
        dist.barrier()
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
