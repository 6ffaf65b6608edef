#!/usr/bin/env python3
"""Benchmark of the fused LB-MHD stream-collide step (MLUPS and fraction of
the HBM roofline).

Workload (default): decaying 2D MHD turbulence on an 8192 x 8192 periodic
lattice (random-phase modes 4 <= |k| <= 8, rms 0.04, C_S = 0.1,
tau = 0.51), FP32 storage and arithmetic, 500 steps timed after warm-up.
The state (10 GB per buffer) is far larger than L2, so no flush is needed
between steps.  The same run also times, on the same lattice, the paper's
kinetic LES (les = 2; the fused one-launch kernel and the two-pass
kernels), the FP64, double-word (FF), FP32-deviation and FP16-deviation
storage forms (fewer steps), an end-to-end pass through the host C ABI
(host fields in, host moments out), the 256-run ensemble, the adjoint
(gradients), and the CPU oracle on a bounded sample.

One JSON line is printed by rank 0.  Under torchrun each rank advances its
own independent lattice (different seed; weak scaling, no data exchange);
the timed region is bracketed by a barrier and the maximum over ranks is
reported.

``--impl reference`` times the FP64 CPU oracle instead, on a bounded
sample (a 512 x 512 lattice of the same recipe) on the host cores.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "MLUPS and % of GB300 HBM roofline, plain FP64 vs FP32/batched vs FP64 oracle"
WORKLOAD = ("decaying 2D MHD turbulence 8192x8192, modes 4<=|k|<=8 rms 0.04, C_S=0.1, tau=0.51, "
            "s5=s6=1.2, s7=s8=1.3")
DTYPES = {"fp64": "f64", "fp32": "f32", "fp32_dev": "f32 (f32 deviation storage)",
          "fp16_dev": "f32 (f16 deviation storage)",
          "ff": "double-word f32 pairs (48-bit significand), storage and arithmetic"}
# Free MRT rates of the turbulence runs (the paper leaves s_5..s_8 open).
# Tying them to s_nu (the BGK-equivalent choice) is unstable at tau = 0.51
# in developed MHD turbulence: a 1e-12 perturbation reaches 9% in 300 steps
# at 512^2 without LES, while with these rates it stays at 1e-11.
TURB_RATES = dict(s5=1.2, s6=1.2, s7=1.3, s8=1.3)


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clock / throttle samples while the timed region runs."""

    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, dev_id: str):
        self.dev_id = dev_id
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", self.dev_id, f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.t.join(timeout=2)

    def summary(self):
        rows = []
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) != 7:
                continue
            try:
                rows.append((float(parts[0]), float(parts[1]), parts[3:]))
            except ValueError:
                continue
        if not rows:
            return None
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for _, _, r in rows for i, v in enumerate(r)
                          if v.lower() == "active"})
        return {"sm_mhz": statistics.median(r[0] for r in rows),
                "sm_max_mhz": max(r[1] for r in rows), "reasons": reasons,
                "samples": len(rows)}


def dev_id_for_smi():
    import torch

    try:
        props = torch.cuda.get_device_properties(torch.cuda.current_device())
        return "%08x:%02x:%02x.0" % (props.pci_domain_id, props.pci_bus_id, props.pci_device_id)
    except Exception:
        vis = os.environ.get("CUDA_VISIBLE_DEVICES", "0").split(",")[0]
        return vis if vis.isdigit() else "0"


def cpu_count():
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count() or 1


# The oracle's sample of the bench workload: one lattice of the same
# turbulence recipe and rates for the cpu_baseline figures and for the
# reference arm (the 8192^2 lattice does not fit the oracle's time budget).
ORACLE_SAMPLE_N = 512


def cpu_model():
    """The host CPU's model name (lscpu, else /proc/cpuinfo)."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.strip().startswith("Model name:"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    try:
        for line in open("/proc/cpuinfo"):
            if line.lower().startswith(("model name", "cpu model")):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    return "unknown"


def oracle_sample():
    from oracle import oracle
    from paper_1607_08675_gb300 import inputs

    oracle.build()
    n = ORACLE_SAMPLE_N
    p = oracle.params(tau_nu=0.51, tau_eta=0.51, C_S=0.1, **TURB_RATES)
    return oracle, p, oracle.init(*inputs.turbulence(n, n, seed=1))


def time_oracle(budget_s: float = 15.0):
    """The FP64 CPU oracle, as it stands, on the ORACLE_SAMPLE_N^2 sample:
    one thread for a third of the budget, then every host core (the same
    bits either way).  Returns a cpu_baseline record."""
    oracle, p, st = oracle_sample()
    n = ORACLE_SAMPLE_N
    cores = cpu_count()
    out = {}
    for key, threads, share in (("value_1thread", 1, 1 / 3), ("value_allcores", cores, 2 / 3)):
        t0 = time.perf_counter()
        st = oracle.step(st, p, 1, nthreads=threads)
        one = time.perf_counter() - t0
        steps = max(1, int(budget_s * share / max(one, 1e-6)))
        t0 = time.perf_counter()
        st = oracle.step(st, p, steps, nthreads=threads)
        dt = time.perf_counter() - t0
        out[key] = n * n * steps / dt / 1e6
        out[key.replace("value", "steps")] = steps
        out[key.replace("value", "seconds")] = dt
    return {"value": out["value_allcores"], "unit": "MLUPS", "cores": cores, "kind": "oracle",
            "cpu_model": cpu_model(), **out,
            "sample": f"{n}x{n} lattice of the same turbulence recipe and rates, FP64 oracle "
                      f"steps on 1 thread and on {cores} threads (value = all cores)"}


def run_reference(args):
    """The reference arm: the FP64 CPU oracle, as it stands, on the host
    cores.  One bench step is one oracle step on a sample lattice of the
    same recipe, sized so that the whole --warmup W --steps K run takes about
    two minutes."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    oracle, p, st = oracle_sample()
    n = ORACLE_SAMPLE_N
    cores = cpu_count()
    st = oracle.step(st, p, args.warmup, nthreads=cores)
    t0 = time.perf_counter()
    oracle.step(st, p, args.steps, nthreads=cores)
    dt = time.perf_counter() - t0
    value = n * n * args.steps / dt / 1e6
    sample = (f"{n}x{n} lattice of the same turbulence recipe per step (the 8192^2 "
              f"lattice does not fit the oracle's time budget), FP64 oracle, {cores} threads; "
              "the same sample as the GPU arm's cpu_baseline")
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": "MLUPS",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * dt / max(1, args.steps), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "sample": sample},
        "cpu_baseline": {"value": value, "unit": "MLUPS", "cores": cores, "kind": "oracle",
                         "cpu_model": cpu_model(), "sample": sample},
        "e2e": {"value": value, "unit": "MLUPS", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }), flush=True)


def max_over_ranks(x: float, dist=None) -> float:
    """Largest value of x over the ranks of the default process group (x
    itself without one).  Works over NCCL (CUDA tensor) and gloo (CPU)."""
    if dist is None or not dist.is_initialized():
        return x
    import torch

    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([float(x)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(world: int, cells_per_rank: int, steps: int, seconds: float) -> float:
    """Whole-job MLUPS of `world` independent lattices timed together (weak
    scaling): all ranks' node updates over the slowest rank's time."""
    return world * cells_per_rank * steps / seconds / 1e6


def kernel_source_hash() -> str:
    """Hash of the step kernel's sources: DRAM counters taken from another
    version of the kernel are not reported."""
    import hashlib

    h = hashlib.sha256()
    for f in ("lbmhd_step.cu", "lbmhd_step_body.cuh", "lbmhd_device.cuh"):
        with open(os.path.join(ROOT, "paper_1607_08675_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def measured_traffic(prec: str, cells: int):
    """ncu DRAM bytes (read + write) per launch for this lattice, from
    profiles/step_kernel_traffic.txt ("source <hash>" and "<precision>
    <bytes per node>" lines), or None when absent or stale."""
    path = os.path.join(ROOT, "profiles", "step_kernel_traffic.txt")
    try:
        with open(path) as fh:
            rows = [ln.split() for ln in fh if ln.strip() and not ln.startswith("#")]
    except OSError:
        return None
    kv = {r[0]: r[1] for r in rows if len(r) >= 2}
    if kv.get("source") != kernel_source_hash() or prec not in kv:
        return None
    return float(kv[prec]) * cells


def run_batched(L, args, stream, rank, hbm, barrier, max_over_ranks):
    """The ensemble workload: 256 runs with sizes drawn among {128, 256, 512,
    1024}^2, own seeds, C_S in [0.05, 0.2], tau in [0.51, 0.7]; FP32; one
    persistent kernel (autotuned shape) under a CUDA graph, against the same
    runs advanced one after another by their own single-lattice launches."""
    import torch

    from paper_1607_08675_gb300 import inputs

    runs = inputs.ensemble(nruns=args.batch_runs, seed=7 + rank)
    nx = [r["nx"] for r in runs]
    ny = [r["ny"] for r in runs]
    tau = [r["tau"] for r in runs]
    cs = [r["C_S"] for r in runs]
    cells = sum(a * b for a, b in zip(nx, ny))
    steps = args.batch_steps
    b = L.lbmhd_batch_create(nx, ny, tau, tau, cs,
                             L.lbmhd_params_default(precision="fp32", stream=stream,
                                                    **TURB_RATES))
    tuned = L.lbmhd_batch_autotune(b, None, 8)
    shape = L.lbmhd_batch_get_launch(b)
    for i, r in enumerate(runs):
        f = inputs.turbulence(r["nx"], r["ny"], seed=r["seed"])
        L.lbmhd_batch_init(b, i, *f)
    L.lbmhd_batch_step(b, 16)
    barrier()
    l0 = L.lbmhd_batch_launch_count(b)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    L.lbmhd_batch_step(b, steps)
    e1.record(stream)
    e1.synchronize()
    L.lbmhd_batch_sync(b)
    t_batch = max_over_ranks(e0.elapsed_time(e1) / 1e3)
    launches = L.lbmhd_batch_launch_count(b) - l0
    L.lbmhd_batch_destroy(b)
    # the same runs, one lattice at a time, each by its own launches
    t_seq = 0.0
    for i, r in enumerate(runs):
        h = L.lbmhd_create(r["nx"], r["ny"], L.lbmhd_params_default(
            precision="fp32", tau_nu=r["tau"], tau_eta=r["tau"], C_S=r["C_S"], stream=stream,
            **TURB_RATES))
        L.lbmhd_init(h, *inputs.turbulence(r["nx"], r["ny"], seed=r["seed"]))
        L.lbmhd_step(h, 3)
        a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a0.record(stream)
        L.lbmhd_step(h, steps)
        a1.record(stream)
        a1.synchronize()
        t_seq += a0.elapsed_time(a1) / 1e3
        L.lbmhd_destroy(h)
    t_seq = max_over_ranks(t_seq)
    world = int(os.environ.get("WORLD_SIZE", "1"))
    mlups = world * cells * steps / t_batch / 1e6
    # the same ensemble with the paper's kinetic LES (les = 2, Delta = 2):
    # the fused kernel over every run's strip-segments, one launch per step
    # (152 B/node), against the runs one after another with their own
    # single-lattice launches of the same kernel; at least MIN_LEG_S of
    # device time
    kw = dict(TURB_RATES, les=2, delta=2.0)
    kb = L.lbmhd_batch_create(nx, ny, tau, tau, cs,
                              L.lbmhd_params_default(precision="fp32", stream=stream, **kw))
    kshape = L.lbmhd_batch_get_launch(kb)
    for i, r in enumerate(runs):
        L.lbmhd_batch_init(kb, i, *inputs.turbulence(r["nx"], r["ny"], seed=r["seed"]))
    L.lbmhd_batch_step(kb, 8)
    barrier()
    e0.record(stream)
    L.lbmhd_batch_step(kb, 4)
    e1.record(stream)
    e1.synchronize()
    ksteps = steps_for(e0.elapsed_time(e1) / 1e3 / 4)
    e0.record(stream)
    L.lbmhd_batch_step(kb, ksteps)
    e1.record(stream)
    e1.synchronize()
    L.lbmhd_batch_sync(kb)
    tk_batch = max_over_ranks(e0.elapsed_time(e1) / 1e3)
    L.lbmhd_batch_destroy(kb)
    tk_seq = 0.0
    for i, r in enumerate(runs):
        h = L.lbmhd_create(r["nx"], r["ny"], L.lbmhd_params_default(
            precision="fp32", tau_nu=r["tau"], tau_eta=r["tau"], C_S=r["C_S"], stream=stream,
            **kw))
        L.lbmhd_init(h, *inputs.turbulence(r["nx"], r["ny"], seed=r["seed"]))
        L.lbmhd_step(h, 3)
        a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a0.record(stream)
        L.lbmhd_step(h, ksteps)
        a1.record(stream)
        a1.synchronize()
        tk_seq += a0.elapsed_time(a1) / 1e3
        L.lbmhd_destroy(h)
    tk_seq = max_over_ranks(tk_seq)
    kinetic = {"MLUPS": world * cells * ksteps / tk_batch / 1e6,
               "sequential_MLUPS": world * cells * ksteps / tk_seq / 1e6,
               "speedup": tk_seq / tk_batch, "steps": ksteps, "seconds": tk_batch,
               "hbm_frac": cells * ksteps * 152 / tk_batch / 1e9 / hbm,
               "kernel": "fused" if kshape[0] == 1 else "two-pass",
               "note": "les=2 ensemble: the fused kernel over every run's strip-segments, one "
                       "launch per step (152 B/node), vs the runs one by one with the fused "
                       "single-lattice kernel"}
    return {"MLUPS": mlups, "sequential_MLUPS": world * cells * steps / t_seq / 1e6,
            "kinetic_les": kinetic,
            "speedup": t_seq / t_batch, "runs": len(runs), "cells": cells, "steps": steps,
            "launch": {"vec": shape[0], "block": shape[1], "steps_per_launch": shape[2]},
            "autotune_trial_MLUPS": tuned, "persistent_launches": int(launches),
            "hbm_frac": cells * steps * 152 / t_batch / 1e9 / hbm,
            "sizes": {str(k): nx.count(k) for k in sorted(set(nx))}}


def run_adjoint(args):
    """The gradient workload: Orszag-Tang 512^2 with the seeded perturbation,
    tau_nu = tau_eta = 0.6, trial C_S = 0.1; loss = 1/2 sum |u - u_ref|^2 +
    |B - B_ref|^2 against a run with C_S = 0.12 after 500 steps; FP32
    forward with FP64 checkpoints every 50 steps, hand-written adjoint
    backward.  Checked against the FP64 adjoint and a central finite
    difference of the FP64 forward in C_S."""
    import torch

    from paper_1607_08675_gb300 import autograd as AG, inputs, lbmhd as L

    n, steps, every = args.adj_n, args.adj_steps, 50
    f = [torch.tensor(a, dtype=torch.float64, device="cuda")
         for a in inputs.orszag_tang(n, n, seed=0)]
    refs = {}
    with torch.no_grad():
        for prec in ("fp32", "ff", "fp64"):  # the reference run in the trial's precision
            refs[prec] = AG.rollout(*f, 0.12, 0.6, 0.6, steps, every=every, precision=prec)

    def loss_of(out, prec="fp64"):
        return 0.5 * sum(((o - r) ** 2).sum() for o, r in zip(out[1:], refs[prec][1:]))

    # one untimed pass of the whole gradient path (library and torch kernels load)
    w = [t.clone().requires_grad_(True) for t in f]
    loss_of(AG.rollout(*w, 0.1, 0.6, 0.6, 2 * every, every=every, precision="fp32"),
            "fp32").backward()
    res = {}
    for prec in ("fp32", "ff", "fp64"):
        leaves = [t.clone().requires_grad_(True) for t in f]
        th = [torch.tensor(v, dtype=torch.float64, requires_grad=True) for v in (0.1, 0.6, 0.6)]
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        out = AG.rollout(*leaves, *th, steps, every=every, precision=prec)
        loss = loss_of(out, prec)
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        loss.backward()
        torch.cuda.synchronize()
        t2 = time.perf_counter()
        res[prec] = {"loss": loss.item(), "dC_S": th[0].grad.item(),
                     "dtau_nu": th[1].grad.item(), "dtau_eta": th[2].grad.item(),
                     "du0_norm": float(torch.linalg.norm(torch.stack([l.grad for l in leaves[1:3]]))),
                     "dB0_norm": float(torch.linalg.norm(torch.stack([l.grad for l in leaves[3:5]]))),
                     "forward_s": t1 - t0, "backward_s": t2 - t1}
    h = 1e-6 * 0.1
    with torch.no_grad():
        lp = loss_of(AG.rollout(*f, 0.1 + h, 0.6, 0.6, steps, every=every)).item()
        lm = loss_of(AG.rollout(*f, 0.1 - h, 0.6, 0.6, steps, every=every)).item()
    fd = (lp - lm) / (2 * h)
    r64, r32 = res["fp64"], res["fp32"]
    return {"workload": f"Orszag-Tang {n}x{n}, {steps} steps, checkpoints every {every}, "
                        "loss vs C_S = 0.12 run",
            "fp32": r32, "ff": res["ff"], "fp64": r64, "fd_dC_S": fd,
            "fd_rel_err_fp64": abs(r64["dC_S"] - fd) / abs(fd),
            "fp32_vs_fp64_rel": {k: abs(r32[k] - r64[k]) / abs(r64[k])
                                 for k in ("dC_S", "dtau_nu", "dtau_eta", "du0_norm", "dB0_norm")},
            "ff_vs_fp64_rel": {k: abs(res["ff"][k] - r64[k]) / abs(r64[k])
                               for k in ("dC_S", "dtau_nu", "dtau_eta", "du0_norm", "dB0_norm")},
            "node_steps_per_s_fp32": n * n * steps / (r32["forward_s"] + r32["backward_s"])}


def shell_spectrum(a, b):
    """Shell-binned spectrum E(k) = 1/2 sum_{k-1/2 <= |k| < k+1/2} |FFT|^2 / N^2 of
    the planar field (a, b)."""
    import numpy as np

    ny, nx = a.shape
    fa, fb = np.fft.fft2(a) / (nx * ny), np.fft.fft2(b) / (nx * ny)
    e = 0.5 * (np.abs(fa) ** 2 + np.abs(fb) ** 2)
    kx = np.fft.fftfreq(nx, 1.0 / nx)
    ky = np.fft.fftfreq(ny, 1.0 / ny)
    k = np.rint(np.sqrt(kx[None, :] ** 2 + ky[:, None] ** 2)).astype(int)
    return np.bincount(k.ravel(), weights=e.ravel())


def field_errors(got, ref):
    """Per field (rho-1, ux, uy, bx, by): max and rms error relative to the
    reference field's max and rms."""
    import numpy as np

    out = {}
    for name, a, b in zip(("rho-1", "ux", "uy", "bx", "by"), got, ref):
        if name == "rho-1":
            a, b = a - 1.0, b - 1.0
        d = a - b
        out[name] = {"max": float(np.max(np.abs(d)) / np.max(np.abs(b))),
                     "rms": float(np.sqrt(np.mean(d * d)) / np.sqrt(np.mean(b * b)))}
    return out


def spectrum_errors(got, ref, kmax=64):
    import numpy as np

    res = {}
    for name, (i, j) in (("E_K", (1, 2)), ("E_M", (3, 4))):
        eg, er = shell_spectrum(got[i], got[j])[1:kmax], shell_spectrum(ref[i], ref[j])[1:kmax]
        res[name] = float(np.max(np.abs(eg - er) / np.maximum(er, 1e-300)))
    return res


def precision_study(args):
    """Errors of every field of the reduced-precision forms.
    (1) 1024^2 turbulence, 2000 steps, against the FP64 CPU oracle (fields and
        shell spectra up to |k| = 64); the FP64 GPU run is included.
    (2) 8192^2 turbulence, 500 steps, against the FP64 GPU run (which matches
        the oracle to 1e-12 where the oracle can run)."""
    import torch

    from oracle import oracle
    from paper_1607_08675_gb300 import build, lbmhd as L

    build.build()
    oracle.build()
    torch.cuda.set_device(0)
    kw = dict(tau_nu=0.51, tau_eta=0.51, C_S=0.1, **TURB_RATES)
    precs = ("fp64", "ff", "fp32", "fp32_dev", "fp16_dev")

    def gpu_run(n, fields, steps, prec):
        h = L.lbmhd_create(n, n, L.lbmhd_params_default(precision=prec, **kw))
        L.lbmhd_init(h, *fields)
        L.lbmhd_step(h, steps)
        m = L.lbmhd_moments(h)
        L.lbmhd_destroy(h)
        return m

    n, steps = args.study_n1, args.study_steps1
    fields = make_fields(n, 1)
    t0 = time.perf_counter()
    ref = oracle.moments(oracle.step(oracle.init(*fields), oracle.params(**kw), steps,
                                     nthreads=cpu_count()))
    t_orc = time.perf_counter() - t0
    for prec in precs:
        m = gpu_run(n, fields, steps, prec)
        print(json.dumps({"study": f"turbulence {n}x{n}, {steps} steps, vs FP64 CPU oracle",
                          "precision": prec, "fields": field_errors(m, ref),
                          "spectra_max_rel": spectrum_errors(m, ref),
                          "oracle_seconds": t_orc}), flush=True)
    n, steps = args.study_n2, args.study_steps2
    fields = make_fields(n, 1)
    ref = gpu_run(n, fields, steps, "fp64")
    for prec in precs[1:]:
        m = gpu_run(n, fields, steps, prec)
        print(json.dumps({"study": f"turbulence {n}x{n}, {steps} steps, vs FP64 GPU run",
                          "precision": prec, "fields": field_errors(m, ref)}), flush=True)


def make_fields(n, seed):
    from paper_1607_08675_gb300 import inputs

    return inputs.turbulence(n, n, seed=seed)


def timed_steps(L, h, stream, steps, warmup):
    """Device time (s) of `steps` steps on the handle's stream, after warm-up."""
    import torch

    L.lbmhd_step(h, warmup)
    stream.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    L.lbmhd_step(h, steps)
    e1.record(stream)
    e1.synchronize()
    return e0.elapsed_time(e1) / 1e3


# Every secondary leg times at least this much device time, whatever --steps
# is, so that its figure does not hang on a handful of launches.
MIN_LEG_S = 0.1


def steps_for(seconds_per_step, min_s=MIN_LEG_S, floor=2):
    """Steps that fill min_s of device time at the probed rate."""
    return max(floor, int(math.ceil(min_s / max(seconds_per_step, 1e-9))))


def timed_leg(L, h, stream, warmup, max_over_ranks_, step=None):
    """(steps, seconds) of a leg timed for at least MIN_LEG_S: a 2-step probe
    after the warm-up sets the step count; max over ranks.  step: the step
    call (default lbmhd_step)."""
    import torch

    step = step or L.lbmhd_step

    def run(n):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        step(h, n)
        e1.record(stream)
        e1.synchronize()
        return e0.elapsed_time(e1) / 1e3

    step(h, warmup)
    stream.synchronize()
    steps = steps_for(run(2) / 2)
    return steps, max_over_ranks_(run(steps))


def run_ours(args):
    import numpy as np
    import torch

    from paper_1607_08675_gb300 import build, lbmhd as L

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    if rank == 0:
        build.build()
    if dist:
        dist.barrier()
    L.lib()

    n = args.n
    fields = make_fields(n, seed=1 + rank)
    stream = torch.cuda.Stream()
    kw = dict(tau_nu=0.51, tau_eta=0.51, C_S=0.1, stream=stream, **TURB_RATES)
    hbm, peak_kind = peaks()

    def barrier():
        torch.cuda.synchronize()
        if dist:
            dist.barrier()

    def max_over_ranks_(x):
        return max_over_ranks(x, dist)

    # ---- headline: the chosen precision -----------------------------------
    prec = args.precision
    h = L.lbmhd_create(n, n, L.lbmhd_params_default(precision=prec, **kw))
    L.lbmhd_init(h, *fields)
    L.lbmhd_step(h, args.warmup)
    barrier()
    launches0 = L.lbmhd_launch_count(h)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(dev_id_for_smi()) as clk:
        barrier()
        e0.record(stream)
        L.lbmhd_step(h, args.steps)
        e1.record(stream)
        e1.synchronize()
        barrier()
    dt = max_over_ranks_(e0.elapsed_time(e1) / 1e3)
    launches = L.lbmhd_launch_count(h) - launches0
    L.lbmhd_sync(h)
    cells = n * n
    value = job_rate(world, cells, args.steps, dt)
    bpc = L.lbmhd_bytes_per_cell(prec)
    per_launch_s = (e0.elapsed_time(e1) / 1e3) / args.steps
    achieved = bpc * cells / per_launch_s / 1e9
    L.lbmhd_destroy(h)
    del h

    # ---- other storage forms on the same lattice ---------------------------
    variants = {}
    if not args.no_variants:
        # the paper's kinetic LES, FP32: the fused one-launch kernel (default;
        # algorithmic bytes per node 19 reads + 19 writes, as a plain step) and
        # the two-pass kernels (19 reads + 5 writes, 19 + 5 reads + 19 writes)
        # and the cross-helicity closure (les = 3) with the fused kernel
        for kname, kles, kvec, kbytes in (("fp32_kinetic_les", 2, 1, 152),
                                          ("fp32_kinetic_les_two_pass", 2, 0, 268),
                                          ("fp32_cross_helicity", 3, 1, 152)):
            hk = L.lbmhd_create(n, n, L.lbmhd_params_default(
                precision="fp32", **dict(kw, les=kles, delta=2.0)))
            L.lbmhd_set_launch(hk, kvec, 256)
            L.lbmhd_init(hk, *fields)
            barrier()
            ksteps, t = timed_leg(L, hk, stream, max(3, args.warmup // 10), max_over_ranks_)
            L.lbmhd_destroy(hk)
            what = ("les=2 (filtered equilibria, Delta=2), " if kles == 2 else
                    "les=3 (cross-helicity closure, Delta=2), ")
            variants[kname] = {
                "MLUPS": world * cells * ksteps / t / 1e6, "steps": ksteps, "seconds": t,
                "bytes_per_cell": kbytes,
                "hbm_frac": kbytes * cells * ksteps / t / 1e9 / hbm,
                "note": what + ("fused: one launch per step" if kvec else "moments pass + step")}
        for vp in ("fp64", "ff", "fp32_dev", "fp16_dev"):
            if vp == prec:
                continue
            hv = L.lbmhd_create(n, n, L.lbmhd_params_default(precision=vp, **kw))
            L.lbmhd_init(hv, *fields)
            barrier()
            vsteps, t = timed_leg(L, hv, stream, max(3, args.warmup // 10), max_over_ranks_)
            L.lbmhd_destroy(hv)
            vb = L.lbmhd_bytes_per_cell(vp)
            variants[vp] = {
                "MLUPS": world * cells * vsteps / t / 1e6, "steps": vsteps, "seconds": t,
                "bytes_per_cell": vb,
                "hbm_frac": vb * cells * vsteps / t / 1e9 / hbm,
            }

    # ---- the 3D extension (D3Q27 + D3Q7 vector), decaying 3D turbulence -----
    # 45 values read and written per node: 360 B (FP32), 720 B (FP64)
    variants3d = {}
    if not args.no_variants:
        from paper_1607_08675_gb300 import inputs

        for vp, n3 in (("fp32", args.n3), ("fp16_dev", args.n3), ("fp64", max(16, args.n3 // 2)),
                       ("ff", max(16, args.n3 // 2))):
            h3 = L.lbmhd3_create(n3, n3, n3, L.lbmhd_params_default(
                precision=vp, tau_nu=0.51, tau_eta=0.51, C_S=0.1, les=1, stream=stream))
            L.lbmhd3_init(h3, *inputs.turbulence3d(n3, n3, n3, seed=1 + rank))
            barrier()
            s3, t = timed_leg(L, h3, stream, 3, max_over_ranks_, step=L.lbmhd3_step)
            b3 = L.lbmhd3_bytes_per_cell(vp)
            L.lbmhd3_destroy(h3)
            variants3d[vp] = {
                "MLUPS": world * n3 ** 3 * s3 / t / 1e6, "steps": s3, "seconds": t,
                "lattice": f"{n3}^3", "bytes_per_cell": b3,
                "hbm_frac": b3 * n3 ** 3 * s3 / t / 1e9 / hbm,
                "note": "3D decaying turbulence (band 2 <= |n| <= 4, rms 0.04), local LES rates"}
        # the gradient closures, fraction at the one-pass bound of 360 B/node:
        # the warp-specialised kernel (default), the fused kernel with two
        # barriers per plane, and the two-pass kernels (a moments pass reading
        # 45 planes and writing 7, then the step: 596 B/node)
        kernel_names = {0: "fused", 1: "two-pass", 2: "two-pass", 3: "warp-specialised"}
        for name, les, launch in (("fp32_kinetic_les", 2, None), ("fp32_cross_helicity", 3, None),
                                  ("fp32_kinetic_les_fused", 2, (0, 4)),
                                  ("fp32_kinetic_les_two_pass", 2, (2, 128))):
            n3 = args.n3
            h3 = L.lbmhd3_create(n3, n3, n3, L.lbmhd_params_default(
                precision="fp32", tau_nu=0.51, tau_eta=0.51, C_S=0.1, delta=2.0, les=les,
                stream=stream))
            if launch:
                L.lbmhd3_set_launch(h3, *launch)
            kname = kernel_names[L.lbmhd3_get_launch(h3)[0]]
            L.lbmhd3_init(h3, *inputs.turbulence3d(n3, n3, n3, seed=1 + rank))
            barrier()
            s3, t = timed_leg(L, h3, stream, 3, max_over_ranks_, step=L.lbmhd3_step)
            L.lbmhd3_destroy(h3)
            b3 = L.lbmhd3_bytes_per_cell("fp32")
            variants3d[name] = {
                "MLUPS": world * n3 ** 3 * s3 / t / 1e6, "steps": s3, "seconds": t,
                "lattice": f"{n3}^3", "bytes_per_cell": b3,
                "hbm_frac": b3 * n3 ** 3 * s3 / t / 1e9 / hbm,
                "kernel": kname,
                "note": ("the paper's filtered equilibria" if les == 2 else
                         "cross-helicity closure") + (", moments pass + step" if kname == "two-pass"
                                                      else ", one launch per step")}

    # ---- the FP64 diagnostics reduction on the same lattice ----------------
    # algorithmic bytes: the 19 stored planes, read once (the tiles' halo
    # rows come from L2)
    diagnostics = None
    if not args.no_variants:
        hd = L.lbmhd_create(n, n, L.lbmhd_params_default(precision=prec, **kw))
        L.lbmhd_init(hd, *fields)
        L.lbmhd_step(hd, 2)
        L.lbmhd_diagnostics(hd)
        barrier()
        d0, d1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        reps = 2
        for attempt in range(2):  # a probe, then enough calls for MIN_LEG_S
            d0.record(stream)
            for _ in range(reps):
                L.lbmhd_diagnostics(hd)
            d1.record(stream)
            d1.synchronize()
            t = d0.elapsed_time(d1) / 1e3 / reps
            if attempt == 0:
                reps = steps_for(t)
        t = max_over_ranks_(t)
        L.lbmhd_destroy(hd)
        dbytes = L.lbmhd_bytes_per_cell(prec) // 2
        diagnostics = {"ms": 1e3 * t, "calls": reps, "seconds": t * reps,
                       "bytes_per_cell": dbytes,
                       "GBps": dbytes * cells / t / 1e9, "hbm_frac": dbytes * cells / t / 1e9 / hbm,
                       "note": "lbmhd_diagnostics (12 FP64 sums, div B, |j|^2) of the "
                               f"{prec} state, per call"}

    # ---- end to end through the host C ABI --------------------------------
    e2e = None
    if not args.no_e2e:
        he = L.lbmhd_create(n, n, L.lbmhd_params_default(precision=prec, **kw))
        # the inputs and outputs live in pinned host memory, as a serving
        # caller would keep them
        pin_in = [torch.from_numpy(a).pin_memory().numpy() for a in fields]
        pin_out = [torch.empty((n, n), dtype=torch.float64).pin_memory().numpy()
                   for _ in range(5)]
        L.lbmhd_init(he, *pin_in)  # allocate/warm the path once
        L.lbmhd_step(he, 3)
        L.lbmhd_moments_into(he, *pin_out)
        barrier()
        t0 = time.perf_counter()
        L.lbmhd_init(he, *pin_in)
        L.lbmhd_step(he, args.steps)
        L.lbmhd_moments_into(he, *pin_out)
        t_e2e = max_over_ranks_(time.perf_counter() - t0)
        L.lbmhd_destroy(he)
        assert all(np.isfinite(a).all() for a in pin_out)
        e2e = {"value": world * cells * args.steps / t_e2e / 1e6, "unit": "MLUPS",
               "h2d_bytes_per_step": 5 * 8 * cells / args.steps,
               "d2h_bytes_per_step": 5 * 8 * cells / args.steps,
               "job": f"lbmhd_init (5 pinned host FP64 fields) + lbmhd_step({args.steps}) + "
                      "lbmhd_moments (5 pinned host FP64 fields); bytes amortised per step"}

    # ---- gradients through the hand-written adjoint ------------------------
    adjoint = None
    if not args.no_adjoint and rank == 0:
        adjoint = run_adjoint(args)

    # ---- batched ensemble vs sequential per-run launches --------------------
    batched = None
    if not args.no_batch:
        batched = run_batched(L, args, stream, rank, hbm, barrier, max_over_ranks_)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        cpu = time_oracle(budget_s=args.cpu_budget)

    traffic = measured_traffic(prec, cells)

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "MLUPS", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": DTYPES[prec].split(" ")[0], "data": "synthetic",
            "config": {"workload": WORKLOAD, "nx": n, "ny": n, "precision": prec,
                       "storage": DTYPES[prec],
                       "l2": "state larger than L2 (%.1f GB per buffer), no flush"
                             % (bpc / 2 * cells / 1e9),
                       "parallelism": f"{world} independent lattice(s), one per GPU"},
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s",
                         "frac": achieved / hbm, "traffic": traffic,
                         "peak_source": f"{peak_kind} copy bandwidth (MEASURED_PEAKS.json)",
                         "bytes_per_cell": bpc},
            "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": int(launches),
            "diagnostics": diagnostics,
            "clocks": clk.summary(), "variants": variants, "variants_3d": variants3d,
            "batched": batched,
            "adjoint": adjoint,
        }
        print(json.dumps(line), flush=True)
    if dist:
        dist.barrier()
        dist.destroy_process_group()


def run_decomp(args):
    """One n x n lattice cut into row slabs (decomp.SlabRunner): slab s on
    rank s * world // k, halos over NCCL between ranks (decomp.exchange), the
    rows that need no ghost row computed while the halo is in flight.  Every
    rank times the same steps; value = lattice node updates per second of the
    job (strong scaling: the lattice is fixed as ranks are added)."""
    import torch

    from paper_1607_08675_gb300 import build, decomp, lbmhd as L

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    if rank == 0:
        build.build()
    if dist:
        dist.barrier()
    L.lib()
    n, prec = args.n, args.precision
    k = args.decomp_slabs or world
    owner = [s * world // k for s in range(k)]
    mine = [s for s in range(k) if owner[s] == rank]
    kw = dict(tau_nu=0.51, tau_eta=0.51, C_S=0.1, precision=prec, **TURB_RATES)
    if args.les:
        kw.update(les=args.les, delta=2.0)
    runner = decomp.SlabRunner(n, n, k, slabs=mine,
                               comm=decomp.DistComm(owner) if world > 1 else None,
                               overlap=not args.no_overlap, **kw)
    runner.init(*make_fields(n, seed=1))
    hbm, _ = peaks()

    def barrier():
        torch.cuda.synchronize()
        if dist:
            dist.barrier()

    runner.step(args.warmup)
    barrier()
    launches0 = sum(L.lbmhd_launch_count(h) for h in runner.h.values())
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(dev_id_for_smi()) as clk:
        barrier()
        e0.record(runner.main)
        runner.step(args.steps)
        e1.record(runner.main)
        e1.synchronize()
        barrier()
    mine_t = e0.elapsed_time(e1) / 1e3
    dt = max_over_ranks(mine_t, dist)
    launches = sum(L.lbmhd_launch_count(h) for h in runner.h.values()) - launches0
    my_rows = sum(runner.rows[s][1] - runner.rows[s][0] for s in mine)
    per_rank = n * my_rows * args.steps / mine_t / 1e6
    rates = [per_rank]
    if dist:
        t = torch.tensor([per_rank], dtype=torch.float64, device="cuda")
        out = [torch.zeros_like(t) for _ in range(world)]
        dist.all_gather(out, t)
        rates = [float(x.item()) for x in out]
    vb = L.lbmhd_bytes_per_cell(prec) // 38
    halo_total = decomp.halo_bytes_per_step(n, n, k, args.les or 1, vb)
    value = n * n * args.steps / dt / 1e6
    bpc = L.lbmhd_bytes_per_cell(prec)
    runner.sync()
    runner.close()
    if rank == 0:
        print(json.dumps({
            "metric": METRIC, "value": value, "unit": "MLUPS", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps,
            "higher_is_better": True, "scaling": "strong", "vs_baseline": None,
            "dtype": DTYPES[prec].split(" ")[0], "data": "synthetic",
            "config": {"workload": WORKLOAD + ", one lattice cut into row slabs",
                       "nx": n, "ny": n, "precision": prec, "les": args.les or 1,
                       "parallelism": f"y-slab decomposition: {k} slab(s) over {world} rank(s)",
                       "l2": "state larger than L2, no flush"},
            "decomp": {"slabs": k, "ranks": world, "overlap": not args.no_overlap,
                       "halo_bytes_per_step": halo_total,
                       "halo_bytes_per_step_rank0": runner_halo(n, k, mine, args.les or 1, vb),
                       "per_rank_MLUPS": rates,
                       "hbm_frac_of_job": value * 1e6 * bpc / 1e9 / hbm / world},
            "gpu_launches": int(launches), "clocks": clk.summary(),
        }), flush=True)
    if dist:
        dist.barrier()
        dist.destroy_process_group()


def run_decomp3(args):
    """One n3^3 lattice cut into z-slabs (decomp.SlabRunner3): slab s on
    rank s * world // k, halos over NCCL between ranks, the planes that need
    no ghost plane computed while the halo is in flight; value = lattice
    node updates per second of the job (strong scaling)."""
    import torch

    from paper_1607_08675_gb300 import build, decomp, inputs, lbmhd as L

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    if rank == 0:
        build.build()
    if dist:
        dist.barrier()
    L.lib()
    n, prec = args.n3, args.precision
    les = args.les or 1
    k = args.decomp_slabs or world
    owner = [s * world // k for s in range(k)]
    mine = [s for s in range(k) if owner[s] == rank]
    kw = dict(tau_nu=0.51, tau_eta=0.51, C_S=0.1, precision=prec, les=les, delta=2.0)
    runner = decomp.SlabRunner3(n, n, n, k, slabs=mine,
                                comm=decomp.DistComm(owner) if world > 1 else None,
                                overlap=not args.no_overlap, **kw)
    runner.init(*inputs.turbulence3d(n, n, n, seed=1))
    hbm, _ = peaks()

    def barrier():
        torch.cuda.synchronize()
        if dist:
            dist.barrier()

    runner.step(args.warmup)
    barrier()
    launches0 = sum(L.lbmhd3_launch_count(h) for h in runner.h.values())
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(dev_id_for_smi()) as clk:
        barrier()
        e0.record(runner.main)
        runner.step(args.steps)
        e1.record(runner.main)
        e1.synchronize()
        barrier()
    mine_t = e0.elapsed_time(e1) / 1e3
    dt = max_over_ranks(mine_t, dist)
    launches = sum(L.lbmhd3_launch_count(h) for h in runner.h.values()) - launches0
    my_planes = sum(runner.planes[s][1] - runner.planes[s][0] for s in mine)
    per_rank = n * n * my_planes * args.steps / mine_t / 1e6
    rates = [per_rank]
    if dist:
        t = torch.tensor([per_rank], dtype=torch.float64, device="cuda")
        out = [torch.zeros_like(t) for _ in range(world)]
        dist.all_gather(out, t)
        rates = [float(x.item()) for x in out]
    bpc = L.lbmhd3_bytes_per_cell(prec)
    halo_total = decomp.halo_bytes_per_step3(n, n, n, k, les, bpc // 90)
    value = n ** 3 * args.steps / dt / 1e6
    runner.sync()
    runner.close()
    if rank == 0:
        print(json.dumps({
            "metric": METRIC, "value": value, "unit": "MLUPS", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps,
            "higher_is_better": True, "scaling": "strong", "vs_baseline": None,
            "dtype": DTYPES[prec].split(" ")[0], "data": "synthetic",
            "config": {"workload": "3D decaying turbulence (D3Q27 + D3Q7), one lattice cut into z-slabs",
                       "nx": n, "ny": n, "nz": n, "precision": prec, "les": les,
                       "parallelism": f"z-slab decomposition: {k} slab(s) over {world} rank(s)",
                       "l2": "state larger than L2, no flush"},
            "decomp": {"slabs": k, "ranks": world, "overlap": not args.no_overlap,
                       "halo_bytes_per_step": halo_total,
                       "per_rank_MLUPS": rates,
                       "hbm_frac_of_job": value * 1e6 * bpc / 1e9 / hbm / world},
            "gpu_launches": int(launches), "clocks": clk.summary(),
        }), flush=True)
    if dist:
        dist.barrier()
        dist.destroy_process_group()


def runner_halo(n, k, mine, les, vb):
    """Bytes the slabs `mine` receive per step."""
    from paper_1607_08675_gb300 import decomp

    msgs = decomp.halo_messages(n, k, decomp.ghost_rows(les))
    return sum(m.nvalues(n) for m in msgs if m.dst in mine) * vb


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=500)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--precision", choices=list(DTYPES), default="fp32")
    ap.add_argument("--n", type=int, default=8192)
    ap.add_argument("--n3", type=int, default=256, help="edge of the 3D lattice legs")
    ap.add_argument("--no-variants", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-batch", action="store_true")
    ap.add_argument("--no-adjoint", action="store_true")
    ap.add_argument("--adj-n", type=int, default=512)
    ap.add_argument("--adj-steps", type=int, default=500)
    ap.add_argument("--batch-runs", type=int, default=256)
    ap.add_argument("--batch-steps", type=int, default=1000)
    ap.add_argument("--precision-study", action="store_true",
                    help="print per-field errors of every storage form instead of timing")
    ap.add_argument("--study-n1", type=int, default=1024)
    ap.add_argument("--study-steps1", type=int, default=2000)
    ap.add_argument("--study-n2", type=int, default=8192)
    ap.add_argument("--study-steps2", type=int, default=500)
    ap.add_argument("--cpu-budget", type=float, default=15.0)
    ap.add_argument("--decomp3", action="store_true",
                    help="one n3^3 3D lattice cut into z-slabs over the ranks (strong scaling)")
    ap.add_argument("--decomp", action="store_true",
                    help="one lattice cut into row slabs over the ranks (strong scaling)")
    ap.add_argument("--decomp-slabs", type=int, default=0,
                    help="slabs of the decomposed lattice (default: one per rank)")
    ap.add_argument("--les", type=int, default=0, help="closure of the decomposed run")
    ap.add_argument("--no-overlap", action="store_true",
                    help="decomposed run: exchange, then step (no overlap)")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.precision_study:
        precision_study(args)
    elif args.impl == "reference":
        run_reference(args)
    elif args.decomp3:
        run_decomp3(args)
    elif args.decomp:
        run_decomp(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
