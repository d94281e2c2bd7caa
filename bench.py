#!/usr/bin/env python
"""Benchmark of the mini-batch quasi-Newton proximal iteration (Algorithm 4.1).

Workload (default "ls128"): nonlinear Lippmann-Schwinger model, 128^3 grid
(voxel = wavelength/4) padded to 256^3, 20 random ellipsoids (contrast in
[0, 0.04]) plus a Gaussian background, L = 60 plane waves on a 45-degree cone,
128x128 detector, 30 dB noise, mini-batch 8 (S = 8 subsets), BiCGSTAB tolerance
1e-4, isotropic TV lambda = 1e-3, box [0, 0.06], 20 dual iterations.  All inputs
are seeded synthetic data.

A step is one iteration k > S of Algorithm 4.1 on one GPU: the gradient of one
subset (7-8 illuminations, forward and adjoint LS solves), the SR1 update and
the weighted proximal mapping.  The first S iterations (which only set up the
per-subset metrics) run during set-up, so the timed steps are in the
quasi-Newton phase.  Metric: illumination-gradients per second (whole job);
MQNPM iterations/s and the plain cuFFT one-illumination-per-launch path are
reported beside it.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl mine|reference]
For N > 1 run under torchrun; every rank runs an independent reconstruction
(replicas; no collective on the data path) and rank 0 prints the JSON line.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import synth  # noqa: E402

METRIC = "illum-gradients/s + MQNPM iters/s at 128^3 vs plain GPU path; % HBM peak"
UNIT = "illum-gradients/s"
# Mean BiCGSTAB iterations (forward + adjoint) per illumination-gradient that the
# GPU path measures on ls128 at tolerance 1e-4 in the timed iterations
# (k = 29..38: 3 forward + 2 adjoint), used only to scale the bounded oracle
# sample of the reference arm to one illumination-gradient.
LS128_ITERS_PER_ILLUM = 5.0
# Iterations of Algorithm 4.1 from x0 = 0 completed when the timed steps end.
SETUP_ITERS = 38


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def fp32_peak_tflops():
    """FP32 FMA peak from the unit counts and the clock: 152 SMs x 128 FP32
    lanes x 2 flops per FMA x the maximum SM clock (MEASURED_PEAKS.json, else
    the nominal 2070 MHz)."""
    mhz = 2070.0
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            mhz = float(json.load(f).get("sm_max_mhz", mhz))
    except Exception:
        pass
    return 152 * 128 * 2 * mhz * 1e6 / 1e12


# ------------------------------------------------------- pass-3 DRAM traffic
# DRAM traffic (dram__bytes_read.sum + dram__bytes_write.sum) of k_pass3 at
# n = 128 from one ncu capture of `bench.py --green-only --batch 4 --tile 0`
# (4 slots per launch, the default z-pass shape), per slot.  It applies only
# while the sources the kernel is compiled from are the captured ones (digest
# below) and the run uses the captured z-pass shape (tile bits 2-3);
# otherwise the bench reports traffic as null.
PASS3_CAPTURE = {"n": 128, "bytes_per_slot": 126320192, "z_tile_bits": 0, "sources_sha256_16": "ecfa54238ba59598"}
PASS3_SOURCES = ("common.cuh", "fft.cuh", "green_passes.cuh", "green_inst.cu")


def pass3_alu_view(n: int, prof: dict, ms: float):
    """Pass 3 as the FP32-issue-bound kernel it is: FFT flops by the usual
    convention (5 P log2 P per P-point complex transform, two per column, plus
    6 per point for the K_hat product) over its live time, against the FP32
    FMA peak.  The convention counts the full transforms, so it is an upper
    estimate of the arithmetic done by the pruned ones."""
    P = 2 * n
    flops_slot = P * P * (2 * 5 * P * math.log2(P) + 6 * P)
    achieved = flops_slot * prof["slot_launches"] / (ms / 1e3) / 1e12 if ms > 0 else 0.0
    peak = fp32_peak_tflops()
    return {"bound": "alu", "kernel": "k_pass3", "achieved": round(achieved, 2), "peak": round(peak, 1),
            "unit": "TFLOP/s", "frac": round(achieved / peak, 4), "flops_per_slot": int(flops_slot),
            "convention": "5 P log2 P per transform + 6 per K_hat product; peak = 152 SM x 128 FP32 lanes x 2 x sm_max_mhz"}


def pass3_traffic(n: int, slots_per_launch: float, tile: int):
    """Captured per-slot traffic x slots per launch, or None if stale."""
    if (tile >> 2) & 3 != PASS3_CAPTURE["z_tile_bits"]:
        return None
    import hashlib
    d = os.path.join(os.path.dirname(os.path.abspath(__file__)), "paper_2307_02043_gb300", "csrc")
    hsh = hashlib.sha256()
    try:
        for f in PASS3_SOURCES:
            with open(os.path.join(d, f), "rb") as fh:
                hsh.update(fh.read())
    except OSError:
        return None
    if hsh.hexdigest()[:16] != PASS3_CAPTURE["sources_sha256_16"] or n != PASS3_CAPTURE["n"]:
        return None
    return int(PASS3_CAPTURE["bytes_per_slot"] * slots_per_launch)


class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = None
        self.skip = 0

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits",
                 "-lms", "50"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
            return
        # wait for the first sample so that the timed region is covered; samples
        # taken before the timed region starts are dropped at stop()
        self.skip = 0
        t0 = time.perf_counter()
        while time.perf_counter() - t0 < 5.0:
            with open(self.path) as f:
                lines = f.read().splitlines()
            if lines:
                self.skip = len(lines)
                break
            time.sleep(0.02)

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as f:
            lines = f.read().splitlines()
        if len(lines) > self.skip:
            lines = lines[self.skip:]
        for line in lines:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, val in zip(names, parts[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(nm)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ------------------------------------------------------------ problem set-up
# Start of the LS adjoint solves per workload (mqnpm_config.adjoint_start):
# at b = G^H S^T r by default; at 0 where the extra apply of the b start
# saves no BiCGSTAB iteration (measured on GB300: ls192, contrast up to 0.05,
# 153.7 illum-gradients/s from 0 against 146.6 from b at the same counts).
ADJOINT_START = {"ls192": "zero"}


def adjoint_start(w, args=None):
    forced = getattr(args, "adjoint_start", None) if args is not None else None
    return forced or ADJOINT_START.get(w.name, "b")


def forward_start(args=None):
    """Start of the warm-started LS forward solves (mqnpm_config.forward_start):
    the stored field refined by one fixed-point step unless forced."""
    forced = getattr(args, "forward_start", None) if args is not None else None
    return forced or "refine"


def subset_of(w):
    so = np.zeros(w.L, dtype=np.int32)
    for s, idx in enumerate(synth.subsets(w)):
        so[idx] = s
    return so


def make_problem(w, dev, torch, binding, seed_shift=0, tile=-1, direct=False, adj="b", fwd="refine"):
    """Synthetic measurements and alpha_s, produced with the library itself."""
    kd = synth.illumination_dirs(w)
    so = subset_of(w)
    subs = synth.subsets(w)
    xt = torch.from_numpy(synth.phantom(w).astype(np.float32)).to(dev).reshape(-1)
    common = dict(model=w.model, h=w.h, kb=w.kb, tv=w.tv, lam=w.lam, box=w.box, krylov_tol=w.krylov_tol,
                  dual_iters=w.dual_iters, gamma=w.gamma, step=w.step, max_batch=max(len(s) for s in subs),
                  krylov_maxit=1000)
    setup = binding.MQNPM(w.n, kd, so, [1.0] * w.S, **dict(common, krylov_tol=1e-6, tile=tile))
    ys = []
    for c0 in range(0, w.L, setup.max_batch):
        il = list(range(c0, min(w.L, c0 + setup.max_batch)))
        y, _ = setup.forward(xt, il)
        ys.append(y)
    y = torch.cat(ys)
    noise = torch.from_numpy(synth.noise_draws(w).astype(np.complex64)).to(dev)
    sigma = torch.linalg.vector_norm(y, dim=1, keepdim=True) / math.sqrt(w.n * w.n) * 10 ** (-w.snr_db / 20)
    y = (y + sigma * noise).contiguous()
    start = torch.from_numpy(synth.power_start(w).astype(np.float32)).to(dev).reshape(-1)
    alpha = [setup.lipschitz(list(s), w.S / w.L, start, iters=10) for s in subs]
    setup.close()
    h = binding.MQNPM(w.n, kd, so, alpha, warm_start=True, tile=tile, direct_launches=direct, adjoint_start=adj,
                      forward_start=fwd, **common)
    h.set_measurements(y.reshape(-1))
    return h, y, alpha, kd, so, subs


# ------------------------------------------------ plain cuFFT comparison path
class PlainPath:
    """One illumination per launch with torch.fft (cuFFT): pad to P^3, full C2C
    FFTs, pointwise multiply, inverse, crop; host-driven BiCGSTAB.  This is the
    baseline the fused path is compared with (same model, same tolerance)."""

    def __init__(self, w, kd, y, torch, dev, adj="b"):
        self.t = torch
        self.adj = adj
        self.w = w
        self.n = w.n
        self.P = 2 * w.n
        self.dev = dev
        self.kd = kd
        self.y = y.view(w.L, w.n, w.n)
        n, P, kb = self.n, self.P, w.kb * w.h   # dimensionless: lengths in voxels
        idx = torch.arange(P, device=dev, dtype=torch.float64)
        off = torch.where(idx < n, idx, idx - P)
        dz, dy, dx = torch.meshgrid(off, off, off, indexing="ij")
        r = torch.sqrt(dx * dx + dy * dy + dz * dz)
        k = torch.exp(1j * kb * r) / (4 * math.pi * r)
        a = (3 / (4 * math.pi)) ** (1 / 3)
        k[0, 0, 0] = (complex(math.cos(kb * a), math.sin(kb * a)) * (1 - 1j * kb * a) - 1) / kb ** 2
        unused = idx == n
        k[unused] = 0
        k[:, unused] = 0
        k[:, :, unused] = 0
        self.K = torch.fft.fftn(kb * kb * k).to(torch.complex64)
        del k, r, dx, dy, dz
        c = (torch.arange(n, device=dev, dtype=torch.float64) - n / 2)
        self.Z, self.Y, self.X = torch.meshgrid(c, c, c, indexing="ij")

    def G(self, v, adj=False):
        t, n, P = self.t, self.n, self.P
        pad = t.zeros((P, P, P), dtype=t.complex64, device=self.dev)
        pad[:n, :n, :n] = v
        F = t.fft.fftn(pad)
        F *= self.K.conj() if adj else self.K
        return t.fft.ifftn(F)[:n, :n, :n]

    def uin(self, l):
        k = self.kd[l]
        ph = self.w.kb * self.w.h * (k[0] * self.X + k[1] * self.Y + k[2] * self.Z)
        return self.t.exp(1j * ph).to(self.t.complex64)

    def bicgstab(self, A, b, x0, tol, maxit=1000):
        t = self.t
        x = x0.clone()
        r = b - A(x)
        rh = r.clone()
        bn = float(t.linalg.vector_norm(b))
        rho_o = alpha = omega = 1.0 + 0j
        v = t.zeros_like(b)
        p = t.zeros_like(b)
        it = 0
        while it < maxit and float(t.linalg.vector_norm(r)) > tol * bn:
            rho = complex(t.vdot(rh.reshape(-1), r.reshape(-1)))
            beta = (rho / rho_o) * (alpha / omega)
            p = r + beta * (p - omega * v)
            v = A(p)
            alpha = rho / complex(t.vdot(rh.reshape(-1), v.reshape(-1)))
            s = r - alpha * v
            it += 1
            if float(t.linalg.vector_norm(s)) <= tol * bn:
                x = x + alpha * p
                break
            tt = A(s)
            omega = complex(t.vdot(tt.reshape(-1), s.reshape(-1))) / float(t.vdot(tt.reshape(-1), tt.reshape(-1)).real)
            x = x + alpha * p + omega * s
            r = s - omega * tt
            rho_o = rho
        return x, it

    def grad(self, x, l, tol):
        t = self.t
        x3 = x.view(self.n, self.n, self.n)
        ui = self.uin(l)
        if self.w.model == "born":          # u = u_in, no solves
            r = self.G(x3 * ui)[-1] - self.y[l]
            lift = t.zeros_like(ui)
            lift[-1] = r
            return (ui.conj() * self.G(lift, adj=True)).real.reshape(-1), 0
        u, itf = self.bicgstab(lambda q: q - self.G(x3 * q), ui, ui, tol)
        r = (u - ui)[-1] - self.y[l]
        lift = t.zeros_like(ui)
        lift[-1] = r
        b = self.G(lift, adj=True)
        z0 = b if self.adj == "b" else t.zeros_like(b)   # the library's start
        z, ita = self.bicgstab(lambda q: q - self.G(x3 * q, adj=True), b, z0, tol)
        return (u.conj() * z).real.reshape(-1), itf + ita


# -------------------------------------------------------------- oracle (CPU)
def aggregate_ranks(torch, dist, device, ms, ms_e2e, illum, illum_e2e):
    """Whole-job figures of replicated runs: the slowest rank's times (max) and
    the illumination-gradients of all ranks (sum).  dist = None for one rank."""
    if dist is None:
        return float(ms), float(ms_e2e), float(illum), float(illum_e2e)
    tt = torch.tensor([float(ms), float(ms_e2e)], dtype=torch.float64, device=device)
    dist.all_reduce(tt, op=dist.ReduceOp.MAX)
    cnt = torch.tensor([float(illum), float(illum_e2e)], dtype=torch.float64, device=device)
    dist.all_reduce(cnt, op=dist.ReduceOp.SUM)
    return float(tt[0]), float(tt[1]), float(cnt[0]), float(cnt[1])


def run_reference(args, world, rank):
    """--impl reference: the FP64 oracle on the host cores, bounded samples."""
    if rank != 0:
        return
    w = synth.workload(args.workload)
    x_np = synth.phantom(w)
    from oracle import physics
    kd = synth.illumination_dirs(w)
    m = physics.Model(w.n, kd[:1], "ls", kb=w.kb, h=w.h, tol=1e-30, maxit=1)
    uin = m.u_in(0)
    A = lambda p: p - m.G(x_np * p)  # noqa: E731
    for _ in range(args.warmup):
        m.G(x_np * uin)
    times = []
    c0, w0 = time.process_time(), time.perf_counter()
    for _ in range(args.steps):
        t0 = time.perf_counter()
        physics.bicgstab(A, uin, uin, 1e-30, 1)     # one BiCGSTAB iteration (+ initial residual)
        times.append(time.perf_counter() - t0)
    cores = round((time.process_time() - c0) / (time.perf_counter() - w0), 1)   # threads actually busy
    t_iter = statistics.mean(times) * 2.0 / 3.0     # 3 applies timed, 2 per iteration
    per_illum = t_iter * LS128_ITERS_PER_ILLUM + 2 * (t_iter / 2)
    value = 1.0 / per_illum
    sample = ("FP64 oracle, one BiCGSTAB iteration of one LS forward solve at n=%d per step, scaled to an "
              "illumination-gradient by %.0f iterations (fwd+adj) + 2 Green's applies" % (w.n, LS128_ITERS_PER_ILLUM))
    out = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * statistics.mean(times),
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
           "data": "synthetic", "config": {"workload": w.name, "n": w.n, "L": w.L, "batch": w.batch},
           "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
           "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def prox_only(args, torch, binding):
    """Weighted proximal mappings on the workload grid with S_eff = S rank-one
    terms (a small case for profiler captures): prints time and phase trace."""
    w = synth.workload(args.workload)
    dev = torch.device("cuda", 0)
    h = binding.MQNPM(w.n, synth.illumination_dirs(w), subset_of(w), [1.0] * w.S, tv=w.tv, lam=w.lam,
                      box=w.box, dual_iters=w.dual_iters, max_batch=1)
    g = torch.Generator(device=dev).manual_seed(0)
    x_true = torch.from_numpy(synth.phantom(w).astype(np.float32)).to(dev).reshape(-1)
    v = x_true + 0.01 * torch.randn(w.N, device=dev, generator=g)
    U = 0.02 * torch.randn(w.S * w.N, device=dev, generator=g)
    tau, c = 50.0, w.S * w.lam
    P = torch.zeros(3 * w.N, device=dev)
    for _ in range(args.warmup):
        h.wprox(v, tau, U, c, P_warm=P)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(args.steps):
        h.wprox(v, tau, U, c, P_warm=P)
    e1.record()
    torch.cuda.synchronize()
    print(json.dumps({"workload": w.name, "S_eff": w.S, "dual_iters": w.dual_iters,
                      "ms_per_prox": round(e0.elapsed_time(e1) / args.steps, 3), "trace_us": h.prox_trace()}),
          flush=True)
    h.close()


def green_only(args, torch, binding):
    """Batched Green's applies on the workload grid (a small case for profiler
    captures): prints per-pass times and achieved GB/s as one JSON line."""
    w = synth.workload(args.workload)
    dev = torch.device("cuda", 0)
    h = binding.MQNPM(w.n, synth.illumination_dirs(w), subset_of(w), [1.0] * w.S, max_batch=args.batch, h=w.h, kb=w.kb,
                      tile=args.tile)
    g = torch.Generator(device=dev).manual_seed(0)
    v = torch.randn(args.batch * w.N, dtype=torch.complex64, device=dev, generator=g)
    for _ in range(args.warmup):
        h.green_apply(v)
    h.profile_begin(args.steps)
    for _ in range(args.steps):
        h.green_apply(v)
    prof = h.profile_end()
    N = w.N
    per_slot = [24 * N, 48 * N, 64 * N, 48 * N, 24 * N]   # plain prologue/epilogue
    slots = prof["slot_launches"]
    res = {"workload": w.name, "batch": args.batch, "applies": prof["calls"],
           "pass_ms": [round(t / prof["calls"], 4) for t in prof["pass_ms"]],
           "pass_GBps": [round(b * slots / (t / 1e3) / 1e9, 1) for b, t in zip(per_slot, prof["pass_ms"])]}
    print(json.dumps(res), flush=True)
    h.close()


def grad_only(args, torch, binding):
    """Mini-batch gradients of the workload (a small case for profiler captures:
    no set-up solves, zero measurements, x = phantom / 2): prints per-pass times."""
    w = synth.workload(args.workload)
    dev = torch.device("cuda", 0)
    subs = synth.subsets(w)
    h = binding.MQNPM(w.n, synth.illumination_dirs(w), subset_of(w), [1.0] * w.S, model=w.model, h=w.h, kb=w.kb,
                      krylov_tol=w.krylov_tol, max_batch=max(len(q) for q in subs), tile=args.tile)
    h.set_measurements(torch.zeros(w.L * w.n * w.n, dtype=torch.complex64, device=dev))
    x = 0.5 * torch.from_numpy(synth.phantom(w).astype(np.float32)).to(dev).reshape(-1)
    illum = [int(i) for i in subs[0]]
    for _ in range(args.warmup):
        h.grad_batch(x, illum, 1.0)
    h.profile_begin(4096)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    its = None
    for _ in range(args.steps):
        _, _, its = h.grad_batch(x, illum, 1.0)
    e1.record()
    torch.cuda.synchronize()
    prof = h.profile_end()
    print(json.dumps({"workload": w.name, "illuminations": len(illum), "ms_per_gradient": round(
        e0.elapsed_time(e1) / args.steps, 3), "krylov_iters": its, "applies": prof["calls"],
        "pass_ms": [round(t, 3) for t in prof["pass_ms"]]}), flush=True)
    h.close()


def prepare_uneven(torch, binding, dev):
    """Measurements and alpha_s of every request of the uneven mix (set-up, not timed)."""
    prepared = []
    for w in synth.uneven_requests():
        subs = synth.subsets(w)
        kd = synth.illumination_dirs(w)
        so = subset_of(w)
        xt = torch.from_numpy(synth.phantom(w).astype(np.float32)).to(dev).reshape(-1)
        mb = max(len(q) for q in subs)
        setup = binding.MQNPM(w.n, kd, so, [1.0] * w.S, krylov_tol=1e-6, krylov_maxit=1000, max_batch=mb)
        ys = [setup.forward(xt, list(range(c0, min(w.L, c0 + mb))))[0] for c0 in range(0, w.L, mb)]
        y = torch.cat(ys)
        noise = torch.from_numpy(synth.noise_draws(w).astype(np.complex64)).to(dev)
        sigma = torch.linalg.vector_norm(y, dim=1, keepdim=True) / math.sqrt(w.n * w.n) * 10 ** (-w.snr_db / 20)
        y = (y + sigma * noise).contiguous()
        start = torch.from_numpy(synth.power_start(w).astype(np.float32)).to(dev).reshape(-1)
        alpha = [setup.lipschitz(list(q), w.S / w.L, start, iters=10) for q in subs]
        setup.close()
        del xt
        prepared.append((w, kd, so, alpha, y, mb))
    torch.cuda.synchronize()
    return prepared


def serve_uneven_run(prepared, budget, shared, torch, binding, dev, max_group_slots=16):
    """One pass of the request loop over the uneven mix.  Requests are admitted
    in order while their workspace fits the HBM budget (the library's own
    budget check at create refuses the rest, which wait for a retirement) and
    retired after `outer_iters` iterations.  shared = False: the active
    requests step one after another, each on its own workspace of one
    mini-batch.  shared = True: the active requests of one grid form a group
    whose subset gradients run as one batch of slots (shared launches, up to
    max_group_slots slots per chunk); a request is admitted only while its
    grid's group, rebuilt with one slot per illumination of its members'
    mini-batches, still fits the budget; each round steps every group once.
    Per-iteration latency: the time from the start of the call that advances a
    request to its end."""
    queue = list(range(len(prepared)))
    active = {}        # request index -> [handle, x, iterations done]
    used = [0]
    peak = [0]
    tiles = {}
    groups = {}        # n -> (Group, member ids)
    lat_ms, illum_done = [], 0
    builds = [0, 0.0]  # group (re)builds, host seconds spent in them
    per_grid = {}      # n -> [step ms, illumination-gradients, Krylov iterations]
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]

    def build_group(n, ids, allow_fewer):
        """(Re)build grid n's group for the members ids with one slot per
        illumination of their mini-batches (up to max_group_slots).  Without
        allow_fewer a group that does not fit the budget is not built (None);
        with it the slot count is halved until it fits."""
        cur = groups.pop(n, None)
        if cur is not None:
            used[0] -= cur[0].workspace_bytes
            cur[0].close()
        slots = min(max_group_slots, sum(prepared[i][5] for i in ids))
        t_build = time.perf_counter()
        while True:
            try:
                g = binding.Group([active[i][0] for i in ids], max_slots=slots,
                                  hbm_budget_bytes=max(1, budget - used[0]))
                break
            except binding.MQNPMError as err:
                if err.code == 2 and not allow_fewer:
                    return None
                if err.code != 2 or slots == 1:
                    raise
                slots = max(1, slots // 2)
        used[0] += g.workspace_bytes
        peak[0] = max(peak[0], used[0])
        groups[n] = (g, ids)
        builds[0] += 1
        builds[1] += time.perf_counter() - t_build
        return g

    def admit():
        while queue:
            i = queue[0]
            w, kd, so, alpha, y, mb = prepared[i]
            if budget - used[0] <= 0:                 # a zero budget would mean "no limit"
                return
            try:
                h = binding.MQNPM(w.n, kd, so, alpha, tv=w.tv, lam=w.lam, box=w.box, krylov_tol=w.krylov_tol,
                                  krylov_maxit=1000, dual_iters=w.dual_iters, gamma=w.gamma, step=w.step,
                                  max_batch=1 if shared else mb, warm_start=True, hbm_budget_bytes=budget - used[0],
                                  tile=tiles.get(w.n, -1))
            except binding.MQNPMError as err:
                if err.code == 2 and active:          # over budget: wait for a retirement
                    return
                raise
            h.set_measurements(y.reshape(-1))
            tiles[w.n] = h.tile_info()["tile"]
            used[0] += h.workspace_bytes
            active[i] = [h, torch.zeros(w.N, dtype=torch.float32, device=dev), 0]
            if shared:
                # a request is admitted with its share of its grid's shared slots
                ids = sorted(j for j in active if prepared[j][0].n == w.n)
                if build_group(w.n, ids, allow_fewer=len(active) == 1) is None:
                    used[0] -= h.workspace_bytes
                    h.close()
                    del active[i]
                    return                            # wait for a retirement
            peak[0] = max(peak[0], used[0])
            queue.pop(0)

    def retire(i):
        h = active[i][0]
        used[0] -= h.workspace_bytes
        n = prepared[i][0].n
        h.close()
        del active[i]
        # the grid's group keeps its reservation until it is rebuilt for the
        # remaining members (and is freed with the grid's last member)
        if n in groups and not any(prepared[j][0].n == n for j in active):
            g, _ = groups.pop(n)
            used[0] -= g.workspace_bytes
            g.close()

    def group_for(n, ids):
        cur = groups.get(n)
        if cur is not None and cur[1] == ids:
            return cur[0]
        return build_group(n, ids, allow_fewer=True)

    admit()
    admitted_first = len(active)
    ev[2].record()
    while active:
        if shared:
            by_n = {}
            for i in sorted(active):
                by_n.setdefault(prepared[i][0].n, []).append(i)
            for n, ids in sorted(by_n.items()):
                g = group_for(n, ids)
                ev[0].record()
                infos = g.step([active[i][1] for i in ids], allow_not_converged=True)
                ev[1].record()
                ev[1].synchronize()
                t = ev[0].elapsed_time(ev[1])
                pg = per_grid.setdefault(n, [0.0, 0, 0])
                pg[0] += t
                for i, info in zip(ids, infos):
                    lat_ms.append(t)
                    illum_done += info["n_illum"]
                    pg[1] += info["n_illum"]
                    pg[2] += info["krylov_iters_total"]
                    active[i][2] += 1
            for i in [i for i in list(active) if active[i][2] >= prepared[i][0].outer_iters]:
                retire(i)
            admit()
        else:
            for i in list(active):
                h, x, done = active[i]
                ev[0].record()
                info = h.step(x, allow_not_converged=True)
                ev[1].record()
                ev[1].synchronize()
                lat_ms.append(ev[0].elapsed_time(ev[1]))
                illum_done += info["n_illum"]
                pg = per_grid.setdefault(prepared[i][0].n, [0.0, 0, 0])
                pg[0] += lat_ms[-1]
                pg[1] += info["n_illum"]
                pg[2] += info["krylov_iters_total"]
                active[i][2] += 1
                if active[i][2] >= prepared[i][0].outer_iters:
                    retire(i)
                    admit()
    ev[3].record()
    torch.cuda.synchronize()
    total_ms = ev[2].elapsed_time(ev[3])
    lat = np.array(lat_ms)
    return {"mode": "shared launches per grid" if shared else "one request after another",
            "peak_workspace_gb": round(peak[0] / 2 ** 30, 2), "admitted_at_start": admitted_first,
            "iterations": int(lat.size), "illum_gradients_per_s": round(illum_done / (total_ms / 1e3), 2),
            "iteration_latency_ms": {"p50": round(float(np.percentile(lat, 50)), 3),
                                     "p99": round(float(np.percentile(lat, 99)), 3),
                                     "max": round(float(lat.max()), 3)},
            "total_ms": round(total_ms, 1), "green_tile_per_grid": {str(k): v for k, v in tiles.items()},
            "group_builds": builds[0], "group_build_ms": round(1e3 * builds[1], 1),
            "slowest_iterations_ms": [round(float(v), 1) for v in sorted(lat_ms)[-8:]],
            "per_grid": {str(k): {"step_ms": round(v[0], 1), "illum_gradients": v[1], "krylov_iters": v[2]}
                         for k, v in sorted(per_grid.items())}}


def serve_uneven(args, torch, binding):
    """Uneven request mix (16 reconstructions, grids 64^3-160^3, L in {24, 48, 60},
    mini-batch 4-8): the request loop with shared launches per grid (the
    served figures) and, for comparison, one request after another.  Prints
    both as one JSON line."""
    dev = torch.device("cuda", 0)
    prepared = prepare_uneven(torch, binding, dev)
    budget = int(args.hbm_budget_gb * 2 ** 30)
    shared = serve_uneven_run(prepared, budget, True, torch, binding, dev)
    serial = serve_uneven_run(prepared, budget, False, torch, binding, dev)
    print(json.dumps({"workload": "uneven16", "requests": len(prepared),
                      "grids": sorted({p[0].n for p in prepared}), "hbm_budget_gb": args.hbm_budget_gb,
                      "illum_gradients_per_s": shared["illum_gradients_per_s"],
                      "iteration_latency_ms": shared["iteration_latency_ms"],
                      "shared": shared, "serial": serial,
                      "speedup_shared_vs_serial": round(shared["illum_gradients_per_s"] /
                                                        serial["illum_gradients_per_s"], 3)}), flush=True)


def weighted_vs_unweighted_prox(torch, h, x, infos, w):
    """The cost claim of Section 1: the weighted proximal mapping (inside the
    timed steps, rank-S metric) against the unweighted one of the same size and
    dual iterations (metric tau* I, the prox of a plain proximal-gradient step),
    timed here on the last iterate."""
    tau = float(infos[-1]["tau_star"])
    c = w.step * w.lam
    P = torch.zeros(3 * w.N, dtype=torch.float32, device=x.device)
    out = torch.empty_like(x)
    for _ in range(2):
        P.zero_()
        h.wprox(x, tau, None, c, P_warm=P, out=out)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    reps = 5
    e0.record()
    for _ in range(reps):
        h.wprox(x, tau, None, c, P_warm=P, out=out)
    e1.record()
    torch.cuda.synchronize()
    unweighted = e0.elapsed_time(e1) / reps
    weighted = statistics.mean(i["ms_prox"] for i in infos)
    return {"weighted_ms": round(weighted, 3), "unweighted_ms": round(unweighted, 3),
            "ratio": round(weighted / unweighted, 2) if unweighted > 0 else None,
            "dual_iters": w.dual_iters, "weighted_rank": w.S}


def prox_bytes(trace: dict, rank: int, N: int) -> int:
    """Algorithmic bytes of one weighted proximal mapping from the barrier
    counts of its phase trace (float32 vectors, N voxels, rank-S metric):
    Gram set-up (4S + 4) N; per divergence pass with the first Newton
    evaluation (R, U, v, status in; d, x out) (25 + 4S) N; per further Newton
    evaluation (U, v, d, status in, x out) (13 + 4S) N; per fix-up after a
    rejected trial (12 + 4S) N; per dual
    update (x, R, P in; P, R out) 52 N; unweighted x pass (R, v in, x out)
    20 N.  The last evaluation's fix-up passes no barrier and is not counted."""
    c = trace.get("counts", {})
    S = rank
    b = 0
    b += c.get("gram", 0) * (4 * S + 4)
    b += c.get("div_UTd", 0) * (25 + 4 * S)
    b += c.get("newton_eval", 0) * (13 + 4 * S)
    b += c.get("x_fixup", 0) * (12 + 4 * S)
    b += c.get("dual_update", 0) * 52
    b += c.get("x_plain", 0) * 20
    if S == 0:   # the final x pass has no barrier after it
        b += 20
    return int(b * N)


def prox_roofline(trace: dict, rank: int, N: int, ms: float):
    peak, kind = peaks()
    by = prox_bytes(trace, rank, N)
    ach = by / (ms / 1e3) / 1e9 if ms > 0 else 0.0
    return {"bound": "hbm", "kernel": "k_wprox (one cooperative launch per proximal mapping)",
            "achieved": round(ach, 1), "peak": peak, "unit": "GB/s", "frac": round(ach / peak, 4),
            "peak_kind": kind, "algorithmic_bytes_per_launch": by, "ms_per_launch": round(ms, 3),
            "rank": rank, "barrier_counts": trace.get("counts", {}),
            "note": "U rows (4 S N bytes) are re-read by every pass; at 128^3 and S = 8 they fit the 129 MB L2, so "
                    "DRAM traffic can be below these algorithmic bytes"}


def plain_vs_fused(w, kd, y, alpha, so, subs, x, tile, torch, binding, dev, adj="b"):
    """The same gradient (one whole subset, same x, same measurements, Krylov
    tolerance and solver starts: forward at u_in, adjoint at b = G^H S^T r or
    at 0 as the workload's) on both arms: the fused library call on a handle
    without warm start, and the plain torch.fft (cuFFT) path with one
    illumination per launch.  Reports per-illumination and per-Krylov-
    iteration times and the speedup at equal solver work."""
    il = [int(i) for i in subs[0]]
    scale = w.S / w.L
    hc = binding.MQNPM(w.n, kd, so, alpha, model=w.model, h=w.h, kb=w.kb, tv=w.tv, lam=w.lam, box=w.box,
                       krylov_tol=w.krylov_tol, krylov_maxit=1000, dual_iters=w.dual_iters, max_batch=len(il),
                       warm_start=False, tile=tile, adjoint_start=adj)
    hc.set_measurements(y.reshape(-1))
    hc.grad_batch(x, il, scale, allow_not_converged=True)          # warm-up
    reps = 3
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record()
    for _ in range(reps):
        _, _, its = hc.grad_batch(x, il, scale, allow_not_converged=True)
    e1.record()
    torch.cuda.synchronize()
    f_ms = e0.elapsed_time(e1) / reps
    hc.close()
    f_iters = sum(a + b for a, b in its)
    plain = PlainPath(w, kd, y, torch, dev, adj)
    plain.grad(x, il[0], w.krylov_tol)                                # warm-up
    torch.cuda.synchronize()
    p0, p1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    p0.record()
    p_iters = 0
    for l in il:
        _, it = plain.grad(x, l, w.krylov_tol)
        p_iters += it
    p1.record()
    torch.cuda.synchronize()
    p_ms = p0.elapsed_time(p1)
    del plain
    born = w.model == "born"
    fused = {"value": round(len(il) / (f_ms / 1e3), 3), "unit": UNIT, "ms_per_illum": round(f_ms / len(il), 3),
             "krylov_iters": f_iters, "illuminations": len(il),
             "ms_per_krylov_iter_per_illum": None if born else round(f_ms / max(1, f_iters), 4),
             "what": "libmqnpm grad_batch, all %d illuminations of subset 0 in one batch, %s" % (
                 len(il), "first Born" if born else "BiCGSTAB forward from u_in, adjoint from b (no warm start)")}
    plain_d = {"value": round(len(il) / (p_ms / 1e3), 3), "unit": UNIT, "ms_per_illum": round(p_ms / len(il), 3),
               "krylov_iters": p_iters, "illuminations": len(il),
               "ms_per_krylov_iter_per_illum": None if born else round(p_ms / max(1, p_iters), 4),
               "what": "torch.fft (cuFFT) padded %d^3, one illumination per launch, %s" % (
                   2 * w.n, "Born (two applies)" if born else "host-driven BiCGSTAB, forward from u_in, adjoint from b")}
    return fused, plain_d, round(fused["value"] / plain_d["value"], 2)


def cpu_oracle_timings(w, x_np, alpha_np):
    """The FP64 oracle as it stands on the host cores (scipy.fft with one
    worker per available core): one whole illumination-gradient of the workload
    (BiCGSTAB forward from u_in and adjoint from 0, the oracle's starts, at the
    workload's tolerance) and
    one weighted proximal mapping of its size (rank S, J dual iterations)."""
    from oracle import physics
    from oracle import wprox as owprox
    kd = synth.illumination_dirs(w)
    m = physics.Model(w.n, kd[:1], w.model, kb=w.kb, h=w.h, tol=w.krylov_tol)
    y0 = np.zeros(w.n * w.n, dtype=np.complex128)
    c0, t0 = time.process_time(), time.perf_counter()
    _, _, its = m.loss_grad(x_np, 0, y0)
    t_grad = time.perf_counter() - t0
    busy = (time.process_time() - c0) / t_grad
    rng = np.random.default_rng(5)
    U = rng.standard_normal((w.S, w.n, w.n, w.n)) * 0.05
    t0 = time.perf_counter()
    owprox.wprox(x_np, 1.5, U, w.step * w.S * w.lam, w.box[0], w.box[1], w.tv, w.dual_iters,
                 newton_tol=1e-6)
    t_prox = time.perf_counter() - t0
    return t_grad, its, t_prox, busy


def cpu_ls32_end_to_end(outer: int = 10):
    """The small nonlinear configuration end to end on the oracle: 32^3, L = 8,
    S = 4, 10 outer iterations of Algorithm 4.1 from x0 = 0 (data simulated by
    the oracle at its own Krylov tolerance 1e-6)."""
    from oracle import bqnpm, physics
    w = synth.workload("ls32")
    kd = synth.illumination_dirs(w)
    m = physics.Model(w.n, kd, "ls", kb=w.kb, h=w.h, tol=w.krylov_tol)
    t0 = time.perf_counter()
    ys = physics.simulate(m, synth.phantom(w), synth.noise_draws(w), w.snr_db)
    subs = synth.subsets(w)
    alpha = [m.lipschitz(s, w.S / w.L, synth.power_start(w), 10) for s in subs]
    t_setup = time.perf_counter() - t0
    opt = bqnpm.BQNPM(m, ys, subs, alpha, lam=w.lam, box=w.box, kind=w.tv, step=w.step, gamma=w.gamma,
                      dual_iters=w.dual_iters)
    t0 = time.perf_counter()
    opt.run(np.zeros((w.n,) * 3), outer)
    return t_setup, time.perf_counter() - t0


def run_workload(w, args, torch, binding, dev, local, world, rank, dist, full=True):
    """Set-up, timed MQNPM iterations (inputs resident in HBM), the end-to-end
    repeat through host buffers and the per-kernel figures of one workload."""
    h, y, alpha, kd, so, subs = make_problem(w, dev, torch, binding, tile=args.tile,
                                             direct=getattr(args, "direct_launches", False),
                                             adj=adjoint_start(w, args), fwd=forward_start(args))
    x = torch.zeros(w.N, dtype=torch.float32, device=dev)
    shard = bool(getattr(args, "shard", False))
    if shard:
        # the subset's illuminations split over the ranks, one all-reduce of the
        # gradient, the rest of the iteration replicated (Eq. 4.1)
        from paper_2307_02043_gb300.sharded import ShardedStep
        sharded_step = ShardedStep(h, rank, world)
        step = sharded_step.step
    else:
        step = lambda xx: h.step(xx, allow_not_converged=True)  # noqa: E731
    # Set-up iterations from x0 = 0: the S initial steps of Algorithm 4.1 and the
    # reconstruction up to iteration SETUP_ITERS, so that the warm-up and timed
    # steps sit where the paper's BQNPM-I reached ASPM's best SNR (38 iterations).
    for _ in range(max(w.S, SETUP_ITERS - args.warmup - args.steps)):
        step(x)
    for _ in range(args.warmup):
        step(x)
    torch.cuda.synchronize()
    # the end-to-end run below repeats the same iterations from this state
    state0, x0 = h.save_state(), x.cpu()
    # ---- timed region: inputs resident in HBM, no pass timers (so that every
    # BiCGSTAB solve runs as one graph launch with its loop on the device)
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    clocks = ClockSampler(local)
    clocks.start()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    illum_done = 0
    infos = []
    launches0 = h.launch_count
    nvtx = getattr(torch.cuda, "nvtx", None)   # a "timed" range for profiler captures
    if full and nvtx is not None:
        nvtx.range_push("timed")
    e0.record(stream)
    for _ in range(args.steps):
        info = step(x)
        infos.append(info)
        illum_done += len(subs[info["subset"]])
    e1.record(stream)
    torch.cuda.synchronize()
    if full and nvtx is not None:
        nvtx.range_pop()
    launches = h.launch_count - launches0
    prox_trace = h.prox_trace()
    if world > 1:
        dist.barrier()
    clk = clocks.stop()
    ms = e0.elapsed_time(e1)
    # ---- end-to-end through the public call with host buffers, same iterations
    h.load_state(state0)
    xh = torch.empty(w.N, dtype=torch.float32).pin_memory()
    xh.copy_(x0)
    torch.cuda.synchronize()
    f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    xd = torch.empty_like(x)
    e2e_illum = 0
    e2e_infos = []
    f0.record(stream)
    for _ in range(args.steps):
        xd.copy_(xh, non_blocking=True)
        info = step(xd)
        e2e_infos.append(info)
        e2e_illum += len(subs[info["subset"]])
        xh.copy_(xd, non_blocking=True)
    f1.record(stream)
    torch.cuda.synchronize()
    ms_e2e = f0.elapsed_time(f1)
    # ---- the same iterations once more with the pass timers (six events per
    # Green's apply; the BiCGSTAB iterations then replay one graph each with a
    # host check in between) for the per-pass times and the roofline
    h.load_state(state0)
    del state0
    xp = x0.to(dev)
    h.profile_begin(8192)
    prof_infos = [step(xp) for _ in range(args.steps)]
    prof = h.profile_end()
    prof_same = [i["krylov_iters_total"] for i in prof_infos] == [i["krylov_iters_total"] for i in infos]
    del xp
    if full and args.log_jsonl and rank == 0:
        with open(args.log_jsonl, "w") as f:
            for i in infos:
                f.write(json.dumps({k: (round(v, 6) if isinstance(v, float) else v) for k, v in i.items()}) + "\n")
    wprox_ratio = weighted_vs_unweighted_prox(torch, h, x, infos, w)
    # ---- max over ranks
    t_max, ms_e2e, illum_total, e2e_total = aggregate_ranks(torch, dist if world > 1 else None, dev, ms, ms_e2e,
                                                            illum_done, e2e_illum)
    if shard:   # every rank stepped the same reconstruction: count its illuminations once
        illum_total, e2e_total = float(illum_done), float(e2e_illum)
    value = illum_total / (t_max / 1e3)
    iters_per_s = (1 if shard else world) * args.steps / (t_max / 1e3)
    e2e_value = e2e_total / (ms_e2e / 1e3)
    # ---- roofline of the dominant Green's pass
    N = w.N
    n = w.n
    per_slot = [28 * N, 48 * N, 64 * N, 48 * N, 32 * N]
    names = ["x_fwd", "y_fwd", "z_conv", "y_inv", "x_inv"]
    pms = prof["pass_ms"]
    dom = int(np.argmax(pms))
    bytes_dom = per_slot[dom] * prof["slot_launches"] + (8 * (n + 1) ** 3 * prof["calls"] if dom == 2 else 0)
    peak, peak_kind = peaks()
    achieved = bytes_dom / (pms[dom] / 1e3) / 1e9 if pms[dom] > 0 else 0.0
    # GB/s only where the bytes per slot do not depend on the fused prologue or
    # epilogue (the x passes move 20-52 N bytes per slot depending on the kind)
    passes = {nm: {"ms": round(t, 3), "GB/s": round(per_slot[i] * prof["slot_launches"] / (t / 1e3) / 1e9, 1)
                   if t > 0 and nm not in ("x_fwd", "x_inv") else None} for i, (nm, t) in enumerate(zip(names, pms))}
    kit = [i["krylov_iters_max"] for i in infos]
    kit_per_illum = [i["krylov_iters_total"] / max(1, i["n_illum"]) for i in infos]
    out = {
        "metric": METRIC, "value": round(value, 3), "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(t_max / args.steps, 3), "higher_is_better": True,
        "scaling": "strong" if shard else "weak", "vs_baseline": None, "dtype": "c64/f32 (FP64 reductions)",
        "data": "synthetic",
        "config": {"workload": w.name, "n": n, "padded": 2 * n, "L": w.L, "batch": max(len(s) for s in subs),
                   "S": w.S, "model": "lippmann-schwinger" if w.model == "ls" else "first-born",
                   "krylov_tol": w.krylov_tol if w.model == "ls" else None, "dual_iters": w.dual_iters,
                   "tv": w.tv, "phase": "k > S (SR1-weighted)", "l2": "inputs larger than L2",
                   "krylov_start": "forward solves warm-started from each illumination's last field%s; "
                                   "adjoint solves from %s" % (
                                       ", refined by one fixed-point step" if forward_start(args) == "refine" else "",
                                       "b = G^H S^T r" if adjoint_start(w, args) == "b" else "0")
                   if w.model == "ls" else None,
                   "parallelism": ("illumination-sharded x%d (one all-reduce per step)" % world) if shard
                   else ("replicas" if world > 1 else "single-gpu")},
        "mqnpm_iters_per_s": round(iters_per_s, 3),
        "roofline": {"bound": "hbm", "kernel": "k_pass3 (" + names[dom] + ")" if dom == 2 else names[dom],
                     "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                     "frac": round(achieved / peak, 4),
                     "traffic": pass3_traffic(n, prof["slot_launches"] / max(1, prof["calls"]), h.tile_info()["tile"])
                     if dom == 2 else None,
                     "peak_kind": peak_kind,
                     "algorithmic_bytes_per_slot": per_slot[dom],
                     "algorithmic_bytes_per_launch": int(bytes_dom / max(1, prof["calls"])),
                     "launches": prof["calls"], "slots_per_launch": round(prof["slot_launches"] / max(1, prof["calls"]), 2)},
        "roofline_alu": pass3_alu_view(n, prof, pms[2]) if prof["calls"] else None,
        "roofline_prox": prox_roofline(prox_trace, infos[-1]["rank"], N, infos[-1]["ms_prox"]),
        "passes": passes,
        "passes_note": "pass times from a repeat of the timed iterations with CUDA events around every pass "
                       "(same Krylov counts: %s)" % prof_same,
        "green_applies": prof["calls"],
        "green_tile": h.tile_info(),
        "phase_ms": {k: round(statistics.mean(i["ms_" + k] for i in infos), 3) for k in ("gradient", "metric", "prox")},
        "newton_iters_max": [i["newton_iters_max"] for i in infos],
        "prox_trace_us": prox_trace,
        "krylov_iters_max_per_step": kit,
        "krylov_iters_per_illum": [round(k, 2) for k in kit_per_illum],
        "gpu_launches": int(launches),
        "clocks": clk,
        "wprox_vs_unweighted": wprox_ratio,
        "e2e": {"value": round(e2e_value, 3), "unit": UNIT, "h2d_bytes_per_step": 4 * N, "d2h_bytes_per_step": 4 * N,
                "iterations": "the timed k = %d..%d again, from a checkpoint" % (infos[0]["k"], infos[-1]["k"]),
                "pass_events": "none, like the timed region",
                "same_krylov_iters": [i["krylov_iters_total"] for i in e2e_infos] ==
                                     [i["krylov_iters_total"] for i in infos]},
    }
    if prof["calls"] == 0:
        out["roofline"] = out["roofline_prox"]
        out["roofline_note"] = ("every Green's apply of this model touches one z-plane (first-Born data, adjoint "
                                "right-hand sides) and the pass timers cover full applies only; the dominant "
                                "kernel is the weighted proximal mapping")
    out["config"]["iterations"] = "k = %d..%d from x0 = 0" % (infos[0]["k"], infos[-1]["k"])
    h.close()
    if rank == 0 and not args.no_plain:
        fused, plain_d, sp = plain_vs_fused(w, kd, y, alpha, so, subs, x, args.tile, torch, binding, dev,
                                            adjoint_start(w, args))
        out["fused_cold"] = fused
        out["plain_gpu"] = plain_d
        out["speedup_vs_plain"] = sp
        out["speedup_vs_plain_note"] = ("same subset, x, tolerance and solver starts on both arms (forward "
                                        "u_in, adjoint b: equal solver work); the headline value above "
                                        "warm-starts the forward solves")
        if fused["ms_per_krylov_iter_per_illum"] and plain_d["ms_per_krylov_iter_per_illum"]:
            out["speedup_per_krylov_iter"] = round(plain_d["ms_per_krylov_iter_per_illum"] /
                                                   fused["ms_per_krylov_iter_per_illum"], 2)
    return out, x


# ---------------------------------------------------------------------- main
def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="mine", choices=["mine", "reference"])
    ap.add_argument("--workload", default="ls128")
    ap.add_argument("--no-plain", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-born", action="store_true", help="skip the born128 figures of the default line")
    ap.add_argument("--direct-launches", action="store_true",
                    help="launch every kernel directly instead of through the captured BiCGSTAB graphs (for launch "
                         "lists of profilers that do not descend into conditional graph nodes)")
    ap.add_argument("--shard", action="store_true",
                    help="one reconstruction with each subset's illuminations split over the ranks and the gradient "
                         "summed by an all-reduce (strong scaling) instead of one replica per rank")
    ap.add_argument("--green-only", action="store_true",
                    help="small case for profiler captures: batched Green's applies of the workload grid")
    ap.add_argument("--batch", type=int, default=2, help="slots per apply in --green-only mode")
    ap.add_argument("--log-jsonl", default=None,
                    help="write one JSON line per timed MQNPM iteration (step info) to this file")
    ap.add_argument("--adjoint-start", choices=["b", "zero"], default=None,
                    help="start of the LS adjoint solves (default: the workload's, b unless listed in ADJOINT_START)")
    ap.add_argument("--forward-start", choices=["refine", "stored"], default=None,
                    help="start of the warm-started LS forward solves (default: refine, one fixed-point step)")
    ap.add_argument("--tile", type=int, default=-1,
                    help="launch-shape tile of the Green's passes (-1: autotuned when a handle is created)")
    ap.add_argument("--serve-uneven", action="store_true",
                    help="uneven request mix: admission by HBM budget, round-robin iterations, latency percentiles")
    ap.add_argument("--hbm-budget-gb", type=float, default=24.0, help="HBM budget of --serve-uneven")
    ap.add_argument("--grad-only", action="store_true",
                    help="small case for profiler captures: mini-batch gradients of the workload")
    ap.add_argument("--prox-only", action="store_true",
                    help="small case for profiler captures: weighted proximal mappings on the workload grid")
    args = ap.parse_args()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, world, rank)
        return
    import torch
    import torch.distributed as dist
    from paper_2307_02043_gb300 import binding

    if args.green_only:
        green_only(args, torch, binding)
        return
    if args.prox_only:
        prox_only(args, torch, binding)
        return
    if args.grad_only:
        grad_only(args, torch, binding)
        return
    if args.serve_uneven:
        serve_uneven(args, torch, binding)
        return

    if args.warmup < 3:
        args.warmup = 3
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        dist.init_process_group("nccl", device_id=dev)
    w = synth.workload(args.workload)
    out, x = run_workload(w, args, torch, binding, dev, local, world, rank, dist, full=True)
    if rank == 0 and world == 1 and args.workload == "ls128" and not args.no_born:
        # the other 128^3 configuration of the metric, same steps and warm-up
        wb = synth.workload("born128")
        ob, _ = run_workload(wb, args, torch, binding, dev, local, world, rank, dist, full=False)
        keep = ("value", "unit", "ms_per_step", "mqnpm_iters_per_s", "roofline", "roofline_note", "phase_ms",
                "gpu_launches", "clocks", "e2e", "fused_cold", "plain_gpu", "speedup_vs_plain", "newton_iters_max",
                "wprox_vs_unweighted", "config")
        out["born128"] = {k: ob[k] for k in keep if k in ob}
    if rank == 0 and not args.no_cpu:
        x_np = x.cpu().numpy().astype(np.float64).reshape(w.n, w.n, w.n)
        t_grad, its, t_prox, busy = cpu_oracle_timings(w, x_np, None)
        t_setup32, t_run32 = cpu_ls32_end_to_end()
        from oracle import physics as _ph
        out["cpu_baseline"] = {
            "value": round(1.0 / t_grad, 6), "unit": UNIT, "cores": _ph.FFT_WORKERS, "kind": "oracle",
            "sample": "FP64 oracle (scipy.fft, %d workers): one whole %d^3 illumination-gradient at the last "
                      "iterate, BiCGSTAB forward from u_in + adjoint from 0 at tol %g (%d + %d iterations, %.1f s)"
                      % (_ph.FFT_WORKERS, w.n, w.krylov_tol, its[0], its[1], t_grad),
            "busy_threads": round(busy, 1),
            "wprox_s": round(t_prox, 2),
            "wprox_sample": "one weighted proximal mapping, %d^3, rank %d, %d dual iterations" % (w.n, w.S,
                                                                                                 w.dual_iters),
            "ls32_end_to_end_s": round(t_run32, 2),
            "ls32_sample": "32^3, L = 8, S = 4: 10 outer iterations of Algorithm 4.1 from x0 = 0 (%.1f s of "
                           "data simulation and alpha_s before them)" % t_setup32}
    if rank == 0:
        print(json.dumps(out), flush=True)
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
