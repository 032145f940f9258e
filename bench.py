#!/usr/bin/env python
"""Benchmark of the multidirect-forcing IB hot path on one GB300 per rank.

Workload (synthetic, shaped like the paper's particle clusters): 64
monodisperse spheres of D = 24 cells (1810 Fibonacci markers each) placed
without overlap in a centred cluster box at volume fraction 0.2 of a 256^3
periodic grid; 32-mode Fourier velocity field; Ns = 5 forcing passes;
dt = 1e-3; the paper's three-point kernel; sequential particle order.

One step = every row of the hot path:
  particle_volume_integrals(u)  (I^n)
  -> ib_multidirect_forcing      (Algorithm 1, Ns passes)
  -> particle_force_torque       (F_ib, T_ib)
  -> particle_volume_integrals(u) (I^{n+1})
  -> particle_collide_update     (collision + Newton-Euler + centroid)

Metric: marker updates per second = M * Ns * steps / time (a marker update
is one marker through one interpolate + force + spread pass).  The headline
`value` is the plain FP64 form (FP64 fields, the paper's precision); the
mixed form (FP32 fields, FP64 forces, reductions and updates) is reported
beside it under "fp32".  Between timed steps L2 is flushed by writing a
512 MiB buffer (outside the timed events).

Roofline bytes are the compulsory ones of the method: per step
B_IB = 6 s B + 24 M (read and write u on the B band cells once, write the
marker forces) plus 3 s N_int per volume-integral call (s = bytes per field
scalar, N_int = cells of the particles' volume integrals).

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gbib|reference]
For N > 1 (torchrun) every rank runs an independent replica of the workload
(different seed); value = all ranks' marker updates / max rank time.
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

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "IB marker interp+spread updates/s"
WORKLOAD = dict(N=256, P=64, D=24.0, phi=0.2, K=32, Ns=5, dt=1e-3)
WORKLOAD_NAME = "cluster-256^3-64xD24-phi0.2-Ns5"
PEAKS_PATH = os.path.join(ROOT, "MEASURED_PEAKS.json")
FALLBACK_HBM = 6800.0


def max_over_ranks(t, device=None):
    """Largest per-rank time: the job's time when every rank runs a replica."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(t)
    tt = torch.tensor([float(t)], dtype=torch.float64, device=device)
    dist.all_reduce(tt, op=dist.ReduceOp.MAX)
    return float(tt.item())


def job_value(markers_per_rank, Ns, world, t_job):
    """Whole-job marker updates per second over all replicas."""
    return world * markers_per_rank * Ns / t_job


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def make_case(seed):
    from paper_2408_14140_gb300 import synth
    w = WORKLOAD
    return synth.cluster_case(N=w["N"], P=w["P"], D_cells=w["D"], phi=w["phi"], K=w["K"],
                              Ns=w["Ns"], dt=w["dt"], seed=seed, build_field=False)


def band_cells(case, kernel_width=3):
    """Unique cells in the markers' kernel supports (the algorithmic band)."""
    X = case.R + np.repeat(case.Xr, np.diff(case.moff), axis=0)
    s = (X - np.asarray(case.org)) / case.h - 0.5
    first = np.floor(s + 0.5).astype(np.int64) - 1
    n = np.asarray(case.n, dtype=np.int64)
    cells = []
    for dz in range(kernel_width):
        for dy in range(kernel_width):
            for dx in range(kernel_width):
                c = (first + np.array([dx, dy, dz])) % n
                cells.append((c[:, 2] * n[1] + c[:, 1]) * n[0] + c[:, 0])
    return int(np.unique(np.concatenate(cells)).size)


def wavefront_levels(case, kernel_width=3, return_levels=False):
    """Wavefronts of the sequential particle order (same conflict test as the
    library: centre distance < rho_p + rho_q + sqrt(3) W h + h/16)."""
    P = case.P
    rho = np.array([np.max(np.linalg.norm(case.R[case.moff[p]:case.moff[p + 1]], axis=1))
                    for p in range(P)])
    L = np.asarray(case.n) * case.h
    lev = np.zeros(P, dtype=int)
    for p in range(P):
        d = case.Xr[:p] - case.Xr[p]
        d -= L * np.rint(d / L)
        conf = np.sqrt(np.sum(d * d, axis=1)) < (rho[:p] + rho[p] + np.sqrt(3) * kernel_width * case.h
                                                  + case.h / 16)
        lev[p] = 1 + (lev[:p][conf].max() if conf.any() else -1)
    if return_levels:
        return lev
    return int(lev.max() + 1) if P else 0


def level_band_cells(case, kernel_width=3):
    """(band cells, markers) of every wavefront: the cells a wavefront's gather
    kernel must read and write once per pass, and the markers it spreads."""
    lev = wavefront_levels(case, kernel_width, return_levels=True)
    out = []
    for L in range(int(lev.max()) + 1 if case.P else 0):
        ps = np.nonzero(lev == L)[0]
        sub = case.__class__(**{**case.__dict__})
        idx = np.concatenate([np.arange(case.moff[p], case.moff[p + 1]) for p in ps])
        sub.Xr = case.Xr[ps]
        sub.R = case.R[idx]
        sub.moff = np.concatenate([[0], np.cumsum(np.diff(case.moff)[ps])])
        out.append((band_cells(sub, kernel_width), int(idx.size)))
    return out


def recorded_traffic(kernel, tag):
    """DRAM bytes per launch of `kernel` recorded under profiles/ by an ncu
    capture (profiles/traffic_<kernel>_<tag>.txt), or None when the kernel's
    source changed since (hash mismatch) or nothing was recorded."""
    import hashlib
    path = os.path.join(ROOT, "profiles", "traffic_%s_%s.txt" % (kernel, tag))
    try:
        rec = dict(line.split(":", 1) for line in open(path) if ":" in line and not line.startswith("#"))
        src = os.path.join(ROOT, rec["source"].strip())
        sha = hashlib.sha256(open(src, "rb").read()).hexdigest()
        if rec.get("source_sha256", "").strip() != sha:
            return None
        return float(rec["bytes_per_launch"])
    except Exception:
        return None


def step_bytes(case, s, band=None):
    """Compulsory bytes of one hot-path step by the method's own count:
    B_IB = 6 s B + 24 M (read and write u on the band once, write F) and
    3 s N_int per volume-integral call (two calls per step)."""
    B = band_cells(case) if band is None else band
    b_ib = 6 * s * B + 24 * case.M
    b_vol = 3 * s * interior_cells(case)
    return b_ib, b_vol


def interior_cells(case):
    """Cells a volume integral reads (alpha > 0 or the box walk): sum of
    (4/3) pi (R + sqrt(3) h / 2)^3 / h^3 per particle, an algorithmic bound."""
    r = case.radius / case.h + 0.8661
    return float(np.sum(4.0 / 3.0 * np.pi * r ** 3))


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []
        self.skip = 0

    def start(self):
        """Starts sampling and returns once the first sample is in (at most
        3 s), so that the timed region that follows is sampled from its
        start; samples taken before start() returns are left out."""
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q,
                 "--format=csv,noheader,nounits", "-lms", "50"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.th = threading.Thread(target=self._read, daemon=True)
            self.th.start()
        except Exception:
            self.proc = None
            return
        for _ in range(60):
            if self.lines or self.proc.poll() is not None:
                break
            time.sleep(0.05)
        self.skip = len(self.lines)

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines[self.skip:]:
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
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def peaks():
    try:
        with open(PEAKS_PATH) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM, "fallback"


# --------------------------------------------------------------------------
# GPU arm
# --------------------------------------------------------------------------
class Runner:
    """Device state of one workload replica and the hot-path step."""

    def __init__(self, case, prec, device, delta=0, order=0):
        import torch
        from paper_2408_14140_gb300 import api, synth
        self.torch, self.api = torch, api
        self.case = case
        self.prec = prec
        self.dev = device
        self.delta, self.order = delta, order
        self.ctx = api.Context()
        # the step's first volume integrals run on a side stream (own context)
        # while the forcing call prepares; its passes wait for them
        self.ctx_v = api.Context()
        # the volume integrals after the forcing reuse the cells and alpha the
        # ones before it kept (the particles do not move in between)
        self.plan = api.PvfPlan(self.ctx_v, case.P, int(2 * np.max(case.radius) / case.h + 4) ** 3)
        self.side = torch.cuda.Stream(device=device)
        # CTAs per particle of the first volume integrals, which run beside
        # the forcing's preparation kernels and take SMs from them (measured
        # best: 2 for FP32 fields, 3 for FP64 fields, whose preparation is
        # longer)
        self.v0_split = 3 if prec == api.IB_F64 else 2
        self.ev_v = torch.cuda.Event()
        self.ctx.set_field_wait(self.ev_v)
        dt = api.field_dtype(prec)
        self.u = synth.fourier_eval_torch(case.n, case.meta["modes"], case.h, case.org,
                                          device=device).to(dt).contiguous()
        _, self.parts, self.marks = self._small(case)
        P, M = case.P, case.M
        z = lambda *s: torch.zeros(s, dtype=torch.float64, device=device)  # noqa: E731
        self.F = z(M, 3)
        self.I0 = (z(P, 3), z(P, 3), z(P))
        self.I1 = (z(P, 3), z(P, 3), z(P))
        self.Fib, self.Tib, self.Fc = z(P, 3), z(P, 3), z(P, 3)

    def _small(self, case):
        torch = self.torch

        def t(a, dtype=torch.float64):
            return torch.as_tensor(np.asarray(a)).to(device=self.dev, dtype=dtype).contiguous()

        parts = dict(Xr=t(case.Xr), Ur=t(case.Ur), Wr=t(case.Wr), radius=t(case.radius),
                     rho_p=t(case.rho_p), moff=t(case.moff, torch.int32))
        marks = dict(R=t(case.R), dV=t(case.dV))
        return None, parts, marks

    def status(self):
        self.ctx.status()
        self.ctx_v.status()

    def step(self):
        c, ctx, torch = self.case, self.ctx, self.torch
        main = torch.cuda.current_stream()
        self.side.wait_stream(main)
        with torch.cuda.stream(self.side):
            # a few CTAs per particle: the preparation's kernels keep most SMs
            self.ctx_v.set_volume_split(self.v0_split)
            self.ctx_v.particle_volume_integrals_keep(self.u, c.h, self.parts, self.plan, out=self.I0)
            self.ev_v.record(self.side)
        ctx.ib_multidirect_forcing(self.u, c.h, self.parts, self.marks, c.Ns, c.dt, F_out=self.F,
                                   delta=self.delta, order=self.order)
        # the second volume integrals (field after forcing) beside the marker
        # force and torque sums (forces only)
        self.side.wait_stream(main)
        with torch.cuda.stream(self.side):
            # the plan's cells over a full wave of CTAs (automatic split)
            self.ctx_v.set_volume_split(0)
            self.ctx_v.particle_volume_integrals_plan(self.u, c.h, self.parts, self.plan, out=self.I1)
        ctx.particle_force_torque(self.parts, self.marks, self.F, c.rho_f, out=(self.Fib, self.Tib))
        main.wait_stream(self.side)
        ctx.particle_collide_update(self.parts, c.n, c.h, c.phys(), c.dt, self.Fib, self.Tib,
                                    self.I1[0], self.I0[0], self.I1[1], self.I0[1], Fc_out=self.Fc)


def launches_per_step(Ns, levels):
    """Library kernels per step on this workload: volume 1 x 2 calls;
    multidirect forcing: prep, marker radii, conflicts, levels, marker order,
    tile count, slot scan (counts, flags and compaction in one single-pass
    scan), fill, pair-count scan, sort, per-cell lists, level ranges, tile
    order (13), one interpolation and one gather kernel per wavefront and
    pass, the persistent remainder kernel (1); force/torque 1; collision +
    Newton-Euler 2."""
    return 2 + 13 + 2 * Ns * levels + 1 + 1 + 2


def capture(runner):
    """The runner's step captured into a CUDA graph (None when capture fails:
    the step then runs as eager launches)."""
    torch = runner.torch
    stream = torch.cuda.current_stream()
    try:
        g = torch.cuda.CUDAGraph()
        s = torch.cuda.Stream()
        s.wait_stream(stream)
        with torch.cuda.stream(s):
            runner.step()  # warm allocations on the capture stream
        stream.wait_stream(s)
        torch.cuda.synchronize()
        with torch.cuda.graph(g):
            runner.step()
        return g
    except Exception as e:  # capture unsupported: fall back to eager launches
        print("# graph capture failed, eager launches: %s" % e, file=sys.stderr)
        torch.cuda.synchronize()
        return None


def timed(run, torch, n, flush):
    """Device time (ms) of each of n calls of run(), L2 flushed before each
    (outside its event pair), events on the launching stream."""
    stream = torch.cuda.current_stream()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(n)]
    for a, b in ev:
        flush.fill_(1.0)
        a.record(stream)
        run()
        b.record(stream)
    torch.cuda.synchronize()
    return [a.elapsed_time(b) for a, b in ev]


def time_steps(runner, steps, warmup, flush, use_graph, replays=(0, 0)):
    """Exactly `steps` timed steps after `warmup` untimed ones (CUDA-graph
    replays when capture works), then `replays` = (repeats, count) more
    blocks of `count` timed replays each (the per-step mean of each block)."""
    torch = runner.torch
    graph = capture(runner) if use_graph else None
    run = graph.replay if graph is not None else runner.step
    for _ in range(warmup):
        run()
    torch.cuda.synchronize()
    runner.status()
    ms = timed(run, torch, steps, flush)
    blocks = [statistics.fmean(timed(run, torch, replays[1], flush)) for _ in range(replays[0])]
    runner.status()
    return ms, graph is not None, blocks


def kernel_timing(runner, steps, flush):
    """Per-phase device time of the library's kernels (CUDA events recorded by
    the library on the launching stream) over `steps` eager steps, summed over
    the runner's contexts (the side-stream context runs the volume integrals)."""
    torch = runner.torch
    ctxs = [runner.ctx] + ([runner.ctx_v] if getattr(runner, "ctx_v", None) is not None else [])
    for ctx in ctxs:
        for ph in runner.api.PHASES:
            ctx.read_timing(ph)
        ctx.set_timing(True)
    for _ in range(steps):
        flush.fill_(1.0)
        runner.step()
    torch.cuda.synchronize()
    out = {}
    for ctx in ctxs:
        ctx.set_timing(False)
        for ph in runner.api.PHASES:
            ms, n = ctx.read_timing(ph)
            if n:
                m0, n0 = out.get(ph, (0.0, 0))
                out[ph] = (m0 + ms, n0 + n)
    return out


def e2e_steps(runner, steps, partners=()):
    """Same step through the public API with host buffers: every step copies
    its inputs from pinned host memory to the device, runs, and reads its
    results back.  With partner replicas the steps are pipelined over the
    replicas in turn: step k+1's inputs upload (one copy stream) while step k
    computes and step k-1's results download (another copy stream).  A
    replica's next upload waits for its previous download, so with three
    replicas that wait no longer gates the next step's upload."""
    torch = runner.torch
    reps = [runner] + list(partners)

    def dev_in(r):
        return [r.u, r.parts["Xr"], r.parts["Ur"], r.parts["Wr"], r.parts["radius"], r.parts["rho_p"],
                r.parts["moff"], r.marks["R"], r.marks["dV"]]

    def dev_out(r):
        return [r.u, r.parts["Xr"], r.parts["Ur"], r.parts["Wr"], r.F]

    host_in = [t.detach().cpu().pin_memory() for t in dev_in(runner)]
    host_out = [[torch.empty(t.shape, dtype=t.dtype, pin_memory=True) for t in dev_out(r)] for r in reps]
    bi = sum(t.numel() * t.element_size() for t in host_in)
    bo = sum(t.numel() * t.element_size() for t in host_out[0])
    s_in, s_out = torch.cuda.Stream(), torch.cuda.Stream()
    s_c = torch.cuda.current_stream()
    freed = [None] * len(reps)  # replica k's previous results downloaded
    for r in reps[1:]:  # warm-up of the partners (a first call sizes its launches)
        for _ in range(2):
            r.step()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for k in range(steps):
        j = k % len(reps)
        r = reps[j]
        with torch.cuda.stream(s_in):
            if freed[j] is not None:
                s_in.wait_event(freed[j])
            for d, h in zip(dev_in(r), host_in):
                d.copy_(h, non_blocking=True)
            ready = torch.cuda.Event()
            ready.record(s_in)
        s_c.wait_event(ready)
        r.step()
        done = torch.cuda.Event()
        done.record(s_c)
        with torch.cuda.stream(s_out):
            s_out.wait_event(done)
            for d, h in zip(dev_out(r), host_out[j]):
                h.copy_(d, non_blocking=True)
            freed[j] = torch.cuda.Event()
            freed[j].record(s_out)
    torch.cuda.synchronize()
    dt = (time.perf_counter() - t0) / steps
    for r in reps:
        r.status()
    return dt, bi, bo


def oracle_step(c, u, Xr, Ur, Wr):
    """One full FP64 hot-path step of the oracle (the step the GPU runs)."""
    import oracle
    a0 = oracle.volume_integrals(c.n, c.h, c.org, u, Xr, c.radius)
    u1, F, _ = oracle.multidirect(c.n, c.h, c.org, u, Xr, Ur, Wr, c.moff, c.R, c.dV, c.Ns, c.dt)
    fo, to = oracle.force_torque(c.moff, c.R, c.dV, F, c.rho_f)
    a1 = oracle.volume_integrals(c.n, c.h, c.org, u1, Xr, c.radius)
    X1, U1, W1, Fc = oracle.collide_update(Xr, Ur, Wr, c.radius, c.rho_p, c.n, c.h, c.phys(),
                                           c.dt, fo, to, a1[0], a0[0], a1[1], a0[1])
    return dict(u=u1, F=F, Iu0=a0[0], Irxu0=a0[1], vol0=a0[2], F_ib=fo, T_ib=to, Iu1=a1[0],
                Irxu1=a1[1], vol1=a1[2], Xr=X1, Ur=U1, Wr=W1, Fc=Fc)


def cpu_baseline(case_np, threads, min_seconds=5.0, max_steps=6):
    """The oracle as it stands, full hot-path steps of the same workload on
    `threads` host threads (OpenMP), repeated until >= min_seconds."""
    import oracle
    c = case_np
    oracle.build()
    old = oracle.num_threads()
    oracle.set_num_threads(threads)
    try:
        used = oracle.num_threads()
        steps = 0
        u = c.u.copy()
        Xr, Ur, Wr = c.Xr.copy(), c.Ur.copy(), c.Wr.copy()
        t0 = time.perf_counter()
        while True:
            o = oracle_step(c, u, Xr, Ur, Wr)
            u, Xr, Ur, Wr = o["u"], o["Xr"], o["Ur"], o["Wr"]
            steps += 1
            el = time.perf_counter() - t0
            if el >= min_seconds or steps >= max_steps:
                break
    finally:
        oracle.set_num_threads(old)
    return el / steps, steps, used


def precision_errors(case, device):
    """Pattern (1): each output array of one GPU step, FP64 and FP32 fields,
    against the oracle's FP64 step on the same inputs (for FP32 fields the
    oracle takes the FP32-rounded field, promoted).  Normwise
    max|gpu - oracle| / max|oracle| per array."""
    import torch
    from paper_2408_14140_gb300 import api
    out = {}
    for prec, name in ((api.IB_F64, "f64_fields"), (api.IB_F32, "f32_fields")):
        r = Runner(case, prec, device)
        u_in = r.u.double().cpu().numpy()
        r.step()
        torch.cuda.synchronize()
        r.status()
        g = dict(u=r.u, F=r.F, Iu0=r.I0[0], Irxu0=r.I0[1], vol0=r.I0[2], F_ib=r.Fib, T_ib=r.Tib,
                 Iu1=r.I1[0], Irxu1=r.I1[1], vol1=r.I1[2], Xr=r.parts["Xr"], Ur=r.parts["Ur"],
                 Wr=r.parts["Wr"], Fc=r.Fc)
        g = {k: v.double().cpu().numpy() for k, v in g.items()}
        o = oracle_step(case, u_in, case.Xr, case.Ur, case.Wr)
        err = {}
        for k, ov in o.items():
            den = float(np.max(np.abs(ov)))
            err[k] = float(np.max(np.abs(g[k] - ov)) / den) if den > 0 else float(np.max(np.abs(g[k])))
        out[name] = {k: float("%.3g" % v) for k, v in err.items()}
        r.ctx.close()
        r.ctx_v.close()
        del r
    out["gate"] = {"f64_fields": 1e-12, "f32_fields": 2e-5}
    out["metric"] = "max|gpu - oracle| / max|oracle| per array, one full step"
    return out


BATCHED = dict(ncases=256, grids=(32, 48, 64, 96, 128), P_max=8, D_lo=8.0, D_hi=24.0, K=8, Ns=3)
BATCHED_NAME = "batched-256-cases-{32..128}^3-1..8xD8..24-Ns3"


class BatchRunner:
    """Device state of the batched workload (independent periodic cases
    through the batch entry points) and its hot-path step."""

    def __init__(self, cases, prec, device):
        import torch
        from paper_2408_14140_gb300 import api, synth
        self.torch, self.api, self.cases, self.dev = torch, api, cases, device
        self.ctx = api.Context()
        dt = api.field_dtype(prec)
        self.fields = [synth.fourier_eval_torch(c.n, c.meta["modes"], c.h, c.org, device=device)
                       .to(dt).contiguous() for c in cases]
        pl, ml = [], []
        for c in cases:
            _, p, m = api.device_case(c.__class__(**{**c.__dict__, "u": np.zeros((3, 1, 1, 1))}), prec, device)
            pl.append(p)
            ml.append(m)
        self.parts, self.marks, self.ranges, _ = api.pack_batch(pl, ml)
        self.hs = [c.h for c in cases]
        self.shapes = [c.n for c in cases]
        self.phys = [c.phys() for c in cases]
        P, M = self.parts["Xr"].shape[0], self.marks["R"].shape[0]
        z = lambda *sh: torch.zeros(sh, dtype=torch.float64, device=device)  # noqa: E731
        self.F = z(M, 3)
        self.I0 = (z(P, 3), z(P, 3), z(P))
        self.I1 = (z(P, 3), z(P, 3), z(P))
        self.Fib, self.Tib, self.Fc = z(P, 3), z(P, 3), z(P, 3)
        self.M = M
        self.Ns = cases[0].Ns
        self.dt = cases[0].dt
        # the case table uploaded once: the batch calls below stage nothing
        # on the host, so the step can be captured into a CUDA graph
        self.table = api.BatchTable(self.ctx, self.fields, self.hs, self.ranges, P, phys=self.phys)

    def status(self):
        self.ctx.status()

    def step(self):
        ctx, t = self.ctx, self.table
        ctx.ib_batch_table_volume_integrals(t, self.parts, out=self.I0)
        ctx.ib_batch_table_multidirect_forcing(t, self.parts, self.marks, self.Ns, self.dt, F_out=self.F)
        ctx.particle_force_torque(self.parts, self.marks, self.F, 1.0, out=(self.Fib, self.Tib))
        ctx.ib_batch_table_volume_integrals(t, self.parts, out=self.I1)
        ctx.ib_batch_table_collide_update(t, self.parts, self.dt, self.Fib, self.Tib, self.I1[0], self.I0[0],
                                          self.I1[1], self.I0[1], Fc_out=self.Fc)

    def close(self):
        self.table.close()
        self.ctx.close()


def run_batched(args, device, hbm):
    """The batched workload: every case advanced by one hot-path step per
    step, all cases in the same launches (FP32 fields), the case table
    uploaded once and the step replayed from a CUDA graph.  The fields
    (2.3 GB) exceed L2, so no flush is needed between steps."""
    import torch
    from paper_2408_14140_gb300 import synth
    b = BATCHED
    cases = synth.batched_cases(b["ncases"], seed=0, grids=b["grids"], P_max=b["P_max"], D_lo=b["D_lo"],
                                D_hi=b["D_hi"], K=b["K"], Ns=b["Ns"])
    r = BatchRunner(cases, 1, device)
    steps = max(3, min(args.steps // 10, 20))
    # launch choices picked by the autotuner on this workload (the tuning
    # steps also serve as warm-up)
    from paper_2408_14140_gb300 import autotune
    tuned = autotune.tune([r.ctx], r.step, warmup=1, reps=3, steps_per_rep=1)
    graph = capture(r) if not args.no_graph else None
    run = graph.replay if graph is not None else r.step
    for _ in range(args.warmup):
        run()
    torch.cuda.synchronize()
    r.ctx.status()
    a, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    for _ in range(steps):
        run()
    e.record()
    torch.cuda.synchronize()
    r.ctx.status()
    step_s = a.elapsed_time(e) / 1000.0 / steps
    # per-phase device time
    for ph in r.api.PHASES:
        r.ctx.read_timing(ph)
    r.ctx.set_timing(True)
    for _ in range(3):
        r.step()
    torch.cuda.synchronize()
    r.ctx.set_timing(False)
    kt = {}
    for ph in r.api.PHASES:
        ms, n = r.ctx.read_timing(ph)
        if n:
            kt[ph] = (ms, n)
    # compulsory bytes by the method's count, summed over the cases
    s = 4
    B = sum(band_cells(c) for c in cases)
    nlev = max(wavefront_levels(c) for c in cases)
    b_ib = 6 * s * B + 24 * r.M
    b_vol = 3 * s * sum(interior_cells(c) for c in cases)
    ms_g, n_g = kt.get("mdf_gather", (float("nan"), 1))
    g_dur = ms_g / n_g / 1000.0
    per_launch = b_ib / (r.Ns * nlev)
    step_b = b_ib + 2 * b_vol
    out = {"workload": BATCHED_NAME, "cases": len(cases), "particles": int(r.parts["Xr"].shape[0]),
           "markers": r.M, "cells": int(sum(np.prod(c.n) for c in cases)), "band_cells": B,
           "levels": nlev, "Ns": r.Ns, "dtype": "f32 fields, f64 forces/reductions",
           "value": r.M * r.Ns / step_s, "unit": "marker-updates/s", "ms_per_step": step_s * 1000.0,
           "steps": steps, "launch": ("cuda-graph replay" if graph is not None else "eager") +
                                     " (case table uploaded once)",
           "autotune": {"choice": tuned["choice"],
                        "table": [{"choice": c, "ms": round(ms, 3)} for c, ms in tuned["table"]]},
           "l2": "inputs larger than L2 (2.3 GB of fields)",
           "phases_us": {k: round(v[0] / v[1] * 1000.0, 2) for k, v in kt.items()},
           "roofline": {"bound": "hbm", "kernel": "k_gather_level", "achieved": per_launch / g_dur / 1e9,
                        "peak": hbm, "unit": "GB/s", "frac": per_launch / g_dur / 1e9 / hbm,
                        "algorithmic_bytes_per_launch": per_launch, "duration_us": g_dur * 1e6,
                        "step": {"algorithmic_bytes": step_b, "b_ib": b_ib, "b_vol_per_call": b_vol,
                                 "ms": step_s * 1000.0, "achieved": step_b / step_s / 1e9,
                                 "frac": step_b / step_s / 1e9 / hbm}}}
    del graph
    r.close()
    return out


def run_serving(args):
    """The served workload: a Poisson request stream through the
    continuous-batching loop, mixed FP32/FP64 fields, and the same trace
    all-FP32 and all-FP64 for the precision comparison."""
    from paper_2408_14140_gb300 import api, serve
    out = {"workload": "poisson-%g/s-%gs-grids48..192-1..32xD8..24-20steps-Ns3-tgv" % (
        args.serve_rate, args.serve_seconds)}
    results = {}
    cfg = serve.ServeConfig(rate=args.serve_rate, seconds=args.serve_seconds, fp64_fraction=0.25, seed=0)
    base = serve.make_trace(cfg)
    # a short untimed trace first: the first served requests of a process pay
    # one-time costs (contexts' workspace growth, pinned staging)
    warm = serve.ServeConfig(rate=args.serve_rate, seconds=0.3, fp64_fraction=0.5, seed=1)
    wsrv = serve.Server(warm)
    wsrv.run(serve.make_trace(warm))
    wsrv.close()
    graphs = serve.ServeConfig(rate=args.serve_rate, seconds=args.serve_seconds, fp64_fraction=0.25, seed=0,
                               graph_after=4)
    for name, prec, c in (("mixed", None, cfg), ("fp32", api.IB_F32, cfg), ("fp64", api.IB_F64, cfg),
                          ("mixed_graph_replay", None, graphs)):
        trace = [serve.Request(r.rid, r.arrival, r.case, r.prec if prec is None else prec) for r in base]
        srv = serve.Server(c)
        t0 = time.perf_counter()
        srv.run(trace)
        wall = time.perf_counter() - t0
        srv.close()
        s = serve.summarize(trace, c, wall)
        s.update(srv.stats())
        s["graph_after"] = c.graph_after
        for p_, nm in ((api.IB_F32, "fp32"), (api.IB_F64, "fp64")):
            lat = np.array([r.latency for r in trace if r.prec == p_ and r.latency is not None])
            if lat.size:
                s["p99_ms_" + nm + "_requests"] = float(np.percentile(lat, 99) * 1e3)
        s["active_peak"] = srv.active_peak
        s["fp64_requests"] = sum(r.prec == api.IB_F64 for r in trace)
        out[name] = s
        results[name] = trace
    # accuracy of the FP32 form: one time step of the first requests alone in
    # FP32 against the same step in FP64 (velocities after the Newton-Euler
    # update; over many coupled steps the stiff collision law amplifies any
    # difference, so the per-step figure is the meaningful one)
    one = serve.ServeConfig(rate=args.serve_rate, seconds=args.serve_seconds, steps=1, seed=0)
    err = {"Ur": 0.0, "Wr": 0.0}
    for r in base[:16]:
        a = serve.serve_alone(one, serve.Request(r.rid, r.arrival, r.case, api.IB_F32))
        b = serve.serve_alone(one, serve.Request(r.rid, r.arrival, r.case, api.IB_F64))
        for k in err:
            x, y = a[k].numpy(), b[k].numpy()
            err[k] = max(err[k], float(np.max(np.abs(x - y)) / max(np.max(np.abs(y)), 1e-300)))
    out["fp32_vs_fp64_one_step"] = {"requests": 16, "max_rel_diff": err}
    out["budget_bytes"] = serve.ServeConfig().budget_bytes
    out["max_active"] = serve.ServeConfig().max_active
    return out


DENSE = dict(N=384, P=512, D=16.0, phi=0.3, K=16, Ns=3, dt=1e-3, min_gap=0.25)
DENSE_NAME = "dense-384^3-512xD16-phi0.3-Ns3"


def make_dense_case(seed=1):
    from paper_2408_14140_gb300 import synth
    w = DENSE
    return synth.cluster_case(N=w["N"], P=w["P"], D_cells=w["D"], phi=w["phi"], K=w["K"], Ns=w["Ns"],
                              dt=w["dt"], seed=seed, min_gap_cells=w["min_gap"], build_field=False)


def roofline_of(case, s, lb, step_s, kt, hbm, hbm_src, traffic):
    """Roofline objects from the method's compulsory bytes (B_IB per step,
    B_IB / (Ns * wavefronts) per gather launch, 3 s N_int per volume call)."""
    B = sum(bl for bl, _ in lb) if lb else band_cells(case)
    b_ib, b_vol = step_bytes(case, s, band_cells(case))
    nlev = max(1, len(lb))
    ms_g, n_g = kt.get("mdf_gather", (float("nan"), 1))
    g_dur = ms_g / n_g / 1000.0
    per_launch = b_ib / (case.Ns * nlev)
    ach = per_launch / g_dur / 1e9
    step_b = b_ib + 2 * b_vol
    ach_s = step_b / step_s / 1e9
    return {"bound": "hbm", "kernel": "k_gather_level", "achieved": ach, "peak": hbm, "unit": "GB/s",
            "frac": ach / hbm, "traffic": traffic, "peak_source": hbm_src,
            "algorithmic_bytes_per_launch": per_launch, "duration_us": g_dur * 1e6,
            "launches_per_step": case.Ns * nlev,
            "step": {"algorithmic_bytes": step_b, "b_ib": b_ib, "b_vol_per_call": b_vol,
                     "ms": step_s * 1000.0, "achieved": ach_s, "frac": ach_s / hbm},
            "band_cells_sum_over_wavefronts": B}


def config_of(case, fields, B, nlev, world):
    """The workload's description (the same for both arms)."""
    return {"workload": WORKLOAD_NAME, "grid": [256, 256, 256], "particles": case.P,
            "markers": case.M, "Ns": case.Ns, "kernel": "roma3", "order": "sequential",
            "fields": fields, "band_cells": B, "levels": nlev,
            "parallelism": "replicas" if world > 1 else "single-gpu",
            "l2": "flushed (512 MiB write) between timed steps"}


def run_gpu(args):
    import torch
    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    device = torch.device("cuda", torch.cuda.current_device())
    from paper_2408_14140_gb300 import api, build

    if rank == 0 or not os.path.exists(build.LIB):
        build.build()
    if world > 1:
        dist.barrier()
    case = make_case(seed=rank)
    M, Ns = case.M, case.Ns
    flush = torch.empty(512 << 20 >> 2, dtype=torch.float32, device=device)
    hbm, hbm_src = peaks()
    B = band_cells(case)
    lb = level_band_cells(case)
    nlev = len(lb)

    results = {}
    precs = {"both": (api.IB_F64, api.IB_F32), "f32": (api.IB_F32,), "f64": (api.IB_F64,)}[args.prec]
    reps = (0, 0) if world > 1 or args.no_replays else (5, 100)
    for prec in precs:
        r = Runner(case, prec, device)
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()
        clk = ClockSampler(local)
        clk.start()
        ms, graphed, blocks = time_steps(r, args.steps, args.warmup, flush, not args.no_graph, reps)
        clocks = clk.stop()
        t_rank = max_over_ranks(sum(ms) / 1000.0, device)
        kt = kernel_timing(r, max(3, min(args.steps, 10)), flush)
        e2e = None
        if not args.no_e2e:
            # two more replicas: uploads and downloads overlap compute
            partners = [Runner(case, prec, device) for _ in range(2)]
            e2e = e2e_steps(r, max(6, min(args.steps, 30)), partners)
            del partners
        results[prec] = dict(ms=ms, t=t_rank, graphed=graphed, clocks=clocks, kt=kt, e2e=e2e, blocks=blocks)
        r.ctx.close()
        r.ctx_v.close()
        del r
    if rank != 0:
        if world > 1:
            dist.barrier()
            dist.destroy_process_group()
        return

    def form(prec):
        res = results[prec]
        s = 8 if prec == api.IB_F64 else 4
        step_s = res["t"] / args.steps
        o = {"value": job_value(M, Ns, world, step_s), "unit": "marker-updates/s",
             "ms_per_step": step_s * 1000.0,
             "launch": "cuda-graph replay" if res["graphed"] else "eager",
             "roofline": roofline_of(case, s, lb, step_s, res["kt"], hbm, hbm_src,
                                     recorded_traffic("k_gather_level", "f64" if s == 8 else "f32")),
             "phases_us": {k: round(v[0] / v[1] * 1000.0, 2) for k, v in res["kt"].items()},
             "clocks": res["clocks"]}
        if res["blocks"]:
            o["replays"] = {"repeats": len(res["blocks"]), "per_repeat": reps[1],
                            "ms_per_step_each": [round(x, 4) for x in res["blocks"]],
                            "ms_per_step_median": statistics.median(res["blocks"]),
                            "value_median": M * Ns / (statistics.median(res["blocks"]) / 1000.0)}
        if res["e2e"]:
            dt, bi, bo = res["e2e"]
            o["e2e"] = {"value": world * M * Ns / dt, "unit": "marker-updates/s",
                        "h2d_bytes_per_step": bi, "d2h_bytes_per_step": bo,
                        "pipeline": "3 device replicas in turn, one copy stream per direction"}
        return o

    head = api.IB_F64 if api.IB_F64 in results else api.IB_F32
    h = form(head)
    line = {
        "metric": METRIC,
        "value": h["value"],
        "unit": "marker-updates/s",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": h["ms_per_step"],
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f64" if head == api.IB_F64 else "f32 fields, f64 forces/reductions",
        "data": "synthetic",
        "config": config_of(case, "f64" if head == api.IB_F64 else "f32", B, nlev, world),
        "e2e": h.get("e2e"),
        "gpu_launches": args.steps * launches_per_step(Ns, nlev),
        "launch": h["launch"],
        "roofline": h["roofline"],
        "phases_us": h["phases_us"],
        "clocks": h["clocks"],
    }
    if "replays" in h:
        line["replays"] = h["replays"]
    if api.IB_F32 in results and head != api.IB_F32:
        line["fp32"] = form(api.IB_F32)
        line["fp32"]["dtype"] = "f32 fields, f64 forces/reductions"
    if world == 1 and not args.no_variants:
        # the same workload with the other particle order and the other kernel
        # (FP32 fields), each a full step timed like the main line
        line["variants"] = {}
        for name, delta, order, mode in (("simultaneous_order", 0, 1, "gather"), ("peskin4_kernel", 1, 0, "gather"),
                                         ("atomic_spread", 0, 0, "atomic")):
            rv = Runner(case, api.IB_F32, device, delta=delta, order=order)
            rv.ctx.set_spread_mode(mode)
            msv, gv, _ = time_steps(rv, max(3, args.steps // 4), args.warmup, flush, not args.no_graph)
            ktv = kernel_timing(rv, 3, flush)
            tv = sum(msv) / 1000.0 / len(msv)
            line["variants"][name] = {"value": M * Ns / tv, "unit": "marker-updates/s",
                                      "ms_per_step": tv * 1000.0, "steps": len(msv), "spread": mode,
                                      "dtype": "f32 fields, f64 forces/reductions",
                                      "launch": "cuda-graph replay" if gv else "eager",
                                      "phases_us": {k: round(v[0] / v[1] * 1000.0, 2) for k, v in ktv.items()}}
            rv.ctx.close()
            rv.ctx_v.close()
            del rv
    if world == 1 and not args.no_dense:
        line["dense"] = run_dense(args, device, flush, hbm, hbm_src)
    if world == 1 and not args.no_single_level:
        line["single_level_step"] = run_single_level(args, device, flush, hbm)
    if world == 1 and not args.no_batched:
        line["batched"] = run_batched(args, device, hbm)
    if world == 1 and not args.no_serve:
        line["serving"] = run_serving(args)
    if world == 1 and not args.no_cpu_baseline:
        from paper_2408_14140_gb300 import synth
        case.u = synth.fourier_eval_torch(case.n, case.meta["modes"], case.h, case.org,
                                          device=device).cpu().numpy()
        line["precision"] = precision_errors(case, device)
        t_all, n_all, thr = cpu_baseline(case, os.cpu_count() or 1)
        t_one, n_one, _ = cpu_baseline(case, 1, min_seconds=5.0, max_steps=3)
        line["cpu_baseline"] = {"value": M * Ns / t_all, "unit": "marker-updates/s",
                                "cores": thr, "kind": "oracle",
                                "sample": "%d full FP64 step(s) of the same workload on %d OpenMP threads "
                                          "(only the interpolation and volume-integral loops are "
                                          "threaded; the forcing loop is serial)" % (n_all, thr),
                                "single_thread": {"value": M * Ns / t_one, "ms_per_step": t_one * 1000.0,
                                                  "sample": "%d full FP64 step(s), 1 thread" % n_one},
                                "all_core": {"value": M * Ns / t_all, "ms_per_step": t_all * 1000.0,
                                             "threads": thr, "nproc": os.cpu_count()}}
    print(json.dumps(line))
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()


class LevelRunner(Runner):
    """The whole single-level step of Sec. 3.1 on the bench workload: the
    momentum predictor (Step 1), the hot path (Step 2 with the volume
    integrals, reductions and particle update) and the level projection
    (Step 3), one after another on the same field."""

    def __init__(self, case, prec, device):
        super().__init__(case, prec, device)
        torch = self.torch
        n = case.n
        self.p = torch.zeros((n[2], n[1], n[0]), dtype=self.u.dtype, device=device)
        self.u_star = torch.empty_like(self.u)
        self.mu = 1e-3

    def step(self):
        c, ctx, torch = self.case, self.ctx, self.torch
        ctx.fluid_predictor(self.u, self.p, c.h, c.rho_f, self.mu, (0.0, 0.0, 0.0), c.dt, u_star=self.u_star)
        self.u, self.u_star = self.u_star, self.u
        super().step()
        ctx.level_projection(self.u, self.p, c.h, c.rho_f, c.dt)


def run_single_level(args, device, flush, hbm):
    """NEXT row: the full single-level step on the 256^3 / 64 x D24 workload,
    FP32 and FP64 fields, CUDA-graph replayed.  Compulsory bytes of the fluid
    calls: the predictor reads u (3 s N) and p (s N) and writes u* (3 s N);
    the projection reads and writes u and p (8 s N); the FFT passes between
    are the solver's own traffic."""
    from paper_2408_14140_gb300 import api
    case = make_case(seed=0)
    N = int(np.prod(case.n))
    out = {"workload": WORKLOAD_NAME + "+predictor+projection", "grid": list(case.n),
           "l2": "flushed (512 MiB write) between timed steps"}
    for prec, name in ((api.IB_F32, "fp32"), (api.IB_F64, "fp64")):
        r = LevelRunner(case, prec, device)
        ms, graphed, _ = time_steps(r, max(3, min(args.steps // 4, 10)), args.warmup, flush, not args.no_graph)
        kt = kernel_timing(r, 3, flush)
        s = 8 if prec == api.IB_F64 else 4
        step_s = sum(ms) / 1000.0 / len(ms)
        o = {"ms_per_step": step_s * 1000.0, "value": case.M * case.Ns / step_s, "unit": "marker-updates/s",
             "steps": len(ms), "launch": "cuda-graph replay" if graphed else "eager",
             "phases_us": {k: round(v[0] / v[1] * 1000.0, 2) for k, v in kt.items()}}
        for ph, nbytes in (("fluid_predictor", 7 * s * N), ("fluid_projection", 8 * s * N)):
            if ph in kt:
                dur = kt[ph][0] / kt[ph][1] / 1000.0
                o[ph] = {"algorithmic_bytes": nbytes, "duration_us": dur * 1e6,
                         "achieved_gbs": nbytes / dur / 1e9, "frac_of_peak": nbytes / dur / 1e9 / hbm}
        out[name] = o
        r.ctx.close()
        r.ctx_v.close()
        del r
    return out


def run_dense(args, device, flush, hbm, hbm_src):
    """The dense cluster: 384^3, 512 spheres of D = 16 at volume fraction 0.3
    (gaps below h, collision forces active), Ns = 3, FP32 fields with FP64
    forces and reductions, the whole step replayed from a CUDA graph."""
    from paper_2408_14140_gb300 import api
    case = make_dense_case()
    lb = level_band_cells(case)
    r = Runner(case, api.IB_F32, device)
    steps = max(5, min(args.steps // 4, 50))
    ms, graphed, _ = time_steps(r, steps, args.warmup, flush, not args.no_graph)
    kt = kernel_timing(r, 3, flush)
    step_s = sum(ms) / 1000.0 / len(ms)
    contacts = int(np.count_nonzero(np.any(r.Fc.cpu().numpy() != 0, axis=1)))
    out = {"workload": DENSE_NAME, "grid": [384, 384, 384], "particles": case.P, "markers": case.M,
           "Ns": case.Ns, "levels": len(lb), "band_cells": band_cells(case),
           "dtype": "f32 fields, f64 forces/reductions", "value": case.M * case.Ns / step_s,
           "unit": "marker-updates/s", "ms_per_step": step_s * 1000.0, "steps": len(ms),
           "launch": "cuda-graph replay" if graphed else "eager",
           "l2": "flushed (512 MiB write) between timed steps",
           "particles_in_contact": contacts,
           "gpu_launches_per_step": launches_per_step(case.Ns, len(lb)),
           "roofline": roofline_of(case, 4, lb, step_s, kt, hbm, hbm_src, None),
           "phases_us": {k: round(v[0] / v[1] * 1000.0, 2) for k, v in kt.items()}}
    r.ctx.close()
    r.ctx_v.close()
    return out


def run_reference(args):
    """The FP64 oracle timed on the host cores on this workload (the reference
    arm for a paper with no published implementation)."""
    rank, world, _ = dist_env()
    if rank != 0:
        return
    from paper_2408_14140_gb300 import synth
    import oracle
    case = make_case(seed=0)
    case.u = synth.fourier_eval(case.n, case.meta["modes"], case.h, case.org)
    oracle.build()
    c = case
    st = dict(u=c.u.copy(), Xr=c.Xr.copy(), Ur=c.Ur.copy(), Wr=c.Wr.copy())

    def step():
        o = oracle_step(c, st["u"], st["Xr"], st["Ur"], st["Wr"])
        st.update(u=o["u"], Xr=o["Xr"], Ur=o["Ur"], Wr=o["Wr"])

    for _ in range(args.warmup):
        step()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        step()
    dt = (time.perf_counter() - t0) / args.steps
    v = c.M * c.Ns / dt
    thr = oracle.num_threads()
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "marker-updates/s",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": dt * 1000.0, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": config_of(c, "f64", band_cells(c), wavefront_levels(c), world),
            "cpu_baseline": {"value": v, "unit": "marker-updates/s", "cores": thr,
                             "kind": "oracle",
                             "sample": "%d full FP64 steps of the same workload on %d OpenMP threads "
                                       "(the forcing loop is serial)" % (args.steps, thr)},
            "e2e": {"value": v, "unit": "marker-updates/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gbib", choices=["gbib", "reference"])
    ap.add_argument("--no-graph", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--prec", default="both", choices=["both", "f32", "f64"])
    ap.add_argument("--no-batched", action="store_true")
    ap.add_argument("--no-variants", action="store_true")
    ap.add_argument("--no-serve", action="store_true")
    ap.add_argument("--no-dense", action="store_true")
    ap.add_argument("--no-single-level", action="store_true")
    ap.add_argument("--no-replays", action="store_true")
    ap.add_argument("--serve-rate", type=float, default=200.0)
    ap.add_argument("--serve-seconds", type=float, default=2.0)
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
