"""Continuous-batching request loop over the batch entry points.

Each request is an independent periodic case -- its own grid, background
flow and spheres -- that runs ``steps`` time steps of the hot path of
Sec. 3.1 (Step 2) on a prescribed flow:

    u <- background flow (restored every step)
    (I_u, I_w, V)_old = PVF volume integrals (Eq. pr2)
    F = multidirect forcing, Ns passes (Algorithm 1)      -> u corrected
    (F_ib, T_ib)  = marker force and torque sums (Eq. pr2)
    (I_u, I_w, V)_new = PVF volume integrals
    collision forces (Eq. DKT_model) + Newton-Euler update (Eq. pr2)

The server keeps every admitted request's field, background flow, particle
state and markers resident on the device.  Requests wait in one queue per
field precision and are admitted first come, first served within it, while
the shared device-memory budget and the precision's slot count allow (a
blocked head of one precision does not hold back the other).  Each loop
iteration advances every active request by one time step through one
sequence of batch launches per precision -- the batch's case table
re-uploaded asynchronously once per change of its active set, the
precisions on separate streams so their steps overlap on the device, and
(optionally) a step replayed from a CUDA graph while the active set stays
the same -- so requests that arrived at different times share the same
kernels.  A request that has run all its
steps has its particle state copied to pinned host memory; its latency runs
from its arrival to that copy's completion.

Only argument marshalling and bookkeeping happen here (PyTorch holds the
device memory); every step of the method runs in the library's kernels.
"""
from __future__ import annotations

import math
import time
from dataclasses import dataclass

import numpy as np
import torch

from . import api, synth


@dataclass
class ServeConfig:
    rate: float = 200.0            # Poisson arrival rate (requests/s)
    seconds: float = 2.0           # length of the arrival trace
    grids: tuple = tuple(range(48, 193, 16))
    P_max: int = 32
    D_lo: float = 8.0
    D_hi: float = 24.0
    Ns: int = 3
    steps: int = 20
    dt: float = 1e-3
    U0: float = 1.0                # Taylor-Green amplitude
    fp64_fraction: float = 0.0     # share of requests served with FP64 fields
    budget_bytes: int = 32 << 30   # device memory for resident requests
    max_active: int = 64           # active requests per field precision
    graph_after: int = 0           # replay a group's step from a CUDA graph once its
                                   # active set has not changed for this many steps (0: never;
                                   # on a Poisson stream the set changes every few steps and a
                                   # capture costs more host time than its replays save)
    volume_split: int = 8          # CTAs per particle of the volume integrals: fixed, so a
                                   # request's sums do not depend on which requests share its batch
    seed: int = 0


@dataclass
class Request:
    rid: int
    arrival: float                 # seconds from the start of the trace
    case: synth.Case
    prec: int
    bytes: int = 0
    # device state (while active)
    u: torch.Tensor | None = None
    u_bg: torch.Tensor | None = None
    parts: dict | None = None
    marks: dict | None = None
    steps_done: int = 0
    # completion
    host: dict | None = None
    event: torch.cuda.Event | None = None
    done_time: float | None = None

    @property
    def latency(self):
        return None if self.done_time is None else self.done_time - self.arrival


def make_trace(cfg: ServeConfig):
    """Seeded Poisson arrivals with their cases (geometry only; the flow is
    the Taylor-Green vortex evaluated on the device at admission)."""
    rng = synth.SplitMix64(cfg.seed)
    out, t, rid = [], 0.0, 0
    while True:
        u = rng.uniform()
        t += -math.log(1.0 - u) / cfg.rate
        if t >= cfg.seconds:
            break
        N = int(cfg.grids[rng.randint(0, len(cfg.grids) - 1)])
        P = rng.randint(1, cfg.P_max)
        case = synth.random_case(N, P, cfg.D_lo, cfg.D_hi, 0, cfg.Ns, rng, cfg.dt, field_kind="none")
        prec = api.IB_F64 if rng.uniform() < cfg.fp64_fraction else api.IB_F32
        out.append(Request(rid, t, case, prec))
        rid += 1
    return out


def request_bytes(case: synth.Case, prec: int) -> int:
    """Device bytes a request holds while active: field and background flow,
    markers and their per-call state, particles (estimate, with the batch's
    flat copies)."""
    s = 8 if prec == api.IB_F64 else 4
    cells = int(np.prod(case.n))
    fields = 2 * 3 * cells * s
    markers = case.M * (3 * 8 + 8) * 2 + case.M * (3 * 8 + 16 * s + 8 + 27 * 4 * 2)
    particles = case.P * (3 * 3 * 8 + 16) * 4
    return fields + markers + particles + (1 << 16)


def admit_count(waiting_bytes, used: int, budget: int, n_active: int, max_active: int) -> int:
    """How many requests at the head of the FIFO queue (their device bytes
    in arrival order) are admitted now: while a slot is free and the head
    fits in what is left of the budget.  A head that does not fit blocks the
    requests behind it (no overtaking)."""
    k = 0
    for b in waiting_bytes:
        if n_active + k >= max_active or used + b > budget:
            break
        used += b
        k += 1
    return k


class Group:
    """Active requests of one field precision: their flat batch arrays, the
    batch's case table on the device, and the group's own stream, so that the
    two precisions' steps overlap on the device."""

    def __init__(self, prec: int, ctx: api.Context, device):
        self.prec = prec
        self.ctx = ctx
        # the FP64 group's steps are the slower ones and set the latency
        # tail, so its stream gets the higher scheduling priority
        self.stream = torch.cuda.Stream(device=device, priority=-1 if prec == api.IB_F64 else 0)
        self.active: list[Request] = []
        self.dirty = True
        self.table = None
        self.graph = None
        self.stable = 0          # steps since the active set last changed
        self.graph_steps = 0     # steps replayed from a graph
        self.eager_steps = 0
        self.host_s = {"rebuild": 0.0, "eager": 0.0, "capture": 0.0, "replay": 0.0}  # host seconds

    def rebuild(self, device):
        """Lay the active requests out as one flat particle/marker set; the
        requests' particle tensors become views of the flat arrays; upload the
        batch's case table once."""
        reqs = self.active
        self.parts, self.marks, self.ranges, _ = api.pack_batch([r.parts for r in reqs],
                                                                [r.marks for r in reqs])
        for r, (p0, p1) in zip(reqs, self.ranges):
            for k in ("Xr", "Ur", "Wr"):
                r.parts[k] = self.parts[k][p0:p1]
        self.fields = [r.u for r in reqs]
        self.bgs = [r.u_bg for r in reqs]
        hs = [r.case.h for r in reqs]
        phys = [r.case.phys() for r in reqs]
        P, M = self.parts["Xr"].shape[0], self.marks["R"].shape[0]
        f64 = dict(dtype=torch.float64, device=device)
        self.F = torch.empty((M, 3), **f64)
        self.Fib = torch.empty((P, 3), **f64)
        self.Tib = torch.empty((P, 3), **f64)
        self.Fc = torch.empty((P, 3), **f64)
        self.I_old = (torch.empty((P, 3), **f64), torch.empty((P, 3), **f64), torch.empty((P,), **f64))
        self.I_new = (torch.empty((P, 3), **f64), torch.empty((P, 3), **f64), torch.empty((P,), **f64))
        if self.table is None:
            self.table = api.BatchTable(self.ctx, self.fields, hs, self.ranges, P, phys=phys)
        else:  # re-upload on the group's stream: no device-wide wait
            self.table.update(self.fields, hs, self.ranges, P, phys=phys, stream=self.stream)
        self.graph = None
        self.stable = 0
        self.dirty = False

    def launch(self, cfg: ServeConfig):
        """One time step of every active request (enqueued on the current stream)."""
        torch._foreach_copy_(self.fields, self.bgs)
        c, t = self.ctx, self.table
        c.ib_batch_table_volume_integrals(t, self.parts, out=self.I_old)
        c.ib_batch_table_multidirect_forcing(t, self.parts, self.marks, cfg.Ns, cfg.dt, F_out=self.F)
        c.particle_force_torque(self.parts, self.marks, self.F, 1.0, out=(self.Fib, self.Tib))
        c.ib_batch_table_volume_integrals(t, self.parts, out=self.I_new)
        c.ib_batch_table_collide_update(t, self.parts, cfg.dt, self.Fib, self.Tib, self.I_new[0], self.I_old[0],
                                        self.I_new[1], self.I_old[1], Fc_out=self.Fc)

    def step(self, cfg: ServeConfig, device):
        if not self.active:
            return
        # every device operation of the group (its allocations included) runs
        # on the group's stream, so it is ordered after the group's last step
        with torch.cuda.stream(self.stream):
            t0 = time.perf_counter()
            if self.dirty:
                self.rebuild(device)
            t1 = time.perf_counter()
            self.host_s["rebuild"] += t1 - t0
            if self.graph is not None:
                self.graph.replay()
                self.graph_steps += 1
                self.host_s["replay"] += time.perf_counter() - t1
            else:
                self.launch(cfg)
                self.eager_steps += 1
                self.stable += 1
                t2 = time.perf_counter()
                self.host_s["eager"] += t2 - t1
                if cfg.graph_after and self.stable >= cfg.graph_after:
                    # the step's launch sequence, captured once for the steps
                    # that follow while the active set stays the same (the
                    # eager steps have sized the workspace)
                    g = torch.cuda.CUDAGraph()
                    with torch.cuda.graph(g, stream=self.stream):
                        self.launch(cfg)
                    self.graph = g
                    # capture records the work without running it: this step ran eagerly
                    self.host_s["capture"] += time.perf_counter() - t2
        for r in self.active:
            r.steps_done += 1


class Server:
    """Admission by device-memory budget, one batch step per group and
    iteration.  Each field precision has its own FIFO queue, slot count and
    stream; the device-memory budget is shared."""

    def __init__(self, cfg: ServeConfig, device="cuda"):
        self.cfg = cfg
        self.device = device
        self.groups = {p: Group(p, api.Context(), device) for p in (api.IB_F32, api.IB_F64)}
        for g in self.groups.values():
            g.ctx.set_volume_split(cfg.volume_split)
        self.waiting = {p: [] for p in self.groups}
        self.finishing: list[Request] = []
        self.used = 0
        self.active_peak = 0

    def n_active(self):
        return sum(len(g.active) for g in self.groups.values())

    def n_waiting(self):
        return sum(len(q) for q in self.waiting.values())

    def admit(self, r: Request):
        c = r.case
        dt = api.field_dtype(r.prec)
        g = self.groups[r.prec]
        with torch.cuda.stream(g.stream):  # the request's memory belongs to its group's stream
            r.u_bg = synth.taylor_green_torch(c.n, self.cfg.U0, c.h, device=self.device, dtype=dt)
            r.u = torch.empty_like(r.u_bg)

            # pinned, non-blocking uploads: a pageable copy would make the
            # host wait for the group's queued steps
            def up(a, dtype=torch.float64):
                return torch.as_tensor(np.ascontiguousarray(a)).to(dtype).pin_memory().to(
                    self.device, non_blocking=True)

            r.parts = dict(Xr=up(c.Xr), Ur=up(c.Ur), Wr=up(c.Wr), radius=up(c.radius), rho_p=up(c.rho_p),
                           moff=up(c.moff, torch.int32))
            r.marks = dict(R=up(c.R), dV=up(c.dV))
        self.used += r.bytes
        g.active.append(r)
        g.dirty = True

    def retire(self, r: Request):
        g = self.groups[r.prec]
        g.active.remove(r)
        g.dirty = True
        r.host = {k: torch.empty(r.parts[k].shape, dtype=torch.float64, pin_memory=True)
                  for k in ("Xr", "Ur", "Wr")}
        with torch.cuda.stream(g.stream):
            for k, t in r.host.items():
                t.copy_(r.parts[k], non_blocking=True)
            r.event = torch.cuda.Event()
            r.event.record(g.stream)
        r.u = r.u_bg = None
        self.finishing.append(r)

    def poll(self, now_fn):
        still = []
        for r in self.finishing:
            if r.event.query():
                r.done_time = now_fn()
                self.used -= r.bytes
            else:
                still.append(r)
        self.finishing = still

    def run(self, trace: list[Request], sync_every_step: bool = False):
        """Serve the trace in real time; returns the requests (with latencies)."""
        cfg = self.cfg
        for r in trace:
            r.bytes = request_bytes(r.case, r.prec)
            if r.bytes > cfg.budget_bytes:
                raise ValueError("request %d needs %d bytes, over the budget" % (r.rid, r.bytes))
        pending = list(trace)
        t0 = time.perf_counter()
        now = lambda: time.perf_counter() - t0
        # each group's steps in flight (events on its stream): a group with
        # `depth` steps outstanding waits its turn, the other goes on, so one
        # precision's pace does not gate the other's
        inflight = {p: [] for p in self.groups}
        depth = 1 if sync_every_step else 3
        while pending or self.n_waiting() or self.n_active() or self.finishing:
            tnow = now()
            while pending and pending[0].arrival <= tnow:
                r = pending.pop(0)
                self.waiting[r.prec].append(r)
            for p, q in self.waiting.items():
                k = admit_count([r.bytes for r in q], self.used, cfg.budget_bytes, len(self.groups[p].active),
                                cfg.max_active)
                for _ in range(k):
                    self.admit(q.pop(0))
            self.active_peak = max(self.active_peak, self.n_active())
            if self.n_active():
                stepped = False
                for p, g in self.groups.items():
                    q = inflight[p]
                    while q and q[0].query():
                        q.pop(0)
                    if not g.active or len(q) >= depth:
                        continue
                    g.step(cfg, self.device)
                    for r in [r for r in g.active if r.steps_done >= cfg.steps]:
                        self.retire(r)
                    ev = torch.cuda.Event()
                    ev.record(g.stream)
                    q.append(ev)
                    stepped = True
                if sync_every_step:
                    for q in inflight.values():
                        for ev in q:
                            ev.synchronize()
                        q.clear()
                elif not stepped:
                    # every active group has `depth` steps outstanding: wait for
                    # the oldest step of either group (whichever finishes first)
                    oldest = [q[0] for q in inflight.values() if q]
                    while oldest and not any(ev.query() for ev in oldest):
                        time.sleep(20e-6)
            else:
                self.poll(now)
                if not self.finishing:
                    nxt = pending[0].arrival if pending else tnow
                    time.sleep(max(0.0, min(nxt - now(), 0.002)))
                continue
            self.poll(now)
        torch.cuda.synchronize()
        for g in self.groups.values():
            g.ctx.status()
        return trace

    def stats(self):
        host = {}
        for g in self.groups.values():
            for k, v in g.host_s.items():
                host[k] = round(host.get(k, 0.0) + v, 4)
        return {"graph_steps": sum(g.graph_steps for g in self.groups.values()),
                "eager_steps": sum(g.eager_steps for g in self.groups.values()),
                "host_seconds": host}

    def close(self):
        torch.cuda.synchronize()
        for g in self.groups.values():
            if g.table is not None:
                g.table.close()
            g.graph = None
            g.ctx.close()


def serve_alone(cfg: ServeConfig, r: Request, device="cuda"):
    """Run one request by itself (a batch of one) for cfg.steps steps and
    return its final particle state on the host."""
    srv = Server(cfg, device)
    r.bytes = request_bytes(r.case, r.prec)
    srv.admit(r)
    g = srv.groups[r.prec]
    for _ in range(cfg.steps):
        g.step(cfg, device)
    g.stream.synchronize()
    out = {k: r.parts[k].cpu() for k in ("Xr", "Ur", "Wr")}
    for gg in srv.groups.values():
        gg.ctx.status()
    srv.close()
    return out


def summarize(trace: list[Request], cfg: ServeConfig, wall: float):
    lat = np.array([r.latency for r in trace if r.latency is not None])
    mk = sum(r.case.M for r in trace) * cfg.Ns * cfg.steps
    return {
        "requests": len(trace),
        "completed": int(lat.size),
        "p50_ms": float(np.percentile(lat, 50) * 1e3) if lat.size else None,
        "p99_ms": float(np.percentile(lat, 99) * 1e3) if lat.size else None,
        "mean_ms": float(lat.mean() * 1e3) if lat.size else None,
        "wall_s": wall,
        "throughput_req_s": len(trace) / wall,
        "marker_updates_per_s": mk / wall,
    }
