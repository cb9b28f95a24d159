"""Serving loop on the batch API (continuous batching).

Requests -- a rotating square patch (Section 5.1.1) or an Evrard sphere
(Section 5.1.2, hydrodynamics only) of some size, to be advanced some number
of steps -- arrive over time. A request is admitted as soon as the batch has
a free instance slot and its particles fit in the device arena (a fixed
budget of device memory, allocated once); its state then stays resident on
the device until it has taken all its steps. All admitted requests advance
together: each tick runs sph_batch_step over every resident instance for up
to `quantum` steps, then retires the finished ones (their results are copied
to the host and their arena range freed) and admits waiting requests, so new
work joins while older work is still running. Arrivals are served in order
(a request that does not fit waits, and so do the ones behind it). With
`tick_s` set, a tick takes as many steps as fit in about tick_s seconds at
the throughput measured so far (at least one, at most `quantum`), so a
request that arrives during a tick waits about tick_s, whatever the number
of resident particles.

Latency of a request = done - arrival, split into three parts:
  tick wait = first admission chance - arrival (the tick running when it
              arrived had to end first),
  queueing  = admitted - first admission chance (no free slot or memory, or
              an earlier request still waiting),
  run       = done - admitted (resident, sharing the device with the others).

A request's result is the same, bit for bit, as stepping it alone with
sph_step: instances of a batch never interact, and a run split over several
calls gives the same bits as one call.

Host-side scheduling only: every step runs in libsph.
"""
from __future__ import annotations

import dataclasses
import math
import time
from collections import deque

import numpy as np

from . import ics

OUT_FIELDS = ("x", "y", "z", "vx", "vy", "vz", "h", "u", "rho", "p", "c", "ax", "ay", "az", "du")


@dataclasses.dataclass
class Request:
    rid: int
    arrival: float          # seconds after the start of the stream (or ticks, virtual clock)
    kind: str               # "patch" or "evrard"
    n: int                  # particles (a patch rounds to a cube)
    steps: int
    seed: int
    omega: float = 5.0
    chance: float = math.nan   # first admission attempt at or after arrival
    admitted: float = math.nan
    done: float = math.nan
    result: dict | None = None


def make_stream(count: int, rate: float, seed: int, n_min: int = 8000, n_max: int = 1_000_000,
                steps: tuple = (10, 100), evrard_share: float = 0.5) -> list:
    """Poisson arrivals at `rate` per second; N log-uniform in [n_min, n_max]
    (a patch takes the nearest cube), steps uniform in [steps[0], steps[1]],
    a patch with omega ~ U[2, 8] or an Evrard sphere."""
    rng = np.random.Generator(np.random.PCG64(seed))
    t = np.cumsum(rng.exponential(1.0 / rate, size=count))
    out = []
    for k in range(count):
        n = int(round(math.exp(rng.uniform(math.log(n_min), math.log(n_max)))))
        kind = "evrard" if rng.uniform() < evrard_share else "patch"
        if kind == "patch":
            side = max(2, int(round(n ** (1.0 / 3.0))))
            n = side ** 3
        st = int(rng.integers(steps[0], steps[1] + 1))
        out.append(Request(k, float(t[k]), kind, n, st, seed * 100003 + k,
                           float(rng.uniform(2.0, 8.0))))
    return out


def initial_state(req: Request, precision: int = 0, **knobs):
    if req.kind == "patch":
        s, p = ics.square_patch(round(req.n ** (1.0 / 3.0)), seed=req.seed, omega=req.omega)
    else:
        s, p = ics.evrard(req.n, seed=req.seed)
    p.precision = precision
    for k, v in knobs.items():
        setattr(p, k, v)
    return s, p


class Arena:
    """First-fit allocator of particle ranges in [0, capacity)."""

    def __init__(self, capacity: int):
        self.free = [(0, capacity)]  # sorted, coalesced (start, length)

    def take(self, n: int):
        for q, (a, ln) in enumerate(self.free):
            if ln >= n:
                if ln == n:
                    self.free.pop(q)
                else:
                    self.free[q] = (a + n, ln - n)
                return a
        return None

    def fits(self, n: int) -> bool:
        return any(ln >= n for _, ln in self.free)

    def give(self, a: int, n: int):
        self.free.append((a, n))
        self.free.sort()
        merged = []
        for s, ln in self.free:
            if merged and merged[-1][0] + merged[-1][1] == s:
                merged[-1] = (merged[-1][0], merged[-1][1] + ln)
            else:
                merged.append((s, ln))
        self.free = merged


@dataclasses.dataclass
class _Resident:
    req: Request
    first: int
    params: object
    left: int
    time: object  # device tensor (1,)


class Server:
    """Resident state of up to max_instances requests in one arena of
    `capacity` particles; one batch context steps them together."""

    def __init__(self, capacity: int, max_instances: int = 256, quantum: int = 10,
                 device: int = 0, stream=None, nnz_per_particle: int = 160,
                 result_fields: tuple = OUT_FIELDS + ("nnb",), keep_result=None,
                 tick_s: float | None = None):
        import torch

        from . import binding
        self.B = binding
        self.torch = torch
        self.dev = torch.device("cuda", device)
        self.stream = stream
        self.capacity = int(capacity)
        self.max_instances = int(max_instances)
        self.quantum = int(quantum)
        self.tick_s = tick_s
        self.rate = None  # particle-steps per second of the ticks so far
        self.result_fields = tuple(result_fields)
        self.keep_result = keep_result  # None: keep every result on the host
        self.ctx = binding.Context(capacity, nnz_capacity=nnz_per_particle * capacity,
                                   device=device, max_instances=max_instances)
        f64 = dict(dtype=torch.float64, device=self.dev)
        self.arr = {f: torch.zeros(capacity, **f64)
                    for f in binding.STATE_FIELDS + binding.OUT_FIELDS}
        self.arr["nnb"] = torch.zeros(capacity, dtype=torch.int32, device=self.dev)
        self.arena = Arena(capacity)
        self.active: list[_Resident] = []
        self.ticks = 0
        self.status = binding.SPH_OK

    @staticmethod
    def bytes_per_particle(max_instances: int = 256, nnz_per_particle: int = 160) -> float:
        """Device bytes per particle of capacity: context scratch plus arena."""
        from . import binding
        n = 1_000_000
        ctx = binding.ctx_bytes(n, nnz_per_particle * n, max_instances) / n
        arena = 8 * (len(binding.STATE_FIELDS) + len(binding.OUT_FIELDS)) + 4
        return ctx + arena

    def can_admit(self, n: int) -> bool:
        return len(self.active) < self.max_instances and self.arena.fits(n)

    def admit(self, req: Request, state: dict, params, now: float):
        torch = self.torch
        first = self.arena.take(req.n)
        assert first is not None
        self.ctx.lists_clear(first, req.n, stream=self.stream)  # as on a fresh context
        for f in self.B.STATE_FIELDS:
            self.arr[f][first:first + req.n].copy_(torch.from_numpy(np.ascontiguousarray(state[f])),
                                                   non_blocking=True)
        req.admitted = now
        self.active.append(_Resident(req, first, params, req.steps,
                                     torch.zeros(1, dtype=torch.float64, device=self.dev)))

    def tick(self) -> list:
        """Advance every resident request by min(quantum, fewest steps left);
        returns the requests that finished, with their results on the host."""
        torch = self.torch
        if not self.active:
            return []
        k = min(self.quantum, min(r.left for r in self.active))
        resident = sum(r.req.n for r in self.active)
        if self.tick_s is not None and self.rate is not None:
            k = max(1, min(k, int(self.tick_s * self.rate / resident)))
        t0 = time.perf_counter()
        self.ctx.batch_set([r.req.n for r in self.active], [r.params for r in self.active],
                           first=[r.first for r in self.active], stream=self.stream)
        arrays = dict(self.arr)
        arrays["dt"] = torch.zeros(len(self.active), dtype=torch.float64, device=self.dev)
        arrays["time"] = torch.cat([r.time for r in self.active])
        self.ctx.batch_step(arrays, nsteps=k, stream=self.stream)
        self.ticks += 1
        done, keep = [], []
        for i, r in enumerate(self.active):
            r.time = arrays["time"][i:i + 1]
            r.left -= k
            (done if r.left == 0 else keep).append(r)
        for r in done:  # results go to the host, then the range is free
            sl = slice(r.first, r.first + r.req.n)
            res = {f: self.arr[f][sl].cpu().numpy() for f in self.result_fields}
            res["time"] = float(r.time.item())
            if self.keep_result is None or self.keep_result(r.req):
                r.req.result = res
            self.arena.give(r.first, r.req.n)
        st = self.ctx.sync(self.stream)
        if st != self.B.SPH_OK:
            self.status = st
        r_now = resident * k / max(time.perf_counter() - t0, 1e-9)
        self.rate = r_now if self.rate is None else 0.5 * (self.rate + r_now)
        self.active = keep
        return [r.req for r in done]


def serve(server: Server, requests: list, states: dict, clock: str = "real") -> dict:
    """Run a request stream to completion. states[rid] = (state, params).
    clock "real": arrival times are seconds of wall time from the start;
    "virtual": one tick is one time unit (deterministic, for tests)."""
    pending = deque(sorted(requests, key=lambda r: (r.arrival, r.rid)))
    t0 = time.perf_counter()
    vt = 0.0

    def now():
        return time.perf_counter() - t0 if clock == "real" else vt

    finished = []
    while pending or server.active:
        t = now()
        for r in pending:  # admission chances come between ticks
            if r.arrival > t:
                break
            if math.isnan(r.chance):
                r.chance = t
        while pending and pending[0].arrival <= t and server.can_admit(pending[0].n):
            r = pending.popleft()
            server.admit(r, *states[r.rid], now=t)
        if not server.active:
            if pending and not server.can_admit(pending[0].n) and not server.active:
                raise RuntimeError(f"request {pending[0].rid} ({pending[0].n} particles) "
                                   f"exceeds the arena of {server.capacity}")
            if pending:
                if clock == "real":
                    time.sleep(max(0.0, pending[0].arrival - now()))
                else:
                    vt = max(vt, pending[0].arrival)
            continue
        out = server.tick()
        if clock == "virtual":
            vt += 1.0
        t = now()
        for r in out:
            r.done = t
        finished.extend(out)
    return summarize(finished)


def _pct(v) -> dict:
    return {"p50": float(np.percentile(v, 50)), "p99": float(np.percentile(v, 99))}


def summarize(reqs: list) -> dict:
    lat = np.array([r.done - r.arrival for r in reqs])
    upd = sum(r.n * r.steps for r in reqs)
    first = min(r.arrival for r in reqs)
    last_arrival = max(r.arrival for r in reqs)
    end = max(r.done for r in reqs)
    out = {"requests": len(reqs), "updates": upd,
           "latency_p50": float(np.percentile(lat, 50)), "latency_p99": float(np.percentile(lat, 99)),
           "makespan": end - first, "served_updates_per_s": upd / max(end - first, 1e-12),
           "offered_updates_per_s": upd / max(last_arrival - first, 1e-12)}
    if all(not math.isnan(r.chance) and not math.isnan(r.admitted) for r in reqs):
        out["split"] = {
            "tick_wait": _pct([r.chance - r.arrival for r in reqs]),
            "queueing": _pct([r.admitted - r.chance for r in reqs]),
            "run": _pct([r.done - r.admitted for r in reqs])}
    return out


def fifo_single(requests: list, run_time: dict) -> dict:
    """One request at a time through the single-instance path, in arrival
    order: run_time[rid] is its measured time alone; request k starts when it
    has arrived and request k - 1 is done."""
    end = 0.0
    for r in sorted(requests, key=lambda r: (r.arrival, r.rid)):
        start = max(r.arrival, end)
        r.chance = r.arrival  # nothing runs in ticks here: no tick wait
        r.admitted = start
        end = start + run_time[r.rid]
        r.done = end
    return summarize(requests)
