"""Request loop for channel-flow solves on one GPU (continuous batching).

Requests arrive over time (e.g. a Poisson process); each is a channel solve to be run
until the residual of W falls below a tolerance or a step cap is hit.  The loop keeps
every admitted request's state on the device in a batch slot, admits waiting requests in
arrival order as soon as a slot and enough of the HBM budget are free, advances all
admitted requests together (one batch step = one graph replay of all of them), checks
residuals every `check_every` steps, and retires finished requests, freeing their slot
and memory for the next arrivals.  Per request it records arrival, admission and
completion times (wall clock from the start of the run), steps and final residual, from
which time-to-steady-state percentiles and aggregate throughput follow.

All numerical work runs in the CUDA library (ugks_batch_*); this module only schedules.
"""
from __future__ import annotations

import dataclasses
import time
from collections import deque
from dataclasses import dataclass, field

import numpy as np


@dataclass
class Request:
    rid: int
    arrival: float          # seconds after the start of the run
    cfg: object             # inputs.Config
    prim: tuple             # initial (rho, U, V, T) per cell
    admitted: float = None
    finished: float = None
    steps: int = 0
    residual: float = None
    converged: bool = False
    slot: int = None
    state: tuple = None     # final (f, W) when keep_state is set


@dataclass
class ServeStats:
    requests: list = field(default_factory=list)
    wall: float = 0.0
    batch_steps: int = 0
    vc_updates: float = 0.0
    peak_bytes: int = 0
    peak_active: int = 0

    def tts(self):
        """time to steady state (finish - arrival) of finished requests, seconds"""
        return np.array([r.finished - r.arrival for r in self.requests if r.finished is not None])

    def summary(self) -> dict:
        t = self.tts()
        done = [r for r in self.requests if r.finished is not None]
        return {
            "requests": len(self.requests),
            "finished": len(done),
            "converged": sum(r.converged for r in done),
            "p50_s": float(np.percentile(t, 50)) if len(t) else None,
            "p99_s": float(np.percentile(t, 99)) if len(t) else None,
            "mean_s": float(t.mean()) if len(t) else None,
            "wall_s": self.wall,
            "batch_steps": self.batch_steps,
            "vc_per_s": self.vc_updates / self.wall if self.wall > 0 else 0.0,
            "peak_bytes": self.peak_bytes,
            "peak_active": self.peak_active,
        }


class Server:
    """Continuous-batching loop over a batch engine.

    batch: an object with admit(cfg) -> slot, retire(slot), instance(slot) (with
    init_maxwellian, residual, get_state), step(n), sync(), bytes_used; `state_bytes(cfg)`
    gives the device bytes a request needs.  Both are injectable so the scheduling can be
    tested without a GPU.
    """

    def __init__(self, batch, state_bytes, hbm_budget: int, max_slots: int, tol: float = 1e-6,
                 max_steps: int = 20000, check_every: int = 20, clock=time.perf_counter,
                 sleep=time.sleep, keep_state: bool = False):
        self.batch = batch
        self.state_bytes = state_bytes
        self.budget = int(hbm_budget)
        self.max_slots = int(max_slots)
        self.tol = float(tol)
        self.max_steps = int(max_steps)
        self.check_every = int(check_every)
        self.clock = clock
        self.sleep = sleep
        self.keep_state = keep_state

    def run(self, requests) -> ServeStats:
        reqs = sorted(requests, key=lambda r: (r.arrival, r.rid))
        pending = deque(reqs)     # not yet arrived
        waiting = deque()         # arrived, not admitted (FIFO)
        active = {}               # slot -> Request
        used = 0
        st = ServeStats(requests=reqs)
        t0 = self.clock()
        now = lambda: self.clock() - t0
        while pending or waiting or active:
            t = now()
            while pending and pending[0].arrival <= t:
                waiting.append(pending.popleft())
            # admission in arrival order: the head waits until it fits (no overtaking)
            while waiting and len(active) < self.max_slots:
                r = waiting[0]
                need = self.state_bytes(r.cfg)
                if self.budget and used + need > self.budget:
                    if not active:
                        raise RuntimeError(f"request {r.rid} needs {need} B, over the budget")
                    break
                waiting.popleft()
                r.slot = self.batch.admit(r.cfg)
                self.batch.instance(r.slot).init_maxwellian(*r.prim)
                r.admitted = now()
                active[r.slot] = r
                used += need
            st.peak_bytes = max(st.peak_bytes, used)
            st.peak_active = max(st.peak_active, len(active))
            if not active:
                if pending:
                    self.sleep(max(0.0, pending[0].arrival - now()))
                continue
            # steps to the next residual check, limited by the closest step cap
            n = min(self.check_every, min(self.max_steps - r.steps for r in active.values()))
            self.batch.step(n)
            st.batch_steps += n
            for r in active.values():
                r.steps += n
                st.vc_updates += n * r.cfg.nx * r.cfg.ny * r.cfg.nu * r.cfg.nv
            self.batch.sync()
            done = []
            for slot, r in active.items():
                res = float(np.max(self.batch.instance(slot).residual()))
                r.residual = res
                if res < self.tol or r.steps >= self.max_steps:
                    r.converged = res < self.tol
                    done.append(slot)
            for slot in done:
                r = active.pop(slot)
                if self.keep_state:
                    r.state = self.batch.instance(slot).get_state()
                self.batch.retire(slot)
                used -= self.state_bytes(r.cfg)
                r.finished = now()
        st.wall = now()
        return st


def make_requests(cfgs, arrivals, prims):
    return [Request(rid=k, arrival=float(a), cfg=c, prim=p)
            for k, (c, a, p) in enumerate(zip(cfgs, arrivals, prims))]


class ModeSwitchingBatch:
    """A batch engine whose step mode follows the work in flight: one persistent launch per
    step (six grid barriers) when the active instances hold at least `persistent_min_vc`
    velocity-cells, else seven phase launches, whose fixed cost is lower for small batches.
    The mode does not change results (the same phase code runs either way)."""

    def __init__(self, batch, persistent_min_vc: int):
        self._b = batch
        self._min = int(persistent_min_vc)
        self._vc = {}

    def __getattr__(self, name):
        return getattr(self._b, name)

    def admit(self, cfg):
        slot = self._b.admit(cfg)
        self._vc[slot] = cfg.nx * cfg.ny * cfg.nu * cfg.nv
        return slot

    def retire(self, slot):
        self._b.retire(slot)
        self._vc.pop(slot, None)

    def step(self, n: int = 1):
        want = sum(self._vc.values()) >= self._min
        if want != self._b.persistent:
            self._b.set_persistent(want)
        self._b.step(n)


def gpu_server(hbm_budget: int, max_slots: int, stream=None, persistent_min_vc: int = 200_000_000,
               **kw) -> Server:
    """A Server over the CUDA batch engine."""
    from . import ugks
    batch = ugks.Batch(max_slots, hbm_budget, stream=stream)
    engine = ModeSwitchingBatch(batch, persistent_min_vc) if batch.persistent else batch
    srv = Server(engine, lambda c: ugks.state_bytes(c, ugks.FP32F), hbm_budget, max_slots, **kw)
    srv.batch_handle = batch
    return srv


def replace(cfg, **kw):
    return dataclasses.replace(cfg, **kw)
