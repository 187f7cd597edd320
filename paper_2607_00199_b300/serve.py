"""Continuous-batching serving loop for independent moving-mesh simulations.

Requests (2D periodic moving-mesh Taylor-Green vortex runs of different size K,
order N, motion and Reynolds number) arrive over time.  The loop keeps each
admitted request's fields, geometry and motion state on the device (one
GB_MIXED solver each), admits waiting requests first-come-first-served as
soon as the HBM budget has room, and on every tick advances all active
requests one SARK step: one gb_group_step per order N, i.e. one persistent
launch per stage over the tiles of every request of that order.  Requests
that arrive while others are running join at the next tick; finished ones
release their memory.  Per-step latency (tick time seen by each active
request), completion latency (arrival to last step) and the aggregate
DOF-stage rate are recorded.
"""
import time
from collections import deque

import numpy as np

from . import gb, inputs, state


def predicted_device_bytes(K, N):
    """Device memory of a GB_MIXED solver of K elements and order N (from the
    library's layout: 5 field arrays of ceil16(K) x S floats, mesh records,
    permutation, vertex arrays, operator tables, diagnostics scratch)."""
    Np = (N + 1) * (N + 2) // 2
    S = ((6 * Np - 4 + 7) // 8) * 8 + 4
    Kpad = (K + 15) // 16 * 16
    nv = K // 2
    return 5 * Kpad * S * 4 + 2 * 32 * K + 4 * K + 3 * 16 * nv + 16 + 4 + (1 << 17) + 8 * (Np + 5 + 5 * 1184)


class Admission:
    """First-come-first-served admission against a device-memory budget (host logic only)."""

    def __init__(self, budget_bytes, max_active=1 << 30):
        self.budget = int(budget_bytes)
        self.max_active = int(max_active)
        self.used = 0
        self.active = 0
        self.waiting = deque()
        self.peak = 0

    def arrive(self, req, nbytes):
        if nbytes > self.budget:
            raise ValueError('request %s needs %d bytes, more than the whole budget' % (req.get('id'), nbytes))
        self.waiting.append((req, int(nbytes)))

    def admit(self):
        """Pop and return the waiting requests that fit now, in arrival order."""
        out = []
        while self.waiting and self.active < self.max_active and self.used + self.waiting[0][1] <= self.budget:
            req, nb = self.waiting.popleft()
            self.used += nb
            self.active += 1
            self.peak = max(self.peak, self.used)
            out.append((req, nb))
        return out

    def release(self, nbytes):
        self.used -= int(nbytes)
        self.active -= 1


class Request:
    def __init__(self, spec, stream, jitter=0.0, cfl=0.5, precision=gb.GB_MIXED):
        self.spec = spec
        n, N = spec['n'], spec['N']
        self.mesh = inputs.periodic_square_mesh(n, jitter=jitter)
        self.solver = gb.Solver(self.mesh, N, spec['Ma'], spec['Re'], precision=precision, stream=stream)
        self.solver.set_motion(spec['A'], spec['T'])
        xy = self.solver.nodes()
        rho, u, v = inputs.taylor_green(xy[..., 0], xy[..., 1], spec['Ma'])
        self.q0 = state.equilibrium_fields(rho, u, v, self.solver.c)
        self.solver.set_fields(self.q0, 0.0)
        self.dt = inputs.cfl_dt(self.mesh, N, self.solver.c, cfl)
        self.steps_done = 0
        self.dof = self.solver.K * self.solver.Np * 6


class Server:
    """Runs a request stream to completion; see the module docstring.

    Set-up of an admitted request (mesh, initial state, device upload) runs on
    worker threads and a separate CUDA stream, overlapping the ticks of the
    requests already running; a request joins the batch at the first tick after
    its set-up has finished."""

    def __init__(self, budget_bytes, stream, steps_per_request=500, max_active=1024, capacity=1024,
                 time_scale=1.0, keep_fields=False, setup_stream=None, workers=2):
        self.adm = Admission(budget_bytes, max_active)
        self.stream = stream
        self.setup_stream = setup_stream
        self.workers = int(workers)
        self.steps = int(steps_per_request)
        self.capacity = int(capacity)
        self.groups = {}
        self.time_scale = float(time_scale)     # arrival times are divided by this (1 = real time)
        self.keep_fields = keep_fields
        self.results = {}
        # the CUDA device current where the server is built: the worker threads that create the
        # requests' solvers make it current too (a thread's current device defaults to 0)
        import torch
        self.device = torch.cuda.current_device() if torch.cuda.is_available() else None

    def _group(self, N):
        if N not in self.groups:
            self.groups[N] = gb.Group(self.capacity, self.stream)
        return self.groups[N]

    def run(self, requests, sync=None):
        """requests: dicts with id, arrival (s), n, N, A, T, Re, Ma.  sync(): device
        synchronisation of the serving stream (e.g. a torch stream's synchronize)."""
        from concurrent.futures import ThreadPoolExecutor
        pending = sorted(requests, key=lambda r: r['arrival'])
        pi = 0
        setup_stream = self.setup_stream if self.setup_stream is not None else self.stream
        preparing = {}               # id -> (future, nbytes)
        active = {}                  # id -> (Request, nbytes)
        step_lat, done_lat = [], []
        total_dof_stages = 0
        ticks = 0
        def _bind():
            if self.device is not None:
                import torch
                torch.cuda.set_device(self.device)
        pool = ThreadPoolExecutor(max_workers=self.workers, initializer=_bind)
        t0 = time.perf_counter()
        try:
            while pi < len(pending) or self.adm.waiting or preparing or active:
                now = time.perf_counter() - t0
                while pi < len(pending) and pending[pi]['arrival'] / self.time_scale <= now:
                    spec = pending[pi]
                    self.adm.arrive(spec, predicted_device_bytes(2 * spec['n'] ** 2, spec['N']))
                    pi += 1
                for spec, nb in self.adm.admit():
                    preparing[spec['id']] = (pool.submit(Request, spec, setup_stream), nb)
                for rid in [r for r, (fut, nb) in preparing.items() if fut.done()]:
                    fut, nb = preparing.pop(rid)
                    rq = fut.result()
                    if setup_stream != self.stream:
                        rq.solver.set_stream(self.stream)
                    active[rid] = (rq, nb)
                if not active:
                    time.sleep(0.0005)
                    continue
                tick0 = time.perf_counter()
                byN = {}
                for rid, (rq, nb) in active.items():
                    byN.setdefault(rq.spec['N'], []).append(rq)
                for N, lst in byN.items():
                    self._group(N).step([r.solver for r in lst], [r.dt for r in lst], 1)
                if sync is not None:
                    sync()
                tick = time.perf_counter() - tick0
                ticks += 1
                finished = []
                for rid, (rq, nb) in active.items():
                    rq.steps_done += 1
                    step_lat.append(tick)
                    total_dof_stages += rq.dof * 4
                    if rq.steps_done >= self.steps:
                        finished.append(rid)
                for rid in finished:
                    rq, nb = active.pop(rid)
                    q, t = rq.solver.fields()          # synchronises; raises on a device status flag
                    done_lat.append(time.perf_counter() - t0 - rq.spec['arrival'] / self.time_scale)
                    if self.keep_fields:
                        self.results[rid] = q
                    rq.solver.close()
                    self.adm.release(nb)
        finally:
            pool.shutdown(wait=True)
            for g in self.groups.values():
                g.close()
            self.groups = {}
        wall = time.perf_counter() - t0
        pct = lambda a, p: float(np.percentile(np.asarray(a), p)) if a else None
        return {'requests': len(requests), 'ticks': ticks, 'wall_s': wall,
                'dof_stage_per_s': total_dof_stages / wall if wall > 0 else None,
                'step_latency_ms': {'p50': pct(step_lat, 50) * 1e3, 'p99': pct(step_lat, 99) * 1e3},
                'completion_latency_s': {'p50': pct(done_lat, 50), 'p99': pct(done_lat, 99)},
                'peak_device_bytes': self.adm.peak, 'budget_bytes': self.adm.budget}
