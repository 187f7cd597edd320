"""Continuous-batching serving loop for independent moving-mesh simulations.

Requests (2D periodic moving-mesh Taylor-Green vortex runs of different size K,
order N, motion and Reynolds number) arrive over time.  The loop keeps each
admitted request's fields, geometry and motion state on the device (one
GB_MIXED solver each), admits waiting requests first-come-first-served as soon
as the device-memory budget has room (by default a fraction of the free device
memory), and steps them in units that run at their own cadence on their own
CUDA streams, so that their work overlaps on the device:

  * small requests (K below `large_k`) are batched in a group per (N, size class
    of K): one launch per stage over the tiles of every member (gb_group_step);
  * a large request, which fills the GPU by itself, is a unit of its own, stepped
    with gb_step on the launch shape its tuner picks (the tcgen05 kernel for N <= 4);
    at most `large_streams` of them run at a time, first come first served, on
    low-priority streams, while the groups of small requests use high-priority
    streams, so that short requests are not held behind long ones.

Whenever a unit's previous launch has completed (polled with CUDA events), its
finished members leave (their memory is released) and its next launch of a few
steps is enqueued; requests whose set-up (worker threads, a side stream) has
finished join their unit before its next launch.  Recorded: per-step device time
of each unit (seen by each member), completion latency (arrival to last step),
and, given each request's time alone, its slowdown (completion latency over the
time alone); the aggregate DOF-stage rate is all updates over the wall time.
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


_MESHES = {}


def _mesh(n, jitter):
    # the seeded meshes depend only on (n, jitter): generated once per process, shared read-only
    key = (int(n), float(jitter))
    if key not in _MESHES:
        _MESHES[key] = inputs.periodic_square_mesh(n, jitter=jitter)
    return _MESHES[key]


class Request:
    def __init__(self, spec, stream, jitter=0.0, cfl=0.5, precision=gb.GB_MIXED):
        self.spec = spec
        n, N = spec['n'], spec['N']
        self.mesh = _mesh(n, jitter)
        self.solver = gb.Solver(self.mesh, N, spec['Ma'], spec['Re'], precision=precision, stream=stream)
        self.solver.set_motion(spec['A'], spec['T'])
        xy = self.solver.nodes()
        rho, u, v = inputs.taylor_green(xy[..., 0], xy[..., 1], spec['Ma'])
        self.q0 = state.equilibrium_fields(rho, u, v, self.solver.c)
        self.solver.set_fields(self.q0, 0.0)
        self.dt = inputs.cfl_dt(self.mesh, N, self.solver.c, cfl)
        self.steps_done = 0
        self.dof = self.solver.K * self.solver.Np * 6


def size_class(K):
    """Bit length of K - 1: meshes of (2^(c-1), 2^c] elements share a class."""
    return int(K - 1).bit_length()


class _Unit:
    """A group of small requests of one (N, size class), or one large request, with its
    own CUDA stream; at most one launch of a few steps in flight."""

    def __init__(self, stream, group=None):
        self.stream = stream          # torch.cuda.Stream
        self.group = group            # gb.Group or None (a single large request)
        self.members = []
        self.inflight = None          # (start event, end event, steps, members)


class Server:
    """Runs a request stream to completion; see the module docstring.

    budget_bytes None: `budget_fraction` of the device memory free when the server is
    built.  alone_ms: optional {(K, N): ms per step of a request running alone}, for the
    slowdown statistics."""

    def __init__(self, budget_bytes=None, stream=None, steps_per_request=500, max_active=1024, capacity=1024,
                 time_scale=1.0, keep_fields=False, setup_stream=None, workers=None, large_k=32768,
                 group_steps=4, large_steps=8, budget_fraction=0.8, large_streams=4, alone_ms=None):
        import torch
        self.torch = torch
        # the CUDA device current where the server is built: the worker threads that create the
        # requests' solvers make it current too (a thread's current device defaults to 0)
        self.device = torch.cuda.current_device() if torch.cuda.is_available() else None
        if budget_bytes is None:
            free, _ = torch.cuda.mem_get_info()
            budget_bytes = int(budget_fraction * free)
        self.adm = Admission(budget_bytes, max_active)
        self.stream = stream
        self.setup_stream = setup_stream
        import os
        self.workers = int(workers) if workers else max(2, min(8, (os.cpu_count() or 2) // 2))
        self.steps = int(steps_per_request)
        self.capacity = int(capacity)
        self.large_k = int(large_k)
        self.group_steps, self.large_steps = int(group_steps), int(large_steps)
        self.time_scale = float(time_scale)     # arrival times are divided by this (1 = real time)
        self.keep_fields = keep_fields
        self.alone_ms = alone_ms or {}
        self.results = {}
        self.units = {}
        # large requests: at most `large_streams` in flight (first come, first served), each on
        # one of these low-priority streams; groups of small requests get high-priority streams
        lo, hi = torch.cuda.Stream.priority_range() if hasattr(torch.cuda.Stream, 'priority_range') else (0, -1)
        self._prio_small = hi
        self._large_pool = [torch.cuda.Stream(priority=lo) for _ in range(max(1, int(large_streams)))]
        self._large_busy = [False] * len(self._large_pool)
        self._large_wait = []          # large requests waiting for a stream

    def _place(self, rq):
        """Put a set-up request into its unit (or the queue of large requests)."""
        K, N = rq.solver.K, rq.spec['N']
        if K >= self.large_k:
            self._large_wait.append(rq)
            self._start_large()
            return
        key = ('group', N, size_class(K))
        if key not in self.units:
            st = self.torch.cuda.Stream(priority=self._prio_small)
            self.units[key] = _Unit(st, gb.Group(self.capacity, st.cuda_stream))
        u = self.units[key]
        rq.solver.set_stream(u.stream.cuda_stream)
        u.members.append(rq)

    def _start_large(self):
        while self._large_wait and not all(self._large_busy):
            i = self._large_busy.index(False)
            rq = self._large_wait.pop(0)
            u = _Unit(self._large_pool[i])
            u.slot = i
            self._large_busy[i] = True
            rq.solver.set_stream(u.stream.cuda_stream)
            u.members.append(rq)
            self.units[('large', rq.spec['id'])] = u

    def _launch(self, u):
        steps = min(r.steps_left for r in u.members)
        steps = min(steps, self.group_steps if u.group is not None else self.large_steps)
        torch = self.torch
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(u.stream)
        if u.group is not None:
            u.group.step([r.solver for r in u.members], [r.dt for r in u.members], steps)
        else:
            r = u.members[0]
            r.solver.step(r.dt, steps)
        e1.record(u.stream)
        u.inflight = (e0, e1, steps, list(u.members))

    def run(self, requests, sync=None):
        """requests: dicts with id, arrival (s), n, N, A, T, Re, Ma."""
        from concurrent.futures import ThreadPoolExecutor
        pending = sorted(requests, key=lambda r: r['arrival'])
        pi = 0
        setup_stream = self.setup_stream if self.setup_stream is not None else self.stream
        preparing = {}               # id -> (future, nbytes)
        nbytes_of = {}
        step_lat, done_lat, slowdown = [], [], []
        total_dof_stages = 0
        launches = 0

        def _bind():
            if self.device is not None:
                self.torch.cuda.set_device(self.device)
        pool = ThreadPoolExecutor(max_workers=self.workers, initializer=_bind)
        t0 = time.perf_counter()
        try:
            while (pi < len(pending) or self.adm.waiting or preparing or self._large_wait or
                   any(u.members for u in self.units.values())):
                progressed = False
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
                    rq.steps_left = self.steps
                    nbytes_of[rid] = nb
                    self._place(rq)
                    progressed = True
                for key, u in list(self.units.items()):
                    if u.inflight is not None and u.inflight[1].query():
                        e0, e1, steps, members = u.inflight
                        ms = e0.elapsed_time(e1) / steps
                        u.inflight = None
                        for rq in members:
                            rq.steps_left -= steps
                            step_lat.extend([ms] * steps)
                            total_dof_stages += rq.dof * 4 * steps
                            if rq.steps_left <= 0:
                                q, _ = rq.solver.fields()   # completed work; raises on a device status flag
                                lat = time.perf_counter() - t0 - rq.spec['arrival'] / self.time_scale
                                done_lat.append(lat)
                                alone = self.alone_ms.get((rq.solver.K, rq.spec['N']))
                                if alone:
                                    slowdown.append(lat / (alone * 1e-3 * self.steps))
                                if self.keep_fields:
                                    self.results[rq.spec['id']] = q
                                u.members.remove(rq)
                                rq.solver.close()
                                self.adm.release(nbytes_of.pop(rq.spec['id']))
                        progressed = True
                        if u.group is None and not u.members:
                            del self.units[key]
                            self._large_busy[u.slot] = False
                            self._start_large()
                            continue
                    if u.inflight is None and u.members:
                        self._launch(u)
                        launches += 1
                        progressed = True
                if not progressed:
                    time.sleep(0.0002)
        finally:
            pool.shutdown(wait=True)
            for u in self.units.values():
                u.stream.synchronize()
                if u.group is not None:
                    u.group.close()
            self.units = {}
        wall = time.perf_counter() - t0
        pct = lambda a, p: float(np.percentile(np.asarray(a), p)) if a else None
        out = {'requests': len(requests), 'launches': launches, 'wall_s': wall,
               'dof_stage_per_s': total_dof_stages / wall if wall > 0 else None,
               'step_latency_ms': {'p50': pct(step_lat, 50), 'p99': pct(step_lat, 99)},
               'completion_latency_s': {'p50': pct(done_lat, 50), 'p99': pct(done_lat, 99)},
               'peak_device_bytes': self.adm.peak, 'budget_bytes': self.adm.budget}
        if slowdown:
            out['slowdown_vs_alone'] = {'p50': pct(slowdown, 50), 'p99': pct(slowdown, 99),
                                        'mean': float(np.mean(slowdown))}
        return out
