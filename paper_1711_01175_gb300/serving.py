"""Serving loop: continuous batching of independent wave solves on one GPU.

Requests arrive over time (each its own mesh, degree, medium, point force and
step count).  The server admits a waiting request as soon as it fits the
memory budget and the occupancy bound, keeps every admitted solve's fields on
the device, and advances all admitted solves of one degree together through a
`dgw_batch` (one batched stage launch per stage over the elements of every
solve, replayed from a CUDA graph of two LSRK steps recorded once per batch).
Solves of different degrees run in separate batches on separate streams, so
their work overlaps on the device.  A composition change rewrites the graph's
descriptors for later replays while earlier ticks still run.  Latency is
arrival -> result on the host.

`one_at_a_time` is the reference policy: requests are served strictly in
arrival order, each alone with dgw_step.
"""
from __future__ import annotations

import ctypes
import time
from collections import deque

import numpy as np

from . import capi
from .solver import Solver, reference_nodes


def bytes_per_request(E, N, precision):
    """Device memory a solve holds: three FP64 state-sized buffers (u, the
    context's second buffer, res), the metric terms in the path's precision,
    mass weights and the neighbour map."""
    nel = E ** 3
    Np = (N + 1) ** 3
    real = 8 if precision == "fp64" else 4
    per_node = 3 * 9 * 8 + 10 * real + 8 + 6 * (N + 1) ** 2 * 4 / Np
    return int(nel * Np * per_node + nel * 200)


class _Solve:
    def __init__(self, req, precision, stream):
        import torch
        r, _ = reference_nodes(req.N)
        d = req.payload if req.payload else req.build(r)
        m = d["mesh"]
        self.req = req
        self.solver = Solver(req.N, tau=1, precision=precision)
        self.solver.upload_mesh(d["x"], m.etoe, m.etof, m.orient, m.bc)
        self.solver.upload_material(d["rho"], d["lam"], d["mu"])
        self.solver.set_point_force(**d["source"])
        self.dt = self.solver.dt_cfl()
        with torch.cuda.stream(stream):
            self.u = torch.zeros((9, m.nel, (req.N + 1) ** 3), dtype=torch.float64, device="cuda")
            self.res = torch.zeros_like(self.u)
        self.steps_done = 0         # steps enqueued so far
        self.bytes = bytes_per_request(req.E, req.N, precision)

    def close(self):
        self.solver.close()
        self.u = self.res = None


class _Group:
    """The batch of one degree, its stream and its ticks in flight."""

    def __init__(self, N, precision, max_solves=capi.DGW_BATCH_MAX_SOLVES):
        import torch
        self.N = N
        self.stream = torch.cuda.Stream()
        st, self.h = capi.dgw_batch_create(torch.cuda.current_device(), N, 0 if precision == "fp64" else 1, 1,
                                           max_solves)
        if st != 0:
            raise capi.DGWError(st, capi.dgw_last_error(None))
        self.capacity = max_solves
        self.solves = []            # the batch's composition for the next tick
        self.dirty = False
        self.inflight = deque()     # (sequence number, event, solves that end with this tick)

    def reset(self):
        n = len(self.solves)
        P = ctypes.c_void_p * max(n, 1)
        D = ctypes.c_double * max(n, 1)
        st = capi.dgw_batch_set(self.h, n, P(*[s.solver._ctx.value for s in self.solves]),
                                P(*[s.u.data_ptr() for s in self.solves]),
                                P(*[s.res.data_ptr() for s in self.solves]),
                                D(*[s.dt for s in self.solves]),
                                D(*[s.steps_done * s.dt for s in self.solves]),
                                ctypes.c_void_p(self.stream.cuda_stream))
        if st != 0:
            raise capi.DGWError(st, capi.dgw_batch_last_error(self.h))
        self.dirty = False

    def close(self):
        capi.dgw_batch_destroy(self.h)


def _finish(solve, t0):
    """Result on the host: the final state's energy and the state itself."""
    u = solve.u.cpu().numpy()
    e = solve.solver.energy(solve.u)
    return dict(rid=solve.req.rid, energy=e, state=u, done=time.perf_counter() - t0)


def _nodes(req):
    return req.E ** 3 * (req.N + 1) ** 3


def continuous_batching(requests, precision="mixed", memory_budget=40e9, pairs_per_tick=4, keep_states=False,
                        max_active_nodes=None, ticks_in_flight=2):
    """Serve `requests` (sorted by arrival) with continuous batching.

    The loop keeps up to `ticks_in_flight` ticks enqueued per batch, so the
    device never waits for the host: a tick is up to `pairs_per_tick` step
    pairs of the batch's current composition.  The host knows in advance how
    many steps each solve has been given, so a solve whose last step is in a
    tick leaves the composition of the next one before that tick has run; its
    result is read (on a separate stream) once its tick's event has
    completed.  Between ticks the loop admits arrived requests (their set-up
    overlaps the device work; they join at their batch's next tick).

    Admission is FIFO and bounded three times: by a batch's capacity
    (DGW_BATCH_MAX_SOLVES solves of one degree), by the memory budget, and by
    `max_active_nodes` (default: two waves of resident threads on the device)
    so that batching fills the GPU with small solves without turning the
    queue into processor sharing, which on a saturated device finishes every
    request later than first-come first-served.

    Finished solves release their device memory when no tick is in flight
    (freeing device memory waits for the whole device) or when admission is
    short of memory."""
    import torch
    if max_active_nodes is None:
        props = torch.cuda.get_device_properties(torch.cuda.current_device())
        max_active_nodes = 2 * props.multi_processor_count * props.max_threads_per_multi_processor
    for r in requests:
        if bytes_per_request(r.E, r.N, precision) > memory_budget:
            raise ValueError(f"request {r.rid} needs more device memory than the budget")
    pending = deque(sorted(requests, key=lambda r: r.arrival))
    waiting = deque()
    groups = {}
    used = 0                # bytes of admitted solves, including retired ones not yet released
    active_nodes = 0        # nodes of solves not yet retired
    retired = []
    results = {}
    readout = torch.cuda.Stream()
    seq = 0
    t0 = time.perf_counter()

    def release():
        nonlocal used
        for s in retired:
            used -= s.bytes
            s.close()
        retired.clear()

    def admit():
        nonlocal used, active_nodes
        now = time.perf_counter() - t0
        while pending and pending[0].arrival <= now:
            waiting.append(pending.popleft())
        while waiting:
            req = waiting[0]
            need = bytes_per_request(req.E, req.N, precision)
            if used + need > memory_budget:
                if not retired:
                    break
                release()
                continue
            if active_nodes > 0 and active_nodes + _nodes(req) > max_active_nodes:
                break
            g = groups.get(req.N)
            if g is not None and len(g.solves) >= g.capacity:
                break
            waiting.popleft()
            if g is None:
                g = groups[req.N] = _Group(req.N, precision)
            s = _Solve(req, precision, g.stream)
            used += s.bytes
            active_nodes += _nodes(req)
            g.solves.append(s)
            g.dirty = True

    while pending or waiting or any(g.solves or g.inflight for g in groups.values()):
        admit()
        for g in groups.values():
            while g.solves and len(g.inflight) < ticks_in_flight:
                if g.dirty:
                    g.reset()
                k = min(pairs_per_tick, min((s.req.steps - s.steps_done) // 2 for s in g.solves))
                st = capi.dgw_batch_run(g.h, k, ctypes.c_void_p(g.stream.cuda_stream))
                if st != 0:
                    raise capi.DGWError(st, capi.dgw_batch_last_error(g.h))
                for s in g.solves:
                    s.steps_done += 2 * k
                ending = [s for s in g.solves if s.steps_done >= s.req.steps]
                if ending:
                    g.solves = [s for s in g.solves if s.steps_done < s.req.steps]
                    g.dirty = True
                ev = torch.cuda.Event()
                ev.record(g.stream)
                g.inflight.append((seq, ev, ending))
                seq += 1
        busy = [g for g in groups.values() if g.inflight]
        if not busy:
            release()
            if pending and not waiting:
                time.sleep(max(0.0, pending[0].arrival - (time.perf_counter() - t0)))
            continue
        g = min(busy, key=lambda gg: gg.inflight[0][0])
        _, ev, ending = g.inflight.popleft()
        ev.synchronize()
        if ending:
            with torch.cuda.stream(readout):
                for s in ending:
                    r = _finish(s, t0)
                    r["latency"] = r["done"] - s.req.arrival
                    if not keep_states:
                        r.pop("state")
                    results[s.req.rid] = r
                    active_nodes -= _nodes(s.req)
                    retired.append(s)
    release()
    for g in groups.values():
        g.close()
    return results, time.perf_counter() - t0


def one_at_a_time(requests, precision="mixed", keep_states=False):
    """Serve `requests` strictly in arrival order, one solve at a time (dgw_step)."""
    import torch
    stream = torch.cuda.Stream()
    results = {}
    t0 = time.perf_counter()
    for req in sorted(requests, key=lambda r: r.arrival):
        wait = req.arrival - (time.perf_counter() - t0)
        if wait > 0:
            time.sleep(wait)
        s = _Solve(req, precision, stream)
        with torch.cuda.stream(stream):
            s.solver.step(s.u, s.res, s.dt, req.steps, t0=0.0, stream=stream)
        stream.synchronize()
        s.steps_done = req.steps
        r = _finish(s, t0)
        r["latency"] = r["done"] - req.arrival
        if not keep_states:
            r.pop("state")
        results[req.rid] = r
        s.close()
    return results, time.perf_counter() - t0


def summarize(results, wall):
    lat = np.array([r["latency"] for r in results.values()]) * 1e3
    return {"requests": len(results), "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
            "mean_ms": float(lat.mean()), "solves_per_s": len(results) / wall, "wall_s": wall}
