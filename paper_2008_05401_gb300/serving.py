"""Continuous-batching request loop over the C ABI (host-side scheduling only).

A request asks for S proposals of n chains of one model at lattice side L.  The
server keeps every admitted job's chain state resident in device memory and,
at each scheduling step:

  1. admits waiting requests in arrival order while the context's HBM budget
     accepts their job memory (``crbm_init_chains`` returns CRBM_ENOMEM when it
     does not; the request then waits for memory to be released);
  2. groups the active jobs that can share a launch (same model kind,
     filter-bank shape and precision), at most 16 per launch; every group has
     two CUDA streams and keeps up to two batches in flight, one per stream:
     whenever a stream of the group is idle (polled through CUDA events,
     never by blocking) it enqueues the group's jobs that are not in flight
     -- a request that arrives while the group's batch runs starts at once on
     the other stream instead of waiting for that batch's quantum --, running
     q = min(quantum, smallest remaining S of the launch) proposals.  The
     quantum adapts so that a launch takes about `target_launch_s`.  Slow
     groups never hold back fast ones, and groups and batches overlap on the
     device (the launch timeline is kept, see ``timeline``);
  3. retires finished jobs (results read back, memory released) as soon as
     their launch completes and records each request's latency.

Random streams are keyed by (seed, chain id, step), and the kernel continues
each chain's sums in place, so a request's result is bit-identical whether it
runs alone or in any mix and however its proposals are split into quanta.
All sampling runs in the CUDA library; this module only schedules.
"""
from __future__ import annotations

import time
from dataclasses import dataclass, field

import numpy as np

from .binding import FP64, Context, CrbmError


@dataclass
class Request:
    rid: int
    kind: int
    L: int
    T: np.ndarray
    J: tuple
    S: int
    model: tuple                      # (W, h_bias, v_bias)
    seed: int = 0
    chain_id_base: int = 0
    init_bits: np.ndarray | None = None
    precision: int = FP64
    arrival: float = 0.0


@dataclass
class Result:
    rid: int
    bits: np.ndarray
    step: int
    sums: np.ndarray
    accepts: np.ndarray
    recomputes: np.ndarray
    logpi: np.ndarray
    F: np.ndarray
    E: np.ndarray
    arrival: float
    admitted: float
    finished: float

    @property
    def latency(self):
        return self.finished - self.arrival


@dataclass
class _Active:
    req: Request
    job: object
    remaining: int
    admitted: float
    group: tuple = field(default=())


class _Group:
    """Jobs that can share a launch (same kind, filter shape, precision) and the
    state of that group's two streams: the launches in flight on each and an
    adaptive quantum that aims each launch at `target_s` seconds."""

    def __init__(self, key, streams, quantum):
        self.key = key
        self.streams = streams
        self.quantum = quantum
        self.in_flight = []          # [(end_event, start_event, chunk, q, stream index)]
        self.finished = []           # [(job, stream index)]: read back once that stream is idle

    def busy(self, si):
        return any(f[4] == si for f in self.in_flight)


class Server:
    def __init__(self, device: int = 0, hbm_budget_bytes: int = 8 << 30, quantum: int = 64,
                 max_jobs_per_launch: int = 16, target_launch_s: float = 0.02, adaptive: bool = True):
        import torch
        self.torch = torch
        self.ctx = Context(device, hbm_budget_bytes)
        self.quantum = quantum
        self.adaptive = adaptive
        self.target = target_launch_s
        self.max_per_launch = max_jobs_per_launch
        self.pending: list[Request] = []
        self.active: list[_Active] = []
        self.results: dict[int, Result] = {}
        self.failed: dict[int, str] = {}      # request id -> error (the request is dropped)
        self._models: dict[bytes, int] = {}
        self._groups: dict[tuple, _Group] = {}
        self.launches = 0
        self.proposals = 0
        # every launch as (group key, stream index, start event, end event), and
        # an event recorded when the server started, against which the
        # device-side start and end times of the launches are measured
        self.timeline = []
        self.t0_event = torch.cuda.Event(enable_timing=True)
        self.t0_event.record(torch.cuda.current_stream(device))

    def close(self):
        for g in self._groups.values():
            for st in g.streams:
                st.synchronize()
        for a in self.active:
            a.job.release()
        self.active = []
        self.ctx.close()

    # ---------------------------------------------------------------- requests
    def submit(self, req: Request):
        self.pending.append(req)

    def _model_id(self, req):
        W, hb, vb = req.model
        W = np.ascontiguousarray(W, dtype=np.float64)
        hb = np.ascontiguousarray(hb, dtype=np.float64)
        key = bytes([req.kind]) + W.tobytes() + hb.tobytes() + np.float64(vb).tobytes() + bytes(W.shape)
        if key not in self._models:
            self._models[key] = self.ctx.load_model(req.kind, W, vb, hb)
        return self._models[key], (req.kind, W.shape[0], W.shape[1])

    def _admit(self, now):
        still = []
        for req in sorted(self.pending, key=lambda r: (r.arrival, r.rid)):
            if req.arrival > now:
                still.append(req)
                continue
            try:
                mid, group = self._model_id(req)
                job = self.ctx.new_job(mid, req.kind, req.L, req.T, req.J, req.seed, req.chain_id_base,
                                       req.init_bits, req.precision)
            except CrbmError as e:
                if e.code == -2 and self.active:   # over the HBM budget: wait for memory
                    still.append(req)
                    continue
                self.failed[req.rid] = str(e)     # a bad request fails alone
                continue
            self.active.append(_Active(req, job, req.S, time.perf_counter(), group + (req.precision,)))
        self.pending = still

    # ---------------------------------------------------------------- scheduling
    def _group(self, key):
        if key not in self._groups:
            dev = self.ctx.device
            self._groups[key] = _Group(key, [self.torch.cuda.Stream(device=dev), self.torch.cuda.Stream(device=dev)],
                                       self.quantum)
        return self._groups[key]

    def _complete(self, g: _Group):
        """Retire the group's finished launches (non-blocking, in any order of
        the two streams); True if any finished."""
        done_any = False
        done = [f for f in g.in_flight if f[0].query()]
        g.in_flight = [f for f in g.in_flight if all(f is not d for d in done)]
        for f in done:
            end, start, chunk, q, si = f
            if self.adaptive:
                dt = start.elapsed_time(end) * 1e-3
                if dt > 0:
                    g.quantum = int(min(4096, max(1, g.quantum * min(4.0, max(0.25, self.target / dt)))))
            for a in chunk:
                a.remaining -= q
                if a.remaining <= 0:
                    g.finished.append((a, si))
            done_any = True
        # reading a job back synchronises its stream: only once nothing is in flight on it
        keep = []
        for a, si in g.finished:
            if g.busy(si):
                keep.append((a, si))
            else:
                self._retire(a)
        g.finished = keep
        return done_any

    def _launch(self, g: _Group, members, si):
        busy = {id(a) for f in g.in_flight for a in f[2]}
        ready = sorted((a for a in members if a.remaining > 0 and id(a) not in busy), key=lambda a: a.remaining)
        n = 0
        stream = g.streams[si]
        for i in range(0, len(ready), self.max_per_launch):
            chunk = ready[i:i + self.max_per_launch]
            q = min(g.quantum, min(a.remaining for a in chunk))
            start = self.torch.cuda.Event(enable_timing=True)
            end = self.torch.cuda.Event(enable_timing=True)
            start.record(stream)
            self.ctx.run_batch([a.job for a in chunk], q, precision=g.key[-1], stream=stream)
            end.record(stream)
            g.in_flight.append((end, start, chunk, q, si))
            self.timeline.append((g.key, si, start, end))
            self.proposals += q * sum(a.job.n for a in chunk)
            self.launches += 1
            n += 1
        return n

    def step(self):
        """One scheduling pass: retire what finished, admit arrivals, keep every
        group's stream busy.  Returns the number of launches made."""
        progressed = any([self._complete(g) for g in self._groups.values()])
        self.active = [a for a in self.active if a.remaining > 0]
        self._admit(time.perf_counter())
        by_group: dict[tuple, list[_Active]] = {}
        for a in self.active:
            by_group.setdefault(a.group, []).append(a)
        launched = 0
        for key, members in by_group.items():
            g = self._group(key)
            for si in (0, 1):                   # an idle stream of the group takes the jobs not in flight
                if not g.busy(si):
                    launched += self._launch(g, members, si)
                    break
        return launched + int(progressed)

    def _retire(self, a: _Active):
        bits, step = a.job.state()
        sums, acc, rec = a.job.observables()
        lp, F, E = a.job.energies()
        a.job.release()
        self.results[a.req.rid] = Result(a.req.rid, bits, step, sums, acc, rec, lp, F, E, a.req.arrival,
                                         a.admitted, time.perf_counter())

    def cancel(self, rid: int) -> bool:
        """Drop a waiting or running request; its job memory is released."""
        for i, r in enumerate(self.pending):
            if r.rid == rid:
                del self.pending[i]
                return True
        for a in self.active:
            if a.req.rid == rid:
                g = self._group(a.group)
                for st in g.streams:
                    st.synchronize()
                self._complete(g)
                if a in self.active and a.remaining > 0:
                    a.job.release()
                    self.active.remove(a)
                return True
        return False

    def idle(self):
        return not self.pending and not self.active

    def run(self, requests, realtime: bool = True, timeout_s: float = 600.0):
        """Serve `requests` (arrival times in seconds from now when realtime,
        else all present at once); returns the results by request id."""
        t0 = time.perf_counter()
        for r in requests:
            r.arrival = t0 + (r.arrival if realtime else 0.0)
            self.submit(r)
        while not self.idle():
            if time.perf_counter() - t0 > timeout_s:
                raise TimeoutError("serving loop exceeded its time limit")
            if self.step() == 0:
                time.sleep(0.0002)
        return self.results

    def launch_intervals(self):
        """Device-side (start, end) of every launch in seconds after the
        server started, with its group key and stream index (after the work
        has finished)."""
        self.torch.cuda.synchronize(self.ctx.device)
        return [(key, si, self.t0_event.elapsed_time(a) * 1e-3, self.t0_event.elapsed_time(b) * 1e-3)
                for key, si, a, b in self.timeline]

    def stats(self, t_start: float | None = None):
        lat = np.array([r.latency for r in self.results.values()])
        if not len(lat):
            return {}
        span = max(r.finished for r in self.results.values()) - (
            t_start if t_start is not None else min(r.arrival for r in self.results.values()))
        return {"requests": len(lat), "p50_latency_s": float(np.percentile(lat, 50)),
                "p99_latency_s": float(np.percentile(lat, 99)), "proposals_per_s": self.proposals / span,
                "launches": self.launches, "wall_s": span}


def synthetic_requests(n: int, rate_hz: float = 200.0, seed: int = 2008054010, max_proposals: int = 10 ** 4,
                       min_proposals: int = 10 ** 2, precision: int = FP64, models=None):
    """Poisson arrivals mixing Ising (L in {16,32,64,128,256}) and Kitaev (L in 4..12)
    jobs, T uniform over each model's range, proposals log-uniform, 1-64 chains."""
    import crbm_workloads as wl
    g = np.random.default_rng(seed)
    if models is None:
        models = {0: wl.gaussian_crbm(4, 5, 0.1, seed=seed), 1: wl.gaussian_crbm(4, 3, 0.05, seed=seed + 1)}
    t = 0.0
    out = []
    base = 0
    for rid in range(n):
        t += g.exponential(1.0 / rate_hz)
        kind = int(g.integers(0, 2))
        n_ch = int(g.integers(1, 65))
        S = int(round(np.exp(g.uniform(np.log(min_proposals), np.log(max_proposals)))))
        if kind == 0:
            L = int(g.choice([16, 32, 64, 128, 256]))
            T = g.uniform(1.5, 3.5, size=n_ch)
            J = (1.0,)
        else:
            L = int(g.integers(4, 13))
            T = np.exp(g.uniform(np.log(0.005), np.log(1.0), size=n_ch))
            J = (1.0, 1.0, 1.0)
        out.append(Request(rid, kind, L, T, J, S, models[kind], seed=seed, chain_id_base=base,
                           precision=precision, arrival=t))
        base += n_ch
    return out
