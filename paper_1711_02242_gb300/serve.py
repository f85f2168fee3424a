"""Continuous-batching server for AFQMC run requests on one GPU.

Requests (a Hamiltonian, a trial, walker count and step count) arrive over
time.  The server owns one device buffer and carves each admitted run's
workspace out of it (first fit, 256-byte aligned): a request is admitted as
soon as its footprint (afqmc_workspace_size) fits, and its walker state stays
resident until it finishes.  Every tick advances every active run by one
chunk of steps, each run on its own CUDA stream (with its own CUDA-graph
replay), so the runs' kernels overlap on the GPU; runs that arrive meanwhile
join at the next tick as memory frees up.  Runs never interact, so each
result is the same as that run stepped alone.
"""
from __future__ import annotations

import dataclasses
import time

import numpy as np

from . import AfqmcRun, afqmc_workspace_size, default_params


class DevicePool:
    """First-fit allocator over one caller-owned uint8 device tensor."""

    def __init__(self, nbytes: int, device="cuda:0"):
        import torch

        self.buf = torch.empty(nbytes, dtype=torch.uint8, device=device)
        base = self.buf.data_ptr()
        self.skew = (-base) % 256
        self.size = nbytes - self.skew
        self.free = [(0, self.size)]  # sorted (offset, length)

    def alloc(self, n: int):
        n = (n + 255) // 256 * 256
        for k, (off, ln) in enumerate(self.free):
            if ln >= n:
                if ln == n:
                    self.free.pop(k)
                else:
                    self.free[k] = (off + n, ln - n)
                return off, n
        return None

    def release(self, off: int, n: int):
        self.free.append((off, n))
        self.free.sort()
        merged = []
        for o, ln in self.free:
            if merged and merged[-1][0] + merged[-1][1] == o:
                merged[-1] = (merged[-1][0], merged[-1][1] + ln)
            else:
                merged.append((o, ln))
        self.free = merged

    def view(self, off: int, n: int):
        return self.buf[self.skew + off: self.skew + off + n]

    def free_bytes(self) -> int:
        return sum(ln for _, ln in self.free)


@dataclasses.dataclass
class Request:
    rid: int
    arrival: float  # seconds after the stream starts
    h1: np.ndarray
    L: np.ndarray
    trial: np.ndarray
    nwalkers: int
    nsteps: int
    seed: int
    energy_period: int = 50
    # filled by the server
    admit: float = float("nan")
    finish: float = float("nan")
    energies: np.ndarray | None = None


class Server:
    def __init__(self, pool_bytes: int, precision: int = 2, chunk_steps: int = 10,
                 device="cuda:0", qr_period: int = 5, dt: float = 0.005,
                 max_active: int | None = None):
        """max_active bounds the runs advanced per tick (slots); None: memory only."""
        self.max_active = max_active
        self.pool = DevicePool(pool_bytes, device)
        self.precision = precision
        self.chunk = chunk_steps
        self.device = device
        self.qr_period = qr_period
        self.dt = dt

    def params(self, r: Request):
        M, N = r.trial.shape
        return default_params(M, N, r.L.shape[0], r.nwalkers, dt=self.dt, seed=r.seed,
                              qr_period=self.qr_period, energy_period=r.energy_period,
                              precision=self.precision, use_graph=1,
                              max_records=max(1, r.nsteps // max(1, r.energy_period)))

    def footprint(self, r: Request) -> int:
        return afqmc_workspace_size(self.params(r)) + 256

    def run(self, requests, realtime: bool = True):
        """Serve `requests` (sorted by arrival).  With realtime, arrivals are
        honoured on the wall clock; otherwise all requests are present at
        t = 0.  Returns the requests with admit/finish times and energies."""
        import torch

        pending = sorted(requests, key=lambda r: r.arrival)
        for r in pending:
            if self.footprint(r) > self.pool.size:
                raise ValueError(f"request {r.rid} needs more than the whole pool")
        queue, active, done = [], [], []
        t0 = time.perf_counter()
        clock = (lambda: time.perf_counter() - t0) if realtime else (lambda: float("inf"))
        while pending or queue or active:
            now = clock()
            while pending and pending[0].arrival <= now:
                queue.append(pending.pop(0))
            # admission in arrival order while a slot is free and the footprint fits
            while queue and (self.max_active is None or len(active) < self.max_active):
                r = queue[0]
                blk = self.pool.alloc(self.footprint(r))
                if blk is None:
                    break
                queue.pop(0)
                stream = torch.cuda.Stream(device=self.device)
                run = AfqmcRun(r.h1, r.L, r.trial, self.params(r), device=self.device,
                               stream=stream, workspace=self.pool.view(*blk))
                r.admit = time.perf_counter() - t0
                active.append([r, run, blk, 0])
            if not active:
                if pending:
                    time.sleep(max(0.0, min(0.01, pending[0].arrival - clock())))
                continue
            # one tick: every active run advances one chunk on its own stream
            for a in active:
                r, run = a[0], a[1]
                n = min(self.chunk, r.nsteps - a[3])
                run.propagate(n)
                a[3] += n
            for a in active:
                a[1].stream.synchronize()
            still = []
            for a in active:
                r, run, blk, steps = a
                if steps >= r.nsteps:
                    r.energies = run.energy_log()
                    r.finish = time.perf_counter() - t0
                    run.close()
                    self.pool.release(*blk)
                    done.append(r)
                else:
                    still.append(a)
            active = still
        return done


def latency_stats(done):
    lat = np.array([r.finish - r.arrival for r in done])
    return {"p50_s": float(np.percentile(lat, 50)), "p99_s": float(np.percentile(lat, 99)),
            "mean_s": float(lat.mean()), "max_s": float(lat.max())}
