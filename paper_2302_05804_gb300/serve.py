"""Continuous-batching server for EM deconvolution jobs.

Jobs (sky patches of uneven size, exposure count and PSF size) arrive over
time. Every job runs either the direct FP32 form (persistent direct kernel)
or the FFT form (persistent FFT kernels of the same step), as the server is
configured. Each admitted job owns a library context (its x, y, u and PSFs stay
resident in device memory) and joins the running batch: every
``emd_batch_step`` advances ALL admitted jobs by one EM iteration in a
single persistent-kernel launch (replayed from a CUDA graph). New jobs are
admitted between steps whenever a batch slot is free and their device
footprint (``emd_ctx_bytes``) fits the HBM budget; their host-to-device
uploads and set-up kernels run on their own streams while earlier jobs keep
iterating. A finished job is read back, its context freed, and its slot and
memory go to the next job in the queue (first come, first served).

Latency of a job = time its result is on the host - its arrival time.
"""
from __future__ import annotations

import math
import time
from dataclasses import dataclass, field

import numpy as np

from . import emd


@dataclass
class JobSpec:
    """One deconvolution request."""
    jid: int
    arrival: float          # seconds after the start of the run
    H: int
    W: int
    n: int
    K: int
    r: int = 1
    iters: int = 50


@dataclass
class JobData:
    y: np.ndarray
    v: np.ndarray
    f: np.ndarray
    mask: np.ndarray


@dataclass
class JobResult:
    jid: int
    arrival: float
    admitted: float
    finished: float
    x: np.ndarray | None = None
    loglik: float | None = None

    @property
    def latency(self):
        return self.finished - self.arrival


def poisson_trace(n_jobs: int, rate: float, seed: int = 4004, s_range=(128, 2048),
                  n_range=(4, 40), k_range=(15, 43), iters: int = 50, r: int = 1):
    """Poisson arrivals at `rate` jobs/s; side log-uniform in s_range, n
    uniform in n_range, odd K uniform in k_range."""
    g = np.random.Generator(np.random.PCG64(seed))
    t = 0.0
    out = []
    ks = np.arange(k_range[0] | 1, k_range[1] + 1, 2)
    for j in range(n_jobs):
        t += g.exponential(1.0 / rate)
        S = int(round(math.exp(g.uniform(math.log(s_range[0]), math.log(s_range[1])))))
        n = int(g.integers(n_range[0], n_range[1] + 1))
        K = int(g.choice(ks))
        out.append(JobSpec(j, t, S, S, n, K, r, iters))
    return out


class DataPool:
    """Job inputs cut from one resident synthetic frame set: a job of side S
    with n exposures and K x K PSFs takes an S x S window of n exposures
    (cycling through the pool's exposures) and the central K x K of their
    PSFs, renormalised. Only the inputs are shared; every job is solved
    independently."""

    def __init__(self, problem):
        self.p = problem

    def make(self, spec: JobSpec) -> JobData:
        p = self.p
        g = np.random.Generator(np.random.PCG64(spec.jid))
        H, W = spec.H, spec.W
        i0 = int(g.integers(0, p.H - H + 1))
        j0 = int(g.integers(0, p.W - W + 1))
        ts = [(spec.jid + t) % p.n for t in range(spec.n)]
        y = np.ascontiguousarray(p.y[ts, i0:i0 + H, j0:j0 + W])
        v = np.ascontiguousarray(p.v[ts, i0:i0 + H, j0:j0 + W])
        m = np.ascontiguousarray(p.mask[ts, i0:i0 + H, j0:j0 + W])
        c, h = p.K // 2, spec.K // 2
        f = p.f[ts, c - h:c + h + 1, c - h:c + h + 1].astype(np.float64)
        f = (f / f.sum(axis=(1, 2), keepdims=True)).astype(np.float32)
        return JobData(y, v, np.ascontiguousarray(f), m)


class Server:
    """Admission + continuous batching over the library's batch API.

    Preparation threads turn arrived requests into ready contexts
    (inputs cut, context created, frames uploaded on the job's own stream)
    while the stepping thread keeps the batch running; contexts are created
    only while the HBM budget allows. The stepping thread adds ready jobs
    between steps, steps, and retires finished jobs (read back, freed)."""

    def __init__(self, hbm_budget: float = 80e9, max_slots: int = 64, keep_results: bool = False,
                 precision: int = 0, prep_threads: int = 4):
        import threading
        import torch
        self.torch = torch
        self.budget = hbm_budget
        self.max_slots = max_slots
        self.keep = keep_results
        self.precision = precision  # EMD_PREC_FP32 (direct) or EMD_PREC_FFT_FP32
        self.prep_threads = max(1, prep_threads)
        self.batch = emd.emd_batch_create(max_slots)
        self.used = 0
        self.lock = threading.Condition()
        self.ready: list[dict] = []
        self.active: dict[int, dict] = {}  # slot -> record
        self.results: list[JobResult] = []
        self.steps = 0
        self.t0 = time.perf_counter()
        self.error = None

    def now(self):
        return time.perf_counter() - self.t0

    def close(self):
        for rec in list(self.active.values()) + self.ready:
            if "slot" in rec:
                emd.emd_batch_remove(self.batch, rec["slot"])
            emd.emd_destroy(rec["ctx"])
        self.active.clear()
        self.ready.clear()
        emd.emd_batch_destroy(self.batch)
        self.batch = None

    # -- preparation threads ----------------------------------------------------
    def _prepare(self, it, it_lock, data_of, realtime):
        """One preparation worker: takes the next request in arrival order and
        readies its context. Cutting the inputs, uploading them and creating
        the device buffers take host time per job; several workers overlap
        them (numpy copies and the library calls release the GIL)."""
        try:
            while not self.error:
                with it_lock:
                    spec = next(it, None)
                if spec is None:
                    return
                if realtime:
                    delay = spec.arrival - self.now()
                    if delay > 0:
                        time.sleep(delay)
                need = emd.emd_ctx_bytes_precision(spec.H, spec.W, spec.n, spec.K, spec.r,
                                                   self.precision)
                with self.lock:
                    # wait for memory and for a slot to be in sight (a job
                    # larger than the budget runs alone)
                    while (self.used + need > self.budget and self.used > 0) or \
                            len(self.ready) + len(self.active) >= self.max_slots + 4:
                        self.lock.wait(0.05)
                    self.used += need
                data = data_of(spec)
                stream = self.torch.cuda.Stream()
                ctx = emd.emd_create(spec.H, spec.W, spec.n, spec.K, spec.r)
                emd.emd_set_stream(ctx, stream)
                emd.emd_set_frames(ctx, data.y, data.v, data.f, data.mask)
                if self.precision:
                    emd.emd_set_precision(ctx, self.precision)
                with self.lock:
                    # ready jobs are admitted in arrival order
                    rec = dict(spec=spec, ctx=ctx, bytes=need, stream=stream, prepared=self.now())
                    k = len(self.ready)
                    while k > 0 and self.ready[k - 1]["spec"].arrival > spec.arrival:
                        k -= 1
                    self.ready.insert(k, rec)
                    self.lock.notify_all()
        except Exception as e:  # surfaced by run()
            self.error = e

    # -- stepping thread ----------------------------------------------------------
    def _admit(self):
        with self.lock:
            while self.ready and len(self.active) < self.max_slots:
                rec = self.ready.pop(0)
                rec["slot"] = emd.emd_batch_add(self.batch, rec["ctx"], rec["spec"].iters)
                rec["admitted"] = self.now()
                self.active[rec["slot"]] = rec

    def _retire(self):
        done = [s for s in self.active if emd.emd_batch_remaining(self.batch, s) == 0]
        if not done:
            return 0
        emd.emd_batch_sync(self.batch)
        for s in done:
            rec = self.active.pop(s)
            spec = rec["spec"]
            x = np.empty((spec.r * spec.H, spec.r * spec.W), np.float32)
            emd.emd_get_x(rec["ctx"], x)
            res = JobResult(spec.jid, spec.arrival, rec["admitted"], self.now(),
                            x if self.keep else None)
            emd.emd_batch_remove(self.batch, s)
            emd.emd_destroy(rec["ctx"])
            with self.lock:
                self.used -= rec["bytes"]
                self.lock.notify_all()
            self.results.append(res)
        return len(done)

    def run(self, trace, data_of, time_limit: float | None = None, realtime: bool = True):
        """Serve `trace` (JobSpecs sorted by arrival). data_of(spec) -> JobData.
        With realtime=False every job is visible at t = 0 (saturation run)."""
        import threading
        self.t0 = time.perf_counter()
        total = len(trace)
        it, it_lock = iter(list(trace)), threading.Lock()
        preps = [threading.Thread(target=self._prepare, args=(it, it_lock, data_of, realtime),
                                  daemon=True) for _ in range(self.prep_threads)]
        for t in preps:
            t.start()
        while len(self.results) < total:
            if self.error:
                raise self.error
            self._admit()
            if self.active:
                emd.emd_batch_step(self.batch)
                self.steps += 1
                self._retire()
            else:
                with self.lock:
                    if not self.ready:
                        self.lock.wait(0.01)
            if time_limit and self.now() > time_limit:
                break
        for t in preps:
            t.join(timeout=60)
        emd.emd_batch_sync(self.batch)
        if self.error:
            raise self.error
        return self.results

    @staticmethod
    def summary(results, trace_len=None):
        if not results:
            return {}
        lat = np.array([r.latency for r in results])
        span = max(r.finished for r in results) - min(r.arrival for r in results)
        return {"jobs": len(results), "jobs_per_s": len(results) / span,
                "p50_s": float(np.percentile(lat, 50)), "p99_s": float(np.percentile(lat, 99)),
                "mean_s": float(lat.mean()), "span_s": span}
