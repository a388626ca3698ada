"""Continuous-batching server for clustering and query jobs on one GPU.

Jobs arrive at any time (``submit``).  A scheduler thread admits them in
arrival order as soon as a worker slot and enough of the HBM budget are free
(first fit: a later job that fits may pass an earlier one that does not, but a
job that has waited longer than ``max_bypass_s`` blocks further bypassing until
it is admitted).  Each worker owns a CUDA stream and runs its work through the
library's C ABI; ctypes releases the GIL during the calls, so admitted work runs
concurrently and its kernels overlap on the device.

Continuous batching: a small job (a query, or a clustering job of at most
``pack_pairs`` pairs) is admitted together with every other small job that is
admissible in the same scheduling tick (up to ``pack_jobs`` jobs and
``pack_max_cells`` DP cells): their DTW work -- all pairs of each set, every
query row -- is planned as one batch and runs as one set of cost-sorted
persistent launches (``batch_run_once``: stream-ordered buffers, no device
synchronisation), on a high-priority stream; then each clustering job's
k-medoids runs on its own matrix.  A large clustering job runs alone on a
low-priority stream (``dtw_pairwise`` with host offsets, then k-medoids).  The
library launches that DTW kernel with one block per chunk of pairs rather than
a persistent grid, so the high-priority work of later small jobs is scheduled
on SMs as its blocks retire instead of waiting for the whole matrix.

Two job kinds:

* ``ClusterJob`` -- upload a set of series, build its DTW matrix D
  (``dtw_pairwise``), cluster it (``kmedoids_fit``).  With ``keep`` the series
  and D stay resident on the device under ``set_id`` (the paper's k-medoids and
  MIP both consume D; queries reuse the series).
* ``QueryJob`` -- one query against a resident set (``dtw_query``): one row
  of D.  It waits until its set is resident.

Memory: a job is admitted only if its footprint (inputs, D, scratch) fits in
the budget next to what is resident and running; resident sets no job uses are
evicted least-recently-used first to make room.  A job larger than the whole
budget is rejected at submission.

Latency of a job = completion time - submission time; ``stats()`` reports
p50/p99 per kind, served GCUPS (in-band DP cells of finished jobs / wall
time) and the admission queue's high-water mark.
"""

from __future__ import annotations

import collections
import dataclasses
import threading
import time
from concurrent.futures import Future

import numpy as np

_PAD_FLOATS = 700  # per-series padding of the library's staging copy, upper bound


def band_cells(n: int, m: int, w: int) -> int:
    """In-band cells of one pair (n <= m), default band reading max(w, m-n)."""
    if n > m:
        n, m = m, n
    w = m - 1 if w < 0 else min(max(w, m - n), m - 1)
    a = min(n, max(0, m - w))
    s1 = a * (a + 1) // 2 + a * w + (n - a) * m
    b = min(n, w)
    s2 = b + ((n - w) * (n - w + 1) // 2 if n > w else 0)
    return s1 - s2 + n


@dataclasses.dataclass
class ClusterJob:
    set_id: str
    values: np.ndarray        # float32, concatenated series
    offsets: np.ndarray       # int64, p+1
    window: int
    k: int
    init_medoids: np.ndarray  # int64, k distinct
    keep: bool = True
    max_iter: int = 100

    kind = "cluster"

    @property
    def p(self) -> int:
        return len(self.offsets) - 1

    def cells(self) -> int:
        lens = np.diff(self.offsets)
        if np.all(lens == lens[0]):
            return self.p * (self.p - 1) // 2 * band_cells(int(lens[0]), int(lens[0]), self.window)
        tot = 0
        for i in range(self.p):
            for j in range(i + 1, self.p):
                tot += band_cells(int(lens[i]), int(lens[j]), self.window)
        return tot

    def resident_bytes(self) -> int:
        return 4 * self.values.size + 8 * self.offsets.size + 4 * self.p * self.p

    def transient_bytes(self) -> int:
        return 4 * (self.values.size + self.p * _PAD_FLOATS) + 8 * self.p + 4 * self.p + 4096


@dataclasses.dataclass
class QueryJob:
    set_id: str
    query: np.ndarray  # float32
    window: int

    kind = "query"

    def transient_bytes(self, p: int) -> int:
        return 4 * (self.query.size + _PAD_FLOATS) + 4 * p + 4096


@dataclasses.dataclass
class Resident:
    values: object
    offsets: object
    D: object
    lens: np.ndarray
    nbytes: int
    users: int = 0
    last_use: float = 0.0
    offsets_host: np.ndarray | None = None


class GpuExecutor:
    """Runs jobs on the GPU through the library (one CUDA stream per worker)."""

    def __init__(self, device: int = 0):
        import torch

        self.torch = torch
        self.device = torch.device("cuda", device)

    def make_stream(self, high_priority: bool = False):
        lo, hi = self.torch.cuda.Stream.priority_range()
        return self.torch.cuda.Stream(device=self.device, priority=hi if high_priority else lo)

    def _upload(self, a):
        return self.torch.from_numpy(a).pin_memory().to(self.device, non_blocking=True)

    def _cluster_result(self, job, D, stream):
        from . import api

        torch = self.torch
        init = torch.as_tensor(job.init_medoids, dtype=torch.int32).to(self.device,
                                                                       non_blocking=True)
        med, lab, cost, iters = api.kmedoids_fit(D, job.k, init, job.max_iter, stream=stream)
        return {"medoids": med.cpu().numpy(), "labels": lab.cpu().numpy(), "cost": cost,
                "iters": iters}

    def run_cluster(self, job: ClusterJob, stream):
        """A large clustering job alone: the all-pairs matrix from host offsets, k-medoids."""
        torch = self.torch
        from . import api

        with torch.cuda.device(self.device), torch.cuda.stream(stream):
            v = self._upload(job.values)
            o = self._upload(job.offsets)
            D = api.dtw_pairwise(v, o, job.window, offsets_host=job.offsets, stream=stream)
            result = self._cluster_result(job, D, stream)
            stream.synchronize()
        return result, Resident(v, o, D, np.diff(job.offsets), job.resident_bytes(),
                                offsets_host=job.offsets)

    def run_query(self, job: QueryJob, res: Resident, stream):
        torch = self.torch
        from . import api

        with torch.cuda.device(self.device), torch.cuda.stream(stream):
            q = self._upload(job.query)
            row = api.dtw_query(q, res.values, res.offsets, job.window,
                                offsets_host=res.offsets_host, stream=stream)
            out = row.cpu().numpy()
            stream.synchronize()
        return {"row": out}

    def run_group(self, group, stream):
        """Small jobs admitted together: one batch for all their DTW work, then k-medoids
        per clustering job.  `group` is a list of (job, resident set or None); returns a
        list of (result, new resident set or None)."""
        torch = self.torch
        from . import api

        with torch.cuda.device(self.device), torch.cuda.stream(stream):
            jobs, keep = [], []
            for job, res in group:
                if job.kind == "cluster":
                    v = self._upload(job.values)
                    o = self._upload(job.offsets)
                    jobs.append({"values": v, "offsets": o, "offsets_host": job.offsets,
                                 "window": job.window})
                    keep.append((v, o))
                else:
                    q = self._upload(job.query)
                    jobs.append({"values": res.values, "offsets": res.offsets,
                                 "offsets_host": res.offsets_host, "query": q,
                                 "window": job.window})
                    keep.append(q)
            outs = api.batch_run_once(jobs, stream=stream)
            results = []
            for (job, res), out, kept in zip(group, outs, keep):
                if job.kind == "cluster":
                    v, o = kept
                    results.append((self._cluster_result(job, out, stream),
                                    Resident(v, o, out, np.diff(job.offsets),
                                             job.resident_bytes(), offsets_host=job.offsets)))
                else:
                    results.append(({"row": out.cpu().numpy()}, None))
            stream.synchronize()
        return results


class DTWServer:
    def __init__(self, executor=None, *, slots: int = 4, hbm_budget: int = 16 << 30,
                 max_bypass_s: float = 2.0, pack_pairs: int = 20000, pack_jobs: int = 32,
                 pack_max_cells: float = 2e10):
        self.ex = executor if executor is not None else GpuExecutor()
        self.slots = slots
        self.budget = int(hbm_budget)
        self.max_bypass_s = max_bypass_s
        self.pack_pairs = pack_pairs
        self.pack_jobs = pack_jobs
        self.pack_max_cells = pack_max_cells
        self._lock = threading.Condition()
        self._pending = collections.deque()  # (t_submit, job, future)
        self._free_slots = list(range(slots))
        # per slot: a low-priority stream for large jobs, a high-priority one for groups
        self._streams = [self.ex.make_stream() for _ in range(slots)]
        self._fast_streams = [self._make_fast_stream() for _ in range(slots)]
        self._groups = []  # sizes of the groups run, for stats()
        self._running_bytes = 0
        self._resident: dict[str, Resident] = {}
        self._resident_bytes = 0
        self._closing = False
        self._records = []  # (kind, t_submit, t_done, cells)
        self._queue_hwm = 0
        self._t0 = time.perf_counter()
        self._busy = 0
        self._sched = threading.Thread(target=self._schedule, daemon=True)
        self._sched.start()

    # ------------------------------------------------------------ public API

    def submit(self, job) -> Future:
        fut = Future()
        need = self._footprint(job)
        if need > self.budget:
            fut.set_exception(MemoryError(
                f"job needs {need} bytes, more than the HBM budget of {self.budget}"))
            return fut
        with self._lock:
            self._pending.append((time.perf_counter(), job, fut))
            self._queue_hwm = max(self._queue_hwm, len(self._pending))
            self._lock.notify_all()
        return fut

    def drain(self, timeout: float | None = None):
        """Wait until every submitted job has finished."""
        t_end = None if timeout is None else time.perf_counter() + timeout
        with self._lock:
            while self._pending or self._busy:
                left = None if t_end is None else t_end - time.perf_counter()
                if left is not None and left <= 0:
                    raise TimeoutError("jobs still pending")
                self._lock.wait(timeout=left if left is not None else 0.5)

    def close(self):
        with self._lock:
            self._closing = True
            self._lock.notify_all()
        self._sched.join(timeout=10)

    def resident_sets(self):
        with self._lock:
            return dict(self._resident)

    def stats(self) -> dict:
        with self._lock:
            recs = list(self._records)
            hwm = self._queue_hwm
        out = {"jobs": len(recs), "queue_high_water": hwm}
        with self._lock:
            groups = list(self._groups)
        if groups:
            out["groups"] = {"count": len(groups), "jobs_packed": int(sum(g for g in groups if g > 1)),
                             "largest": int(max(groups)), "mean": float(np.mean(groups))}
        for kind in ("cluster", "query"):
            lat = np.array([d - s for k, s, d, _ in recs if k == kind])
            if lat.size:
                out[kind] = {"n": int(lat.size), "p50_ms": float(np.percentile(lat, 50) * 1e3),
                             "p99_ms": float(np.percentile(lat, 99) * 1e3),
                             "max_ms": float(lat.max() * 1e3)}
        if recs:
            t0 = min(s for _, s, _, _ in recs)
            t1 = max(d for _, _, d, _ in recs)
            cells = sum(c for *_, c in recs)
            out["wall_s"] = t1 - t0
            out["served_gcups"] = cells / max(t1 - t0, 1e-9) / 1e9
            out["cells"] = cells
            # time from the last submission to the last result: the queue's drain
            out["drain_s"] = t1 - max(s for _, s, _, _ in recs)
        return out

    # -------------------------------------------------------------- internals

    def _make_fast_stream(self):
        try:
            return self.ex.make_stream(high_priority=True)
        except TypeError:  # an executor without stream priorities
            return self.ex.make_stream()

    def _cells(self, job) -> float:
        if job.kind == "cluster":
            return float(job.cells())
        res = self._resident.get(job.set_id)
        if res is None:
            return 0.0
        return float(sum(band_cells(len(job.query), int(l), job.window) for l in res.lens))

    def _small(self, job) -> bool:
        return job.kind == "query" or job.p * (job.p - 1) // 2 <= self.pack_pairs

    def _reserve(self, job):
        """Account an admitted job's footprint; returns (bytes, resident set used or None)."""
        if job.kind == "cluster":
            need, res = self._footprint(job), None
        else:
            res = self._resident[job.set_id]
            res.users += 1
            need = job.transient_bytes(len(res.lens))
        self._running_bytes += need
        return need, res

    def _footprint(self, job) -> int:
        if job.kind == "cluster":
            return job.resident_bytes() + job.transient_bytes()
        res = self._resident.get(job.set_id)
        p = len(res.lens) if res is not None else 0
        return job.transient_bytes(p)

    def _evict_for(self, need: int) -> bool:
        """Evict unused resident sets (LRU) until `need` bytes fit; True if they do."""
        def free():
            return self.budget - self._resident_bytes - self._running_bytes

        if need <= free():
            return True
        victims = sorted((r.last_use, sid) for sid, r in self._resident.items() if r.users == 0)
        waiting = {j.set_id for _, j, _ in self._pending if j.kind == "query"}
        for _, sid in victims:
            if sid in waiting:
                continue
            r = self._resident.pop(sid)
            self._resident_bytes -= r.nbytes
            if need <= free():
                return True
        return need <= free()

    def _admissible(self, job) -> bool:
        if job.kind == "query":
            res = self._resident.get(job.set_id)
            if res is None:
                return False  # its set is not resident (yet)
            return self._evict_for(job.transient_bytes(len(res.lens)))
        return self._evict_for(self._footprint(job))

    def _schedule(self):
        while True:
            with self._lock:
                while not self._closing and (not self._pending or not self._free_slots):
                    self._lock.wait(timeout=0.05)
                if self._closing:
                    return
                now = time.perf_counter()
                chosen = None
                for idx, (t_sub, job, fut) in enumerate(self._pending):
                    if self._admissible(job):
                        chosen = idx
                        break
                    if now - t_sub > self.max_bypass_s:
                        break  # this one has waited long enough: no bypassing it
                if chosen is None:
                    self._lock.wait(timeout=0.01)
                    continue
                entry = self._pending[chosen]
                del self._pending[chosen]
                group = [entry]
                if self._small(entry[1]):
                    # pack every other small job admissible now (arrival order)
                    cells = self._cells(entry[1])
                    need, res = self._reserve(entry[1])
                    members = [(entry, need, res)]
                    idx = 0
                    while idx < len(self._pending) and len(members) < self.pack_jobs:
                        e = self._pending[idx]
                        if not self._small(e[1]) and now - e[0] > self.max_bypass_s:
                            break  # a large job that has waited long enough is not bypassed
                        c = self._cells(e[1]) if self._small(e[1]) else None
                        if (c is not None and cells + c <= self.pack_max_cells
                                and self._admissible(e[1])):
                            del self._pending[idx]
                            n2, r2 = self._reserve(e[1])
                            members.append((e, n2, r2))
                            cells += c
                            continue
                        idx += 1
                    group = members
                    stream_set = self._fast_streams
                else:
                    need, res = self._reserve(entry[1])
                    group = [(entry, need, res)]
                    stream_set = self._streams
                slot = self._free_slots.pop()
                self._busy += len(group)
                self._groups.append(len(group))
            threading.Thread(target=self._work_group, args=(slot, stream_set[slot], group),
                             daemon=True).start()

    def _run(self, group, stream):
        """Results of a group: (result, new resident or None, error or None, cells) per job."""
        out = []
        if len(group) > 1 or (hasattr(self.ex, "run_group") and self._small(group[0][0][1])):
            if hasattr(self.ex, "run_group"):
                try:
                    res = self.ex.run_group([(e[1], r) for e, _, r in group], stream)
                    return [(result, resident, None) for result, resident in res]
                except Exception as err:  # the whole group fails together
                    return [(None, None, err) for _ in group]
        for (t_sub, job, fut), need, res in group:  # one by one
            try:
                if job.kind == "cluster":
                    result, resident = self.ex.run_cluster(job, stream)
                else:
                    result, resident = self.ex.run_query(job, res, stream), None
                out.append((result, resident, None))
            except Exception as err:  # reported through the job's future
                out.append((None, None, err))
        return out

    def _work_group(self, slot, stream, group):
        outcomes = self._run(group, stream)
        t_done = time.perf_counter()
        finished = []
        with self._lock:
            for ((t_sub, job, fut), need, res), (result, resident, err) in zip(group, outcomes):
                self._running_bytes -= need
                if job.kind == "query":
                    res.users -= 1
                    res.last_use = t_done
                    cells = sum(band_cells(len(job.query), int(l), job.window) for l in res.lens)
                else:
                    cells = job.cells()
                    if resident is not None and job.keep:
                        old = self._resident.pop(job.set_id, None)
                        if old is not None:
                            self._resident_bytes -= old.nbytes
                        resident.last_use = t_done
                        self._resident[job.set_id] = resident
                        self._resident_bytes += resident.nbytes
                self._busy -= 1
                if err is None:
                    self._records.append((job.kind, t_sub, t_done, cells))
                finished.append((fut, result, err))
            self._free_slots.append(slot)
            self._lock.notify_all()
        for fut, result, err in finished:
            if err is not None:
                fut.set_exception(err)
            else:
                fut.set_result(result)


# ------------------------------------------------------------ job streams


def poisson_stream(n_jobs: int, rate: float = 20.0, seed: int = 4, n_range=(100, 5000),
                   len_range=(128, 1024), k_range=(2, 12), query_frac: float = 0.3,
                   window_frac: float = 0.1):
    """Arrival times and jobs of a Poisson stream of clustering and query jobs.

    Clustering jobs: N ~ U[n_range] series of one length L ~ U[len_range] from
    the five class generators, window floor(window_frac * L), k ~ U[k_range].
    A query job asks one new series of the same length against the set of an
    earlier clustering job.  Returns a list of (t_arrival_s, job).
    """
    from . import synth

    rng = np.random.default_rng(seed)
    t = 0.0
    out = []
    sets = []
    for i in range(n_jobs):
        t += rng.exponential(1.0 / rate)
        if sets and rng.random() < query_frac:
            sid, L, w = sets[int(rng.integers(0, len(sets)))]
            q = synth.five_class_set(1, L, seed=seed * 100003 + i)[0]
            out.append((t, QueryJob(sid, q, w)))
            continue
        N = int(rng.integers(n_range[0], n_range[1] + 1))
        L = int(rng.integers(len_range[0], len_range[1] + 1))
        k = int(rng.integers(k_range[0], k_range[1] + 1))
        w = int(window_frac * L)
        v, o, _ = synth.five_class_set(N, L, seed=seed * 100003 + i)
        sid = f"set{i}"
        out.append((t, ClusterJob(sid, v, o, w, k, synth.init_medoids(N, k, seed + i))))
        sets.append((sid, L, w))
    return out


def replay(server: DTWServer, arrivals, realtime: bool = True):
    """Submit jobs at their arrival times (or all at once); returns the futures."""
    t0 = time.perf_counter()
    futs = []
    for t, job in arrivals:
        if realtime:
            delay = t - (time.perf_counter() - t0)
            if delay > 0:
                time.sleep(delay)
        futs.append(server.submit(job))
    return futs
