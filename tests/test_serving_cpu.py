"""Scheduling logic of the continuous-batching server, with a fake executor (no GPU)."""

import threading
import time

import numpy as np
import pytest

from paper_2307_04904_gb300 import serving, synth


class FakeExecutor:
    """Sleeps instead of computing; records how many jobs run at once."""

    def __init__(self, t_cluster=0.02, t_query=0.005):
        self.t_cluster, self.t_query = t_cluster, t_query
        self.lock = threading.Lock()
        self.running = 0
        self.max_running = 0
        self.order = []

    def make_stream(self):
        return None

    def _enter(self, tag):
        with self.lock:
            self.running += 1
            self.max_running = max(self.max_running, self.running)
            self.order.append(tag)

    def _leave(self):
        with self.lock:
            self.running -= 1

    def run_cluster(self, job, stream):
        self._enter(job.set_id)
        time.sleep(self.t_cluster)
        self._leave()
        return ({"p": job.p},
                serving.Resident(None, None, None, np.diff(job.offsets), job.resident_bytes()))

    def run_query(self, job, res, stream):
        self._enter("q:" + job.set_id)
        time.sleep(self.t_query)
        self._leave()
        return {"row": np.zeros(len(res.lens), np.float32)}


def _cluster(i, N=50, L=64, keep=True):
    v, o = synth.random_walk_set(N, L, seed=i)
    return serving.ClusterJob(f"s{i}", v, o, 6, 3, synth.init_medoids(N, 3, i), keep=keep)


def test_all_jobs_finish_and_run_concurrently():
    ex = FakeExecutor()
    srv = serving.DTWServer(ex, slots=4, hbm_budget=1 << 30)
    futs = [srv.submit(_cluster(i)) for i in range(12)]
    for i, f in enumerate(futs):
        assert f.result(timeout=10)["p"] == 50
    srv.drain(timeout=10)
    assert ex.max_running > 1
    st = srv.stats()
    assert st["jobs"] == 12 and st["cluster"]["n"] == 12
    assert st["cluster"]["p99_ms"] >= st["cluster"]["p50_ms"] > 0
    srv.close()


def test_admission_by_footprint():
    ex = FakeExecutor()
    job = _cluster(0, N=100, L=64, keep=False)
    need = job.resident_bytes() + job.transient_bytes()
    # room for one job at a time although four slots are free
    srv = serving.DTWServer(ex, slots=4, hbm_budget=int(need * 1.5))
    futs = [srv.submit(_cluster(i, N=100, L=64, keep=False)) for i in range(6)]
    for f in futs:
        f.result(timeout=10)
    assert ex.max_running == 1
    srv.close()


def test_job_larger_than_budget_is_rejected():
    srv = serving.DTWServer(FakeExecutor(), slots=2, hbm_budget=1000)
    with pytest.raises(MemoryError):
        srv.submit(_cluster(0)).result(timeout=5)
    srv.close()


def test_query_waits_for_its_set_and_lru_eviction():
    ex = FakeExecutor(t_cluster=0.05)
    one = _cluster(0, N=60, L=64)
    # one running job plus two and a half resident sets
    srv = serving.DTWServer(ex, slots=2,
                            hbm_budget=int(one.transient_bytes() + 3.5 * one.resident_bytes()))
    q = serving.QueryJob("s0", synth.random_walk_set(1, 64, seed=9)[0], 6)
    fq = srv.submit(q)  # submitted before its set exists: must wait
    f0 = srv.submit(_cluster(0, N=60, L=64))
    assert fq.result(timeout=10)["row"].shape == (60,)
    f0.result(timeout=10)
    assert ex.order.index("s0") < ex.order.index("q:s0")
    # more sets than fit: older unused ones are evicted, the newest stays resident
    for i in range(1, 5):
        srv.submit(_cluster(i, N=60, L=64)).result(timeout=10)
    res = srv.resident_sets()
    assert "s4" in res and len(res) <= 3 and "s0" not in res
    srv.close()


def test_band_cells_matches_closed_form():
    assert serving.band_cells(512, 512, 51) == 50084
    assert serving.band_cells(128, 128, 12) == 3044
    import oracle

    for n, m, w in [(80, 394, 19), (300, 300, -1), (64, 2048, 102), (10, 12, 0)]:
        assert serving.band_cells(n, m, w) == oracle.band_cells(n, m, w)


def test_poisson_stream_shape():
    arr = serving.poisson_stream(40, rate=20.0, seed=4, n_range=(20, 40), len_range=(32, 48))
    ts = [t for t, _ in arr]
    assert all(b > a for a, b in zip(ts, ts[1:]))
    kinds = [j.kind for _, j in arr]
    assert kinds[0] == "cluster" and "query" in kinds
    for _, j in arr:
        if j.kind == "query":
            assert any(c.kind == "cluster" and c.set_id == j.set_id for _, c in arr)


class FakeGroupExecutor(FakeExecutor):
    """A FakeExecutor that also runs packed groups, recording their sizes and kinds."""

    def __init__(self, **kw):
        super().__init__(**kw)
        self.groups = []

    def make_stream(self, high_priority=False):
        return "fast" if high_priority else "slow"

    def run_group(self, group, stream):
        assert stream == "fast"
        with self.lock:
            self.groups.append(sorted(j.kind for j, _ in group))
        self._enter(f"group{len(group)}")
        time.sleep(self.t_cluster)
        self._leave()
        out = []
        for job, res in group:
            if job.kind == "cluster":
                out.append(({"p": job.p}, serving.Resident(None, None, None, np.diff(job.offsets),
                                                           job.resident_bytes())))
            else:
                out.append(({"row": np.zeros(len(res.lens), np.float32)}, None))
        return out


def test_small_jobs_admitted_together_share_one_group():
    """Small jobs waiting at the same tick are packed into one group (one batch on the
    device, high-priority stream); a job above pack_pairs runs alone; every future gets
    its own result."""
    ex = FakeGroupExecutor(t_cluster=0.05)
    srv = serving.DTWServer(ex, slots=1, hbm_budget=1 << 30, pack_pairs=2000)
    big = _cluster(99, N=120, L=128)  # 7140 pairs: above pack_pairs
    first = srv.submit(_cluster(0))  # occupies the only slot while the rest queue
    time.sleep(0.01)
    futs = [srv.submit(_cluster(i)) for i in range(1, 9)] + [srv.submit(big)]
    assert first.result(timeout=10)["p"] == 50
    for f in futs[:-1]:
        assert f.result(timeout=10)["p"] == 50
    assert futs[-1].result(timeout=10)["p"] == 120
    srv.drain(timeout=10)
    st = srv.stats()
    srv.close()
    # the eight queued small jobs went out in one group; the large one alone, not as a group
    assert ["cluster"] * 8 in ex.groups
    assert st["groups"]["largest"] == 8 and st["jobs"] == 10
    assert "99" not in "".join(ex.order[:-1]) and ex.order[-1] == "s99"


def test_queries_join_groups_once_their_set_is_resident():
    ex = FakeGroupExecutor(t_cluster=0.03)
    srv = serving.DTWServer(ex, slots=2, hbm_budget=1 << 30)
    c = _cluster(1)
    assert srv.submit(c).result(timeout=10)["p"] == 50
    q = [serving.QueryJob("s1", np.zeros(64, np.float32), 6) for _ in range(5)]
    futs = [srv.submit(j) for j in q]
    for f in futs:
        assert f.result(timeout=10)["row"].shape == (50,)
    srv.drain(timeout=10)
    srv.close()
    assert any("query" in g for g in ex.groups)
