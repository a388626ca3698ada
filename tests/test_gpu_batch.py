"""GPU parity of the batched path (include/dtwgb_batch.h) against the oracle.

A batch mixes ragged sets with a per-pair window (per mille of the longer
series), a uniform set, a strict packed set and a query job.  Every output
value must equal the oracle's float mirror bit for bit (same per-pair band,
same float operations), whatever the planner chose: graph or not, sorted or
not, autotuned or not.
"""

import numpy as np
import pytest
import torch

import oracle
from paper_2307_04904_gb300 import api, synth

pytestmark = pytest.mark.gpu


def _series(values, offsets, i):
    return values[offsets[i]:offsets[i + 1]]


def _w_of(job, n, m):
    return job["window_permille"] * max(n, m) // 1000 if job.get("window_permille") else job["window"]


def _expected(job, values, offsets, q=None):
    """Float-mirror values of a job, pair by pair, with the pair's own band."""
    p = len(offsets) - 1
    strict = job.get("strict", False)
    if q is not None:
        out = np.empty(p, np.float32)
        for i in range(p):
            s = _series(values, offsets, i)
            out[i] = oracle.dtw_f32_mirror(q, s, _w_of(job, len(q), len(s)), strict)
        return out
    D = np.zeros((p, p), np.float32)
    for a in range(p):
        for b in range(a + 1, p):
            x, y = _series(values, offsets, a), _series(values, offsets, b)
            D[a, b] = D[b, a] = oracle.dtw_f32_mirror(x, y, _w_of(job, len(x), len(y)), strict)
    if job.get("packed"):
        a, b = np.triu_indices(p, 1)
        return D[a, b]
    return D


def _make_jobs(seed=0):
    specs = []
    lens = synth.ragged_lengths(30, 40, 400, seed=seed + 1)
    v, o, _ = synth.five_class_set(30, lens, seed=seed + 1)
    specs.append(({"window_permille": 50}, v, o, None))
    v, o = synth.random_walk_set(25, 128, seed=seed + 2)
    specs.append(({"window": 12}, v, o, None))
    lens = synth.ragged_lengths(20, 30, 200, seed=seed + 3)
    v, o, _ = synth.five_class_set(20, lens, seed=seed + 3)
    specs.append(({"window": 10, "strict": True, "packed": True}, v, o, None))
    lens = synth.ragged_lengths(40, 100, 700, seed=seed + 4)
    v, o, _ = synth.five_class_set(40, lens, seed=seed + 4)
    q = synth.five_class_set(1, 333, seed=seed + 5)[0]
    specs.append(({"window": 40}, v, o, q))
    jobs = []
    for spec, v, o, q in specs:
        j = dict(spec)
        j.setdefault("window", -1)
        j["values"] = torch.from_numpy(v).cuda()
        j["offsets"] = torch.from_numpy(o).cuda()
        if q is not None:
            j["query"] = torch.from_numpy(q).cuda()
        jobs.append(j)
    return specs, jobs


def _check(batch, specs):
    outs = batch.run()
    torch.cuda.synchronize()
    for (spec, v, o, q), out in zip(specs, outs):
        exp = _expected(spec, v, o, q)
        got = out.cpu().numpy()
        assert got.shape == exp.shape
        assert np.array_equal(got.view(np.uint32), exp.view(np.uint32))


@pytest.mark.parametrize("graph,unsorted", [(True, False), (False, False), (True, True)])
def test_batch_mixed_jobs(graph, unsorted):
    specs, jobs = _make_jobs()
    b = api.Batch(jobs, graph=graph, unsorted=unsorted)
    info = b.info()
    assert info["jobs"] == 4 and info["graph"] == int(graph)
    assert info["pairs"] == 30 * 29 // 2 + 25 * 24 // 2 + 20 * 19 // 2 + 40
    _check(b, specs)
    _check(b, specs)  # a second replay gives the same values
    b.close()


def test_batch_autotune_and_cache(tmp_path, monkeypatch):
    monkeypatch.setenv("DTWGB_TUNE_CACHE", str(tmp_path / "tune.jsonl"))
    specs, jobs = _make_jobs(seed=10)
    b = api.Batch(jobs, graph=True, autotune=True)
    assert b.info()["buckets_tuned"] >= 1
    _check(b, specs)
    b.close()
    # the same buckets again: answered by the cache, nothing is timed
    b2 = api.Batch(jobs, graph=True, autotune=True)
    assert b2.info()["buckets_tuned"] == 0
    _check(b2, specs)
    b2.close()


def test_batch_picks_up_new_data_in_the_same_buffers():
    specs, jobs = _make_jobs(seed=20)
    b = api.Batch(jobs, graph=True)
    _check(b, specs)
    # overwrite the first job's values in place; the next replay must follow them
    spec, v, o, q = specs[0]
    v2 = synth.five_class_set(30, np.diff(o), seed=99)[0]
    jobs[0]["values"].copy_(torch.from_numpy(v2))
    specs[0] = (spec, v2, o, q)
    _check(b, specs)
    b.close()


def test_batch_class_breakdown_covers_all_pairs():
    specs, jobs = _make_jobs(seed=30)
    b = api.Batch(jobs, graph=False)
    cls = b.classes()
    assert sum(c["items"] for c in cls) == b.info()["pairs"]
    cells = 0
    for spec, v, o, q in specs:
        lens = np.diff(o)
        if q is not None:
            pairs = [(len(q), int(l)) for l in lens]
        else:
            pairs = [(int(lens[a]), int(lens[c])) for a in range(len(lens)) for c in range(a + 1, len(lens))]
        for n, m in pairs:
            w = _w_of(spec, n, m)
            strict = spec.get("strict", False)
            if strict and abs(n - m) > w:
                continue
            cells += oracle.band_cells(n, m, w, strict)
    assert b.info()["cells"] == cells
    b.close()


def test_batch_rejects_invalid_job():
    v, o = synth.random_walk_set(3, 10, seed=1)
    bad = o.copy()
    bad[2] = bad[1]
    job = {"values": torch.from_numpy(v).cuda(), "offsets": torch.from_numpy(bad).cuda(),
           "window": 2}
    with pytest.raises(api.DTWError) as e:
        api.Batch([job])
    assert e.value.code == api.DTW_EINVAL


def test_batch_ragged_long_sample():
    """600 series with lengths in [64, 2048], per-pair window 5 % of the longer series."""
    lens = synth.ragged_lengths(600, 64, 2048, seed=2)
    v, o, _ = synth.five_class_set(600, lens, seed=2)
    job = {"values": torch.from_numpy(v).cuda(), "offsets": torch.from_numpy(o).cuda(),
           "window_permille": 50}
    b = api.Batch([job], graph=True, autotune=True)
    D = b.run()[0]
    torch.cuda.synchronize()
    D = D.cpu().numpy()
    assert np.array_equal(D, D.T) and np.all(np.diag(D) == 0)
    rng = np.random.default_rng(3)
    a = rng.integers(0, 600, 400)
    c = rng.integers(0, 600, 400)
    for i, j in zip(a, c):
        if i == j:
            continue
        x, y = _series(v, o, i), _series(v, o, j)
        w = 50 * max(len(x), len(y)) // 1000
        assert D[i, j] == oracle.dtw_f32_mirror(x, y, w)
        ref = oracle.dtw(x, y, w)
        assert abs(D[i, j] - ref) <= 1e-5 * ref
    b.close()


@pytest.mark.parametrize("family", ["tstrip:4", "tstrip:8", "tstrip:16", "strip:4", "rot:12",
                                    "two:6", "two:8", "two:10"])
def test_batch_forced_family(family, monkeypatch):
    # every pair through one family (the transposed strip holds pairs whose shorter series
    # has at most 32 K values; longer ones fall back to the column strip): same bits
    monkeypatch.setenv("DTWGB_BATCH_FAMILY", family)
    specs, jobs = _make_jobs(seed=40)
    b = api.Batch(jobs, graph=True)
    kinds = {c["kind"] for c in b.classes()}
    if family.startswith("tstrip"):
        assert "tstrip" in kinds
    if family.startswith("two"):
        assert "tworow" in kinds
    _check(b, specs)
    _check(b, specs)
    b.close()


def test_batch_full_ragged_workload_sampled():
    """The whole batched ragged workload, 4000 series with lengths uniform in [64, 2048] and a
    per-pair band of 5 % of the longer series (widened to |n - m|), planned and run as the
    benchmark runs it (graph, autotuned).  The 8M-pair matrix is symmetric with a zero
    diagonal; 20000 random pairs, every pair among the 20 shortest and the 20 longest series,
    and each of those 40 against 25 random others are compared with the oracle: bit for bit
    with the float mirror and within 1e-5 of the float64 value."""
    n = 4000
    lens = synth.ragged_lengths(n, 64, 2048, seed=2)
    v, o, _ = synth.five_class_set(n, lens, seed=2)
    job = {"values": torch.from_numpy(v).cuda(), "offsets": torch.from_numpy(o).cuda(),
           "window_permille": 50}
    b = api.Batch([job], graph=True, autotune=True)
    assert b.info()["pairs"] == n * (n - 1) // 2
    D = b.run()[0]
    torch.cuda.synchronize()
    D = D.cpu().numpy()
    b.close()
    assert np.all(np.diag(D) == 0) and np.array_equal(D, D.T)
    rng = np.random.default_rng(4)
    order = np.argsort(lens, kind="stable")
    ext = np.concatenate([order[:20], order[-20:]])
    ea, eb = np.triu_indices(len(ext), 1)
    sa = np.concatenate([rng.integers(0, n, 20000), ext[ea], np.repeat(ext, 25)])
    sb = np.concatenate([rng.integers(0, n, 20000), ext[eb], rng.integers(0, n, 25 * len(ext))])
    keep = sa != sb
    sa, sb = sa[keep], sb[keep]
    assert len(sa) >= 20000
    w = np.maximum(lens[sa], lens[sb]) * 50 // 1000
    mir = oracle.pairs_w_f32_mirror(v, o, sa, sb, w)
    ref = oracle.pairs_w(v, o, sa, sb, w)
    got = D[sa, sb]
    bad = np.flatnonzero(got.view(np.uint32) != mir.view(np.uint32))
    assert bad.size == 0, f"{bad.size} pairs differ from the float mirror, first {(sa[bad[0]], sb[bad[0]])}"
    rel = np.abs(got.astype(np.float64) - ref) / ref
    assert rel.max() <= 1e-5, rel.max()


def test_run_once_equals_plain_calls():
    """dtw_batch_run_once (stream-ordered pool, every class on the caller's stream, no
    device synchronisation) gives every job the bits of dtw_pairwise / dtw_query, and a
    second call on new data in fresh buffers does too."""
    for seed in (50, 51):
        specs, jobs = _make_jobs(seed=seed)
        for j, (spec, v, o, q) in zip(jobs, specs):
            j["offsets_host"] = o
        stream = torch.cuda.Stream()
        with torch.cuda.stream(stream):
            outs = api.batch_run_once(jobs, stream=stream)
        stream.synchronize()
        for (spec, v, o, q), out in zip(specs, outs):
            exp = _expected(spec, v, o, q)
            got = out.cpu().numpy()
            assert np.array_equal(got.view(np.uint32), exp.view(np.uint32))


def test_host_offsets_flag_equals_device_offsets():
    lens = synth.ragged_lengths(30, 60, 300, seed=61)
    v, o, _ = synth.five_class_set(30, lens, seed=61)
    vt, ot = torch.from_numpy(v).cuda(), torch.from_numpy(o).cuda()
    for w in (8, 40):
        a = api.dtw_pairwise(vt, ot, w)
        b = api.dtw_pairwise(vt, None, w, offsets_host=o)
        assert torch.equal(a, b)
        q = torch.from_numpy(synth.five_class_set(1, 150, seed=62)[0]).cuda()
        assert torch.equal(api.dtw_query(q, vt, ot, w), api.dtw_query(q, vt, None, w, offsets_host=o))
