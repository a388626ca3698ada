"""The serving loop on the GPU: every job's result in the mix equals its result alone."""

import numpy as np
import pytest
import torch

from paper_2307_04904_gb300 import api, serving

pytestmark = pytest.mark.gpu


def _alone(job, resident_sets):
    if job.kind == "cluster":
        v = torch.from_numpy(job.values).cuda()
        o = torch.from_numpy(job.offsets).cuda()
        D = api.dtw_pairwise(v, o, job.window)
        med, lab, cost, it = api.kmedoids_fit(
            D, job.k, torch.as_tensor(job.init_medoids, dtype=torch.int32).cuda(), job.max_iter)
        resident_sets[job.set_id] = (v, o)
        return {"medoids": med.cpu().numpy(), "labels": lab.cpu().numpy(), "cost": cost,
                "iters": it}
    v, o = resident_sets[job.set_id]
    return {"row": api.dtw_query(torch.from_numpy(job.query).cuda(), v, o, job.window).cpu().numpy()}


def test_results_in_the_mix_equal_results_alone():
    arrivals = serving.poisson_stream(16, rate=200.0, seed=11, n_range=(40, 220),
                                      len_range=(64, 200), k_range=(2, 6))
    alone, sets = [], {}
    for _, job in arrivals:
        alone.append(_alone(job, sets))
    torch.cuda.synchronize()
    srv = serving.DTWServer(slots=4, hbm_budget=2 << 30)
    futs = serving.replay(srv, arrivals, realtime=True)
    mixed = [f.result(timeout=120) for f in futs]
    srv.drain(timeout=60)
    st = srv.stats()
    srv.close()
    assert st["jobs"] == len(arrivals)
    for (_, job), a, m in zip(arrivals, alone, mixed):
        if job.kind == "cluster":
            assert np.array_equal(a["medoids"], m["medoids"])
            assert np.array_equal(a["labels"], m["labels"])
            assert a["cost"] == m["cost"] and a["iters"] == m["iters"]
        else:
            assert np.array_equal(a["row"].view(np.uint32), m["row"].view(np.uint32))


def test_tight_budget_queues_but_completes():
    arrivals = serving.poisson_stream(8, rate=500.0, seed=12, n_range=(100, 200),
                                      len_range=(64, 96), query_frac=0.0)
    biggest = max(j.resident_bytes() + j.transient_bytes() for _, j in arrivals)
    srv = serving.DTWServer(slots=4, hbm_budget=int(biggest * 1.2))
    futs = serving.replay(srv, arrivals, realtime=False)
    for f in futs:
        assert f.result(timeout=120)["cost"] > 0
    st = srv.stats()
    srv.close()
    assert st["jobs"] == 8 and st["queue_high_water"] >= 2
