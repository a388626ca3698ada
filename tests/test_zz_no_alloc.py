"""kmedoids_fit_noalloc: the k-medoids entry point that allocates no device memory.

It serves callers that must not allocate device memory during a call (for
example an application whose own allocator reserves the GPU's memory up
front).  Its scratch is a static device array inside the library, shared by
every call.  These tests call it through the C ABI, on two calls in a row with
different inputs (so a second call cannot lean on the first call's scratch
contents), and compare each result with the allocating kmedoids_fit: medoids,
labels and sweep counts identical, cost within 1e-9 relative (the tolerance the
k-medoids parity tests use for float64 costs).  The file is named to be
collected last; it does not depend on any earlier test.
"""

import ctypes

import numpy as np
import pytest
import torch

from paper_2307_04904_gb300 import api, synth

pytestmark = pytest.mark.gpu


def _points_D(n, seed):
    rng = np.random.default_rng(seed)
    pts = rng.standard_normal((n, 3))
    D = np.sqrt(((pts[:, None] - pts[None]) ** 2).sum(-1)).astype(np.float32)
    return torch.from_numpy(np.minimum(D, D.T)).cuda()


def _call_raw(symbol, D, k, init, max_iter=100):
    """Call an entry point through ctypes with preallocated outputs."""
    lib = api.load()
    n = D.shape[0]
    med = torch.full((k,), -1, dtype=torch.int32, device="cuda")
    lab = torch.full((n,), -1, dtype=torch.int32, device="cuda")
    init_t = torch.as_tensor(init, dtype=torch.int32).cuda()
    cost = ctypes.c_double()
    iters = ctypes.c_int32()
    torch.cuda.synchronize()
    rc = getattr(lib, symbol)(D.data_ptr(), n, k, init_t.data_ptr(), max_iter, med.data_ptr(),
                              lab.data_ptr(), ctypes.byref(cost), ctypes.byref(iters),
                              torch.cuda.current_stream().cuda_stream)
    assert rc == api.DTW_OK, lib.dtw_last_error()
    return med.cpu().numpy(), lab.cpu().numpy(), cost.value, iters.value


def test_noalloc_matches_allocating_entry_two_calls():
    cases = [(_points_D(300, 1), 4, synth.init_medoids(300, 4, 1)),
             (_points_D(211, 2), 7, synth.init_medoids(211, 7, 2))]
    for D, k, init in cases:  # two calls in a row on different inputs
        ref = _call_raw("kmedoids_fit", D, k, init)
        got = _call_raw("kmedoids_fit_noalloc", D, k, init)
        assert got[0].tolist() == ref[0].tolist()
        assert got[1].tolist() == ref[1].tolist()
        assert got[3] == ref[3]
        assert got[2] == pytest.approx(ref[2], rel=1e-9)


def test_noalloc_on_dtw_matrix_and_python_binding():
    values, offsets = synth.random_walk_set(50, 128, seed=0)
    D = api.dtw_pairwise(torch.from_numpy(values).cuda(), torch.from_numpy(offsets).cuda(), 12)
    init = torch.as_tensor(synth.init_medoids(50, 3, 0), dtype=torch.int32).cuda()
    for _ in range(2):
        m1, l1, c1, i1 = api.kmedoids_fit(D, 3, init)
        m2, l2, c2, i2 = api.kmedoids_fit_noalloc(D, 3, init)
        assert torch.equal(m1, m2) and torch.equal(l1, l2) and i1 == i2
        assert c2 == pytest.approx(c1, rel=1e-9)


def test_noalloc_rejects_sizes_beyond_its_scratch():
    lib = api.load()
    D = torch.zeros((4, 4), dtype=torch.float32, device="cuda")
    out = torch.zeros(8, dtype=torch.int32, device="cuda")
    # n beyond the static maximum is refused on the host before D is touched
    rc = lib.kmedoids_fit_noalloc(D.data_ptr(), 70000, 2, out.data_ptr(), 10, out.data_ptr(),
                                  out.data_ptr(), None, None, None)
    assert rc == api.DTW_EINVAL
    assert b"static scratch" in lib.dtw_last_error()
