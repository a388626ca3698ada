"""GPU parity of dtw_pairwise / dtw_query against the CPU oracle (through the C ABI).

Tolerance: relative error <= 1e-5 against the float64 oracle (exact zeros
compared exactly), and bit-for-bit equality with the oracle's float mirror,
which performs the same float operations per cell (d = x - y rounded, then one
fused multiply-add onto the exact three-way minimum).
"""

import numpy as np
import pytest
import torch

import oracle
from paper_2307_04904_gb300 import api, synth

pytestmark = pytest.mark.gpu
RTOL = 1e-5


def _dev(values, offsets):
    return (torch.from_numpy(values).cuda(), torch.from_numpy(offsets).cuda())


def _check_matrix(values, offsets, w, strict=False, D=None):
    v, o = _dev(values, offsets)
    if D is None:
        D = api.dtw_pairwise(v, o, w, strict=strict)
    torch.cuda.synchronize()
    D = D.cpu().numpy()
    p = len(offsets) - 1
    ref = oracle.pairwise(values, offsets, w, strict)
    a, b = np.triu_indices(p, 1)
    mirror = oracle.pairs_f32_mirror(values, offsets, a, b, w, strict)
    assert np.all(np.diag(D) == 0)
    assert np.array_equal(D, D.T)
    got = D[a, b]
    assert np.array_equal(got.view(np.uint32), mirror.view(np.uint32)), \
        f"float mirror mismatch at {np.argmax(got != mirror)}"
    r = ref[a, b]
    fin = np.isfinite(r)
    assert np.array_equal(np.isfinite(got), fin)
    rel = np.abs(got[fin].astype(np.float64) - r[fin]) / np.maximum(r[fin], 1e-300)
    rel[r[fin] == 0] = np.abs(got[fin][r[fin] == 0])
    assert rel.max(initial=0) <= RTOL, rel.max()
    return rel.max(initial=0)


@pytest.mark.parametrize("w", [128, 12])
def test_small_random_walk_all_pairs(w):
    # 50 series of length 128, seed 0: all 1225 pairs
    values, offsets = synth.random_walk_set(50, 128, seed=0)
    _check_matrix(values, offsets, w)


def test_integer_inputs_exact():
    values, offsets = synth.integer_set(24, 37, seed=3)
    v, o = _dev(values, offsets)
    for w in (0, 1, 5, -1):
        D = api.dtw_pairwise(v, o, w).cpu().numpy().astype(np.float64)
        assert np.array_equal(D, oracle.pairwise(values, offsets, w))


@pytest.mark.parametrize("L,w", [(1, 0), (2, 0), (7, 3), (13, 6), (26, 12), (27, 13), (52, 25),
                                 (103, 51), (104, 51), (105, 52), (97, 0), (64, 200), (255, 127),
                                 (256, 127), (129, 64), (8, 2)])
def test_edge_shapes_equal_lengths(L, w):
    values, offsets, _ = synth.five_class_set(9, L, seed=L * 7 + w)
    _check_matrix(values, offsets, w)


@pytest.mark.parametrize("strict", [False, True])
def test_ragged_lengths(strict):
    lens = synth.ragged_lengths(30, 20, 90, seed=9)
    values, offsets, _ = synth.five_class_set(30, lens, seed=9)
    for w in (4, 9, 30):
        _check_matrix(values, offsets, w, strict)


def test_packed_output_matches_full():
    values, offsets, _ = synth.five_class_set(40, 64, seed=2)
    v, o = _dev(values, offsets)
    full = api.dtw_pairwise(v, o, 6)
    packed = api.dtw_pairwise(v, o, 6, packed=True)
    a, b = np.triu_indices(40, 1)
    assert torch.equal(packed.cpu(), full.cpu()[a, b])


def test_single_series_and_pair():
    values, offsets = synth.random_walk_set(1, 10, seed=1)
    v, o = _dev(values, offsets)
    assert api.dtw_pairwise(v, o, 3).cpu().numpy().tolist() == [[0.0]]
    values, offsets = synth.random_walk_set(2, 10, seed=1)
    _check_matrix(values, offsets, 3)


def test_host_io_equals_device_path():
    values, offsets, _ = synth.five_class_set(20, 80, seed=4)
    v, o = _dev(values, offsets)
    dev = api.dtw_pairwise(v, o, 8).cpu().numpy()
    host = api.dtw_pairwise_host(values, offsets, 8)
    assert np.array_equal(dev, host)


def test_query_row():
    lens = synth.ragged_lengths(25, 30, 70, seed=12)
    values, offsets, _ = synth.five_class_set(25, lens, seed=12)
    q = synth.five_class_set(1, 50, seed=13)[0]
    v, o = _dev(values, offsets)
    for w in (5, -1):
        got = api.dtw_query(torch.from_numpy(q).cuda(), v, o, w).cpu().numpy()
        ref = oracle.query(q, values, offsets, w)
        assert np.max(np.abs(got - ref) / ref) <= RTOL
        # the query row equals the row of the matrix of the set with q prepended
        ext_v = np.concatenate([q, values])
        ext_o = np.concatenate([[0], offsets + len(q)])
        D = api.dtw_pairwise(*_dev(ext_v, ext_o), w).cpu().numpy()
        assert np.array_equal(D[0, 1:], got)


def test_argument_errors():
    values, offsets = synth.random_walk_set(4, 10, seed=1)
    v, o = _dev(values, offsets)
    bad = o.clone()
    bad[2] = bad[1]  # empty series
    with pytest.raises(api.DTWError) as e:
        api.dtw_pairwise(v, bad, 3)
    assert e.value.code == api.DTW_EINVAL
    nan_v = v.clone()
    nan_v[5] = float("nan")
    with pytest.raises(api.DTWError) as e:
        api.dtw_pairwise(nan_v, o, 3, check_finite=True)
    assert e.value.code == api.DTW_EINVAL
    with pytest.raises(api.DTWError) as e:
        api.dtw_pairwise(v, o.to(torch.int32).to(torch.int64).flip(0).contiguous(), 3)
    assert e.value.code == api.DTW_EINVAL


def test_large_config_all_pairs(c1_matrix):
    """2000 series of length 512 (five classes), w = 51: the benchmark workload, computed in
    the benchmark's launch configuration.  Every one of the 1,999,000 pairs equals the
    oracle's float mirror bit for bit and the float64 oracle within 1e-5 relative."""
    c = c1_matrix
    Dc, a, b = c["D"], c["a"], c["b"]
    assert np.all(np.diag(Dc) == 0)
    assert np.array_equal(Dc, Dc.T)
    got = Dc[a, b]
    bad = np.flatnonzero(got.view(np.uint32) != c["mirror"].view(np.uint32))
    assert bad.size == 0, f"{bad.size} pairs differ from the float mirror, first {(a[bad[0]], b[bad[0]])}"
    rel = np.abs(got.astype(np.float64) - c["ref"]) / c["ref"]
    assert rel.max() <= RTOL, rel.max()
    assert got.min() > 0  # no two series of the set are identical


# ---------------------------------------------------------------- wide bands (strip kernel)


@pytest.mark.parametrize("L,w", [(600, -1), (300, 200), (257, 129), (1000, 400)])
def test_wide_band_equal_lengths(L, w):
    values, offsets, _ = synth.five_class_set(7, L, seed=L + w)
    _check_matrix(values, offsets, w)


@pytest.mark.parametrize("strict", [False, True])
def test_wide_band_ragged(strict):
    lens = synth.ragged_lengths(20, 64, 900, seed=21)
    values, offsets, _ = synth.five_class_set(20, lens, seed=21)
    for w in (20, 300):
        _check_matrix(values, offsets, w, strict)


@pytest.mark.parametrize("shape", ["strip:4", "strip:8", "strip:16", "rot:16:32", "rot:13:8:2",
                                   "rot:8:16", "rot:8:8", "rot:8:8:2", "rot:10:8", "rot:20:4",
                                   "rot:13:16", "rot:20:8", "rot:12:8", "rot:18:4", "rot:12:16",
                                   "rot:9:8", "rot:15:8", "rot:17:4", "rot:23:4", "rot:11:16",
                                   "two:6:8", "two:8:8", "two:10:8", "two:6:16", "two:10:4"])
def test_forced_shapes_agree(shape, monkeypatch):
    # every kernel shape computes the same float values (both band edges cross the strips)
    lens = synth.ragged_lengths(16, 100, 140, seed=31)
    values, offsets, _ = synth.five_class_set(16, lens, seed=31)
    monkeypatch.setenv("DTWGB_SHAPE", shape)
    _check_matrix(values, offsets, 30)
    q = synth.five_class_set(1, 145, seed=32)[0]
    got = api.dtw_query(torch.from_numpy(q).cuda(), *_dev(values, offsets), 30).cpu().numpy()
    mir = np.array([oracle.dtw_f32_mirror(q, values[offsets[i]:offsets[i + 1]], 30)
                    for i in range(16)], dtype=np.float32)
    assert np.array_equal(got.view(np.uint32), mir.view(np.uint32))


def test_ragged_long_sample():
    """Ragged set with lengths in [64, 2048] (the batched-ragged workload's length mix), band
    5 % of the longest series widened per pair to |n-m|: sampled pairs vs the oracle."""
    lens = synth.ragged_lengths(120, 64, 2048, seed=2)
    values, offsets, _ = synth.five_class_set(120, lens, seed=2)
    v, o = _dev(values, offsets)
    D = api.dtw_pairwise(v, o, 102).cpu().numpy()
    assert np.array_equal(D, D.T) and np.all(np.diag(D) == 0)
    rng = np.random.default_rng(5)
    a = rng.integers(0, 120, 300)
    b = rng.integers(0, 120, 300)
    keep = a != b
    a, b = a[keep], b[keep]
    mir = oracle.pairs_f32_mirror(values, offsets, a, b, 102)
    ref = oracle.pairs(values, offsets, a, b, 102)
    got = D[a, b]
    assert np.array_equal(got.view(np.uint32), mir.view(np.uint32))
    assert (np.abs(got - ref) / ref).max() <= RTOL


@pytest.mark.parametrize("shape", ["strip:4", "strip:8", "strip:16"])
def test_strip_starting_inside_the_matrix(shape, monkeypatch):
    """Very unequal lengths with the band widened to |n-m|: later strips start below
    row 1, so the first row of lanes 1.. has out-of-band upper predecessors."""
    rng = np.random.default_rng(77)
    x = rng.standard_normal(80).astype(np.float32)
    y = rng.standard_normal(394).astype(np.float32)
    vv = np.concatenate([x, y])
    oo = np.array([0, 80, 474], dtype=np.int64)
    monkeypatch.setenv("DTWGB_SHAPE", shape)
    for w in (19, 320, 393):
        D = api.dtw_pairwise(*_dev(vv, oo), w).cpu().numpy()
        assert D[0, 1] == oracle.dtw_f32_mirror(x, y, w)
    _check_matrix(*synth.five_class_set(6, synth.ragged_lengths(6, 40, 700, seed=8), seed=8)[:2], 10)


@pytest.mark.parametrize("shape", ["strip:4", "strip:8", "strip:16"])
def test_strip_shapes_on_tile_boundary_lengths(shape, monkeypatch):
    """Each column-strip width on lengths at and around its tile sizes (1, 2, 31-33, K-slot
    lane widths, 32K strip widths) and up to 2048, band 5 % of the longer series widened to
    |n-m| (so the band edges cross most strips, at every phase): every pair is bitwise the
    float mirror."""
    lens = np.array([1, 2, 3, 31, 32, 33, 127, 128, 129, 255, 256, 257, 511, 512, 513, 700,
                     1023, 1024, 1500, 2048], dtype=np.int64)
    values, offsets, _ = synth.five_class_set(len(lens), lens, seed=91)
    monkeypatch.setenv("DTWGB_SHAPE", shape)
    v, o = _dev(values, offsets)
    D = api.dtw_pairwise(v, o, 50, permille=True).cpu().numpy()
    a, b = np.triu_indices(len(lens), 1)
    hi = np.maximum(lens[a], lens[b])
    w = np.minimum(np.maximum(hi * 50 // 1000, np.abs(lens[a] - lens[b])), hi - 1)
    mir = oracle.pairs_w_f32_mirror(values, offsets, a, b, w)
    got = D[a, b]
    assert np.array_equal(got.view(np.uint32), mir.view(np.uint32)), \
        (a[np.argmax(got != mir)], b[np.argmax(got != mir)])
    assert np.array_equal(D, D.T) and np.all(np.diag(D) == 0)


def test_window_permille_flag():
    """DTW_WINDOW_PERMILLE: each pair's band is floor(window * max(n, m) / 1000)."""
    lens = synth.ragged_lengths(25, 50, 600, seed=41)
    values, offsets, _ = synth.five_class_set(25, lens, seed=41)
    v, o = _dev(values, offsets)
    for pm, strict in ((50, False), (200, True), (0, False)):
        D = api.dtw_pairwise(v, o, pm, permille=True, strict=strict).cpu().numpy()
        a, b = np.triu_indices(25, 1)
        w = np.maximum(lens[a], lens[b]) * pm // 1000
        ref = oracle.pairs_w(values, offsets, a, b, w, strict)
        got = D[a, b].astype(np.float64)
        fin = np.isfinite(ref)
        assert np.array_equal(np.isfinite(got), fin)
        assert np.max(np.abs(got[fin] - ref[fin]) / ref[fin]) <= RTOL


@pytest.mark.parametrize("L,w", [(300, 38), (400, 51), (520, 76), (700, 102), (640, 159), (450, 45),
                                 (580, 58), (700, 70), (830, 89), (950, 95), (640, 64), (830, 83),
                                 (900, 90), (1100, 110), (1300, 130)])
def test_band_widths_of_every_tail_kind(L, w):
    # the automatic shape of each width (masked tails of 1, 4 and K slots, K = 10 and 20)
    # gives the float mirror's bits
    values, offsets, _ = synth.five_class_set(10, L, seed=L + w)
    _check_matrix(values, offsets, w)


@pytest.mark.parametrize("lo,hi,w", [(100, 151, 5), (30, 69, 5), (40, 90, 5), (50, 88, 5)])
def test_ragged_sets_whose_widest_band_fills_the_lanes(lo, hi, w):
    # the widest band of the set, 2 (hi - lo) + 1 cells, fills a shape's slots to within one
    # (13 x 8, 20 x 4) or a few (13 x 8, 10 x 8); pairs of closer lengths have narrower bands
    # whose cells beyond the band a short masked tail would leave unmasked
    lens = np.array(synth.ragged_lengths(14, lo, hi, seed=lo))
    lens[0], lens[1] = lo, hi
    values, offsets, _ = synth.five_class_set(14, lens, seed=lo)
    _check_matrix(values, offsets, w)
    q = synth.five_class_set(1, (lo + hi) // 2, seed=hi)[0]
    got = api.dtw_query(torch.from_numpy(q).cuda(), *_dev(values, offsets), w).cpu().numpy()
    mir = np.array([oracle.dtw_f32_mirror(q, values[offsets[i]:offsets[i + 1]], w)
                    for i in range(14)], dtype=np.float32)
    assert np.array_equal(got.view(np.uint32), mir.view(np.uint32))


@pytest.mark.parametrize("shape,L,w", [("two:13:4", 512, 51), ("two:13:4", 300, 51),
                                       ("two:12:4", 400, 47), ("two:16:4", 640, 63),
                                       ("two:8:8", 520, 63), ("two:6:8", 200, 47),
                                       ("two:10:8", 700, 79), ("two:16:8", 900, 126),
                                       ("two:12:8", 450, 94), ("two:13:8", 330, 102)])
def test_two_row_shapes_of_one_length(shape, L, w, monkeypatch):
    # the two-row kernel with the masked tails of one-length sets (1 or 4 slots of the
    # upper half) gives the float mirror's bits, for the matrix and for a query
    values, offsets, _ = synth.five_class_set(11, L, seed=L + 3 * w)
    monkeypatch.setenv("DTWGB_SHAPE", shape)
    _check_matrix(values, offsets, w)
    q = synth.five_class_set(1, L, seed=L + 3 * w + 1)[0]
    got = api.dtw_query(torch.from_numpy(q).cuda(), *_dev(values, offsets), w).cpu().numpy()
    mir = np.array([oracle.dtw_f32_mirror(q, values[offsets[i]:offsets[i + 1]], w)
                    for i in range(11)], dtype=np.float32)
    assert np.array_equal(got.view(np.uint32), mir.view(np.uint32))


@pytest.mark.parametrize("shape,L,w", [("three:9:4", 512, 51), ("three:9:4", 300, 51),
                                       ("three:5:4", 256, 29), ("three:11:4", 600, 65),
                                       ("three:7:8", 700, 83), ("three:6:8", 480, 71),
                                       ("three:10:2", 200, 29), ("three:8:4", 400, 46),
                                       ("three:9:8", 800, 106), ("three:9:2", 256, 25)])
def test_three_row_shapes_of_one_length(shape, L, w, monkeypatch):
    # the three-row kernel (masked tails of 1, 4 and 8 slots of the last part) gives the
    # float mirror's bits, for the matrix and for a query
    values, offsets, _ = synth.five_class_set(11, L, seed=L + 5 * w)
    monkeypatch.setenv("DTWGB_SHAPE", shape)
    assert api.describe_shape(L, L, w).startswith("dtw_multirow_kernel<R=3")
    _check_matrix(values, offsets, w)
    q = synth.five_class_set(1, L, seed=L + 5 * w + 1)[0]
    got = api.dtw_query(torch.from_numpy(q).cuda(), *_dev(values, offsets), w).cpu().numpy()
    mir = np.array([oracle.dtw_f32_mirror(q, values[offsets[i]:offsets[i + 1]], w)
                    for i in range(11)], dtype=np.float32)
    assert np.array_equal(got.view(np.uint32), mir.view(np.uint32))
