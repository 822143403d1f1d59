"""Host logic of bench.py: image sets of every workload, sampling of image ids, workload labels (no GPU)."""
import importlib.util
import os

import numpy as np
import pytest

import blinksynth as bs

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def bench():
    spec = importlib.util.spec_from_file_location("bench_mod", os.path.join(ROOT, "bench.py"))
    m = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(m)
    return m


@pytest.mark.parametrize("name", ["tiny", "coarse", "precision", "uneven", "fullband"])
def test_image_sets_cover_every_image_once(bench, name):
    w = bs.WORKLOADS[name]
    ns = w.samples_per_chunk
    sets = bench.image_sets({"sets": w.sets()}, w, ns)
    # packed per set, contiguous, one image per (integration, output channel)
    assert sum(c for _, _, c, _ in sets) == (ns // w.samples_per_int) * w.n_out_chan
    first = 0
    for st, f, c, side in sets:
        assert f == first and side == st.n_pix and c == (ns // w.samples_per_int) * (st.n_fine // w.chan_avg)
        first += c
    if name == "uneven":
        assert [s for _, _, _, s in sets] == [256, 512, 1024, 512]


def test_pick_images_spreads_over_sets_and_stays_in_range(bench):
    w = bs.WORKLOADS["uneven"]
    sets = bench.image_sets({"sets": w.sets()}, w, w.samples_per_chunk)
    picks = bench.pick_images(sets, 64)
    assert {q for q, _ in picks} == set(range(len(sets)))
    for q, i in picks:
        assert 0 <= i < sets[q][2]
    assert len(picks) == len(set(picks))
    # one image: one pick
    one = bench.image_sets({"sets": bs.WORKLOADS["tiny"].sets()}, bs.WORKLOADS["tiny"], 10)
    assert bench.pick_images(one, 16) == [(0, 0)]


def test_sample_ids_are_sorted_unique_and_cover_both_ends(bench):
    ids = bench.oracle_sample_ids(38400, 64)
    assert ids[0] == 0 and ids[-1] == 38399 and np.all(np.diff(ids) > 0)


def test_workload_labels(bench):
    assert "38,400" not in bench.workload_label("fullband", bs.WORKLOADS["fullband"])
    assert bench.workload_label("fullband", bs.WORKLOADS["fullband"]).startswith("fullband: 50 ms chunk, 144 tiles")
    assert bench.workload_label("uneven", bs.WORKLOADS["uneven"]).startswith("uneven: 144 tiles")


def test_calibration_generators_are_seeded_and_shaped(bench):
    g1, g2 = bench.bench_gains(8, 16), bench.bench_gains(8, 16)
    assert g1.shape == (8, 16, 2) and g1.dtype == np.complex64 and np.array_equal(g1, g2)
    assert 0.5 <= np.abs(g1).min() and np.abs(g1).max() <= 1.5
    J = bench.bench_jones(8, 16)
    assert J.shape == (8, 16, 2, 2) and np.array_equal(J, bench.bench_jones(8, 16))


def test_oracle_images_of_picked_sets_use_each_sets_calibration(bench):
    # the per-set slice of a call-wide calibration array reaches the oracle: the picked images equal direct
    # oracle calls on each set with its own channels, flags and gains
    import oracle
    w = bs.WORKLOADS["uneven"]
    inp = bs.build_workload("uneven", n_samples=10)
    small = [type(st)(fine0=st.fine0, n_fine=2, n_pix=64, flags=st.flags) for st in inp["sets"]]
    inp = dict(inp, sets=small)
    sets = bench.image_sets(inp, w, 10)
    gains = bench.bench_gains(w.n_fine // w.chan_avg, w.n_tiles)
    picks = [(0, 1), (2, 0), (3, 1)]
    got = bench.oracle_sets_images(oracle, inp, w, sets, picks, 2, gains)
    for (q, i), img in zip(picks, got):
        st = small[q]
        ref = oracle.pipeline(inp["volt"], inp["enu"], inp["freqs"], w.samples_per_int, w.chan_avg, 64,
                              ids=np.array([i]), flags=st.flags, fine0=st.fine0, n_fine=st.n_fine,
                              gains=gains[st.fine0:st.fine0 + st.n_fine].astype(np.complex128))["images"][0]
        assert np.array_equal(img, ref)


def test_oracle_images_of_picked_sets_use_the_kernel(bench):
    import oracle
    w = bs.WORKLOADS["tiny"]
    inp = bs.build_workload("tiny")
    sets = bench.image_sets(inp, w, 10)
    st = sets[0][0]
    inp = dict(inp, sets=[type(st)(fine0=st.fine0, n_fine=st.n_fine, n_pix=64, flags=st.flags)])
    sets = bench.image_sets(inp, w, 10)
    got = bench.oracle_sets_images(oracle, inp, w, sets, [(0, 0)], 1, None, 4)[0]
    ref = oracle.pipeline(inp["volt"], inp["enu"], inp["freqs"], 10, 1, 64, support=4)["images"][0]
    assert np.array_equal(got, ref)
    assert not np.array_equal(got, oracle.pipeline(inp["volt"], inp["enu"], inp["freqs"], 10, 1, 64)["images"][0])
