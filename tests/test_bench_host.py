"""Host logic of bench.py (CPU only): the stated error of a frame against the
oracle, the subsampled scenes used for profiler captures, and the keys under
which committed kernel counters are matched to the current sources."""
import importlib.util
import os

import numpy as np
import pytest

import oracle

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def bench():
    spec = importlib.util.spec_from_file_location("bench_under_test", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def test_code_only_ignores_comments_and_spacing(bench):
    a = "int x = 1; // one\n/* block\n comment */ float y;\n"
    b = "int   x = 1;\n\n float y;  // other words"
    assert bench._code_only(a) == bench._code_only(b) == "int x = 1; float y;"
    assert bench._code_only("int x = 2;") != bench._code_only(a)


def test_kernel_source_sets_exist_and_hash(bench):
    csrc = os.path.join(ROOT, "paper_1309_1114_gb300", "csrc")
    for name, files in bench.KERNEL_SOURCES.items():
        for f in files:
            assert os.path.exists(os.path.join(csrc, f)), (name, f)
        h = bench.source_hash(files)
        assert len(h) == 16 and h == bench.source_hash(tuple(reversed(files)))
    assert bench.source_hash(bench.KERNEL_SOURCES["item_kernel"]) != \
        bench.source_hash(bench.KERNEL_SOURCES["absorb_kernel"])
    assert bench.tile_kernel_name(32, False) == "item_kernel<32, 0>"
    assert bench.tile_kernel_name(64, True) == "item_kernel<64, 1>"


def test_workload_labels_are_distinct(bench):
    labels = [w["label"] for w in bench.WORKLOADS.values()]
    assert len(labels) == len(set(labels))


def test_subsample_keeps_the_camera_and_draws_distinct_particles(bench):
    wl = bench.WORKLOADS["uniform"]
    full = bench.make_scene(wl)
    sub = bench.make_scene(wl, 1000)
    assert sub.n == 1000 and full.n > 1000
    assert sub.cams[0] == full.cams[0]
    # every drawn particle is one of the full set's, none twice
    pairs = set(zip(full.parts["x"].tolist(), full.parts["y"].tolist(), full.parts["z"].tolist()))
    drawn = list(zip(sub.parts["x"].tolist(), sub.parts["y"].tolist(), sub.parts["z"].tolist()))
    assert len(set(drawn)) == 1000 and all(p in pairs for p in drawn)


def test_stated_error_of_the_oracle_image_is_zero_and_a_planted_error_is_seen(bench):
    wl = bench.WORKLOADS["uniform"]
    sc = bench.make_scene(wl)
    cam = sc.cams[0]
    o = oracle.render(sc.parts, sc.palette, cam, {}, nthreads=os.cpu_count() or 1)
    e = bench.stated_error(sc, cam, o, {}, 1e-4)
    assert e["n_pixels"] >= 1024 and e["max_rel"] < 1e-12 and e["within_tol"]
    # one channel of the brightest pixel (always among the picks) off by 1 %
    g = o.copy()
    j, i = np.unravel_index(np.argmax(g.sum(axis=2)), g.shape[:2])
    g[j, i, 0] *= 1.01
    e = bench.stated_error(sc, cam, g, {}, 1e-4)
    assert 0.009 < e["max_rel"] < 0.011 and not e["within_tol"]


def test_committed_counter_entries_are_well_formed(bench):
    """Every entry of profiles/traffic.json names its kernel and workload, its
    positive DRAM bytes per launch, the source files of its kernel, and the
    capture command (one pass of the plain program, then ncu with the clocks
    left alone)."""
    import json
    with open(os.path.join(ROOT, "profiles", "traffic.json")) as f:
        d = json.load(f)
    labels = {w["label"] for w in bench.WORKLOADS.values()}
    assert d
    for key, e in d.items():
        kernel, _, label = key.partition("@")
        assert label in labels, key
        base = kernel.split("<")[0]
        assert base in bench.KERNEL_SOURCES, key
        assert e["dram_bytes_per_launch"] > 0
        assert e["sources"] == ", ".join(bench.KERNEL_SOURCES[base])
        assert len(e["source_hash"]) == 16
        cmd = e["command"]
        assert cmd.startswith("python bench.py") and " && ncu " in cmd
        assert "--clock-control none" in cmd
        if "captured_bytes_per_launch" in e:     # a subsample capture scaled to the full launch
            assert "--subsample" in cmd and e["dram_bytes_per_launch"] > e["captured_bytes_per_launch"]
        lim = e.get("limiter")
        if lim:
            assert os.path.exists(os.path.join(ROOT, lim["profile"]))
