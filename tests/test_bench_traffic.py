"""bench.py's `roofline.traffic`: the DRAM bytes of a committed ncu capture,
scaled to the bench launch by its point-slices, reported only while the fine
kernel's own code hashes to the capture's source hash.  Edits elsewhere in
heat2d.cu (other kernels, host code) keep the figure; an edit to the fine
kernel's body or launch code drops it to null."""
import json
import os
import shutil

import pytest

import bench

UNITS = 8 * 512 * 128 * 128


def _copy_sources(tmp_path):
    out = []
    for p in bench.FINE_SRCS:
        q = tmp_path / os.path.basename(p)
        shutil.copy(p, q)
        out.append(str(q))
    return out


def _traffic_file(tmp_path, sha):
    t = {"k_heat2d_fine<ff>": {"dram_bytes": 1000, "units": 10, "source_sha": sha}}
    f = tmp_path / "traffic.json"
    f.write_text(json.dumps(t))
    return str(f)


@pytest.mark.parametrize("kernel,base", [("k_heat2d_split", "k_heat2d_split"),
                                         ("k_heat2d_fine<float>", "k_heat2d_fine")])
def test_committed_figure_follows_the_hash(kernel, base):
    t = json.load(open(bench.TRAFFIC))[kernel]
    got = bench.traffic_for(kernel, UNITS)
    if bench.src_hash(bench.FINE_SRCS, base) == t["source_sha"]:
        assert got == t["dram_bytes"] * UNITS / t["units"]
    else:
        assert got is None


def test_the_split_kernel_has_its_own_hash(tmp_path, monkeypatch):
    """An edit to the split kernel drops its figure and keeps the FP32 one."""
    srcs = _copy_sources(tmp_path)
    monkeypatch.setattr(bench, "FINE_SRCS", srcs)
    t = {"k_heat2d_split": {"dram_bytes": 10, "units": 1, "source_sha": bench.src_hash(srcs, "k_heat2d_split")},
         "k_heat2d_fine<float>": {"dram_bytes": 10, "units": 1, "source_sha": bench.src_hash(srcs)}}
    f = tmp_path / "traffic.json"
    f.write_text(json.dumps(t))
    monkeypatch.setattr(bench, "TRAFFIC", str(f))
    assert bench.traffic_for("k_heat2d_split", 2) == 20
    heat2d = next(p for p in srcs if p.endswith("heat2d.cu"))
    text = open(heat2d).read()
    marker = "k_heat2d_split(Heat2dArgs a) {"
    open(heat2d, "w").write(text.replace(marker, marker + "\n    // edited", 1))
    assert bench.traffic_for("k_heat2d_split", 2) is None
    assert bench.traffic_for("k_heat2d_fine<float>", 2) == 20


def test_edits_outside_the_fine_kernel_keep_the_figure(tmp_path, monkeypatch):
    srcs = _copy_sources(tmp_path)
    monkeypatch.setattr(bench, "FINE_SRCS", srcs)
    monkeypatch.setattr(bench, "TRAFFIC", _traffic_file(tmp_path, bench.src_hash(srcs)))
    assert bench.traffic_for("k_heat2d_fine<ff>", 20) == 2000
    heat2d = next(p for p in srcs if p.endswith("heat2d.cu"))
    with open(heat2d, "a") as f:
        f.write("\n// a host-side edit after the fine kernel\n")
    assert bench.traffic_for("k_heat2d_fine<ff>", 20) == 2000
    assert bench.traffic_for("k_heat2d_fine<float>", 20) is None   # no entry


def test_an_edit_in_the_fine_kernel_drops_the_figure(tmp_path, monkeypatch):
    srcs = _copy_sources(tmp_path)
    monkeypatch.setattr(bench, "FINE_SRCS", srcs)
    monkeypatch.setattr(bench, "TRAFFIC", _traffic_file(tmp_path, bench.src_hash(srcs)))
    heat2d = next(p for p in srcs if p.endswith("heat2d.cu"))
    text = open(heat2d).read()
    body = bench._fine_kernel_source(text)
    assert "k_heat2d_fine" in body
    marker = "template <class V, int RX, int RY, bool CL>"
    open(heat2d, "w").write(text.replace(marker, marker + "\n// edited", 1))
    assert bench.traffic_for("k_heat2d_fine<ff>", 20) is None
