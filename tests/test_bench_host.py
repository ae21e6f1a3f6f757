"""Host logic of bench.py's roofline accounting (no GPU): algorithmic bytes per launch and per
right-hand side of each timed kernel group, and the rule that a committed DRAM-traffic figure
is used only while its kernel source is unchanged."""
import hashlib
import json
import os

import bench


def test_algorithmic_bytes():
    N, nX, ncut = 128 ** 3, 279550, 810004
    geo = N * 6  # phase code (2 B) and voxel scale (4 B)
    assert bench.algorithmic_bytes("apply_uncut_f32", N, nX, ncut, True) == (0, 72 * N + geo)
    assert bench.algorithmic_bytes("prec_f32", N, nX, ncut, True) == (0, 48 * (N + nX))
    # on-the-fly cut tets (the default): per launch each cut tet's record (68 reals) and 9 ints;
    # per right-hand side 72 B per enriched node (d read, q updated)
    assert bench.algorithmic_bytes("apply_cut_f32", N, nX, ncut, True) == (308 * ncut, 72 * nX)
    assert bench.algorithmic_bytes("apply_cut_f64", N, nX, ncut, True) == (580 * ncut, 144 * nX)
    # cached matrices: 1232 B per cut tet and launch, 72 B per enriched node and right-hand side
    assert bench.algorithmic_bytes("apply_cut_f32", N, nX, ncut, True, cut_cache=True) == (1232 * ncut, 72 * nX)
    assert bench.algorithmic_bytes("no_such_group", N, nX, ncut, True) is None


def test_traffic_is_used_only_for_the_captured_source(tmp_path, monkeypatch):
    src_dir = tmp_path / "paper_2601_02172_gb300" / "csrc"
    src_dir.mkdir(parents=True)
    (src_dir / "k.cu").write_text("kernel v1")
    sha = hashlib.sha256(b"kernel v1").hexdigest()[:16]
    (tmp_path / "profiles").mkdir()
    entry = {"kernels": ["k"], "source": "k.cu", "source_sha": sha, "dram_bytes_per_rhs": 123.0}
    (tmp_path / "profiles" / "traffic.json").write_text(json.dumps({"grp": entry}))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.traffic_for("grp")["dram_bytes_per_rhs"] == 123.0
    assert bench.traffic_for("other") is None
    (src_dir / "k.cu").write_text("kernel v2")  # the kernel changed since the capture
    assert bench.traffic_for("grp") is None
    # several source files: the sha covers them in order
    (src_dir / "h.cuh").write_text("header v1")
    sha2 = hashlib.sha256(b"kernel v2" + b"header v1").hexdigest()[:16]
    entry2 = {"kernels": ["k"], "source": ["k.cu", "h.cuh"], "source_sha": sha2, "dram_bytes_per_rhs": 7.0}
    (tmp_path / "profiles" / "traffic.json").write_text(json.dumps({"grp": entry2}))
    assert bench.traffic_for("grp")["dram_bytes_per_rhs"] == 7.0
    (src_dir / "h.cuh").write_text("header v2")
    assert bench.traffic_for("grp") is None


def test_committed_traffic_entries_name_existing_sources():
    d = json.load(open(os.path.join(bench.ROOT, "profiles", "traffic.json")))
    for k, ent in d.items():
        if k.startswith("_"):
            continue
        srcs = ent["source"] if isinstance(ent["source"], list) else [ent["source"]]
        for f in srcs:
            assert os.path.exists(os.path.join(bench.ROOT, "paper_2601_02172_gb300", "csrc", f)), k
