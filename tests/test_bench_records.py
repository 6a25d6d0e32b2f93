"""bench.py's recorded DRAM traffic (profiles/force_kernel_traffic.txt) is
used only for the workload, launch shape and force-kernel sources it was
measured on; the source hash ignores comments and blank space."""
import os
import shutil
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import bench  # noqa: E402

FORMS = {"x1": "scalar f32", "x2": "paired f32x2", "xe": "entry-paired f32x2"}


def _launch(shape):
    """The bench line's launch record for a record's 'R,W,T,form' key."""
    R, W, T, form = shape.split(",")
    return {"sinks_per_thread": int(R), "warps_per_group": int(W), "tile_j": int(T), "arith": FORMS[form]}


def _records():
    recs, rec = [], {}
    with open(os.path.join(ROOT, "profiles", "force_kernel_traffic.txt")) as f:
        for line in f:
            if not line.strip():
                if rec:
                    recs.append(rec)
                rec = {}
            elif "=" in line and not line.lstrip().startswith("#"):
                k, v = line.split("=", 1)
                rec[k.strip()] = v.strip()
    if rec:
        recs.append(rec)
    return recs


def test_a_record_is_used_only_for_its_workload_shape_and_sources(monkeypatch):
    recs = _records()
    assert recs and all({"workload", "launch", "kernel_hash", "bytes_per_launch"} <= set(r) for r in recs)
    r = recs[0]
    launch = _launch(r["launch"])
    other_form = "scalar f32" if launch["arith"] != "scalar f32" else "entry-paired f32x2"
    monkeypatch.setattr(bench, "kernel_hash", lambda: r["kernel_hash"])
    assert bench._recorded_traffic(r["workload"], launch) == float(r["bytes_per_launch"])
    assert bench._recorded_traffic("plummer_4m", launch) is None            # another workload
    assert bench._recorded_traffic(r["workload"], dict(launch, tile_j=1024)) is None   # another shape
    assert bench._recorded_traffic(r["workload"], dict(launch, arith=other_form)) is None   # another form
    monkeypatch.setattr(bench, "kernel_hash", lambda: "0" * 12)
    assert bench._recorded_traffic(r["workload"], launch) is None            # other sources


def test_the_source_hash_ignores_comments_but_not_code(tmp_path, monkeypatch):
    csrc = tmp_path / "paper_1812_07313_gb300" / "csrc"
    csrc.mkdir(parents=True)
    for f in bench.KERNEL_SOURCES:
        shutil.copy(os.path.join(ROOT, "paper_1812_07313_gb300", "csrc", f), csrc / f)
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    h0 = bench.kernel_hash()
    assert len(h0) == 12
    f = csrc / bench.KERNEL_SOURCES[0]
    text = f.read_text()
    f.write_text("// a new comment line\n" + text.replace("\n", "\n\n", 3) + "\n/* and a block comment */\n")
    assert bench.kernel_hash() == h0
    f.write_text(text.replace("#pragma once", "#pragma once\nstatic const int qg_unused_marker = 1;", 1))
    assert bench.kernel_hash() != h0
