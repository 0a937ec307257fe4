"""Host-side helpers of bench.py (no GPU): warm-up rounding to whole step graphs,
the FP64 flop count taken from the committed instruction counters, and the DRAM
traffic entries that are used only while their source files are unchanged."""
import json
import os
import sys
import types

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_warmup_rounds_up_to_whole_step_graphs():
    ns = types.SimpleNamespace
    # graph length: the rebuild period if even, else twice it (every-step lists: 2)
    assert bench.warmup_steps(ns(warmup=5, rebin=10)) == 10
    assert bench.warmup_steps(ns(warmup=10, rebin=10)) == 10
    assert bench.warmup_steps(ns(warmup=11, rebin=10)) == 20
    assert bench.warmup_steps(ns(warmup=3, rebin=1)) == 4
    assert bench.warmup_steps(ns(warmup=3, rebin=5)) == 10
    assert bench.warmup_steps(ns(warmup=5, rebin=0)) == 6
    for w in range(3, 30):
        for r in range(1, 13):
            n = bench.warmup_steps(ns(warmup=w, rebin=r))
            glen = r if r % 2 == 0 else 2 * r
            assert n >= w and n % glen == 0 and n - w < glen


def test_fp64_flops_come_from_the_committed_counters():
    with open(os.path.join(ROOT, "profiles", "fp64_collide_ops.json")) as fh:
        ent = json.load(fh)["d2q9"]
    pc = ent["per_cell"]
    # the per-cell figures are the captured totals over the lattice
    for k in ("dfma", "dadd", "dmul"):
        assert ent[k] == pc[k] * ent["cells"]
    assert pc["instructions"] == pc["dfma"] + pc["dadd"] + pc["dmul"]
    assert pc["flops"] == 2 * pc["dfma"] + pc["dadd"] + pc["dmul"]
    fl, ceiling, src = bench.collide_fp64_ops(9)
    assert (fl, src) == (pc["flops"], "ncu instruction counts")
    # 2 FP64 instructions per clock per SM at this mix, 152 SMs at 2.07 GHz
    assert abs(ceiling - 2 * fl / pc["instructions"] * 152 * 2.07e9 / 1e12) < 1e-12
    assert bench.collide_fp64_ops(19)[2].endswith("(estimate)")


def test_traffic_entries_follow_their_sources(tmp_path, monkeypatch):
    with open(bench.TRAFFIC_FILE) as fh:
        t = json.load(fh)
    for name in ("k_collide_stream", "k_moments + k_couple"):
        ent = t[name]
        fresh = ent["source_sha"] == bench._src_hash(ent["source"])
        want = ent["dram_bytes_per_launch"] if fresh else None
        assert bench._traffic(name, ent["workload"]) == want
        assert bench._traffic(name, "another-workload") is None
    # an entry whose hash matches the sources is used, a changed source voids it
    cur = {k: dict(v, source_sha=bench._src_hash(v["source"])) for k, v in t.items()
           if isinstance(v, dict)}
    cur["k_collide_stream"]["source_sha"] = "0" * 16
    p = tmp_path / "traffic.json"
    p.write_text(json.dumps(cur))
    monkeypatch.setattr(bench, "TRAFFIC_FILE", str(p))
    assert bench._traffic("k_collide_stream", "c2-fp32") is None
    assert bench._traffic("k_moments + k_couple", "c2-fp32") == \
        t["k_moments + k_couple"]["dram_bytes_per_launch"]
