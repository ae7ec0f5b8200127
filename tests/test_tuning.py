"""The stored autotune table (host logic only; no GPU)."""
import json

from paper_2410_22686_gb300 import capi, tuning


def test_fields_match_the_c_struct():
    assert tuple(f for f, _ in capi.pc_tiles._fields_) == tuning.FIELDS


def test_key_normalises_precision_aliases():
    assert tuning.key(2, 255, 256, "fp32") == tuning.key(2, 255, 256, "mixed") == "2d_m255_n256_mixed"
    assert tuning.key(3, 63, 128, "bf16s") == "3d_m63_n128_bf16s"
    assert tuning.key(2, 255, 256, "fp32", "fst") == "2d_m255_n256_mixed_fst"
    assert tuning.key(2, 255, 256, "fp64", "mg") == "2d_m255_n256_fp64"


def test_lookup_reads_entries(tmp_path, monkeypatch):
    path = tmp_path / "t.json"
    path.write_text(json.dumps({"entries": {"2d_m15_n16_fp64": {"mg_cx": 8, "mg_ctas": 4, "mv_tj": 16,
                                                                  "pro_pch": 2, "fft_stream": 1, "mg_march": 1,
                                                                  "mg_seg": 8}}}))
    monkeypatch.setattr(tuning, "_cache", tuning.load(str(path)))
    assert tuning.lookup(2, 15, 16, "fp64") == {"mg_cx": 8, "mg_ctas": 4, "mv_tj": 16, "pro_pch": 2,
                                                "fft_stream": 1, "mg_march": 1, "mg_seg": 8}
    assert tuning.lookup(2, 15, 32, "fp64") is None
    assert tuning.lookup(2, 15, 16, "fp64", "fst") is None  # sine-transform shapes are keyed apart


def test_missing_table_is_empty(tmp_path):
    assert tuning.load(str(tmp_path / "none.json")) == {}


def test_workloads_cover_the_bench_shapes():
    keys = {tuning.key(*w) for w in tuning.WORKLOADS}
    for k in ("2d_m255_n256_mixed", "2d_m255_n256_fp64", "2d_m255_n256_bf16s", "3d_m63_n128_mixed",
              "2d_m127_n128_fp64", "2d_m31_n32_fp64_fst", "2d_m255_n256_mixed_fst", "2d_m255_n256_fp64_fst"):
        assert k in keys


def test_stored_table_is_well_formed():
    entries = tuning.load()
    for k, e in entries.items():
        assert set(e) <= set(tuning.FIELDS), k
        assert e["mg_cx"] in (0, 8, 16)
        assert 0 <= e["mg_ctas"] <= 64 and 0 <= e["mv_tj"] <= 4096 and 0 <= e["pro_pch"] <= 64
        assert e["fft_stream"] in (0, 1)
        assert e.get("fst_stream", 0) in (0, 1, 2, 3)


def test_write_missing_tunes_only_the_absent_shapes(tmp_path, monkeypatch):
    """``--write --missing`` keeps the stored entries and tunes only the shapes the table
    lacks (the tuner itself is replaced by a stub: no GPU)."""
    import torch
    path = tmp_path / "t.json"
    keep = {"mg_cx": 8, "mg_ctas": 4, "mv_tj": 16, "pro_pch": 2, "fft_stream": 1, "mg_march": 0, "mg_seg": 0,
            "fst_stream": 0}
    first = tuning.WORKLOADS[0]
    path.write_text(json.dumps({"entries": {tuning.key(*first): keep}}))
    tuned = []

    def stub(dim, m1, n, precision, spatial, reps):
        tuned.append((dim, m1, n, precision, spatial))
        return {f: 0 for f in tuning.FIELDS}

    monkeypatch.setattr(tuning, "_tune_one", stub)
    monkeypatch.setattr(torch.cuda, "get_device_name", lambda *a: "stub")
    assert tuning.main(["--write", "--missing", "--out", str(path)]) == 0
    entries = tuning.load(str(path))
    assert entries[tuning.key(*first)] == keep
    assert first not in tuned and len(tuned) == len(tuning.WORKLOADS) - 1
    assert set(entries) == {tuning.key(*w) for w in tuning.WORKLOADS}
