"""Host-side helpers of bench.py that need no GPU."""
import bench


def test_code_text_ignores_comments_and_blank_lines_but_not_code():
    a = "int f(int x) {  // the first\n\n  /* a block\n     comment */\n  return x + 1;\n}\n"
    b = "int f(int x) {\n  return x + 1;   // edited comment\n}\n"
    c = "int f(int x) {\n  return x + 2;\n}\n"
    assert bench.code_text(a) == bench.code_text(b) == "int f(int x) {\n  return x + 1;\n}"
    assert bench.code_text(c) != bench.code_text(b)


def test_profiled_traffic_needs_a_matching_source_hash(tmp_path, monkeypatch):
    """A summary whose source_sha256 differs from the current kernel sources
    yields no traffic figure (the counters were taken on other code)."""
    prof = tmp_path / "profiles"
    prof.mkdir()
    good = prof / f"k_{bench.NX}x{bench.NY}_fp32.md"
    good.write_text(f"- dram_bytes_per_launch: 123\n- source_sha256: `{bench.sources_sha()}`\n")
    stale = prof / f"s_{bench.NX}x{bench.NY}_fp32.md"
    stale.write_text("- dram_bytes_per_launch: 456\n- source_sha256: `deadbeef`\n")
    real_sha = bench.sources_sha()
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    monkeypatch.setattr(bench, "sources_sha", lambda: real_sha)
    assert bench.profiled_traffic("k") == 123
    assert bench.profiled_traffic("s") is None
    assert bench.profiled_traffic("missing") is None
