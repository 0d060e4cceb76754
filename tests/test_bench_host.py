"""bench.py host logic that needs no GPU: the kernel-source digest that ties
the committed ncu traffic figures to the kernels they were taken on, and
the reading of that file."""
import bench


def test_source_code_drops_comments_and_blank_lines():
    src = "int a; // one\n\n/* two\n   lines */ int b;\n  // only a comment\nint c;  /* tail */\n"
    assert bench.source_code(src) == "int a;\n  int b;\nint c;"


def test_digest_ignores_comments_but_not_code(tmp_path, monkeypatch):
    csrc = tmp_path / "paper_2209_01983_gb300" / "csrc"
    csrc.mkdir(parents=True)
    (csrc / "k.cu").write_text("__global__ void k() { int x = 1; }  // first\n")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    d0 = bench.source_digest()
    (csrc / "k.cu").write_text("// a new header comment\n__global__ void k() { int x = 1; }\n")
    assert bench.source_digest() == d0
    (csrc / "k.cu").write_text("__global__ void k() { int x = 2; }\n")
    assert bench.source_digest() != d0


def test_traffic_table_only_for_matching_digest(tmp_path, monkeypatch):
    csrc = tmp_path / "paper_2209_01983_gb300" / "csrc"
    csrc.mkdir(parents=True)
    (csrc / "k.cu").write_text("__global__ void k() {}\n")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    f = tmp_path / "traffic.txt"
    monkeypatch.setattr(bench, "TRAFFIC_FILE", str(f))
    rows = "fp32_mixed mix_nodes node 133.7 140 3\n"
    f.write_text(f"# source-digest: {bench.source_digest()}\n" + rows)
    table, _ = bench.load_traffic()
    assert table == {("fp32_mixed", "mix_nodes"): 133.7}
    f.write_text("# source-digest: 0000000000000000\n" + rows)
    table, note = bench.load_traffic()
    assert table == {} and "changed" in note


def test_oracle_all_cores_replicas():
    # one spawned replica per host core, timed together: at least one core's
    # worth of throughput and no more than cores times the best single rate
    rate, cores, secs = bench.oracle_rate_all_cores(8, 0.1, 3, 1, timeout_s=120)
    single, _, _ = bench.oracle_rate(8, 0.1, 3, 1)
    assert cores >= 1 and secs > 0
    assert 0.2 * single < rate < 4.0 * cores * single
