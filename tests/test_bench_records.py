"""bench.py's stored DRAM-traffic records: the default workload's record must
belong to the tensor-core kernel source as it stands (a kernel change without a
new capture would silently report traffic as unmeasured), and the source hash
must ignore comments and white space only."""
import bench


def test_default_workload_traffic_record_matches_the_kernel_source():
    key = f"{bench._source_hash()}:fhn3d_256:f16x10"
    assert key in bench.NCU_TRAFFIC, (key, sorted(bench.NCU_TRAFFIC))
    # mean DRAM bytes per k_mode_tc launch at 256^3: near the 1.82 GB the
    # launches must move (operand planes once, outputs once), never far above
    assert 1.5e9 < bench.NCU_TRAFFIC[key] < 2.0e9


def test_source_hash_ignores_comments_and_spacing(tmp_path, monkeypatch):
    src_dir = tmp_path / "paper_2310_07551_gb300" / "csrc"
    src_dir.mkdir(parents=True)
    code = "int f(int a) { return a + 1; }\n// Pointwise kernels of the split-BF16 step.\nint g;\n"
    (src_dir / "tc.cu").write_text(code)
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    h0 = bench._source_hash()
    (src_dir / "tc.cu").write_text("// note\nint f(int a)  {\n  return a + 1; /* c */ }\n"
                                   "// Pointwise kernels of the split-BF16 step.\nint g2;\n")
    assert bench._source_hash() == h0          # comments, spacing, and code after the cut
    (src_dir / "tc.cu").write_text(code.replace("a + 1", "a + 2"))
    assert bench._source_hash() != h0
