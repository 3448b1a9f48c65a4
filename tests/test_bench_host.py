"""Host-side arithmetic of the benchmark's roofline entries (no GPU)."""
import bench


def test_fp32_peak_from_unit_counts():
    # 152 SMs x 128 FP32 lanes x 2 FLOP per FMA x 2.070 GHz
    assert abs(bench.FP32_PEAK_TFLOPS - 80.54784) < 1e-9


def test_flop_entry_counts_the_folded_line_operator():
    # per DoF and direction 2n + 5 FLOP; 6D, n = 4: 6 * 13 = 78, + 3 in the stage update
    e = bench.flop_entry(1 << 30, 5.57, 6, 4, True)
    assert e["per_dof"] == 81
    assert abs(e["achieved_tflops"] - 81 * (1 << 30) / 5.57e-3 / 1e12) < 1e-9
    assert abs(e["frac"] - e["achieved_tflops"] / bench.FP32_PEAK_TFLOPS) < 1e-12
    assert bench.flop_entry(1000, 1.0, 4, 3, False)["per_dof"] == 4 * 11


def test_algorithmic_bytes_per_dof():
    b = bench.BYTES_PER_DOF
    assert b["stage_fp32w_fp64u"] == 24 and b["apply_fp32"] == 8 and b["apply_fp64"] == 16


def test_kernel_hash_ignores_comments_only(tmp_path, monkeypatch):
    """The recorded DRAM bytes stay keyed to the stage kernel's code: a comment
    or whitespace edit keeps the hash, a code edit changes it."""
    csrc = tmp_path / "paper_2002_08110_gb300" / "csrc"
    csrc.mkdir(parents=True)
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    monkeypatch.setattr(bench, "KERNEL_SOURCES", ["k.cu"])
    (csrc / "k.cu").write_text("// one\nint f(int x) { return x + 1; }  /* two */\n")
    h0 = bench.kernel_hash()
    (csrc / "k.cu").write_text("// changed comment\nint  f(int x)\n{ return x + 1; }\n/* other\n block */\n")
    assert bench.kernel_hash() == h0
    (csrc / "k.cu").write_text("// one\nint f(int x) { return x + 2; }\n")
    assert bench.kernel_hash() != h0
