"""Host logic of bench.py that needs no GPU: the code-only source digest that keys the committed ncu
summaries, and the reading of a summary's DRAM traffic."""
import os

import bench


def test_source_code_only_drops_comments_and_blank_lines():
    a = "int x = 1;  // one\n\n/* block\n   comment */\nint y = x / 2;\n"
    b = "// header\nint x = 1;\n   \nint y = x / 2;   // half\n"
    assert bench.source_code_only(a) == bench.source_code_only(b) == "int x = 1;\nint y = x / 2;"
    assert bench.source_code_only("int x = 2;") != bench.source_code_only("int x = 1;")


def test_digest_follows_code_not_comments(monkeypatch, tmp_path):
    csrc = tmp_path / "paper_2001_07979_gb300" / "csrc"
    csrc.mkdir(parents=True)
    for f in bench.KERNEL_SOURCES:
        (csrc / f).write_text(f"// {f}\nint {f.replace('.', '_')} = 1;\n")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    d0 = bench.kernel_source_digest()
    (csrc / bench.KERNEL_SOURCES[0]).write_text(f"// another comment\n\nint {bench.KERNEL_SOURCES[0].replace('.', '_')} = 1;"
                                                "  /* trailing */\n")
    assert bench.kernel_source_digest() == d0
    (csrc / bench.KERNEL_SOURCES[0]).write_text("int changed = 2;\n")
    assert bench.kernel_source_digest() != d0


def test_traffic_only_for_matching_digest_and_type(monkeypatch, tmp_path):
    (tmp_path / "profiles").mkdir()
    digest = bench.kernel_source_digest()
    summary = (f"# a capture\nkernel_source_sha256_16 = {digest}\nmsg_dtype = f32\n"
               "dram_bytes_per_frame_later_iteration = 1000\ndram_bytes_per_frame_first_iteration = 10\n")
    (tmp_path / "profiles" / "k.txt").write_text(summary)
    real_root = bench.ROOT
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    monkeypatch.setattr(bench, "kernel_source_digest", lambda: digest)
    # row form: the per-edge kernel runs the iterations after the second; 4 frames of 3 iterations, 2 launches
    assert bench.kernel_traffic([3, 3, 3, 3], 2, "k.txt", "f32", rows=True) == 4 * 1000 / 2
    # per-edge form: first iteration once per frame, later ones after it
    assert bench.kernel_traffic([2, 1], 3, "k.txt", "f32") == (2 * 10 + 1 * 1000) / 3
    assert bench.kernel_traffic([3], 1, "k.txt", "f16", rows=True) is None
    monkeypatch.setattr(bench, "kernel_source_digest", lambda: "0" * 16)
    assert bench.kernel_traffic([3], 1, "k.txt", "f32", rows=True) is None
    assert os.path.isdir(real_root)


def test_fer_upper_bound_is_clopper_pearson():
    # no error in n frames: 1 - 0.05^(1/n), about 3/n (the rule of three)
    assert bench.fer_upper95(0, 8192) == 1.0 - 0.05 ** (1.0 / 8192)
    assert abs(bench.fer_upper95(0, 8192) * 8192 - 3.0) < 0.01
    # k errors: the upper end of the one-sided 95% interval, where P(X <= k) = 0.05 for X ~ Bin(n, p)
    import math
    for k, n in ((1, 100), (5, 2048), (24, 2048)):
        p = bench.fer_upper95(k, n)
        cdf = sum(math.comb(n, i) * p ** i * (1 - p) ** (n - i) for i in range(k + 1))
        assert abs(cdf - 0.05) < 1e-6, (k, n, cdf)
    assert bench.fer_upper95(3, 3) == 1.0
