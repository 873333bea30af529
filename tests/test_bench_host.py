"""Host arithmetic of bench.py's roofline object (CPU only)."""
import json
import os

import bench

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_algorithmic_bytes_of_the_bulk_step():
    """Bulk grid 512 x 512 x 16 (padded 1024 x 1024 x 32): the x-pass spectrum
    holds 3 components x 16 planes x 512 rows x 513 complex FP32; the tensor
    octant 6 components x 17 x 513 x 513 FP32; fields are 16-byte float4."""
    cfg = dict(nx=512, ny=512, nz=16)
    b = bench.algorithmic_bytes(cfg, (1024, 1024, 32))
    cells = 512 * 512 * 16
    w1 = 3 * 16 * 512 * 513 * 8
    octant = 6 * 17 * 513 * 513 * 4
    assert w1 == 100_859_904 and octant == 107_372_952
    assert b["yz_fused"] == 2 * w1 + octant == 309_092_760
    assert b["x_fwd"] == b["x_inv"] == cells * 16 + w1
    # RK4 stages read/write 64, 96, 96 and 80 bytes per cell (no maps)
    assert b["local_stage"] == cells * 84
    assert bench.algorithmic_bytes(cfg, (1024, 1024, 32), axis_map=True)["local_stage"] == cells * 100


def test_film_spectrum_has_four_tensor_components():
    """One z plane: N_xz = N_yz = 0, so the octant keeps four components."""
    b = bench.algorithmic_bytes(dict(nx=512, ny=128, nz=1), (1024, 256, 1))
    assert b["yz_fused"] == 2 * (3 * 128 * 513 * 8) + 4 * 1 * 129 * 513 * 4


def test_traffic_is_reported_only_for_the_captured_sources(monkeypatch, tmp_path):
    entry = {"dram_bytes_per_launch": 123456, "source_digest": "ab" * 8}
    (tmp_path / "profiles").mkdir()
    (tmp_path / "profiles" / "traffic.json").write_text(json.dumps({"bulk": {"yzq_kernel": entry}}))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    monkeypatch.setattr(bench, "source_digest", lambda kernel=None: entry["source_digest"])
    assert bench.load_traffic("bulk", "yzq_kernel") == entry["dram_bytes_per_launch"]
    monkeypatch.setattr(bench, "source_digest", lambda kernel=None: "0" * 16)
    assert bench.load_traffic("bulk", "yzq_kernel") is None


def test_committed_traffic_entries_name_known_kernels():
    t = json.load(open(os.path.join(ROOT, "profiles", "traffic.json")))
    for wl, entries in t.items():
        if wl.startswith("_"):
            continue
        for kernel, e in entries.items():
            assert kernel in bench.KERNEL_TU and e["dram_bytes_per_launch"] > 0


def test_kernel_digests_cover_their_translation_unit_and_headers_only():
    """A kernel's digest covers the file that defines it and every local
    header it includes (through other headers too), and nothing else."""
    plane = bench.kernel_sources("yzh_kernel")
    for f in ("paper_2602_12242_gb300/csrc/demag_plane.cu", "paper_2602_12242_gb300/csrc/regfft.cuh",
              "paper_2602_12242_gb300/csrc/fft.cuh", "paper_2602_12242_gb300/csrc/bulk.cuh",
              "paper_2602_12242_gb300/csrc/cluster.cuh", "paper_2602_12242_gb300/csrc/common.cuh", "include/mx.h"):
        assert f in plane
    assert not any(f.endswith(("fno.cu", "cnn.cu", "api.cu", "local.cu", "demag_quad.cu")) for f in plane)
    quad = bench.kernel_sources("yzq_kernel")
    assert "paper_2602_12242_gb300/csrc/demag_quad.cu" in quad
    assert not any(f.endswith(("demag_plane.cu", "bulk.cuh")) for f in quad)
    local = bench.kernel_sources("local_kernel")
    assert "paper_2602_12242_gb300/csrc/local.cuh" in local
    assert not any(f.endswith("demag_plane.cu") for f in local)
    assert bench.source_digest("xfk_kernel") == bench.source_digest("yzh_kernel") != bench.source_digest("local_kernel")
    assert bench.source_digest("yzq_kernel") != bench.source_digest("yzh_kernel")


def test_kernel_digest_ignores_comments_and_layout(tmp_path):
    a, b, c = tmp_path / "a.cu", tmp_path / "b.cu", tmp_path / "c.cu"
    a.write_text("int f(int x) {  // doubles\n  return 2 * x; /* the\n result */\n}\n")
    b.write_text("int f(int x) {\n return 2 * x;\n}\n")
    c.write_text("int f(int x) { return 3 * x; }\n")
    assert bench._code_text(str(a)) == bench._code_text(str(b)) != bench._code_text(str(c))


def test_algorithmic_bytes_of_the_fused_stage():
    """The fused inverse-x + local slot counts the spectrum read and the local
    stage without the H_demag write and read (32 B per cell less than the two
    separate kernels)."""
    import bench
    cfg = {"nx": 512, "ny": 512, "nz": 16}
    ab = bench.algorithmic_bytes(cfg, (1024, 1024, 32), axis_map=True)
    nc = 512 * 512 * 16
    assert ab["x_inv"] + ab["local_stage"] - ab["x_inv_local"] == 32 * nc
