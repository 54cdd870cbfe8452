"""The benchmark's byte model (the roofline's algorithmic bytes) against the
per-pass accounting of the solve: B(N) = 12 N^2 (N+1) c + 2 N^3 r + (N+1)^3 r
per solve; the field solve P1 + P2 + 3 (P3 + P4 + P5); the non-cubic model
equal to the cubic one on a cube.  No GPU."""
import os

import bench


def test_solve_bytes_sum_to_B():
    for N in (32, 256, 512):
        for c, r in ((8, 4), (16, 8)):
            B = 12 * N * N * (N + 1) * c + 2 * N ** 3 * r + (N + 1) ** 3 * r
            assert sum(bench.pass_bytes(N, c, r)) == B


def test_field_bytes():
    pb = bench.pass_bytes(256, 8, 4)
    assert bench.field_bytes(256, 8, 4) == pb[0] + pb[1] + 3 * (pb[2] + pb[3] + pb[4])


def test_noncubic_model_on_a_cube():
    for N in (16, 64):
        assert bench.pass_bytes3((N, N, N), 8, 4) == bench.pass_bytes(N, 8, 4)
    # the 1 x 1 x 2 box has twice the points and one more spectrum plane per z
    a = bench.pass_bytes3((32, 32, 64), 8, 4)
    assert a[0] == 32 * 32 * 64 * 4 + 64 * 32 * 33 * 8


def test_kernel_source_hash_is_stable():
    assert bench.kernel_src_sha() == bench.kernel_src_sha()
    assert len(bench.kernel_src_sha()) == 16


def _ncu_csv(path, launches):
    """A synthetic ncu --csv log: one row per (launch, metric)."""
    hdr = ['"ID"', '"Kernel Name"', '"Metric Name"', '"Metric Unit"', '"Metric Value"']
    rows = [",".join(hdr)]
    for i, (name, t_ns, rd, wr) in enumerate(launches):
        for m, u, v in (("gpu__time_duration.sum", "ns", t_ns), ("dram__bytes_read.sum", "byte", rd),
                        ("dram__bytes_write.sum", "Mbyte", wr / 1e6)):
            rows.append('"%d","%s","%s","%s","%s"' % (i, name, m, u, v))
    with open(path, "w") as f:
        f.write("==PROF== a line ncu writes\n" + "\n".join(rows) + "\n")


def test_summarize_traffic_and_launches(tmp_path):
    import json
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    plan = [("void fsp::k_roots<float>(x)", 6000, 100, 0)]
    passes = ["void fast::k_fast_r2c<float, 8>(a)", "void fast::k_fast_col<float, 16, 0>(a)",
              "void fast::k_fast_col<float, 16, 2>(a)", "void fast::k_fast_col<float, 16, 1>(a)",
              "void fast::k_fast_c2r<float, 8>(a)"]
    launches = plan + [(n, 1000 * (j + 1), 1e6 * (j + 1), 2e6) for _ in range(2) for j, n in enumerate(passes)]
    csv = tmp_path / "t.csv"
    _ncu_csv(csv, launches)
    log = tmp_path / "pc.log"
    log.write_text(json.dumps({"profile_case": "f32", "ok": True, "launches_per_solve": [["f32", 5]]}) + "\n")
    run = [sys.executable, os.path.join(root, "bench.py"), "--n", "8", "--out-dir", str(tmp_path),
           "--ncu-csv", str(csv)]
    subprocess.run(run + ["--summarize", "traffic", "--case-log", str(log)], check=True)
    d = json.loads((tmp_path / "solve_n8_dram_traffic.json").read_text())
    assert d["f32"]["per_launch_bytes"] == [1e6 * (j + 1) + 2e6 for j in range(5)]
    assert d["f32"]["kernels"] == passes
    md = (tmp_path / "solve_n8_dram_traffic.md").read_text()
    assert "| 3 | `void fast::k_fast_col<float, 16, 2>` | 3.0 | 2.0 | 3.0 |" in md
    subprocess.run(run + ["--summarize", "launches"], check=True)
    md = (tmp_path / "bench_n8_launch_list.md").read_text()
    assert "| `void fast::k_fast_col<float, 16, 2>` | 2 | 6.0 |" in md
