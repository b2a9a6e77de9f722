"""Host-side tools of bench.py: the ncu CSV digests (launch-list table,
DRAM traffic record) and the rule that a committed traffic figure applies
only to the workload, precision and kernel sources it was captured on."""

import json
import os

import bench

HDR = ('"ID","Process ID","Process Name","Host Name","Kernel Name","Context","Stream",'
       '"Block Size","Grid Size","Device","CC","Section Name","Metric Name","Metric Unit",'
       '"Metric Value"\n')


def _row(i, kernel, metric, value):
    return (f'"{i}","1","python","h","{kernel}","1","7","(128, 1, 1)","(8, 1, 1)","0","10.3",'
            f'"Command line profiler metrics","{metric}","",'
            f'"{value}"\n')


def _csv(tmp_path, rows):
    p = tmp_path / "x.csv"
    p.write_text("==PROF== Connected\n" + HDR + "".join(rows))
    return str(p)


def test_summarize_launches_shares_rates_and_pipes(tmp_path):
    k1 = "void hz::(anonymous namespace)::slab_factor_fused_kernel<float, 6, 3, 5, 3>(hz::Args)"
    k2 = "op_pair_kernel_c64(hz::Args)"
    rows = [_row(0, k1, "gpu__time_duration.sum", "3,000,000"),
            _row(0, k1, "dram__bytes_read.sum", "3,000,000"),
            _row(0, k1, "sm__pipe_fma_cycles_active.avg.pct_of_peak_sustained_active", "5"),
            _row(1, k2, "gpu__time_duration.sum", "1,000,000"),
            _row(1, k2, "dram__bytes_read.sum", "2,000,000"),
            _row(1, k2, "sm__pipe_fma_cycles_active.avg.pct_of_peak_sustained_active", "7"),
            _row(2, k2, "gpu__time_duration.sum", "1,000,000"),
            _row(2, k2, "dram__bytes_read.sum", "4,000,000"),
            _row(2, k2, "sm__pipe_fma_cycles_active.avg.pct_of_peak_sustained_active", "9")]
    t = bench.summarize_launches(_csv(tmp_path, rows)).splitlines()
    assert "DRAM GB/s" in t[0] and "FMA pipe %" in t[0]
    first = [c.strip() for c in t[2].split("|")]
    assert first[1] == "`slab_factor_fused_kernel<float, 6, 3, 5, 3>`"
    assert first[2:6] == ["1", "3.000", "0.600", "3000.0"]   # 3 of 5 ms, one launch
    second = [c.strip() for c in t[3].split("|")]
    assert second[2:6] == ["2", "2.000", "0.400", "1000.0"]
    assert second[6] == "3"                                # 6 MB in 2 ms = 3 GB/s
    assert second[7] == "8.0"                              # mean of 7 and 9


def test_traffic_record_applies_only_to_its_workload_and_sources(tmp_path, monkeypatch):
    rows = [_row(0, "void slab_factor_fused_kernel<float, 6, 3, 5, 3>(A)", "dram__bytes_read.sum", "100"),
            _row(0, "void slab_factor_fused_kernel<float, 6, 3, 5, 3>(A)", "dram__bytes_write.sum", "300"),
            _row(1, "void slab_factor_fused_kernel<float, 6, 3, 5, 3>(A)", "dram__bytes_read.sum", "200"),
            _row(1, "void slab_factor_fused_kernel<float, 6, 3, 5, 3>(A)", "dram__bytes_write.sum", "200")]
    root = tmp_path / "root"
    (root / "profiles").mkdir(parents=True)
    csrc = root / "paper_1412_0464_gb300" / "csrc"
    csrc.mkdir(parents=True)
    for f in bench.TRAFFIC_KERNELS["slab_factor"][1]:
        (csrc / f).write_text("// " + f)
    monkeypatch.setattr(bench, "ROOT", str(root))
    out = bench.write_traffic(_csv(tmp_path, rows), "ncu ...", "wl A")
    assert out["kernels"]["slab_factor"]["dram_bytes_per_launch"] == 400.0
    assert bench._traffic("slab_factor", "wl A", "mixed") == 400.0
    assert bench._traffic("slab_factor", "wl B", "mixed") is None
    assert bench._traffic("slab_factor", "wl A", "fp64") is None
    (csrc / "slab.cuh").write_text("// changed")
    assert bench._traffic("slab_factor", "wl A", "mixed") is None
    assert json.load(open(os.path.join(root, "profiles", "traffic.json")))["bench_workload"] == "wl A"
