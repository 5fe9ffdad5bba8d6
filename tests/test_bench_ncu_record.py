"""The DRAM-traffic record that the benchmark reads (profiles/dram_traffic.json)
is written from ncu's CSV launch logs by bench.py itself: checked here on a small
hand-made log (plan kernels, one apply, two SpMV steps), and the committed
record's layout."""
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402

HEADER = '"ID","Kernel Name","Metric Name","Metric Unit","Metric Value"\n'


def _log(tmp_path, launches):
    rows = ["==PROF== Connected to process 1\n", HEADER]
    for i, (name, rd, wr, ns) in enumerate(launches):
        rows.append(f'"{i}","{name}","dram__bytes_read.sum","byte","{rd:,}"\n')
        rows.append(f'"{i}","{name}","dram__bytes_write.sum","byte","{wr}"\n')
        rows.append(f'"{i}","{name}","gpu__time_duration.sum","nsecond","{ns}"\n')
    p = tmp_path / "launches.csv"
    p.write_text("".join(rows))
    return str(p)


def test_summary_of_one_apply_and_two_steps(tmp_path):
    log = _log(tmp_path, [
        ("void radix_sort::DeviceRadixSortOnesweepKernel<int>(int *)", 100, 50, 1000),
        ("nap::<unnamed>::k_classify(const int *)", 200, 80, 2000),
        ("void nap::k_gather2<double>(const T1 *, int)", 1000, 800, 3000),
        ("void nap::k_pack<double>(const T1 *)", 900, 700, 2500),
        ("void nap::k_transfer<double>(const T1 *)", 900, 700, 2000),
        ("void nap::k_unpack<double>(const T1 *)", 1200, 900, 3500),
        ("void nap::k_spmv_s<0, 0, 8, 32>(SellView)", 5000, 100, 9000),
        ("void nap::k_spmv_s<0, 0, 8, 32>(SellView)", 5100, 100, 9100),
        ("void nap::k_spmv_s<0, 0, 8, 32>(SellView)", 4900, 100, 8900),
    ])
    r = bench.ncu_summary(log, nsteps=2, per_step=1)
    assert [k["kernel"] for k in r["per_kernel"]] == [
        "k_gather2<double>", "k_pack<double>", "k_transfer<double>", "k_unpack<double>",
        "k_spmv_s<0, 0, 8, 32>"]
    assert r["apply_bytes"] == 1800 + 1600 + 1600 + 2100 + 5100
    assert r["apply_us_serialised"] == 20.0
    assert r["spmv_step_kernels"] == ["k_spmv_s<0, 0, 8, 32>"]
    assert r["spmv_step_bytes"] == (5200 + 5000) / 2
    assert r["spmv_step_us"] == 9.0


def test_fp32_steps_take_two_launches(tmp_path, monkeypatch):
    log = _log(tmp_path, [
        ("nap::<unnamed>::k_sell_fill(const int *)", 10, 10, 100),
        ("nap::k_to_f32(const double *)", 40, 20, 500),
        ("void nap::k_spmv_s<1, 0, 8, 32>(SellView)", 3000, 60, 5000),
        ("nap::k_to_f32(const double *)", 40, 20, 600),
        ("void nap::k_spmv_s<1, 0, 8, 32>(SellView)", 3000, 60, 5200),
        ("nap::k_to_f32(const double *)", 40, 20, 400),
        ("void nap::k_spmv_s<1, 0, 8, 32>(SellView)", 3000, 60, 5400),
    ])
    out = tmp_path / "dram_traffic.json"
    monkeypatch.setattr(bench, "kernel_hash", lambda: "h")
    d = bench.write_ncu_records([f"w|f32|phased|sell={log}"], str(out))
    assert json.loads(out.read_text()) == d and d["kernel_hash"] == "h"
    r = d["records"]["w|f32|phased|sell"]
    assert r["spmv_step_kernels"] == ["k_to_f32", "k_spmv_s<1, 0, 8, 32>"]
    # per step: the FP32 copy of x and the SpMV, averaged over the two steps
    assert r["spmv_step_bytes"] == 60 + 3060 and r["apply_bytes"] == 60 + 3060


def test_committed_record_layout():
    d = json.load(open(os.path.join(ROOT, "profiles", "dram_traffic.json")))
    assert len(d["kernel_hash"]) == 16
    for key, r in d["records"].items():
        assert len(key.split("|")) == 4
        assert r["apply_bytes"] > 0 and r["spmv_step_bytes"] > 0
        assert r["apply_bytes"] == sum(k["dram_read"] + k["dram_write"] for k in r["per_kernel"])
