"""The benchmark's JSON contract, on CPU: the reference arm (the oracle timed on
host cores) at a small size, its silence on ranks other than 0, and the
at-scale config block shared by both arms."""

import importlib.util
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def load_bench():
    spec = importlib.util.spec_from_file_location("bench_under_test", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def run_bench(extra_env=None, *args):
    env = dict(os.environ)
    env.update(extra_env or {})
    return subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), *args], capture_output=True, text=True,
                          env=env, cwd=ROOT, timeout=300)


def test_reference_arm_line():
    r = run_bench(None, "--impl", "reference", "--steps", "2", "--warmup", "1", "--log2-buckets", "12",
                  "--log2-batch", "10")
    assert r.returncode == 0, r.stderr
    line = json.loads(r.stdout.strip().splitlines()[-1])
    bench = load_bench()
    assert line["impl"] == "reference" and line["metric"] == bench.METRIC and line["unit"] == bench.UNIT
    assert line["higher_is_better"] is True and line["steps"] == 2 and line["warmup"] == 1 and line["n_gpus"] == 1
    assert line["value"] > 0 and line["ms_per_step"] > 0
    cb = line["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == line["value"] and cb["unit"] == bench.UNIT
    assert "1024 lookups per step" in cb["sample"]
    # one step is 1024 lookups: the rate and the step time agree
    assert abs(line["value"] - 1024 / (line["ms_per_step"] / 1e3) / 1e9) <= 0.05 * line["value"] + 1e-6
    e2e = line["e2e"]
    assert e2e == {"value": line["value"], "unit": bench.UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
    cfg = line["config"]
    assert cfg["n_buckets"] == 4096 and cfg["batch"] == 1024 and cfg["entries"] == int(0.9 * 4096 * 8)
    assert cfg["workload"] == "plain Cuckoo++ at scale: 2^12 buckets x 8 slots, LF 0.9, 1024-key bulk_lookup"
    assert cfg["l2"].startswith("inputs not larger than L2")


def test_reference_arm_only_rank0_prints():
    r = run_bench({"RANK": "1", "WORLD_SIZE": "2", "LOCAL_RANK": "1"}, "--impl", "reference", "--steps", "1",
                  "--warmup", "1", "--log2-buckets", "10", "--log2-batch", "8")
    assert r.returncode == 0, r.stderr
    assert r.stdout.strip() == ""


def test_default_scale_config():
    bench = load_bench()
    sys_argv = sys.argv
    try:
        sys.argv = ["bench.py"]
        args = bench.parse()
    finally:
        sys.argv = sys_argv
    cfg = bench.scale_config(args, 120_795_955)
    assert cfg["workload"] == "plain Cuckoo++ at scale: 2^24 buckets x 8 slots, LF 0.9, 16M-key bulk_lookup"
    assert cfg["n_buckets"] == 1 << 24 and cfg["batch"] == 1 << 24 and cfg["timers"] is False
    assert cfg["l2"] == "inputs larger than L2 (table 4.3 GB, keys 256 MB); no flush"
    # the committed DRAM-traffic capture is of this configuration
    assert (args.log2_buckets, args.log2_batch, args.load_factor, args.neg_rate) == bench.TRAFFIC_CONFIG


def test_roofline_byte_counts():
    """Algorithmic bytes: 32 per bucket read (primary or secondary) and per
    record examined, plus 25 of streamed key and result per lookup; line bytes:
    128 per line request (one per bucket read, one per second-line read) plus
    the same 25."""
    bench = load_bench()
    n, prim, sec, rec, line1 = 1000, 1000, 64, 500, 225
    counts = [prim, sec, rec, line1]
    assert bench.alg_bytes_of(counts, n) == 32 * (prim + sec + rec) + 25 * n
    assert bench.lines_of(counts) == prim + sec + line1
    assert bench.line_bytes_of(counts, n) == 128 * (prim + sec + line1) + 25 * n
    # the headline batch's counts give the per-lookup figures the bench reports
    assert abs(bench.alg_bytes_of([1.0, 0.0645, 0.5], 1) - 75.06) < 0.01


def test_traffic_record_and_read(tmp_path):
    """--record-traffic turns an ncu --csv log of the lookup kernel (units as
    ncu prints them) into the traffic data file, stamped with the current
    sources' sha256; the bench reports it only while that stamp matches."""
    bench = load_bench()
    name = "void ckpp::<unnamed>::lookup_kernel<0, 0, 0, 0>(ckpp::TableView)"
    head = '"ID","Process ID","Kernel Name","Metric Name","Metric Unit","Metric Value"\n'
    rows = [("0", "dram__bytes_read.sum", "Gbyte", "2.5"), ("0", "dram__bytes_write.sum", "Mbyte", "1,500.5"),
            ("0", "gpu__time_duration.sum", "ns", "400000"), ("1", "dram__bytes_read.sum", "Gbyte", "9.0")]
    csv_path = tmp_path / "t.csv"
    csv_path.write_text("==PROF== noise\n" + head + "".join(f'"{i}","1","{name}","{m}","{u}","{v}"\n'
                                                           for i, m, u, v in rows))
    bench.TRAFFIC_FILE = str(tmp_path / "traffic.json")
    bench.record_traffic(str(csv_path))
    d = json.loads(open(bench.TRAFFIC_FILE).read())
    assert d["traffic_bytes_per_launch"] == 2_500_000_000 + 1_500_500_000
    assert d["gpu_time_us"] == 400.0 and d["sources_sha256"] == bench.sources_sha256()
    assert bench.profiled_traffic() == float(d["traffic_bytes_per_launch"])
    d["sources_sha256"] = "0" * 64
    open(bench.TRAFFIC_FILE, "w").write(json.dumps(d))
    assert bench.profiled_traffic() is None


def test_committed_traffic_file_names_the_lookup_sources():
    bench = load_bench()
    d = json.loads(open(os.path.join(ROOT, "profiles", "lookup_traffic.json")).read())
    assert tuple(d["sources"]) == bench.LOOKUP_SOURCES
    assert d["config"] == dict(zip(("log2_buckets", "log2_batch", "load_factor", "neg_rate"), bench.TRAFFIC_CONFIG))
