"""Host logic of the benchmark that needs no GPU: the DRAM-traffic figure is reported only for the sources
it was measured on."""
import bench


def _ncu_csv(path, read, write, unit="byte"):
    path.write_text(
        '"ID","Kernel Name","dram__bytes_read.sum","dram__bytes_write.sum"\n'
        f'"","","{unit}","{unit}"\n'
        f'"0","eval_direct_async_kernel","{read}","{write}"\n')
    return str(path)


def test_traffic_keyed_by_source_hash(tmp_path, monkeypatch):
    traffic = tmp_path / "traffic.txt"
    traffic.write_text("# header\nsome old line | 1 512 1 4 1 | 1280644864 | old format\n")
    monkeypatch.setattr(bench, "TRAFFIC_FILE", str(traffic))
    shape = {"variant": 1, "nb": 512, "ppc": 1, "stages": 4, "order": 1}
    assert bench._profiled_traffic(shape) is None  # nothing recorded for these sources
    bench.record_traffic(_ncu_csv(tmp_path / "a.csv", "979.5", "301.25", "Mbyte"), shape, "profiles/x.md")
    assert bench._profiled_traffic(shape) == 979.5e6 + 301.25e6
    other = dict(shape, stages=6)
    assert bench._profiled_traffic(other) is None  # another launch shape
    # a second record of the same shape replaces the first
    bench.record_traffic(_ncu_csv(tmp_path / "b.csv", "1000", "24"), shape, "profiles/x.md")
    assert bench._profiled_traffic(shape) == 1024.0
    assert traffic.read_text().count(bench.WORKLOAD) == 1
    # after an edit of the kernel sources the figure no longer applies
    monkeypatch.setattr(bench, "eval_source_hash", lambda: "0123456789abcdef")
    assert bench._profiled_traffic(shape) is None


def test_source_hash_covers_the_evaluation_sources():
    h = bench.eval_source_hash()
    assert len(h) == 16 and int(h, 16) >= 0
    assert "bspline_eval_kernels.cuh" in bench.EVAL_SOURCES and "bspline_lib.cu" in bench.EVAL_SOURCES
