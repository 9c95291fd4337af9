"""Host-side helpers of bench.py (no GPU): the roofline's DRAM traffic comes
from the record that --record-traffic writes from an ncu CSV log, and only
while the G1 source it was taken on is unchanged; the whole-path work
figures add up."""

import bench

HDR = ['"ID"', '"Process ID"', '"Process Name"', '"Host Name"', '"Kernel Name"', '"Context"', '"Stream"',
       '"Block Size"', '"Grid Size"', '"Device"', '"CC"', '"Section Name"', '"Metric Name"',
       '"Metric Unit"', '"Metric Value"']


def _row(i, kernel, metric, unit, value):
    return ",".join('"%s"' % v for v in (i, 1, "python", "h", kernel, 1, 7, "(128, 1, 1)", "(608, 1, 1)",
                                          0, "10.3", "Command line profiler metrics", metric, unit, value))


def _tree(tmp_path, kernel_text):
    (tmp_path / "profiles").mkdir()
    src = tmp_path / "paper_1010_1386_gb300" / "csrc"
    src.mkdir(parents=True)
    (src / "kernels_g1.cu").write_text(kernel_text)
    csv = tmp_path / "g1.csv"
    lines = ["==PROF== Connected to process 1", ",".join(HDR)]
    i = 0
    for step in range(2):  # two steps of two launches each: only the last step counts
        for k, mb in (("void g1_kernel<40>(G1Args)", 10.0 + step), ("void g1_kernel<32>(G1Args)", 2.0)):
            lines.append(_row(i, k, "dram__bytes_read.sum", "Mbyte", "%.1f" % mb))
            lines.append(_row(i, k, "dram__bytes_write.sum", "Kbyte", "500"))
            i += 1
        lines.append(_row(i, "g2n_kernel(G2nArgs)", "dram__bytes_read.sum", "Mbyte", "99"))
        i += 1
    csv.write_text("\n".join(lines) + "\n")
    return csv


def test_g1_traffic_only_for_the_recorded_source(tmp_path, monkeypatch):
    text = "// kernel\n"
    csv = _tree(tmp_path, text)
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    bench.record_traffic(str(csv), "ncu ...")
    assert bench.g1_traffic() == 11e6 + 0.5e6 + 2e6 + 0.5e6
    (tmp_path / "paper_1010_1386_gb300" / "csrc" / "kernels_g1.cu").write_text(text + "// changed\n")
    assert bench.g1_traffic() is None


def test_g1_traffic_missing_record_is_null(tmp_path, monkeypatch):
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.g1_traffic() is None


def test_whole_path_work_adds_up():
    info = {"modmul_eval": 1e9, "modmul_prs": 3e9, "modmul_interp": 5e8, "modmul_crt": 5e8}
    w = bench.whole_path_work(info, 100, 10.0, 20.0)
    assert w["total"] == 5e9 and w["per_resultant"] == 5e7
    assert abs(w["whole_path_timad_s"] - 4 * 5e9 / 1e-2 / 1e12) < 1e-9
    assert abs(w["whole_path_frac"] - w["whole_path_timad_s"] / 20.0) < 1e-12
