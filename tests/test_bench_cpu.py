"""Host-side helpers of bench.py (no GPU): the roofline's DRAM traffic is
read from the committed ncu summary only while the G1 source it was taken on
is unchanged, and the whole-path work figures add up."""
import hashlib
import os

import bench


def _tree(tmp_path, kernel_text, recorded_sha, traffic="3.83e8"):
    (tmp_path / "profiles").mkdir()
    src = tmp_path / "paper_1010_1386_gb300" / "csrc"
    src.mkdir(parents=True)
    (src / "kernels_g1.cu").write_text(kernel_text)
    (tmp_path / "profiles" / "g1_images_batch512.md").write_text(
        "# G1\n\nkernels_g1.cu sha256: %s\n\ndram bytes per G1 stage: %s\n" % (recorded_sha, traffic))


def test_g1_traffic_only_for_the_profiled_source(tmp_path, monkeypatch):
    text = "// kernel\n"
    sha = hashlib.sha256(text.encode()).hexdigest()
    _tree(tmp_path, text, sha)
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.g1_traffic() == 3.83e8
    (tmp_path / "paper_1010_1386_gb300" / "csrc" / "kernels_g1.cu").write_text(text + "// changed\n")
    assert bench.g1_traffic() is None


def test_g1_traffic_missing_profile_is_null(tmp_path, monkeypatch):
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.g1_traffic() is None


def test_committed_profile_names_a_sha_and_a_traffic():
    text = open(os.path.join(os.path.dirname(bench.__file__), "profiles", "g1_images_batch512.md")).read()
    assert "kernels_g1.cu sha256:" in text and "dram bytes per G1 stage:" in text


def test_whole_path_work_adds_up():
    info = {"modmul_eval": 1e9, "modmul_prs": 3e9, "modmul_interp": 5e8, "modmul_crt": 5e8}
    w = bench.whole_path_work(info, 100, 10.0, 20.0)
    assert w["total"] == 5e9 and w["per_resultant"] == 5e7
    assert abs(w["whole_path_timad_s"] - 4 * 5e9 / 1e-2 / 1e12) < 1e-9
    assert abs(w["whole_path_frac"] - w["whole_path_timad_s"] / 20.0) < 1e-12
