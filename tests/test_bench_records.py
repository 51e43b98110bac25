"""Host logic of bench.py's profile records (no GPU): a figure taken from a committed ncu summary is
reported only while the hash of the kernel and launch set-up sources and the kernel variant match
the ones recorded beside it; otherwise the bench line carries null."""
import pytest

import bench


def _write(tmp_path, name, text):
    d = tmp_path / "profiles"
    d.mkdir(exist_ok=True)
    (d / name).write_text(text)


def test_record_matches_only_same_sources_and_variant(tmp_path, monkeypatch):
    sha = bench.kernel_sources_sha1()
    _write(tmp_path, "launches_nside512_200k_seg.md",
           f"text\n<!-- machine-readable (read by bench.py): traffic_bytes_per_step=123456 variant=6 csrc_sha1={sha} -->\n")
    _write(tmp_path, "pair_kernel_far_nside128_200k_seg.md",
           f"<!-- machine-readable (read by bench.py): fma_pipe_busy=0.777 variant=6 csrc_sha1={sha} -->\n")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    monkeypatch.setattr(bench, "kernel_sources_sha1", lambda: sha)
    assert bench.profiled_traffic(6) == 123456
    assert bench.profiled_fma_busy(6) == pytest.approx(0.777)
    assert bench.profiled_traffic(5) is None          # another variant
    assert bench.profiled_fma_busy(-1) is None


def test_record_nulled_when_sources_change(tmp_path, monkeypatch):
    _write(tmp_path, "launches_nside512_200k_seg.md",
           "<!-- machine-readable (read by bench.py): traffic_bytes_per_step=99 variant=6 csrc_sha1=" + "0" * 40 + " -->\n")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    monkeypatch.setattr(bench, "kernel_sources_sha1", lambda: "f" * 40)
    assert bench.profiled_traffic(6) is None


def test_missing_summary_gives_none(tmp_path, monkeypatch):
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    monkeypatch.setattr(bench, "kernel_sources_sha1", lambda: "a" * 40)
    assert bench.profiled_traffic(6) is None
    assert bench.profiled_fma_busy(6) is None


def test_hash_covers_kernel_and_launch_sources():
    """The hash changes with any of the sources that decide the pair kernels' work and traffic."""
    import hashlib
    import os

    h = hashlib.sha1()
    for f in ("map.cu", "pipeline.cuh", "isw_internal.cuh", "pack.cu", "api.cu", "kernels.cuh"):
        with open(os.path.join(bench.ROOT, "paper_1204_5041_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    assert bench.kernel_sources_sha1() == h.hexdigest()
