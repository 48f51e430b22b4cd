"""bench.py's host side without a GPU: the reference arm's JSON line (the
oracle timed on the host cores) and the profile records keyed to the
step-kernel source."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def test_reference_arm_prints_one_complete_line():
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "2", "--warmup", "1"],
                       cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert key in d, key
    assert d["impl"] == "reference"
    assert d["steps"] == 2 and d["warmup"] == 1
    assert d["value"] > 0 and d["higher_is_better"] is True
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["cpu_baseline"]["cores"] >= 1
    assert d["e2e"]["value"] == d["value"]
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["d2h_bytes_per_step"] == 0


def test_profile_record_applies_only_to_its_kernel(tmp_path, monkeypatch):
    import bench
    digest = bench.kernel_hash()
    assert len(digest) == 16 and int(digest, 16) >= 0
    assert bench.kernel_hash() == digest  # deterministic
    prof = tmp_path / "profiles"
    prof.mkdir()
    (prof / "rec.txt").write_text("# comment line\n"
                                  "step_fp32_8192 0123456789abcdef 1.0\n"
                                  f"step_fp32_8192 {digest} 6940000000\n"
                                  f"other_tag {digest} 5\n")
    # kernel_hash reads the sources under ROOT: point only the records elsewhere
    real_root = bench.ROOT
    monkeypatch.setattr(bench, "kernel_hash", lambda sources=bench.STEP_SOURCES: digest)
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.profile_record("rec.txt", "step_fp32_8192") == pytest.approx(6.94e9)
    assert bench.profile_record("rec.txt", "other_tag") == 5.0
    assert bench.profile_record("rec.txt", "missing") is None
    assert bench.profile_record("absent.txt", "step_fp32_8192") is None
    (prof / "stale.txt").write_text("step_fp32_8192 0123456789abcdef 1.0\n")
    assert bench.profile_record("stale.txt", "step_fp32_8192") is None
    assert os.path.isdir(os.path.join(real_root, "profiles"))


def test_paired_kernel_records_follow_their_own_sources():
    """The paired kernel's records are keyed by the hash of its own sources
    (the single-step kernel's plus its file and headers), not the step hash."""
    import bench
    step, pair = bench.kernel_hash(), bench.kernel_hash(bench.PAIR_SOURCES)
    assert step != pair and len(pair) == 16
    assert set(bench.STEP_SOURCES) < set(bench.PAIR_SOURCES)
    ipl = bench.pair_record("pair_fp32_warp_instr_per_lu")
    assert ipl is None or 5.0 < ipl < 20.0
    traffic = bench.pair_record("pair_fp32_8192")
    # near the algorithmic bytes of a paired launch (52 per update, two steps): a
    # little under them when written lines are still in L2 at the launch's end,
    # well over them only if tiles re-read their input
    algorithmic = 52 * 2 * 8192 * 8192
    assert traffic is None or 0.9 * algorithmic < traffic < 1.2 * algorithmic
