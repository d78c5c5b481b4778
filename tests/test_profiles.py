"""The committed profiles.  The DRAM-traffic record of the grid-update kernel
is consistent: read + write add up to the per-launch figure the bench
reports, that figure is within a few per cent of the algorithmic 20 bytes per
point (no wasted re-reads), and the bench uses it only while the kernel source
is the one the counters were taken on.  Every ncu summary gives the command
that produced it, which runs committed files only and keeps the GPU clocks
unlocked (--clock-control none)."""
import json
import os
import re
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def _record():
    with open(os.path.join(ROOT, "profiles", "traffic.json")) as f:
        return json.load(f)


def test_traffic_record_adds_up_and_is_near_the_algorithmic_bytes():
    rec = _record()
    assert "so8" in rec
    for key, e in rec.items():
        assert re.fullmatch(r"so\d+", key)
        assert re.fullmatch(r"[0-9a-f]{16}", e["source_sha"])
        total = e["dram_bytes_read"] + e["dram_bytes_write"]
        assert abs(total - e["bytes_per_launch_512"]) <= 1e-9 * total
        # u^n, u^-, c and d read once and u^+ written once per point
        algorithmic = 20.0 * 512 ** 3
        assert 0.98 <= total / algorithmic <= 1.10, (key, total / algorithmic)


def test_bench_reports_traffic_only_for_the_source_it_was_taken_on(tmp_path, monkeypatch):
    sha = bench.kernel_source_sha()
    assert re.fullmatch(r"[0-9a-f]{16}", sha)
    e = _record()["so8"]
    got = bench.kernel_traffic(8)
    if e["source_sha"] == sha:
        assert got == e["bytes_per_launch_512"]
    else:
        assert got is None
    # a record taken on another source is not used
    fake = tmp_path / "profiles"
    fake.mkdir()
    (fake / "traffic.json").write_text(json.dumps({"so8": dict(e, source_sha="0" * 16)}))
    real_join = os.path.join

    def join(*parts):
        if parts[:3] == (bench.ROOT, "profiles", "traffic.json"):
            return str(fake / "traffic.json")
        return real_join(*parts)

    monkeypatch.setattr(bench.os.path, "join", join)
    assert bench.kernel_traffic(8) is None


def _profile_commands():
    out = {}
    pdir = os.path.join(ROOT, "profiles")
    for f in sorted(os.listdir(pdir)):
        if f.endswith(".md"):
            text = open(os.path.join(pdir, f)).read()
            out[f] = re.findall(r"```\n(.*?)```", text, flags=re.S)
    return out


def test_every_profile_gives_a_command_that_runs_committed_files_only():
    cmds = _profile_commands()
    assert cmds
    for f, blocks in cmds.items():
        assert blocks, "%s has no command" % f
        text = "\n".join(blocks).replace("\\\n", " ")
        assert "_work" not in text, f
        for line in text.splitlines():
            for m in re.finditer(r"python (?:-m ([\w.]+)|([\w/]+\.py))", line):
                if m.group(1):
                    path = os.path.join(ROOT, *m.group(1).split(".")) + ".py"
                else:
                    path = os.path.join(ROOT, m.group(2))
                assert os.path.isfile(path), (f, line)
            for part in line.split("&&"):
                if part.strip().startswith("ncu"):
                    assert "--clock-control none" in part, (f, line)
