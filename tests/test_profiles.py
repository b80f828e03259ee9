"""The committed ncu summaries that bench.py reads for its roofline fields:
each names the full command that produced it and the hash of the kernel
sources it was taken on, and carries the per-launch figures bench.py looks
up (traffic, instruction count, limiter).  Whether the hash still matches
the sources is bench.py's decision at run time (it then reports no
traffic), so it is not asserted here."""
import glob
import os

import bench

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_every_summary_names_its_command_and_sources():
    files = sorted(glob.glob(os.path.join(ROOT, "profiles", "*.txt")))
    assert files
    for f in files:
        text = open(f).read()
        assert "# Command" in text or "#   ncu" in text, f
        assert "--clock-control none" in text, f
        assert "kernel_sources_sha256:" in text, f


def test_bench_profiles_exist_and_carry_their_keys():
    for (workload, p), name in bench.PROFILES.items():
        assert workload in bench.WORKLOADS
        assert p in (0, 1, 2)
        path = os.path.join(ROOT, "profiles", name)
        assert os.path.exists(path), name
        kv = {}
        for ln in open(path):
            if ":" in ln and not ln.startswith("#"):
                k, v = ln.split(":", 1)
                kv[k.strip()] = v.strip()
        for key in ("kernel_sources_sha256", "traffic_bytes_per_launch", "inst_per_launch", "limiter"):
            assert key in kv, (name, key)
        assert int(kv["traffic_bytes_per_launch"]) > 0
        assert int(kv["inst_per_launch"]) > 0
        assert kv["limiter"] in ("issue", "latency", "hbm")
