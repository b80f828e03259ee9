#!/usr/bin/env python
"""Benchmark of the two-layer decode (whole-archive decode, unified seek,
batched decode, seek serving) on synthetic data shaped like the paper's
workloads.

Headline (the JSON line's value): whole-archive decode of 256 MiB of
synthetic FASTQ (seed 1; header/150-base read/'+'/quality records), 16 KiB
blocks (16,384 blocks), encoded by the library's host encoder.  A step is
one ace_decode_all: every block's three rANS streams decoded and its literals
and absolute-offset matches resolved into the output, on the GPU, with a
256 MiB L2 flush between steps.

Also measured, each at the size its configuration states:
  - plain small: 1 MiB mixed data (seed 0), decode latency, graph replay,
    the seek of block 37 with the three-phase check;
  - FASTQ: 10,000 random single-block seeks, plain (one launch sequence and
    a synchronise each) and batched through the decoded-block cache; the end
    to end time through the C ABI from pinned host memory;
  - genome: 1 GiB repetitive genome (seed 3), whole decode, levels;
  - batched: 4,096 uneven objects (log-uniform 4 KiB - 64 MiB, four
    profiles, 4/16/64 KiB blocks) in one CUDA-graph replay against one
    launch sequence per object;
  - serving: 8 resident archives of 5 GiB (40 GiB decompressed) under a
    20 GB device working-set budget, Poisson arrivals 10k - 1M requests/s;
  - beyond device memory: a 50 GB genome whose archive stays in host
    memory, the range decode of blocks 0..1000 and a long range streamed to
    host memory in sub-ranges;
  - the GPU encoder on the FASTQ and genome workloads, beside the host
    encoder (the batched, serving and host-resident workloads are encoded
    with it);
  - the oracle on the host cores beside each decode.
--quick caps the batched objects at 2 MiB, the served archives at 256 MiB
and the host-resident genome at 4 GiB (labelled as reduced in the output).

Prints one JSON line.  Under torchrun each rank decodes its own replica
(replicas only: no data-path collective).
"""
import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

# workload name -> (profile, decompressed bytes, seed, log2 block size, min match)
WORKLOADS = {
    "fastq-256MiB-16KiB-blocks": ("fastq", 1 << 28, 1, 14, 16),
    "mixed-1MiB-16KiB-blocks": ("mixed", 1 << 20, 0, 14, 4),
    "genome-1GiB-16KiB-blocks": ("genome", 1 << 30, 3, 14, 20),
    "text-128MiB-16KiB-blocks": ("text", 1 << 27, 5, 14, 4),  # --workload only: the text profile of configs 4-5
}
WORKLOAD = "fastq-256MiB-16KiB-blocks"
MIN_MATCH = {"fastq": 16, "genome": 20, "text": 4, "mixed": 4}
SEEK_SEED = 2
REF_SAMPLE = 8 << 20   # the reference arm decodes this many bytes of the workload per step
E2E_INFLIGHT = 3       # end-to-end steps in flight, each with its own stream and device buffers
SPEC_HBM_GBS = 7900.0  # nominal GB300 HBM3e bandwidth (spec sheet)
SCHEDULERS_PER_SM = 4  # warp schedulers per SM: one warp instruction each per cycle
METRIC = "decompressed GB/s (% HBM roofline); 16KB seek p50/p99 us, batched vs plain"
KERNEL_SOURCES = ["paper_2606_24531_gb300/csrc/ace.cu", "paper_2606_24531_gb300/csrc/ace_device.cuh"]
PROFILES_DIR = os.path.join(ROOT, "profiles")
# committed ncu summaries of the dominant kernel, per (workload, pass: 0 tokens, 1 literals, 2 matches)
PROFILES = {("fastq-256MiB-16KiB-blocks", 0): "token_pass_fastq256.txt",
            ("fastq-256MiB-16KiB-blocks", 1): "literal_pass_fastq256.txt",
            ("fastq-256MiB-16KiB-blocks", 2): "match_pass_fastq256.txt",
            ("genome-1GiB-16KiB-blocks", 2): "match_pass_genome1g.txt"}


def kernel_sha():
    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        with open(os.path.join(ROOT, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def profile_summary(path):
    """The key: value lines of a committed ncu summary, if it was taken on the
    current kernel sources (else None)."""
    try:
        kv = {}
        with open(path) as f:
            for ln in f:
                if ":" in ln and not ln.startswith("#"):
                    k, v = ln.split(":", 1)
                    kv[k.strip()] = v.strip()
        if kv.get("kernel_sources_sha256") == kernel_sha():
            return kv
    except OSError:
        pass
    return None


def cpu_model():
    """The host CPU's model line from /proc/cpuinfo (the part number on Arm)."""
    try:
        with open("/proc/cpuinfo") as f:
            lines = f.read().splitlines()
    except OSError:
        return "unknown"
    for key in ("model name", "CPU part", "Hardware"):
        for ln in lines:
            if ln.startswith(key):
                return ln.split(":", 1)[1].strip()
    return "unknown"


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "sm_max_mhz": 2070.0}, "fallback"


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during a region."""

    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.f = tempfile.TemporaryFile(mode="w+")
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(gpu_index), "--query-gpu=" + self.Q,
                                       "--format=csv,noheader,nounits", "-lms", "100"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.p = None

    def stop(self):
        if self.p is None:
            return None
        self.p.terminate()
        self.p.wait()
        self.f.seek(0)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.f:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            for n, v in zip(names, parts[4:8]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def make_data(name, limit=None):
    import synth

    profile, total, seed, log2b, min_match = WORKLOADS[name]
    data = synth.generate(profile, total, seed)
    if limit is not None and limit < data.size:
        data = np.ascontiguousarray(data[:limit])
    return data, log2b, min_match


def make_workload(name, limit=None):
    """The workload's data and its archive from the library's host encoder;
    limit takes a prefix of the data."""
    from paper_2606_24531_gb300 import ace

    data, log2b, min_match = make_data(name, limit)
    arc, stats = ace.ace_encode(data, log2b, min_match, stats=True)
    return data, arc, stats


def max_over_ranks(x, dist, device):
    """The largest of every rank's x (the job's step time is its slowest rank's)."""
    import torch

    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def archive_bytes_read(arc):
    """Bytes of an archive a whole decode reads: all of it but the dependency
    table (header, directory, stream payloads)."""
    hdr = arc[:64].view(np.uint64)
    return int(arc.size) - (int(hdr[6]) - int(hdr[5]))


def stream_bytes(arc):
    """Stored bytes of the literal, length and offset streams over all blocks."""
    hdr = arc[:64].view(np.uint64)
    nb, dir_off = int(hdr[3]), int(hdr[4])
    d = arc[dir_off:dir_off + 64 * nb].view(np.uint32).reshape(nb, 16)[:, 6:9].astype(np.int64)
    return [int(x) for x in d.sum(axis=0)], nb


def algorithmic_bytes(arc, stats, total):
    """The plain definition's bytes (compressed bytes read + match-source
    bytes read + output bytes written) for the whole decode, and split over
    the three passes of the pass schedule: tokens read the directory and the
    length and offset streams; literals read the directory and the literal
    streams and write the literals; matches read each match's source bytes
    (min(length, distance)) and write the matched bytes.  The 16-byte match
    records the passes exchange are the design's own intermediate data and
    are counted apart."""
    sb, nb = stream_bytes(arc)
    whole = archive_bytes_read(arc) + stats["match_src_bytes"] + total
    return {
        "whole": whole,
        "whole_upper": archive_bytes_read(arc) + stats["match_bytes"] + total,
        "passes": [64 * nb + sb[1] + sb[2],
                   64 * nb + sb[0] + stats["literal_bytes"],
                   stats["match_src_bytes"] + stats["match_bytes"]],
        "intermediate_records": 16 * stats["n_matches"],
    }


def timed(stream, fn, steps, warmup, flush=None):
    """Device time (ms) of fn() per step: CUDA events on stream, an L2 flush
    (a fill larger than L2) before each step outside the events."""
    import torch

    out = []
    for k in range(warmup + steps):
        if flush is not None:
            flush.fill_(k & 255)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        fn()
        e1.record(stream)
        e1.synchronize()
        if k >= warmup:
            out.append(e0.elapsed_time(e1))
    return out


def pass_times(ace, da, out, stream, flush, steps):
    """Mean ms of each pass of the pass schedule (events between them)."""
    import torch

    per = [[], [], []]
    passes = (ace.ACE_PASS_TOKENS, ace.ACE_PASS_LITERALS, ace.ACE_PASS_MATCH)
    for k in range(steps + 2):
        flush.fill_(k & 255)
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
        ev[0].record(stream)
        for p in passes:
            ace.ace_decode_pass(da.idx, p, out, da.total, da.d_scratch, da.scratch_bytes, None, stream)
            ev[p + 1].record(stream)
        ev[3].synchronize()
        if k >= 2:
            for p in range(3):
                per[p].append(ev[p].elapsed_time(ev[p + 1]))
    return [statistics.mean(x) for x in per]


def oracle_baseline(data, arc, what):
    """The oracle (plain sequential C decoder, one host thread) decoding arc,
    checked against data."""
    import oracle

    t0 = time.perf_counter()
    ref = oracle.decode(arc)
    dt = time.perf_counter() - t0
    assert np.array_equal(ref, data), "oracle decode differs from the original"
    return {"value": data.size / dt / 1e9, "unit": "GB/s", "cores": 1, "kind": "oracle",
            "sample": "%s, one thread (%.2f s)" % (what, dt)}


def run_reference(args, rank):
    """The reference arm: the oracle (plain sequential C encoder and decoder,
    test infrastructure) on the host cores.  Each step decodes a bounded
    sample of the workload, a prefix encoded by the oracle's own encoder;
    this arm never loads the GPU library."""
    if rank != 0:
        return
    import oracle

    data, log2b, min_match = make_data(args.workload, REF_SAMPLE)
    arc = oracle.encode(data, log2b, min_match, 16)
    t_all = []
    for k in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        out = oracle.decode(arc)
        t1 = time.perf_counter()
        if k >= args.warmup:
            t_all.append(t1 - t0)
    assert np.array_equal(out, data)
    ms = 1e3 * statistics.mean(t_all)
    gbs = data.size / (ms / 1e3) / 1e9
    sample = ("the first %d bytes of the workload, encoded by the oracle's encoder, decoded whole each step, "
              "one thread" % data.size)
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": gbs, "unit": "GB/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "u8", "data": "synthetic",
        "config": {"workload": args.workload, "sample_bytes": int(data.size),
                   "blocks": int(data.size >> log2b)},
        "cpu_baseline": {"value": gbs, "unit": "GB/s", "cores": 1, "kind": "oracle", "sample": sample},
        "e2e": {"value": gbs, "unit": "GB/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }), flush=True)


def roofline_of(alg, ms_pass, ms_whole, peaks, peak_kind, sm_count, clocks, workload):
    """The roofline of the dominant kernel (the slowest pass of the pass
    schedule), on the plain definition's bytes, plus the whole decode.  When
    the committed ncu summary of that kernel matches the current sources, its
    DRAM traffic and instruction count give the traffic field and the issue
    roofline (warp instructions per second against 4 per SM per cycle at the
    sampled SM clock); the summary's limiter names the bound."""
    names = ["decode_kernel<false, PASS_TOKENS>", "decode_kernel<false, PASS_LITERALS>",
             "match_level_kernel + match_small_kernel"]
    top = max(range(3), key=lambda p: ms_pass[p])
    hbm_peak = peaks["hbm_gbs"]
    achieved = alg["passes"][top] / (ms_pass[top] / 1e3) / 1e9
    pf = PROFILES.get((workload, top))
    prof = profile_summary(os.path.join(PROFILES_DIR, pf)) if pf else None
    sm_mhz = (clocks or {}).get("sm_mhz") or peaks.get("sm_max_mhz", 2070.0)
    issue = None
    if prof and "inst_per_launch" in prof:
        inst = float(prof["inst_per_launch"])
        ips = inst / (ms_pass[top] / 1e3)
        ipeak = sm_count * SCHEDULERS_PER_SM * sm_mhz * 1e6
        issue = {"achieved": ips, "peak": ipeak, "unit": "warp-inst/s", "frac": ips / ipeak,
                 "inst_per_launch": inst, "sm_mhz": sm_mhz,
                 "peak_basis": "%d SMs x %d schedulers x the median sampled SM clock" % (sm_count, SCHEDULERS_PER_SM)}
    hbm = {"achieved": achieved, "peak": hbm_peak, "unit": "GB/s", "frac": achieved / hbm_peak,
           "peak_kind": peak_kind + " (MEASURED_PEAKS.json hbm_gbs)" if peak_kind == "measured" else peak_kind}
    bound = (prof or {}).get("limiter", "hbm")
    r = {"bound": "alu" if bound == "issue" and issue else "hbm", "kernel": names[top],
         "traffic": int(prof["traffic_bytes_per_launch"]) if prof and "traffic_bytes_per_launch" in prof else None,
         "algorithmic_bytes": alg["passes"][top], "hbm": hbm, "issue": issue,
         "passes": {n: {"ms": ms_pass[p], "algorithmic_bytes": alg["passes"][p],
                        "achieved_gbs": alg["passes"][p] / (ms_pass[p] / 1e3) / 1e9,
                        "frac": alg["passes"][p] / (ms_pass[p] / 1e3) / 1e9 / hbm_peak}
                    for p, n in enumerate(["tokens", "literals", "matches"])},
         "intermediate_record_bytes": alg["intermediate_records"],
         "whole_decode": {"algorithmic_bytes": alg["whole"], "algorithmic_bytes_upper": alg["whole_upper"],
                          "achieved_gbs": alg["whole"] / (ms_whole / 1e3) / 1e9,
                          "frac": alg["whole"] / (ms_whole / 1e3) / 1e9 / hbm_peak},
         "spec_sheet": {"peak_gbs": SPEC_HBM_GBS, "frac_of_spec": achieved / SPEC_HBM_GBS,
                        "label": "fraction of the nominal HBM3e bandwidth, not a measurement"}}
    if r["bound"] == "alu":
        r.update({"achieved": issue["achieved"], "peak": issue["peak"], "unit": "warp-inst/s", "frac": issue["frac"]})
    else:
        r.update({"achieved": achieved, "peak": hbm_peak, "unit": "GB/s", "frac": achieved / hbm_peak})
    return r


def decode_config(ace, DeviceArchive, name, dev, stream, flush, steps, warmup, data=None, arc=None, stats=None,
                  seeks=0, verify_block=None, oracle_sample=None):
    """Whole decode of one workload at its stated size: device ms per step
    (L2 flushed between steps), pass breakdown, graph replay, roofline of the
    whole decode, levels; optionally plain seeks, the three-phase check of
    one block, and the oracle beside it."""
    import torch

    if data is None:
        data, arc, stats = make_workload(name)
    da = DeviceArchive(arc, max_seek_blocks=1024, device=dev)
    info = da.info
    total = info["total_size"]
    out = torch.empty(total, dtype=torch.uint8, device=dev)
    d_data = torch.from_numpy(data).to(dev)
    da.decode_all(out)
    st = da.sync()
    assert st == ace.ACE_OK, ace.ace_status_str(st)
    assert torch.equal(out, d_data), "decode differs from the original (%s)" % name
    ms = timed(stream, lambda: da.decode_all(out), steps, warmup, flush)
    assert da.sync() == ace.ACE_OK
    ms_pass = pass_times(ace, da, out, stream, flush, max(5, min(steps, 20)))
    assert da.sync() == ace.ACE_OK
    graph = torch.cuda.CUDAGraph()
    cap = torch.cuda.Stream(dev)
    cap.wait_stream(stream)
    with torch.cuda.graph(graph, stream=cap):
        ace.ace_decode_all(da.idx, out, total, da.d_scratch, da.scratch_bytes, None, cap)
    torch.cuda.synchronize()
    gms = timed(stream, graph.replay, max(10, min(steps, 50)), 2, flush)
    assert da.sync() == ace.ACE_OK
    assert torch.equal(out, d_data), "graph-replayed decode differs from the original (%s)" % name
    del graph
    peaks, peak_kind = measured_peaks()
    alg = algorithmic_bytes(arc, stats, total)
    m = statistics.mean(ms)
    sm_count = torch.cuda.get_device_properties(dev).multi_processor_count
    res = {"workload": name, "bytes": total, "blocks": info["n_blocks"], "block_size": info["block_size"],
           "archive_bytes": int(arc.size), "ratio": total / arc.size, "ms_per_step": m,
           "ms_median": statistics.median(ms), "GBps": total / (m / 1e3) / 1e9,
           "passes_ms": {"tokens": ms_pass[0], "literals": ms_pass[1], "matches": ms_pass[2]},
           "graph_replay": {"ms_median": statistics.median(gms), "GBps": total / (statistics.median(gms) / 1e3) / 1e9},
           "roofline_whole": {"algorithmic_bytes": alg["whole"], "achieved_gbs": alg["whole"] / (m / 1e3) / 1e9,
                              "peak": peaks["hbm_gbs"], "frac": alg["whole"] / (m / 1e3) / 1e9 / peaks["hbm_gbs"]},
           "roofline": roofline_of(alg, ms_pass, m, peaks, peak_kind, sm_count, None, name),
           "levels": {"count": info["n_levels"],
                      "blocks_per_level": [int(x) for x in ace.ace_index_levels(da.idx, min(info["n_levels"], 64),
                                                                                stream)]},
           "matches": stats["n_matches"], "literal_fraction": stats["literal_bytes"] / total}
    B = info["block_size"]
    if verify_block is not None:
        import oracle

        b = verify_block
        s = da.seek(b * B, B)
        assert da.sync() == ace.ACE_OK
        assert torch.equal(s, d_data[b * B:(b + 1) * B])
        lat = []
        for _ in range(20):
            t0 = time.perf_counter()
            da.seek(b * B, B, out=s)
            assert da.sync() == ace.ACE_OK
            lat.append(time.perf_counter() - t0)
        rep, _ = da.verify(b * B, B, oracle.fnv1a64(data[b * B:(b + 1) * B]))
        res["seek_block"] = {"block": b, "p50_us": 1e6 * float(np.percentile(lat[5:], 50)),
                             "three_phase": {k: int(rep[k]) for k in ("phase1_ok", "phase2_ok", "phase3_ok")}}
    if oracle_sample is not None:
        s_data, s_arc, what = oracle_sample(data, arc)
        res["cpu_baseline"] = oracle_baseline(s_data, s_arc, what)
    res["_handles"] = (da, out, d_data, data, arc, stats, alg, ms_pass)
    return res


def measure_seeks(ace, da, d_data, n_seeks, dev, stream):
    """n_seeks random single-block seeks: plain (ace_seek + ace_sync each)
    and batched 256 at a time through a decoded-block cache (a request's
    latency runs from its batch's submission to its completion)."""
    import torch
    import synth
    from paper_2606_24531_gb300.serve import SeekCache

    info = da.info
    nb, B = info["n_blocks"], info["block_size"]
    blocks = synth.uniform(SEEK_SEED, n_seeks, 0, nb - 1)
    seek_out = torch.empty(B, dtype=torch.uint8, device=dev)
    for b in synth.uniform(SEEK_SEED + 100, 20, 0, nb - 1):  # warm-up (first launches load the kernels)
        ace.ace_seek(da.idx, int(b) * B, B, seek_out, B, da.d_scratch, da.scratch_bytes, stream)
        assert ace.ace_sync(da.idx, da.d_scratch, stream) == ace.ACE_OK
    lat = []
    for i, b in enumerate(blocks):
        b = int(b)
        t0 = time.perf_counter()
        ace.ace_seek(da.idx, b * B, B, seek_out, B, da.d_scratch, da.scratch_bytes, stream)
        s = ace.ace_sync(da.idx, da.d_scratch, stream)
        lat.append(time.perf_counter() - t0)
        assert s == ace.ACE_OK
        if i % 997 == 0:
            assert torch.equal(seek_out, d_data[b * B:(b + 1) * B])
    lat_us = np.array(lat) * 1e6
    sc = SeekCache([da], n_slots=16384, max_reqs=256, pool_bytes=256 * B + 4096, device=dev)
    sc.seek_many([(0, int(b) * B, B) for b in synth.uniform(SEEK_SEED + 100, 256, 0, nb - 1)])  # warm-up
    sc.reset()
    blat, bt0 = [], time.perf_counter()
    for s0 in range(0, len(blocks), 256):
        bb = np.asarray(blocks[s0:s0 + 256], np.uint64)
        t0 = time.perf_counter()
        r = sc.plan_arrays(np.zeros(len(bb), np.uint32), bb * np.uint64(B), np.full(len(bb), B, np.uint64))
        sc.run_batch(r)
        t1 = time.perf_counter()
        blat += [t1 - t0] * len(bb)
        if s0 % 2560 == 0:
            b, o = int(bb[0]), int(r[0]["out_off"])
            assert torch.equal(sc.pool[o:o + B], d_data[b * B:(b + 1) * B])
    bwall = time.perf_counter() - bt0
    blat_us = np.array(blat) * 1e6
    sc.close()
    return {"kind": "plain: ace_seek + ace_sync per 16 KiB block", "n": len(lat),
            "p50_us": float(np.percentile(lat_us, 50)), "p99_us": float(np.percentile(lat_us, 99)),
            "mean_us": float(lat_us.mean()), "seeks_per_s": len(lat) / float(np.sum(lat)),
            "batched": {"kind": "ace_seek_batch, 256 per batch, decoded-block cache",
                        "p50_us": float(np.percentile(blat_us, 50)), "p99_us": float(np.percentile(blat_us, 99)),
                        "seeks_per_s": len(blat) / bwall},
            "paper_context_us": 334.0}


def measure_e2e(ace, da, arc, data, total, steps, dev, dist, world):
    """End to end through the C ABI from pinned host memory: every step
    uploads the archive, builds its index, decodes and downloads the output;
    E2E_INFLIGHT steps are in flight on their own streams and buffers, so one
    step's copies overlap another's decode."""
    import torch

    h_arc = torch.from_numpy(arc).pin_memory()
    slots = []
    for _ in range(E2E_INFLIGHT):
        st2 = torch.cuda.Stream(dev)
        slots.append({
            "stream": st2,
            "d_arc": torch.empty(arc.size, dtype=torch.uint8, device=dev),
            "d_index": torch.empty(da.index_bytes, dtype=torch.uint8, device=dev),
            "d_scratch": torch.empty(da.scratch_bytes, dtype=torch.uint8, device=dev),
            "out": torch.empty(total, dtype=torch.uint8, device=dev),
            "h_out": torch.empty(total, dtype=torch.uint8).pin_memory(),
            "idx": None,
        })
    for sl in slots:
        ace.ace_scratch_init(da.idx, sl["d_scratch"], da.scratch_bytes, sl["stream"])
    torch.cuda.synchronize()

    def e2e_step(sl):
        with torch.cuda.stream(sl["stream"]):
            sl["d_arc"].copy_(h_arc, non_blocking=True)
        sl["idx"] = ace.ace_index_build(sl["d_arc"], arc.size, arc[:64], sl["d_index"], da.index_bytes,
                                        sl["stream"])
        ace.ace_decode_all(sl["idx"], sl["out"], total, sl["d_scratch"], da.scratch_bytes, None, sl["stream"])
        with torch.cuda.stream(sl["stream"]):
            sl["h_out"].copy_(sl["out"], non_blocking=True)

    def e2e_finish(sl):
        st_ = ace.ace_sync(sl["idx"], sl["d_scratch"], sl["stream"])
        ace.ace_index_free(sl["idx"])
        sl["idx"] = None
        assert st_ == ace.ACE_OK

    n_e2e = max(4, min(steps, 20))
    depth = len(slots)
    for k in range(depth):  # warm-up
        e2e_step(slots[k])
    for sl in slots:
        e2e_finish(sl)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    t0 = time.perf_counter()
    for k in range(n_e2e):
        if k >= depth:
            e2e_finish(slots[k % depth])  # the step that last used this slot
        e2e_step(slots[k % depth])
    for k in range(max(0, n_e2e - depth), n_e2e):
        e2e_finish(slots[k % depth])
    e2e_s = (time.perf_counter() - t0) / n_e2e
    if dist:
        e2e_s = max_over_ranks(e2e_s, dist, dev)
    for sl in slots:
        assert np.array_equal(sl["h_out"].numpy()[:4096], data[:4096])
        assert np.array_equal(sl["h_out"].numpy()[-4096:], data[-4096:])
    del slots
    return {"value": world * total / e2e_s / 1e9, "unit": "GB/s",
            "h2d_bytes_per_step": int(arc.size), "d2h_bytes_per_step": int(total),
            "includes": "per step: H2D of the archive from pinned memory, index build, decode, "
                        "D2H of the output to pinned memory; %d steps in flight on as many streams" % E2E_INFLIGHT}


def measure_batched(ace, dev, stream, flush, max_size, reduced):
    """4,096 uneven objects in one persistent launch replayed as a CUDA graph
    (autotuned launch shape and schedule), against one ace_decode_all launch
    sequence per object; every object checked against its original."""
    import torch
    from paper_2606_24531_gb300.batch import DeviceBatch, autotune, make_objects, time_per_object

    t0 = time.perf_counter()
    bdatas, barcs, bstats = make_objects(4096, seed=4, max_size=max_size, stats=True, encoder="gpu", device=dev)
    prep_s = time.perf_counter() - t0
    db = DeviceBatch(barcs, device=dev)
    tuned = autotune(db, reps=2, cache_key=None)
    graph = db.capture()
    graph.replay()
    assert db.sync() == ace.ACE_OK
    for i, d in enumerate(bdatas):
        assert torch.equal(db.output(i), torch.from_numpy(d).to(dev)), "batched object %d differs" % i
    btotal = sum(int(d.size) for d in bdatas)
    bt = timed(stream, graph.replay, 5, 1, flush)
    assert db.sync() == ace.ACE_OK
    del graph
    per_obj_ms = time_per_object(db.items, [db.output(i) for i in range(len(bdatas))], reps=2)
    alg = sum(algorithmic_bytes(a, s, int(d.size))["whole"] for d, a, s in zip(bdatas, barcs, bstats))
    peaks, _ = measured_peaks()
    gms = float(np.median(bt))
    # the oracle on the first objects, about 128 MiB of them
    k, acc = 0, 0
    while k < len(bdatas) and acc < (128 << 20):
        acc += int(bdatas[k].size)
        k += 1
    import oracle

    t1 = time.perf_counter()
    for i in range(k):
        assert np.array_equal(oracle.decode(barcs[i]), bdatas[i])
    odt = time.perf_counter() - t1
    res = {"workload": "batched-4096-objects-4KiB-%s" % ("2MiB-reduced" if reduced else "64MiB"),
           "objects": len(bdatas), "bytes": btotal, "archive_bytes": int(sum(a.size for a in barcs)),
           "max_object": max_size, "blocks": int(sum(int(a[24:32].view(np.uint64)[0]) for a in barcs)),
           "graph_ms": gms, "graph_GBps": btotal / (gms / 1e3) / 1e9,
           "per_object_launches_ms": per_obj_ms, "per_object_GBps": btotal / (per_obj_ms / 1e3) / 1e9,
           "roofline_whole": {"algorithmic_bytes": alg, "achieved_gbs": alg / (gms / 1e3) / 1e9,
                              "peak": peaks["hbm_gbs"], "frac": alg / (gms / 1e3) / 1e9 / peaks["hbm_gbs"]},
           "tuned": {k_: tuned[k_] for k_ in ("warps_per_cta", "window", "schedule", "copy_width")},
           "host_prep_s": prep_s,
           "cpu_baseline": {"value": acc / odt / 1e9, "unit": "GB/s", "cores": 1, "kind": "oracle",
                            "sample": "the first %d objects (%d bytes), one thread (%.2f s)" % (k, acc, odt)}}
    if reduced:
        res["reduced"] = "objects capped at %d bytes (--quick)" % max_size
    db.close()
    return res


def measure_serve(ace, DeviceArchive, dev, arch_bytes, budget, reduced):
    """Seek serving: 8 resident archives (two per profile, 16 KiB blocks,
    5-byte offsets), Poisson arrivals of seeks at uniform offsets with
    log-uniform lengths from one block to 1 MiB, continuous batching under a
    device working-set budget, against one ace_seek per request; a sample of
    results checked against the plain path (alone vs in the mix)."""
    import threading

    import torch
    import synth
    from paper_2606_24531_gb300.serve import Server, plain_latencies

    profs = ["fastq", "fastq", "genome", "genome", "text", "text", "mixed", "mixed"]
    t0 = time.perf_counter()
    datas = [None] * len(profs)

    def gen(k):
        datas[k] = synth.generate(profs[k], arch_bytes, 10 + k)

    th = [threading.Thread(target=gen, args=(k,)) for k in range(len(profs))]
    for t in th:
        t.start()
    for t in th:
        t.join()
    sdas = []
    for k, p in enumerate(profs):  # encoded on the GPU, the archives staying resident
        arc = ace.ace_encode_gpu(torch.from_numpy(datas[k]).to(dev), 14, MIN_MATCH[p], off_width=5)
        sdas.append(DeviceArchive(arc.cpu().numpy(), max_seek_blocks=1024, device=dev))
        del arc
        torch.cuda.empty_cache()
    prep_s = time.perf_counter() - t0
    sizes = np.array([x.total for x in sdas], np.uint64)
    srv = Server(sdas, budget_bytes=budget, device=dev)
    tq, aq, cq, lq = synth.requests(6, 3000, 3e4, sizes, 1 << 14, 1 << 20)
    srv.run(tq, aq, cq, lq, time_limit_s=2.0)  # warm-up (first launches, first cached blocks), not reported
    rows = []
    rng = np.random.default_rng(9)
    for lam in (1e4, 3e4, 1e5, 3e5, 1e6):
        nreq = int(min(100000, max(20000, 2 * lam)))
        tq, aq, cq, lq = synth.requests(5, nreq, lam, sizes, 1 << 14, 1 << 20)
        keep = set(int(x) for x in rng.integers(0, nreq, 16))
        res = srv.run(tq, aq, cq, lq, keep=keep, time_limit_s=4.0)
        lt = res["latency_ns"][res["latency_ns"] >= 0] / 1e3
        for rid, got in res["kept"].items():  # the same bytes alone (plain seek) as in the mix
            a, c, n = int(aq[rid]), int(cq[rid]), int(lq[rid])
            assert np.array_equal(got, datas[a][c:c + n]), "served result %d differs" % rid
        rows.append({"rate_per_s": lam, "requests": nreq, "served": res["served"], "rejected": res["rejected"],
                     "p50_us": float(np.percentile(lt, 50)) if lt.size else None,
                     "p99_us": float(np.percentile(lt, 99)) if lt.size else None,
                     "GBps": res["bytes"] / res["seconds"] / 1e9, "batches": res["batches"],
                     "evicted_blocks": res["evicted"], "checked_alone_vs_mix": len(res["kept"])})
    tq, aq, cq, lq = synth.requests(5, 500, 1e4, sizes, 1 << 14, 1 << 20)
    pl = plain_latencies(sdas, [x.d_scratch for x in sdas], aq, cq, lq) / 1e3
    out = {"workload": "serve-8x%dMiB-16KiB-blocks%s" % (arch_bytes >> 20, "-reduced" if reduced else ""),
           "archives": len(sdas), "archive_bytes": arch_bytes, "decompressed_total": int(sizes.sum()),
           "compressed_resident": int(sum(x.d_arc.numel() for x in sdas)),
           "budget_bytes": budget, "working_set_bytes": srv.working_set_bytes(), "streams": srv.n_streams,
           "by_rate": rows, "host_prep_s": prep_s,
           "plain": {"p50_us": float(np.percentile(pl, 50)), "p99_us": float(np.percentile(pl, 99)),
                     "GBps": float(lq.sum()) / (float(pl.sum()) / 1e6) / 1e9}}
    if reduced:
        out["reduced"] = "archives of %d bytes under a %d-byte budget (--quick)" % (arch_bytes, budget)
    srv.close()
    for x in sdas:
        x.close()
    del datas
    torch.cuda.synchronize()
    return out


def measure_beyond_vram(ace, dev, stream, total_bytes, reduced):
    """Range decode of an archive kept in host memory (the paper's 50 GB
    genome case, where output plus archive exceed a GPU's memory): the
    archive's bytes pinned and mapped, read by the GPU in place; the index
    built on the device.  Times the range decode of blocks 0..1000, a long
    range streamed to host memory in sub-ranges, and a whole decode into
    device memory with the archive still on the host."""
    import torch
    import synth
    from paper_2606_24531_gb300.archive import HostArchive

    t0 = time.perf_counter()
    data = synth.generate("genome", total_bytes, 3)
    d_in = torch.from_numpy(data).to(dev)
    arc = ace.ace_encode_gpu(d_in, 14, 20).cpu().numpy()  # on the GPU; the archive then lives on the host
    del d_in
    torch.cuda.empty_cache()
    prep_s = time.perf_counter() - t0
    t0 = time.perf_counter()
    ha = HostArchive(arc, max_seek_blocks=4096, device=dev)
    index_ms = 1e3 * (time.perf_counter() - t0)
    B = ha.block_size
    first = torch.empty(1001 * B, dtype=torch.uint8, device=dev)
    lat = []
    for k in range(13):
        t1 = time.perf_counter()
        ace.ace_seek(ha.idx, 0, 1001 * B, first, first.numel(), ha.d_scratch, ha.scratch_bytes, stream)
        st = ace.ace_sync(ha.idx, ha.d_scratch, stream)
        lat.append(time.perf_counter() - t1)
        assert st == ace.ACE_OK
    assert torch.equal(first, torch.from_numpy(data[:1001 * B]).to(dev))
    span = min(8 << 30, ha.total)
    h_out = torch.empty(span, dtype=torch.uint8).pin_memory()
    ha.decode_range_to_host(0, 64 * B, h_out[:64 * B], chunk_blocks=4096)  # warm-up
    t1 = time.perf_counter()
    ha.decode_range_to_host(0, span, h_out, chunk_blocks=4096)
    stream_s = time.perf_counter() - t1
    hv = h_out.numpy()
    for c in np.linspace(0, span - 4096, 64).astype(np.int64):
        assert np.array_equal(hv[c:c + 4096], data[c:c + 4096]), "streamed range differs at %d" % c
    del h_out, hv
    whole = None
    free, _ = torch.cuda.mem_get_info(dev)
    if ha.total + (2 << 30) < free:
        out = torch.empty(ha.total, dtype=torch.uint8, device=dev)
        ha.decode_all(out)
        assert ha.sync() == ace.ACE_OK
        ms = timed(stream, lambda: ha.decode_all(out), 3, 1)
        assert ha.sync() == ace.ACE_OK
        for c in np.linspace(0, ha.total - 4096, 64).astype(np.int64):
            assert torch.equal(out[c:c + 4096].cpu(), torch.from_numpy(data[c:c + 4096]))
        whole = {"ms": statistics.median(ms), "GBps": ha.total / (statistics.median(ms) / 1e3) / 1e9,
                 "where": "archive in host memory, output in device memory"}
        del out
    res = {"workload": "genome-%dB-16KiB-blocks-host-resident%s" % (total_bytes, "-reduced" if reduced else ""),
           "bytes": ha.total, "blocks": ha.info["n_blocks"], "archive_bytes": int(arc.size),
           "index_build_ms": index_ms, "host_prep_s": prep_s,
           "range_blocks_0_1000": {"p50_ms": 1e3 * float(np.percentile(lat[3:], 50)),
                                   "p99_ms": 1e3 * float(np.percentile(lat[3:], 99)),
                                   "paper_context_ms": 0.654},
           "streamed_to_host": {"bytes": span, "seconds": stream_s, "GBps": span / stream_s / 1e9,
                                "sub_range_blocks": 4096},
           "whole_decode": whole}
    ha.close()
    del data, arc
    torch.cuda.empty_cache()
    return res


def measure_encoder(ace, dev, stream):
    """The GPU encoder on the headline workload and the genome: encode time
    (input resident in device memory, archive left there), ratio beside the
    host encoder's, and the archive checked by a GPU decode."""
    import torch
    from paper_2606_24531_gb300.archive import DeviceArchive

    rows = {}
    for name in ("fastq-256MiB-16KiB-blocks", "genome-1GiB-16KiB-blocks"):
        data, log2b, mm = make_data(name)
        d_in = torch.from_numpy(data).to(dev)
        ace.ace_encode_gpu(d_in, log2b, mm)  # warm-up
        torch.cuda.synchronize()
        ts = []
        for _ in range(3):
            t0 = time.perf_counter()
            arc, st = ace.ace_encode_gpu(d_in, log2b, mm, stats=True)
            torch.cuda.synchronize()
            ts.append(time.perf_counter() - t0)
        h = arc.cpu().numpy()
        t0 = time.perf_counter()
        host = ace.ace_encode(data, log2b, mm)
        host_s = time.perf_counter() - t0
        da = DeviceArchive(h, device=dev)
        out = da.decode_all()
        assert da.sync() == ace.ACE_OK and torch.equal(out[:data.size], d_in), "GPU-encoded archive differs"
        da.close()
        rows[name] = {"gpu_encode_s": statistics.median(ts), "gpu_GBps": data.size / statistics.median(ts) / 1e9,
                      "ratio": data.size / h.size, "host_encode_s": host_s, "host_ratio": data.size / host.size,
                      "host_threads": os.cpu_count(), "levels": st["n_levels"]}
        del d_in, arc, out
        torch.cuda.empty_cache()
    return rows


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--seeks", type=int, default=10000)
    ap.add_argument("--workload", default=WORKLOAD, choices=sorted(WORKLOADS),
                    help="headline decode workload (the default is the headline one)")
    ap.add_argument("--no-extras", action="store_true", help="decode steps only (for profiler runs)")
    ap.add_argument("--no-serve", action="store_true", help="skip the serving measurement")
    ap.add_argument("--no-batched", action="store_true", help="skip the batched measurement")
    ap.add_argument("--no-beyond-vram", action="store_true", help="skip the host-resident range decode")
    ap.add_argument("--quick", action="store_true",
                    help="reduced batched (2 MiB objects) and serving (256 MiB archives) configurations")
    args = ap.parse_args()
    assert args.warmup >= 3 or args.no_extras, "at least 3 warm-up steps"

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank)
        return

    import torch
    import __graft_entry__

    __graft_entry__.build()
    from paper_2606_24531_gb300 import ace
    from paper_2606_24531_gb300.archive import DeviceArchive

    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream(dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    sm_count = torch.cuda.get_device_properties(dev).multi_processor_count
    peaks, peak_kind = measured_peaks()

    # ---- the headline: whole decode of the workload, steps timed between barriers
    data, arc, stats = make_workload(args.workload)
    t0 = time.perf_counter()
    da = DeviceArchive(arc, max_seek_blocks=512, device=dev)
    index_ms = 1e3 * (time.perf_counter() - t0)
    info = da.info
    total = info["total_size"]
    out = torch.empty(total, dtype=torch.uint8, device=dev)
    d_data = torch.from_numpy(data).to(dev)
    da.decode_all(out)
    st = da.sync()
    assert st == ace.ACE_OK, ace.ace_status_str(st)
    assert torch.equal(out, d_data), "decode differs from the original"
    for _ in range(args.warmup):
        da.decode_all(out)
    torch.cuda.synchronize()
    sampler = ClockSampler(local)
    time.sleep(0.2)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    times = timed(stream, lambda: da.decode_all(out), args.steps, 0, flush)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    clocks = sampler.stop()
    st = da.sync()
    assert st == ace.ACE_OK, ace.ace_status_str(st)
    assert torch.equal(out, d_data), "decode differs from the original after the timed steps"
    ms = statistics.mean(times)
    if dist:
        ms = max_over_ranks(ms, dist, dev)
    value = world * total / (ms / 1e3) / 1e9
    ms_pass = pass_times(ace, da, out, stream, flush, max(5, min(args.steps, 20)))
    assert da.sync() == ace.ACE_OK
    alg = algorithmic_bytes(arc, stats, total)
    result = {
        "metric": METRIC, "value": value, "unit": "GB/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "u8", "data": "synthetic",
        "config": {"workload": args.workload, "blocks": info["n_blocks"], "block_size": info["block_size"],
                   "archive_bytes": int(arc.size), "ratio": total / arc.size, "levels": info["n_levels"],
                   "literal_fraction": stats["literal_bytes"] / total, "matches": stats["n_matches"],
                   "schedule": "passes (tokens, literals, matches by level)",
                   "l2": "flushed between timed steps (256 MiB fill)", "parallelism": "replicas"},
        "roofline": roofline_of(alg, ms_pass, ms, peaks, peak_kind, sm_count, clocks, args.workload),
        "gpu_launches": (3 + info["n_levels"]) * args.steps,  # per step: header reset, tokens, literals, a match launch per level
        "clocks": clocks,
        "index_build_ms": index_ms,
        "ms_median": statistics.median(times),
        "sm_count": sm_count,
        "levels": {"count": info["n_levels"],
                   "blocks_per_level": [int(x) for x in ace.ace_index_levels(da.idx, min(info["n_levels"], 64),
                                                                             stream)]},
    }
    if not args.no_extras:
        fused = timed(stream, lambda: da.decode_all(out, tune=ace.make_tune(schedule=ace.ACE_SCHEDULE_FUSED)),
                      10, 2, flush)
        assert da.sync() == ace.ACE_OK and torch.equal(out, d_data)
        result["fused_schedule"] = {"ms_median": statistics.median(fused),
                                    "GBps": total / (statistics.median(fused) / 1e3) / 1e9}
        result["seek"] = measure_seeks(ace, da, d_data, args.seeks, dev, stream)
        result["e2e"] = measure_e2e(ace, da, arc, data, total, args.steps, dev, dist, world)
        if rank == 0:
            result["cpu_baseline"] = oracle_baseline(data, arc, "the whole archive")
            result["cpu_baseline"].update({"cpu": os.uname().machine, "cpu_model": cpu_model(),
                                           "nproc": os.cpu_count(), "affinity": len(os.sched_getaffinity(0))})
        da.close()
        del out, d_data
        # ---- the other configurations, each at its stated size
        cfgs = {}
        small = decode_config(ace, DeviceArchive, "mixed-1MiB-16KiB-blocks", dev, stream, flush, 20, 3,
                              verify_block=37, oracle_sample=lambda d, a: (d, a, "the whole archive"))
        small.pop("_handles")
        cfgs["plain_small"] = small
        gen = decode_config(ace, DeviceArchive, "genome-1GiB-16KiB-blocks", dev, stream, flush, 10, 3,
                            oracle_sample=lambda d, a: (d, a, "the whole archive"))
        gen.pop("_handles")
        cfgs["genome"] = gen
        torch.cuda.empty_cache()
        cfgs["gpu_encoder"] = measure_encoder(ace, dev, stream)
        if not args.no_batched:
            cfgs["batched"] = measure_batched(ace, dev, stream, flush, (1 << 21) if args.quick else (1 << 26),
                                              args.quick)
            torch.cuda.empty_cache()
        if not args.no_serve:
            if args.quick:
                cfgs["serve"] = measure_serve(ace, DeviceArchive, dev, 256 << 20, 4 * 10**9, True)
            else:
                cfgs["serve"] = measure_serve(ace, DeviceArchive, dev, 5 << 30, 20 * 10**9, False)
            torch.cuda.empty_cache()
        if not args.no_beyond_vram:
            cfgs["beyond_vram"] = measure_beyond_vram(ace, dev, stream, (4 << 30) if args.quick else 50 * 10**9,
                                                      args.quick)
        result["configs"] = cfgs
    if rank == 0:
        print(json.dumps(result), flush=True)
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
