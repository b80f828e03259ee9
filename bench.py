#!/usr/bin/env python
"""Benchmark: whole-archive two-layer decode of FASTQ-shaped data.

Workload: 256 MiB of synthetic FASTQ (seed 1; header/150-base read/'+'/
quality records), 16 KiB blocks (16,384 blocks), encoded by the library's
host encoder.  A step is one ace_decode_all: every block's three rANS
streams decoded and its literals and absolute-offset matches resolved into
the output, on the GPU.  Also measured: 10,000 random single-block seeks
(seed 2), one launch sequence plus a synchronise per seek; the end-to-end
time through the C ABI from pinned host memory; the CPU oracle on the host
cores.

Prints one JSON line.  Under torchrun each rank decodes its own replica of
the archive (replicas only: no data-path collective).
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
}
WORKLOAD = "fastq-256MiB-16KiB-blocks"
SEEK_SEED = 2
REF_SAMPLE = 8 << 20  # the reference arm decodes this many bytes of the workload per step
E2E_INFLIGHT = 3      # end-to-end steps in flight, each with its own stream and device buffers
SPEC_HBM_GBS = 7900.0  # nominal GB300 HBM3e bandwidth (spec sheet)
METRIC = "decompressed GB/s (% HBM roofline); 16KB seek p50/p99 us, batched vs plain"
KERNEL_SOURCES = ["paper_2606_24531_gb300/csrc/ace.cu", "paper_2606_24531_gb300/csrc/ace_device.cuh"]
PROFILE_SUMMARY = os.path.join(ROOT, "profiles", "literal_pass_fastq256.txt")


def kernel_sha():
    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        with open(os.path.join(ROOT, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def profiled_traffic():
    """dram read+write bytes per literal-pass launch from the committed ncu summary,
    if it was taken on the current kernel sources."""
    try:
        kv = {}
        with open(PROFILE_SUMMARY) as f:
            for ln in f:
                if ":" in ln:
                    k, v = ln.split(":", 1)
                    kv[k.strip()] = v.strip()
        if kv.get("kernel_sources_sha256") == kernel_sha():
            return int(kv["traffic_bytes_per_launch"])
    except (OSError, KeyError, ValueError):
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
        return {"hbm_gbs": 6800.0}, "fallback"


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


def make_workload(name, limit=None):
    """The workload's data and archive; limit takes a prefix of the data."""
    import synth
    from paper_2606_24531_gb300 import ace

    profile, total, seed, log2b, min_match = WORKLOADS[name]
    data = synth.generate(profile, total, seed)
    if limit is not None and limit < data.size:
        data = np.ascontiguousarray(data[:limit])
    arc, stats = ace.ace_encode(data, log2b, min_match, stats=True)
    return data, arc, stats


def max_over_ranks(x, dist, device):
    """The largest of every rank's x (the job's step time is its slowest rank's)."""
    import torch

    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def run_reference(args, rank):
    """The oracle (plain sequential C decoder) on the host cores."""
    if rank != 0:
        return
    import oracle

    data, arc, _ = make_workload(args.workload, REF_SAMPLE)
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
    sample = "the first %d bytes of the workload, encoded alike, decoded whole each step, one thread" % data.size
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": gbs, "unit": "GB/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "u8", "data": "synthetic",
        "config": {"workload": args.workload, "blocks": int(data.size >> WORKLOADS[args.workload][3])},
        "cpu_baseline": {"value": gbs, "unit": "GB/s", "cores": 1, "kind": "oracle", "sample": sample},
        "e2e": {"value": gbs, "unit": "GB/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--seeks", type=int, default=10000)
    ap.add_argument("--workload", default=WORKLOAD, choices=sorted(WORKLOADS),
                    help="decode workload (the default is the headline one)")
    ap.add_argument("--no-extras", action="store_true", help="decode steps only (for profiler runs)")
    ap.add_argument("--no-serve", action="store_true", help="skip the serving measurement")
    ap.add_argument("--serve-archive-mib", type=int, default=256, help="size of each served archive")
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

    data, arc, stats = make_workload(args.workload)
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream(dev)
    t0 = time.perf_counter()
    da = DeviceArchive(arc, max_seek_blocks=512, device=dev)
    index_ms = 1e3 * (time.perf_counter() - t0)
    info = da.info
    total = info["total_size"]
    out = torch.empty(total, dtype=torch.uint8, device=dev)
    d_data = torch.from_numpy(data).to(dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)

    # correctness before timing: bit-exact against the original bytes
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
    # one step = ace_decode_all, issued as its three passes so that events
    # between them time each pass on its own
    ev = [tuple(torch.cuda.Event(enable_timing=True) for _ in range(4)) for _ in range(args.steps)]
    passes = (ace.ACE_PASS_TOKENS, ace.ACE_PASS_LITERALS, ace.ACE_PASS_MATCH)
    for k in range(args.steps):
        flush.fill_(k & 255)  # L2 flush between timed steps, outside the events
        ev[k][0].record(stream)
        for p in passes:
            ace.ace_decode_pass(da.idx, p, out, total, da.d_scratch, da.scratch_bytes, None, stream)
            ev[k][p + 1].record(stream)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    clocks = sampler.stop()
    st = da.sync()
    assert st == ace.ACE_OK, ace.ace_status_str(st)
    times = [e[0].elapsed_time(e[3]) for e in ev]
    ms = statistics.mean(times)
    ms_median = statistics.median(times)
    ms_pass = [statistics.mean(e[p].elapsed_time(e[p + 1]) for e in ev) for p in range(3)]
    if dist:
        ms = max_over_ranks(ms, dist, dev)
    value = world * total / (ms / 1e3) / 1e9

    peaks, peak_kind = measured_peaks()
    hdr = arc[:64].view(np.uint64)
    deps_bytes = int(hdr[6]) - int(hdr[5])  # payload_off - deps_off: not read by a whole decode
    # algorithmic bytes per pass: the token pass reads the directory and the
    # length and offset streams and writes a 16-byte record per match; the
    # literal pass reads the directory, the literal streams and the records
    # and writes every literal; the match pass reads the records and every
    # match's source bytes and writes the matched bytes
    nb = info["n_blocks"]
    dir_off = int(hdr[4])
    sb = arc[dir_off:dir_off + 64 * nb].view(np.uint32).reshape(nb, 16)[:, 6:9].astype(np.int64).sum(axis=0)
    rec_b = 16 * stats["n_matches"]
    alg = [64 * nb + int(sb[1] + sb[2]) + rec_b,
           64 * nb + int(sb[0]) + rec_b + stats["literal_bytes"],
           rec_b + stats["match_src_bytes"] + stats["match_bytes"]]
    # the whole decode by the plain definition: archive bytes read (the
    # dependency table aside) + match source bytes (min(len, distance); the
    # upper variant counts len) + output bytes written
    whole = (arc.size - deps_bytes) + stats["match_src_bytes"] + total
    whole_upper = (arc.size - deps_bytes) + stats["match_bytes"] + total
    names = ["decode_kernel<false, PASS_TOKENS>", "decode_kernel<false, PASS_LITERALS>", "match_level_kernel"]
    top = max(range(3), key=lambda p: ms_pass[p])
    achieved = alg[top] / (ms_pass[top] / 1e3) / 1e9
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                "frac": achieved / peaks["hbm_gbs"], "traffic": profiled_traffic() if top == 1 else None,
                "kernel": names[top], "algorithmic_bytes": alg[top], "peak_kind": peak_kind,
                "passes": {n: {"ms": ms_pass[p], "algorithmic_bytes": alg[p],
                               "achieved_gbs": alg[p] / (ms_pass[p] / 1e3) / 1e9}
                           for p, n in enumerate(["tokens", "literals", "matches"])},
                "whole_decode": {"algorithmic_bytes": whole, "algorithmic_bytes_upper": whole_upper,
                                 "achieved_gbs": whole / (ms / 1e3) / 1e9,
                                 "frac": whole / (ms / 1e3) / 1e9 / peaks["hbm_gbs"]},
                "spec_sheet": {"peak_gbs": SPEC_HBM_GBS, "frac_of_spec": achieved / SPEC_HBM_GBS,
                               "label": "fraction of the nominal HBM3e bandwidth, not a measurement"}}

    result = {
        "metric": METRIC, "value": value, "unit": "GB/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "u8", "data": "synthetic",
        "config": {"workload": args.workload, "blocks": info["n_blocks"], "block_size": info["block_size"],
                   "archive_bytes": int(arc.size), "ratio": total / arc.size, "levels": info["n_levels"],
                   "literal_fraction": stats["literal_bytes"] / total, "matches": stats["n_matches"],
                   "l2": "flushed between timed steps (256 MiB fill)", "parallelism": "replicas"},
        "roofline": roofline,
        "gpu_launches": (3 + info["n_levels"]) * args.steps,  # per step: header reset, tokens, literals, a match launch per level
        "clocks": clocks,
        "index_build_ms": index_ms,
        "ms_median": ms_median,
        "sm_count": torch.cuda.get_device_properties(dev).multi_processor_count,
        "levels": {"count": info["n_levels"],
                   "blocks_per_level": [int(x) for x in ace.ace_index_levels(da.idx, min(info["n_levels"], 64),
                                                                             stream)]},
    }

    if not args.no_extras:
        # the same decode replayed from a CUDA graph: launch overhead out of
        # the step (it matters for small archives)
        graph = torch.cuda.CUDAGraph()
        cap = torch.cuda.Stream(dev)
        cap.wait_stream(stream)
        with torch.cuda.graph(graph, stream=cap):
            ace.ace_decode_all(da.idx, out, total, da.d_scratch, da.scratch_bytes, None, cap)
        torch.cuda.synchronize()
        gts = []
        for k in range(max(10, min(args.steps, 50))):
            flush.fill_(k & 255)
            g0, g1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            g0.record(stream)
            graph.replay()
            g1.record(stream)
            g1.synchronize()
            gts.append(g0.elapsed_time(g1))
        st = da.sync()
        assert st == ace.ACE_OK, ace.ace_status_str(st)
        assert torch.equal(out, d_data), "graph-replayed decode differs from the original"
        result["graph_replay"] = {"ms_median": statistics.median(gts),
                                  "GBps": total / (statistics.median(gts) / 1e3) / 1e9}
        del graph

        # plain seeks: one seek launch sequence + a synchronise per request
        import synth

        nb = info["n_blocks"]
        blocks = synth.uniform(SEEK_SEED, args.seeks, 0, nb - 1)
        B = info["block_size"]
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
        # batched: the same 10,000 seeks in batches of 256 through one
        # decoded-block cache (one closure, one decode, one copy per batch);
        # a request's latency runs from its batch's submission to completion
        from paper_2606_24531_gb300.serve import SeekCache

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
        result["seek"] = {"kind": "plain: ace_seek + ace_sync per 16 KiB block", "n": len(lat),
                          "p50_us": float(np.percentile(lat_us, 50)),
                          "p99_us": float(np.percentile(lat_us, 99)),
                          "mean_us": float(lat_us.mean()),
                          "seeks_per_s": len(lat) / float(np.sum(lat)),
                          "batched": {"kind": "ace_seek_batch, 256 per batch, decoded-block cache",
                                      "p50_us": float(np.percentile(blat_us, 50)),
                                      "p99_us": float(np.percentile(blat_us, 99)),
                                      "seeks_per_s": len(blat) / bwall},
                          "paper_context_us": 334.0}

        # end to end through the C ABI from pinned host memory: every step
        # uploads the archive, builds its index, decodes and downloads the
        # output; E2E_INFLIGHT steps are in flight on their own streams and
        # device buffers, so one step's copies overlap another's decode
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

        n_e2e = max(4, min(args.steps, 20))
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
        result["e2e"] = {"value": world * total / e2e_s / 1e9, "unit": "GB/s",
                         "h2d_bytes_per_step": int(arc.size), "d2h_bytes_per_step": int(total),
                         "includes": "per step: H2D of the archive from pinned memory, index build, decode, "
                                     "D2H of the output to pinned memory; %d steps in flight on as many streams"
                                     % E2E_INFLIGHT}
        del slots

        # batched: 4,096 uneven objects (log-uniform 4 KiB .. 2 MiB, four
        # profiles, 4/16/64 KiB blocks) in one persistent launch replayed as a
        # CUDA graph, against one ace_decode_all launch per object
        from paper_2606_24531_gb300.batch import DeviceBatch, autotune, make_objects, time_per_object

        bdatas, barcs = make_objects(4096, seed=4, max_size=1 << 21)
        db = DeviceBatch(barcs, device=dev)
        tuned = autotune(db, reps=2, cache_key=None)
        graph = db.capture()
        graph.replay()
        assert db.sync() == ace.ACE_OK
        btotal = sum(d.size for d in bdatas)
        chk = torch.cat([torch.from_numpy(d) for d in bdatas[:64]]).to(dev)
        assert torch.equal(torch.cat([db.output(i) for i in range(64)]), chk)
        bt = []
        for _ in range(5):
            flush.fill_(1)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            graph.replay()
            e1.record(stream)
            e1.synchronize()
            bt.append(e0.elapsed_time(e1))
        per_obj_ms = time_per_object(db.items, [db.output(i) for i in range(len(bdatas))], reps=2)
        result["batched"] = {"objects": len(bdatas), "bytes": btotal, "max_object": 1 << 21,
                             "graph_ms": float(np.median(bt)),
                             "graph_GBps": btotal / (float(np.median(bt)) / 1e3) / 1e9,
                             "per_object_launches_ms": per_obj_ms,
                             "per_object_GBps": btotal / (per_obj_ms / 1e3) / 1e9,
                             "tuned": {k: tuned[k] for k in ("warps_per_cta", "window")}}
        db.close()

        # serving: 8 resident archives (two per profile, 16 KiB blocks),
        # Poisson arrivals of seeks at uniform offsets with log-uniform lengths
        # from one block to 1 MiB, continuous batching on two streams under a
        # device working-set budget, against one ace_seek per request
        if not args.no_serve:
            import synth
            from paper_2606_24531_gb300.serve import Server, plain_latencies

            profs = ["fastq", "fastq", "genome", "genome", "text", "text", "mixed", "mixed"]
            mmp = {"fastq": 16, "genome": 20, "text": 4, "mixed": 4}
            arch_bytes = args.serve_archive_mib << 20
            sdas = []
            for k, p in enumerate(profs):
                dk = synth.generate(p, arch_bytes, 10 + k)
                sdas.append(DeviceArchive(ace.ace_encode(dk, 14, mmp[p]), max_seek_blocks=1024, device=dev))
            sizes = np.array([x.total for x in sdas], np.uint64)
            budget = min(20 << 30, 4 << 30)
            srv = Server(sdas, budget_bytes=budget, n_streams=2, max_batch=256, pool_bytes=96 << 20, device=dev)
            rows = []
            for lam in (1e4, 3e4, 1e5, 3e5, 1e6):
                nreq = int(min(max(lam * 1.0, 2000), 100000))
                tq, aq, cq, lq = synth.requests(5, nreq, lam, sizes, 1 << 14, 1 << 20)
                res = srv.run(tq, aq, cq, lq, time_limit_s=3.0)
                lt = res["latency_ns"][res["latency_ns"] >= 0] / 1e3
                rows.append({"rate_per_s": lam, "requests": nreq, "served": res["served"],
                             "p50_us": float(np.percentile(lt, 50)), "p99_us": float(np.percentile(lt, 99)),
                             "GBps": res["bytes"] / res["seconds"] / 1e9, "batches": res["batches"],
                             "cache_resets": res["resets"]})
            tq, aq, cq, lq = synth.requests(5, 500, 1e4, sizes, 1 << 14, 1 << 20)
            pl = plain_latencies(sdas, [x.d_scratch for x in sdas], aq, cq, lq) / 1e3
            srv.close()
            result["serve"] = {"archives": len(sdas), "archive_bytes": arch_bytes,
                               "decompressed_total": int(sizes.sum()), "budget_bytes": budget,
                               "working_set_bytes": srv.working_set_bytes(), "by_rate": rows,
                               "plain": {"p50_us": float(np.percentile(pl, 50)),
                                         "p99_us": float(np.percentile(pl, 99)),
                                         "GBps": float(lq.sum()) / (float(pl.sum()) / 1e6) / 1e9}}
            for x in sdas:
                x.close()

        # the oracle on the host cores (rank 0 only)
        if rank == 0:
            import oracle

            # bounded: workloads above 256 MiB are sampled by their first 256 MiB
            s_data, s_arc = data, arc
            if data.size > (1 << 28):
                s_data, s_arc, _ = make_workload(args.workload, 1 << 28)
            t0 = time.perf_counter()
            ref = oracle.decode(s_arc)
            dt = time.perf_counter() - t0
            assert np.array_equal(ref, s_data)
            what = ("the whole archive" if s_data.size == data.size
                    else "the first %d bytes of the workload, encoded alike" % s_data.size)
            # the oracle's seek: its closure decoded from the archive alone
            sb = synth.uniform(SEEK_SEED + 200, 10, 0, (s_data.size >> WORKLOADS[args.workload][3]) - 1)
            Bs = 1 << WORKLOADS[args.workload][3]
            t0 = time.perf_counter()
            for b in sb:
                oracle.seek(s_arc, int(b) * Bs, Bs)
            seek_ms = 1e3 * (time.perf_counter() - t0) / len(sb)
            result["cpu_baseline"] = {"value": s_data.size / dt / 1e9, "unit": "GB/s", "cores": 1,
                                      "kind": "oracle",
                                      "sample": "%s, one thread (%.1f s)" % (what, dt),
                                      "seek_ms": seek_ms, "cpu": os.uname().machine, "cpu_model": cpu_model(),
                                      "nproc": os.cpu_count(), "affinity": len(os.sched_getaffinity(0))}
    if rank == 0:
        print(json.dumps(result), flush=True)
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
