#!/usr/bin/env python
"""Read-mapping throughput on one GB300: reads/s mapped, all hits, k = 5 % of 100 bp.

Workload (default): human-scale synthetic genome of 3.1 Gbp (45 % repeat families, 1 % tandem
runs) and 10,000,000 reads of 100 bp (95 % sampled with 1-4 % errors, 5 % random), indexed in
device-resident batches of 2^20 reads, q = 16, k = 5, all-hits mode.  One step maps all
10,000,000 reads (10 batches: peanut_index_reads + peanut_map each).

  value : reads/s with the reads already in device memory (peanut_index_reads_device +
          peanut_map_device), timed with CUDA events on the mapping stream.
  e2e   : reads/s through the host API (peanut_index_reads from pinned host memory +
          peanut_map returning host arrays), host<->device copies inside the timed region.
  roofline : the verification kernel (the largest launch-list share), algorithmic INT32
          operations per launch over its CUDA-event duration, against the INT32 issue peak derived
          from the SM count and clock; roofline_scan: the two reference-scan kernels, algorithmic
          bytes per launch against the measured HBM copy bandwidth.
  cpu_baseline : the CPU oracle on a bounded sample of the same workload (see --help).

Launch: `python bench.py [--gpus N --steps K --warmup W]`; for N > 1 under torchrun, each rank
maps its own 10,000,000 reads against its own copy of the reference (weak scaling, no data-path
collective).  `--impl reference` times the CPU oracle instead (rank 0 only).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "reads/sec mapped (all-hits, k=5%) on 1 GB300 vs oracle; p50/p99 request latency"
UNIT = "reads/s"
HIT_BYTES = 4 + 1 + 8 + 1  # read_id, strand, end_pos, dist of one result
N_SM, INT32_LANES_PER_SM, SM_MAX_MHZ = 152, 128, 2070.0  # GB300


def parse_args():
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", default="human_3g1_10m")
    ap.add_argument("--ref-len", type=int, default=None, help="scale the reference down (same recipe)")
    ap.add_argument("--reads", type=int, default=None, help="scale the read count down")
    ap.add_argument("--batch", type=int, default=1 << 20)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-slice", type=int, default=30_000_000,
                    help="reference prefix (bp) of the CPU-baseline sample")
    return ap.parse_args()


def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons while the timed region runs."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() in ("active", "0x1", "1"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm)}


def traffic_per_unit(name: str, kernel_src_sha: str):
    """DRAM bytes per unit of work of a kernel, from the committed ncu summary
    profiles/<name>_traffic.json, if it was taken on the current kernel source; else None."""
    p = os.path.join(ROOT, "profiles", f"{name}_traffic.json")
    try:
        with open(p) as f:
            d = json.load(f)
        if d.get("source_sha256") != kernel_src_sha:
            return None
        return float(d["dram_bytes_per_word_column"])
    except Exception:
        return None


def source_sha() -> str:
    h = hashlib.sha256()
    for f in ("map.cu", "prims.cuh", "internal.cuh"):
        with open(os.path.join(ROOT, "paper_1403_1706_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()


def make_inputs(args, rank):
    import synth
    w = synth.WORKLOADS[args.workload]
    n = args.ref_len or w["ref_len"]
    nr = args.reads or w["n_reads"]
    t0 = time.time()
    ref = synth.make_reference(n, 1403, w["repeat_frac"], w["tandem_frac"])
    seed = 1706 + list(synth.WORKLOADS).index(args.workload) + 1000 * rank
    reads = synth.make_reads(ref, nr, seed, lengths=w["lengths"], sub_rate=w.get("sub_rate"),
                             indel_rate=w.get("indel_rate"), rate_range=w.get("rate_range"),
                             random_frac=w["random_frac"])
    return ref, reads, w, time.time() - t0


def cpu_baseline(ref, reads, w, slice_len, batch):
    """The oracle on a bounded sample: the reads whose planted origin lies in the first
    `slice_len` bases (plus the unmappable ones at their natural rate), as many as one read
    batch holds per base of reference, mapped against that prefix; single thread."""
    import oracle
    n = ref.size
    slice_len = min(slice_len, n)
    want = max(1, int(round(batch * slice_len / n)))
    inside = (reads.truth_end >= 0) & (reads.truth_end < slice_len - 1)
    rnd = reads.truth_end < 0
    idx = np.flatnonzero(inside | (rnd & (np.arange(reads.n) % max(1, n // slice_len) == 0)))[:want]
    sub = reads.subset(idx)
    q, k = w["q"], w["k"]
    t0 = time.perf_counter()
    h = oracle.map_filter(ref[:slice_len], sub.seq, sub.offsets, k, q, "all")
    dt = time.perf_counter() - t0
    return {"value": sub.n / dt, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"{sub.n} reads (origin in the first {slice_len} bp, one batch's density) vs the "
                      f"first {slice_len} bp of the {n} bp reference; {len(h)} hits; {dt:.1f} s single-thread"}


def run_reference(args, rank, world):
    if rank != 0:
        return 0
    ref, reads, w, _ = make_inputs(args, 0)
    steps, secs = [], []
    res = None
    for i in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        res = cpu_baseline(ref, reads, w, args.cpu_slice // 2, args.batch)
        if i >= args.warmup:
            steps.append(res["value"])
            secs.append(time.perf_counter() - t0)
    v = statistics.mean(steps)
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * statistics.mean(secs),
            "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u32", "data": "synthetic",
            "config": {"workload": args.workload, "sample": res["sample"]},
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": res["sample"]},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def main():
    args = parse_args()
    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group(backend="nccl" if args.impl == "ours" else "gloo")
    if args.impl == "reference":
        return run_reference(args, rank, world)

    import torch
    torch.cuda.set_device(local)
    from paper_1403_1706_gb300 import peanut
    peanut.load()

    ref, reads, w, t_gen = make_inputs(args, rank)
    q, k = w["q"], w["k"]
    stream = torch.cuda.current_stream()
    t0 = time.time()
    R = peanut.pack_reference(ref, stream=stream)
    t_pack = time.time() - t0

    # batches: rebased offsets, device and pinned host copies of the reads
    B = args.batch
    bounds = [(a, min(reads.n, a + B)) for a in range(0, reads.n, B)]
    d_seq = torch.from_numpy(reads.seq).to("cuda")
    h_seq = torch.empty(reads.seq.size, dtype=torch.uint8, pin_memory=True)
    h_seq.numpy()[:] = reads.seq
    batches = []
    for a, b in bounds:
        o0, o1 = int(reads.offsets[a]), int(reads.offsets[b])
        offs = (reads.offsets[a:b + 1] - np.uint64(o0)).astype(np.uint64)
        batches.append(dict(n=b - a, o0=o0, o1=o1, h_off=offs,
                            d_off=torch.from_numpy(offs.astype(np.int64)).to("cuda"),
                            d_seq=d_seq[o0:o1], h_seq=h_seq.numpy()[o0:o1]))
    kw = dict(k=k) if isinstance(k, int) else dict(k_permille=50)

    def step_device(stats=None):
        n_res = 0
        for bt in batches:
            RB = peanut.index_reads_device(R, bt["d_seq"], bt["d_off"], q, stream=stream, **kw)
            H = peanut.map_device(R, RB)
            n_res += H.n
            if stats is not None:
                stats.append(peanut.get_map_stats(RB))
            H.free()
            RB.free()
        return n_res

    def step_host():
        n_res = 0
        for bt in batches:
            RB = peanut.index_reads(R, bt["h_seq"], bt["h_off"], q, stream=stream, **kw)
            h = peanut.map_arrays(R, RB)
            n_res += h.n
            h.free()
            RB.free()
        return n_res

    def barrier():
        if world > 1:
            import torch.distributed as dist
            dist.barrier()
        torch.cuda.synchronize()

    from paper_1403_1706_gb300.shard import max_over_ranks, sum_over_ranks
    units = sum_over_ranks(reads.n, device="cuda")  # every rank maps its own read set
    bases = sum_over_ranks(reads.seq.size, device="cuda")

    t0 = time.time()
    for _ in range(args.warmup):
        n_res = step_device()
    t_warm = time.time() - t0

    # timed: device-resident inputs
    stats = []
    barrier()
    l0 = peanut.kernel_launches()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        ev0.record(stream)
        for _ in range(args.steps):
            n_res = step_device(stats)
        ev1.record(stream)
        torch.cuda.synchronize()
    launches = peanut.kernel_launches() - l0
    ms = max_over_ranks(ev0.elapsed_time(ev1), device="cuda") / args.steps
    value = units / (ms / 1e3)
    clocks = clk.summary()

    # end to end through the host API
    e2e = None
    if not args.no_e2e:
        barrier()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(args.steps):
            n_res_h = step_host()
        e1.record(stream)
        torch.cuda.synchronize()
        ems = max_over_ranks(e0.elapsed_time(e1), device="cuda") / args.steps
        h2d = sum(int(bt["h_seq"].nbytes) + int(bt["h_off"].nbytes) for bt in batches)
        e2e = {"value": units / (ems / 1e3), "unit": UNIT, "h2d_bytes_per_step": h2d,
               "d2h_bytes_per_step": int(n_res_h) * HIT_BYTES, "ms_per_step": ems}

    # rooflines: the verification count pass (largest launch-list share; integer-ALU bound) and the
    # reference scan (the memory-bound kernel)
    peak, peak_kind = load_peaks()
    n_ref = ref.size
    int_peak_tops = INT32_LANES_PER_SM * N_SM * SM_MAX_MHZ * 1e6 / 1e12
    v_ops = statistics.mean(34.0 * s["candidate_word_columns"] for s in stats)
    v_ms = statistics.mean(s["ms_verify_kernel"] for s in stats)
    v_ach = v_ops / (v_ms / 1e3) / 1e12
    per_wc = traffic_per_unit("verify_k", source_sha())
    v_wc = statistics.mean(s["candidate_word_columns"] for s in stats)
    roof = {"bound": "alu", "achieved": v_ach, "peak": int_peak_tops, "unit": "TOP/s", "frac": v_ach / int_peak_tops,
            "traffic": per_wc * v_wc if per_wc is not None else None, "kernel": "verify_k (count pass)",
            "algorithmic_int32_ops_per_launch": v_ops, "avg_launch_ms": v_ms,
            "peak_source": "derived: 152 SMs x 128 INT32 lanes x 2070 MHz"}
    per_launch = [n_ref * (0.25 + 8.0) + s["present_probes"] * 8.0 + s["hits"] * (4.0 + 1.0 + 8.0) for s in stats]
    algo_bytes = statistics.mean(per_launch)
    avg_ms = statistics.mean(s["ms_scan_kernel"] for s in stats)
    achieved = algo_bytes / (avg_ms / 1e3) / 1e9
    roof_scan = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                 "traffic": None, "kernel": "probe_ref_k + expand_k",
                 "algorithmic_bytes_per_launch": algo_bytes, "avg_launch_ms": avg_ms, "peak_source": peak_kind}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(ref, reads, w, args.cpu_slice, args.batch)

    stage = {k2: statistics.mean(s[k2] for s in stats) for k2 in
             ("ms_scan", "ms_scan_kernel", "ms_bin", "ms_windows", "ms_windows_sweep", "ms_lowcx", "ms_compact",
              "ms_verify", "ms_verify_kernel", "ms_output")}
    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "u32", "data": "synthetic",
            "config": {"workload": args.workload, "reference_bp": int(n_ref), "reads_per_gpu": int(reads.n),
                       "read_len": list(w["lengths"]), "k": k, "q": q, "batch_reads": B, "mode": "all",
                       "parallelism": f"read-sharded x{world}",
                       "l2": "no flush: every batch streams a 0.78 GB packed reference and probes a 1 GiB "
                             "index (> 129 MB L2)"},
            "e2e": e2e, "gpu_launches": int(launches), "clocks": clocks, "roofline": roof,
            "roofline_scan": roof_scan, "cpu_baseline": cpu,
            "results_per_step": int(n_res), "bases_per_s": bases / (ms / 1e3),
            "stage_ms_per_batch": stage,
            "hits_per_batch": statistics.mean(s["hits"] for s in stats),
            "candidates_per_batch": statistics.mean(s["candidates"] for s in stats),
            "candidate_columns_per_batch": statistics.mean(s["candidate_columns"] for s in stats),
            "lowcx_reads_per_batch": statistics.mean(s["lowcx_reads"] for s in stats),
            "lowcx_ranges_per_batch": statistics.mean(s["lowcx_ranges"] for s in stats),
            "present_probes_per_batch": statistics.mean(s["present_probes"] for s in stats),
            "setup_s": {"generate": t_gen, "pack": t_pack, "warmup": t_warm},
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
