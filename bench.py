#!/usr/bin/env python
"""Read-mapping throughput on one GB300: reads/s mapped, all hits, k = 5 % of 100 bp.

Workload (default): human-scale synthetic genome of 3.1 Gbp (45 % repeat families, 1 % tandem
runs) and 10,000,000 reads of 100 bp (95 % sampled with 1-4 % errors, 5 % random), indexed in
device-resident batches of 2^20 reads, q = 16, k = 5, all-hits mode.  One step maps all
10,000,000 reads (10 batches: peanut_index_reads + peanut_map each).

  value : reads/s of the engine with the reads already in device memory and the results left
          there (peanut_engine_submit_device / peanut_engine_wait_device), timed with CUDA events
          on the bench's stream; `plain` is the per-batch path (peanut_index_reads_device +
          peanut_map_device), `plain_tuned` the same at the engine's tuned setting.
  e2e   : reads/s through the host API (peanut_engine_submit from pinned host memory +
          peanut_engine_wait returning host arrays), host<->device copies inside the timed region.
  serving : a short Poisson request stream through the engine: p50 / p99 request latency.
  roofline : the q'-gram filter on candidate ranges (the largest launch-list share), algorithmic
          INT32 instructions per launch over its CUDA-event duration, against the measured integer
          issue rate of the in-repo microbenchmark; roofline_verify: the bit-vector verification
          kernel, the same way; roofline_scan: the two reference-scan kernels, algorithmic bytes per
          launch against the measured HBM copy bandwidth, and their L2 probe rate against the
          measured random-probe rate.
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
# Myers' column step on one 64-bit word, counted as the fewest 32-bit ALU instructions it needs:
# Xv = Eq | Mv (2), Eq & Pv (2), the carried add (2), Xh (2, one 3-input logic op per half),
# Ph (2), Mh (2), the two carried one-bit shifts (4 funnel shifts), Pv (2), Mv (2)
ALG_OPS_PER_WORD_COLUMN = 20
# The q'-gram filter per reference position scanned, in 32-bit ALU instructions: the 4-gram code
# (a funnel shift and a shift), the set lookup's word index and bit test and the count (4), the
# byte compares of the tracked 4-grams (xor, mask, add, zero-byte mask, shift, accumulate: 6)
FILTER_OPS_PER_POSITION = 12


def int_peaks(peanut, stream=None):
    """The in-repo integer issue-rate microbenchmark (peanut_int_peak), every kind once."""
    out = {}
    for kind, iters in (("lop3", 20000), ("shf", 20000), ("iadd", 20000), ("imad", 20000), ("popc", 20000),
                        ("myers_w1", 6000), ("myers_w2", 3000), ("probe_l2", 400), ("probe_hbm", 100)):
        r = peanut.int_peak(kind, iters, stream)
        out[kind] = {"ops_per_s": r["ops_per_s"], "ms": r["ms"], "ops": r["ops"],
                     "unit": ("word-columns/s" if kind.startswith("myers") else
                              "8-byte loads/s" if kind.startswith("probe") else "instructions/s")}
    return out


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
    ap.add_argument("--cpu-slice", type=int, default=100_000_000,
                    help="reference prefix (bp) of the CPU-baseline sample")
    ap.add_argument("--mode", choices=["plain", "batched", "serve", "qstudy", "post"], default="plain",
                    help="plain: one batch per launch sequence (the headline); batched: uneven batches of "
                         "50-250 bp reads through the engine vs the plain path; serve: a Poisson request "
                         "stream through the engine vs one request at a time; qstudy: index variants and the "
                         "q / L2-residency trade-off on one batch; post: the postprocessing of one batch's "
                         "hits (starts, ranks, qualities, alignments)")
    ap.add_argument("--requests", type=int, default=None, help="serve: number of requests")
    ap.add_argument("--rate", type=float, default=None, help="serve: mean arrivals per second")
    ap.add_argument("--executors", type=int, default=2, help="engine: launches in flight")
    ap.add_argument("--no-check", action="store_true", help="batched: skip the identical-output check")
    ap.add_argument("--no-serve", action="store_true", help="plain: skip the short serving leg")
    ap.add_argument("--no-graph-arm", action="store_true", help="plain: skip the engine-with-graphs arm")
    ap.add_argument("--no-refindex", action="store_true",
                    help="plain: skip the reference-side q-group index comparison arm")
    ap.add_argument("--serve-requests", type=int, default=30, help="plain: requests of the serving leg")
    ap.add_argument("--qstudy-configs", default=None,
                    help="qstudy: the settings to run, q:stride:layout joined by commas (default: all 13)")
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


def traffic_per_unit(name: str, unit: str, kernel_src_sha: str):
    """DRAM bytes per unit of work of a kernel, from the committed ncu summary
    profiles/<name>_traffic.json, if it was taken on the current kernel source; else None."""
    p = os.path.join(ROOT, "profiles", f"{name}_traffic.json")
    try:
        with open(p) as f:
            d = json.load(f)
        if d.get("source_sha256") != kernel_src_sha:
            return None
        return float(d[f"dram_bytes_per_{unit}"])
    except Exception:
        return None


def source_sha() -> str:
    """Hash of the mapping kernels' source (map.cu and the shared headers)."""
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


def cpu_baseline(ref, reads, w, slice_len, batch, threads=None):
    """The oracle on a bounded sample: the reads whose planted origin lies in the first
    `slice_len` bases (plus the unmappable ones at their natural rate), as many as one read batch
    holds per base of reference, mapped against that prefix.  The sample's reads are split over
    `threads` host threads (default: every core), each an independent oracle call that scans the
    whole prefix (ctypes releases the GIL); value = sample reads / wall time.  The per-read rate
    stands for the full workload because the sample is as dense on the prefix as a batch is on
    the whole reference: it is an extrapolation from the sample, labelled as such."""
    import oracle
    from concurrent.futures import ThreadPoolExecutor
    threads = threads or os.cpu_count() or 1
    n = ref.size
    slice_len = min(slice_len, n)
    want = max(1, int(round(batch * slice_len / n)))
    inside = (reads.truth_end >= 0) & (reads.truth_end < slice_len - 1)
    rnd = reads.truth_end < 0
    idx = np.flatnonzero(inside | (rnd & (np.arange(reads.n) % max(1, n // slice_len) == 0)))[:want]
    sub = reads.subset(idx)
    q, k = w["q"], w["k"]
    prefix = ref[:slice_len]
    shards = [sub.subset(np.arange(t, sub.n, threads)) for t in range(threads)]  # interleaved: balanced
    t0 = time.perf_counter()
    with ThreadPoolExecutor(threads) as ex:
        parts = list(ex.map(lambda sh: oracle.map_filter(prefix, sh.seq, sh.offsets, k, q, "all"), shards))
    dt = time.perf_counter() - t0
    nh = sum(len(h) for h in parts)
    return {"value": sub.n / dt, "unit": UNIT, "cores": threads, "kind": "oracle",
            "extrapolated": True,
            "sample": f"{sub.n} reads (origin in the first {slice_len} bp, one {batch}-read batch's density on "
                      f"the {n} bp reference) mapped against that prefix, split over {threads} threads; "
                      f"{nh} hits; {dt:.1f} s wall; reads/s extrapolated per read to the full workload (optimistic: "
                      f"the oracle's cost per low-complexity read grows with the reference length)"}


def run_reference(args, rank, world):
    if rank != 0:
        return 0
    ref, reads, w, _ = make_inputs(args, 0)
    steps, secs = [], []
    res = None
    for i in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        res = cpu_baseline(ref, reads, w, args.cpu_slice, args.batch)
        if i >= args.warmup:
            steps.append(res["value"])
            secs.append(time.perf_counter() - t0)
    v = statistics.mean(steps)
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * statistics.mean(secs),
            "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u32", "data": "synthetic",
            "config": {"workload": args.workload, "sample": res["sample"]},
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": res["cores"], "kind": "oracle",
                             "extrapolated": True, "sample": res["sample"]},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def _k_of(m):
    return (int(m) * 50 + 999) // 1000


def _q_class(m):
    return min(int(m) // (_k_of(m) + 1), 16)


def run_batched(args, rank, world, local):
    """Uneven batches (2^16-2^21 reads, log-uniform sizes) of reads of 50, 75, 100, 150 and 250 bp
    (2 % errors, k = ceil(0.05 L)) on the 3.1 Gbp reference.  Plain arm: every batch mapped
    with one launch sequence per q class (the largest q its reads admit: 12 for 50 bp, 15 for
    75 bp, 16 for the rest), reads resident in HBM.  Batched arm: the engine, every batch one
    device submission, coalesced into autotuned launches on `executors` streams."""
    import torch
    import synth
    from paper_1403_1706_gb300 import peanut
    from paper_1403_1706_gb300.shard import max_over_ranks, sum_over_ranks
    torch.cuda.set_device(local)
    peanut.load()
    w = synth.WORKLOADS["uneven_3g1_10m"]
    n_ref = args.ref_len or w["ref_len"]
    n_reads = args.reads or w["n_reads"]
    t0 = time.time()
    ref = synth.make_reference(n_ref, 1403, w["repeat_frac"], w["tandem_frac"])
    lengths = w["lengths"]
    per = [n_reads // len(lengths) + (1 if i < n_reads % len(lengths) else 0) for i in range(len(lengths))]
    cls_reads = [synth.make_reads(ref, per[i], 4000 + 10 * i + 1000 * rank, lengths=(L,),
                                  rate_range=w["rate_range"], random_frac=w["random_frac"])
                 for i, L in enumerate(lengths)]
    bounds = synth.uneven_batches(n_reads, 77 + rank)
    # batch b holds, of every length, its share of the batch size (reads grouped by length)
    cum = np.cumsum([0] + per)
    cuts = [[int(round(bb * p / n_reads)) for p in per] for bb in bounds]
    cuts[-1] = list(per)
    seqs, offs, groups = [], [], []
    for b in range(len(bounds) - 1):
        parts, o = [], [np.zeros(1, np.uint64)]
        grp = []  # (q, first read, end read) within the batch
        at_read, at_base = 0, 0
        for i, L in enumerate(lengths):
            a, e = cuts[b][i], cuts[b + 1][i]
            sub = cls_reads[i].slice(a, e)
            parts.append(sub.seq)
            o.append(sub.offsets[1:] + np.uint64(at_base))
            q = _q_class(L)
            if grp and grp[-1][0] == q:
                grp[-1] = (q, grp[-1][1], at_read + sub.n)
            else:
                grp.append((q, at_read, at_read + sub.n))
            at_read += sub.n
            at_base += int(sub.seq.size)
        seqs.append(np.concatenate(parts))
        offs.append(np.concatenate(o))
        groups.append(grp)
    t_gen = time.time() - t0
    stream = torch.cuda.current_stream()
    R = peanut.pack_reference(ref, stream=stream)
    d_batches, h_batches = [], []
    for sq, of, grp in zip(seqs, offs, groups):
        d_seq = torch.from_numpy(sq).to("cuda")
        d_off = torch.from_numpy(of.astype(np.int64)).to("cuda")
        h_seq = torch.empty(sq.size, dtype=torch.uint8, pin_memory=True)
        h_seq.numpy()[:] = sq
        h_off = torch.empty(of.size, dtype=torch.int64, pin_memory=True)
        h_off.numpy()[:] = of.astype(np.int64)
        sub_dev = []
        for q, a, e in grp:
            # the plain path maps a q class in as few launch sequences as keep a launch's expected
            # q-gram hits (random hits of the class's longest reads, twice for repeats) below 2^31
            lmax = max(L for L in lengths if _q_class(L) == q)
            nq = lmax - q + 1
            hpr = nq * 2.0 * 2.0 * n_ref / float(1 << (2 * q)) + nq
            cap = max(1, min(1 << 21, int(2.0 ** 31 / hpr)))
            for x in range(a, e, cap):
                y = min(e, x + cap)
                o0 = int(of[x])
                sub_dev.append((q, x, d_seq[o0:int(of[y])], (d_off[x:y + 1] - o0).contiguous()))
        d_batches.append((d_seq, d_off, sub_dev))
        h_batches.append((h_seq, h_off))
    torch.cuda.synchronize()

    def plain_step(collect=False):
        n_res, out = 0, []
        for d_seq, d_off, sub_dev in d_batches:
            parts = []
            for q, a, ds, do in sub_dev:
                B = peanut.index_reads_device(R, ds, do, q, k_permille=50, stream=stream)
                H = peanut.map_device(R, B)
                n_res += H.n
                if collect:
                    h = H.to_numpy()
                    h["read"] += a
                    parts.append(h)
                H.free()
                B.free()
            if collect:
                out.append(np.concatenate(parts))
        return n_res, out

    E = peanut.Engine(R, k_permille=50, executors=args.executors, autotune=True)

    def engine_step(collect=False):  # results stay in device memory, as in the plain arm
        tickets = [E.submit_device(d_seq, d_off, "all", result_on_device=True) for d_seq, d_off, _ in d_batches]
        n_res, out = 0, []
        for t in tickets:
            h = E.wait_device(t)
            n_res += h.n
            if collect:
                out.append(h.to_numpy())
            h.free()
        return n_res, out

    def engine_host_step():
        tickets = [E.submit(h_seq.numpy(), h_off.numpy().view(np.uint64), "all") for h_seq, h_off in h_batches]
        n_res = 0
        for t in tickets:
            h = E.wait_arrays(t)
            n_res += h.n
            h.free()
        return n_res

    # warm-up: tunes the engine; the first step checks that both arms return the same hits
    t0 = time.time()
    identical = None
    for i in range(args.warmup):
        check = i == 0 and not args.no_check
        _, a = plain_step(check)
        _, b = engine_step(check)
        if check:
            identical = all(np.array_equal(x, y) for x, y in zip(a, b)) and len(a) == len(b)
            del a, b
    t_warm = time.time() - t0

    def timed(fn):
        torch.cuda.synchronize()
        if world > 1:
            import torch.distributed as dist
            dist.barrier()
        l0 = peanut.kernel_launches()
        t = time.perf_counter()
        n = 0
        for _ in range(args.steps):
            n = fn()
        torch.cuda.synchronize()
        dt = (time.perf_counter() - t) / args.steps
        return max_over_ranks(dt, device="cuda"), n, (peanut.kernel_launches() - l0) // args.steps

    units = sum_over_ranks(n_reads, device="cuda")
    with ClockSampler(local) as clk:
        dt_b, n_b, launches_b = timed(lambda: engine_step()[0])
    clocks = clk.summary()
    dt_p, n_p, launches_p = timed(lambda: plain_step()[0])
    engine_host_step()  # warm-up of the host path (page-locked result blocks)
    dt_e, n_e, _ = timed(engine_host_step)
    st = E.stats()
    bases = sum_over_ranks(sum(int(x.size) for x in seqs), device="cuda")
    if rank == 0:
        line = {
            "metric": METRIC, "value": units / dt_b, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * dt_b, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "u32", "data": "synthetic", "mode": "batched",
            "config": {"workload": "uneven_3g1_10m", "reference_bp": int(n_ref), "reads_per_gpu": int(n_reads),
                       "read_len": list(lengths), "k": "ceil(0.05 L)", "errors": "2% of length",
                       "batches": len(bounds) - 1, "batch_reads": [int(min(np.diff(bounds))), int(max(np.diff(bounds)))],
                       "order": "reads of a batch grouped by length", "executors": args.executors,
                       "parallelism": f"read-sharded x{world}", "l2": "no flush: 0.78 GB packed reference + "
                       "index probes per launch (> 129 MB L2)"},
            "plain": {"value": units / dt_p, "ms_per_step": 1e3 * dt_p, "gpu_launches": int(launches_p),
                      "launch_sequences_per_step": sum(len(d[2]) for d in d_batches),
                      "q": {str(L): _q_class(L) for L in lengths}, "stride": 1},
            "vs_plain": dt_p / dt_b, "identical_output": identical,
            "e2e": {"value": units / dt_e, "unit": UNIT, "ms_per_step": 1e3 * dt_e,
                    "h2d_bytes_per_step": int(sum(h.numel() + 8 * o.numel() for h, o in h_batches)),
                    "d2h_bytes_per_step": int(n_e) * HIT_BYTES},
            "gpu_launches": int(launches_b), "clocks": clocks, "results_per_step": int(n_b),
            "bases_per_s": bases / dt_b, "engine": st,
            "setup_s": {"generate": t_gen, "warmup": t_warm},
        }
        print(json.dumps(line), flush=True)
    E.free()
    return 0


def run_qstudy(args, rank, world, local):
    """The index variants and the q / L2-residency trade-off on one 2^20-read batch of the 3.1 Gbp
    workload (100 bp, k = 5): for each q, sampling stride and layout of the batch index, the plain
    path's index and map times, its stage times and the index size.  At q <= 14 the (I, S) table
    (4^q / 4 bytes) fits the 129 MB L2; every lower q multiplies the random q-gram hits by 4.  Every
    setting must give the same hits (checked against the first)."""
    import torch
    import synth
    from paper_1403_1706_gb300 import peanut
    torch.cuda.set_device(local)
    peanut.load()
    w = synth.WORKLOADS["human_3g1_10m"]
    n_ref = args.ref_len or w["ref_len"]
    ref = synth.make_reference(n_ref, 1403, w["repeat_frac"], w["tandem_frac"])
    seed = 1706 + list(synth.WORKLOADS).index("human_3g1_10m")
    reads = synth.make_reads(ref, args.reads or (1 << 20), seed, lengths=w["lengths"], rate_range=w["rate_range"],
                             random_frac=w["random_frac"])
    stream = torch.cuda.current_stream()
    R = peanut.pack_reference(ref, stream=stream)
    d_seq = torch.from_numpy(reads.seq).to("cuda")
    d_off = torch.from_numpy(reads.offsets.astype(np.int64)).to("cuda")
    configs = [(16, 1, "interleaved"), (16, 1, "sampled_s"), (16, 1, "w64"), (16, 16, "interleaved"),
               (16, 16, "sampled_s"), (16, 16, "w64"), (16, 4, "interleaved"), (15, 1, "interleaved"),
               (15, 3, "interleaved"), (15, 15, "interleaved"), (14, 4, "interleaved"), (14, 14, "interleaved"),
               (13, 13, "interleaved")]
    if args.qstudy_configs:
        configs = [(int(a), int(b), c) for a, b, c in (x.split(":") for x in args.qstudy_configs.split(","))]
    rows, ref_hits = [], None
    for q, stride, layout in configs:
        def once():
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            B = peanut.index_reads_device(R, d_seq, d_off, q, k=5, stride=stride, layout=layout, stream=stream)
            torch.cuda.synchronize()
            t1 = time.perf_counter()
            H = peanut.map_device(R, B)
            torch.cuda.synchronize()
            t2 = time.perf_counter()
            st = peanut.get_map_stats(B)
            h = H.to_numpy()
            H.free()
            B.free()
            return t1 - t0, t2 - t1, st, h
        once()  # warm-up (builds the reference's frequent-q-gram table for this q)
        ti, tm, st, h = once()
        if ref_hits is None:
            ref_hits = h
        groups = (1 << (2 * q)) // 32
        rows.append({"q": q, "stride": stride, "layout": layout,
                     "index_table_bytes": groups * (8 if layout == "interleaved" else 6),
                     "index_ms": 1e3 * ti, "map_ms": 1e3 * tm, "ms_probe_kernel": st["ms_probe_kernel"],
                     "ms_scan_kernel": st["ms_scan_kernel"], "ms_windows": st["ms_windows"],
                     "ms_filter_kernel": st["ms_filter_kernel"], "ms_verify_kernel": st["ms_verify_kernel"],
                     "hits": st["hits"], "present_probes": st["present_probes"], "candidates": st["candidates"],
                     "results": st["results"], "identical": bool(np.array_equal(h, ref_hits))})
        print(json.dumps(rows[-1]), file=sys.stderr, flush=True)
    if rank == 0:
        best = min(rows, key=lambda r: r["index_ms"] + r["map_ms"])
        line = {"metric": METRIC, "mode": "qstudy", "value": reads.n / ((best["index_ms"] + best["map_ms"]) / 1e3),
                "unit": UNIT, "n_gpus": world, "steps": 1, "warmup": 1, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "u32", "data": "synthetic",
                "config": {"workload": "human_3g1_10m (one batch)", "reference_bp": int(n_ref), "reads": int(reads.n),
                           "k": 5, "l2_bytes": 129 << 20},
                "study": rows, "identical_output": all(r["identical"] for r in rows)}
        print(json.dumps(line), flush=True)
    return 0


def run_post(args, rank, world, local):
    """The postprocessing of one 2^20-read batch of the 3.1 Gbp workload (100 bp, k = 5, all hits,
    q = 16, stride 16, the engine's tuned setting): alignment start, hit-rank and quality
    (peanut_annotate_hits), then the alignment of every hit (peanut_hit_alignments); the median
    of three runs each, CUDA events on the batch's stream, hits per second."""
    import torch
    import synth
    from paper_1403_1706_gb300 import peanut
    torch.cuda.set_device(local)
    peanut.load()
    w = synth.WORKLOADS["human_3g1_10m"]
    n_ref = args.ref_len or w["ref_len"]
    ref = synth.make_reference(n_ref, 1403, w["repeat_frac"], w["tandem_frac"])
    seed = 1706 + list(synth.WORKLOADS).index("human_3g1_10m")
    reads = synth.make_reads(ref, args.reads or (1 << 20), seed, lengths=w["lengths"], rate_range=w["rate_range"],
                             random_frac=w["random_frac"])
    stream = torch.cuda.current_stream()
    R = peanut.pack_reference(ref, stream=stream)
    d_seq = torch.from_numpy(reads.seq).to("cuda")
    d_off = torch.from_numpy(reads.offsets.astype(np.int64)).to("cuda")
    B = peanut.index_reads_device(R, d_seq, d_off, 16, k=5, stride=16, stream=stream)
    dh = peanut.map_device(R, B, "all")

    def timed(fn, reps=3):
        out, ts = None, []
        for _ in range(reps + 1):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            e0.record(stream)
            out = fn()
            e1.record(stream)
            torch.cuda.synchronize()
            ts.append(e0.elapsed_time(e1))
        return out, statistics.median(ts[1:])

    (start, _, _), ms_ann = timed(lambda: peanut.annotate_hits(R, B, dh))
    (ops, nops), ms_cig = timed(lambda: peanut.hit_alignments(R, B, dh, start))
    n = dh.n
    runs = nops.cpu().numpy().view(np.uint16)
    line = {"metric": "hits/sec postprocessed (start, rank, quality and extended CIGAR of every hit)", "mode": "post",
            "value": n / ((ms_ann + ms_cig) / 1e3), "unit": "hits/s",
            "n_gpus": world, "steps": 3, "warmup": 1, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "u32", "data": "synthetic",
            "config": {"workload": "human_3g1_10m (one batch)", "reference_bp": int(n_ref), "reads": int(reads.n),
                       "k": 5, "q": 16, "stride": 16, "mode": "all"},
            "hits": int(n), "ms_annotate": ms_ann, "ms_alignments": ms_cig,
            "annotate_hits_per_s": n / (ms_ann / 1e3), "alignment_hits_per_s": n / (ms_cig / 1e3),
            "mean_runs_per_hit": float(runs.mean()) if n else 0.0, "max_runs_per_hit": int(runs.max()) if n else 0}
    if rank == 0:
        print(json.dumps(line), flush=True)
    dh.free()
    B.free()
    return 0


def serve_stream(peanut, R, ref, n_req, rate, seed, executors, warmup, clock_gpu=None, log=None):
    """A Poisson request stream (sizes log-uniform in 10^3..10^6 reads, lengths 75-250 bp, 1-4 %
    errors, k = ceil(0.05 L), half the requests in best-stratum mode) on a resident reference.
    Engine: requests submitted from pinned host memory at their arrival times, each result
    waited for on its own thread; latency = result in hand - arrival.  Baseline: one request at a
    time through the plain path (peanut_index_reads + peanut_map per q class of the request), a
    FIFO queue over the measured service times.  Returns the measurements as a dict."""
    import torch
    import synth
    w = synth.WORKLOADS["serve_3g1"]
    t0 = time.time()
    arrivals, sizes, modes = synth.request_stream(seed, n_req, rate, w["req_min"], w["req_max"])
    reqs = []
    for i in range(n_req):
        rd = synth.make_reads(ref, int(sizes[i]), 9000 + i + 100 * seed, lengths=w["lengths"],
                              rate_range=w["rate_range"], random_frac=w["random_frac"])
        h_seq = torch.empty(rd.seq.size, dtype=torch.uint8, pin_memory=True)
        h_seq.numpy()[:] = rd.seq
        # the baseline maps each q class of the request as its own batch
        cls = np.array([_q_class(m) for m in range(256)])[rd.lengths]
        order = np.argsort(cls, kind="stable")
        groups = []
        for q in np.unique(cls):
            idx = order[cls[order] == q]
            sub = rd.subset(idx)
            groups.append((int(q), idx.astype(np.int64), sub.seq, sub.offsets))
        reqs.append((h_seq, rd.offsets, groups, rd.n))
    t_gen = time.time() - t0
    E = peanut.Engine(R, k_permille=50, executors=executors, autotune=True)
    # warm-up: the largest request through both paths (tunes the engine's classes, builds the
    # reference's per-q tables)
    warm = int(np.argmax(sizes))
    for _ in range(max(1, warmup)):
        E.wait(E.submit(reqs[warm][0].numpy(), reqs[warm][1], "all"))
    for q, idx, sq, of in reqs[warm][2]:
        B = peanut.index_reads(R, sq, of, q, k_permille=50)
        peanut.map(R, B, "all")
        B.free()

    done = [0.0] * n_req
    nres = [0] * n_req
    waiters = []

    def waiter(i, t):
        h = E.wait_arrays(t)
        done[i] = time.perf_counter()
        nres[i] = h.n
        h.free()

    l0 = peanut.kernel_launches()
    clk = ClockSampler(clock_gpu) if clock_gpu is not None else None
    if clk:
        clk.__enter__()
    start = time.perf_counter()
    for i in range(n_req):
        delay = start + float(arrivals[i]) - time.perf_counter()
        if delay > 0:
            time.sleep(delay)
        t = E.submit(reqs[i][0].numpy(), reqs[i][1], str(modes[i]))
        th = threading.Thread(target=waiter, args=(i, t))
        th.start()
        waiters.append(th)
    for th in waiters:
        th.join()
    if clk:
        clk.__exit__()
    launches = peanut.kernel_launches() - l0
    lat = np.array([done[i] - (start + float(arrivals[i])) for i in range(n_req)])
    span = max(done) - (start + float(arrivals[0]))
    total_reads = int(sum(r[3] for r in reqs))
    st = E.stats()
    E.free()

    service = []
    for i in range(n_req):
        t = time.perf_counter()
        for q, idx, sq, of in reqs[i][2]:
            B = peanut.index_reads(R, sq, of, q, k_permille=50)
            h = peanut.map_arrays(R, B, str(modes[i]))  # a read's stratum lies within its class
            h.free()
            B.free()
        service.append(time.perf_counter() - t)
    fin, plain_lat = 0.0, []
    for i in range(n_req):
        fin = max(float(arrivals[i]), fin) + service[i]
        plain_lat.append(fin - float(arrivals[i]))
    plain_lat = np.array(plain_lat)
    plain_span = fin - float(arrivals[0])
    pct = lambda a: {"p50": float(np.percentile(a, 50)), "p99": float(np.percentile(a, 99)),
                     "max": float(a.max())}
    return {
        "value": total_reads / span, "unit": UNIT, "span_s": span, "requests": n_req, "rate_per_s": rate,
        "request_reads": [int(sizes.min()), int(sizes.max())], "reads": total_reads,
        "offered_reads_per_s": total_reads / max(float(arrivals[-1]), 1e-9),
        "modes": {m: int((modes == m).sum()) for m in ("all", "best")},
        "latency_s": pct(lat),
        "one_at_a_time": {"value": total_reads / plain_span, "latency_s": pct(plain_lat),
                          "service_s_total": float(sum(service)),
                          "note": "plain path per q class of each request, FIFO queue from measured "
                                  "service times"},
        "h2d_bytes": int(sum(r[0].numel() + 8 * (r[3] + 1) for r in reqs)),
        "d2h_bytes": int(sum(nres)) * HIT_BYTES, "results": int(sum(nres)), "gpu_launches": int(launches),
        "clocks": clk.summary() if clk else None, "engine": st, "generate_s": t_gen,
    }


def run_serve(args, rank, world, local):
    """The serving configuration (serve_3g1): a Poisson request stream of 100 requests at 50/s on
    the resident 3.1 Gbp reference, through the engine and one request at a time (serve_stream)."""
    import torch
    import synth
    from paper_1403_1706_gb300 import peanut
    torch.cuda.set_device(local)
    peanut.load()
    w = synth.WORKLOADS["serve_3g1"]
    n_ref = args.ref_len or w["ref_len"]
    n_req = args.requests or w["n_requests"]
    t0 = time.time()
    ref = synth.make_reference(n_ref, 1403, w["repeat_frac"], w["tandem_frac"])
    t_ref = time.time() - t0
    rate = args.rate or w["rate_per_s"]
    R = peanut.pack_reference(ref)
    sv = serve_stream(peanut, R, ref, n_req, rate, 91 + rank, args.executors, args.warmup, clock_gpu=local)
    if rank == 0:
        line = {
            "metric": METRIC, "value": sv["value"], "unit": UNIT, "n_gpus": world, "steps": 1,
            "warmup": args.warmup, "ms_per_step": 1e3 * sv["span_s"], "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "u32", "data": "synthetic", "mode": "serve",
            "config": {"workload": "serve_3g1", "reference_bp": int(n_ref), "requests": n_req,
                       "rate_per_s": rate, "request_reads": sv["request_reads"],
                       "reads": sv["reads"], "read_len": [75, 250], "k": "ceil(0.05 L)",
                       "modes": sv["modes"], "executors": args.executors,
                       "offered_reads_per_s": sv["offered_reads_per_s"]},
            "latency_s": sv["latency_s"], "one_at_a_time": sv["one_at_a_time"],
            "e2e": {"value": sv["value"], "unit": UNIT, "h2d_bytes_per_step": sv["h2d_bytes"],
                    "d2h_bytes_per_step": sv["d2h_bytes"]},
            "gpu_launches": sv["gpu_launches"], "clocks": sv["clocks"], "results": sv["results"],
            "engine": sv["engine"], "setup_s": {"generate": t_ref + sv["generate_s"]},
        }
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
    if args.mode == "batched":
        rc = run_batched(args, rank, world, local)
    elif args.mode == "qstudy":
        rc = run_qstudy(args, rank, world, local)
    elif args.mode == "serve":
        rc = run_serve(args, rank, world, local)
    elif args.mode == "post":
        rc = run_post(args, rank, world, local)
    else:
        rc = None
    if rc is not None:
        if world > 1:
            import torch.distributed as dist
            dist.destroy_process_group()
        return rc

    import torch
    torch.cuda.set_device(local)
    from paper_1403_1706_gb300 import peanut
    peanut.load()

    ref, reads, w, t_gen = make_inputs(args, rank)
    q, k = w["q"], w["k"]
    stream = torch.cuda.current_stream()
    ipk = int_peaks(peanut, stream)
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

    def step_device(stats=None, qs=(q, 1), ri=False):
        n_res = 0
        for bt in batches:
            RB = peanut.index_reads_device(R, bt["d_seq"], bt["d_off"], qs[0], stream=stream, stride=qs[1],
                                           ref_index=ri, **kw)
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

    # the engine over the same device-resident batches of 2^20 reads: launches of at most one
    # batch, (q, stride) autotuned, `executors` launches in flight
    E = peanut.Engine(R, **kw, executors=args.executors, max_reads=B, autotune=True)

    def step_engine():  # results stay in device memory, as in the plain arm
        tickets = [E.submit_device(bt["d_seq"], bt["d_off"], "all", result_on_device=True) for bt in batches]
        n = 0
        for t in tickets:
            h = E.wait_device(t)
            n += h.n
            h.free()
        return n

    def step_engine_host():
        tickets = [E.submit(bt["h_seq"], bt["h_off"], "all") for bt in batches]
        n = 0
        for t in tickets:
            h = E.wait_arrays(t)
            n += h.n
            h.free()
        return n

    t0 = time.time()
    identical = None
    for i in range(args.warmup):
        n_res = step_device()
        n_eng = step_engine()
        if i == 0 and not args.no_check:  # both paths return the same hits, batch by batch
            identical = True
            tickets = [E.submit_device(bt["d_seq"], bt["d_off"], "all") for bt in batches]
            for bt, t in zip(batches, tickets):
                RB = peanut.index_reads_device(R, bt["d_seq"], bt["d_off"], q, stream=stream, **kw)
                want = peanut.map_device(R, RB)
                a = want.to_numpy()
                want.free()
                RB.free()
                h = E.wait_arrays(t)
                identical &= (h.n == a.size and np.array_equal(h.read, a["read"]) and
                              np.array_equal(h.strand, a["strand"]) and
                              np.array_equal(h.end.astype(np.int64), a["end"]) and
                              np.array_equal(h.dist, a["dist"].astype(np.uint8)))
                h.free()
            identical = bool(identical)
    t_warm = time.time() - t0

    def timed(fn, clocks=False, engine=True):
        barrier()
        l0 = peanut.kernel_launches()
        e0 = E.stats() if engine else None
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        clk = ClockSampler(local) if clocks else None
        if clk:
            clk.__enter__()
        ev0.record(stream)
        n = 0
        for _ in range(args.steps):
            n = fn()
        ev1.record(stream)
        torch.cuda.synchronize()
        if clk:
            clk.__exit__()
        e1 = E.stats() if engine else None
        delta = None if not engine else {f: e1[f] - e0[f] for f in ("map_runs", "hits", "candidate_word_columns", "present_probes",
                                               "candidate_columns", "useful_columns", "filter_positions",
                                               "ms_filter_kernel",
                                               "bases_scanned", "ms_verify_kernel", "ms_scan_kernel",
                                               "ms_admit", "ms_launch", "ms_assemble", "ms_download")}
        ms = max_over_ranks(ev0.elapsed_time(ev1), device="cuda") / args.steps
        return ms, n, peanut.kernel_launches() - l0, delta, (clk.summary() if clk else None)

    # timed: plain path (one launch sequence per batch, q = 16, every q-gram), device-resident
    stats = []
    ms_p, n_res, launches_p, _, _ = timed(lambda: step_device(stats))
    # timed: engine, device-resident (the headline)
    ms, n_eng, launches, edelta, clocks = timed(step_engine, clocks=True)
    value = units / (ms / 1e3)

    # end to end through the host API (engine submissions from pinned host memory)
    e2e = None
    if not args.no_e2e:
        step_engine_host()  # warm-up of the host path (page-locked result blocks)
        ems, n_res_h, _, hdelta, _ = timed(step_engine_host)
        h2d = sum(int(bt["h_seq"].nbytes) + int(bt["h_off"].nbytes) for bt in batches)
        e2e = {"value": units / (ems / 1e3), "unit": UNIT, "h2d_bytes_per_step": h2d,
               "d2h_bytes_per_step": int(n_res_h) * HIT_BYTES, "ms_per_step": ems,
               "api": "peanut_engine_submit + peanut_engine_wait",
               "engine_ms_per_step": {f[3:]: hdelta[f] / args.steps
                                      for f in ("ms_admit", "ms_launch", "ms_assemble", "ms_download")},
               "pageable_result_blocks": E.stats()["pageable_result_blocks"]}
    est = E.stats()
    E.free()

    # the same engine with each launch's sync-free stretches run as CUDA graphs (graphs = 1)
    engine_graphs = None
    if not args.no_graph_arm:
        EG = peanut.Engine(R, **kw, executors=args.executors, max_reads=B, autotune=True, graphs=True)

        def step_engine_graphs():
            tickets = [EG.submit_device(bt["d_seq"], bt["d_off"], "all", result_on_device=True) for bt in batches]
            n = 0
            for t in tickets:
                h = EG.wait_device(t)
                n += h.n
                h.free()
            return n
        n_g = step_engine_graphs()  # warm-up (tunes the engine's class)
        step_engine_graphs()
        ms_g, n_g2, launches_g, _, _ = timed(step_engine_graphs, engine=False)
        gst = EG.stats()
        EG.free()
        engine_graphs = {"value": units / (ms_g / 1e3), "ms_per_step": ms_g, "gpu_launches": int(launches_g),
                         "graph_segments": gst["graph_segments"], "map_runs": gst["map_runs"],
                         "results_per_step": int(n_g2), "same_result_count": int(n_g2) == int(n_eng),
                         "note": "peanut_engine_params.graphs = 1: the scan, binning + short-read windows, filter "
                                 "+ verification count pass and write pass of every launch captured as CUDA "
                                 "graphs (instantiated per launch)"}

    # the plain path at the engine's tuned setting: isolates what batching and overlap add
    tuned = next((c for c in est["classes"] if c["q_class"] == q), None)
    plain_tuned = None
    if tuned is not None:
        qs_t = (tuned["q"], tuned["stride"])
        step_device(qs=qs_t)  # warm-up at this setting
        stats_t = []
        ms_t, _, launches_t, _, _ = timed(lambda: step_device(stats_t, qs=qs_t), engine=False)
        plain_tuned = {"value": units / (ms_t / 1e3), "ms_per_step": ms_t, "q": qs_t[0], "stride": qs_t[1],
                       "gpu_launches": int(launches_t),
                       "stage_ms_per_batch": {k2: statistics.mean(x[k2] for x in stats_t) for k2 in
                                              ("ms_scan_kernel", "ms_probe_kernel", "ms_bin", "ms_windows",
                                               "ms_lowcx", "ms_compact", "ms_verify", "ms_filter_kernel",
                                               "ms_verify_kernel")},
                       "per_batch": {k2: statistics.mean(x[k2] for x in stats_t) for k2 in
                                     ("hits", "present_probes", "candidates", "filter_live", "candidate_columns",
                                      "useful_columns", "results")}}

    # the reference-side q-group index as a comparison: the same batches at the tuned setting with
    # their q-grams looked up in the reference's own index instead of streaming the reference
    refidx = None
    if tuned is not None and not args.no_refindex:
        qs_t = (tuned["q"], tuned["stride"])
        torch.cuda.synchronize()
        t0 = time.time()
        peanut.index_reference(R, qs_t[0], stream)
        torch.cuda.synchronize()
        t_build = time.time() - t0
        same = True
        for bt in batches[:1]:  # identical hits, batch 0, both scans
            hs = []
            for ri in (False, True):
                RB = peanut.index_reads_device(R, bt["d_seq"], bt["d_off"], qs_t[0], stream=stream, stride=qs_t[1],
                                               ref_index=ri, **kw)
                H = peanut.map_device(R, RB)
                hs.append(H.to_numpy())
                H.free()
                RB.free()
            same = bool(np.array_equal(hs[0], hs[1]))
        step_device(qs=qs_t, ri=True)
        stats_r = []
        ms_r, _, launches_r, _, _ = timed(lambda: step_device(stats_r, qs=qs_t, ri=True), engine=False)
        refidx = {"value": units / (ms_r / 1e3), "ms_per_step": ms_r, "q": qs_t[0], "stride": qs_t[1],
                  "gpu_launches": int(launches_r), "build_s": t_build, "identical_output_batch0": same,
                  "scan_kernel_ms_per_batch": statistics.mean(x["ms_scan_kernel"] for x in stats_r),
                  "streaming_scan_kernel_ms_per_batch": (plain_tuned["stage_ms_per_batch"]["ms_scan_kernel"]
                                                         if plain_tuned else None),
                  "stage_ms_per_batch": {k2: statistics.mean(x[k2] for x in stats_r) for k2 in
                                         ("ms_scan_kernel", "ms_bin", "ms_windows", "ms_lowcx", "ms_compact",
                                          "ms_verify", "ms_filter_kernel", "ms_verify_kernel")},
                  "note": "plain path at the engine's tuned setting, hits from the reference's own q-group "
                          "index (peanut_index_reference, ref_index = 1) instead of the streaming scan"}

    # a short serving leg: the serving configuration's request stream (sizes log-uniform in
    # 10^3..10^6 reads, 50 requests/s), fewer requests, on the same resident reference
    serving = None
    if not args.no_serve:
        sv = serve_stream(peanut, R, ref, args.serve_requests, 50.0, 91 + rank, args.executors, 1)
        serving = {k2: sv[k2] for k2 in ("value", "unit", "requests", "rate_per_s", "request_reads", "reads",
                                          "offered_reads_per_s", "modes", "latency_s", "one_at_a_time",
                                          "span_s")}

    # rooflines: the verification count pass (largest launch-list share; integer-ALU bound) and the
    # reference scan (the memory-bound kernels), from the runs' CUDA-event kernel times
    peak, peak_kind = load_peaks()
    n_ref = ref.size
    int_peak_tops = ipk["lop3"]["ops_per_s"] / 1e12
    step_peak = ipk["myers_w2"]["ops_per_s"]
    l2_probe_peak = ipk["probe_l2"]["ops_per_s"]
    sha = source_sha()
    per_wc = traffic_per_unit("verify_k", "word_column", sha)
    per_pos = traffic_per_unit("qfilter_k", "position", sha)
    peak_note = ("measured: in-repo microbenchmark, 3-input logic (lop3.b32) issue rate "
                 "(peanut_int_peak kind 0), same process, before the timed region")

    def rooflines(runs, wc, ms_v, probes, hits, bases, ms_s, fpos, ms_f, note):
        # the q'-gram filter: the dominant kernel by launch-list share (profiles/launches_*.md)
        f_ops = FILTER_OPS_PER_POSITION * fpos / runs
        f_ms = ms_f / runs
        f_ach = f_ops / (f_ms / 1e3) / 1e12
        filt = {"bound": "alu", "achieved": f_ach, "peak": int_peak_tops, "unit": "TOP/s",
                "frac": f_ach / int_peak_tops, "traffic": per_pos * fpos / runs if per_pos is not None else None,
                "kernel": "qfilter_k", "algorithmic_int32_ops_per_launch": f_ops,
                "ops_per_position": FILTER_OPS_PER_POSITION, "positions_per_launch": fpos / runs,
                "avg_launch_ms": f_ms, "launches": runs, "peak_source": peak_note, "timing": note}
        v_ops = ALG_OPS_PER_WORD_COLUMN * wc / runs
        v_ms = ms_v / runs
        v_ach = v_ops / (v_ms / 1e3) / 1e12
        roof = {"bound": "alu", "achieved": v_ach, "peak": int_peak_tops, "unit": "TOP/s",
                "frac": v_ach / int_peak_tops,
                "traffic": per_wc * wc / runs if per_wc is not None else None, "kernel": "verify_k (count pass)",
                "algorithmic_int32_ops_per_launch": v_ops, "ops_per_word_column": ALG_OPS_PER_WORD_COLUMN,
                "avg_launch_ms": v_ms, "launches": runs, "peak_source": peak_note,
                "word_columns_per_s": wc / runs / (v_ms / 1e3),
                "step_frac": wc / runs / (v_ms / 1e3) / step_peak,
                "step_peak_word_columns_per_s": step_peak, "timing": note}
        algo = (bases * (0.25 + 8.0) + probes * 8.0 + hits * (4.0 + 1.0 + 8.0)) / runs
        s_ms = ms_s / runs
        ach = algo / (s_ms / 1e3) / 1e9
        scan = {"bound": "hbm", "achieved": ach, "peak": peak, "unit": "GB/s", "frac": ach / peak,
                "traffic": None, "kernel": "probe_ref_k + expand_k", "algorithmic_bytes_per_launch": algo,
                "avg_launch_ms": s_ms, "launches": runs, "peak_source": peak_kind, "timing": note,
                "l2_probes_per_s": bases / runs / (s_ms / 1e3),
                "l2_probe_frac": bases / runs / (s_ms / 1e3) / l2_probe_peak,
                "l2_probe_peak_per_s": l2_probe_peak}
        return filt, roof, scan

    filt, roof, roof_scan = rooflines(
        edelta["map_runs"], edelta["candidate_word_columns"], edelta["ms_verify_kernel"], edelta["present_probes"],
        edelta["hits"], edelta["bases_scanned"], edelta["ms_scan_kernel"], edelta["filter_positions"],
        edelta["ms_filter_kernel"],
        f"engine runs, {args.executors} launches in flight: kernels share the GPU with the other stream's work")
    filt_p, roof_p, roof_scan_p = rooflines(
        len(stats), sum(s["candidate_word_columns"] for s in stats), sum(s["ms_verify_kernel"] for s in stats),
        sum(s["present_probes"] for s in stats), sum(s["hits"] for s in stats), n_ref * len(stats),
        sum(s["ms_scan_kernel"] for s in stats), sum(s["filter_positions"] for s in stats),
        sum(s["ms_filter_kernel"] for s in stats), "plain path, one launch sequence at a time")
    plain = {"value": units / (ms_p / 1e3), "ms_per_step": ms_p, "gpu_launches": int(launches_p),
             "q": q, "stride": 1, "roofline": filt_p, "roofline_verify": roof_p, "roofline_scan": roof_scan_p,
             "results_per_step": int(n_res),
             "stage_ms_per_batch": {k2: statistics.mean(s[k2] for s in stats) for k2 in
                                    ("ms_scan", "ms_scan_kernel", "ms_probe_kernel", "ms_bin", "ms_windows",
                                     "ms_windows_sweep", "ms_lowcx", "ms_compact", "ms_verify",
                                     "ms_filter_kernel", "ms_verify_kernel", "ms_output")},
             "per_batch": {k2: statistics.mean(s[k2] for s in stats) for k2 in
                           ("hits", "present_probes", "candidates", "prefilter_columns", "filter_positions",
                            "filter_live", "candidate_columns", "useful_columns", "lowcx_reads", "lowcx_ranges",
                            "lowcx_rest_segments", "results")}}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(ref, reads, w, args.cpu_slice, args.batch)

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "u32", "data": "synthetic",
            "config": {"workload": args.workload, "reference_bp": int(n_ref), "reads_per_gpu": int(reads.n),
                       "read_len": list(w["lengths"]), "k": k, "q": "autotuned per q class (plain: 16)",
                       "batch_reads": B, "mode": "all", "executors": args.executors,
                       "parallelism": f"read-sharded x{world}",
                       "l2": "no flush: every batch streams a 0.78 GB packed reference and probes a 1 GiB "
                             "index (> 129 MB L2)"},
            "e2e": e2e, "gpu_launches": int(launches), "clocks": clocks, "roofline": filt,
            "roofline_verify": roof, "roofline_scan": roof_scan, "cpu_baseline": cpu,
            "path": "engine (peanut_engine_submit_device / peanut_engine_wait)",
            "plain": plain, "plain_tuned": plain_tuned, "vs_plain": ms_p / ms,
            "vs_plain_tuned": plain_tuned["ms_per_step"] / ms if plain_tuned else None,
            "identical_output": identical, "serving": serving, "plain_refindex": refidx,
            "engine_graphs": engine_graphs,
            "int_peak": {kk: {"per_s": v["ops_per_s"], "unit": v["unit"],
                              "per_sm_per_clock": (v["ops_per_s"] / (152 * clocks["sm_mhz"] * 1e6)
                                                   if clocks and clocks.get("sm_mhz") else None)}
                         for kk, v in ipk.items()},
            "verify_useful_column_fraction": (edelta["useful_columns"] / edelta["candidate_columns"]
                                              if edelta["candidate_columns"] else None),
            "engine": {"classes": est["classes"], "launches": est["launches"],
                       "hbm_reserved_peak": est["hbm_reserved_peak"],
                       "engine_ms_per_step": {f[3:]: edelta[f] / args.steps
                                              for f in ("ms_admit", "ms_launch", "ms_assemble", "ms_download")}},
            "results_per_step": int(n_eng), "bases_per_s": bases / (ms / 1e3),
            "setup_s": {"generate": t_gen, "pack": t_pack, "warmup": t_warm},
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
