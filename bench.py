#!/usr/bin/env python
"""Benchmark of the MaxSSmap hot path on GB300 (one JSON line on rank 0).

One step = the whole hot path over one batch: phase one (exact MSS scan of every read on
both strands along every genome diagonal, per-fragment maxima, top-2 fragments, best-diagonal
rescan) and phase two (banded NW) for every read of the batch.  Default workload: the
bacterial-genome shape, a 4.6 Mbp synthetic genome (GC 50.8%, 2% exact 1-5 kbp repeat
copies), F = 2048, 200,000 reads of 100 bp and 200,000 of 150 bp at 10/20/30% substitutions
with up to two geometric gaps <= 30 bp, scores 5/-4, banded NW 5/-4/-10/-1 with W = 32.  The
400,000 reads are dealt into batches of 50,000 (read b, b + 8, b + 16, ...: every batch has
the same mix) and the steps cycle through the batches.

Metric: GCUPS = sum over reads of m * Gp * 2 strands / step time (the paper reports
wall-clock minutes; cells per second is the standard unit of alignment scans), and reads/s.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl mine|reference]

--impl reference times the CPU oracle (the plain definition, single-threaded C, run as one
process per host core over read shards) on a bounded sample of the same workload.
Multi-GPU (torchrun): every rank maps its own batch of reads against its own genome replica
(independent problems, weak scaling, no data-path collective).
"""
from __future__ import annotations

import argparse
import json
import multiprocessing as mp
import os
import statistics
import subprocess
import sys
import tempfile
import time
from concurrent.futures import ProcessPoolExecutor

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import gen  # noqa: E402

METRIC = "GCUPS (exact MSS scan of every read, both strands, every diagonal + top-2 + banded NW)"
L2_FLUSH_BYTES = 512 << 20


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="mine", choices=["mine", "reference"])
    ap.add_argument("--workload", default="bact-4.6M")
    ap.add_argument("--reads", type=int, default=0, help="override the read count (testing only)")
    ap.add_argument("--batch", type=int, default=50_000, help="reads per step (the workload is dealt into batches)")
    ap.add_argument("--genome", type=int, default=0, help="override the genome length (testing only)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--cpu-reads-per-core", type=int, default=2)
    ap.add_argument("--autotune", action="store_true",
                    help="pick the scan shape and fragment length with mss_autotune on a read sample first")
    ap.add_argument("--autotune-reads", type=int, default=256)
    ap.add_argument("--threads", type=int, default=0, choices=[0, 128, 256],
                    help="scan threads per CTA (0: the library's default)")
    ap.add_argument("--read-step", type=int, default=1, choices=[1, 2],
                    help="2: MaxSSmap_fast (every other read base in phase one)")
    ap.add_argument("--no-proposal", action="store_true", help="skip the learned-proposal measurement")
    ap.add_argument("--prop-train-reads", type=int, default=20_000)
    ap.add_argument("--prop-steps", type=int, default=400)
    ap.add_argument("--prop-eval-reads", type=int, default=8_000)
    return ap.parse_args()


def workload(args, rank: int):
    wl = gen.workloads()[args.workload]
    if args.reads or args.genome:
        wl = gen.scaled(wl, genome_len=args.genome or None, reads=args.reads or None)
    genome = gen.make_genome(wl.genome, wl.seed)      # identical on every rank
    reads = gen.read_set(wl, genome, rank)             # reads drawn per rank
    return wl, genome, reads.seq, reads.offsets


def batches(seq, off, batch: int):
    """The workload dealt into ceil(R / batch) batches of equal mix: (seq, offsets) per batch."""
    R = off.shape[0] - 1
    nb = max(1, -(-R // max(1, batch)))
    out = []
    for b in range(nb):
        idx = gen.batch_index(R, nb, b)
        lens = (off[idx + 1] - off[idx]).astype(np.int64)
        o = np.zeros(idx.shape[0] + 1, dtype=np.int64)
        np.cumsum(lens, out=o[1:])
        starts = np.repeat(off[idx] - o[:-1], lens)
        s = seq[np.arange(o[-1], dtype=np.int64) + starts]
        out.append((s, o))
    return out


# DRAM bytes (read + write) of one k_scan launch of the default workload (bact-4.6M, one
# 50,000-read batch, F = 2048, read step 1), from an ncu capture of that launch with
# dram__bytes_read.sum and dram__bytes_write.sum (one pass; the command and the figures are in
# profiles/launches_bact-4.6M_50k-read-batch.md).  Other workloads report no traffic.
SCAN_DRAM_BYTES_DEFAULT = 9.018112e6


def workload_config(wl, genome, lengths, F: int, args, world: int = 1) -> dict:
    """The `config` object both arms report for the same workload."""
    Gp = -(-int(genome.shape[0]) // F) * F
    R = int(lengths.shape[0])
    nb = max(1, -(-R // max(1, args.batch)))
    return {"workload": wl.name, "genome_bp": int(genome.shape[0]), "frag_len": F, "padded_bp": Gp,
            "reads": R, "batch_reads": -(-R // nb), "batches": nb,
            "read_lengths": sorted(set(np.asarray(lengths).tolist())),
            "scores": [wl.match, wl.mismatch], "nw": list(wl.nw),
            "parallelism": f"replicas x{world} (read batches per GPU)", "read_step": args.read_step}


def cells_of(lengths: np.ndarray, G: int, F: int, step: int = 1) -> int:
    """Scan cells: read positions taking part (every base, or every other one with read step 2)
    x padded diagonals x 2 strands."""
    Gp = -(-G // F) * F
    return int(((lengths.astype(np.int64) + step - 1) // step).sum()) * Gp * 2


# ------------------------------------------------------------------------------- CPU oracle
def _oracle_job(args):
    import oracle
    genome, F, seq, off, match, mismatch, nw, step = args
    oracle.map_batch(genome, F, seq, off, match, mismatch, nw=nw, step=step)
    return int(off.shape[0] - 1)


def cpu_sample(seq, off, n):
    R = off.shape[0] - 1
    idx = np.linspace(0, R - 1, n).astype(np.int64)
    lens = (off[idx + 1] - off[idx]).astype(np.int64)
    o = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(lens, out=o[1:])
    s = np.concatenate([seq[off[i]:off[i + 1]] for i in idx])
    return s, o


def time_oracle(wl, genome, seq, off, cores, reads_per_core, pool, step=1):
    n = max(1, cores * reads_per_core)
    s, o = cpu_sample(seq, off, n)
    bounds = np.linspace(0, n, cores + 1).astype(int)
    jobs = []
    for a, b in zip(bounds[:-1], bounds[1:]):
        if b <= a:
            continue
        jobs.append((genome, wl.frag_len, np.ascontiguousarray(s[o[a]:o[b]]),
                     np.ascontiguousarray(o[a:b + 1] - o[a]), wl.match, wl.mismatch, wl.nw, step))
    t0 = time.perf_counter()
    done = sum(pool.map(_oracle_job, jobs))
    dt = time.perf_counter() - t0
    cells = cells_of(np.diff(o), genome.shape[0], wl.frag_len, step)
    return cells, done, dt


def host_cores() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    wl, genome, seq, off = workload(args, 0)
    cores = host_cores()
    with ProcessPoolExecutor(max_workers=cores, mp_context=mp.get_context("spawn")) as pool:
        for _ in range(args.warmup):
            time_oracle(wl, genome, seq, off, cores, 1, pool, args.read_step)
        tot_cells = tot_reads = 0
        tot_t = 0.0
        for _ in range(args.steps):
            c, r, dt = time_oracle(wl, genome, seq, off, cores, 1, pool, args.read_step)
            tot_cells += c
            tot_reads += r
            tot_t += dt
    gcups = tot_cells / tot_t / 1e9
    lens = sorted(set(np.diff(off).tolist()))
    span = f"{lens[0]}-{lens[-1]} bp" if len(lens) > 3 else "/".join(str(x) for x in lens) + " bp"
    sample = (f"{cores} reads per step (one per core, evenly spaced over the workload's {span} reads), "
              f"phase one + banded NW")
    line = {
        "impl": "reference", "metric": METRIC, "value": round(gcups, 4), "unit": "GCUPS", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(tot_t / args.steps * 1e3, 3),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int64", "data": "synthetic",
        "config": workload_config(wl, genome, np.diff(off), wl.frag_len, args, args.gpus),
        "reads_per_s": round(tot_reads / tot_t, 3),
        "cpu_baseline": {"value": round(gcups, 4), "unit": "GCUPS", "cores": cores, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": round(gcups, 4), "unit": "GCUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# ------------------------------------------------------------------------------- clocks
class ClockSampler:
    FIELDS = ["clocks.sm", "clocks.max.sm", "power.draw", "clocks_event_reasons.active",
              "clocks_event_reasons.hw_slowdown", "clocks_event_reasons.hw_thermal_slowdown",
              "clocks_event_reasons.sw_thermal_slowdown", "clocks_event_reasons.sw_power_cap"]

    def __init__(self, gpu_index: int):
        self.proc = None
        # samples go to a file given by MSS_CLOCK_LOG, else to a temporary file removed after reading
        self.keep = "MSS_CLOCK_LOG" in os.environ
        self.path = os.environ.get("MSS_CLOCK_LOG") or os.path.join(tempfile.gettempdir(),
                                                                      f"mss_clocks_{os.getpid()}.csv")
        try:
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={','.join(self.FIELDS)}",
                                          "--format=csv,noheader,nounits", "-lms", "200", "-i", str(gpu_index)],
                                         stdout=self.fh, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self) -> dict | None:
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.fh.close()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as fh:
            lines = fh.readlines()
        if not self.keep:
            os.remove(self.path)
        for line in lines:
            p = [x.strip() for x in line.split(",")]
            if len(p) < 8:
                continue
            try:
                sm.append(float(p[0]))
                mx.append(float(p[1]))
            except ValueError:
                continue
            for n, v in zip(names, p[4:8]):
                if v.lower() == "active":
                    reasons.add(n)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


# ------------------------------------------------------------------------------- learned proposal
def measure_proposal(torch, mss, g, wl, genome, max_len, args, stream) -> dict:
    """The second half of the metric: learned proposal + exact rescoring (+ exhaustive fallback
    below a threshold) against the exhaustive scan, on held-out reads of the workload's recipe
    drawn from the same genome.  The model is trained here on exhaustive-scan labels of
    separate training reads; the threshold is chosen on a validation set (the smallest one
    that reaches 99.5% top-1 agreement), then reads/s and agreement are measured on a test set.
    Outside the timed region of the main metric."""
    from paper_1403_2136_gb300.proposal import evaluate, exhaustive_labels, pick_tau, train
    K = 64
    rs = wl.reads
    def draw(n, seed):
        per = [max(1, n * r.count // sum(x.count for x in rs)) for r in rs]
        parts = [gen.make_reads(genome, gen.ReadSpec(**{**r.__dict__, "count": c}), seed + i)
                 for i, (r, c) in enumerate(zip(rs, per))]
        return gen.concat_reads(parts)
    tr = draw(args.prop_train_reads, wl.seed * 97 + 11)
    va = draw(args.prop_eval_reads // 2, wl.seed * 97 + 23)
    te = draw(args.prop_eval_reads, wl.seed * 97 + 37)
    dev = lambda x: torch.from_numpy(np.ascontiguousarray(x)).cuda()  # noqa: E731
    d_tseq, d_toff = dev(tr.seq), dev(tr.offsets)
    t0 = time.perf_counter()
    labels = exhaustive_labels(torch, g, d_tseq, d_toff, tr.count, max_len, wl.match, wl.mismatch)
    label_s = time.perf_counter() - t0
    prop = mss.Proposal(seed=1)
    t0 = time.perf_counter()
    losses = train(torch, prop, g, d_tseq, d_toff, tr.lengths, labels, wl.frag_len, max_len, args.prop_steps, 256,
                   2e-3, 0.05, log=None)
    torch.cuda.synchronize()
    train_s = time.perf_counter() - t0
    prop.build_index(g, max_len)
    taus = [-1e30, 0.3, 0.4, 0.5, 0.6, 0.7, 0.8, 0.9, 1.01]
    d_vseq, d_voff = dev(va.seq), dev(va.offsets)
    ex_v = exhaustive_labels(torch, g, d_vseq, d_voff, va.count, max_len, wl.match, wl.mismatch)
    val = evaluate(torch, prop, g, d_vseq, d_voff, va.count, max_len, wl.match, wl.mismatch, K, taus, ex_v, 1.0)
    tau = pick_tau(val)
    d_eseq, d_eoff = dev(te.seq), dev(te.offsets)
    exhaustive_labels(torch, g, d_eseq, d_eoff, te.count, max_len, wl.match, wl.mismatch)   # warm-up
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    ex = exhaustive_labels(torch, g, d_eseq, d_eoff, te.count, max_len, wl.match, wl.mismatch)
    ex_ms = (time.perf_counter() - t0) * 1e3
    res = {r["tau"]: r for r in evaluate(torch, prop, g, d_eseq, d_eoff, te.count, max_len, wl.match, wl.mismatch, K,
                                         sorted({-1e30, tau}), ex, ex_ms)}
    chosen, free = res[tau], res[-1e30]
    # end to end: reads uploaded from pinned host memory, hits read back, inside the timing
    h_seq, h_off = torch.from_numpy(te.seq).pin_memory(), torch.from_numpy(te.offsets).pin_memory()
    h_hits = torch.empty(te.count * 32, dtype=torch.uint8).pin_memory()
    d_out = torch.empty(te.count * 32, dtype=torch.uint8, device="cuda")
    reps = 3
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(reps):
        d_eseq.copy_(h_seq, non_blocking=True)
        d_eoff.copy_(h_off, non_blocking=True)
        prop.map_reads(g, d_eseq, d_eoff, te.count, max_len, wl.match, wl.mismatch, K, tau, d_out)
        h_hits.copy_(d_out)
    torch.cuda.synchronize()
    te_s = (time.perf_counter() - t0) / reps
    prop.close()
    return {"workload": f"{wl.name.split(':')[0]} genome, held-out reads of its recipe", "K": K, "tau": tau,
            "tau_rule": "smallest threshold with >= 99.5% top-1 agreement on a validation set",
            "train": {"reads": tr.count, "steps": args.prop_steps, "batch": 256, "label_s": round(label_s, 2),
                      "train_s": round(train_s, 2), "loss_first": round(losses[0], 4) if losses else None,
                      "loss_last": round(float(np.mean(losses[-20:])), 4) if losses else None},
            "validation_reads": va.count, "eval_reads": te.count,
            "reads_per_s": chosen["reads_per_s"], "exhaustive_reads_per_s": round(te.count / (ex_ms / 1e3), 1),
            "speedup_vs_exhaustive": chosen["speedup_vs_exhaustive"],
            "top1_agreement": chosen["top1_agreement"], "recall_at_64": chosen["recall_at_64"],
            "fallback_fraction": round(chosen["fallback_reads"] / te.count, 5),
            "changed_mappings": chosen["changed_mappings"],
            "no_fallback": {"reads_per_s": free["reads_per_s"], "top1_agreement": free["top1_agreement"],
                            "recall_at_64": free["recall_at_64"], "speedup_vs_exhaustive": free["speedup_vs_exhaustive"]},
            "e2e": {"reads_per_s": round(te.count / te_s, 1), "h2d_bytes_per_step": int(te.seq.nbytes + te.offsets.nbytes),
                    "d2h_bytes_per_step": int(te.count * 32)}}


# ------------------------------------------------------------------------------- GPU arm
def peak_nominal_tcups(sms: int, clk_mhz: float) -> float:
    """Nominal two-pipe figure: 2 int16 ops per cell (add-relu, max); packed 16-bit x2 work runs
    on two pipes of 16 lanes per SM sub-partition each (integer/DPX and FMA), so at most
    2 pipes x 16 lanes x 2 halves / 2 ops = 32 cells per clock per sub-partition, 4 per SM."""
    return sms * 4 * 32 * clk_mhz * 1e6 / 1e12


def peak_measured_tcups(probe, sms: int, clk_mhz: float):
    """Measured two-pipe figure: the library's probe with PRMT (integer pipe) and f16 FMA-relu
    (FMA pipe) interleaved keeps both 16-lane pipes busy; each packed warp-instruction is 64
    lane operations and a cell needs 2, so cells per SM clock = rate x 32."""
    if not probe:
        return None
    return probe["prmt_and_fma_relu"] * 32 * sms * clk_mhz * 1e6 / 1e12


def mix_ceiling_tcups(probe, sms: int, clk_mhz: float):
    """The scan's own instruction mix measured in isolation (2 PRMT + 2 f16 FMA-relu + 1 three-
    input max per 2 lane pairs of 32 threads x 2 cells = 128 cells per 5 warp-instructions)."""
    if not probe:
        return None
    return probe["scan_mix"] * 128 / 5 * sms * clk_mhz * 1e6 / 1e12


def scan_lanes(max_len: int, match: int, mismatch: int, variant: int) -> str:
    """The 16-bit lanes the scan ran on: f16 x2 (integers up to 2048, exact) when every partial
    sum fits and both scores have an f16 form with a zero low byte, else int16 x2; a tuned
    variant (>= 0) decides by itself."""
    f16_ok = (max_len * match <= 2048 and all(float(np.float16(v)) == v and
              (int(np.array(v, np.float16).view(np.uint16)) & 0xFF) == 0 for v in (match, mismatch)))
    v = variant if variant >= 0 else (1 if f16_ok else 0)
    return "f16x2, exact integers <= 2048" if v == 1 else "int16x2"


def bench_line(*, gcups, t, world, args, reads_s, e2e, launches, sms, probe, max_len, wl, genome, lengths,
               frag_len, tune, tuned, cells_timed, scan_ms, cpu, clk, probe_mhz=None) -> dict:
    """The JSON line of the GPU arm from the measured values (no device work here).  The probe
    rates are per SM clock at probe_mhz, the clock the library counts them at (the device's
    maximum SM clock, which the sampled clocks show the GPU running at under load)."""
    clk_mhz = probe_mhz or 2070.0
    nominal = peak_nominal_tcups(sms, clk_mhz)
    measured = peak_measured_tcups(probe, sms, clk_mhz)
    peak = measured if measured else nominal
    # the integer/DPX pipe alone, measured by the same probe: warp-instructions per SM clock x
    # 32 threads x 2 lanes / 2 ops per cell
    dpx_only = probe["dpx_add_max"] * 32 * sms * clk_mhz * 1e6 / 1e12 if probe else None
    mix = mix_ceiling_tcups(probe, sms, clk_mhz)
    lanes = scan_lanes(max_len, wl.match, wl.mismatch, tune["variant"])
    default_run = (wl.name == gen.workloads()[args.workload].name and args.workload == "bact-4.6M"
                   and args.read_step == 1 and not args.autotune and frag_len == 2048 and args.batch == 50_000
                   and args.threads == 0)
    traffic = SCAN_DRAM_BYTES_DEFAULT if default_run else None
    scan_mean_ms = statistics.mean(scan_ms)
    achieved = cells_timed / (sum(scan_ms) * 1e-3) / 1e12
    src = (f"measured: pipe probe with PRMT (integer pipe) and packed f16 FMA-relu (FMA pipe) interleaved, "
           f"both 16-lane pipes busy: {probe['prmt_and_fma_relu']:.3f} warp-instructions per SM clock x 32 cells "
           f"x {sms} SMs x {clk_mhz:.0f} MHz" if measured else
           f"nominal: {sms} SMs x 4 sub-partitions x 32 cells/clk x {clk_mhz:.0f} MHz")
    return {
        "metric": METRIC, "value": round(gcups, 3), "unit": "GCUPS", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(t * 1e3 / args.steps, 3), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f16" if lanes.startswith("f16") else "int16",
        "data": "synthetic",
        "config": {**workload_config(wl, genome, lengths, frag_len, args, world),
                   "l2": f"flushed between timed steps ({L2_FLUSH_BYTES >> 20} MiB write)",
                   "scan_tune": tune, "autotune": tuned, "scan_lanes": lanes},
        "reads_per_s": round(reads_s, 1),
        "e2e": e2e,
        "gpu_launches": int(launches),
        "roofline": {"bound": "alu", "kernel": "k_scan (phase-one scan + per-read fragment top-4)",
                     "achieved": round(achieved, 3), "peak": round(peak, 3), "unit": "Tcell/s",
                     "frac": round(achieved / peak, 4), "traffic": traffic, "peak_source": src,
                     "peak_nominal": round(nominal, 3), "frac_of_nominal": round(achieved / nominal, 4),
                     "scan_ms_per_step": round(scan_mean_ms, 3),
                     "peak_dpx_pipe_only": round(dpx_only, 3) if dpx_only else None,
                     "frac_of_dpx_pipe_only": round(achieved / dpx_only, 4) if dpx_only else None,
                     "mix_ceiling": round(mix, 3) if mix else None,
                     "frac_of_mix_ceiling": round(achieved / mix, 4) if mix else None,
                     "probe_warp_instr_per_sm_clk": {k: round(v, 4) for k, v in probe.items()} if probe else None},
        "cpu_baseline": cpu,
        "clocks": clk,
    }


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    import torch
    import torch.distributed as dist

    import paper_1403_2136_gb300 as mss

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    wl, genome, seq, off = workload(args, rank)
    lengths = np.diff(off)
    R = int(lengths.shape[0])
    max_len = int(lengths.max())
    nm, nmm, go, ge, W = wl.nw
    parts = batches(seq, off, args.batch)
    nb = len(parts)

    # CPU baseline first (rank 0, N = 1), before the GPU is busy
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        cores = host_cores()
        with ProcessPoolExecutor(max_workers=cores, mp_context=mp.get_context("spawn")) as pool:
            c, r, dt = time_oracle(wl, genome, seq, off, cores, args.cpu_reads_per_core, pool, args.read_step)
        cpu = {"value": round(c / dt / 1e9, 4), "unit": "GCUPS", "cores": cores, "kind": "oracle",
               "sample": f"{r} reads ({args.cpu_reads_per_core} per core, evenly spaced over the workload), "
                         f"phase one + banded NW, {dt:.1f} s wall on {cores} processes",
               "reads_per_s": round(r / dt, 3)}

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    props = torch.cuda.get_device_properties(dev)
    g = mss.mss_load_genome(genome, frag_len=wl.frag_len, max_read_len=max_len)
    info = g.info()
    mss.mss_set_read_step(g, args.read_step)
    if args.threads:
        mss.mss_set_tune(g, threads=args.threads)
    mss.mss_scan_timing(g, True)
    stream = torch.cuda.Stream(device=dev)
    d_parts = [(torch.from_numpy(s).to(dev), torch.from_numpy(o).to(dev), int(o.shape[0] - 1)) for s, o in parts]
    Rb = max(p[2] for p in d_parts)
    d_hits = torch.empty(Rb * 32, dtype=torch.uint8, device=dev)
    d_alns = torch.empty(Rb * 24, dtype=torch.uint8, device=dev)
    stride = 4 * max_len + 64
    d_cig = torch.empty(Rb * stride, dtype=torch.uint8, device=dev)
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)

    def part_cells(F):
        return [cells_of(np.diff(o), genome.shape[0], F, args.read_step) for _, o in parts]

    cells_b = part_cells(wl.frag_len)
    tuned = None
    if args.autotune:
        # an evenly spaced sample of the reads (all lengths), outside the timed region
        n = min(R, args.autotune_reads)
        s_seq, s_off = cpu_sample(seq, off, n)
        t0 = time.perf_counter()
        tuned = mss.mss_autotune(g, torch.from_numpy(s_seq).to(dev), torch.from_numpy(s_off).to(dev), n, max_len,
                                 wl.match, wl.mismatch, allow_frag_len=True, stream=stream)
        tuned["sample_reads"] = n
        tuned["seconds"] = round(time.perf_counter() - t0, 1)
        info = g.info()
        cells_b = part_cells(info["frag_len"])

    def step(b):
        d_seq, d_off, Rk = d_parts[b]
        mss.mss_map_reads_device(g, d_seq, d_off, Rk, max_len, wl.match, wl.mismatch, d_hits, stream=stream)
        mss.nw_align_device(g, d_seq, d_off, Rk, max_len, d_hits, d_alns, d_cig, stride, nm, nmm, go, ge, W,
                            stream=stream)

    with torch.cuda.stream(stream):
        for i in range(args.warmup):
            step(i % nb)
        mss.mss_sync(g, stream=stream)
        # instruction rates per SM clock and the clock they are counted at, outside the timed region
        probe, probe_mhz = mss.mss_probe_pipes() if rank == 0 else (None, None)
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
              for _ in range(args.steps)]
        scan_ms = []
        clocks = ClockSampler(local) if rank == 0 else None
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize(dev)
        launches0 = mss.mss_launch_count(g)
        for k in range(args.steps):
            flush.fill_(k & 0xFF)                    # evict the genome and workspaces from L2
            ev[k][0].record(stream)
            step(k % nb)
            ev[k][1].record(stream)
            scan_ms.append(mss.mss_scan_time_ms(g))  # waits for this step's scan
        torch.cuda.synchronize(dev)
        launches = mss.mss_launch_count(g) - launches0
        if world > 1:
            dist.barrier()
        clk = clocks.stop() if clocks else None
        mss.mss_sync(g, stream=stream)
    step_ms = [a.elapsed_time(b) for a, b in ev]
    t_local = sum(step_ms) / 1e3
    t = t_local
    if world > 1:
        tt = torch.tensor([t_local], dtype=torch.float64, device=dev)
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        t = float(tt.item())
    cells_timed = sum(cells_b[k % nb] for k in range(args.steps))
    reads_timed = sum(d_parts[k % nb][2] for k in range(args.steps))
    gcups = cells_timed * world / t / 1e9
    reads_s = reads_timed * world / t

    # end to end through the host-pointer call (pinned host buffers, copies inside the timing)
    e2e = None
    if not args.no_e2e:
        h_parts = [(torch.from_numpy(s).pin_memory(), torch.from_numpy(o).pin_memory()) for s, o in parts]
        h_hits = torch.empty(Rb * 32, dtype=torch.uint8).pin_memory()
        h_alns = torch.empty(Rb * 24, dtype=torch.uint8).pin_memory()
        h_cig = torch.empty(Rb * stride, dtype=torch.uint8).pin_memory()

        def e2e_step(b):
            h_seq, h_off = h_parts[b]
            Rk = int(h_off.shape[0] - 1)
            mss.mss_map_align(g, h_seq, h_off, wl.match, wl.mismatch, wl.nw, h_hits[:Rk * 32], h_alns[:Rk * 24],
                              h_cig[:Rk * stride], stride, stream=stream)

        e2e_step(0)
        if world > 1:
            dist.barrier()
        e2e_steps = max(1, args.steps)
        t0 = time.perf_counter()
        for k in range(e2e_steps):
            e2e_step(k % nb)
        te = time.perf_counter() - t0
        if world > 1:
            tt = torch.tensor([te], dtype=torch.float64, device=dev)
            dist.all_reduce(tt, op=dist.ReduceOp.MAX)
            te = float(tt.item())
        e_cells = sum(cells_b[k % nb] for k in range(e2e_steps))
        e_reads = sum(int(parts[k % nb][1].shape[0] - 1) for k in range(e2e_steps))
        h2d = sum(int(parts[k % nb][0].nbytes + parts[k % nb][1].nbytes) for k in range(e2e_steps)) // e2e_steps
        d2h = sum(int(parts[k % nb][1].shape[0] - 1) * (32 + 24 + stride) for k in range(e2e_steps)) // e2e_steps
        e2e = {"value": round(e_cells * world / te / 1e9, 3), "unit": "GCUPS",
               "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
               "reads_per_s": round(e_reads * world / te, 1)}

    prop = None
    if rank == 0 and not args.no_proposal:
        # on the default stream: the proposal helpers pass no stream to the library, so torch's
        # copies and the library's launches are ordered on the same stream
        torch.cuda.synchronize(dev)
        prop = measure_proposal(torch, mss, g, wl, genome, max_len, args, None)

    if rank == 0:
        line = bench_line(
            gcups=gcups, t=t, world=world, args=args, reads_s=reads_s, e2e=e2e, launches=launches,
            sms=props.multi_processor_count, probe=probe, probe_mhz=probe_mhz, max_len=max_len, wl=wl, genome=genome,
            lengths=lengths, frag_len=info["frag_len"], tune=mss.mss_get_tune(g), tuned=tuned,
            cells_timed=cells_timed, scan_ms=scan_ms, cpu=cpu, clk=clk)
        if prop is not None:
            line["proposal"] = prop
        print(json.dumps(line), flush=True)
    g.close()
    if world > 1:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
