"""The GPU arm's JSON line is assembled from measured values by a pure function; these CPU
checks run it on made-up measurements so that a mistake in the assembly shows here, not on the
GPU machine.  The keys follow the benchmark contract (metric, value, unit, config, e2e, roofline,
cpu_baseline, clocks, gpu_launches, ...)."""
import json
import sys

import numpy as np

import bench
import gen


def _line(monkeypatch, variant=-1, workload="bact-4.6M"):
    monkeypatch.setattr(sys, "argv", ["bench.py", "--workload", workload])
    args = bench.parse()
    wl = gen.workloads()[args.workload]
    genome = np.zeros(4_600_000, dtype=np.uint8)
    lengths = np.array([100] * 4 + [150] * 4, dtype=np.int64)
    cells = bench.cells_of(lengths, genome.shape[0], wl.frag_len)
    tune = {"variant": variant, "pairs": 0, "queries": 0, "ctas_per_sm": 0, "min_items_per_cta": 0, "threads": 0}
    return bench.bench_line(
        gcups=20000.0, t=68.6, world=1, args=args, reads_s=17500.0,
        e2e={"value": 19900.0, "unit": "GCUPS", "h2d_bytes_per_step": 10, "d2h_bytes_per_step": 20},
        launches=18, sms=152, probe={"dpx_add_max": 1.97, "fma_relu": 1.9, "prmt_and_fma_relu": 3.5, "prmt": 1.9, "max3": 1.9, "scan_mix": 2.5, "dpx_and_fma_relu": 2.3}, probe_mhz=2070.0, max_len=int(lengths.max()), wl=wl, genome=genome,
        lengths=lengths, frag_len=wl.frag_len, tune=tune, tuned=None, cells_timed=3 * cells, scan_ms=[22748.0] * 3,
        cpu={"value": 7.4, "unit": "GCUPS", "cores": 16, "kind": "oracle", "sample": "32 reads"},
        clk={"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "reasons": [], "samples": 300})


def test_line_has_the_contract_keys(monkeypatch):
    line = _line(monkeypatch)
    json.dumps(line)
    for k in ["metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "scaling",
              "vs_baseline", "dtype", "data", "config", "e2e", "gpu_launches", "roofline", "cpu_baseline", "clocks"]:
        assert k in line, k
    assert line["config"]["workload"].startswith("bact-4.6M")
    assert line["higher_is_better"] is True and line["scaling"] == "weak" and line["n_gpus"] == 1
    r = line["roofline"]
    for k in ["bound", "achieved", "peak", "unit", "frac", "traffic"]:
        assert k in r, k
    assert abs(r["frac"] - r["achieved"] / r["peak"]) < 1e-3
    assert r["traffic"] == bench.SCAN_DRAM_BYTES_DEFAULT      # default workload: the captured bytes
    # the measured both-pipe probe rate (3.5 warp-instructions per SM clock) x 32 cells
    assert abs(r["peak"] - 3.5 * 32 * 152 * 2070e6 / 1e12) < 1e-3
    assert abs(r["mix_ceiling"] - 2.5 * 128 / 5 * 152 * 2070e6 / 1e12) < 1e-3
    assert abs(r["peak_nominal"] - 152 * 4 * 32 * 2070e6 / 1e12) < 1e-3
    assert abs(r["achieved"] - 3 * bench.cells_of(np.array([100] * 4 + [150] * 4), 4_600_000, 2048) /
               (3 * 22.748) / 1e12) < 1e-3
    assert line["config"]["scan_lanes"].startswith("f16x2") and line["dtype"] == "f16"
    assert line["config"]["batches"] == 1 and line["config"]["batch_reads"] == 8
    assert line["gpu_launches"] == 18


def test_other_workload_reports_no_traffic(monkeypatch):
    line = _line(monkeypatch, workload="chrom-230M")
    assert line["roofline"]["traffic"] is None


def test_scan_lanes():
    assert bench.scan_lanes(150, 5, -4, -1).startswith("f16x2")
    assert bench.scan_lanes(2000, 2, -3, -1) == "int16x2"     # partial sums above 2048
    assert bench.scan_lanes(100, 9, -1, -1) == "int16x2"      # f16(9) = 0x4880: nonzero low byte
    assert bench.scan_lanes(150, 5, -4, 0) == "int16x2"       # a tuned variant decides


def test_batches_deal_the_reads_evenly():
    wl = gen.scaled(gen.workloads()["bact-4.6M"], genome_len=20_000, reads=40)
    genome = gen.make_genome(wl.genome, wl.seed)
    reads = gen.read_set(wl, genome)
    parts = bench.batches(reads.seq, reads.offsets, 8)
    assert len(parts) == 5
    for b, (s, o) in enumerate(parts):
        idx = gen.batch_index(reads.count, 5, b)
        assert o.shape[0] - 1 == idx.shape[0]
        for j, i in enumerate(idx):
            assert s[o[j]:o[j + 1]].tobytes() == reads.read(int(i))
        assert sorted(set(np.diff(o).tolist())) == [100, 150]     # both lengths in every batch
