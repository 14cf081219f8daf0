"""Training and evaluation of the learned fragment proposal (host orchestration only).

Labels come from the exhaustive scan: for each training read its best fragment, strand and
second-best fragment.  A training step takes B reads (on their labelled strand) against the
candidate set of the batch (every read's best fragment and its second-best fragment as a hard
negative); the loss is the softmax cross-entropy of the read's best fragment.  Evaluation maps
held-out reads with the proposal (top K per read, exact rescoring, exhaustive fallback below a
score threshold) and compares with the exhaustive scan: top-1 agreement (the chosen fragment's
exact score equals the exhaustive best score: equal-score fragments are equally valid), strict
fragment agreement, recall at K (the exhaustive best fragment is among the candidates), and
the speedup over the exhaustive scan on the same GPU.

Every compute step runs in libmaxss kernels; this module draws batches and keeps score.

    python -m paper_1403_2136_gb300.proposal [--genome-len N] [--train-reads N] [--steps N] ...
"""
from __future__ import annotations

import argparse
import dataclasses
import json
import os
import sys
import time

import numpy as np

from . import HIT_DTYPE, MssError, Proposal, hits_from_bytes, mss_load_genome, mss_map_reads_device, mss_sync


def _dev(torch, x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def exhaustive_labels(torch, g, d_seq, d_off, R, max_len, match, mismatch, stream=None):
    d_hits = torch.empty(R * 32, dtype=torch.uint8, device="cuda")
    mss_map_reads_device(g, d_seq, d_off, R, max_len, match, mismatch, d_hits, stream=stream)
    mss_sync(g, stream=stream)
    return hits_from_bytes(d_hits.cpu()).copy()


def train(torch, prop: Proposal, g, d_seq, d_off, lens, labels, F: int, max_len: int, steps: int, batch: int,
          lr: float, temperature: float, seed: int = 1, log_every: int = 50, log=None):
    """Contrastive training on exhaustive-scan labels.  Returns the list of step losses."""
    rng = np.random.default_rng(seed)
    ok = np.nonzero((labels["best_score"] > 0) & ((labels["flags"] & 1) == 0))[0]  # confidently mapped reads
    win = F + max_len - 1
    B = min(batch, ok.size)
    d_rcodes = torch.empty(B * max_len, dtype=torch.uint8, device="cuda")
    d_rlens = torch.empty(B, dtype=torch.int32, device="cuda")
    d_ccodes = torch.empty(2 * B * win, dtype=torch.uint8, device="cuda")
    d_clens = torch.empty(2 * B, dtype=torch.int32, device="cuda")
    losses = []
    for step in range(steps):
        pick = rng.choice(ok, size=B, replace=False)
        strand = labels["strand"][pick].astype(np.int8)
        prop.read_codes(d_seq, d_off, _dev(torch, pick.astype(np.int32)), _dev(torch, strand), B, max_len, d_rcodes,
                        d_rlens)
        b1 = labels["best_frag"][pick]
        b2 = labels["second_frag"][pick]
        cand = np.unique(np.concatenate([b1, b2[b2 >= 0]]))
        pos = {int(f): i for i, f in enumerate(cand)}
        lab = np.array([pos[int(f)] for f in b1], dtype=np.int32)
        C = cand.size
        prop.window_codes(g, _dev(torch, cand.astype(np.int64) * F), C, win, win, d_ccodes, d_clens)
        loss = prop.train_step(d_rcodes, d_rlens, max_len, B, int(lens[pick].max()), d_ccodes, d_clens, win, C, win,
                               _dev(torch, lab), lr=lr, temperature=temperature)
        losses.append(loss)
        if log is not None and (step % log_every == 0 or step == steps - 1):
            log(f"step {step} loss {loss:.4f} (B={B}, C={C})")
    return losses


def evaluate(torch, prop: Proposal, g, d_seq, d_off, R, max_len, match, mismatch, K, taus, exhaustive_hits,
             exhaustive_ms):
    """Proposal mapping at each threshold tau vs the exhaustive result."""
    out = []
    d_out = torch.empty(R * 32, dtype=torch.uint8, device="cuda")
    d_cand = torch.empty(R * K, dtype=torch.int32, device="cuda")
    d_top = torch.empty(R, dtype=torch.float32, device="cuda")
    ex = exhaustive_hits
    for tau in taus:
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        nfb = prop.map_reads(g, d_seq, d_off, R, max_len, match, mismatch, K, tau, d_out, d_cand=d_cand, d_top=d_top)
        torch.cuda.synchronize()
        ms = (time.perf_counter() - t0) * 1e3
        h = hits_from_bytes(d_out.cpu())
        cand = d_cand.cpu().numpy().reshape(R, K)
        agree = float(np.mean(h["best_score"] == ex["best_score"]))
        strict = float(np.mean(h["best_frag"] == ex["best_frag"]))
        recall = float(np.mean([ex["best_frag"][i] in cand[i] for i in range(R)]))
        out.append({"tau": tau, "fallback_reads": nfb, "top1_agreement": round(agree, 5),
                    "strict_fragment_agreement": round(strict, 5), f"recall_at_{K}": round(recall, 5),
                    "ms": round(ms, 1), "reads_per_s": round(R / (ms / 1e3), 1),
                    "speedup_vs_exhaustive": round(exhaustive_ms / ms, 2),
                    "changed_mappings": int(np.sum(h["best_score"] != ex["best_score"]))})
    return out


def main(argv=None):
    import torch

    import gen

    ap = argparse.ArgumentParser()
    ap.add_argument("--workload", default="chrom-230M", choices=["chrom-230M", "ancient-2.4G"],
                    help="genome and read shape (the genome is scaled to --genome-len)")
    ap.add_argument("--genome-len", type=int, default=23_000_000, help="genome length (0: the workload's own)")
    ap.add_argument("--train-reads", type=int, default=60_000)
    ap.add_argument("--eval-reads", type=int, default=20_000)
    ap.add_argument("--steps", type=int, default=800)
    ap.add_argument("--batch", type=int, default=256)
    ap.add_argument("--lr", type=float, default=2e-3)
    ap.add_argument("--temperature", type=float, default=0.05)
    ap.add_argument("--K", type=int, default=64)
    ap.add_argument("--taus", type=str, default="-1e30,0.5,0.7,0.8,0.9", help="comma-separated; pass as --taus=...")
    ap.add_argument("--checkpoint", type=str, default="")
    args = ap.parse_args(argv)
    log = lambda m: print(m, file=sys.stderr, flush=True)  # noqa: E731

    wl = gen.workloads()[args.workload]
    if args.genome_len:
        wl = gen.scaled(wl, genome_len=args.genome_len)
    t0 = time.perf_counter()
    genome = gen.make_genome(wl.genome, wl.seed)
    log(f"genome of {genome.shape[0]} bases in {time.perf_counter() - t0:.1f} s")
    F = 2048
    spec = wl.reads[0]
    max_len = 250 if spec.lognormal is None else int(spec.lognormal[3])
    tr = gen.make_reads(genome, dataclasses.replace(spec, count=max(args.train_reads, 1)), wl.seed * 7 + 1)
    ev = gen.make_reads(genome, dataclasses.replace(spec, count=args.eval_reads), wl.seed * 7 + 2)
    g = mss_load_genome(genome, frag_len=F, max_read_len=max_len)
    NF = g.info()["num_frags"]
    d_tseq, d_toff = _dev(torch, tr.seq), _dev(torch, tr.offsets)
    t0 = time.perf_counter()
    labels = exhaustive_labels(torch, g, d_tseq, d_toff, tr.count, max_len, wl.match, wl.mismatch)
    label_s = time.perf_counter() - t0
    log(f"labels for {tr.count} reads in {label_s:.1f} s")
    prop = Proposal(seed=1)
    t0 = time.perf_counter()
    losses = train(torch, prop, g, d_tseq, d_toff, tr.lengths, labels, F, max_len, args.steps, args.batch, args.lr,
                   args.temperature, log=log) if args.steps > 0 else []
    torch.cuda.synchronize()
    train_s = time.perf_counter() - t0
    if args.checkpoint:
        prop.save(args.checkpoint)
    t0 = time.perf_counter()
    prop.build_index(g, max_len)
    torch.cuda.synchronize()
    index_s = time.perf_counter() - t0
    d_eseq, d_eoff = _dev(torch, ev.seq), _dev(torch, ev.offsets)
    exhaustive_labels(torch, g, d_eseq, d_eoff, ev.count, max_len, wl.match, wl.mismatch)  # warm-up
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    ex = exhaustive_labels(torch, g, d_eseq, d_eoff, ev.count, max_len, wl.match, wl.mismatch)
    ex_ms = (time.perf_counter() - t0) * 1e3
    taus = [float(x) for x in args.taus.split(",")]
    res = evaluate(torch, prop, g, d_eseq, d_eoff, ev.count, max_len, wl.match, wl.mismatch, args.K, taus, ex, ex_ms)
    line = {"metric": "learned proposal + exact rescoring vs exhaustive scan (top-1 agreement, recall, speedup)",
            "workload": wl.name, "genome_bp": int(genome.shape[0]), "frag_len": F, "num_frags": int(NF),
            "train_reads": tr.count, "train_steps": args.steps, "batch": args.batch,
            "loss_first": round(losses[0], 4) if losses else None,
            "loss_last": round(float(np.mean(losses[-20:])), 4) if losses else None,
            "loss_curve": [round(float(np.mean(c)), 4) for c in np.array_split(np.asarray(losses), min(10, len(losses)))]
            if losses else [],
            "label_s": round(label_s, 2), "train_s": round(train_s, 2), "index_s": round(index_s, 2),
            "eval_reads": ev.count, "exhaustive_ms": round(ex_ms, 1),
            "exhaustive_reads_per_s": round(ev.count / (ex_ms / 1e3), 1), "K": args.K, "results": res}
    print(json.dumps(line), flush=True)
    prop.close()
    g.close()


if __name__ == "__main__":
    main()
