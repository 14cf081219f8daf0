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


def mine_hard(torch, prop: Proposal, g, d_seq, d_off, R, max_len, match, mismatch, K, stream=None):
    """The model's own top K fragments of every training read over the whole fragment index
    (index rebuilt with the current weights): the hard negatives of the next steps."""
    prop.build_index(g, max_len, stream=stream)
    d_out = torch.empty(R * 32, dtype=torch.uint8, device="cuda")
    d_cand = torch.empty(R * K, dtype=torch.int32, device="cuda")
    prop.map_reads(g, d_seq, d_off, R, max_len, match, mismatch, K, -1e30, d_out, d_cand=d_cand, stream=stream)
    torch.cuda.synchronize()
    return d_cand.cpu().numpy().reshape(R, K)


def train(torch, prop: Proposal, g, d_seq, d_off, lens, labels, F: int, max_len: int, steps: int, batch: int,
          lr: float, temperature: float, seed: int = 1, log_every: int = 50, log=None, mine_every: int = 0,
          hard: int = 0, match: int = 5, mismatch: int = -4, K: int = 64):
    """Contrastive training on exhaustive-scan labels.  The candidates of a step are the best
    and second-best fragments of its reads and, with mining on, each read's `hard` highest-
    ranked wrong fragments from the model's own top K over the whole index (refreshed every
    `mine_every` steps).  Returns the list of step losses."""
    rng = np.random.default_rng(seed)
    ok = np.nonzero((labels["best_score"] > 0) & ((labels["flags"] & 1) == 0))[0]  # confidently mapped reads
    win = F + max_len - 1
    B = min(batch, ok.size)
    cmax = min(1024, B * (2 + hard))
    d_rcodes = torch.empty(B * max_len, dtype=torch.uint8, device="cuda")
    d_rlens = torch.empty(B, dtype=torch.int32, device="cuda")
    d_ccodes = torch.empty(cmax * win, dtype=torch.uint8, device="cuda")
    d_clens = torch.empty(cmax, dtype=torch.int32, device="cuda")
    losses = []
    mined = None
    R = lens.shape[0]
    for step in range(steps):
        if hard > 0 and mine_every > 0 and step % mine_every == 0 and step > 0:
            mined = mine_hard(torch, prop, g, d_seq, d_off, R, max_len, match, mismatch, K)
        pick = rng.choice(ok, size=B, replace=False)
        strand = labels["strand"][pick].astype(np.int8)
        prop.read_codes(d_seq, d_off, _dev(torch, pick.astype(np.int32)), _dev(torch, strand), B, max_len, d_rcodes,
                        d_rlens)
        b1 = labels["best_frag"][pick]
        b2 = labels["second_frag"][pick]
        parts = [b1, b2[b2 >= 0]]
        if mined is not None:
            m = mined[pick]
            wrong = m != b1[:, None]
            # the first `hard` wrong fragments of each read's ranked list
            rank = np.cumsum(wrong, axis=1)
            parts.append(m[wrong & (rank <= hard) & (m >= 0)])
        positives = np.unique(b1)
        negatives = np.setdiff1d(np.concatenate(parts[1:]), positives)[:cmax - positives.size]
        cand = np.concatenate([positives, negatives])
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


def _genome_for(gen, spec: str):
    """'name' or 'name@length' (the workload's genome recipe, scaled to length)."""
    name, _, ln = spec.partition("@")
    wl = gen.workloads()[name]
    if ln:
        wl = gen.scaled(wl, genome_len=int(ln))
    return wl, gen.make_genome(wl.genome, wl.seed)


def pick_tau(rows, target: float = 0.995):
    """The smallest threshold whose top-1 agreement reaches the target (rows of evaluate());
    the largest threshold when none does."""
    ok = [r for r in rows if r["top1_agreement"] >= target]
    return min(ok, key=lambda r: r["tau"])["tau"] if ok else max(r["tau"] for r in rows)


def at_scale(torch, gen, prop, args, rspec, max_len, F, taus, log):
    """All --scale-reads reads through the proposal without fallback (top K, exact rescoring),
    timed; an evenly spaced subsample through the exhaustive scan, timed; agreement and the
    fallback fraction at each threshold on the subsample (a read below the threshold falls back
    and then agrees by construction).  Running the fallback for every read of the full set is
    left out when it would take the exhaustive scan's time (the rate is reported)."""
    spec, _, _ = args.evals.split(",")[0].partition(":")
    ewl, eg = _genome_for(gen, spec)
    t0 = time.perf_counter()
    ev = gen.make_reads(eg, dataclasses.replace(rspec, count=args.scale_reads), ewl.seed * 7 + 3)
    log(f"{ev.count} reads drawn in {time.perf_counter() - t0:.1f} s")
    g = mss_load_genome(eg, frag_len=F, max_read_len=max_len)
    NF = g.info()["num_frags"]
    t0 = time.perf_counter()
    prop.build_index(g, max_len)
    torch.cuda.synchronize()
    index_s = time.perf_counter() - t0
    R, K = ev.count, args.K
    d_seq, d_off = _dev(torch, ev.seq), _dev(torch, ev.offsets)
    d_out = torch.empty(R * 32, dtype=torch.uint8, device="cuda")
    d_cand = torch.empty(R * K, dtype=torch.int32, device="cuda")
    d_top = torch.empty(R, dtype=torch.float32, device="cuda")
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    prop.map_reads(g, d_seq, d_off, R, max_len, ewl.match, ewl.mismatch, K, -1e30, d_out, d_cand=d_cand, d_top=d_top)
    torch.cuda.synchronize()
    prop_s = time.perf_counter() - t0
    h = hits_from_bytes(d_out.cpu())
    top = d_top.cpu().numpy()
    cand = d_cand.cpu().numpy().reshape(R, K)
    sub = np.linspace(0, R - 1, min(R, args.subsample)).astype(np.int64)
    sr = ev.subset(sub)
    d_sseq, d_soff = _dev(torch, sr.seq), _dev(torch, sr.offsets)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    ex = exhaustive_labels(torch, g, d_sseq, d_soff, sr.count, max_len, ewl.match, ewl.mismatch)
    ex_s = time.perf_counter() - t0
    g.close()
    agree = h["best_score"][sub] == ex["best_score"]
    recall = float(np.mean([ex["best_frag"][i] in cand[s] for i, s in enumerate(sub)]))
    rows = []
    ex_rate = sr.count / ex_s
    for tau in taus:
        fb = top[sub] < tau
        frac = float(np.mean(fb))
        # proposal for every read, then the exhaustive scan for the fallback fraction
        rate = 1.0 / (prop_s / R + frac / ex_rate)
        rows.append({"tau": tau, "fallback_fraction": round(frac, 5),
                     "top1_agreement": round(float(np.mean(agree | fb)), 5),
                     "reads_per_s_with_fallback": round(rate, 1), "speedup_vs_exhaustive": round(rate / ex_rate, 3)})
    return {"genome": ewl.name, "genome_bp": int(eg.shape[0]), "num_frags": int(NF), "index_s": round(index_s, 2),
            "reads": R, "K": K, "proposal_s": round(prop_s, 2), "proposal_reads_per_s": round(R / prop_s, 1),
            "subsample": sr.count, "exhaustive_s": round(ex_s, 2), "exhaustive_reads_per_s": round(ex_rate, 2),
            "recall_at_K_subsample": round(recall, 5), "top1_agreement_no_fallback": round(float(np.mean(agree)), 5),
            "taus": rows}


def main(argv=None):
    import torch

    import gen

    ap = argparse.ArgumentParser()
    ap.add_argument("--train-genome", default="bact-4.6M", help="genome of the training labels: name[@length]")
    ap.add_argument("--read-shape", default="chrom-230M", help="workload whose read recipe draws the reads")
    ap.add_argument("--train-reads", type=int, default=60_000)
    ap.add_argument("--steps", type=int, default=800)
    ap.add_argument("--batch", type=int, default=256)
    ap.add_argument("--lr", type=float, default=2e-3)
    ap.add_argument("--temperature", type=float, default=0.05)
    ap.add_argument("--mine-every", type=int, default=0, help="refresh the hard negatives every N steps (0: off)")
    ap.add_argument("--hard", type=int, default=2, help="hard negatives per read from the model's own top K")
    ap.add_argument("--K", type=int, default=64)
    ap.add_argument("--evals", default="chrom-230M@23000000",
                    help="comma-separated evaluation genomes name[@length][:reads] (held-out reads of the read "
                         "shape; the read count overrides --eval-reads for that genome)")
    ap.add_argument("--eval-reads", type=int, default=20_000, help="held-out reads per genome (half choose tau)")
    ap.add_argument("--taus", type=str, default="-1e30,0.3,0.4,0.5,0.6,0.7,0.8,0.9",
                    help="comma-separated; pass as --taus=...")
    ap.add_argument("--scale-reads", type=int, default=0,
                    help="instead of the evaluation above: map this many reads of the read shape on the first "
                         "evaluation genome with the proposal (no fallback), and compare a subsample with the "
                         "exhaustive scan")
    ap.add_argument("--subsample", type=int, default=20_000, help="exhaustive subsample of --scale-reads")
    ap.add_argument("--checkpoint", type=str, default="", help="save the trained weights here")
    ap.add_argument("--load", type=str, default="", help="start from these weights")
    ap.add_argument("--pooling", choices=["max", "mean"], default="max",
                    help="how the last layer's positions become one vector (a checkpoint's own setting wins)")
    args = ap.parse_args(argv)
    log = lambda m: print(m, file=sys.stderr, flush=True)  # noqa: E731

    F = 2048
    rspec = gen.workloads()[args.read_shape].reads[0]
    max_len = 250 if rspec.lognormal is None else int(rspec.lognormal[3])
    wl, genome = _genome_for(gen, args.train_genome)
    tr = gen.make_reads(genome, dataclasses.replace(rspec, count=max(args.train_reads, 1)), wl.seed * 7 + 1)
    g = mss_load_genome(genome, frag_len=F, max_read_len=max_len)
    d_tseq, d_toff = _dev(torch, tr.seq), _dev(torch, tr.offsets)
    t0 = time.perf_counter()
    labels = exhaustive_labels(torch, g, d_tseq, d_toff, tr.count, max_len, wl.match, wl.mismatch)
    label_s = time.perf_counter() - t0
    log(f"labels for {tr.count} reads on {genome.shape[0]} bp in {label_s:.1f} s")
    prop = Proposal(seed=1)
    prop.pooling = args.pooling
    if args.load:
        prop.load(args.load)
    t0 = time.perf_counter()
    losses = train(torch, prop, g, d_tseq, d_toff, tr.lengths, labels, F, max_len, args.steps, args.batch, args.lr,
                   args.temperature, log=log, mine_every=args.mine_every, hard=args.hard if args.mine_every else 0,
                   match=wl.match, mismatch=wl.mismatch, K=args.K) if args.steps > 0 else []
    torch.cuda.synchronize()
    train_s = time.perf_counter() - t0
    if args.checkpoint:
        prop.save(args.checkpoint)
    g.close()
    del d_tseq, d_toff

    taus = [float(x) for x in args.taus.split(",")]
    if args.scale_reads > 0:
        scale = at_scale(torch, gen, prop, args, rspec, max_len, F, taus, log)
        print(json.dumps({"metric": "learned proposal at scale (no fallback) vs an exhaustive subsample",
                          "train_genome": wl.name, "train_reads": tr.count, "train_steps": args.steps,
                          "pooling": prop.pooling, "loaded": args.load or None, **scale}), flush=True)
        prop.close()
        return
    evals = []
    for spec in args.evals.split(","):
        spec, _, nr = spec.partition(":")
        ewl, eg = _genome_for(gen, spec)
        ev = gen.make_reads(eg, dataclasses.replace(rspec, count=int(nr) if nr else args.eval_reads), ewl.seed * 7 + 2)
        half = ev.count // 2
        sets = [ev.subset(np.arange(0, half)), ev.subset(np.arange(half, ev.count))]
        g = mss_load_genome(eg, frag_len=F, max_read_len=max_len)
        NF = g.info()["num_frags"]
        t0 = time.perf_counter()
        prop.build_index(g, max_len)
        torch.cuda.synchronize()
        index_s = time.perf_counter() - t0
        rows = []
        for part in sets:
            d_eseq, d_eoff = _dev(torch, part.seq), _dev(torch, part.offsets)
            exhaustive_labels(torch, g, d_eseq, d_eoff, part.count, max_len, ewl.match, ewl.mismatch)  # warm-up
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            ex = exhaustive_labels(torch, g, d_eseq, d_eoff, part.count, max_len, ewl.match, ewl.mismatch)
            ex_ms = (time.perf_counter() - t0) * 1e3
            rows.append((part, d_eseq, d_eoff, ex, ex_ms))
        # tau chosen on the first half, reported on the second
        part, d_eseq, d_eoff, ex, ex_ms = rows[0]
        val = evaluate(torch, prop, g, d_eseq, d_eoff, part.count, max_len, ewl.match, ewl.mismatch, args.K, taus, ex,
                       ex_ms)
        tau = pick_tau(val)
        part, d_eseq, d_eoff, ex, ex_ms = rows[1]
        test = evaluate(torch, prop, g, d_eseq, d_eoff, part.count, max_len, ewl.match, ewl.mismatch, args.K,
                        sorted(set([-1e30, tau])), ex, ex_ms)
        evals.append({"genome": ewl.name, "genome_bp": int(eg.shape[0]), "num_frags": int(NF),
                      "index_s": round(index_s, 2), "eval_reads": part.count,
                      "exhaustive_reads_per_s": round(part.count / (ex_ms / 1e3), 1),
                      "tau_chosen_on_validation": tau, "validation": val, "test": test})
        log(json.dumps(evals[-1]))
        g.close()
    line = {"metric": "learned proposal + exact rescoring vs exhaustive scan (top-1 agreement, recall, speedup)",
            "train_genome": wl.name, "train_genome_bp": int(genome.shape[0]), "frag_len": F,
            "read_shape": args.read_shape, "train_reads": tr.count, "train_steps": args.steps, "batch": args.batch,
            "mine_every": args.mine_every, "hard": args.hard if args.mine_every else 0, "pooling": prop.pooling,
            "loss_first": round(losses[0], 4) if losses else None,
            "loss_last": round(float(np.mean(losses[-20:])), 4) if losses else None,
            "loss_curve": [round(float(np.mean(c)), 4) for c in np.array_split(np.asarray(losses), min(10, len(losses)))]
            if losses else [],
            "label_s": round(label_s, 2), "train_s": round(train_s, 2), "K": args.K, "evals": evals}
    print(json.dumps(line), flush=True)
    prop.close()


if __name__ == "__main__":
    main()
