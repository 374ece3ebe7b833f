"""Train the capacity predictor's network (run on a GPU).

    python -m paper_2401_02756_gb300.train_predictor --samples 10000 \\
        --out paper_2401_02756_gb300/predictor_weights.npz

Each sample is a read set of the batched-build distribution
(``synth.batch_sample`` under its own seed, so no training sample is one of
the benchmark's).  Its features are the sketch registers from
``dbg_sketch_reads`` and its label is ln of the exact distinct-vertex count
from the builder itself (``dbg_insert_reads`` + ``dbg_stats``).  The samples
are split 80 / 10 / 10 into training, validation (to keep the best weights)
and test sets; the network is trained with the library's Adam step on
mini-batches.  The report (``.json`` beside the weights) gives the test
set's relative errors of the network and of the HyperLogLog estimate, and the
margin: the largest ratio true / predicted over all samples, plus 2 %.

Read sets are generated on CPU worker processes (started with ``spawn``
before the first GPU call) while the GPU builds earlier ones.
"""

from __future__ import annotations

import argparse
import json
import math
import multiprocessing as mp
import os
import time

import numpy as np

from . import dbg, synth
from .predictor import REG_STRIDE

TRAIN_SEED = 17  # sample seed of the training distribution (the benchmark uses 4)


def label_samples(n: int, seed: int, workers: int, log=print):
    """Registers (int32 [n, REG_STRIDE]) and exact distinct counts of n samples."""
    import torch
    ctx = mp.get_context("spawn")
    regs = torch.zeros(n, REG_STRIDE, dtype=torch.int32, device="cuda")
    D = np.zeros(n, dtype=np.int64)
    ks = np.zeros(n, dtype=np.int32)
    graphs = {}
    t0 = time.time()
    with ctx.Pool(workers) as pool:
        for done, (i, k, packed, offsets, edges) in enumerate(
                pool.imap_unordered(synth.batch_sample_arrays, [(i, seed) for i in range(n)],
                                   chunksize=2)):
            p = torch.from_numpy(np.concatenate([packed, np.zeros(16, np.uint8)])).cuda()
            o = torch.from_numpy(offsets.view(np.int64)).cuda()
            dbg.sketch(k, p, o, registers=regs[i])
            if k not in graphs:
                # the largest sample (2 Mbp at 60x, 0.5 % errors) has about 2e7 vertices
                graphs[k] = dbg.Graph(k, 48_000_000)
            g = graphs[k]
            g.reset()
            g.insert(p, o)
            nv, ne = g.stats()
            if ne != edges:
                raise RuntimeError(f"sample {i}: {ne} edges counted, {edges} expected")
            D[i], ks[i] = nv, k
            if log and (done + 1) % 1000 == 0:
                log(f"  labelled {done + 1}/{n} ({time.time() - t0:.0f} s)")
    for g in graphs.values():
        g.close()
    if np.any(regs[:, -1].cpu().numpy() != dbg.OK):
        raise RuntimeError("a sketch reported an error")
    return regs, D, ks


def train(regs, D, split, steps: int, batch: int, lr: float, seed: int, log=print):
    """Train on the rows in split["train"], keep the weights best on
    split["val"]; returns the parameters (device float32)."""
    import torch
    n = regs.shape[0]
    X = torch.empty(n, dbg.MLP_INPUTS, dtype=torch.float32, device="cuda")
    dbg.mlp_features(regs, X, n, stride=REG_STRIDE)
    T = torch.from_numpy(np.log(D.astype(np.float64)).astype(np.float32)).cuda()
    tr = torch.from_numpy(split["train"]).cuda()
    va = split["val"]
    P = torch.empty(dbg.MLP_PARAMS, dtype=torch.float32, device="cuda")
    dbg.mlp_init(P, seed)
    P[-1] = float(T[tr].mean())  # the output bias starts at the mean label
    G, M, V = (torch.zeros_like(P) for _ in range(3))
    w = torch.empty(dbg.mlp_work_floats(batch), dtype=torch.float32, device="cuda")
    wv = torch.empty(dbg.mlp_work_floats(len(va)), dtype=torch.float32, device="cuda")
    yv = torch.empty(len(va), dtype=torch.float32, device="cuda")
    Xv, Tv = X[torch.from_numpy(va).cuda()].contiguous(), T[torch.from_numpy(va).cuda()]
    gen = torch.Generator(device="cpu").manual_seed(seed)
    best, best_err = P.clone(), float("inf")
    loss = torch.zeros(1, dtype=torch.float32, device="cuda")
    for s in range(1, steps + 1):
        idx = tr[torch.randint(0, len(tr), (batch,), generator=gen).cuda()]
        xb, tb = X[idx].contiguous(), T[idx].contiguous()
        rate = lr * 0.5 * (1 + math.cos(math.pi * (s - 1) / steps))  # cosine decay
        dbg.mlp_train_step(P, G, M, V, s, max(rate, 1e-7), xb, tb, w, loss=loss)
        if s % 100 == 0 or s == steps:
            dbg.mlp_forward(P, Xv, yv, wv)
            err = float((yv - Tv).abs().mean())
            if err < best_err:
                best, best_err = P.clone(), err
            if log and s % 1000 == 0:
                log(f"  step {s}: batch loss {float(loss):.5f}, val mean |ln error| {err:.5f}")
    return best


def evaluate(P, regs, D, rows):
    """Relative errors of the network and of HyperLogLog on the given rows."""
    import torch
    from .predictor import CapacityPredictor
    pred = CapacityPredictor(params=P, margin=1.0)
    sel = regs[torch.from_numpy(rows).cuda()].contiguous()
    out = pred.predict_registers(sel, len(rows))
    mlp = np.array([p.mlp for p in out])
    hll = np.array([p.hll for p in out])
    return mlp, hll


def _summary(est, truth):
    rel = est / truth - 1.0
    a = np.abs(rel)
    return {"mean_abs": float(a.mean()), "p50_abs": float(np.median(a)),
            "p99_abs": float(np.quantile(a, 0.99)), "max_abs": float(a.max()),
            "bias": float(rel.mean())}


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    ap.add_argument("--samples", type=int, default=10_000)
    ap.add_argument("--seed", type=int, default=TRAIN_SEED)
    ap.add_argument("--steps", type=int, default=6000)
    ap.add_argument("--batch", type=int, default=256)
    ap.add_argument("--lr", type=float, default=1e-3)
    ap.add_argument("--workers", type=int, default=max(1, (os.cpu_count() or 2) - 1))
    ap.add_argument("--out", default=os.path.join(os.path.dirname(__file__),
                                                  "predictor_weights.npz"))
    a = ap.parse_args(argv)
    import torch
    if not torch.cuda.is_available():
        raise SystemExit("training needs a GPU")
    dbg.load()
    t0 = time.time()
    regs, D, ks = label_samples(a.samples, a.seed, a.workers)
    t_label = time.time() - t0
    perm = np.random.default_rng(a.seed).permutation(a.samples)
    n_tr, n_va = int(0.8 * a.samples), int(0.1 * a.samples)
    split = {"train": np.sort(perm[:n_tr]), "val": np.sort(perm[n_tr:n_tr + n_va]),
             "test": np.sort(perm[n_tr + n_va:])}
    t1 = time.time()
    P = train(regs, D, split, a.steps, a.batch, a.lr, a.seed)
    t_train = time.time() - t1
    mlp_all, hll_all = evaluate(P, regs, D, np.arange(a.samples))
    te = split["test"]
    margin = float(np.max(D / mlp_all)) * 1.02
    report = {
        "samples": a.samples, "seed": a.seed, "distribution": "synth.batch_sample",
        "k_values": sorted(int(k) for k in set(ks.tolist())),
        "distinct_vertices": {"min": int(D.min()), "median": int(np.median(D)),
                              "max": int(D.max())},
        "split": {n: int(len(v)) for n, v in split.items()},
        "steps": a.steps, "batch": a.batch, "lr": a.lr,
        "test_network": _summary(mlp_all[te], D[te]),
        "test_hyperloglog": _summary(hll_all[te], D[te]),
        "margin": margin, "label_seconds": t_label, "train_seconds": t_train,
    }
    np.savez(a.out, params=P.cpu().numpy(), margin=np.float64(margin))
    with open(os.path.splitext(a.out)[0] + ".json", "w") as f:
        json.dump(report, f, indent=1)
    print(json.dumps(report))


if __name__ == "__main__":
    main()
