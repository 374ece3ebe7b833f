"""Write ``workload_digests.json``: the oracle's graph of each full-size
benchmark workload, recorded as exact per-shard digests.

Only :mod:`oracle` and the seeded generator are called here; nothing comes
from the CUDA path.  For each workload the oracle builds the graph in
``shard_mod`` passes (vertices whose FNV-1a shard is ``p``), and for each pass
records the number of vertices, the sum of the counters and the SHA-256 of
the shard's sorted export (uint64 keys, then uint32 [n, 4] counters, both
little-endian).  A GPU export, split with :func:`oracle.shard_of_keys`,
must reproduce every digest bit for bit.

The batched workload (``batch256``: 256 samples of ``synth.batch_samples``)
is recorded one digest per sample, unsharded.

Usage: ``python tests/golden/make_golden.py [workload ...]`` (default: the
three plain-build workloads and ``batch256``; the 100 Mbp one and the batch
take tens of minutes each).
"""

import hashlib
import json
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_2401_02756_gb300 import synth  # noqa: E402

OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "workload_digests.json")
SHARDS = {"10kb_k21": 1, "5mbp_50x_k31": 2, "100mbp_30x_k31": 8}


def digest(keys: np.ndarray, counts: np.ndarray) -> str:
    h = hashlib.sha256()
    h.update(np.ascontiguousarray(keys, dtype="<u8").tobytes())
    h.update(np.ascontiguousarray(counts, dtype="<u4").tobytes())
    return h.hexdigest()


def _sample_digest(job):
    i, seed = job
    rs = synth.batch_sample(i, seed)
    g = oracle.build_graph(rs.packed, rs.offsets, rs.k, threads=1)
    assert int(g.counts.astype(np.uint64).sum()) == rs.n_edges()
    return i, {"k": rs.k, "n_reads": rs.n_reads, "n_edges": rs.n_edges(),
               "n_vertices": g.n_vertices, "sha256": digest(g.keys, g.counts)}


def batch(data, threads, n=256, seed=4):
    """One oracle build per sample, the samples spread over worker processes."""
    import multiprocessing as mp
    t0 = time.time()
    samples = [None] * n
    with mp.get_context("spawn").Pool(threads) as pool:
        for done, (i, rec) in enumerate(pool.imap_unordered(_sample_digest,
                                                            [(i, seed) for i in range(n)])):
            samples[i] = rec
            if (done + 1) % 32 == 0:
                print(f"batch256: {done + 1}/{n} samples ({time.time() - t0:.0f} s)", flush=True)
    data["batch256"] = {
        "seed": seed, "samples": samples,
        "digest": "sha256 of little-endian uint64 keys then uint32 [n,4] counters, per sample",
    }
    json.dump(data, open(OUT, "w"), indent=1, sort_keys=True)


def main(names):
    data = json.load(open(OUT)) if os.path.exists(OUT) else {}
    threads = os.cpu_count() or 1
    for name in names:
        if name == "batch256":
            batch(data, threads)
            continue
        t0 = time.time()
        rs = synth.WORKLOADS[name]()
        P = SHARDS[name]
        shards = []
        for p in range(P):
            g = oracle.build_graph(rs.packed, rs.offsets, rs.k, shard_mod=P, shard_id=p,
                                   threads=threads)
            shards.append({"n_vertices": g.n_vertices,
                           "n_edges": int(g.counts.astype(np.uint64).sum()),
                           "sha256": digest(g.keys, g.counts)})
            print(f"{name} shard {p}/{P}: {g.n_vertices} vertices ({time.time() - t0:.0f} s)",
                  flush=True)
            del g
        data[name] = {
            "k": rs.k, "n_reads": rs.n_reads, "n_edges": rs.n_edges(),
            "n_vertices": sum(s["n_vertices"] for s in shards),
            "shard_mod": P, "shards": shards,
            "digest": "sha256 of little-endian uint64 keys then uint32 [n,4] counters, per oracle shard",
        }
        assert sum(s["n_edges"] for s in shards) == rs.n_edges()
        json.dump(data, open(OUT, "w"), indent=1, sort_keys=True)
        print(f"{name}: done in {time.time() - t0:.0f} s", flush=True)


if __name__ == "__main__":
    main(sys.argv[1:] or list(SHARDS) + ["batch256"])
