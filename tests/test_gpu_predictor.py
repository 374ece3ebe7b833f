"""The capacity predictor: the committed weights predict the distinct-vertex
count of unseen samples of the batched-build distribution (truth from the
oracle), the sized table holds them, and the training script runs end to end."""

import json
import os

import numpy as np
import pytest

import oracle
from gpu_util import to_device
from paper_2401_02756_gb300 import build, dbg, synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    build.build()
    dbg.load()


def small_samples(n, seed=23):
    # the training distribution restricted to genomes of 5e4 .. 2e5 bases, so
    # the oracle labels each in about a second; seed 23 is used by neither
    # the training set nor the benchmark
    return [synth.batch_sample(i, seed, gmax=2e5) for i in range(n)]


def test_committed_weights_predict_unseen_samples():
    from paper_2401_02756_gb300.predictor import CapacityPredictor, WEIGHTS
    with open(os.path.splitext(WEIGHTS)[0] + ".json") as f:
        report = json.load(f)
    assert report["samples"] >= 10_000
    pred = CapacityPredictor()
    assert 1.0 <= pred.margin < 2.0
    for rs in small_samples(6):
        D = oracle.build_graph(rs.packed, rs.offsets, rs.k).n_vertices
        packed, offsets = to_device(rs)
        p = pred.predict(rs.k, packed, offsets)
        assert abs(p.hll / D - 1) < 0.13, (p.hll, D)  # four HyperLogLog standard errors
        assert abs(p.mlp / D - 1) < max(0.15, 4 * report["test_network"]["p99_abs"]), (p.mlp, D)
        # the table the predictor sizes holds the graph
        g = dbg.Graph(rs.k, pred.capacity(p))
        g.insert(packed, offsets)
        assert g.status() == dbg.OK
        assert g.stats() == (D, rs.n_edges())
        g.close()


def test_batched_predictions_equal_one_by_one():
    import torch
    from paper_2401_02756_gb300.predictor import REG_STRIDE, CapacityPredictor
    pred = CapacityPredictor()
    samples = small_samples(5, seed=29)
    regs = torch.zeros(len(samples), REG_STRIDE, dtype=torch.int32, device="cuda")
    single = []
    for i, rs in enumerate(samples):
        packed, offsets = to_device(rs)
        dbg.sketch(rs.k, packed, offsets, registers=regs[i])
        single.append(pred.predict(rs.k, packed, offsets))
    batched = pred.predict_registers(regs, len(samples))
    for a, b in zip(single, batched):
        assert a.hll == b.hll
        assert a.mlp == pytest.approx(b.mlp, rel=1e-6)


def test_training_script_end_to_end(tmp_path):
    from paper_2401_02756_gb300 import train_predictor
    from paper_2401_02756_gb300.predictor import CapacityPredictor
    out = str(tmp_path / "w.npz")
    train_predictor.main(["--samples", "40", "--steps", "200", "--batch", "16",
                          "--workers", "2", "--out", out])
    with open(str(tmp_path / "w.json")) as f:
        report = json.load(f)
    assert report["split"] == {"train": 32, "val": 4, "test": 4}
    assert report["margin"] >= 1.0
    pred = CapacityPredictor(out)
    assert np.isfinite(pred.params.cpu().numpy()).all()
