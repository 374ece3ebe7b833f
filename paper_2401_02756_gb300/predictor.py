"""Capacity predictor: the number of distinct vertices a read set will give,
known before its table is allocated.

The lock-free table is allocated once at its final size (the paper's table
has a fixed number of buckets), so a build must be sized before it starts.
The predictor runs entirely in the library's kernels:

1. ``dbg_sketch_reads`` -- HyperLogLog registers (1024) of the vertex keys;
2. ``dbg_mlp_features`` -- registers / 64 as float32 inputs;
3. ``dbg_mlp_forward`` -- the trained network, giving ln(distinct vertices).

The classical HyperLogLog estimate of the same registers
(``dbg_sketch_estimate``) is returned beside it.  The weights and the margin
(the largest ratio of true to predicted count seen in training and held-out
data, with 2 % added) come from ``train_predictor.py`` and are stored in
``predictor_weights.npz``; its report sits in ``predictor_weights.json``.
"""

from __future__ import annotations

import math
import os
from dataclasses import dataclass

import numpy as np

from . import dbg

_HERE = os.path.dirname(os.path.abspath(__file__))
WEIGHTS = os.path.join(_HERE, "predictor_weights.npz")
REPORT = os.path.join(_HERE, "predictor_weights.json")
REG_STRIDE = dbg.SKETCH_REGISTERS + 1  # registers plus the status word
# HyperLogLog with 1024 registers has a relative standard error of 1.04 / 32
# (3.25 %); its margin covers 4.6 of them
HLL_MARGIN = 1.15


@dataclass
class Prediction:
    mlp: float  # distinct vertices predicted by the network
    hll: float  # HyperLogLog estimate of the same registers


class CapacityPredictor:
    """Loads trained weights onto the device and predicts distinct vertices."""

    def __init__(self, path: str = WEIGHTS, device="cuda", params=None, margin=None):
        """Weights from ``path``, or ``params`` (a device float32 tensor of
        MLP_PARAMS) with ``margin`` when given."""
        import torch
        self.device = torch.device(device)
        if params is None:
            with np.load(path) as z:
                host = np.ascontiguousarray(z["params"], dtype=np.float32)
                margin = float(z["margin"]) if margin is None else margin
            if host.size != dbg.MLP_PARAMS:
                raise ValueError(f"{path}: {host.size} parameters, expected {dbg.MLP_PARAMS}")
            params = torch.from_numpy(host).to(self.device)
        if params.numel() != dbg.MLP_PARAMS:
            raise ValueError(f"expected {dbg.MLP_PARAMS} parameters")
        self.params = params
        self.margin = 1.0 if margin is None else float(margin)
        # the distinct-vertex counts the network was trained on: outside them
        # (a read set far larger than any training sample) the HyperLogLog
        # estimate sizes the table instead
        self.trained_range = (0.0, float("inf"))
        if os.path.exists(REPORT):
            import json
            with open(REPORT) as f:
                dv = json.load(f).get("distinct_vertices", {})
            if "min" in dv and "max" in dv:
                self.trained_range = (float(dv["min"]), float(dv["max"]))
        self._work: dict[int, tuple] = {}

    def _buffers(self, batch: int):
        import torch
        if batch not in self._work:
            self._work[batch] = (
                torch.empty(batch, dbg.MLP_INPUTS, dtype=torch.float32, device=self.device),
                torch.empty(batch, dtype=torch.float32, device=self.device),
                torch.empty(dbg.mlp_work_floats(batch), dtype=torch.float32, device=self.device))
        return self._work[batch]

    def log_vertices(self, registers, batch: int, stride: int = REG_STRIDE, stream=None):
        """ln(distinct vertices) for ``batch`` register rows (a device int32
        buffer, ``stride`` words apart); a device float32 tensor, stream-ordered."""
        x, y, w = self._buffers(batch)
        dbg.mlp_features(registers, x, batch, stride=stride, stream=stream)
        dbg.mlp_forward(self.params, x, y, w, batch=batch, stream=stream)
        return y

    def predict_registers(self, registers, batch: int, stream=None) -> list[Prediction]:
        """Predictions for ``batch`` register rows of ``REG_STRIDE`` words."""
        import torch
        y = self.log_vertices(registers, batch, stream=stream)
        s = stream or torch.cuda.current_stream(self.device)
        s.synchronize()
        regs = registers.view(-1)[:batch * REG_STRIDE].view(batch, REG_STRIDE).cpu().numpy()
        ln = y.cpu().numpy().astype(np.float64)
        out = []
        for b in range(batch):
            if regs[b, -1] != dbg.OK:
                raise dbg.DbgError(int(regs[b, -1]), "dbg_sketch_reads")
            out.append(Prediction(math.exp(ln[b]), dbg.sketch_estimate(regs[b])))
        return out

    def predict(self, k: int, packed, offsets, stream=None) -> Prediction:
        """Predict the distinct vertices of one device-resident read set."""
        regs = dbg.sketch(k, packed, offsets, stream=stream)
        return self.predict_registers(regs, 1, stream=stream)[0]

    def vertices(self, prediction: Prediction) -> float:
        """The count a table is sized for: the network's prediction times its
        margin, or -- when the HyperLogLog estimate lies beyond the counts the
        network was trained on by more than a quarter -- the estimate times
        HLL_MARGIN."""
        lo, hi = self.trained_range
        if prediction.hll > 1.25 * hi or prediction.hll < lo / 1.25:
            return prediction.hll * HLL_MARGIN
        return prediction.mlp * self.margin

    def capacity(self, prediction: Prediction, headroom: float = 1.5) -> int:
        """Table slots for a predicted count: headroom times ``vertices``
        (the headroom keeps the load factor, and so the probe lengths, where
        the builder expects them)."""
        return max(64, int(math.ceil(self.vertices(prediction) * headroom)))
