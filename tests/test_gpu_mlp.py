"""The capacity predictor's network (FP32 CUDA kernels) against the FP64
reference in ``oracle.mlp``.

Tolerances follow from the arithmetic: every output is a sum of at most
n = 1024 + 2 * 64 products evaluated in float32, so it is within about
n * 2^-24 times the same expression evaluated on absolute values
(``oracle.mlp.abs_forward`` and the absolute-value backward pass below).  The
bound is taken with a factor 8 of slack; a transposed operand, a wrong index
or a dropped term is off by O(1) of that magnitude and fails.  The test inputs
are drawn so that no ReLU input lies within its (slack-free) rounding bound of
zero, so both sides take the same ReLU branches.
"""

import numpy as np
import pytest

from oracle import mlp
from paper_2401_02756_gb300 import build, dbg

pytestmark = pytest.mark.gpu

U = 2.0 ** -24
GAMMA = 8 * (mlp.IN + 2 * mlp.HID + 8) * U


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    build.build()
    dbg.load()


def ambiguous_rows(p, x):
    """Rows with a ReLU input within its float32 rounding bound of zero: n
    terms of magnitude sum a give |error| <= n * 2^-24 * a (Higham, Accuracy
    and Stability of Numerical Algorithms, Sec. 3.1), and the second layer
    inherits the first layer's error through |W2|."""
    _, c = mlp.forward(p, x)
    q = {n: np.abs(a) for n, a in mlp.unpack(p).items()}
    a1 = np.abs(x) @ q["W1"].T + q["b1"]
    a2 = a1 @ q["W2"].T + q["b2"]
    bad1 = np.abs(c["z1"]) <= 2 * (mlp.IN + 2) * U * a1
    bad2 = np.abs(c["z2"]) <= 2 * (mlp.IN + mlp.HID + 4) * U * a2
    return bad1.any(axis=1) | bad2.any(axis=1)


def case(seed: int, batch: int):
    """Seeded parameters (He-uniform scale, small biases), sketch-like inputs
    (register values 0..24 over 64, some inputs never set) and targets around
    ln(1e5); input rows whose ReLU branches rounding could flip are redrawn."""
    rng = np.random.default_rng(seed)
    blocks = {"W1": rng.uniform(-1, 1, (mlp.HID, mlp.IN)) * np.sqrt(6 / mlp.IN),
              "b1": rng.normal(0, 0.1, mlp.HID),
              "W2": rng.uniform(-1, 1, (mlp.HID, mlp.HID)) * np.sqrt(6 / mlp.HID),
              "b2": rng.normal(0, 0.1, mlp.HID),
              "w3": rng.uniform(-1, 1, mlp.HID) * np.sqrt(6 / mlp.HID), "b3": 0.3}
    p = mlp.pack(blocks).astype(np.float32).astype(np.float64)
    dead = rng.integers(0, mlp.IN, 20)
    rows = []
    while len(rows) < batch:
        x = rng.integers(0, 25, (batch, mlp.IN)) / 64.0
        x[:, dead] = 0.0
        rows.extend(x[~ambiguous_rows(p, x)])
    x = np.array(rows[:batch])
    t = rng.normal(11.5, 2.0, batch).astype(np.float32).astype(np.float64)
    return p, x, t


def magnitudes(p, x, t):
    """Absolute-value forward and backward passes: per-output sums of the
    magnitudes of the terms each float32 result is made of."""
    q = {n: np.abs(a) for n, a in mlp.unpack(p).items()}
    a1 = np.abs(x) @ q["W1"].T + q["b1"]
    a2 = a1 @ q["W2"].T + q["b2"]
    ay = a2 @ q["w3"] + q["b3"]
    y, _ = mlp.forward(p, x)
    B = x.shape[0]
    ady = (np.abs(y - t) + GAMMA * ay + np.abs(t)) / B
    g = {"w3": a2.T @ ady, "b3": ady.sum()}
    az2 = np.outer(ady, q["w3"])
    g["W2"], g["b2"] = az2.T @ a1, az2.sum(axis=0)
    az1 = az2 @ q["W2"]
    g["W1"], g["b1"] = az1.T @ np.abs(x), az1.sum(axis=0)
    return a1, a2, ay, mlp.pack(g)


def assert_well_conditioned(p, x):
    assert not ambiguous_rows(p, x).any(), "a ReLU input is within rounding of 0"


def dev(a, dtype="float32"):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a, dtype=dtype)).cuda()


def work(batch):
    import torch
    return torch.zeros(dbg.mlp_work_floats(batch), dtype=torch.float32, device="cuda")


@pytest.mark.parametrize("batch", [1, 31, 33, 257])
def test_forward_matches_reference(batch):
    import torch
    p, x, t = case(100 + batch, batch)
    assert_well_conditioned(p, x)
    y = torch.empty(batch, dtype=torch.float32, device="cuda")
    dbg.mlp_forward(dev(p), dev(x), y, work(batch))
    ref, _ = mlp.forward(p, x)
    bound = GAMMA * mlp.abs_forward(p, x)
    err = np.abs(y.cpu().numpy().astype(np.float64) - ref)
    assert np.all(err <= bound), (err.max(), bound.min())


@pytest.mark.parametrize("batch", [7, 64, 200])
def test_train_step_gradients_loss_and_adam_match_reference(batch):
    import torch
    p, x, t = case(200 + batch, batch)
    assert_well_conditioned(p, x)
    P, G = dev(p), torch.zeros(mlp.N_PARAMS, dtype=torch.float32, device="cuda")
    M = torch.zeros_like(G)
    V = torch.zeros_like(G)
    loss = torch.zeros(1, dtype=torch.float32, device="cuda")
    lr = 1e-3
    dbg.mlp_train_step(P, G, M, V, 1, lr, dev(x), dev(t), work(batch), loss=loss)
    torch.cuda.synchronize()
    ref_loss, ref_g = mlp.loss_and_grads(p, x, t)
    _, _, ay, mag = magnitudes(p, x, t)
    y, _ = mlp.forward(p, x)
    loss_bound = np.mean(np.abs(y - t) * GAMMA * ay) + GAMMA * ref_loss + 1e-30
    assert abs(float(loss.item()) - ref_loss) <= 2 * loss_bound + ref_loss * 1e-6

    g = G.cpu().numpy().astype(np.float64)
    tol = GAMMA * mag
    assert np.all(np.abs(g - ref_g) <= tol), np.max(np.abs(g - ref_g) - tol)
    assert np.array_equal(g == 0.0, ref_g == 0.0)  # the same ReLU branches and dead inputs

    # Adam, step 1: each parameter moves by lr * g / (|g| + eps)
    step = P.cpu().numpy().astype(np.float64) - p
    clear = (np.abs(ref_g) > 2 * tol) & (np.abs(ref_g) > 1e-4)
    assert clear.mean() > 0.5
    expect = -lr * ref_g[clear] / (np.abs(ref_g[clear]) + 1e-8)
    assert np.allclose(step[clear], expect, rtol=2e-4, atol=0)
    assert np.all(step[ref_g == 0.0] == 0.0)
    assert np.all(np.abs(step) <= lr * (1 + 1e-5))
    # the moments use the float32 values of 1 - beta1 and 1 - beta2
    one_m_b1 = float(np.float32(1) - np.float32(0.9))
    one_m_b2 = float(np.float32(1) - np.float32(0.999))
    assert np.allclose(M.cpu().numpy(), one_m_b1 * g, rtol=1e-6, atol=0)
    assert np.allclose(V.cpu().numpy(), one_m_b2 * g * g, rtol=1e-5, atol=1e-44)


def test_several_adam_steps_track_the_reference():
    import torch
    batch, lr, steps = 48, 2e-3, 5
    p, x, t = case(300, batch)
    P = dev(p)
    G = torch.zeros(mlp.N_PARAMS, dtype=torch.float32, device="cuda")
    M, V = torch.zeros_like(G), torch.zeros_like(G)
    w, X, T = work(batch), dev(x), dev(t)
    rp, rm, rv = p.copy(), np.zeros_like(p), np.zeros_like(p)
    for s in range(1, steps + 1):
        dbg.mlp_train_step(P, G, M, V, s, lr, X, T, w)
        _, g = mlp.loss_and_grads(rp, x, t)
        rp, rm, rv = mlp.adam_step(rp, g, rm, rv, s, lr)
    moved = rp - p
    got = P.cpu().numpy().astype(np.float64) - p
    # parameters whose reference gradient never came near 0 follow the same path
    big = np.abs(moved) > 0.5 * steps * lr
    assert big.mean() > 0.3
    assert np.allclose(got[big], moved[big], rtol=2e-2, atol=0)
    # Adam's per-step move is at most lr * (1 - beta1) / sqrt(1 - beta2) when
    # 1 - beta1 > sqrt(1 - beta2) (Kingma & Ba, Sec. 2.1)
    bound = steps * lr * 0.1 / np.sqrt(0.001) * (1 + 1e-4)
    assert np.all(np.abs(moved) <= bound) and np.all(np.abs(got) <= bound)


def test_training_fits_a_learnable_target():
    import torch
    batch, steps = 64, 400
    rng = np.random.default_rng(7)
    x = rng.integers(0, 25, (batch, mlp.IN)) / 64.0
    t = 10.0 + 20.0 * x[:, :64].mean(axis=1)
    P = torch.empty(mlp.N_PARAMS, dtype=torch.float32, device="cuda")
    dbg.mlp_init(P, 11)
    G = torch.zeros_like(P)
    M, V = torch.zeros_like(P), torch.zeros_like(P)
    w, X, T = work(batch), dev(x), dev(t)
    loss = torch.zeros(1, dtype=torch.float32, device="cuda")
    first = None
    for s in range(1, steps + 1):
        dbg.mlp_train_step(P, G, M, V, s, 1e-2, X, T, w, loss=loss)
        if first is None:
            first = float(loss.item())
    last = float(loss.item())
    assert last < 1e-2 * first, (first, last)


def test_init_is_seeded_he_uniform_with_zero_biases():
    import torch
    a = torch.empty(mlp.N_PARAMS, dtype=torch.float32, device="cuda")
    b = torch.empty_like(a)
    c = torch.empty_like(a)
    dbg.mlp_init(a, 5)
    dbg.mlp_init(b, 5)
    dbg.mlp_init(c, 6)
    a, b, c = (v.cpu().numpy().astype(np.float64) for v in (a, b, c))
    assert np.array_equal(a, b) and not np.array_equal(a, c)
    q = mlp.unpack(a)
    for name in ("b1", "b2", "b3"):
        assert not np.any(q[name])
    for name, fan_in in (("W1", mlp.IN), ("W2", mlp.HID), ("w3", mlp.HID)):
        lim = np.sqrt(6.0 / fan_in)
        assert np.all(np.abs(q[name]) <= lim)
        assert np.std(q[name]) == pytest.approx(lim / np.sqrt(3.0), rel=0.1 if name != "w3" else 0.35)
        assert abs(np.mean(q[name])) < 0.1 * lim


@pytest.mark.parametrize("stride", [dbg.SKETCH_REGISTERS + 1, 2048])
def test_features_are_registers_over_64(stride):
    import torch
    batch = 9
    rng = np.random.default_rng(stride)
    regs = rng.integers(0, 56, (batch, stride)).astype(np.int32)
    x = torch.empty(batch, mlp.IN, dtype=torch.float32, device="cuda")
    dbg.mlp_features(dev(regs, "int32"), x, batch, stride=stride)
    assert np.array_equal(x.cpu().numpy(), (regs[:, :mlp.IN] / 64.0).astype(np.float32))
