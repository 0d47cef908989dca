"""Parity of the learned preconditioner's CUDA kernels (BF16 tensor-core
convolutions, FP32 accumulation) with the FP64 CNN oracle (oracle/cnn.py).

Bars: forward output within 1e-2 relative L2 of the oracle run on
BF16-rounded weights and layer inputs; loss within 1e-2; every layer's weight
and bias gradient within 2.5e-2 relative L2 of FP64 backpropagation through
that BF16-rounded network and within 3e-2 of FP64 backpropagation through the
unrounded one; the network inputs of a grid within 1e-5 (FP32); one AdamW
step equal to the textbook update of the GPU's own gradient to FP32 rounding.

The gradient bars come from the arithmetic.  The gradient map that feeds each
tensor-core product is stored in BF16 (unit roundoff 2^-9).  Each level of the
backward pass therefore adds about 0.35 % relative error, and weight
gradients sum over all points with cancellation.  The first layer sits five
levels deep.
"""
import numpy as np
import pytest

import oracle as O
from oracle import cnn
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2103_16120_gb300 as sw  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _build():
    from paper_2103_16120_gb300 import build
    build.build()
    assert torch.cuda.is_available()


def rel(a, b):
    a, b = np.asarray(a, np.float64), np.asarray(b, np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def params(seed):
    P = cnn.init_params(seed)
    rng = np.random.default_rng(seed + 1)
    for k in P:
        if k.endswith(".b"):
            P[k] = 0.05 * rng.standard_normal(P[k].shape)
    return P


def model_with(P):
    m = sw.Model()
    sw.sw_model_set_params(m, cnn.flatten_params(P).astype(np.float32))
    return m


def inputs(seed, B, H, W):
    rng = np.random.default_rng(seed)
    x0 = rng.standard_normal((B, 4, H, W))
    x0[:, 3] = np.sin(np.linspace(-1.5, 1.5, H))[None, :, None]
    return x0


def dev(a):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float32, device="cuda")


@pytest.mark.parametrize("B,H,W", [(1, 8, 64), (2, 16, 128), (1, 32, 256)])
def test_forward_matches_oracle(B, H, W):
    P = params(10 + W)
    m = model_with(P)
    # the oracle sees exactly the BF16 weights and inputs the GPU holds
    x0 = cnn.round_bf16(inputs(20 + W, B, H, W))
    y = torch.empty((B, H, W), dtype=torch.float32, device="cuda")
    sw.sw_model_forward(m, dev(x0), y)
    torch.cuda.synchronize()
    yg = y.cpu().numpy()
    for b in range(B):
        yo, _ = cnn.forward(P, x0[b], bf16=True)
        assert rel(yg[b], yo) <= 1e-2


def test_param_roundtrip_and_count():
    P = params(3)
    m = model_with(P)
    back = sw.sw_model_get_params(m)
    assert back.size == sw.SW_MODEL_PARAMS == cnn.n_params()
    assert np.array_equal(back, cnn.flatten_params(P).astype(np.float32))


@pytest.mark.parametrize("B,H,W", [(2, 8, 64), (1, 16, 128), (2, 32, 256)])
def test_loss_and_gradients_match_oracle(B, H, W):
    P = params(30 + H)
    m = model_with(P)
    x0 = inputs(40 + H, B, H, W)
    target = np.random.default_rng(50 + H).standard_normal((B, H, W))
    loss, g = sw.sw_model_loss_grad(m, dev(x0), dev(target))
    lo, Go = cnn.loss_and_grad(P, [(x0[b], target[b]) for b in range(B)])
    assert abs(loss - lo) <= 1e-2 * lo
    # FP64 backpropagation through the network as the GPU stores it: weights
    # and layer inputs rounded to BF16
    Pr = {k: (cnn.round_bf16(v) if k.endswith(".w") else v) for k, v in P.items()}
    Gr, npts = None, 0
    for b in range(B):
        y, cache = cnn.forward(P, x0[b], bf16=True)
        gb = cnn.backward(Pr, cache, 2.0 * (y - target[b]))
        Gr = gb if Gr is None else {k: Gr[k] + gb[k] for k in Gr}
        npts += y.size
    Gr = {k: v / npts for k, v in Gr.items()}
    Gg = cnn.unflatten_params(g.astype(np.float64))
    for name, _, _, _ in cnn.LAYERS:
        for part in (".w", ".b"):
            assert rel(Gg[name + part], Gr[name + part]) <= 2.5e-2, name + part
            assert rel(Gg[name + part], Go[name + part]) <= 3e-2, name + part


def test_features_match_oracle():
    nx, ny = 128, 64
    Pp = synth.problem(nx, ny, 60)
    g = sw.sw_grid_create(nx, ny)
    sw.sw_elliptic_set_coeffs(g, *[torch.as_tensor(Pp[k], device="cuda") for k in sw.COEFF_KEYS])
    m = model_with(params(4))
    r = np.random.default_rng(61).standard_normal((ny, nx)) * 3e4
    x0 = torch.empty((4, ny, nx), dtype=torch.float32, device="cuda")
    sw.sw_model_features(m, g, dev(r), x0)
    static, d = cnn.static_features(Pp, O.Problem(Pp).diag_L())
    xo, s = cnn.features(r.astype(np.float32).astype(np.float64), static)
    xg = x0.cpu().numpy()
    for c in range(4):
        assert rel(xg[c], xo[c]) <= 1e-5, c
    # the preconditioner output e = s y / d
    e = torch.empty((ny, nx), dtype=torch.float32, device="cuda")
    P = params(4)
    sw.sw_model_apply(m, g, dev(r), e)
    eo = cnn.apply(P, r, static, d, bf16=True)
    assert rel(e.cpu().numpy(), eo) <= 1e-2


def test_adamw_step_is_the_textbook_update():
    B, H, W = 2, 8, 64
    P = params(70)
    m = model_with(P)
    x0, t = dev(inputs(71, B, H, W)), dev(np.random.default_rng(72).standard_normal((B, H, W)))
    _, g = sw.sw_model_loss_grad(m, x0, t)
    lr, wd = 1e-3, 0.01
    sw.sw_model_train_step(m, x0, t, lr=lr, weight_decay=wd)
    got = sw.sw_model_get_params(m).astype(np.float64)
    exp = cnn.flatten_params(cnn.adamw_step(P, cnn.unflatten_params(g.astype(np.float64)), {}, lr, wd=wd))
    p0 = cnn.flatten_params(P)
    # the step itself (about lr per entry) agrees to FP32 rounding
    assert np.max(np.abs((got - p0) - (exp - p0))) <= 1e-6


def test_training_reduces_the_loss():
    B, H, W = 8, 16, 64
    P = params(80)
    m = model_with(P)
    x0 = dev(inputs(81, B, H, W))
    # a smooth target the network can fit
    t = dev(np.stack([np.cos(np.linspace(0, 2 * np.pi, W))[None, :] * np.ones((H, 1))] * B))
    l0 = sw.sw_model_train_step(m, x0, t, lr=3e-3)
    for _ in range(60):
        last = sw.sw_model_train_step(m, x0, t, lr=3e-3)
    assert last < 0.3 * l0


def test_rejects_bad_shapes():
    m = model_with(params(90))
    x0 = dev(inputs(91, 1, 8, 96))
    y = torch.empty((1, 8, 96), dtype=torch.float32, device="cuda")
    with pytest.raises(sw.SwError) as ei:
        sw.sw_model_forward(m, x0, y)
    assert ei.value.status == sw.SW_ERR_INVALID_ARG
