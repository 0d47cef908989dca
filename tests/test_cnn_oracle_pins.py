"""Pins of the CNN oracle (oracle/cnn.py) against definitions that do not go
through its own code: brute-force loops over the padding rule, adjoint
identities, central finite differences, symmetry of the network under
longitude shifts, the closed form of a first AdamW step, and the face
coefficients read back from the operator of the C oracle."""
import math

import numpy as np
import pytest

import oracle as O
from oracle import cnn
import synth


def nb(h, i, H, W):
    """Source point of the padded neighbour (h, i), h in -1..H, i in -1..W."""
    i %= W
    if h < 0:
        return 0, (i + W // 2) % W
    if h >= H:
        return H - 1, (i + W // 2) % W
    return h, i


def test_network_size_and_flops():
    assert cnn.n_params() == 158369
    # FLOPs per grid point: 2*9*(4*32 + 96*32 + 32) at full resolution,
    # 2*9*(32*64 + 128*64)/4 at half and 2*9*64*64/16 at quarter resolution
    assert cnn.forward_flops(128, 256) == 108864 * 256 * 128     # about 3.6 GFLOP


def test_padding_matches_the_neighbour_rule():
    rng = np.random.default_rng(1)
    C_, H, W = 2, 4, 6
    x = rng.standard_normal((C_, H, W))
    p = cnn.pad_sphere(x)
    for h in range(-1, H + 1):
        for i in range(-1, W + 1):
            sh, si = nb(h, i, H, W)
            assert np.array_equal(p[:, h + 1, i + 1], x[:, sh, si])


def test_conv_matches_brute_force_loops():
    rng = np.random.default_rng(2)
    Ci, Co, H, W = 3, 2, 4, 6
    x = rng.standard_normal((Ci, H, W))
    w = rng.standard_normal((Co, Ci, 3, 3))
    b = rng.standard_normal(Co)
    y = cnn.conv3x3(x, w, b)
    for o in range(Co):
        for h in range(H):
            for i in range(W):
                s = b[o]
                for c in range(Ci):
                    for ky in range(3):
                        for kx in range(3):
                            sh, si = nb(h + ky - 1, i + kx - 1, H, W)
                            s += w[o, c, ky, kx] * x[c, sh, si]
                assert abs(y[o, h, i] - s) <= 1e-12 * (1 + abs(s))


@pytest.mark.parametrize("op,adj,shape,oshape", [
    (cnn.pad_sphere, cnn.pad_sphere_adjoint, (3, 4, 8), (3, 6, 10)),
    (cnn.pool2, cnn.pool2_adjoint, (3, 4, 8), (3, 2, 4)),
    (cnn.up2, cnn.up2_adjoint, (3, 2, 4), (3, 4, 8)),
])
def test_adjoint_identities(op, adj, shape, oshape):
    rng = np.random.default_rng(3)
    x = rng.standard_normal(shape)
    g = rng.standard_normal(oshape)
    lhs = float(np.sum(op(x) * g))
    rhs = float(np.sum(x * adj(g)))
    assert abs(lhs - rhs) <= 1e-12 * (abs(lhs) + 1)


def test_conv_backward_is_the_adjoint():
    rng = np.random.default_rng(4)
    x = rng.standard_normal((3, 4, 8))
    w = rng.standard_normal((2, 3, 3, 3))
    b = np.zeros(2)
    gy = rng.standard_normal((2, 4, 8))
    gx, gw, gb = cnn.conv3x3_backward(x, w, gy)
    # y is linear in x and in w: <y, gy> = <x, gx> = <w, gw>
    ygy = float(np.sum(cnn.conv3x3(x, w, b) * gy))
    assert abs(ygy - float(np.sum(x * gx))) <= 1e-11 * abs(ygy)
    assert abs(ygy - float(np.sum(w * gw))) <= 1e-11 * abs(ygy)
    assert np.allclose(gb, gy.sum(axis=(1, 2)))


def _tiny_batch(seed, H=8, W=16, n=2):
    rng = np.random.default_rng(seed)
    return [(rng.standard_normal((4, H, W)), rng.standard_normal((H, W))) for _ in range(n)]


def test_backprop_matches_central_differences():
    P = cnn.init_params(5)
    # non-zero biases so that every ReLU sees both signs
    rng = np.random.default_rng(6)
    for k in P:
        if k.endswith(".b"):
            P[k] = 0.1 * rng.standard_normal(P[k].shape)
    batch = _tiny_batch(7)
    _, G = cnn.loss_and_grad(P, batch)
    h = 1e-6
    for name, _, _, _ in cnn.LAYERS:
        for key, idx in ((name + ".w", (0, 0, 1, 2)), (name + ".w", (-1, -1, 2, 0)), (name + ".b", (0,))):
            Pp = {k: v.copy() for k, v in P.items()}
            Pm = {k: v.copy() for k, v in P.items()}
            Pp[key][idx] += h
            Pm[key][idx] -= h
            fd = (cnn.loss_and_grad(Pp, batch)[0] - cnn.loss_and_grad(Pm, batch)[0]) / (2 * h)
            g = G[key][idx]
            assert abs(fd - g) <= 1e-6 * max(abs(g), 1e-3), (key, idx, fd, g)


def test_network_commutes_with_longitude_shifts():
    P = cnn.init_params(8)
    x0 = np.random.default_rng(9).standard_normal((4, 8, 16))
    y, _ = cnn.forward(P, x0)
    ys, _ = cnn.forward(P, np.roll(x0, 4, axis=2))     # 4 = one point at level 2
    assert np.allclose(ys, np.roll(y, 4, axis=1), rtol=0, atol=1e-12)


def test_round_bf16():
    assert cnn.round_bf16(1.0) == 1.0
    assert cnn.round_bf16(1.0 + 2 ** -8) == 1.0                  # tie to even
    assert cnn.round_bf16(1.0 + 3 * 2 ** -8) == 1.0 + 2 ** -6    # tie to even (up)
    assert cnn.round_bf16(1.0 + 2 ** -7) == 1.0 + 2 ** -7
    x = np.random.default_rng(10).standard_normal(1000)
    assert np.max(np.abs(cnn.round_bf16(x) - x) / np.abs(x)) <= 2 ** -8


def test_first_adamw_step_closed_form():
    P = {"c.w": np.array([1.0, -2.0, 3.0]), "c.b": np.array([0.5])}
    G = {"c.w": np.array([0.3, -4.0, 0.0]), "c.b": np.array([1e-3])}
    lr, wd = 1e-2, 0.1
    out = cnn.adamw_step({k: v.copy() for k, v in P.items()}, G, {}, lr, wd=wd)
    # m_hat = g and v_hat = g^2 after one step: w -= lr (g/(|g| + eps) + wd w)
    exp_w = P["c.w"] - lr * (G["c.w"] / (np.abs(G["c.w"]) + 1e-8) + wd * P["c.w"])
    exp_b = P["c.b"] - lr * (G["c.b"] / (np.abs(G["c.b"]) + 1e-8))
    assert np.allclose(out["c.w"], exp_w, rtol=1e-14, atol=1e-15)
    assert np.allclose(out["c.b"], exp_b, rtol=1e-14, atol=1e-15)


def test_face_features_match_the_operator():
    """The couplings in the features are entries of L read off the C oracle:
    L(delta at (j, i)) at (j, i+1) is ax(i+1/2) when only A11 is non-zero."""
    nx, ny = 16, 8
    P = synth.problem(nx, ny, 11)
    only = {k: np.zeros_like(P[k]) for k in ("A11", "A12", "A21", "A22", "B1", "B2", "C")}
    only["A11"] = P["A11"]
    only_y = dict(only, A11=np.zeros_like(P["A11"]), A22=P["A22"])
    ax, ay = cnn.faces(P)
    for j, i in ((0, 0), (3, 7), (7, 15)):
        d = np.zeros((ny, nx)); d[j, i] = 1.0
        Lx = O.Problem(only).operator(d)
        assert math.isclose(Lx[j, (i + 1) % nx], ax[j, i], rel_tol=1e-13)
        assert math.isclose(Lx[j, (i - 1) % nx], ax[j, (i - 1) % nx], rel_tol=1e-13)
        Ly = O.Problem(only_y).operator(d)
        if j + 1 < ny:
            assert math.isclose(Ly[j + 1, i], ay[j, i], rel_tol=1e-13)
        else:
            assert ay[j, i] == 0.0
    static, dd = cnn.static_features(P, O.Problem(P).diag_L())
    assert np.all(dd > 0) and np.all(static[0] > 0) and np.all(static[1] >= 0)
    assert np.all(static[0] + static[1] <= 1.0 + 1e-12)   # couplings are part of the diagonal


def test_training_reduces_the_loss():
    P = cnn.init_params(12)
    batch = _tiny_batch(13, n=1)
    state = {}
    l0 = cnn.loss_and_grad(P, batch)[0]
    for _ in range(30):
        _, G = cnn.loss_and_grad(P, batch)
        P = cnn.adamw_step(P, G, state, 3e-3)
    assert cnn.loss_and_grad(P, batch)[0] < 0.5 * l0
