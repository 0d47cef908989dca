"""FP64 CPU oracle of the learned preconditioner (the CNN used inside flexible
GCR).  The paper has no learned part; this follows the network fixed for the
project: a three-level U-Net with 3x3 convolutions, 32/64/64 channels,
longitude-periodic and across-pole padding, and the training objective below.

TEST INFRASTRUCTURE ONLY: imported by tests/ and never by the library.  It
shares no code with the CUDA path.  Everything is plain numpy in float64,
channels-first [C, H, W] (one sample) with H = ny latitude rows and W = nx
longitudes, written for a reader to check by eye; nothing is fused.

Network (levels l = 0, 1, 2 have H/2^l x W/2^l points):
    a1 = relu(conv(x0;  4 -> 32))                      level 0
    a2 = relu(conv(pool(a1); 32 -> 64))                level 1
    a3 = relu(conv(pool(a2); 64 -> 64))                level 2
    a4 = relu(conv(cat(up(a3), a2); 128 -> 64))        level 1
    a5 = relu(conv(cat(up(a4), a1); 96 -> 32))         level 0
    y  = conv(a5; 32 -> 1)                             level 0
conv: 3x3 with bias; pool: 2x2 mean; up: nearest-neighbour 2x; cat: channels.

Padding (the operator's boundary rules, applied at every level): periodic in
longitude; the row beyond a pole is the pole row shifted by half a circle,
x[-1, i] = x[0, i + W/2] and x[H, i] = x[H-1, i + W/2].

Inputs and output (a dimensionless correction of the Jacobi scaling):
    d  = |diag(L)|                               per point
    s  = sqrt(mean(r^2))                         per sample
    x0 = [r/s, (ax_w + ax_e)/d, (ay_s + ay_n)/d, sin(phi)]
    e  = s * y / d                               the preconditioned residual
with ax, ay the zonal and meridional face coefficients of L (Eq. 10 in
flux form: a11 / dlam^2 and a22 / dphi^2 at the faces, the mean of the two
adjacent cells, zero on the pole faces).

Training: the target for a pair (R, Phi = L^-1 R) is y* = d Phi / s with
s = rms(R); loss = mean over points and samples of (y - y*)^2; AdamW.
"""
from __future__ import annotations

import math

import numpy as np

LAYERS = (  # (name, c_in, c_out, relu)
    ("c1", 4, 32, True),
    ("c2", 32, 64, True),
    ("c3", 64, 64, True),
    ("c4", 128, 64, True),
    ("c5", 96, 32, True),
    ("c6", 32, 1, False),
)


def n_params() -> int:
    return sum(ci * co * 9 + co for _, ci, co, _ in LAYERS)


def forward_flops(ny: int, nx: int) -> float:
    """Multiply-add FLOPs (2 per MAC) of one forward pass of the convolutions."""
    level = {"c1": 0, "c2": 1, "c3": 2, "c4": 1, "c5": 0, "c6": 0}
    return sum(2.0 * ci * co * 9 * (ny * nx) / 4 ** level[n] for n, ci, co, _ in LAYERS)


# ---------------------------------------------------------------------------
# elementary operations and their adjoints
# ---------------------------------------------------------------------------
def pad_sphere(x):
    """[C, H, W] -> [C, H+2, W+2] with the periodic / across-pole halo."""
    C_, H, W = x.shape
    assert W % 2 == 0
    p = np.zeros((C_, H + 2, W + 2))
    p[:, 1:H + 1, 1:W + 1] = x
    p[:, 0, 1:W + 1] = np.roll(x[:, 0, :], -(W // 2), axis=-1)        # x[-1, i] = x[0, i + W/2]
    p[:, H + 1, 1:W + 1] = np.roll(x[:, H - 1, :], -(W // 2), axis=-1)  # x[H, i] = x[H-1, i + W/2]
    p[:, :, 0] = p[:, :, W]        # periodic longitude (corners included)
    p[:, :, W + 1] = p[:, :, 1]
    return p


def pad_sphere_adjoint(g):
    """Adjoint of pad_sphere: [C, H+2, W+2] -> [C, H, W]."""
    C_, Hp, Wp = g.shape
    H, W = Hp - 2, Wp - 2
    g = g.copy()
    g[:, :, W] += g[:, :, 0]
    g[:, :, 1] += g[:, :, W + 1]
    x = g[:, 1:H + 1, 1:W + 1].copy()
    x[:, 0, :] += np.roll(g[:, 0, 1:W + 1], W // 2, axis=-1)
    x[:, H - 1, :] += np.roll(g[:, H + 1, 1:W + 1], W // 2, axis=-1)
    return x


def conv3x3(x, w, b):
    """y[o, h, i] = b[o] + sum_{c, dy, dx} w[o, c, dy, dx] xp[c, h + dy, i + dx]
    (dy, dx in 0..2 over the padded input xp)."""
    C_, H, W = x.shape
    xp = pad_sphere(x)
    y = np.zeros((w.shape[0], H, W))
    for dy in range(3):
        for dx in range(3):
            patch = xp[:, dy:dy + H, dx:dx + W]                 # [C, H, W]
            y += np.einsum("oc,chw->ohw", w[:, :, dy, dx], patch)
    return y + b[:, None, None]


def conv3x3_backward(x, w, gy):
    """Gradients of conv3x3 with respect to x, w and b, given dLoss/dy = gy."""
    C_, H, W = x.shape
    xp = pad_sphere(x)
    gxp = np.zeros_like(xp)
    gw = np.zeros_like(w)
    for dy in range(3):
        for dx in range(3):
            patch = xp[:, dy:dy + H, dx:dx + W]
            gw[:, :, dy, dx] = np.einsum("ohw,chw->oc", gy, patch)
            gxp[:, dy:dy + H, dx:dx + W] += np.einsum("oc,ohw->chw", w[:, :, dy, dx], gy)
    return pad_sphere_adjoint(gxp), gw, gy.sum(axis=(1, 2))


def pool2(x):
    C_, H, W = x.shape
    return x.reshape(C_, H // 2, 2, W // 2, 2).mean(axis=(2, 4))


def pool2_adjoint(g):
    return np.repeat(np.repeat(g, 2, axis=1), 2, axis=2) / 4.0


def up2(x):
    return np.repeat(np.repeat(x, 2, axis=1), 2, axis=2)


def up2_adjoint(g):
    C_, H, W = g.shape
    return g.reshape(C_, H // 2, 2, W // 2, 2).sum(axis=(2, 4))


def relu(x):
    return np.maximum(x, 0.0)


def round_bf16(x):
    """Round to the nearest value with an 8-bit significand (ties to even), the
    precision of bfloat16 (its exponent range is that of float32)."""
    x = np.asarray(x, dtype=np.float64)
    m, e = np.frexp(x)                    # x = m 2^e, 0.5 <= |m| < 1
    return np.ldexp(np.rint(m * 256.0) / 256.0, e)


# ---------------------------------------------------------------------------
# parameters
# ---------------------------------------------------------------------------
def init_params(seed: int) -> dict:
    """He-normal weights, zero biases (the initial state shared with the GPU
    through the flat vector of flatten_params)."""
    rng = np.random.default_rng(seed)
    P = {}
    for name, ci, co, _ in LAYERS:
        P[name + ".w"] = rng.standard_normal((co, ci, 3, 3)) * math.sqrt(2.0 / (9 * ci))
        P[name + ".b"] = np.zeros(co)
    return P


def flatten_params(P: dict) -> np.ndarray:
    """Flat order: per layer, w as [c_out][c_in][3][3] then b."""
    return np.concatenate([np.concatenate([P[n + ".w"].ravel(), P[n + ".b"]]) for n, _, _, _ in LAYERS])


def unflatten_params(v: np.ndarray) -> dict:
    P, k = {}, 0
    for name, ci, co, _ in LAYERS:
        nw = co * ci * 9
        P[name + ".w"] = np.asarray(v[k:k + nw], dtype=np.float64).reshape(co, ci, 3, 3); k += nw
        P[name + ".b"] = np.asarray(v[k:k + co], dtype=np.float64); k += co
    assert k == len(v)
    return P


# ---------------------------------------------------------------------------
# network
# ---------------------------------------------------------------------------
def forward(P: dict, x0, bf16: bool = False):
    """Forward pass of one sample x0 [4, H, W]; returns (y [H, W], cache).
    bf16=True rounds weights and every layer input to bfloat16 precision
    (the storage format of the GPU path); the arithmetic stays FP64."""
    rd = round_bf16 if bf16 else (lambda a: a)
    W_ = {k: (rd(v) if k.endswith(".w") else v) for k, v in P.items()}
    cache = {}

    def layer(name, x, act):
        xin = rd(x)
        z = conv3x3(xin, W_[name + ".w"], W_[name + ".b"])
        cache[name] = (xin, z)
        return relu(z) if act else z

    a1 = layer("c1", x0, True)
    a2 = layer("c2", pool2(a1), True)
    a3 = layer("c3", pool2(a2), True)
    a4 = layer("c4", np.concatenate([up2(a3), a2]), True)
    a5 = layer("c5", np.concatenate([up2(a4), a1]), True)
    y = layer("c6", a5, False)
    cache["acts"] = (a1, a2, a3, a4, a5)
    return y[0], cache


def backward(P: dict, cache: dict, gy):
    """Gradients of a loss with respect to every parameter, given dLoss/dy
    (gy [H, W]) and the cache of forward (taken without bf16 rounding)."""
    G = {}

    def layer_back(name, g_out, act):
        xin, z = cache[name]
        gz = g_out * (z > 0) if act else g_out
        gx, gw, gb = conv3x3_backward(xin, P[name + ".w"], gz)
        G[name + ".w"], G[name + ".b"] = gw, gb
        return gx

    g_a5 = layer_back("c6", gy[None], False)
    g_cat5 = layer_back("c5", g_a5, True)                    # [96]: up(a4) 0..63, a1 64..95
    g_a4 = up2_adjoint(g_cat5[:64])
    g_a1 = g_cat5[64:].copy()
    g_cat4 = layer_back("c4", g_a4, True)                    # [128]: up(a3) 0..63, a2 64..127
    g_a3 = up2_adjoint(g_cat4[:64])
    g_a2 = g_cat4[64:].copy()
    g_a2 += pool2_adjoint(layer_back("c3", g_a3, True))
    g_a1 += pool2_adjoint(layer_back("c2", g_a2, True))
    layer_back("c1", g_a1, True)
    return G


# ---------------------------------------------------------------------------
# the preconditioner's inputs and output
# ---------------------------------------------------------------------------
def faces(coeffs: dict):
    """Zonal and meridional face coefficients of L (the a11 and a22 terms of
    the flux form): ax[j, i] at (i+1/2, j), ay[j, i] at (i, j+1/2), ay = 0 on
    the north pole face."""
    A11, A22 = coeffs["A11"], coeffs["A22"]
    ny, nx = A11.shape
    dlam, dphi = 2 * math.pi / nx, math.pi / ny
    ax = 0.5 * (A11 + np.roll(A11, -1, axis=1)) / dlam ** 2
    ay = np.zeros_like(A22)
    ay[:-1] = 0.5 * (A22[:-1] + A22[1:]) / dphi ** 2
    return ax, ay


def static_features(coeffs: dict, diag_L):
    """Channels 1..3 of x0 and d = |diag(L)|."""
    ax, ay = faces(coeffs)
    ny, nx = ax.shape
    d = np.abs(diag_L)
    zc = (ax + np.roll(ax, 1, axis=1)) / d
    ay_s = np.zeros_like(ay)
    ay_s[1:] = ay[:-1]
    mc = (ay + ay_s) / d
    phi = -math.pi / 2 + (np.arange(ny) + 0.5) * math.pi / ny
    sl = np.repeat(np.sin(phi)[:, None], nx, axis=1)
    return np.stack([zc, mc, sl]), d


def features(r, static):
    s = math.sqrt(float(np.mean(np.asarray(r) ** 2)))
    s = s if s > 0 else 1.0
    return np.concatenate([np.asarray(r)[None] / s, static]), s


def apply(P: dict, r, static, d, bf16: bool = False):
    """e = s y / d for the residual r."""
    x0, s = features(r, static)
    y, _ = forward(P, x0, bf16=bf16)
    return s * y / d


def target(phi, R, d):
    s = math.sqrt(float(np.mean(np.asarray(R) ** 2)))
    return d * phi / s


def loss_and_grad(P: dict, batch):
    """Mean squared error over points and samples; batch = [(x0, y*), ...]."""
    tot, G = 0.0, None
    npts = 0
    for x0, ys in batch:
        y, cache = forward(P, x0)
        diff = y - ys
        tot += float(np.sum(diff * diff))
        npts += diff.size
        g = backward(P, cache, 2.0 * diff)
        G = g if G is None else {k: G[k] + g[k] for k in G}
    return tot / npts, {k: v / npts for k, v in G.items()}


def adamw_step(P: dict, G: dict, state: dict, lr: float, beta1=0.9, beta2=0.999, eps=1e-8, wd=0.0):
    """One AdamW step (decoupled weight decay on the weights, not the biases);
    state holds m, v and the step count t."""
    t = state.get("t", 0) + 1
    state["t"] = t
    for k in P:
        m = state.setdefault("m." + k, np.zeros_like(P[k]))
        v = state.setdefault("v." + k, np.zeros_like(P[k]))
        m[...] = beta1 * m + (1 - beta1) * G[k]
        v[...] = beta2 * v + (1 - beta2) * G[k] ** 2
        mh = m / (1 - beta1 ** t)
        vh = v / (1 - beta2 ** t)
        decay = wd * P[k] if k.endswith(".w") else 0.0
        P[k] = P[k] - lr * (mh / (np.sqrt(vh) + eps) + decay)
    return P
