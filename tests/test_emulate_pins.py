"""Pins of the reduced-precision emulation (oracle/emulate.py).

* The rounding function against IEEE conversions of numpy (FP16, FP32, with
  subnormals and exact ties) and torch (BF16), and, with an unbounded
  exponent, against the C oracle's own rounding routine.
* The 16-bit storage with row scales: power-of-two scales, stored values on
  the format's grid and bounded by 1, the half-spacing error bound, FP32 on
  the pole band; tiny rows keep their relative accuracy where an unscaled
  IEEE half flushes them to zero (the reason for the scale: 5 exponent bits
  against the paper's 11, Sec. 4.1).
* With every field kept in FP64 the emulated solve is the FP64 oracle's GCR
  iterate for iterate; with the mixed storage it still reaches the FP64 true
  residual (the reliable update, Sec. 4) close to the oracle's solution and
  with about the oracle's iteration count (Sec. 4.3).
"""
import numpy as np
import pytest

import oracle as O
from oracle import emulate as E
import synth

pytestmark = pytest.mark.filterwarnings("ignore::RuntimeWarning")


def wide_sample(seed, n, lo, hi):
    rng = np.random.default_rng(seed)
    return rng.choice([-1.0, 1.0], n) * 10.0 ** rng.uniform(lo, hi, n)


def test_round_fp16_is_ieee_half():
    x = wide_sample(1, 20000, -9, 4.6)           # normals, subnormals, flushes
    got = E.round_fmt(x, *E.FORMATS["fp16"])
    assert np.array_equal(got, x.astype(np.float16).astype(np.float64))
    # exact ties go to the even neighbour
    ties = np.array([1 + 2.0 ** -11, 1 + 3 * 2.0 ** -11, 2.0 ** -24 * 0.5, 2.0 ** -24 * 1.5,
                     2.0 ** -14 * (1 + 2.0 ** -11)])
    assert np.array_equal(E.round_fmt(ties, 10, -14), ties.astype(np.float16).astype(np.float64))
    assert np.array_equal(E.round_fmt(ties, 10, -14),
                          [1.0, 1 + 2.0 ** -9, 0.0, 2.0 ** -23, 2.0 ** -14])


def test_round_fp32_is_ieee_single():
    x = wide_sample(2, 20000, -44, 30)
    got = E.round_fmt(x, *E.FORMATS["fp32"])
    assert np.array_equal(got, x.astype(np.float32).astype(np.float64))


def test_round_bf16_is_torch_bfloat16():
    torch = pytest.importorskip("torch")
    # FP32 inputs, so torch's conversion rounds once
    x = wide_sample(3, 20000, -40, 30).astype(np.float32)
    ref = torch.from_numpy(x).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(E.round_fmt(x.astype(np.float64), *E.FORMATS["bf16"]), ref)


@pytest.mark.parametrize("p", [7, 10, 23])
def test_unbounded_exponent_matches_the_c_oracle(p):
    x = wide_sample(4 + p, 500, -300, 300)
    got = E.round_fmt(x, p, None)
    assert np.array_equal(got, [O.round_bits(v, p) for v in x])


@pytest.mark.parametrize("fmt,p", [("fp16", 10), ("bf16", 7)])
def test_row_scaled_storage(fmt, p):
    rng = np.random.default_rng(5)
    ny, nx, band = 16, 64, 2
    mags = 10.0 ** rng.uniform(-30, 8, ny)
    q = rng.standard_normal((ny, nx)) * mags[:, None]
    s = E.store_q(q, fmt, band)
    for j in range(ny):
        if j < band or j >= ny - band:
            assert np.array_equal(s[j], q[j].astype(np.float32).astype(np.float64))
            continue
        sc = E.row_scale(q[j])
        m, e = np.frexp(sc)
        assert m == 0.5                                   # a power of two
        assert sc / 2 <= np.max(np.abs(q[j])) < sc
        y = s[j] / sc                                     # exact: power of two
        assert np.max(np.abs(y)) <= 1.0
        if fmt == "fp16":
            assert np.array_equal(y, y.astype(np.float16).astype(np.float64))
        # at most half the spacing 2^-(p+1) of the top binade [1/2, 1)
        assert np.max(np.abs(s[j] - q[j])) <= 2.0 ** -(p + 2) * sc
    # without a scale an IEEE half loses rows below its range
    tiny = 1e-9 * rng.standard_normal((4, nx))
    assert np.all(E.round_fmt(tiny, 10, -14) == 0.0)
    kept = E.store_q(tiny, "fp16", 0)
    assert np.max(np.abs(kept - tiny) / np.max(np.abs(tiny))) <= 2.0 ** -11


def test_default_band_is_the_papers():
    import json
    import os
    g = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_constants.json")))
    for nx, b in g["pole_band_rows"]["value"].items():
        assert E.default_band(int(nx) // 2) == b


@pytest.mark.parametrize("nx,ny,seed", [(64, 32, 31), (128, 64, 32)])
def test_fp64_storage_reproduces_the_oracle(nx, ny, seed):
    P = synth.problem(nx, ny, seed)
    o = O.Opts(k=4, tol=1e-10, max_iters=300)
    ref, st = O.Problem(P).gcr(P["R"], o)
    phi, se = E.MixedSolve(P, qfmt="fp64", vfmt="fp64", cfmt="fp64").solve(P["R"], o)
    assert se["iterations"] == st["iterations"] and se["converged"] == 1
    assert np.linalg.norm(phi - ref) <= 1e-12 * np.linalg.norm(ref)
    assert abs(se["true_rel_residual"] - st["true_rel_residual"]) <= 1e-3 * st["true_rel_residual"]


@pytest.mark.parametrize("qfmt", ["fp16", "bf16"])
@pytest.mark.parametrize("nx,ny,seed", [(128, 64, 41), (256, 128, 42)])
def test_mixed_storage_reaches_the_fp64_residual(qfmt, nx, ny, seed):
    P = synth.problem(nx, ny, seed)
    tol = 1e-8
    o = O.Opts(k=4, tol=tol, max_iters=400)
    _, st = O.Problem(P).gcr(P["R"], o)
    exact, _ = O.Problem(P).gcr(P["R"], O.Opts(k=4, tol=1e-13, max_iters=3000))
    phi, se = E.MixedSolve(P, qfmt=qfmt).solve(P["R"], o)
    assert se["converged"] == 1 and se["true_rel_residual"] <= tol
    # the true residual of the result, recomputed by the oracle
    r = O.Problem(P).operator(phi) - P["R"]
    assert np.linalg.norm(r) <= tol * np.linalg.norm(P["R"])
    assert np.linalg.norm(phi - exact) <= 1e-6 * np.linalg.norm(exact)
    # a 16-bit preconditioner costs few iterations (Sec. 4.3)
    assert st["iterations"] - 1 <= se["iterations"] <= 1.5 * st["iterations"] + 2


# ---------------------------------------------------------------------------
# split fluid thickness for the residual (Sec. 4.2, Eq. 14)
# ---------------------------------------------------------------------------

@pytest.fixture(scope="module")
def split_case():
    nx, ny = 256, 128
    st = synth.synthetic_state(nx, ny, 25)
    P = synth.coefficients(st)
    P["R"] = synth.rhs_divergence(nx, ny, 25)
    dphi, _ = O.Problem(P).gcr(P["R"], O.Opts(tol=1e-12))
    return P, st.phi_star.copy(), dphi


def test_numpy_operator_is_the_oracle_operator(split_case):
    P, phin, _ = split_case
    x = np.random.default_rng(1).standard_normal(phin.shape)
    a = O.Problem(P).operator(x)
    assert np.linalg.norm(E.operator_np(P, x) - a) <= 1e-13 * np.linalg.norm(a)
    # Eq. 14 in double precision is L(hat + tilde), by linearity
    hat, tilde = phin, x
    b = E.operator_np(P, tilde, hat=hat, hat_grads=E.face_gradients(hat))
    c = O.Problem(P).operator(hat + tilde)
    assert np.linalg.norm(b - c) <= 1e-13 * np.linalg.norm(c)


def test_split_phi_recovers_the_derivative_terms(split_case):
    """Sec. 4.2: with the derivatives of Phi_hat stored, single-precision r0
    loses far less than with Phi truncated to single precision: about four
    orders of magnitude near the poles, two elsewhere.  The split acts on the
    derivative (A) terms, so they are taken alone (B = C = 0).  The state is
    a full depth (8000 m); the exact solution is one solver increment away."""
    P, phin, dphi = split_case
    Q = dict(P, B1=0 * P["B1"], B2=0 * P["B2"], C=0 * P["C"])
    prob = O.Problem(Q)
    R = prob.operator(phin + dphi)
    r_dp = prob.operator(phin) - R

    def rowrel(r):
        return np.sqrt(np.sum((r - r_dp) ** 2, axis=1)) / np.sqrt(np.sum(r_dp ** 2, axis=1))

    plain = rowrel(E.operator_np(Q, phin.astype(np.float32), np.float32).astype(np.float64) - R)
    ny = phin.shape[0]
    mid = slice(ny // 4, 3 * ny // 4)
    gains = []
    for steps in (0, 1, 10):                      # increments added since the refresh
        hat, _ = E.split_phi(phin - steps * dphi)
        tilde = (phin - hat.astype(np.float64)).astype(np.float32)
        hg = [g.astype(np.float32) for g in E.face_gradients(hat.astype(np.float64))]
        split = rowrel(E.operator_np(Q, tilde, np.float32, hat=hat, hat_grads=hg).astype(np.float64) - R)
        gains.append((max(plain[0], plain[-1]) / max(split[0], split[-1]),
                      np.median(plain[mid]) / np.median(split[mid])))
    pole0, mid0 = gains[0]
    assert pole0 >= 1e4 and mid0 >= 1e2
    # the gain shrinks as Phi_tilde grows: the reason for the periodic refresh
    assert gains[0][0] > gains[1][0] > gains[2][0]
    assert gains[0][1] >= gains[1][1] > gains[2][1]
