"""Pins of the oracle's learned-closure pieces (CPU): the regression statistics, the backpropagated
gradient, and the closure term inside the right-hand side."""
import math

import numpy as np
import pytest

import oracle
import qhfpe_inputs as qi
from oracle import closure as cl


def _small_model(depth=3, closure=2, **kw):
    m = qi.harmonic_two_state(nq=8, n_p=16, depth=depth, closure=closure, **kw)
    return m


@pytest.mark.parametrize("terminator", [False, True])
def test_statistics_reproduce_the_direct_squared_error(terminator):
    """sum_x (c^T G c - 2 c^T h + yy) / n equals the mean of |sum_f c_f phi_f - y|^2 over all samples,
    with y the target tier itself or its residual after the terminator's estimate."""
    m = _small_model(depth=4)
    W = qi.random_state(m, seed=3)
    tier = 3
    p = qi.axis(16, -8, 8)
    dp = p[1] - p[0]
    r0, c0 = (0.7, 1.3) if terminator else (0.0, 0.0)
    w = cl.init_weights(7)
    w[-cl.N_OUT * (cl.N_HID + 1):] = np.random.default_rng(8).normal(size=cl.N_OUT * (cl.N_HID + 1)) * 0.1
    X = cl.inputs(*np.meshgrid(qi.axis(8, -8, 8), p, indexing="ij"), m["eta"]).reshape(-1, 3)
    stats = cl.statistics(W, tier, r0, c0, p, dp)
    L = cl.loss(w, X, stats)
    c, _ = cl.forward(w, X)
    c = c.reshape(8, 16, 10)
    # direct: the terminator's estimate r0 p W^N + c0 (4th-order d/dp) W^N, then the patch combination
    WN, WN1, Wt = W[tier - 1], W[tier - 2], W[tier]
    dWN = (np.roll(WN, 2, -1) - 8 * np.roll(WN, 1, -1) + 8 * np.roll(WN, -1, -1) - np.roll(WN, -2, -1)) / (12 * dp)
    target = Wt - (r0 * p * WN + c0 * dWN)
    pred = np.zeros_like(Wt)
    for b in range(-2, 3):
        pred += c[..., 2 + b] * np.roll(WN, -b, -1) + c[..., 7 + b] * np.roll(WN1, -b, -1)
    direct = (np.abs(pred - target) ** 2).sum() / target.size
    assert L == pytest.approx(direct, rel=1e-12)


@pytest.mark.parametrize("lam", [0.0, 0.3])
def test_backprop_gradient_matches_finite_differences(lam):
    m = _small_model(depth=4)
    W = qi.random_state(m, seed=4)
    stats = cl.statistics(W, 3)
    X = cl.inputs(*np.meshgrid(qi.axis(8, -8, 8), qi.axis(16, -8, 8), indexing="ij"), 0.7).reshape(-1, 3)
    w = cl.init_weights(9)
    rng = np.random.default_rng(10)
    w[-cl.N_OUT * (cl.N_HID + 1):] = rng.normal(size=cl.N_OUT * (cl.N_HID + 1)) * 0.05
    L, g = cl.loss_and_grad(w, X, stats, lam)
    assert L == pytest.approx(cl.loss(w, X, stats, lam), rel=1e-14)
    idx = np.concatenate([rng.choice(768, 6, replace=False),                      # W1
                          768 + rng.choice(256, 3, replace=False),                # b1
                          1024 + rng.choice(65536, 6, replace=False),             # W2
                          cl.N_WEIGHTS - 2570 + rng.choice(2570, 8, replace=False)])  # W4, b4
    for k in idx:
        e = 1e-5
        wp, wm = w.copy(), w.copy()
        wp[k] += e
        wm[k] -= e
        fd = (cl.loss(wp, X, stats, lam) - cl.loss(wm, X, stats, lam)) / (2 * e)
        assert g[k] == pytest.approx(fd, rel=2e-6, abs=1e-10)


def test_zero_coefficients_are_the_terminator():
    m = _small_model(depth=3)
    W = qi.random_state(m, seed=5)
    coef = np.zeros((m["nq"], m["np"], 10))
    L_learned = oracle.Oracle(m, closure_coef=coef).rhs(W)
    assert np.array_equal(L_learned, oracle.Oracle(dict(m, closure=1)).rhs(W))


def test_closure_term_on_plane_waves():
    """Constant coefficients c = e_{2+1} add W^N(l+1) to the terminator's W^(N+1); on
    W^N = exp(i kappa p) the top tier gains d/dp of exp(i kappa dp) W^N, with the 4th-order
    difference's symbol i (8 sin(kappa dp) - sin(2 kappa dp)) / (6 dp)."""
    m = _small_model(depth=2)
    coef = np.zeros((m["nq"], m["np"], 10))
    coef[..., 3] = 1.0
    O = oracle.Oracle(m, closure_coef=coef)
    Ot = oracle.Oracle(dict(m, closure=1))
    n_p, dp = m["np"], O.dp
    k = 3
    kappa = 2 * math.pi * k / (n_p * dp)
    W = np.zeros(O.shape, complex)
    W[2, 1, 0] = np.exp(2j * math.pi * k * np.arange(n_p) / n_p)[None, :] * np.ones((m["nq"], 1))
    out = O.rhs(W, oracle.TIER_UP) - Ot.rhs(W, oracle.TIER_UP)
    symbol = 1j * (8 * math.sin(kappa * dp) - math.sin(2 * kappa * dp)) / (6 * dp)
    expect = symbol * np.exp(1j * kappa * dp) * W[2, 1, 0]
    assert np.allclose(out[2, 1, 0], expect, atol=1e-12)
    assert np.abs(out[:2]).max() < 1e-13


def test_correction_can_cancel_the_terminator_momentum_part():
    """c_2 = -r_0 p removes d/dp (r_0 p W^N) from the terminator's term, leaving c_0 d2W^N/dp2."""
    m = _small_model(depth=2)
    W = qi.random_state(m, seed=6)
    p = qi.axis(m["np"], m["p_min"], m["p_max"])
    r0 = m["eta"]
    coef = np.zeros((m["nq"], m["np"], 10))
    coef[..., 2] = -r0 * p[None, :]
    L_learned = oracle.Oracle(m, closure_coef=coef).rhs(W)
    O_t = oracle.Oracle(dict(m, closure=1))
    L_term = O_t.rhs(W)
    d1 = np.array([1, -8, 0, 8, -1]) / (12 * O_t.dp)
    top = W[2]
    dpw = sum(d1[t] * np.roll(r0 * p * top, 2 - t, axis=-1) for t in range(5))
    diff = L_term - L_learned
    assert np.allclose(diff[2], dpw, atol=1e-11)
    assert np.abs(diff[:2]).max() < 1e-12


# ------------------------------------------------------------------------------------------------
# State-input network (the literal closure): inputs layout, backpropagation, bf16 rounding
# ------------------------------------------------------------------------------------------------
def test_state_inputs_layout_on_an_impulse():
    """A single nonzero value of tier N-1 at (i0, l0) of pair (0, 1) appears in the inputs of exactly
    the nine neighbouring points, at the patch position of its offset (q zero-padded, p periodic)."""
    m = qi.harmonic_two_state(nq=6, n_p=8, depth=3)
    W = np.zeros(qi.state_shape(m), complex)
    i0, l0 = 2, 7
    W[2, 0, 1, i0, l0] = 3.0 - 1.0j
    X = cl.state_inputs(W, 3, m)
    base = 3  # tier N (= tier 2 of the state) comes first
    pair = 0 * 2 + 1
    hits = np.argwhere(np.abs(X[..., 3:]) > 0)
    assert len(hits) == 2 * 9
    for a in (-1, 0, 1):
        for b in (-1, 0, 1):
            i, l = i0 - a, (l0 - b) % 8  # the point whose (a, b) neighbour is (i0, l0)
            c = base + 2 * (9 * pair + 3 * (a + 1) + (b + 1))
            assert X[i, l, c] == 3.0 and X[i, l, c + 1] == -1.0
    assert X[0, 0, 0] == m["q_min"] / 8 and X[0, 1, 1] == (m["p_min"] + 2.0) / 8


def test_state_targets_on_plane_waves():
    """The target is W^(t) less r_0 p W^(t-1) + c_0 dW^(t-1)/dp.  With W^(t-1) = exp(i k p) (a plane wave of
    the periodic p grid) the 4th-order central difference is multiplication by
    i (8 sin(k dp) - sin(2 k dp)) / (6 dp), so W^(t) = r_0 p W^(t-1) + c_0 lambda W^(t-1) gives a zero target,
    and W^(t) = 0 gives minus that element; r_0 = eta and c_0 = eta / beta (high temperature, Sec. II)."""
    m = qi.harmonic_two_state(nq=5, n_p=16, depth=3, eta=0.7, beta=0.48)
    n_p, dp = m["np"], (m["p_max"] - m["p_min"]) / m["np"]
    p = m["p_min"] + dp * np.arange(n_p)
    r0, c0 = 0.7, 0.7 / 0.48
    W = np.zeros(qi.state_shape(m), complex)
    for mode, (j, k) in ((3, (0, 1)), (5, (1, 1))):
        kk = 2 * np.pi * mode / (n_p * dp)
        wave = np.exp(1j * kk * (p - m["p_min"]))
        lam = 1j * (8 * np.sin(kk * dp) - np.sin(2 * kk * dp)) / (6 * dp)
        W[1, j, k] = wave[None, :] * (1.0 + np.arange(5))[:, None]
        W[2, j, k] = (r0 * p + c0 * lam) * W[1, j, k]
    Y = cl.state_targets(W, 2, m)
    assert np.abs(Y).max() < 1e-12 * np.abs(W).max()
    W[2] = 0
    Y = cl.state_targets(W, 2, m)
    ref = -(r0 * p + c0 * 1j * (8 * np.sin(2 * np.pi * 3 / n_p) - np.sin(4 * np.pi * 3 / n_p)) / (6 * dp)) * W[1, 0, 1]
    assert np.allclose(Y[..., 2 * 1] + 1j * Y[..., 2 * 1 + 1], ref, rtol=1e-12, atol=1e-12)


def test_state_gradient_matches_finite_differences():
    S = 1
    n_in, n_out = cl.state_sizes(S)
    rng = np.random.default_rng(7)
    w = np.concatenate([rng.normal(size=int(np.prod(s))) * (0.3 / np.sqrt(s[-1]) if len(s) == 2 else 0.1)
                        for s in cl.state_shapes(S)] + [np.ones(3)])
    X = rng.normal(size=(5, n_in))
    Y = rng.normal(size=(5, n_out))
    L, g = cl.state_loss_and_grad(w, X, Y, S)
    n = len(g)
    for idx in rng.choice(n, 25, replace=False):
        e = np.zeros_like(w)
        e[idx] = 1e-6
        fd = (cl.state_loss_and_grad(w + e, X, Y, S)[0] - cl.state_loss_and_grad(w - e, X, Y, S)[0]) / 2e-6
        assert fd == pytest.approx(g[idx], rel=1e-5, abs=1e-9)


def test_bf16_rounding():
    v = np.array([1.0, 1.0 + 2 ** -8, 1.0 + 2 ** -7, 1.0 + 3 * 2 ** -8, -2.5, 1e-3])
    got = cl.bf16(v)
    assert got[0] == 1.0
    assert got[1] == 1.0                  # halfway between 1 and 1 + 2^-7: ties to even
    assert got[2] == 1.0 + 2 ** -7
    assert got[3] == 1.0 + 2 * 2 ** -7    # halfway: ties to even (odd mantissa rounds up)
    assert got[4] == -2.5
    assert abs(got[5] - 1e-3) < 1e-3 * 2 ** -8
