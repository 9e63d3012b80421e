"""Pins of the oracle's coordinate-dependent (non-Condon) dipole super-operators (Sec. III) against what
the mathematics fixes:

* a coordinate-independent table reduces to the Condon products of the C oracle;
* plane waves along p are eigenvectors of the discrete convolution: a wave e^{2 pi i n l / np} is
  multiplied by mu(q - n dr / 2) from the left and mu(q + n dr / 2) from the right (dr = 2 pi / (np dp)),
  evaluated from the dipole function itself, not from the table's indexing;
* (mu^-> W)^dagger = mu^<- (W^dagger) for a real symmetric dipole;
* the phase-space trace of mu^-> W is the non-Condon trace Tr{mu W}, and with a constant dipole the
  non-Condon trace and response equal the Condon ones.
"""
import numpy as np
import pytest

import oracle
import qhfpe_inputs as qi
from oracle import noncondon as nc


def _model(S=2, nq=10, n_p=16):
    if S == 2:
        return qi.harmonic_two_state(nq=nq, n_p=n_p, depth=1)
    return qi.three_state(nq=nq, n_p=n_p, depth=1, n_matsubara=0)


@pytest.mark.parametrize("S", [2, 3])
def test_constant_dipole_reduces_to_condon(S):
    m = _model(S)
    O = oracle.Oracle(m)
    mu = np.asarray(m["mu"], dtype=np.float64)
    F = [[(lambda c: (lambda q: np.full_like(np.asarray(q, dtype=np.float64), c)))(mu[j, k]) for k in range(S)]
         for j in range(S)]
    T = qi.function_table(m, F)
    W = qi.random_state(m, seed=101)
    for side in (nc.LEFT, nc.RIGHT, nc.COMMUTATOR):
        ref = O.apply_dipole(W, side)
        got = nc.apply_dipole(W, T, side)
        assert np.linalg.norm(got - ref) <= 1e-13 * np.linalg.norm(ref)
    assert abs(nc.trace(W, T, O.dq, O.dp) - O.trace(W)) <= 1e-13 * abs(O.trace(W))


def test_plane_waves_pick_mu_at_half_the_r_offset():
    m = _model(2, nq=6, n_p=16)
    n_p, nq = m["np"], m["nq"]
    dp = (m["p_max"] - m["p_min"]) / n_p
    dr = 2 * np.pi / (n_p * dp)
    a, b = 0.7, 0.15

    def mu01(q):
        return a + b * np.sin(np.asarray(q))

    F = [[None, mu01], [mu01, None]]
    T = qi.function_table(m, F)
    q = qi.axis(nq, m["q_min"], m["q_max"])
    lidx = np.arange(n_p)
    for n in (-5, -1, 0, 2, 7):  # not the Nyquist wave
        wave = np.exp(2j * np.pi * n * lidx / n_p)
        W = np.zeros((1, 2, 2, nq, n_p), dtype=np.complex128)
        W[0, 1, 0] = wave[None, :]  # only W_10 is non-zero
        L = nc.apply_dipole(W, T, nc.LEFT)      # (mu^-> W)_00 = mu_01 * W_10
        R = nc.apply_dipole(W, T, nc.RIGHT)     # (mu^<- W)_11 = W_10 * mu_01
        for i in range(nq):
            assert np.allclose(L[0, 0, 0, i], mu01(q[i] - n * dr / 2) * wave, atol=1e-13)
            assert np.allclose(R[0, 1, 1, i], mu01(q[i] + n * dr / 2) * wave, atol=1e-13)
        assert np.abs(L[0, 1]).max() < 1e-13 and np.abs(R[0, 0]).max() < 1e-13


def test_adjoint_relation_and_trace():
    m = _model(3, nq=8, n_p=16)
    O = oracle.Oracle(m)
    T = qi.function_table(m, qi.linear_dipole(m, slope=0.2))
    W = qi.random_state(m, seed=102)
    dag = lambda X: np.conj(np.transpose(X, (0, 2, 1, 3, 4)))
    L = nc.apply_dipole(W, T, nc.LEFT)
    R = nc.apply_dipole(dag(W), T, nc.RIGHT)
    assert np.linalg.norm(dag(L) - R) <= 1e-13 * np.linalg.norm(L)
    # phase-space trace of mu^-> W: the p-sum of a circulant picks its r = 0 multiplier, mu(q_i)
    ps_trace = sum(L[0, j, j].sum() for j in range(3)) * O.dq * O.dp
    assert abs(ps_trace - nc.trace(W, T, O.dq, O.dp)) <= 1e-12 * abs(ps_trace)


def test_constant_dipole_response_equals_condon_response():
    m = qi.harmonic_two_state(nq=16, n_p=16, depth=2)
    O = oracle.Oracle(m)
    Weq, _ = O.equilibrate(100)
    mu = np.asarray(m["mu"], dtype=np.float64)
    F = [[(lambda c: (lambda q: np.full_like(np.asarray(q, dtype=np.float64), c)))(mu[j, k]) for k in range(2)]
         for j in range(2)]
    R_nc = nc.linear_response(O, Weq, qi.function_table(m, F), 30)
    R_c = O.linear_response(Weq, 30)
    assert np.linalg.norm(R_nc - R_c) <= 1e-12 * np.linalg.norm(R_c)


def test_constant_dipole_first_order_distribution_equals_condon():
    m = qi.harmonic_two_state(nq=16, n_p=16, depth=1)
    O = oracle.Oracle(m)
    Weq, _ = O.equilibrate(80)
    mu = np.asarray(m["mu"], dtype=np.float64)
    F = [[(lambda c: (lambda q: np.full_like(np.asarray(q, dtype=np.float64), c)))(mu[j, k]) for k in range(2)]
         for j in range(2)]
    om = [9.0, -9.0]
    a = nc.first_order_distribution(O, Weq, qi.function_table(m, F), 6, 3, om)
    b = O.first_order_distribution(Weq, 6, 3, om)
    assert np.linalg.norm(a - b) <= 1e-12 * np.linalg.norm(b)
