"""Pins of the oracle's adiabatic-basis wavepacket marginals (Sec. III, "Wavepacket dynamics") against
what the mathematics fixes: the trace is basis-invariant; without diabatic coupling the adiabatic
states are the diabatic ones ordered by energy; for two states the lower eigenvector has a closed
form; a state that is a pure adiabatic population maps to that population; Hermitian states give
Hermitian marginals; the p-sum is the p-integral of a smooth Gaussian."""
import numpy as np
import pytest

import qhfpe_inputs as qi
from oracle import marginals as om


def _grid(m):
    return (m["p_max"] - m["p_min"]) / m["np"]


def test_trace_is_invariant():
    for m in (qi.morse_photoisomerization(nq=64, n_p=16), qi.three_state(nq=12, n_p=8, depth=1, n_matsubara=0)):
        W = qi.random_state(m, seed=81)
        P = om.adiabatic_marginals(W, qi.u_table(m), _grid(m))
        rho = om.coordinate_marginals(W[0], _grid(m))
        S = m["S"]
        tr_ad = sum(P[a, a] for a in range(S))
        tr_di = sum(rho[j, j] for j in range(S))
        assert np.allclose(tr_ad, tr_di, rtol=0, atol=1e-12 * np.abs(tr_di).max())


def test_no_coupling_orders_the_diabatic_states_by_energy():
    m = qi.harmonic_two_state(nq=40, n_p=8, coupling=0.0)
    T = qi.u_table(m)
    W = qi.random_state(m, seed=82)
    P = om.adiabatic_marginals(W, T, _grid(m))
    rho = om.coordinate_marginals(W[0], _grid(m))
    U = om.diabatic_matrix(T)
    for i in range(m["nq"]):
        lo, hi = (0, 1) if U[i, 0, 0] <= U[i, 1, 1] else (1, 0)
        assert P[0, 0, i] == pytest.approx(rho[lo, lo, i], abs=1e-14)
        assert P[1, 1, i] == pytest.approx(rho[hi, hi, i], abs=1e-14)
        # coherences: the same element, signs fixed by the convention (each vector is +e_j)
        assert P[0, 1, i] == pytest.approx(rho[lo, hi, i], abs=1e-14)


def test_two_state_lower_eigenvector_closed_form():
    m = qi.morse_photoisomerization(nq=200, n_p=8)
    T = qi.u_table(m)
    U = om.diabatic_matrix(T)
    V = om.adiabatic_basis(U)
    a, b, c = U[:, 0, 0], U[:, 1, 1], U[:, 0, 1]
    lam = 0.5 * (a + b) - np.sqrt(0.25 * (a - b) ** 2 + c * c)
    # (U - lam) v = 0: v = (c, lam - a) from the first row, or (lam - b, c) from the second; take the
    # one whose large component does not come from a cancellation
    first = np.abs(lam - a) >= np.abs(lam - b)
    v0 = np.where(first, c, lam - b)
    v1 = np.where(first, lam - a, c)
    nrm = np.hypot(v0, v1)
    v0, v1 = v0 / nrm, v1 / nrm
    lead_is_0 = np.abs(v0) >= np.abs(v1) - 1e-9
    sgn = np.where(lead_is_0, np.sign(v0), np.sign(v1))
    assert np.allclose(V[:, 0, 0], sgn * v0, atol=1e-12)
    assert np.allclose(V[:, 1, 0], sgn * v1, atol=1e-12)
    # the eigenvalue equation itself, for both vectors
    for i in range(0, 200, 17):
        w = np.linalg.eigvalsh(U[i])
        for k in range(2):
            assert np.allclose(U[i] @ V[i, :, k], w[k] * V[i, :, k], atol=1e-9 * np.abs(U[i]).max())


def test_pure_adiabatic_population():
    m = qi.morse_photoisomerization(nq=96, n_p=16)
    T = qi.u_table(m)
    V = om.adiabatic_basis(om.diabatic_matrix(T))
    q = qi.axis(m["nq"], m["q_min"], m["q_max"])
    p = qi.axis(m["np"], m["p_min"], m["p_max"])
    dp = _grid(m)
    f = np.exp(-0.5 * ((q - 10.0) / 3.0) ** 2)
    g = np.exp(-0.5 * (p / 2.0) ** 2)
    W = np.zeros((1, 2, 2, m["nq"], m["np"]), dtype=np.complex128)
    a = 1  # the upper adiabatic state
    for j in range(2):
        for k in range(2):
            W[0, j, k] = (f * V[:, j, a] * V[:, k, a])[:, None] * g[None, :]
    P = om.adiabatic_marginals(W, T, dp)
    norm = g.sum() * dp
    assert np.allclose(P[1, 1], f * norm, atol=1e-13)
    assert np.abs(P[0, 0]).max() < 1e-13 and np.abs(P[0, 1]).max() < 1e-13


def test_hermitian_states_give_hermitian_marginals():
    m = qi.three_state(nq=10, n_p=8, depth=1, n_matsubara=0)
    W = qi.random_state(m, seed=83, hermitian=True)
    P = om.adiabatic_marginals(W, qi.u_table(m), _grid(m))
    assert np.allclose(P, np.conj(np.transpose(P, (1, 0, 2))), atol=1e-13)
    for a in range(3):
        assert np.abs(P[a, a].imag).max() < 1e-13


def test_p_sum_is_the_gaussian_integral():
    m = qi.harmonic_two_state(nq=4, n_p=64, pr=(-8.0, 8.0))
    p = qi.axis(m["np"], m["p_min"], m["p_max"])
    sigma = 1.3
    W0 = np.zeros((2, 2, 4, 64), dtype=np.complex128)
    W0[0, 0] = np.exp(-0.5 * (p / sigma) ** 2)[None, :]
    rho = om.coordinate_marginals(W0, _grid(m))
    assert np.allclose(rho[0, 0], np.sqrt(2 * np.pi) * sigma, rtol=1e-12)
