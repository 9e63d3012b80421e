"""Pins of the oracle's nonlinear system-bath coupling, V(q) = q + c2 q^2 (Sec. II keeps V general),
against an independent method (no GPU).

The same hierarchy, Eq. (heom), written for density matrices in a truncated harmonic-oscillator basis,
with every operator of Sec. II taken from its definition as a super-operator and evaluated by operator
algebra alone (no Wigner-space calculus):  Phi X = i[V, X],  Psi X = (V X + X V)/2,  K X = i[T, X] with
T = p^2/2 (the kinetic part of the Liouvillian),  Lambda^(1) = Psi K - K Psi,  Lambda^(2) = Psi Lambda^(1)
- Lambda^(1) Psi.  Expanding the nested commutators gives Lambda^(1) X = (i/2){[V, T], X} and, writing
Lambda^(1) X = -(1/2){A, X}, Lambda^(2) X = (1/4)[[A, V], X]; with [q, p] = i, [V, T] = i A,
A = p + c2 (q p + p q), and [A, V] = -i (1 + 2 c2 q)^2.  The hierarchy uses these closed forms (the
literal nested products of truncated q and p matrices are wrong at the top levels and destabilise it);
a separate test checks them against the literal nested commutators on low-level states.  The oracle
uses the Wigner-space forms it derives from the same definitions (phi(q) = 1 + 2 c2 q):
Phi = -phi d/dp, Lambda^(1) = -p phi - (c2/2) d2/dp dq, Lambda^(2) = c2 phi d/dp.  A wrong sign or
factor in any of them, or a missing Lambda^(2) coupling to W^(n - 2 e_0), moves R1 by far more than the
truncation differences (checked below).
"""
import functools
import math

import numpy as np
import pytest

import oracle
import qhfpe_inputs as qi


def _relerr(a, b):
    return np.linalg.norm(np.ravel(a - b)) / max(np.linalg.norm(np.ravel(b)), 1e-300)


class _HOBasisHEOMGeneralV:
    """Eq. (heom) for density matrices, one Drude mode (K = 0, high temperature), truncated at depth N,
    coupling function V given as a matrix in the oscillator basis."""

    def __init__(self, S, n_v, d, E, Vc, c2, co, depth, mu):
        a = np.diag(np.sqrt(np.arange(1, n_v)), 1)
        q = (a + a.T) / math.sqrt(2)
        p = 1j * (a.T - a) / math.sqrt(2)
        num = np.diag(np.arange(n_v) + 0.5)
        Iv, Ie = np.eye(n_v), np.eye(S)
        H = np.zeros((S * n_v, S * n_v), complex)
        for j in range(S):
            blk = num - d[j] * q + (0.5 * d[j] ** 2 + E[j]) * Iv
            H[j * n_v:(j + 1) * n_v, j * n_v:(j + 1) * n_v] = blk
            for k in range(S):
                if k != j:
                    H[j * n_v:(j + 1) * n_v, k * n_v:(k + 1) * n_v] = Vc[j][k] * Iv
        self.H = H
        self.V = np.kron(Ie, q + c2 * (q @ q))
        self.T = np.kron(Ie, 0.5 * (p @ p))
        self.A = np.kron(Ie, p + c2 * (q @ p + p @ q))
        f = Iv + 2.0 * c2 * q
        self.C2 = np.kron(Ie, -1j * (f @ f))  # [A, V]
        self.mu = np.kron(mu, Iv)
        self.co = co
        self.depth = depth

    def phi(self, X):
        return 1j * (self.V @ X - X @ self.V)

    def psi(self, X):
        return 0.5 * (self.V @ X + X @ self.V)

    def kin(self, X):
        return 1j * (self.T @ X - X @ self.T)

    def lam1_nested(self, X):
        return self.psi(self.kin(X)) - self.kin(self.psi(X))

    def lam2_nested(self, X):
        return self.psi(self.lam1_nested(X)) - self.lam1_nested(self.psi(X))

    def lam1(self, X):
        return -0.5 * (self.A @ X + X @ self.A)

    def lam2(self, X):
        return 0.25 * (self.C2 @ X - X @ self.C2)

    def rhs(self, R):
        g, r, c = self.co["gamma"][0], self.co["r"][0], self.co["c"][0]
        out = []
        N = self.depth
        for n in range(N + 1):
            X = R[n]
            d = -1j * (self.H @ X - X @ self.H) - n * g * X
            if n < N:
                d = d - self.phi(R[n + 1])
            if n > 0:
                d = d - n * g * (r * self.lam1(R[n - 1]) + c * self.phi(R[n - 1]))
            if n > 1:
                d = d - 0.5 * n * (n - 1) * g * g * r * r * self.lam2(R[n - 2])
            out.append(d)
        return np.array(out)

    def rk4(self, R, dt, n):
        for _ in range(n):
            k1 = self.rhs(R)
            k2 = self.rhs(R + 0.5 * dt * k1)
            k3 = self.rhs(R + 0.5 * dt * k2)
            k4 = self.rhs(R + dt * k3)
            R = R + dt / 6 * (k1 + 2 * k2 + 2 * k3 + k4)
        return R


def _model(c2):
    m = qi.harmonic_two_state(nq=48, n_p=48, qr=(-8.0, 8.0), pr=(-8.0, 8.0), displacement=1.0, gap=2.0,
                              coupling=0.3, eta=0.3, gamma=1.0, beta=1.0, depth=3, closure=0, dt=0.01)
    m["v_c2"] = c2
    return m


@functools.lru_cache(maxsize=4)
def _r1_pair(c2, n_t=400, n_v=36):
    """R1 of the oracle and of the density-matrix hierarchy for coupling c2 (each from its own
    equilibrium: the oracle's Boltzmann start relaxed 4000 steps, the canonical state relaxed by the
    ground-state density-matrix hierarchy 2000 steps of 0.02)."""
    m = _model(c2)
    O = oracle.Oracle(m)
    co = O.coefficients()
    Weq, _ = O.equilibrate(4000)
    R1_w = O.linear_response(Weq, n_t)
    depth, beta = m["depth"], m["beta"]
    B1 = _HOBasisHEOMGeneralV(1, n_v, [0.0], [0.0], [[0]], c2, co, depth, np.array([[1.0]]))
    rho0 = np.zeros((depth + 1, n_v, n_v), complex)
    w, U = np.linalg.eigh(B1.H)
    th = U @ np.diag(np.exp(-beta * w)) @ U.conj().T
    rho0[0] = th / np.trace(th)
    rho_eq = B1.rk4(rho0, 0.02, 2000)
    B = _HOBasisHEOMGeneralV(2, n_v, [0.0, 1.0], [0.0, 2.0], [[0, 0.3], [0.3, 0]], c2, co, depth, m["mu"])
    R = np.zeros((depth + 1, 2 * n_v, 2 * n_v), complex)
    R[:, :n_v, :n_v] = rho_eq
    R = np.array([B.mu @ X - X @ B.mu for X in R])
    R1_h = [1j * np.trace(B.mu @ R[0])]
    for _ in range(n_t):
        R = B.rk4(R, m["dt"], 1)
        R1_h.append(1j * np.trace(B.mu @ R[0]))
    return R1_w, np.array(R1_h)


@pytest.mark.parametrize("c2", [0.0, 0.12])
def test_closed_forms_equal_the_nested_commutators(c2):
    """Lambda^(1) = Psi K - K Psi and Lambda^(2) = Psi Lambda^(1) - Lambda^(1) Psi, formed literally from
    the matrices, equal the closed forms on states confined to low levels (where the truncation of the
    basis does not enter)."""
    co = {"gamma": [1.0], "r": [0.3], "c": [0.6]}
    n_v = 40
    B = _HOBasisHEOMGeneralV(1, n_v, [0.0], [0.0], [[0]], c2, co, 2, np.array([[1.0]]))
    rng = np.random.default_rng(2)
    X = np.zeros((n_v, n_v), complex)
    X[:10, :10] = rng.standard_normal((10, 10)) + 1j * rng.standard_normal((10, 10))
    scale = np.abs(X).max()
    assert np.abs(B.lam1_nested(X) - B.lam1(X)).max() < 1e-12 * scale
    assert np.abs(B.lam2_nested(X) - B.lam2(X)).max() < 1e-12 * scale
    if c2 != 0.0:
        assert np.abs(B.lam2(X)).max() > 1e-2 * np.abs(X).max()


def test_general_v_super_operators_reduce_to_the_linear_ones():
    """For V = q the nested commutators give Lambda^(1) = -(1/2){p, .} and Lambda^(2) = 0 (the linear
    coupling of Sec. II), which the density-matrix hierarchy of the other pins uses directly."""
    co = {"gamma": [1.0], "r": [0.3], "c": [0.6]}
    B = _HOBasisHEOMGeneralV(1, 30, [0.0], [0.0], [[0]], 0.0, co, 2, np.array([[1.0]]))
    rng = np.random.default_rng(1)
    X = np.zeros((30, 30), complex)
    X[:8, :8] = rng.standard_normal((8, 8)) + 1j * rng.standard_normal((8, 8))  # low levels only
    a = np.diag(np.sqrt(np.arange(1, 30)), 1)
    p = 1j * (a.T - a) / math.sqrt(2)
    assert _relerr(B.lam1(X), -0.5 * (p @ X + X @ p)) < 1e-12
    assert np.abs(B.lam2(X)).max() < 1e-12 * np.abs(X).max()


def test_zero_c2_is_the_linear_coupling():
    m = qi.harmonic_two_state(nq=16, n_p=16, depth=2, closure=0)
    W = qi.random_state(m, seed=5)
    assert np.array_equal(oracle.Oracle(m).rhs(W), oracle.Oracle(dict(m, v_c2=0.0)).rhs(W))


def test_nonlinear_coupling_requires_truncation():
    m = qi.harmonic_two_state(nq=16, n_p=16, depth=2, closure=1)
    with pytest.raises(ValueError):
        oracle.Oracle(dict(m, v_c2=0.1))


@pytest.mark.slow
def test_nonlinear_linear_response_against_vibrational_basis_heom():
    c2 = 0.12
    R1_w, R1_h = _r1_pair(c2)
    err = _relerr(R1_w, R1_h)
    # the oracle's linear-coupling R1 on the same grid: the nonlinear coupling moves R1 far beyond the
    # agreement of the two truncations (48 x 48 grid, 36 levels; the linear coupling itself is pinned
    # against the same density-matrix hierarchy by the pins of the linear model)
    m0 = _model(0.0)
    O0 = oracle.Oracle(m0)
    R1_w0 = O0.linear_response(O0.equilibrate(4000)[0], len(R1_w) - 1)
    shift = _relerr(R1_w, R1_w0)
    print(f"c2 {c2}: oracle vs density matrix {err:.2e}; nonlinear shift {shift:.2e}")
    assert err < 2e-3
    assert shift > 20 * err
