"""Pins of the CPU oracle to what the paper and the mathematics fix (no GPU).

Each test names what it pins.  None of them re-types the oracle's own formula: they use printed values
(tests/golden), closed forms, exact discrete identities, invariants, special cases and an independent
method (a density-matrix HEOM in a truncated vibrational basis).
"""
import functools
import itertools
import math
import os

import numpy as np
import pytest

import oracle
import qhfpe_inputs as qi

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _model(**kw):
    """Two-state harmonic model; keyword arguments go to qhfpe_inputs.harmonic_two_state."""
    return qi.harmonic_two_state(**kw)


def _relerr(a, b):
    return np.linalg.norm(np.ravel(a - b)) / max(np.linalg.norm(np.ravel(b)), 1e-300)


# ------------------------------------------------------------------------------------------------
# P1: the printed upwind stencil (Sec. III) and the orders of the q- and p-differences
# ------------------------------------------------------------------------------------------------
def _read_stencil():
    rows = {}
    with open(os.path.join(GOLDEN, "upwind_stencil.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            br, d, c = line.split()
            rows.setdefault(br, {})[int(d)] = float(c)
    return rows


def test_upwind_stencil_matches_printed_coefficients():
    """Kinetic term on a unit impulse reproduces the printed coefficients for both signs of p."""
    m = qi.single_state(lambda q: 0 * q, nq=16, n_p=8, depth=0, closure=0)
    O = oracle.Oracle(m)
    W = np.zeros(O.shape, complex)
    i0 = 8
    W[0, 0, 0, i0, :] = 1.0
    out = O.rhs(W, oracle.KINETIC)[0, 0, 0]
    p = qi.axis(m["np"], m["p_min"], m["p_max"])
    dq = O.dq
    gold = _read_stencil()
    for l in range(m["np"]):
        br = "p<0" if p[l] < 0 else "p>=0"
        for d, c in gold[br].items():
            # output row i = i0 - d sees the impulse at offset +d with coefficient c
            got = out[i0 - d, l].real / (-p[l]) * 60 * dq if p[l] != 0 else None
            if got is not None:
                assert got == pytest.approx(c, abs=1e-12)
        # rows outside the stencil's reach see nothing
        for i in range(m["nq"]):
            if (i0 - i) not in gold[br]:
                assert out[i, l] == 0


def test_upwind_stencil_order_and_first_error_term():
    """Exact for q^k, k <= 5; for q^6 at q = 0 the error is -12 dq^5 (p >= 0) and +12 dq^5 (p < 0)
    (the sixth moment of the printed stencil is -+720)."""
    m = qi.single_state(lambda q: 0 * q, nq=16, n_p=4, qr=(-4.0, 4.0), depth=0, closure=0)
    O = oracle.Oracle(m)
    q = qi.axis(m["nq"], m["q_min"], m["q_max"])
    p = qi.axis(m["np"], m["p_min"], m["p_max"])
    i0 = int(np.argmin(abs(q)))
    assert q[i0] == 0
    for k in range(0, 7):
        W = np.zeros(O.shape, complex)
        W[0, 0, 0] = (q ** k)[:, None] * np.ones(m["np"])[None, :]
        out = O.rhs(W, oracle.KINETIC)[0, 0, 0]
        for l in range(m["np"]):
            if p[l] == 0:
                continue
            dq_est = out[3:-3, l].real / (-p[l])
            exact = k * q[3:-3] ** (k - 1) if k > 0 else 0 * q[3:-3]
            if k <= 5:
                assert np.allclose(dq_est, exact, atol=1e-10 * max(1, np.abs(exact).max()))
            else:
                err = dq_est[i0 - 3] - 0.0
                expect = -12 * O.dq ** 5 if p[l] >= 0 else 12 * O.dq ** 5
                assert err == pytest.approx(expect, rel=1e-9)


def test_p_differences_order():
    """d/dp (through the tier-up coupling) is exact for p^k, k <= 4, with error -4 dp^4 at p = 0 for
    p^5; d^2/dp^2 (through the delta-term) exact for k <= 5 with error -8 dp^4 at p = 0 for p^6."""
    m = qi.single_state(lambda q: 0 * q, nq=4, n_p=16, pr=(-4.0, 4.0), depth=1, closure=0,
                        high_temperature=0, use_cdelta=1, n_matsubara=1, beta=1.0, gamma=1.0, eta=1.0)
    O = oracle.Oracle(m)
    co = O.coefficients()
    assert co["cdelta"] != 0
    h = O.hierarchy().tolist()
    up0 = h.index([1, 0])
    p = qi.axis(m["np"], m["p_min"], m["p_max"])
    l0 = int(np.argmin(abs(p)))
    for k in range(0, 7):
        W = np.zeros(O.shape, complex)
        W[up0, 0, 0] = np.ones(m["nq"])[:, None] * (p ** k)[None, :]
        d1 = O.rhs(W, oracle.TIER_UP)[0, 0, 0, 1, 2:-2].real
        ex1 = k * p[2:-2] ** (k - 1) if k else 0 * p[2:-2]
        if k <= 4:
            assert np.allclose(d1, ex1, atol=1e-10 * max(1, abs(ex1).max()))
        elif k == 5:
            assert d1[l0 - 2] == pytest.approx(-4 * O.dp ** 4, rel=1e-9)
        W = np.zeros(O.shape, complex)
        W[0, 0, 0] = np.ones(m["nq"])[:, None] * (p ** k)[None, :]
        d2 = O.rhs(W, oracle.DAMPING)[0, 0, 0, 1, 2:-2].real / co["cdelta"]
        ex2 = k * (k - 1) * p[2:-2] ** (k - 2) if k >= 2 else 0 * p[2:-2]
        if k <= 5:
            assert np.allclose(d2, ex2, atol=1e-9 * max(1, abs(ex2).max()))
        elif k == 6:
            assert d2[l0 - 2] == pytest.approx(-8 * O.dp ** 4, rel=1e-9)


# ------------------------------------------------------------------------------------------------
# P2: the potential kernel of Eq. (quantum-liouvillian)
# ------------------------------------------------------------------------------------------------
def test_potential_kernel_constant_surfaces():
    """Constant surfaces a, b: the 10 block rotates at -i(b - a), the 01 block at -i(a - b), the
    diagonal blocks do not move."""
    a, b = 0.7, 3.2
    m = _model()
    m["U"] = [[lambda q: a + 0 * q, None], [None, lambda q: b + 0 * q]]
    O = oracle.Oracle(m)
    W = qi.random_state(m)
    out = O.rhs(W, oracle.POTENTIAL)
    assert np.abs(out[:, 0, 0]).max() < 1e-12
    assert np.abs(out[:, 1, 1]).max() < 1e-12
    assert _relerr(out[:, 1, 0], -1j * (b - a) * W[:, 1, 0]) < 1e-13
    assert _relerr(out[:, 0, 1], -1j * (a - b) * W[:, 0, 1]) < 1e-13


@pytest.mark.parametrize("surface", ["quadratic", "cubic", "anharmonic"])
def test_potential_kernel_plane_waves(surface):
    """A p-plane wave W = exp(i kappa p) (kappa = 2 pi k/(np dp), |k| < np/2) is an eigenfunction of
    the single-state kernel with eigenvalue i [U(q + kappa/2) - U(q - kappa/2)]; for a quadratic
    surface this is U'(q) d/dp, the classical force term, and for a cubic it adds the Moyal term."""
    funcs = {
        "quadratic": lambda q: 0.3 * q * q - 0.7 * q + 2.0,
        "cubic": lambda q: 0.05 * q ** 3 + 0.5 * q * q,
        "anharmonic": lambda q: 5.0 * ((q / 4.0) ** 2 - 1.0) ** 2,
    }
    U = funcs[surface]
    m = qi.single_state(U, nq=8, n_p=32, depth=0, closure=0)
    O = oracle.Oracle(m)
    q = qi.axis(m["nq"], m["q_min"], m["q_max"])
    lidx = np.arange(m["np"])
    for k in (-15, -7, -1, 1, 5, 15):
        kappa = 2 * math.pi * k / (m["np"] * O.dp)
        W = np.zeros(O.shape, complex)
        W[0, 0, 0] = np.exp(2j * math.pi * k * lidx / m["np"])[None, :] * np.ones((m["nq"], 1))
        out = O.rhs(W, oracle.POTENTIAL)[0, 0, 0]
        lam = 1j * (U(q + kappa / 2) - U(q - kappa / 2))
        assert _relerr(out, lam[:, None] * W[0, 0, 0]) < 1e-12
        if surface == "quadratic":
            force = (0.6 * q - 0.7)[:, None] * (1j * kappa) * W[0, 0, 0]
            assert _relerr(out, force) < 1e-12


def test_potential_kernel_keeps_real_diagonal_blocks_real():
    """With the symmetric Nyquist reading, a real W_jj gives a real potential term for any surface."""
    m = qi.photoisomerization_two_state(nq=8, n_p=16, depth=0, n_matsubara=0)
    m["U"][0][1] = m["U"][1][0] = None
    O = oracle.Oracle(m)
    W = np.zeros(O.shape, complex)
    W[0, 0, 0] = np.random.default_rng(1).uniform(-1, 1, (8, 16))
    out = O.rhs(W, oracle.POTENTIAL)
    assert np.abs(out[0, 0, 0].imag).max() < 1e-12 * np.abs(out).max()
    assert np.abs(out[0, 0, 0]).max() > 1e-3


# ------------------------------------------------------------------------------------------------
# P3: invariants of the full right-hand side
# ------------------------------------------------------------------------------------------------
@pytest.mark.parametrize("kind", ["harmonic", "photoiso"])
def test_rhs_conserves_trace_and_hermiticity(kind):
    if kind == "harmonic":
        m = _model(periodic_q=1)
    else:
        m = qi.photoisomerization_two_state(nq=16, n_p=16, depth=2, n_matsubara=1)
        m["periodic_q"] = 1
    O = oracle.Oracle(m)
    W = qi.random_state(m, hermitian=True, zero_p_edges=2)
    L = O.rhs(W)
    tr = sum(L[0, j, j].sum() for j in range(m["S"]))
    assert abs(tr) < 1e-12 * np.abs(L).sum()
    LH = np.conj(np.swapaxes(L, 1, 2))
    assert _relerr(L, LH) < 1e-13


# ------------------------------------------------------------------------------------------------
# P4: R1(0) = 0 and the closed form of dR1/dt(0)
# ------------------------------------------------------------------------------------------------
def test_linear_response_initial_value_and_slope():
    m = _model()
    O = oracle.Oracle(m)
    rng = np.random.default_rng(3)
    W = np.zeros(O.shape, complex)
    for e in range(O.n_elem):
        blk = np.zeros((m["nq"], m["np"]))
        blk[4:-4, 3:-3] = rng.uniform(0, 1, (m["nq"] - 8, m["np"] - 6))
        W[e, 0, 0] = blk
    X = O.apply_dipole(W, oracle.COMMUTATOR)
    assert abs(O.trace(X)) < 1e-14
    slope = 1j * O.trace(O.rhs(X))
    q = qi.axis(m["nq"], m["q_min"], m["q_max"])
    dU = m["U"][1][1](q) - m["U"][0][0](q)
    expect = 2.0 * (dU * W[0, 0, 0].sum(axis=1)).sum() * O.dq * O.dp
    assert slope.real == pytest.approx(expect, rel=1e-12)
    assert abs(slope.imag) < 1e-12 * abs(expect)


# ------------------------------------------------------------------------------------------------
# P5: identical surfaces -- exact discrete closed form through RK4's amplification polynomial
# ------------------------------------------------------------------------------------------------
def _electronic_liouvillian(H):
    S = H.shape[0]
    I = np.eye(S)
    # d vec(s)/dt = -i (H s - s H), row-major vec
    return -1j * (np.kron(H, I) - np.kron(I, H.T))


def _rk4_poly(A, dt):
    Z = dt * A
    P = np.eye(A.shape[0], dtype=complex)
    term = np.eye(A.shape[0], dtype=complex)
    for k in range(1, 5):
        term = term @ Z / k
        P = P + term
    return P


def _dip(mu, side):
    S = mu.shape[0]
    I = np.eye(S)
    left = np.kron(mu, I)
    right = np.kron(I, mu.T)
    return {oracle.LEFT: left, oracle.RIGHT: right, oracle.COMMUTATOR: left - right}[side]


@pytest.fixture(scope="module")
def identical_surface_case():
    """Periodic q and p make the trace an exact invariant, so the discrete ground problem has an exact
    stationary state; it is reached by propagation (at a larger step, which does not change the null
    vector of the generator) and then used with the response step dt."""
    E, V = 3.0, 0.4
    kw = dict(nq=24, n_p=24, qr=(-9.0, 9.0), pr=(-9.0, 9.0), displacement=0.0, eta=1.0, depth=1, periodic_q=1)
    surf = [[lambda q: 0.5 * q * q, lambda q: V + 0 * q], [lambda q: V + 0 * q, lambda q: 0.5 * q * q + E]]
    m_eq = _model(dt=0.04, **kw)
    m_eq["U"] = surf
    Weq, res = oracle.Oracle(m_eq).equilibrate(5000)
    m = _model(dt=0.02, **kw)
    m["U"] = surf
    O = oracle.Oracle(m)
    H = np.array([[0.0, V], [V, E]])
    return m, O, Weq, res, H


def test_identical_surfaces_linear_response(identical_surface_case):
    m, O, Weq, res, H = identical_surface_case
    assert res < 1e-10
    n = 150
    R1 = O.linear_response(Weq, n)
    mu = m["mu"]
    P = _rk4_poly(_electronic_liouvillian(H), m["dt"])
    s0 = np.zeros(4, complex)
    s0[0] = 1.0
    x = _dip(mu, oracle.COMMUTATOR) @ s0
    trW = Weq[0, 0, 0].sum() * O.dq * O.dp
    ref = []
    for _ in range(n + 1):
        ref.append(1j * (mu.T.reshape(-1) @ x) * trW)
        x = P @ x
    assert _relerr(R1, np.array(ref)) < 1e-10


def test_identical_surfaces_third_order_response(identical_surface_case):
    """Covers the t1-stride / t2-fork / t3 bookkeeping of the third-order protocol."""
    m, O, Weq, res, H = identical_surface_case
    n_t1, stride, t2s, n_t3 = 3, 4, [0, 5, 9], 12
    R3 = O.third_order_response(Weq, n_t1, stride, t2s, n_t3)
    P = _rk4_poly(_electronic_liouvillian(H), m["dt"])
    D = _dip(m["mu"], oracle.COMMUTATOR)
    mu_row = m["mu"].T.reshape(-1)
    trW = Weq[0, 0, 0].sum() * O.dq * O.dp
    s0 = np.zeros(4, complex)
    s0[0] = 1
    Pn = lambda k: np.linalg.matrix_power(P, k)
    ref = np.zeros_like(R3)
    for b, t2 in enumerate(t2s):
        for a in range(n_t1):
            x = D @ Pn(t2) @ D @ Pn(a * stride) @ D @ s0
            for c in range(n_t3 + 1):
                ref[b, a, c] = (1j) ** 3 * (mu_row @ Pn(c) @ x) * trW
    assert _relerr(R3, ref) < 1e-10


# ------------------------------------------------------------------------------------------------
# P6: harmonic single-state equilibrium (classical Boltzmann variances at high temperature)
# ------------------------------------------------------------------------------------------------
@pytest.mark.slow
def test_harmonic_equilibrium_variances():
    beta = 0.48
    m = qi.single_state(lambda q: 0.5 * q * q, nq=48, n_p=48, qr=(-10.0, 10.0), pr=(-10.0, 10.0),
                        beta=beta, eta=1.0, gamma=2.0, depth=4, closure=1, dt=0.02)
    O = oracle.Oracle(m)
    Weq, res = O.equilibrate(2500)
    q = qi.axis(m["nq"], m["q_min"], m["q_max"])
    p = qi.axis(m["np"], m["p_min"], m["p_max"])
    W = Weq[0, 0, 0].real
    Z = W.sum()
    q2 = (W * q[:, None] ** 2).sum() / Z
    p2 = (W * p[None, :] ** 2).sum() / Z
    assert q2 == pytest.approx(1 / beta, rel=2e-3)
    assert p2 == pytest.approx(1 / beta, rel=2e-3)


# ------------------------------------------------------------------------------------------------
# P8: independent method -- density-matrix HEOM in a truncated harmonic-oscillator basis
# ------------------------------------------------------------------------------------------------
class _HOBasisHEOM:
    """The same hierarchy (Eq. (heom), linear coupling, Eq. (GMFP) terminator) written for density
    matrices: Phi rho = i[q, rho], Lambda rho = -(1/2){p, rho}, with q, p in an n_v-level
    oscillator basis (omega = 1) tensored with the electronic states."""

    def __init__(self, S, n_v, d, E, V, co, depth, mu):
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
                    H[j * n_v:(j + 1) * n_v, k * n_v:(k + 1) * n_v] = V[j][k] * Iv
        self.H = H
        self.Q = np.kron(Ie, q)
        self.P = np.kron(Ie, p)
        self.mu = np.kron(mu, Iv)
        self.co = co
        self.depth = depth
        self.S, self.n_v = S, n_v

    def rhs(self, R):
        g, r, c = self.co["gamma"][0], self.co["r"][0], self.co["c"][0]
        H, Q, P = self.H, self.Q, self.P
        phi = lambda X: 1j * (Q @ X - X @ Q)
        lam = lambda X: -0.5 * (P @ X + X @ P)
        out = []
        N = self.depth
        for n in range(N + 1):
            X = R[n]
            d = -1j * (H @ X - X @ H) - n * g * X
            if n < N:
                d = d - phi(R[n + 1])
            else:
                d = d + phi(r * lam(X) + c * phi(X))
            if n > 0:
                d = d - n * g * (r * lam(R[n - 1]) + c * phi(R[n - 1]))
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


@functools.lru_cache(maxsize=1)
def _vib_case():
    """The two-state model shared by the comparisons with the vibrational-basis hierarchy (displaced
    harmonic diabats, coupling 0.3, beta = 1, zeta = 0.3, gamma = 1, depth 3, 48 x 48 grid) with its
    equilibrium in both representations: the oracle's (4000 RK4 steps from the Boltzmann start) and the
    density-matrix one (the canonical state relaxed by the ground-state hierarchy, 2000 steps of 0.02).
    Returns (model, oracle, bath coefficients, W_eq, rho_eq tiers, d, E, V, depth, n_v)."""
    beta, eta, gamma, depth = 1.0, 0.3, 1.0, 3
    d, E, V = [0.0, 1.0], [0.0, 2.0], [[0, 0.3], [0.3, 0]]
    m = _model(nq=48, n_p=48, qr=(-8.0, 8.0), pr=(-8.0, 8.0), displacement=d[1], gap=E[1], coupling=0.3,
               eta=eta, gamma=gamma, beta=beta, depth=depth, dt=0.01)
    O = oracle.Oracle(m)
    co = O.coefficients()
    Weq, _ = O.equilibrate(4000)
    Weq.setflags(write=False)
    n_v = 36
    B1 = _HOBasisHEOM(1, n_v, [0.0], [0.0], [[0]], co, depth, np.array([[1.0]]))
    rho0 = np.zeros((depth + 1, n_v, n_v), complex)
    w, U = np.linalg.eigh(B1.H)
    th = U @ np.diag(np.exp(-beta * w)) @ U.conj().T
    rho0[0] = th / np.trace(th)
    rho_eq = B1.rk4(rho0, 0.02, 2000)
    rho_eq.setflags(write=False)
    return m, O, co, Weq, rho_eq, d, E, V, depth, n_v


@pytest.mark.slow
def test_linear_response_against_vibrational_basis_heom():
    m, O, co, Weq, rho_eq, d, E, V, depth, n_v = _vib_case()
    n_t = 400
    R1_w = O.linear_response(Weq, n_t)

    mu = m["mu"]
    B = _HOBasisHEOM(2, n_v, d, E, V, co, depth, mu)
    R = np.zeros((depth + 1, 2 * n_v, 2 * n_v), complex)
    R[:, :n_v, :n_v] = rho_eq
    R = np.array([B.mu @ X - X @ B.mu for X in R])
    R1_h = [1j * np.trace(B.mu @ R[0])]
    for _ in range(n_t):
        R = B.rk4(R, m["dt"], 1)
        R1_h.append(1j * np.trace(B.mu @ R[0]))
    R1_h = np.array(R1_h)
    # both truncations (48x48 phase-space grid vs 36 vibrational levels) leave ~5e-4
    assert _relerr(R1_w, R1_h) < 1e-3


# ------------------------------------------------------------------------------------------------
# P11: depth 0 with the terminator is the multi-state quantum Fokker-Planck equation, Eq. (heomW)
# ------------------------------------------------------------------------------------------------
def test_depth_zero_terminator_is_quantum_fokker_planck():
    m = _model(depth=0)
    O = oracle.Oracle(m)
    W = qi.random_state(m)
    zeta, beta = m["eta"], m["beta"]
    p = qi.axis(m["np"], m["p_min"], m["p_max"])
    dp = O.dp
    # zeta d/dp (p W + (1/beta) dW/dp) with 4th-order central differences on the periodic p axis
    d1 = np.array([1, -8, 0, 8, -1]) / (12 * dp)
    d2 = np.array([-1, 16, -30, 16, -1]) / (12 * dp * dp)

    def conv(x, c):
        return sum(c[t] * np.roll(x, 2 - t, axis=-1) for t in range(5))

    fp = zeta * conv(p * W, d1) + (zeta / beta) * conv(W, d2)
    ref = O.rhs(W, oracle.KINETIC | oracle.POTENTIAL) + fp
    assert _relerr(O.rhs(W), ref) < 1e-13


# ------------------------------------------------------------------------------------------------
# Bath coefficients against direct quadrature of Eqs. (bath-response), (bath-correlation)
# ------------------------------------------------------------------------------------------------
@pytest.mark.parametrize("beta,gamma", [(0.48, 1.0), (1.0, 2.0), (2.0, 1.0)])
def test_bath_coefficients_reproduce_correlation_functions(beta, gamma):
    from scipy.integrate import quad
    eta, K = 0.7, 400
    g = np.zeros(K + 1); r = np.zeros(K + 1); c = np.zeros(K + 1); cd = np.zeros(1)
    import ctypes
    dp = ctypes.POINTER(ctypes.c_double)
    oracle.lib().oq_bath_coefficients(eta, gamma, beta, K, 0, 1, g.ctypes.data_as(dp), r.ctypes.data_as(dp),
                                      c.ctypes.data_as(dp), cd.ctypes.data_as(dp))
    J_over_w = lambda w: (eta / math.pi) * gamma ** 2 / (gamma ** 2 + w ** 2)
    w_coth = lambda w: w / math.tanh(beta * w / 2) if w > 1e-12 else 2.0 / beta
    for t in (0.3, 1.0, 2.5):
        psi = 2 * quad(J_over_w, 0, np.inf, weight="cos", wvar=t)[0]
        assert sum(r * g * np.exp(-g * t)) == pytest.approx(psi, rel=1e-8)
        C = quad(lambda w: J_over_w(w) * w_coth(w), 0, np.inf, weight="cos", wvar=t, limlst=200)[0]
        assert sum(c * g * np.exp(-g * t)) == pytest.approx(C, rel=1e-6, abs=1e-9)
    # the delta-term carries the neglected Matsubara weight, which vanishes as K grows
    assert abs(cd[0]) < 2 * eta * gamma ** 2 * beta / (4 * math.pi ** 2 * K)
    # high-temperature limit of the zeroth coefficient (end of Sec. II)
    oracle.lib().oq_bath_coefficients(eta, gamma, 1e-4, 0, 0, 0, g.ctypes.data_as(dp), r.ctypes.data_as(dp),
                                      c.ctypes.data_as(dp), cd.ctypes.data_as(dp))
    assert c[0] == pytest.approx(eta / 1e-4, rel=1e-6)


def test_hierarchy_size_and_neighbours():
    for K, N in [(0, 3), (2, 8), (2, 10), (3, 10)]:
        n = oracle.lib().oq_hierarchy(K + 1, N, None)
        assert n == math.comb(N + K + 1, K + 1)
    m = qi.photoisomerization_two_state(nq=4, n_p=8, depth=4, n_matsubara=2)
    O = oracle.Oracle(m)
    h = O.hierarchy()
    assert len({tuple(x) for x in h}) == len(h)
    assert (h.sum(axis=1) <= 4).all() and (np.diff(h.sum(axis=1)) >= 0).all()


# ------------------------------------------------------------------------------------------------
# P9 / P10: spectra identities and pathway additivity
# ------------------------------------------------------------------------------------------------
def test_transient_absorption_two_definitions():
    """w int dw1 I_corr(w, T, w1) over one w1 period equals 2 pi times Eq. (transient-absorption)."""
    rng = np.random.default_rng(5)
    n1, n3, dt1, dt3 = 9, 40, 0.08, 0.01
    R3 = rng.normal(size=(n1, n3 + 1)) + 1j * rng.normal(size=(n1, n3 + 1))
    om = np.linspace(-20, 20, 33)
    a = oracle.transient_absorption_from_corr(R3, dt1, dt3, om, n_omega1=16)
    b = oracle.transient_absorption(R3[0][None, :], dt3, om)[0]
    assert _relerr(a, 2 * math.pi * b) < 1e-12


def test_absorption_of_damped_oscillation():
    """Trapezoid transform of R1 = 2 sin(Et) exp(-G t) against the closed-form Laplace transform."""
    E, G, dt, n = 5.0, 0.5, 1e-3, 60000
    t = np.arange(n + 1) * dt
    R1 = 2 * np.sin(E * t) * np.exp(-G * t)
    om = np.linspace(-10, 10, 41)
    got = oracle.absorption(R1, dt, om)
    ft = -1j * (1 / (G - 1j * (om + E)) - 1 / (G - 1j * (om - E)))
    assert np.allclose(got, om * ft.imag, atol=2e-5)


def test_pathway_split_is_additive():
    m = _model(nq=16, n_p=16, depth=1)
    O = oracle.Oracle(m)
    Weq, _ = O.equilibrate(50)
    args = (2, 3, [0, 4], 6)
    full = O.third_order_response(Weq, *args, first=oracle.COMMUTATOR)
    ket = O.third_order_response(Weq, *args, first=oracle.LEFT)
    bra = O.third_order_response(Weq, *args, first=oracle.RIGHT)
    assert _relerr(ket + bra, full) < 1e-13
    assert np.abs(ket).max() > 1e-3 and np.abs(bra).max() > 1e-3


# ------------------------------------------------------------------------------------------------
# The paper's printed model parameters pin the reading of its Morse surfaces
# ------------------------------------------------------------------------------------------------
def test_morse_reading_reproduces_printed_resonances():
    vals = {}
    with open(os.path.join(GOLDEN, "morse_resonances.txt")) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                k, v = line.split()
                vals[k] = float(v)
    m = qi.morse_photoisomerization()
    q0, q1 = m["q_minima"]
    U00, U11 = m["U"][0][0], m["U"][1][1]
    scale = vals["omega0"]
    nu0 = (U11(q0) - U00(q0)) * scale
    nu1 = (U00(q1) - U11(q1)) * scale
    assert nu0 == pytest.approx(vals["nu0"], rel=1e-3)
    assert nu1 == pytest.approx(vals["nu1"], rel=1e-3)


def test_rhs_rows_equal_the_full_rhs():
    """The sampled-rows entry (used at full problem sizes) returns exactly the rows of the full RHS."""
    for m in (qi.three_state(nq=12, n_p=16, depth=2, n_matsubara=1), qi.harmonic_two_state(nq=16, n_p=16, depth=3)):
        O = oracle.Oracle(m)
        W = qi.random_state(m, seed=77)
        full = O.rhs(W)
        S, nq = m["S"], m["nq"]
        rng = np.random.default_rng(5)
        rows = [(int(rng.integers(full.shape[0])), int(rng.integers(S)), int(rng.integers(S)), int(i))
                for i in (0, 1, nq - 1, nq // 2, 3)]
        got = O.rhs_rows(W, rows)
        for r, (e, j, k, i) in enumerate(rows):
            assert np.array_equal(got[r], full[e, j, k, i])
    with pytest.raises(ValueError):
        O.rhs_rows(W, [(0, 0, 0, nq)])


# ------------------------------------------------------------------------------------------------
# Brownian-oscillator absorption: displaced harmonic surfaces without diabatic coupling, Drude bath
# at high temperature (the K = 0 coefficients of Sec. II), R1 of Eq. (R1)
# ------------------------------------------------------------------------------------------------
def _brownian_oscillator_r1(d, gap, zeta, gamma, beta, t):
    """Closed form (hbar = m = omega_0 = 1).  The energy gap U_1 - U_0 = gap + d^2/2 - d q is linear in
    q and the dynamics is Gaussian, so the second-order cumulant is exact:
        R1(t) = i (K - K*),  K(t) = Tr{e^{i H_0 t} e^{-i H_1 t} rho_eq} = exp(-i (gap + d^2/2) t - g(t)),
        g(t) = int_0^t (t - s) C(s) ds,  C(s) = d^2 [C_sym(s) - (i/2) chi(s)],
    with chi the response of q to a unit momentum kick and C_sym the symmetrised q correlation of the
    oscillator under Drude friction (memory zeta gamma e^{-gamma t}) and the bath force of the high-
    temperature reading, <F(t) F(0)> = (zeta/beta) gamma e^{-gamma |t|}.  Both follow from the linear
    Markovian embedding x = (q, p, z, F): q' = p, p' = -q - z + F, z' = zeta gamma p - gamma z,
    F' = -gamma F + noise, whose stationary covariance solves a Lyapunov equation."""
    from scipy.integrate import cumulative_trapezoid
    from scipy.linalg import expm, solve_continuous_lyapunov
    A = np.array([[0.0, 1.0, 0.0, 0.0], [-1.0, 0.0, -1.0, 1.0], [0.0, zeta * gamma, -gamma, 0.0],
                  [0.0, 0.0, 0.0, -gamma]])
    noise = np.zeros((4, 4))
    noise[3, 3] = 2.0 * (zeta / beta) * gamma ** 2
    Sig = solve_continuous_lyapunov(A, -noise)
    tf = np.linspace(0.0, t[-1], 20001)
    Eh, E3h = expm(A * (tf[1] - tf[0])), expm(A[:3, :3] * (tf[1] - tf[0]))
    M, R = Sig.copy(), np.eye(3)
    csym, chi = np.empty(len(tf)), np.empty(len(tf))
    for k in range(len(tf)):
        csym[k], chi[k] = M[0, 0], R[0, 1]
        M, R = Eh @ M, E3h @ R
    C = d * d * (csym - 0.5j * chi)
    g = cumulative_trapezoid(cumulative_trapezoid(C, tf, initial=0.0), tf, initial=0.0)
    gt = np.interp(t, tf, g.real) + 1j * np.interp(t, tf, g.imag)
    K = np.exp(-1j * (gap + 0.5 * d * d) * t - gt)
    return 1j * (K - np.conj(K)), Sig[0, 0]


def test_brownian_oscillator_absorption_closed_form():
    # small displacement and 15 time units, so that the vibrational recurrences and their damping by
    # the bath shape R1: the closed form with zeta or gamma off by 10-20 % is 1.5e-2 - 2.6e-2 away,
    # without the bath 0.87 away
    d, gap, zeta, gamma, beta = 0.5, 10.0, 1.0, 1.0, 0.48
    m = _model(nq=32, n_p=32, coupling=0.0, displacement=d, gap=gap, eta=zeta, gamma=gamma, beta=beta,
               depth=4, dt=0.01)
    O = oracle.Oracle(m)
    W_eq, _ = O.equilibrate(3000)
    n_t = 1500
    R1 = O.linear_response(W_eq, n_t)
    ref, q_var = _brownian_oscillator_r1(d, gap, zeta, gamma, beta, np.arange(n_t + 1) * m["dt"])
    assert abs(q_var - 1.0 / beta) < 1e-9  # the high-temperature reading: classical <q^2> = 1 / beta
    assert _relerr(R1, ref) < 1e-3  # measured 1.1e-4


@pytest.mark.slow
def test_third_order_response_against_vibrational_basis_heom():
    """Eq. (R3), R3 = i^3 Tr{mu G(t3) mu^x G(t2) mu^x G(t1) mu^x W_eq}, against the same hierarchy written
    for density matrices in a truncated vibrational basis (an independent method), on a small
    schedule: two t1 delays, two waiting times, 100 t3 steps."""
    m, O, co, Weq, rho_eq, d, E, V, depth, n_v = _vib_case()
    n_t1, stride, t2_steps, n_t3 = 2, 20, [0, 30], 100
    R3_w = O.third_order_response(Weq, n_t1, stride, t2_steps, n_t3)

    B = _HOBasisHEOM(2, n_v, d, E, V, co, depth, m["mu"])
    comm = lambda R: np.array([B.mu @ X - X @ B.mu for X in R])
    R = np.zeros((depth + 1, 2 * n_v, 2 * n_v), complex)
    R[:, :n_v, :n_v] = rho_eq
    R = comm(R)
    R3_h = np.zeros((len(t2_steps), n_t1, n_t3 + 1), complex)
    for a in range(n_t1):
        if a > 0:
            R = B.rk4(R, m["dt"], stride)
        X = comm(R)
        done = 0
        for b, t2 in enumerate(t2_steps):
            if t2 > done:
                X = B.rk4(X, m["dt"], t2 - done)
                done = t2
            Y = comm(X)
            R3_h[b, a, 0] = (1j) ** 3 * np.trace(B.mu @ Y[0])
            for c in range(1, n_t3 + 1):
                Y = B.rk4(Y, m["dt"], 1)
                R3_h[b, a, c] = (1j) ** 3 * np.trace(B.mu @ Y[0])
    # the two truncations (48 x 48 phase-space grid vs 36 vibrational levels): measured 4.3e-5
    assert _relerr(R3_w, R3_h) < 5e-4


@pytest.mark.slow
def test_noncondon_linear_response_against_vibrational_basis_heom():
    """A coordinate-dependent transition dipole mu_01(q) = 1 + s q (Sec. III: the dipole operators then
    act as p-convolutions in the Wigner representation) against the vibrational-basis hierarchy, where
    mu(q) is simply the operator 1 + s q."""
    from oracle import noncondon as nc
    s = 0.2
    m, O, co, Weq, rho_eq, d, E, V, depth, n_v = _vib_case()
    n_t = 400
    R1_w = nc.linear_response(O, Weq, qi.function_table(m, qi.linear_dipole(m, slope=s)), n_t)

    B = _HOBasisHEOM(2, n_v, d, E, V, co, depth, m["mu"])
    q = B.Q[:n_v, :n_v]
    B.mu = np.kron(np.asarray(m["mu"], dtype=float), np.eye(n_v) + s * q)
    R = np.zeros((depth + 1, 2 * n_v, 2 * n_v), complex)
    R[:, :n_v, :n_v] = rho_eq
    R = np.array([B.mu @ X - X @ B.mu for X in R])
    R1_h = [1j * np.trace(B.mu @ R[0])]
    for _ in range(n_t):
        R = B.rk4(R, m["dt"], 1)
        R1_h.append(1j * np.trace(B.mu @ R[0]))
    R1_h = np.array(R1_h)
    err = _relerr(R1_w, R1_h)
    assert err < 1e-3  # measured 6.1e-4: the two truncations, as for the Condon R1
    # and the coordinate dependence matters at this size: the Condon response is far away
    assert _relerr(O.linear_response(Weq, n_t), R1_h) > 20 * err


@pytest.mark.slow
def test_adiabatic_marginals_against_vibrational_basis_heom():
    """Adiabatic-basis coordinate distributions (Sec. III, wavepacket dynamics) after a ket-side
    excitation and 2 time units of propagation, against the vibrational-basis hierarchy: there the
    diabatic density rho_jk(q, q) = sum_mn phi_m(q) rho_jk,mn phi_n(q) with the oscillator
    eigenfunctions phi_n, rotated by the eigenvectors of the diabatic matrix U(q) (ascending
    eigenvalue, first largest-magnitude component positive)."""
    from oracle import marginals as mg
    m, O, co, Weq, rho_eq, d, E, V, depth, n_v = _vib_case()
    n_t = 200
    W, _ = O.step(O.apply_dipole(Weq, oracle.LEFT), n_t)
    dp = (m["p_max"] - m["p_min"]) / m["np"]
    P_w = mg.adiabatic_marginals(W, qi.u_table(m), dp)

    B = _HOBasisHEOM(2, n_v, d, E, V, co, depth, m["mu"])
    R = np.zeros((depth + 1, 2 * n_v, 2 * n_v), complex)
    R[:, :n_v, :n_v] = rho_eq
    R = np.array([B.mu @ X for X in R])
    R = B.rk4(R, m["dt"], n_t)
    q = qi.axis(m["nq"], m["q_min"], m["q_max"])
    # oscillator eigenfunctions by the three-term recurrence
    phi = np.zeros((n_v, len(q)))
    phi[0] = np.pi ** -0.25 * np.exp(-0.5 * q * q)
    phi[1] = math.sqrt(2.0) * q * phi[0]
    for n in range(2, n_v):
        phi[n] = math.sqrt(2.0 / n) * q * phi[n - 1] - math.sqrt((n - 1) / n) * phi[n - 2]
    S = 2
    rho_q = np.zeros((S, S, len(q)), complex)
    for j in range(S):
        for k in range(S):
            blk = R[0][j * n_v:(j + 1) * n_v, k * n_v:(k + 1) * n_v]
            rho_q[j, k] = np.einsum("mi,mn,ni->i", phi, blk, phi)
    P_h = np.zeros_like(rho_q)
    for i, x in enumerate(q):
        Umat = np.array([[m["U"][j][k](x) for k in range(S)] for j in range(S)], dtype=float)
        _, vec = np.linalg.eigh(Umat)
        for a in range(S):
            lead = int(np.argmax(np.abs(vec[:, a]) >= np.abs(vec[:, a]).max() - 1e-9))
            if vec[lead, a] < 0:
                vec[:, a] = -vec[:, a]
        P_h[:, :, i] = vec.T @ rho_q[:, :, i] @ vec
    # measured 2.5e-3, limited by the phase-space grid (7.3e-4 on 64 x 64; 48 instead of 36
    # vibrational levels change nothing)
    assert _relerr(P_w, P_h) < 4e-3


@pytest.mark.slow
def test_first_order_distribution_marginals_against_vibrational_basis_heom():
    """The frequency-domain first-order distribution W'(omega_1) of Sec. III (trapezoid Fourier sums of
    the t1 propagation after mu^x, then i [mu^-> F(omega) - mu^<- F(-omega)]), integrated over p, against
    the same construction for density matrices in the vibrational basis, in position representation."""
    m, O, co, Weq, rho_eq, d, E, V, depth, n_v = _vib_case()
    n_t1, stride, omega = 6, 10, np.array([2.0, -2.0, 2.6])
    Wp = O.first_order_distribution(Weq, n_t1, stride, omega)
    dp = (m["p_max"] - m["p_min"]) / m["np"]
    marg_w = Wp[:, 0].sum(axis=-1) * dp  # [omega][S][S][nq]

    B = _HOBasisHEOM(2, n_v, d, E, V, co, depth, m["mu"])
    R = np.zeros((depth + 1, 2 * n_v, 2 * n_v), complex)
    R[:, :n_v, :n_v] = rho_eq
    X = np.array([B.mu @ Y - Y @ B.mu for Y in R])
    dt1 = stride * m["dt"]
    Fp = np.zeros((len(omega), 2 * n_v, 2 * n_v), complex)
    Fm = np.zeros_like(Fp)
    for a in range(n_t1):
        if a > 0:
            X = B.rk4(X, m["dt"], stride)
        wgt = dt1 * (0.5 if a in (0, n_t1 - 1) else 1.0)  # trapezoid rule on t1 = 0 .. (n_t1 - 1) dt1
        for k, om in enumerate(omega):
            Fp[k] += wgt * np.exp(1j * om * a * dt1) * X[0]
            Fm[k] += wgt * np.exp(-1j * om * a * dt1) * X[0]
    q = qi.axis(m["nq"], m["q_min"], m["q_max"])
    phi = np.zeros((n_v, len(q)))
    phi[0] = np.pi ** -0.25 * np.exp(-0.5 * q * q)
    phi[1] = math.sqrt(2.0) * q * phi[0]
    for n in range(2, n_v):
        phi[n] = math.sqrt(2.0 / n) * q * phi[n - 1] - math.sqrt((n - 1) / n) * phi[n - 2]
    for k in range(len(omega)):
        Wk = 1j * (B.mu @ Fp[k] - Fm[k] @ B.mu)
        marg_h = np.array([[np.einsum("mi,mn,ni->i", phi, Wk[j * n_v:(j + 1) * n_v, l * n_v:(l + 1) * n_v], phi)
                            for l in range(2)] for j in range(2)])
        assert _relerr(marg_w[k], marg_h) < 2e-3, omega[k]  # measured 4.9e-4 at each omega


@pytest.mark.slow
def test_three_state_linear_response_against_vibrational_basis_heom():
    """Three displaced harmonic diabats with pairwise constant couplings (the S x S mixing of the
    potential kernel with S = 3) and mu_0j = mu_j0 = 1: R1 against the vibrational-basis hierarchy."""
    beta, eta, gamma, depth = 1.0, 0.3, 1.0, 3
    d, E = [0.0, 1.0, -0.8], [0.0, 2.0, 2.6]
    V = [[0, 0.2, 0.15], [0.2, 0, 0.3], [0.15, 0.3, 0]]
    U = [[(lambda j: (lambda q: 0.5 * (np.asarray(q) - d[j]) ** 2 + E[j]))(j) if j == k else
          (lambda c: (lambda q: np.full(np.shape(q), float(c))))(V[j][k]) for k in range(3)] for j in range(3)]
    mu = np.array([[0.0, 1.0, 1.0], [1.0, 0.0, 0.0], [1.0, 0.0, 0.0]])
    m = dict(name="harmonic_three_state", S=3, nq=48, np=48, q_min=-8.0, q_max=8.0, p_min=-8.0, p_max=8.0,
             U=U, mu=mu, eta=eta, gamma=gamma, beta=beta, n_matsubara=0, high_temperature=1, use_cdelta=0,
             depth=depth, closure=1, dt=0.01, periodic_q=0)
    O = oracle.Oracle(m, qi.u_table(m))
    co = O.coefficients()
    Weq, _ = O.equilibrate(4000)
    n_t = 400
    R1_w = O.linear_response(Weq, n_t)

    n_v = 30
    B1 = _HOBasisHEOM(1, n_v, [0.0], [0.0], [[0]], co, depth, np.array([[1.0]]))
    rho0 = np.zeros((depth + 1, n_v, n_v), complex)
    w, Uv = np.linalg.eigh(B1.H)
    th = Uv @ np.diag(np.exp(-beta * w)) @ Uv.conj().T
    rho0[0] = th / np.trace(th)
    rho_eq = B1.rk4(rho0, 0.02, 2000)
    B = _HOBasisHEOM(3, n_v, d, E, V, co, depth, mu)
    R = np.zeros((depth + 1, 3 * n_v, 3 * n_v), complex)
    R[:, :n_v, :n_v] = rho_eq
    R = np.array([B.mu @ X - X @ B.mu for X in R])
    R1_h = [1j * np.trace(B.mu @ R[0])]
    for _ in range(n_t):
        R = B.rk4(R, m["dt"], 1)
        R1_h.append(1j * np.trace(B.mu @ R[0]))
    assert _relerr(R1_w, np.array(R1_h)) < 1e-3  # measured 1.7e-4


class _HOBasisMultiModeHEOM:
    """The hierarchy of Eq. (heom) with several bath modes k = 0..K (multi-indices |n| <= N, truncation
    at the top) and the delta-term, for density matrices in an n_v-level oscillator basis: Phi rho =
    i[q, rho], Lambda rho = -(1/2){p, rho}; d rho_n = -i[H, rho_n] - sum_k n_k gamma_k rho_n
    + c_delta Phi^2 rho_n - sum_k Phi rho_{n+e_k} - sum_k n_k gamma_k (r_k Lambda + c_k Phi) rho_{n-e_k}."""

    def __init__(self, base, co, depth):
        self.H, self.Q, self.P = base.H, base.Q, base.P
        self.co = co
        K1 = len(co["gamma"])
        self.idx = [n for n in itertools.product(range(depth + 1), repeat=K1) if sum(n) <= depth]
        self.pos = {n: a for a, n in enumerate(self.idx)}

    def rhs(self, R):
        H, Q, P, co = self.H, self.Q, self.P, self.co
        phi = lambda X: 1j * (Q @ X - X @ Q)
        lam = lambda X: -0.5 * (P @ X + X @ P)
        out = np.zeros_like(R)
        for a, n in enumerate(self.idx):
            X = R[a]
            d = -1j * (H @ X - X @ H) - sum(nk * g for nk, g in zip(n, co["gamma"])) * X
            d = d + co["cdelta"] * phi(phi(X))
            for k in range(len(n)):
                up = tuple(n[j] + (j == k) for j in range(len(n)))
                if up in self.pos:
                    d = d - phi(R[self.pos[up]])
                if n[k] > 0:
                    dn = tuple(n[j] - (j == k) for j in range(len(n)))
                    Y = R[self.pos[dn]]
                    d = d - n[k] * co["gamma"][k] * (co["r"][k] * lam(Y) + co["c"][k] * phi(Y))
            out[a] = d
        return out

    def rk4(self, R, dt, n):
        for _ in range(n):
            k1 = self.rhs(R)
            k2 = self.rhs(R + 0.5 * dt * k1)
            k3 = self.rhs(R + 0.5 * dt * k2)
            k4 = self.rhs(R + dt * k3)
            R = R + dt / 6 * (k1 + 2 * k2 + 2 * k3 + k4)
        return R


@pytest.mark.slow
def test_matsubara_linear_response_against_vibrational_basis_heom():
    """Low temperature: the Drude mode plus one Matsubara mode and the delta-term (Eqs. (bath-response),
    (bath-correlation) with K = 1), truncated at depth 3: R1 against the multi-mode vibrational-basis
    hierarchy."""
    beta, eta, gamma, depth = 2.0, 0.3, 1.0, 3
    d, E, V = [0.0, 1.0], [0.0, 2.0], [[0, 0.3], [0.3, 0]]
    m = _model(nq=48, n_p=48, qr=(-8.0, 8.0), pr=(-8.0, 8.0), displacement=d[1], gap=E[1], coupling=0.3,
               eta=eta, gamma=gamma, beta=beta, depth=depth, closure=0, dt=0.01)
    m.update(n_matsubara=1, high_temperature=0, use_cdelta=1)
    O = oracle.Oracle(m)
    co = O.coefficients()
    assert len(co["gamma"]) == 2 and co["cdelta"] != 0.0
    Weq, _ = O.equilibrate(4000)
    n_t = 250
    R1_w = O.linear_response(Weq, n_t)

    n_v = 24
    g1 = _HOBasisMultiModeHEOM(_HOBasisHEOM(1, n_v, [0.0], [0.0], [[0]], co, depth, np.array([[1.0]])), co, depth)
    rho0 = np.zeros((len(g1.idx), n_v, n_v), complex)
    w, U = np.linalg.eigh(g1.H)
    th = U @ np.diag(np.exp(-beta * w)) @ U.conj().T
    rho0[0] = th / np.trace(th)
    rho_eq = g1.rk4(rho0, 0.02, 2000)
    base = _HOBasisHEOM(2, n_v, d, E, V, co, depth, m["mu"])
    g2 = _HOBasisMultiModeHEOM(base, co, depth)
    assert g2.idx == g1.idx and g2.idx[0] == (0, 0)
    R = np.zeros((len(g2.idx), 2 * n_v, 2 * n_v), complex)
    R[:, :n_v, :n_v] = rho_eq
    R = np.array([base.mu @ X - X @ base.mu for X in R])
    R1_h = [1j * np.trace(base.mu @ R[0])]
    for _ in range(n_t):
        R = g2.rk4(R, m["dt"], 1)
        R1_h.append(1j * np.trace(base.mu @ R[0]))
    assert _relerr(R1_w, np.array(R1_h)) < 1e-3  # measured 2.9e-4


@pytest.mark.slow
def test_noncondon_third_order_response_against_vibrational_basis_heom():
    """Eq. (R3) with the coordinate-dependent dipole mu_01(q) = 1 + 0.2 q in all three interactions and
    the trace, against the vibrational-basis hierarchy with the dipole operator 1 + 0.2 q."""
    from oracle import noncondon as nc
    s = 0.2
    m, O, co, Weq, rho_eq, d, E, V, depth, n_v = _vib_case()
    n_t1, stride, t2_steps, n_t3 = 2, 20, [0, 30], 60
    T = qi.function_table(m, qi.linear_dipole(m, slope=s))
    R3_w = nc.third_order_response(O, Weq, T, n_t1, stride, t2_steps, n_t3)

    B = _HOBasisHEOM(2, n_v, d, E, V, co, depth, m["mu"])
    B.mu = np.kron(np.asarray(m["mu"], dtype=float), np.eye(n_v) + s * B.Q[:n_v, :n_v])
    comm = lambda R: np.array([B.mu @ X - X @ B.mu for X in R])
    R = np.zeros((depth + 1, 2 * n_v, 2 * n_v), complex)
    R[:, :n_v, :n_v] = rho_eq
    R = comm(R)
    R3_h = np.zeros((len(t2_steps), n_t1, n_t3 + 1), complex)
    for a in range(n_t1):
        if a > 0:
            R = B.rk4(R, m["dt"], stride)
        X = comm(R)
        done = 0
        for b, t2 in enumerate(t2_steps):
            if t2 > done:
                X = B.rk4(X, m["dt"], t2 - done)
                done = t2
            Y = comm(X)
            R3_h[b, a, 0] = (1j) ** 3 * np.trace(B.mu @ Y[0])
            for c in range(1, n_t3 + 1):
                Y = B.rk4(Y, m["dt"], 1)
                R3_h[b, a, c] = (1j) ** 3 * np.trace(B.mu @ Y[0])
    err = _relerr(R3_w, R3_h)
    assert err < 5e-4  # measured 2.0e-5
    # the coordinate dependence matters here: the Condon R3 is 7.4e-2 away
    assert _relerr(O.third_order_response(Weq, n_t1, stride, t2_steps, n_t3), R3_h) > 100 * err
