"""Seeded synthetic inputs for the multi-state QHFPE workloads.

This module holds model definitions (diabatic surfaces, dipole matrices, bath and grid parameters of
the synthetic workloads shaped like those of Ikeda & Tanimura 2017, Sec. III) and seeded random states.
It holds none of the method's arithmetic: no right-hand side, no bath coefficients, no transforms.
Both the CUDA library's tests/benchmark and the CPU oracle take their inputs from here.

Potential tables follow the documented input contract of the library (and of the oracle): for a
p-grid of np points with spacing dp = (p_max - p_min)/np, the half-offsets are
    s_t = (t - np/2) * pi / (np * dp),   t = 0 .. np,
and the caller supplies T_jk[i][t] = U_jk(q_i + s_t) with q_i = q_min + i*(q_max - q_min)/nq.
"""
import math

import numpy as np

SEED = 1706


def axis(n, lo, hi):
    return lo + np.arange(n, dtype=np.float64) * ((hi - lo) / n)


def half_offsets(n_p, p_min, p_max):
    dp = (p_max - p_min) / n_p
    return (np.arange(n_p + 1, dtype=np.float64) - n_p / 2) * (math.pi / (n_p * dp))


def linear_continuation(f, lo, hi, h=1e-5):
    """f inside [lo, hi]; outside, the tangent line at the nearer edge (limits the stiffness of the
    potential kernel, which samples U up to pi/(2 dp) beyond the box)."""
    flo, fhi = f(lo), f(hi)
    slo = (f(lo + h) - f(lo - h)) / (2 * h)
    shi = (f(hi + h) - f(hi - h)) / (2 * h)

    def g(q):
        q = np.asarray(q, dtype=np.float64)
        out = f(np.clip(q, lo, hi))
        out = np.where(q < lo, flo + slo * (q - lo), out)
        out = np.where(q > hi, fhi + shi * (q - hi), out)
        return out

    return g


def u_table(model):
    """T[j][k][i][t] = U_jk(q_i + s_t), shape [S][S][nq][np+1], float64."""
    S, nq, n_p = model["S"], model["nq"], model["np"]
    q = axis(nq, model["q_min"], model["q_max"])
    s = half_offsets(n_p, model["p_min"], model["p_max"])
    pts = q[:, None] + s[None, :]
    T = np.zeros((S, S, nq, n_p + 1), dtype=np.float64)
    for j in range(S):
        for k in range(S):
            f = model["U"][j][k]
            T[j, k] = f(pts) if f is not None else 0.0
    return np.ascontiguousarray(T)


def function_table(model, F):
    """T[j][k][i][t] = F[j][k](q_i + s_t) for an S x S array of functions of q (None: zero), in the
    potential-table convention; used for coordinate-dependent (non-Condon) dipoles."""
    S, nq, n_p = model["S"], model["nq"], model["np"]
    q = axis(nq, model["q_min"], model["q_max"])
    s = half_offsets(n_p, model["p_min"], model["p_max"])
    pts = q[:, None] + s[None, :]
    T = np.zeros((S, S, nq, n_p + 1), dtype=np.float64)
    for j in range(S):
        for k in range(S):
            if F[j][k] is not None:
                T[j, k] = F[j][k](pts)
    return np.ascontiguousarray(T)


def linear_dipole(model, slope=0.1, q_ref=0.0):
    """A coordinate-dependent transition dipole mu_0j(q) = mu_j0(q) = mu_0j * (1 + slope (q - q_ref))
    (a Herzberg-Teller-like linear dependence), zero elsewhere, on the model's Condon matrix."""
    S = model["S"]
    mu = np.asarray(model["mu"], dtype=np.float64)
    F = [[None] * S for _ in range(S)]
    for j in range(S):
        for k in range(S):
            if mu[j, k] != 0.0:
                c = float(mu[j, k])
                F[j][k] = (lambda c: (lambda q: c * (1.0 + slope * (np.asarray(q) - q_ref))))(c)
    return F


def _const(c):
    return lambda q: np.full(np.shape(q), float(c))


def harmonic_two_state(nq=32, n_p=32, qr=(-8.0, 8.0), pr=(-8.0, 8.0), displacement=1.5, gap=10.0,
                       coupling=0.5, eta=0.5, gamma=1.0, beta=0.48, depth=3, closure=1, dt=0.01,
                       periodic_q=0):
    """Two displaced harmonic diabats with constant diabatic coupling, Drude bath at high temperature
    (K = 0).  beta = 0.48 is the paper's beta*hbar*omega_0 at 300 K (Sec. III)."""
    return dict(
        name="harmonic_two_state", S=2, nq=nq, np=n_p, q_min=qr[0], q_max=qr[1], p_min=pr[0], p_max=pr[1],
        U=[[lambda q: 0.5 * q * q, _const(coupling)],
           [_const(coupling), lambda q: 0.5 * (q - displacement) ** 2 + gap]],
        mu=np.array([[0.0, 1.0], [1.0, 0.0]]),
        eta=eta, gamma=gamma, beta=beta, n_matsubara=0, high_temperature=1, use_cdelta=0,
        depth=depth, closure=closure, dt=dt, periodic_q=periodic_q)


def _ground_double_well(q):
    return 5.0 * ((q / 4.0) ** 2 - 1.0) ** 2


def _excited_anharmonic(q):
    x = q - 3.0
    return 0.5 * x * x + 0.01 * x ** 4 - 0.31


def photoisomerization_two_state(nq=96, n_p=128, qr=(-10.0, 10.0), pr=(-16.0, 16.0), coupling=0.5,
                                 eta=1.0, gamma=1.0, beta=1.0, n_matsubara=2, depth=8, dt=1.6e-3):
    """Quartic double-well ground state (barrier 5, wells at +-4) and a displaced anharmonic excited
    well crossing it at q = 0; constant diabatic coupling; Drude bath with K Matsubara terms and the
    delta-term; surfaces continued linearly outside the q box."""
    lo, hi = qr
    return dict(
        name="photoisomerization_two_state", S=2, nq=nq, np=n_p, q_min=lo, q_max=hi, p_min=pr[0], p_max=pr[1],
        U=[[linear_continuation(_ground_double_well, lo, hi), _const(coupling)],
           [_const(coupling), linear_continuation(_excited_anharmonic, lo, hi)]],
        mu=np.array([[0.0, 1.0], [1.0, 0.0]]),
        eta=eta, gamma=gamma, beta=beta, n_matsubara=n_matsubara, high_temperature=0, use_cdelta=1,
        depth=depth, closure=0, dt=dt, periodic_q=0)


def three_state(nq=256, n_p=256, qr=(-10.0, 10.0), pr=(-16.0, 16.0), coupling=0.5, eta=1.0, gamma=2.0,
                beta=0.5, n_matsubara=2, depth=10, dt=6.5e-4):
    """Ground double well plus two excited anharmonic wells (the second shifted by +1 in q and +2 in
    energy) with pairwise couplings forming an avoided crossing; mu_0j = mu_j0 = 1 for the excited
    states and 0 between them."""
    lo, hi = qr
    e2 = lambda q: _excited_anharmonic(q - 1.0) + 2.0
    c = _const(coupling)
    return dict(
        name="three_state", S=3, nq=nq, np=n_p, q_min=lo, q_max=hi, p_min=pr[0], p_max=pr[1],
        U=[[linear_continuation(_ground_double_well, lo, hi), c, c],
           [c, linear_continuation(_excited_anharmonic, lo, hi), c],
           [c, c, linear_continuation(e2, lo, hi)]],
        mu=np.array([[0.0, 1.0, 1.0], [1.0, 0.0, 0.0], [1.0, 0.0, 0.0]]),
        eta=eta, gamma=gamma, beta=beta, n_matsubara=n_matsubara, high_temperature=0, use_cdelta=1,
        depth=depth, closure=0, dt=dt, periodic_q=0)


def single_state(U, nq=32, n_p=32, qr=(-8.0, 8.0), pr=(-8.0, 8.0), **bath):
    """One electronic state on surface U (used for equilibrium checks)."""
    d = dict(name="single_state", S=1, nq=nq, np=n_p, q_min=qr[0], q_max=qr[1], p_min=pr[0], p_max=pr[1],
             U=[[U]], mu=np.array([[1.0]]), eta=0.5, gamma=1.0, beta=0.48, n_matsubara=0,
             high_temperature=1, use_cdelta=0, depth=3, closure=1, dt=0.01, periodic_q=0)
    d.update(bath)
    return d


def n_elements(model):
    """Number of hierarchy elements C(depth + K + 1, K + 1) (a count, used for sizing buffers)."""
    return math.comb(model["depth"] + model["n_matsubara"] + 1, model["n_matsubara"] + 1)


def state_shape(model, replicas=None):
    shp = (n_elements(model), model["S"], model["S"], model["nq"], model["np"])
    return shp if replicas is None else (replicas,) + shp


def random_state(model, seed=SEED, replicas=None, hermitian=False, zero_p_edges=0):
    """Complex uniform[-1, 1] state.  hermitian: W_kj = conj(W_jk) for every element.
    zero_p_edges: number of p columns set to zero at both ends."""
    rng = np.random.default_rng(seed)
    shp = state_shape(model, replicas)
    W = rng.uniform(-1, 1, shp) + 1j * rng.uniform(-1, 1, shp)
    if hermitian:
        W = 0.5 * (W + np.conj(np.swapaxes(W, -3, -4)))
    if zero_p_edges:
        W[..., :zero_p_edges] = 0
        W[..., -zero_p_edges:] = 0
    return np.ascontiguousarray(W)


WORKLOADS = {  # the named synthetic workloads at their full sizes
    "harmonic_32x32_d3": lambda: harmonic_two_state(),
    "photoiso_96x128_d8": lambda: photoisomerization_two_state(),
    "three_state_256x256_d10": lambda: three_state(),
}


def morse_photoisomerization(nq=512, n_p=128, qr=(-20.0, 80.0), pr=(-25.0, 25.0), bath="underdamped"):
    """The paper's own model (Sec. III), in units of hbar*omega_0 with omega_0 = 100 cm^-1: displaced
    Morse diabats and a Gaussian diabatic coupling.  The printed exponent is read as
    -a_j (q - q_j) with a_j = omega_j / sqrt(2 D_j omega_0), which reproduces the printed resonance
    frequencies (the literal printed form does not).  Baths of Sec. III (T = 300 K, beta = 0.48):
    underdamped zeta = 40 cm^-1, gamma = 500 cm^-1, depth 5; overdamped zeta = 400 cm^-1 with the
    gamma -> infinity limit, i.e. the depth-0 hierarchy with the Eq. (GMFP) terminator (the quantum
    Fokker-Planck equation, where gamma no longer enters)."""
    if bath not in ("underdamped", "overdamped"):
        raise ValueError(bath)
    w0, w1 = 1.0, 0.8
    D0, D1, dE, dV = 700.0, 500.0, 10.0, 6.0
    q0, q1, qs, sig = 0.0, 18.98, 10.28, 2.0
    a0, a1 = w0 / math.sqrt(2 * D0 * w0), w1 / math.sqrt(2 * D1 * w0)
    U00 = lambda q: D0 * (1 - np.exp(-a0 * (np.asarray(q) - q0))) ** 2
    U11 = lambda q: D1 * (1 - np.exp(-a1 * (np.asarray(q) - q1))) ** 2 + dE
    U01 = lambda q: dV * np.exp(-(np.asarray(q) - qs) ** 2 / (2 * sig * sig))
    return dict(
        name="morse_photoisomerization", S=2, nq=nq, np=n_p, q_min=qr[0], q_max=qr[1], p_min=pr[0], p_max=pr[1],
        U=[[U00, U01], [U01, U11]], mu=np.array([[0.0, 1.0], [1.0, 0.0]]),
        eta=0.4 if bath == "underdamped" else 4.0, gamma=5.0, beta=0.48, n_matsubara=0, high_temperature=1,
        use_cdelta=0, depth=5 if bath == "underdamped" else 0, closure=1, dt=1e-3, periodic_q=0, q_minima=(q0, q1))
