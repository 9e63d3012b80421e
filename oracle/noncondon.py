"""Coordinate-dependent (non-Condon) dipole super-operators of Sec. III in plain numpy FP64.

Test infrastructure only: imported by tests/ and never by the library or its binding.

The partial Wigner representations of mu rho and rho mu are the p-convolutions
    (mu^-> W)_jk(p, q) = sum_l mu_jl(p, q) * W_lk(p, q),   (mu^<- W)_jk = sum_l mu*_lk(p, q) * W_jl,
    mu_jk(p, q) = (1 / 2 pi) int dr e^{-i p r} mu_jk(q + r/2)        (hbar = 1),
and mu*(p, q) is the transform of mu(q - r/2).  On the p grid (r grid dr = 2 pi / (np dp), modes
m = -np/2 .. np/2 - 1) the convolution is the circulant matrix
    K[l, l'] = (1/np) sum_m e^{-2 pi i m (l - l') / np} mu(q + r_m / 2)
(for mu^<-: mu(q - r_m / 2)), built here explicitly from this definition -- no FFT.  The Nyquist mode
m = -np/2 takes the symmetric value (mu(q + r_max/2) + mu(q - r_max/2)) / 2, the same reading as for the
potential.  The multipliers come from a table in the potential-table convention:
T[j][k][i][t] = mu_jk(q_i + s_t), s_t = (t - np/2) dr / 2, so r_m / 2 sits at column np/2 + m and
-r_m / 2 at column np/2 - m.

The trace with a coordinate-dependent dipole: Tr{mu W} = sum_jk int dq dp mu_kj(q) W_jk(q, p) (the Wigner
function of the operator mu(q) is mu(q)).
"""
import numpy as np

LEFT, RIGHT, COMMUTATOR = 1, 2, 3


def multipliers(mu_table):
    """(ML, MR): mu(q_i + r_m/2) and mu(q_i - r_m/2), [S][S][nq][np] over m = -np/2 .. np/2 - 1."""
    n_p = mu_table.shape[-1] - 1
    m = np.arange(-n_p // 2, n_p // 2)
    ML = mu_table[..., n_p // 2 + m].copy()
    MR = mu_table[..., n_p // 2 - m].copy()
    nyq = 0.5 * (mu_table[..., 0] + mu_table[..., n_p])
    ML[..., 0] = nyq
    MR[..., 0] = nyq
    return ML, MR


def circulants(mult):
    """K[..., l, l'] = (1/np) sum_m e^{-2 pi i m (l - l')/np} mult[..., m]."""
    n_p = mult.shape[-1]
    m = np.arange(-n_p // 2, n_p // 2)
    d = np.arange(n_p)[:, None] - np.arange(n_p)[None, :]
    E = np.exp(-2j * np.pi * m[:, None, None] * d[None, :, :] / n_p) / n_p
    return np.einsum("...m,mab->...ab", mult, E)


def apply_dipole(W, mu_table, side=COMMUTATOR):
    """mu^-> W (LEFT), mu^<- W (RIGHT) or mu^x W (COMMUTATOR) on every hierarchy element of W
    [n_elem][S][S][nq][np]."""
    ML, MR = multipliers(mu_table)
    KL, KR = circulants(ML), circulants(MR)
    left = np.einsum("jliab,elkib->ejkia", KL, W)
    right = np.einsum("lkiab,ejlib->ejkia", KR, W)
    if side == LEFT:
        return left
    if side == RIGHT:
        return right
    return left - right


def trace(W, mu_table, dq, dp):
    """Tr{mu W^(0)} = sum_jk sum_i mu_kj(q_i) sum_l W^(0)_jk(q_i, p_l) dq dp."""
    n_p = mu_table.shape[-1] - 1
    mu_q = mu_table[..., n_p // 2]  # [S][S][nq]
    return np.einsum("kji,jkil->", mu_q, W[0]) * dq * dp


def linear_response(O, W_eq, mu_table, n_t):
    """R1(t_n) = i Tr{mu G(t_n) mu^x W_eq}, n = 0 .. n_t, with the oracle's RK4 propagator O.step."""
    X = apply_dipole(W_eq, mu_table, COMMUTATOR)
    out = np.zeros(n_t + 1, dtype=np.complex128)
    out[0] = 1j * trace(X, mu_table, O.dq, O.dp)
    for n in range(1, n_t + 1):
        X, _ = O.step(X, 1)
        out[n] = 1j * trace(X, mu_table, O.dq, O.dp)
    return out


def first_order_distribution(O, W_eq, mu_table, n_t1, t1_stride, omega):
    """W'(omega) = i [mu^-> F(omega) - mu^<- F(-omega)], F(omega) = sum_a w_a e^{i omega t_a} X(t_a),
    X(t) = G(t) mu^x W_eq, with the coordinate-dependent dipole (trapezoid weights on t_a = a t1_stride
    dt, n_t1 >= 2); propagation by the oracle's RK4 O.step."""
    assert n_t1 >= 2
    dt1 = t1_stride * O.dt
    wts = np.full(n_t1, dt1)
    wts[0] *= 0.5
    wts[-1] *= 0.5
    omega = np.asarray(omega, dtype=np.float64)
    X = apply_dipole(W_eq, mu_table, COMMUTATOR)
    Fp = np.zeros((len(omega),) + X.shape, dtype=np.complex128)
    Fm = np.zeros_like(Fp)
    for a in range(n_t1):
        if a > 0:
            X, _ = O.step(X, t1_stride)
        for k, om in enumerate(omega):
            Fp[k] += wts[a] * np.exp(1j * om * a * dt1) * X
            Fm[k] += wts[a] * np.exp(-1j * om * a * dt1) * X
    return np.stack([1j * (apply_dipole(Fp[k], mu_table, LEFT) - apply_dipole(Fm[k], mu_table, RIGHT))
                     for k in range(len(omega))])


def third_order_response(O, W_eq, mu_table, n_t1, t1_stride, t2_steps, n_t3, first=COMMUTATOR):
    """R3(t3, t2, t1) = i^3 Tr{mu G(t3) mu^x G(t2) mu^x G(t1) mu^x W_eq} (Eq. (R3)) with the
    coordinate-dependent dipole in every interaction and in the trace, on t1 = a t1_stride dt
    (a < n_t1), t2 in t2_steps dt, t3 = c dt (c <= n_t3); `first` as in Oracle.third_order_response
    (LEFT: mu^->, RIGHT: -mu^<-).  Propagation by the oracle's RK4 O.step.
    Returns [len(t2_steps)][n_t1][n_t3 + 1]."""
    W = apply_dipole(W_eq, mu_table, first)
    if first == RIGHT:
        W = -W
    out = np.zeros((len(t2_steps), n_t1, n_t3 + 1), dtype=np.complex128)
    for a in range(n_t1):
        if a > 0:
            W, _ = O.step(W, t1_stride)
        X = apply_dipole(W, mu_table, COMMUTATOR)
        done = 0
        for b, t2 in enumerate(t2_steps):
            if t2 > done:
                X, _ = O.step(X, t2 - done)
                done = t2
            Y = apply_dipole(X, mu_table, COMMUTATOR)
            out[b, a, 0] = (1j) ** 3 * trace(Y, mu_table, O.dq, O.dp)
            for c in range(1, n_t3 + 1):
                Y, _ = O.step(Y, 1)
                out[b, a, c] = (1j) ** 3 * trace(Y, mu_table, O.dq, O.dp)
    return out
