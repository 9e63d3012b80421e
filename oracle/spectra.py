"""Spectra from response functions -- TEST INFRASTRUCTURE ONLY (part of the CPU oracle).

Fourier-Laplace transforms of Sec. III by the trapezoid rule on the sampled time grid (weight 1/2 at
both ends, no window); frequencies are given explicitly by the caller.
"""
import numpy as np


def _weights(n, dt):
    w = np.full(n, dt)
    w[0] *= 0.5
    w[-1] *= 0.5
    return w


def absorption(R1, dt, omega):
    """Eq. (I1): I(w) = w Im int_0^T dt e^{iwt} R1(t)."""
    R1 = np.asarray(R1)
    t = np.arange(len(R1)) * dt
    w = _weights(len(R1), dt)
    omega = np.asarray(omega, dtype=np.float64)
    ft = np.exp(1j * omega[:, None] * t[None, :]) @ (w * R1)
    return omega * ft.imag


def two_d(R3, dt1, dt3, omega1, omega3):
    """Eqs. (nonreph), (reph), (I3) for one waiting time.  R3: [n_t1][n_t3+1] on t1 = a*dt1,
    t3 = c*dt3.  Returns (I_NR, I_R, I_corr), each [len(omega3)][len(omega1)]."""
    R3 = np.asarray(R3)
    n1, n3 = R3.shape
    t1 = np.arange(n1) * dt1
    t3 = np.arange(n3) * dt3
    w1 = _weights(n1, dt1)
    w3 = _weights(n3, dt3)
    E3 = np.exp(1j * np.asarray(omega3)[:, None] * t3[None, :]) * w3[None, :]
    E1p = np.exp(1j * np.asarray(omega1)[:, None] * t1[None, :]) * w1[None, :]
    E1m = np.exp(-1j * np.asarray(omega1)[:, None] * t1[None, :]) * w1[None, :]
    G = E3 @ R3.T  # [w3][t1]
    nr = (G @ E1p.T).imag
    re = (G @ E1m.T).imag
    return nr, re, nr + re


def transient_absorption(R3_t1zero, dt, omega):
    """Eq. (transient-absorption): I(w, T) = w Im int dt e^{iwt} R3(t, T, 0).
    R3_t1zero: [n_T][n_t+1].  Returns [n_T][len(omega)]."""
    R = np.atleast_2d(np.asarray(R3_t1zero))
    return np.stack([absorption(r, dt, omega) for r in R])


def transient_absorption_from_corr(R3, dt1, dt3, omega3, n_omega1):
    """The alternative definition of Sec. III D: I(w, T) = w int dw1 I_corr(w, T, w1), with the w1
    integral a Riemann sum over one full period [0, 2 pi/dt1) on n_omega1 points."""
    omega1 = np.arange(n_omega1) * (2 * np.pi / dt1 / n_omega1)
    _, _, corr = two_d(R3, dt1, dt3, omega1, omega3)
    return np.asarray(omega3) * corr.sum(axis=1) * (2 * np.pi / dt1 / n_omega1)
