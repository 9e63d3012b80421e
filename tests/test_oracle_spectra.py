"""Pins of the oracle's spectra, each part on its own (no GPU).

Eqs. (nonreph) and (reph) differ only in the sign of omega_1 in the t1 transform, and Eq. (I3) is their
sum.  A sum-only check cannot tell the two parts apart, so these tests drive the oracle with a response
whose transforms are known in closed form and compare each part separately:

* R3(t3, t1) = exp(-(i Omega3 + G3) t3) exp(-(i Omega1 + G1) t1), a product of damped oscillations.
  The trapezoid sum of a sampled exponential is a geometric series, so the discrete transform has an
  exact closed form (a pin to rounding); the continuum double Laplace transform fixes the physics
  (NR peaks at omega1 = +Omega1, R at omega1 = -Omega1) within the quadrature error.
"""
import numpy as np

import oracle


def _trapezoid_geometric(z, n, dt):
    """dt * (z^0/2 + z^1 + ... + z^(n-1) + z^n/2): the trapezoid rule on n+1 samples of z^m."""
    return dt * ((1 - z ** (n + 1)) / (1 - z) - 0.5 * (1 + z ** n))


def _damped_product(n1, n3, dt1, dt3, om1, g1, om3, g3):
    t1 = np.arange(n1) * dt1
    t3 = np.arange(n3) * dt3
    return np.exp(-(1j * om1 + g1) * t1)[:, None] * np.exp(-(1j * om3 + g3) * t3)[None, :]


def test_two_d_parts_equal_the_discrete_geometric_sums():
    """Each of I_NR and I_R equals Im of the product of two closed-form trapezoid sums (Eqs. (nonreph),
    (reph)): the omega_1 exponent is +i omega_1 t1 for NR and -i omega_1 t1 for R."""
    n1, n3, dt1, dt3 = 40, 301, 0.08, 0.01
    Om1, G1, Om3, G3 = 3.0, 0.4, 7.0, 0.6
    R3 = _damped_product(n1, n3, dt1, dt3, Om1, G1, Om3, G3)
    w1 = np.linspace(-6.0, 6.0, 25) + 0.13  # not symmetric about 0
    w3 = np.linspace(2.0, 12.0, 21)
    nr, re, corr = oracle.two_d(R3, dt1, dt3, w1, w3)
    A3 = _trapezoid_geometric(np.exp((1j * w3 - 1j * Om3 - G3) * dt3), n3 - 1, dt3)      # [w3]
    A1p = _trapezoid_geometric(np.exp((1j * w1 - 1j * Om1 - G1) * dt1), n1 - 1, dt1)     # [w1], NR
    A1m = _trapezoid_geometric(np.exp((-1j * w1 - 1j * Om1 - G1) * dt1), n1 - 1, dt1)    # [w1], R
    nr_ref = (A3[:, None] * A1p[None, :]).imag
    re_ref = (A3[:, None] * A1m[None, :]).imag
    scale = np.abs(nr_ref).max()
    assert np.abs(nr - nr_ref).max() < 1e-12 * scale
    assert np.abs(re - re_ref).max() < 1e-12 * scale
    assert np.abs(corr - (nr_ref + re_ref)).max() < 1e-12 * scale
    # the two parts are far apart for this response: exchanging them fails the checks above
    assert np.abs(nr_ref - re_ref).max() > 0.3 * scale


def test_two_d_parts_against_the_double_laplace_transform():
    """Continuum check of Eqs. (nonreph), (reph): with a long, fine time grid the trapezoid sums approach
    Im[i/(G3 - i(w3 - Omega3)) * 1/(G1 - i(+-w1 - Omega1))] for R3 = i exp(...) exp(...) (the factor i
    makes the parts absorptive); the non-rephasing part peaks at omega_1 = +Omega_1 and the rephasing
    part at omega_1 = -Omega_1."""
    dt1, dt3 = 0.01, 0.01
    Om1, G1, Om3, G3 = 4.0, 1.0, 6.0, 1.0
    n1 = n3 = 2401  # t up to 24: exp(-24) truncation
    R3 = 1j * _damped_product(n1, n3, dt1, dt3, Om1, G1, Om3, G3)
    w1 = np.linspace(-8.0, 8.0, 33)
    w3 = np.array([4.0, 6.0, 8.0])
    nr, re, _ = oracle.two_d(R3, dt1, dt3, w1, w3)
    L3 = 1j / (G3 - 1j * (w3 - Om3))
    nr_ref = (L3[:, None] / (G1 - 1j * (w1 - Om1))[None, :]).imag
    re_ref = (L3[:, None] / (G1 - 1j * (-w1 - Om1))[None, :]).imag
    # trapezoid error: the endpoint term dt^2/12 |f'(0)| per axis, relative to |L| ~ 1/G
    tol = 2e-4
    assert np.abs(nr - nr_ref).max() < tol
    assert np.abs(re - re_ref).max() < tol
    # peak positions along omega_1 on the omega_3 = Omega_3 row
    row = 1
    assert w1[np.argmax(np.abs(nr[row]))] == Om1
    assert w1[np.argmax(np.abs(re[row]))] == -Om1
