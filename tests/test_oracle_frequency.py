"""Pins of the oracle's frequency-domain first-order distribution W'(omega_1) (Sec. III, "One-dimensional
spectrum") against relations the mathematics fixes:

* its phase-space trace: Tr W'(omega) = 2i sum_a w_a sin(omega t_a) R1(t_a), with R1 the oracle's linear
  response (Tr{mu^-> Y} = Tr{mu^<- Y} = Tr{mu Y} and R1 = i Tr{mu G mu^x W_eq});
* the paper's reading of the correlation spectrum as the linear absorption of
  W''(t2, omega_1) = G(t2) i [W'(omega_1) + W'(-omega_1)]: Im sum_c w_c e^{i omega_3 t3} Tr{mu G(t3) i mu^x W''}
  equals the correlation spectrum computed from R3, Eqs. (I3), (nonreph), (reph), on the same t1 and t3
  grids (a discrete identity: W' + W'(-omega) carries 2 cos(omega t1) into the t1 sum);
* W'(omega) is linear in the t1 samples: doubling n_t1 at half the stride changes only the quadrature,
  so on a smooth signal the two agree to the trapezoid error, and omega = 0 gives i mu^x sum_a w_a X(t_a).
"""
import numpy as np

import oracle
import qhfpe_inputs as qi
from oracle import spectra


def _model():
    return qi.harmonic_two_state(nq=16, n_p=16, depth=2)


def _eq(O):
    W, _ = O.equilibrate(200)
    return W


def _tr(W, O):
    S = W.shape[1]
    return sum(W[0, j, j].sum() for j in range(S)) * O.dq * O.dp


def test_trace_of_first_order_distribution_is_the_sine_transform_of_R1():
    m = _model()
    O = oracle.Oracle(m)
    Weq = _eq(O)
    n_t1, stride = 12, 3
    omega = np.array([0.0, 7.5, 10.0, 12.5])
    Wp = O.first_order_distribution(Weq, n_t1, stride, omega)
    R1 = O.linear_response(Weq, (n_t1 - 1) * stride)[::stride]
    assert len(R1) == n_t1
    dt1 = stride * m["dt"]
    w = np.full(n_t1, dt1)
    w[0] *= 0.5
    w[-1] *= 0.5
    t = np.arange(n_t1) * dt1
    for k, om in enumerate(omega):
        ref = 2j * np.sum(w * np.sin(om * t) * R1)
        got = _tr(Wp[k], O)
        assert abs(got - ref) <= 1e-12 * max(abs(ref), np.abs(R1).max() * t[-1]), (om, got, ref)


def test_correlation_spectrum_from_second_order_distribution_equals_the_R3_route():
    m = _model()
    O = oracle.Oracle(m)
    Weq = _eq(O)
    n_t1, stride, t2, n_t3 = 8, 4, 10, 40
    omega1 = np.array([8.0, 10.0, 11.5])
    omega3 = np.linspace(6.0, 14.0, 9)
    Wp = O.first_order_distribution(Weq, n_t1, stride, np.concatenate([omega1, -omega1]))
    dt3 = m["dt"]
    t3 = np.arange(n_t3 + 1) * dt3
    w3 = np.full(n_t3 + 1, dt3)
    w3[0] *= 0.5
    w3[-1] *= 0.5
    got = np.zeros((len(omega3), len(omega1)))
    for k in range(len(omega1)):
        W2 = 1j * (Wp[k] + Wp[k + len(omega1)])
        W2, _ = O.step(W2, t2)
        _, tr = O.step(O.apply_dipole(W2, oracle.COMMUTATOR), n_t3)
        sig = 1j * tr  # Tr{mu G(t3) i mu^x W''}
        got[:, k] = (np.exp(1j * omega3[:, None] * t3[None, :]) @ (w3 * sig)).imag
    R3 = O.third_order_response(Weq, n_t1, stride, [t2], n_t3)[0]
    ref = spectra.two_d(R3, stride * m["dt"], dt3, omega1, omega3)[2]
    assert np.abs(ref).max() > 0
    assert np.linalg.norm(got - ref) <= 1e-12 * np.linalg.norm(ref)


def test_zero_frequency_and_quadrature_refinement():
    m = _model()
    O = oracle.Oracle(m)
    Weq = _eq(O)
    # omega = 0: W'(0) = i mu^x F(0), F(0) = sum_a w_a X(t_a)
    n_t1, stride = 6, 5
    W0 = O.first_order_distribution(Weq, n_t1, stride, [0.0])[0]
    X = O.apply_dipole(Weq, oracle.COMMUTATOR)
    dt1 = stride * m["dt"]
    F = np.zeros_like(X)
    for a in range(n_t1):
        if a > 0:
            X, _ = O.step(X, stride)
        F += (0.5 if a in (0, n_t1 - 1) else 1.0) * dt1 * X
    assert np.linalg.norm(W0 - 1j * O.apply_dipole(F, oracle.COMMUTATOR)) <= 1e-13 * np.linalg.norm(W0)
    # the same t1 window sampled twice as finely: the trapezoid sums agree to their O(dt1^2) error
    coarse = O.first_order_distribution(Weq, 11, 4, [9.0])[0]
    fine = O.first_order_distribution(Weq, 21, 2, [9.0])[0]
    err = np.linalg.norm(coarse - fine) / np.linalg.norm(fine)
    assert 1e-8 < err < 1e-2
