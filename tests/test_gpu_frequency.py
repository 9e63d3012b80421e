"""The frequency-domain first-order distribution W'(omega_1) (Sec. III, "One-dimensional spectrum")
through the C ABI: parity with the oracle (every tier, FP64 and mixed forms), and the correlation
spectrum obtained as the linear absorption of W''(t2, omega_1) = G(t2) i [W'(omega_1) + W'(-omega_1)]
against the correlation spectrum of the R3 route, Eq. (I3), computed by the library on the same grids."""
import numpy as np
import pytest

import oracle
import qhfpe_inputs as qi

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _P(model, precision, **kw):
    from paper_1706_09590_gb300 import Propagator
    return Propagator(model, qi.u_table(model), precision=precision, **kw)


def rel(a, b):
    return np.linalg.norm(np.ravel(a - b)) / max(np.linalg.norm(np.ravel(b)), 1e-300)


@pytest.fixture(scope="module")
def setup():
    m = qi.harmonic_two_state(nq=32, n_p=32, depth=3)
    O = oracle.Oracle(m)
    Weq, _ = O.equilibrate(300)
    return m, O, Weq


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-10), ("mixed", 1e-5)])
def test_first_order_distribution_matches_the_oracle(setup, precision, tol):
    m, O, Weq = setup
    n_t1, stride = 16, 4
    omega = np.array([9.0, 10.5, -10.5, 12.0])
    ref = O.first_order_distribution(Weq, n_t1, stride, omega)
    P = _P(m, precision)
    P.set_equilibrium(Weq)
    got = P.first_order_distribution(n_t1, stride, omega)
    assert got.shape == ref.shape
    for k in range(len(omega)):
        assert rel(got[k], ref[k]) < tol, (precision, omega[k], rel(got[k], ref[k]))
    P.close()


def test_correlation_spectrum_through_the_second_order_distribution(setup):
    from paper_1706_09590_gb300 import COMMUTATOR
    m, O, Weq = setup
    n_t1, stride, t2, n_t3 = 16, 4, 30, 200
    omega1 = np.linspace(8.0, 13.0, 6)
    omega3 = np.linspace(6.0, 15.0, 19)
    out = {}
    for precision in ("fp64", "mixed"):
        P = _P(m, precision)
        P.set_equilibrium(Weq)
        Wp = P.first_order_distribution(n_t1, stride, np.concatenate([omega1, -omega1]))
        dt3 = m["dt"]
        t3 = np.arange(n_t3 + 1) * dt3
        w3 = np.full(n_t3 + 1, dt3)
        w3[0] *= 0.5
        w3[-1] *= 0.5
        corr = np.zeros((len(omega3), len(omega1)))
        for k in range(len(omega1)):
            P.set_state(1j * (Wp[k] + Wp[k + len(omega1)]))
            P.step(t2)
            P.apply_dipole(COMMUTATOR)
            sig = 1j * P.step(n_t3, record_trace=True)[0]
            corr[:, k] = (np.exp(1j * omega3[:, None] * t3[None, :]) @ (w3 * sig)).imag
        R3 = P.third_order_response(n_t1, stride, [t2], n_t3)[0]
        ref = P.spectrum_2d(R3, stride * m["dt"], dt3, omega1, omega3)[2]
        out[precision] = corr
        tol = 1e-10 if precision == "fp64" else 1e-4
        print(precision, "W'' route vs R3 route, relative L2:", rel(corr, ref))
        assert rel(corr, ref) < tol
        P.close()
    assert rel(out["mixed"], out["fp64"]) < 1e-4


def test_first_order_distribution_rejects_bad_arguments(setup):
    from paper_1706_09590_gb300 import QhfpeError
    m, O, Weq = setup
    P = _P(m, "fp64")
    with pytest.raises(QhfpeError):  # no equilibrium yet
        P.first_order_distribution(4, 2, [1.0])
    P.set_equilibrium(Weq)
    with pytest.raises(QhfpeError):
        P.first_order_distribution(0, 2, [1.0])
    with pytest.raises(QhfpeError):
        P.first_order_distribution(4, 0, [1.0])
    with pytest.raises(QhfpeError):
        P.first_order_distribution(4, 2, [np.nan])
    P.close()
