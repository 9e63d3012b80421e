"""Coordinate-dependent (non-Condon) dipoles (Sec. III) through the C ABI: the dipole super-operators
on every tier against the numpy oracle (two and three states, FP64 and mixed forms, a replica subset),
a coordinate-independent table against the Condon path, the linear response R1, W'(omega) and the
third-order response R3 (split pathways and plain) against the oracle, the return to the Condon
dipole, and the argument checks."""
import numpy as np
import pytest

import oracle
import qhfpe_inputs as qi
from oracle import noncondon as nc

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


MODELS = {
    "two_state_np64": qi.photoisomerization_two_state(nq=20, n_p=64, depth=2, n_matsubara=1),
    "three_state_np32": qi.three_state(nq=12, n_p=32, depth=1, n_matsubara=1),
    "harmonic_np128": qi.harmonic_two_state(nq=9, n_p=128, depth=2),
}


@pytest.mark.parametrize("name", list(MODELS))
@pytest.mark.parametrize("precision,tol", [("fp64", 1e-12), ("mixed", 2e-6)])
def test_dipole_superoperators_match_the_oracle(name, precision, tol):
    from paper_1706_09590_gb300 import LEFT, RIGHT, COMMUTATOR
    m = MODELS[name]
    T = qi.function_table(m, qi.linear_dipole(m, slope=0.15, q_ref=0.5))
    P = _P(m, precision, n_replicas=3)
    P.set_dipole_table(T)
    for side in (LEFT, RIGHT, COMMUTATOR):
        Ws = [qi.random_state(m, seed=110 + 10 * side + r) for r in range(3)]
        for r, W in enumerate(Ws):
            P.set_state(W, r)
        P.apply_dipole(side, replicas=[0, 2])
        for r, W in enumerate(Ws):
            got = P.get_state(r)
            if r == 1:  # not in the list: unchanged (up to the mixed forms' rounding at set_state)
                assert rel(got[0], W[0]) == 0.0
                continue
            Win = W.copy()
            if precision != "fp64":
                Win[1:] = Win[1:].astype(np.complex64).astype(np.complex128)
            ref = nc.apply_dipole(Win, T, side)
            assert rel(got[0], ref[0]) < (1e-12 if precision == "fp64" else 1e-12 * 100), (side, r)
            assert rel(got, ref) < tol, (name, precision, side, r, rel(got, ref))
    P.close()


def test_constant_table_equals_the_condon_path():
    m = MODELS["two_state_np64"]
    mu = np.asarray(m["mu"], dtype=np.float64)
    F = [[(lambda c: (lambda q: np.full_like(np.asarray(q, dtype=np.float64), c)))(mu[j, k]) for k in range(2)]
         for j in range(2)]
    W = qi.random_state(m, seed=120)
    A, B = _P(m, "fp64"), _P(m, "fp64")
    A.set_dipole_table(qi.function_table(m, F))
    A.set_state(W)
    B.set_state(W)
    A.apply_dipole()
    B.apply_dipole()
    assert rel(A.get_state(0), B.get_state(0)) < 1e-13
    assert abs(A.trace()[0] - B.trace()[0]) <= 1e-13 * abs(B.trace()[0])


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-10), ("mixed", 1e-5)])
def test_linear_response_matches_the_oracle(precision, tol):
    m = qi.harmonic_two_state(nq=32, n_p=32, depth=3)
    O = oracle.Oracle(m)
    Weq, _ = O.equilibrate(300)
    T = qi.function_table(m, qi.linear_dipole(m, slope=0.3))
    ref = nc.linear_response(O, Weq, T, 60)
    P = _P(m, precision)
    P.set_dipole_table(T)
    P.set_equilibrium(Weq)
    got = P.linear_response(60)
    assert rel(got, ref) < tol
    # back to the Condon dipole: the Condon response again
    P.set_dipole_table(None)
    assert rel(P.linear_response(60), O.linear_response(Weq, 60)) < tol
    P.close()


def test_argument_checks():
    from paper_1706_09590_gb300 import QhfpeError
    m = qi.harmonic_two_state(nq=8, n_p=16, depth=1)  # np = 16: no FFT dipole kernel
    P = _P(m, "fp64")
    with pytest.raises(QhfpeError):
        P.set_dipole_table(qi.function_table(m, qi.linear_dipole(m)))
    P.close()
    m = MODELS["two_state_np64"]
    P = _P(m, "fp64")
    T = qi.function_table(m, qi.linear_dipole(m))
    bad = T.copy()
    bad[0, 1, 3, 5] += 1.0  # no longer symmetric in (j, k)
    with pytest.raises(QhfpeError):
        P.set_dipole_table(bad)
    bad = T.copy()
    bad[1, 0, 0, 0] = np.inf
    bad[0, 1, 0, 0] = np.inf
    with pytest.raises(QhfpeError):
        P.set_dipole_table(bad)
    P.close()


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-10), ("mixed", 1e-5)])
def test_first_order_distribution_with_a_coordinate_dependent_dipole(precision, tol):
    m = qi.harmonic_two_state(nq=32, n_p=32, depth=2)
    O = oracle.Oracle(m)
    Weq, _ = O.equilibrate(200)
    T = qi.function_table(m, qi.linear_dipole(m, slope=0.25))
    omega = np.array([9.5, -9.5, 11.0])
    ref = nc.first_order_distribution(O, Weq, T, 10, 4, omega)
    P = _P(m, precision)
    P.set_dipole_table(T)
    P.set_equilibrium(Weq)
    got = P.first_order_distribution(10, 4, omega)
    for k in range(len(omega)):
        assert rel(got[k], ref[k]) < tol, (precision, omega[k], rel(got[k], ref[k]))
    P.close()


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-10), ("mixed", 1e-5)])
def test_third_order_response_matches_the_oracle(precision, tol):
    """Eq. (R3) with the coordinate-dependent dipole in every interaction and the trace: the batched
    schedule (split pathways and the plain commutator) against the oracle's composition."""
    m = qi.harmonic_two_state(nq=32, n_p=32, depth=2)
    O = oracle.Oracle(m)
    Weq, _ = O.equilibrate(300)
    T = qi.function_table(m, qi.linear_dipole(m, slope=0.25))
    args = (3, 4, [0, 6], 12)
    ket = nc.third_order_response(O, Weq, T, *args, first=nc.LEFT)
    bra = nc.third_order_response(O, Weq, T, *args, first=nc.RIGHT)
    P = _P(m, precision)
    P.set_dipole_table(T)
    P.set_equilibrium(Weq)
    got = P.third_order_response(*args, split_pathways=True)
    assert rel(got[0], ket) < tol
    assert rel(got[1], bra) < tol
    assert rel(P.third_order_response(*args, split_pathways=False), ket + bra) < tol
    P.close()
