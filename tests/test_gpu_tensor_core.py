"""The tcgen05 split-bf16 DFT-GEMM potential kernel (QHFPE_MIXED_BF16X3) against the FP64 oracle."""
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


def rel(a, b):
    return np.linalg.norm(np.ravel(a - b)) / max(np.linalg.norm(np.ravel(b)), 1e-300)


def _P(m, precision="bf16x3", **kw):
    from paper_1706_09590_gb300 import Propagator
    return Propagator(m, qi.u_table(m), precision=precision, **kw)


MODELS = {
    "np128_S2": qi.photoisomerization_two_state(nq=20, n_p=128, depth=2, n_matsubara=1),
    "np64_S2": qi.harmonic_two_state(nq=24, n_p=64, depth=2),
    "np128_S1": qi.single_state(lambda q: 5.0 * ((q / 4.0) ** 2 - 1.0) ** 2, nq=12, n_p=128, depth=1),
}


@pytest.mark.parametrize("name", list(MODELS))
def test_potential_term(name):
    m = MODELS[name]
    O = oracle.Oracle(m)
    P = _P(m)
    W = qi.random_state(m, seed=71)
    P.set_state(W)
    Win = P.get_state(0)
    Win[1:] = Win[1:].astype(np.complex64).astype(np.complex128)
    ref = O.rhs(Win, oracle.POTENTIAL)
    got = P.apply_rhs(0, oracle.POTENTIAL)
    err = rel(got, ref)
    print(name, "potential-term relative L2 error", err)
    assert err < 2e-4
    full = rel(P.apply_rhs(0), O.rhs(Win))
    print(name, "full right-hand side relative L2 error", full)
    assert full < 2e-4


def test_linear_response_bf16x3():
    m = qi.harmonic_two_state(nq=32, n_p=64, depth=3)
    O = oracle.Oracle(m)
    Weq, _ = O.equilibrate(300)
    ref = O.linear_response(Weq, 300)
    P = _P(m)
    P.set_equilibrium(Weq)
    got = P.linear_response(300)
    err = rel(got, ref)
    print("R1 relative L2 error (bf16x3)", err)
    assert err < 1e-4


@pytest.mark.parametrize("name", ["np128_S2", "np64_S2"])
def test_potential_term_replicas(name):
    """Several replicas in one launch (tiles whose rows span replicas, elements and q rows, a ragged
    last tile): each replica's right-hand side against the oracle on its own state."""
    m = MODELS[name]
    O = oracle.Oracle(m)
    P = _P(m, n_replicas=3)
    Ws = [qi.random_state(m, seed=90 + r) for r in range(3)]
    for r, W in enumerate(Ws):
        P.set_state(W, r)
    for r in (2, 0, 1):
        Win = P.get_state(r)
        Win[1:] = Win[1:].astype(np.complex64).astype(np.complex128)
        err = rel(P.apply_rhs(r, oracle.POTENTIAL), O.rhs(Win, oracle.POTENTIAL))
        assert err < 2e-4, (name, r, err)
        assert rel(P.apply_rhs(r), O.rhs(Win)) < 2e-4, (name, r)
    P.close()
