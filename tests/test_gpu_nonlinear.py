"""The nonlinear system-bath coupling V(q) = q + c2 q^2 (Sec. II) through the C ABI against the CPU
oracle (whose operators are pinned against the density-matrix hierarchy): each right-hand-side term
alone, RK4 steps with traces, the linear response, a heterogeneous batch with a nonlinear member and
persistent propagation.
Tolerances as in the other parity tests: FP64 1e-12 (one right-hand side) / 1e-11 (steps) / 1e-10
(response), mixed 2e-5 / 1e-5 / 1e-4."""
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


def _P(m, precision="fp64", **kw):
    from paper_1706_09590_gb300 import Propagator
    return Propagator(m, qi.u_table(m), precision=precision, **kw)


def _models():
    h = qi.harmonic_two_state(nq=24, n_p=32, depth=3, closure=0)
    h["v_c2"] = 0.1
    ph = qi.photoisomerization_two_state(nq=20, n_p=64, depth=3, n_matsubara=2)
    ph["v_c2"] = -0.04
    three = qi.three_state(nq=16, n_p=32, depth=2, n_matsubara=1)
    three["v_c2"] = 0.05
    per = qi.harmonic_two_state(nq=18, n_p=32, depth=2, closure=0)
    per["v_c2"] = 0.08
    per["periodic_q"] = 1
    wide = qi.harmonic_two_state(nq=12, n_p=128, pr=(-16.0, 16.0), depth=4, closure=0)
    wide["v_c2"] = 0.1
    return {"harmonic": h, "photoiso_K2": ph, "three_state": three, "periodic": per, "np128": wide}


MODELS = _models()
TERMS = [1, 2, 4, 8, 16, 31]


@pytest.mark.parametrize("name", list(MODELS))
@pytest.mark.parametrize("precision,tol", [("fp64", 1e-12), ("mixed", 2e-5)])
def test_nonlinear_rhs_terms(name, precision, tol):
    m = MODELS[name]
    O = oracle.Oracle(m)
    P = _P(m, precision)
    W = qi.random_state(m, seed=31)
    P.set_state(W)
    Win = P.get_state(0)
    for t in TERMS:
        ref = O.rhs(Win, t)
        got = P.apply_rhs(0, t)
        if np.linalg.norm(ref) == 0:
            assert np.linalg.norm(got) == 0
        else:
            assert rel(got, ref) < tol, (name, t, rel(got, ref))
    P.close()


@pytest.mark.parametrize("name", ["harmonic", "photoiso_K2", "np128"])
@pytest.mark.parametrize("precision,tol", [("fp64", 1e-11), ("mixed", 1e-5)])
def test_nonlinear_steps(name, precision, tol):
    m = MODELS[name]
    W = qi.random_state(m, seed=32, hermitian=True)
    ref_W, ref_tr = oracle.Oracle(m).step(W, 12)
    P = _P(m, precision)
    P.set_state(W)
    tr = P.step(12, record_trace=True)[0]
    assert rel(P.get_state(0), ref_W) < tol
    assert rel(tr, ref_tr) < tol
    P.close()


def test_nonlinear_linear_response_fp64_and_mixed():
    m = MODELS["harmonic"]
    O = oracle.Oracle(m)
    Weq, _ = O.equilibrate(300)
    ref = O.linear_response(Weq, 200)
    for precision, tol in (("fp64", 1e-10), ("mixed", 1e-4)):
        P = _P(m, precision)
        P.set_equilibrium(Weq)
        assert rel(P.linear_response(200), ref) < tol
        P.close()
    # the coupling matters: the linear-coupling response is far away
    lin = dict(m, v_c2=0.0)
    O0 = oracle.Oracle(lin)
    assert rel(O0.linear_response(O0.equilibrate(300)[0], 200), ref) > 1e-3


def test_nonlinear_member_in_a_heterogeneous_batch():
    from paper_1706_09590_gb300 import Batch
    a, b = MODELS["harmonic"], dict(MODELS["harmonic"], v_c2=0.0, nq=28)
    Wa, Wb = qi.random_state(a, seed=33), qi.random_state(b, seed=34)
    alone = []
    for m, W in ((a, Wa), (b, Wb)):
        P = _P(m, "mixed")
        P.set_state(W)
        P.step(10)
        alone.append(P.get_state(0))
        P.close()
    Ps = [_P(a, "mixed"), _P(b, "mixed")]
    Ps[0].set_state(Wa)
    Ps[1].set_state(Wb)
    B = Batch(Ps)
    B.step(10)
    for P, ref in zip(Ps, alone):
        assert rel(P.get_state(0), ref) < 1e-6
    B.close()
    for P in Ps:
        P.close()


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-11), ("mixed", 1e-5)])
def test_nonlinear_persistent_steps(precision, tol):
    """Persistent propagation (one cooperative launch over the batch kernel, which carries the nonlinear
    terms) against the oracle, with the trace reduced in the same launch."""
    m = MODELS["harmonic"]
    W = qi.random_state(m, seed=35)
    P = _P(m, precision)
    P.set_persistent(True)
    P.set_state(W)
    tr = P.step(9, record_trace=True)[0]
    got = P.get_state(0)
    P.close()
    ref_W, ref_tr = oracle.Oracle(m).step(W, 9)
    assert rel(got, ref_W) < tol and rel(tr, ref_tr) < tol, (rel(got, ref_W), rel(tr, ref_tr))


def test_nonlinear_coupling_rejects_closures():
    from paper_1706_09590_gb300 import QhfpeError
    m = dict(qi.harmonic_two_state(nq=16, n_p=32, depth=2, closure=1), v_c2=0.1)
    with pytest.raises(QhfpeError):
        _P(m)
