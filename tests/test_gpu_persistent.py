"""Persistent propagation (qhfpe_set_persistent): whole runs of RK4 steps in one cooperative launch with
grid barriers between the Horner stages and the trace reduced in the same launch, against the graph-
replayed launches and the CPU oracle; the bounded barrier wait gives up with QHFPE_ETIMEOUT when a
block never arrives.

The state is the same arithmetic as the graph path (FP64: equal to 1e-14; FP32: the graph path may use
the q-window kernel, whose rounding order differs), the trace sums differ in reduction order only."""
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


def _P(m, precision, persistent, **kw):
    from paper_1706_09590_gb300 import Propagator
    P = Propagator(m, qi.u_table(m), precision=precision, **kw)
    P.set_persistent(persistent)
    return P


MODELS = {
    "harmonic_32x32_d3": qi.harmonic_two_state(),
    "photoiso_np128": qi.photoisomerization_two_state(nq=20, n_p=128, depth=2, n_matsubara=1),
    "three_state": qi.three_state(nq=16, n_p=32, depth=2, n_matsubara=1),
}


@pytest.mark.parametrize("name", list(MODELS))
@pytest.mark.parametrize("precision,tol_state,tol_oracle", [("fp64", 1e-14, 1e-11), ("mixed", 2e-6, 1e-5)])
def test_persistent_steps_match_graph_and_oracle(name, precision, tol_state, tol_oracle):
    m = MODELS[name]
    W = qi.random_state(m, seed=51, hermitian=True)
    out = {}
    for persistent in (False, True):
        P = _P(m, precision, persistent)
        P.set_state(W)
        tr = P.step(37, record_trace=True)[0]  # a 16-step graph chunk count that does not divide
        out[persistent] = (P.get_state(0), tr)
        P.close()
    (Wg, tg), (Wp, tp) = out[False], out[True]
    assert rel(Wp, Wg) < tol_state
    assert rel(tp, tg) < max(tol_state, 1e-13)
    ref_W, ref_tr = oracle.Oracle(m).step(W, 37)
    assert rel(Wp, ref_W) < tol_oracle and rel(tp, ref_tr) < tol_oracle


def test_persistent_replicas_and_response_schedule():
    """Several replicas in one launch, and the third-order schedule (every phase's delays packed as
    replicas) with split pathways: persistent against graph replay."""
    m = MODELS["harmonic_32x32_d3"]
    O = oracle.Oracle(m)
    Weq, _ = O.equilibrate(200)
    R = {}
    for persistent in (False, True):
        P = _P(m, "fp64", persistent)
        P.set_equilibrium(Weq)
        R[persistent] = P.third_order_response(3, 4, [0, 6], 20, split_pathways=True)
        P.close()
    assert np.abs(R[False]).max() > 0
    assert rel(R[True], R[False]) < 1e-12
    W = qi.random_state(m, seed=52, replicas=5)
    out = {}
    for persistent in (False, True):
        P = _P(m, "mixed", persistent, n_replicas=5)
        for r in range(5):
            P.set_state(W[r], replica=r)
        tr = P.step(20, record_trace=True)
        out[persistent] = (np.stack([P.get_state(r) for r in range(5)]), tr)
        P.close()
    assert rel(out[True][0], out[False][0]) < 2e-6
    assert rel(out[True][1], out[False][1]) < 2e-6


def test_persistent_barrier_gives_up_with_etimeout():
    from paper_1706_09590_gb300 import QhfpeError
    m = MODELS["harmonic_32x32_d3"]
    P = _P(m, "fp64", True)
    assert P.barrier_selftest(0, limit_ms=200) == 0
    assert P.barrier_selftest(1, limit_ms=200) == 5  # QHFPE_ETIMEOUT
    # the context stays usable: a fresh handle propagates
    Q = _P(m, "fp64", True)
    Q.set_state(qi.random_state(m, seed=53))
    Q.step(3)
    assert np.all(np.isfinite(Q.get_state(0)))
    Q.close()
    P.close()
    del QhfpeError
