"""The q-window form of the fused stage kernel (FP32 state, np = 128, one or two electronic states)
against the CPU oracle, and against the other fused stage kernel (QHFPE_FUSED_WINDOW=0).

Cases: two states with two Matsubara terms (six tier neighbours, the most the window kernel takes) on
a q grid that is not a multiple of the tile; two states with the Eq. (GMFP) terminator; one state (16-row
tiles) on a ragged grid; a periodic q axis; the learned closure's extra element slot.  Mixed-form
tolerances as in the other parity tests: 2e-5 on one right-hand side, 1e-5 on 12 RK4 steps.
"""
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


def _models():
    two_k2 = qi.photoisomerization_two_state(nq=26, n_p=128, depth=3, n_matsubara=2)
    term = qi.harmonic_two_state(nq=30, n_p=128, pr=(-16.0, 16.0), depth=3)
    # dt inside the RK4 stability bound (the quartic surface reaches ~900 at q + r/2 on this p grid)
    one = qi.single_state(lambda q: 0.5 * q * q + 0.02 * q ** 4, nq=37, n_p=128, pr=(-16.0, 16.0), depth=3,
                          closure=1, dt=0.001)
    per = qi.photoisomerization_two_state(nq=20, n_p=128, depth=2, n_matsubara=1)
    per["periodic_q"] = 1
    return {"two_state_K2": two_k2, "terminator": term, "one_state": one, "periodic": per}


MODELS = _models()


def _P(m, **kw):
    from paper_1706_09590_gb300 import Propagator
    return Propagator(m, qi.u_table(m), precision="mixed", **kw)


@pytest.mark.parametrize("name", list(MODELS))
def test_window_rhs_against_oracle(name):
    m = MODELS[name]
    P = _P(m)
    W = qi.random_state(m, seed=21)
    P.set_state(W)
    Win = P.get_state(0)
    got = P.apply_rhs(0)
    P.close()
    ref = oracle.Oracle(m).rhs(Win)
    assert np.all(np.isfinite(got))
    assert rel(got, ref) < 2e-5, (name, rel(got, ref))


@pytest.mark.parametrize("name", list(MODELS))
def test_window_steps_against_oracle_and_other_kernel(name, monkeypatch):
    m = MODELS[name]
    W = qi.random_state(m, seed=22, hermitian=True)
    ref_W, ref_tr = oracle.Oracle(m).step(W, 12)
    out = {}
    # a pinned tile skips the timed choice between the forms, so that each form certainly runs
    monkeypatch.setenv("QHFPE_TILE_ROWS", "2")
    for flag in ("1", "0"):
        monkeypatch.setenv("QHFPE_FUSED_WINDOW", flag)
        P = _P(m)
        P.set_state(W)
        tr = P.step(12, record_trace=True)[0]
        assert P.stage_form() == int(flag)
        out[flag] = (P.get_state(0), tr)
        P.close()
    got, tr = out["1"]
    assert rel(got, ref_W) < 1e-5 and rel(tr, ref_tr) < 1e-5, (rel(got, ref_W), rel(tr, ref_tr))
    # the two FP32 kernels differ only in rounding order
    assert rel(got, out["0"][0]) < 2e-6


def test_window_replicas_and_single_replica_rhs(monkeypatch):
    """Three replicas with different states in one launch (replica index of each block), and the
    right-hand side of one replica alone (the launch's first-replica offset), against the oracle."""
    m = MODELS["two_state_K2"]
    monkeypatch.setenv("QHFPE_TILE_ROWS", "2")
    W = qi.random_state(m, seed=24, replicas=3, hermitian=True)
    P = _P(m, n_replicas=3)
    for r in range(3):
        P.set_state(W[r], replica=r)
    tr = P.step(6, record_trace=True)
    assert P.stage_form() == 1
    O = oracle.Oracle(m)
    for r in range(3):
        ref_W, ref_tr = O.step(W[r], 6)
        assert rel(P.get_state(r), ref_W) < 1e-5 and rel(tr[r], ref_tr) < 1e-5
    got = P.apply_rhs(1)
    ref = O.rhs(P.get_state(1))
    assert rel(got, ref) < 2e-5
    P.close()


def test_window_learned_closure_slot():
    """The learned closure's W^(N+1) slot is one more tier-up neighbour of the deepest element: with
    loaded weights the window kernel matches the other kernel."""
    from paper_1706_09590_gb300 import Propagator
    import os
    m = qi.harmonic_two_state(nq=24, n_p=128, pr=(-16.0, 16.0), depth=3, closure=2)
    T = qi.u_table(m)
    rng = np.random.default_rng(3)
    from paper_1706_09590_gb300.qhfpe import CLOSURE_N_WEIGHTS
    w = (0.02 * rng.standard_normal(CLOSURE_N_WEIGHTS)).astype(np.float32)
    W = qi.random_state(m, seed=23)
    res = {}
    for flag in ("1", "0"):
        os.environ["QHFPE_FUSED_WINDOW"] = flag
        os.environ["QHFPE_TILE_ROWS"] = "2"
        try:
            P = Propagator(m, T, precision="mixed")
            P.closure_load(w)
            P.set_state(W)
            P.step(5)
            assert P.stage_form() == int(flag)
            res[flag] = P.get_state(0)
            P.close()
        finally:
            os.environ.pop("QHFPE_FUSED_WINDOW", None)
            os.environ.pop("QHFPE_TILE_ROWS", None)
    assert np.all(np.isfinite(res["1"]))
    assert rel(res["1"], res["0"]) < 2e-6
