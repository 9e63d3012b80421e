"""The three-state workload at its full size (256 x 256 grid, depth 10, three bath modes: 286 hierarchy
elements x 9 electronic pairs, 168.7 M cells) through the C ABI: one right-hand side against the oracle
at sampled rows (all pairs, tier 0 and the deepest tier, q rows at both edges and inside), and a short
transient-absorption schedule (t1 = 0, two waiting times) in the mixed form against the FP64 form."""
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


def _sample_rows(n_elem, S, nq, seed=4):
    rng = np.random.default_rng(seed)
    rows = []
    for e in (0, 1, n_elem // 2, n_elem - 1):
        for j in range(S):
            for k in range(S):
                i = (0, 1, 2, nq - 1, nq - 3, nq // 2, int(rng.integers(nq)))[(3 * j + k + e) % 7]
                rows.append((e, j, k, i))
    for _ in range(16):
        rows.append((int(rng.integers(n_elem)), int(rng.integers(S)), int(rng.integers(S)), int(rng.integers(nq))))
    return rows


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-12), ("mixed", 2e-5)])
def test_full_size_rhs_at_sampled_rows(precision, tol):
    m = qi.three_state()
    assert qi.n_elements(m) == 286
    P = _P(m, precision)
    W = qi.random_state(m, seed=41)
    P.set_state(W)
    del W
    Win = P.get_state(0)
    if precision != "fp64":
        Win[1:] = Win[1:].astype(np.complex64).astype(np.complex128)
    got = P.apply_rhs(0)
    P.close()
    rows = _sample_rows(Win.shape[0], m["S"], m["nq"])
    ref = oracle.Oracle(m).rhs_rows(Win, rows)
    sel = np.stack([got[e, j, k, i] for e, j, k, i in rows])
    assert np.all(np.isfinite(got))
    assert rel(sel, ref) < tol
    for r in range(len(rows)):  # no single row far off
        assert rel(sel[r], ref[r]) < 10 * tol


def test_full_size_transient_absorption_mixed_vs_fp64():
    m = qi.three_state()
    n_eq, t2, n_t3 = 400, [0, 60], 120
    R = {}
    for precision in ("fp64", "mixed"):
        P = _P(m, precision)
        P.equilibrate(n_eq)
        Weq = P.get_state(0)
        P.set_equilibrium(Weq)
        R[precision] = P.third_order_response(1, 1, t2, n_t3)
        P.close()
    assert np.all(np.isfinite(R["fp64"]))
    assert np.abs(R["fp64"]).max() > 0
    err = rel(R["mixed"], R["fp64"])
    print("three-state TAS response, mixed vs FP64 relative L2:", err)
    assert err < 1e-4
