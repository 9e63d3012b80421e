"""The two-state photoisomerization workload at its full size (96 x 128, depth 8, two Matsubara terms and
the delta-term: 165 elements x 4 pairs, 8.11 M cells) over the stated bath and coupling ranges:
eta in {0.1, 1, 5} x diabatic coupling in {0.2, 0.5, 1, 2} (units of omega_0), dt = 0.8 x the
library's stability bound for each case.

* every case: linear response R1, Eq. (R1), and the transient-absorption response R3(t3, T, 0),
  Eq. (transient-absorption), of the mixed form against the FP64 form, from the same FP64 equilibrium
  state (Sec. III), within 1e-4 relative L2; the wall time of each form is printed.  R1 covers one
  time unit and the TAS response T in {0, 0.25} with t3 up to 0.5, except at eta = 5: there the depth-8
  hierarchy truncated at beta = 1 has growing modes (element norms grow about e^(10 t) in FP64 and in
  the mixed form alike, and FP32 rounding is amplified with them), so the comparison stops at t = 0.5
  (R1) and T + t3 = 0.5 (TAS), before the growth reaches the response;
* the benchmark point (eta 1, coupling 0.5): a short propagation of the full hierarchy on the full grid
  against the CPU oracle (FP64 1e-11, mixed 1e-5 after 6 RK4 steps, traces as well);
* the stiffest corner (eta 5, coupling 2): the right-hand side against the oracle at sampled rows.
"""
import time

import numpy as np
import pytest

import oracle
import qhfpe_inputs as qi

pytestmark = pytest.mark.gpu

ETAS = (0.1, 1.0, 5.0)
COUPLINGS = (0.2, 0.5, 1.0, 2.0)


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def rel(a, b):
    return np.linalg.norm(np.ravel(a - b)) / max(np.linalg.norm(np.ravel(b)), 1e-300)


def window(eta):
    """(R1 length, second waiting time, t3 length) in time units: the unstable eta = 5 hierarchy is
    compared before its growing modes reach the response."""
    return (0.5, 0.125, 0.375) if eta >= 5 else (1.0, 0.25, 0.5)


def _case(eta, coupling):
    from paper_1706_09590_gb300 import Propagator
    m = qi.photoisomerization_two_state(eta=eta, coupling=coupling)
    T = qi.u_table(m)
    probe = Propagator(m, T, precision="fp64")
    dt = 0.8 * probe.max_stable_dt()
    probe.close()
    return m, T, dt


@pytest.mark.parametrize("coupling", COUPLINGS)
@pytest.mark.parametrize("eta", ETAS)
def test_mixed_vs_fp64_linear_and_transient_absorption(eta, coupling):
    import torch
    from paper_1706_09590_gb300 import Propagator
    m, T, dt = _case(eta, coupling)
    t_r1, t_T, t_t3 = window(eta)
    n_r1 = int(round(t_r1 / dt))
    t2 = [0, int(round(t_T / dt))]
    n_t3 = int(round(t_t3 / dt))
    E = Propagator(m, T, precision="fp64", dt=dt)
    E.equilibrate(300)
    Weq = E.get_state(0)
    E.close()
    R1, R3, wall = {}, {}, {}
    for prec in ("fp64", "mixed"):
        P = Propagator(m, T, precision=prec, dt=dt)
        P.set_equilibrium(Weq)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        R1[prec] = P.linear_response(n_r1)
        R3[prec] = P.third_order_response(1, 1, t2, n_t3)
        torch.cuda.synchronize()
        wall[prec] = time.perf_counter() - t0
        P.close()
    e1, e3 = rel(R1["mixed"], R1["fp64"]), rel(R3["mixed"], R3["fp64"])
    print(f"eta {eta} coupling {coupling} dt {dt:.3e}: R1 {e1:.2e}, TAS R3 {e3:.2e}; "
          f"wall fp64 {wall['fp64']:.2f} s, mixed {wall['mixed']:.2f} s")
    assert np.all(np.isfinite(R1["fp64"])) and np.all(np.isfinite(R3["fp64"]))
    assert np.abs(R1["fp64"]).max() > 1e-3 and np.abs(R3["fp64"]).max() > 1e-3
    assert e1 < 1e-4
    assert e3 < 1e-4


@pytest.fixture(scope="module")
def bench_point_reference():
    """Six oracle RK4 steps of the full hierarchy at the benchmark point (computed once)."""
    m, T, dt = _case(1.0, 0.5)
    W = qi.random_state(m, seed=77, hermitian=True)
    ref_W, ref_tr = oracle.Oracle(dict(m, dt=dt), T).step(W, 6)
    return m, T, dt, W, ref_W, ref_tr


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-11), ("mixed", 1e-5)])
def test_full_size_steps_against_oracle(bench_point_reference, precision, tol):
    from paper_1706_09590_gb300 import Propagator
    m, T, dt, W, ref_W, ref_tr = bench_point_reference
    P = Propagator(m, T, precision=precision, dt=dt)
    P.set_state(W)
    tr = P.step(6, record_trace=True)[0]
    got = P.get_state(0)
    P.close()
    assert rel(got, ref_W) < tol
    assert rel(tr, ref_tr) < tol


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-12), ("mixed", 2e-5)])
def test_stiffest_case_rhs_at_sampled_rows(precision, tol):
    from paper_1706_09590_gb300 import Propagator
    m, T, dt = _case(5.0, 2.0)
    P = Propagator(m, T, precision=precision, dt=dt)
    W = qi.random_state(m, seed=78)
    P.set_state(W)
    Win = P.get_state(0)
    got = P.apply_rhs(0)
    n_elem = got.shape[0]
    P.close()
    rng = np.random.default_rng(5)
    rows = [(e, j, k, i) for e in (0, 1, n_elem // 2, n_elem - 1) for j in range(2) for k in range(2)
            for i in (0, 2, m["nq"] // 2, m["nq"] - 1)]
    rows += [(int(rng.integers(n_elem)), int(rng.integers(2)), int(rng.integers(2)), int(rng.integers(m["nq"])))
             for _ in range(16)]
    ref = oracle.Oracle(m, T).rhs_rows(Win, rows)
    sel = np.stack([got[e, j, k, i] for e, j, k, i in rows])
    assert rel(sel, ref) < tol
