"""The batched 2D schedule at the full t3 length of the 2D-spectrum workload (harmonic two-state model,
32 x 32, depth 3, t3 = 512 RK4 steps, t1 stride 8, waiting times 0 and 100 steps) against the CPU
oracle on a sub-schedule of the full one: the first two t1 delays and the first two waiting times, both
pathways of the first interaction (Eq. (R3) with the ket-side mu^-> and the bra-side -mu^<- jobs
batched as replicas).  FP64 within 1e-10, the mixed form within 1e-4, as the shorter schedules of the
parity tests."""
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


@pytest.fixture(scope="module")
def reference():
    m = qi.harmonic_two_state()
    O = oracle.Oracle(m)
    Weq, _ = O.equilibrate(300)
    args = (2, 8, [0, 100], 512)
    ket = O.third_order_response(Weq, *args, first=oracle.LEFT)
    bra = O.third_order_response(Weq, *args, first=oracle.RIGHT)
    return m, Weq, args, ket, bra


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-10), ("mixed", 1e-4)])
def test_full_t3_sub_schedule_matches_oracle(reference, precision, tol):
    from paper_1706_09590_gb300 import Propagator
    m, Weq, args, ket, bra = reference
    P = Propagator(m, qi.u_table(m), precision=precision)
    P.set_equilibrium(Weq)
    got = P.third_order_response(*args, split_pathways=True)
    P.close()
    assert np.abs(ket).max() > 0 and np.abs(bra).max() > 0
    assert rel(got[0], ket) < tol and rel(got[1], bra) < tol, (rel(got[0], ket), rel(got[1], bra))
