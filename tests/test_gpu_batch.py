"""Heterogeneous batches through the C ABI: members that differ in q grid and ranges, surfaces, bath,
depth, closure, dt and replica count, advanced together (each Horner stage of the RK4 step of
Eq. (heom), Sec. III, one launch for all members), against the same members stepped alone and against
the oracle; the argument checks."""
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


def _P(m, precision, n_replicas=1):
    from paper_1706_09590_gb300 import Propagator
    return Propagator(m, qi.u_table(m), precision=precision, n_replicas=n_replicas)


# np = 32, two states; everything else differs
MEMBERS = [
    (qi.harmonic_two_state(nq=32, n_p=32, depth=3), 1),
    (qi.harmonic_two_state(nq=20, n_p=32, qr=(-6.0, 7.0), depth=5, closure=0, dt=0.008, eta=0.3), 2),
    (qi.photoisomerization_two_state(nq=40, n_p=32, depth=2, n_matsubara=1, dt=2e-3), 1),
]


# np = 64, three states, different grids, depths and bath modes
MEMBERS_S3 = [
    (qi.three_state(nq=12, n_p=64, depth=1, n_matsubara=1), 2),
    (qi.three_state(nq=20, n_p=64, qr=(-8.0, 9.0), depth=2, n_matsubara=0, dt=5e-4), 1),
]


def _fill(P, k):
    for r in range(P.n_replicas):
        P.set_state(qi.random_state(P.model, seed=300 + 10 * k + r, hermitian=True), r)


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-12), ("mixed", 1e-5)])
@pytest.mark.parametrize("tile", [None, 3])
def test_batch_equals_members_alone(precision, tol, tile, monkeypatch):
    from paper_1706_09590_gb300 import Batch
    if tile is not None:
        monkeypatch.setenv("QHFPE_TILE_ROWS", str(tile))
    batched = [_P(m, precision, n) for m, n in MEMBERS]
    alone = [_P(m, precision, n) for m, n in MEMBERS]
    for k, (a, b) in enumerate(zip(batched, alone)):
        _fill(a, k)
        _fill(b, k)
    B = Batch(batched)
    n_steps = 21  # one captured 16-step chunk and five single steps
    tr_b = B.step(n_steps, record_trace=True)
    if tile is not None:
        assert B.tile_rows() == tile
    for k, (a, b) in enumerate(zip(batched, alone)):
        tr_a = b.step(n_steps, record_trace=True)
        assert tr_b[k].shape == tr_a.shape
        assert rel(tr_b[k], tr_a) <= tol, (k, rel(tr_b[k], tr_a))
        for r in range(a.n_replicas):
            assert rel(a.get_state(r), b.get_state(r)) <= tol, (k, r)
    # without traces, and a second call on the captured graphs
    B.step(3)
    for a, b in zip(batched, alone):
        b.step(3)
        assert rel(a.get_state(a.n_replicas - 1), b.get_state(b.n_replicas - 1)) <= tol
    B.close()


def test_batch_member_against_the_oracle():
    from paper_1706_09590_gb300 import Batch
    Ps = [_P(m, "fp64", n) for m, n in MEMBERS]
    for k, P in enumerate(Ps):
        _fill(P, k)
    W = [P.get_state(P.n_replicas - 1) for P in Ps]
    B = Batch(Ps)
    tr = B.step(4, record_trace=True)
    for k, (m, _) in enumerate(MEMBERS):
        ref_W, ref_tr = oracle.Oracle(m).step(W[k], 4)
        assert rel(Ps[k].get_state(Ps[k].n_replicas - 1), ref_W) < 1e-11, k
        assert rel(tr[k][-1], ref_tr) < 1e-11, k
    B.close()


def test_batch_argument_checks():
    from paper_1706_09590_gb300 import Batch, QhfpeError
    a = _P(MEMBERS[0][0], "fp64")
    with pytest.raises(QhfpeError):  # the same handle twice
        Batch([a, a])
    b = _P(qi.harmonic_two_state(nq=16, n_p=64, depth=2), "fp64")
    with pytest.raises(QhfpeError):  # another np
        Batch([a, b])
    c = _P(MEMBERS[0][0], "mixed")
    with pytest.raises(QhfpeError):  # another precision
        Batch([a, c])
    d = _P(qi.harmonic_two_state(nq=16, n_p=64, depth=2), "bf16x3")
    with pytest.raises(QhfpeError):  # the tensor-core form
        Batch([d])
    for P in (a, b, c, d):
        P.close()


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-12), ("mixed", 1e-5)])
def test_three_state_batch_equals_members_alone(precision, tol):
    from paper_1706_09590_gb300 import Batch
    batched = [_P(m, precision, n) for m, n in MEMBERS_S3]
    alone = [_P(m, precision, n) for m, n in MEMBERS_S3]
    for k, (a, b) in enumerate(zip(batched, alone)):
        _fill(a, k)
        _fill(b, k)
    B = Batch(batched)
    tr_b = B.step(5, record_trace=True)
    for k, (a, b) in enumerate(zip(batched, alone)):
        tr_a = b.step(5, record_trace=True)
        assert rel(tr_b[k], tr_a) <= tol, k
        for r in range(a.n_replicas):
            assert rel(a.get_state(r), b.get_state(r)) <= tol, (k, r)
    B.close()
