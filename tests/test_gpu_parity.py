"""Parity of the CUDA library (through the C ABI) with the FP64 CPU oracle, element by element.

Tolerances: FP64 form 1e-10 relative L2 on states, traces, responses and spectra (the oracle uses
classic RK4 and direct circulant sums, the library the Horner form and FFTs, so only rounding order
differs); mixed forms 1e-4 on responses (the accuracy target for the reduced-precision forms) and
bounds derived from FP32 rounding on single right-hand-side evaluations.
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
    import paper_1706_09590_gb300 as q
    q.lib()


def _P(model, precision="fp64", **kw):
    from paper_1706_09590_gb300 import Propagator
    return Propagator(model, qi.u_table(model), precision=precision, **kw)


def rel(a, b):
    return np.linalg.norm(np.ravel(a - b)) / max(np.linalg.norm(np.ravel(b)), 1e-300)


def _models():
    h = qi.harmonic_two_state()  # 32 x 32, depth 3, terminator
    ph = qi.photoisomerization_two_state(nq=24, n_p=32, depth=3, n_matsubara=2)
    ph_per = qi.photoisomerization_two_state(nq=13, n_p=16, depth=2, n_matsubara=1)
    ph_per["periodic_q"] = 1
    three = qi.three_state(nq=16, n_p=16, depth=2, n_matsubara=1)
    single = qi.single_state(lambda q: 0.5 * q * q, nq=20, n_p=8, depth=0, closure=1)
    big_np = qi.harmonic_two_state(nq=6, n_p=512, qr=(-8, 8), pr=(-40, 40), depth=1)
    # p = 0 falls inside one lane's run of p values (l = 31 with two values per lane): the fused
    # kernel's generic seven-row q-stencil path
    asym_p = qi.photoisomerization_two_state(nq=20, n_p=64, pr=(-7.75, 8.25), depth=2, n_matsubara=1)
    return {"harmonic": h, "photoiso": ph, "ragged_periodic": ph_per, "three_state": three, "single": single,
            "np512": big_np, "asym_p": asym_p}


MODELS = _models()
TERMS = [1, 2, 4, 8, 16, 31]


@pytest.mark.parametrize("name", list(MODELS))
def test_rhs_terms_fp64(name):
    m = MODELS[name]
    O = oracle.Oracle(m)
    P = _P(m)
    W = qi.random_state(m, seed=11)
    P.set_state(W)
    assert rel(P.get_state(0), W) == 0.0
    for t in TERMS:
        ref = O.rhs(W, t)
        got = P.apply_rhs(0, t)
        if np.linalg.norm(ref) == 0:
            assert np.linalg.norm(got) == 0
        else:
            assert rel(got, ref) < 1e-12, (name, t, rel(got, ref))


@pytest.mark.parametrize("name", ["harmonic", "photoiso", "three_state", "asym_p"])
def test_rhs_mixed(name):
    m = MODELS[name]
    O = oracle.Oracle(m)
    P = _P(m, "mixed")
    W = qi.random_state(m, seed=12)
    P.set_state(W)
    got = P.get_state(0)
    # tier 0 is held in FP64, the rest is rounded to FP32
    assert rel(got[0], W[0]) == 0.0
    assert rel(got, W) < 1e-7
    for t in TERMS:
        ref = O.rhs(P.get_state(0).astype(np.complex64).astype(np.complex128), t)
        assert rel(P.apply_rhs(0, t), ref) < 2e-5, (name, t)


@pytest.mark.parametrize("name", ["harmonic", "photoiso", "three_state", "ragged_periodic"])
def test_steps_and_traces_fp64(name):
    m = MODELS[name]
    O = oracle.Oracle(m)
    P = _P(m)
    W = qi.random_state(m, seed=13, hermitian=True)
    ref_W, ref_tr = O.step(W, 12)
    P.set_state(W)
    tr = P.step(12, record_trace=True)[0]
    assert rel(P.get_state(0), ref_W) < 1e-11
    assert rel(tr, ref_tr) < 1e-11
    # chunked graph replays + remainder: 16 + 3 steps equal 19 single steps of the oracle
    ref_W2, ref_tr2 = O.step(ref_W, 19)
    tr2 = P.step(19, record_trace=True)[0]
    assert rel(P.get_state(0), ref_W2) < 1e-11
    assert rel(tr2, ref_tr2) < 1e-11


TILE_MODELS = {
    "photoiso_s2": qi.photoisomerization_two_state(nq=27, n_p=128, depth=2, n_matsubara=2),
    "three_s3": qi.three_state(nq=21, n_p=32, depth=2, n_matsubara=1),
    "single_s1": qi.single_state(lambda q: 0.5 * q * q + 0.05 * q ** 4, nq=37, n_p=64, depth=3, closure=1),
    "asym_p": MODELS["asym_p"],
}


@pytest.mark.parametrize("tile", [1, 2, 3, 4, 6, 8, 16])
@pytest.mark.parametrize("name", list(TILE_MODELS))
@pytest.mark.parametrize("precision,tol", [("fp64", 1e-12), ("mixed", 2e-5)])
def test_rhs_every_tile(name, tile, precision, tol, monkeypatch):
    """The fused stage kernel at each tile height (q rows per block; ragged last tiles, one or several
    runs of rows per warp) against the oracle's right-hand side."""
    m = TILE_MODELS[name]
    monkeypatch.setenv("QHFPE_TILE_ROWS", str(tile))
    P = _P(m, precision)
    P.set_state(qi.random_state(m, seed=31, hermitian=True))
    P.step(1)
    W = P.get_state(0)
    ref = oracle.Oracle(m).rhs(W if precision == "fp64" else W.astype(np.complex64).astype(np.complex128), 31)
    assert rel(P.apply_rhs(0, 31), ref) < tol, (name, tile, precision)


def test_steps_mixed():
    m = MODELS["harmonic"]
    O = oracle.Oracle(m)
    P = _P(m, "mixed")
    W = qi.random_state(m, seed=14, hermitian=True)
    ref_W, ref_tr = O.step(W, 40)
    P.set_state(W)
    tr = P.step(40, record_trace=True)[0]
    assert rel(P.get_state(0)[0], ref_W[0]) < 1e-5
    assert rel(tr, ref_tr) < 1e-5


def test_replicas_independent_and_fork():
    m = MODELS["photoiso"]
    O = oracle.Oracle(m)
    P = _P(m, n_replicas=3)
    Ws = [qi.random_state(m, seed=20 + r) for r in range(3)]
    for r, W in enumerate(Ws):
        P.set_state(W, r)
    tr = P.step(5, record_trace=True)
    for r, W in enumerate(Ws):
        ref_W, ref_tr = O.step(W, 5)
        assert rel(P.get_state(r), ref_W) < 1e-11
        assert rel(tr[r], ref_tr) < 1e-11
    P.fork(1, [0, 2])
    a = P.get_state(1)
    assert rel(P.get_state(0), a) == 0 and rel(P.get_state(2), a) == 0
    # zero steps: only the initial trace
    tr0 = P.step(0, record_trace=True)
    assert tr0.shape == (3, 1)
    assert abs(tr0[1, 0] - O.trace(a)) < 1e-12 * max(1, abs(O.trace(a)))


@pytest.mark.parametrize("side", [1, 2, 3])
def test_dipole(side):
    m = MODELS["three_state"]
    O = oracle.Oracle(m)
    P = _P(m, n_replicas=2)
    W = qi.random_state(m, seed=30)
    P.set_state(W, 0)
    P.set_state(W, 1)
    P.apply_dipole(side, replicas=[1])
    assert rel(P.get_state(1), O.apply_dipole(W, side)) < 1e-15
    assert rel(P.get_state(0), W) == 0
    t = P.trace()
    assert abs(t[1] - O.trace(O.apply_dipole(W, side))) < 1e-12 * max(1.0, abs(t[1]))


def test_equilibrate_fp64():
    m = MODELS["harmonic"]
    O = oracle.Oracle(m)
    P = _P(m)
    ref, ref_res = O.equilibrate(300)
    res = P.equilibrate(300)
    assert rel(P.get_state(0), ref) < 1e-11
    assert res == pytest.approx(ref_res, rel=1e-6)


def test_equilibrate_to_tolerance_fp64():
    """Stationarity-driven equilibration (Sec. III): the run stops at the first check where the
    residual ||L W|| / ||W|| is below tol.  The oracle, propagated the same number of steps, gives the
    same state, a residual below tol, and a residual at tol or above one check earlier."""
    m = MODELS["harmonic"]
    O = oracle.Oracle(m)
    P = _P(m)
    M = 40
    tol = 1e-4  # the Boltzmann start is at 1.9e-3; the oracle passes 1e-4 between 320 and 640 steps
    n, res = P.equilibrate_to(tol, t_max=60.0, check_every=M)
    assert 320 < n <= 640 and n % M == 0
    ref, ref_res = O.equilibrate(n)
    assert rel(P.get_state(0), ref) < 1e-11
    assert res == pytest.approx(ref_res, rel=1e-6)
    assert ref_res < tol
    assert O.equilibrate(n - M)[1] >= tol
    # t_max ends the run when tol cannot be met: 1.05 time units = 105 steps of 0.01 (a partial check)
    n2, res2 = P.equilibrate_to(1e-300, t_max=1.05, check_every=M)
    assert n2 == 105
    ref2, ref_res2 = O.equilibrate(105)
    assert rel(P.get_state(0), ref2) < 1e-11
    assert res2 == pytest.approx(ref_res2, rel=1e-6)


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-10), ("mixed", 1e-4)])
def test_linear_response(precision, tol):
    m = MODELS["harmonic"]
    O = oracle.Oracle(m)
    Weq, _ = O.equilibrate(400)
    ref = O.linear_response(Weq, 300)
    P = _P(m, precision)
    P.set_equilibrium(Weq)
    got = P.linear_response(300)
    assert rel(got, ref) < tol


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-10), ("mixed", 1e-4)])
def test_third_order_response_split(precision, tol):
    m = qi.harmonic_two_state(nq=16, n_p=16, depth=2)
    O = oracle.Oracle(m)
    Weq, _ = O.equilibrate(100)
    args = (3, 4, [0, 3, 7], 10)
    ket = O.third_order_response(Weq, *args, first=oracle.LEFT)
    bra = O.third_order_response(Weq, *args, first=oracle.RIGHT)
    P = _P(m, precision)
    P.set_equilibrium(Weq)
    got = P.third_order_response(*args, split_pathways=True)
    assert rel(got[0], ket) < tol
    assert rel(got[1], bra) < tol
    full = P.third_order_response(*args, split_pathways=False)
    assert rel(full, ket + bra) < tol
    # transient absorption is the n_t1 = 1 schedule
    tas = P.third_order_response(1, 0, [0, 5], 10)
    ref_tas = O.third_order_response(Weq, 1, 0, [0, 5], 10)
    assert rel(tas, ref_tas) < tol


def test_spectra():
    m = MODELS["harmonic"]
    P = _P(m)
    rng = np.random.default_rng(3)
    R1 = rng.normal(size=301) + 1j * rng.normal(size=301)
    om = np.linspace(-20, 20, 57)
    assert rel(P.spectrum_absorption(R1, 0.01, om), oracle.absorption(R1, 0.01, om)) < 1e-12
    R3 = rng.normal(size=(9, 41)) + 1j * rng.normal(size=(9, 41))
    w1 = np.linspace(-15, 15, 31)
    w3 = np.linspace(-12, 12, 25)
    nr, re, corr = P.spectrum_2d(R3, 0.08, 0.01, w1, w3)
    rnr, rre, rcorr = oracle.two_d(R3, 0.08, 0.01, w1, w3)
    assert rel(nr, rnr) < 1e-12 and rel(re, rre) < 1e-12 and rel(corr, rcorr) < 1e-12


def test_bath_and_hierarchy_match_oracle():
    for name in ("photoiso", "three_state", "harmonic"):
        m = MODELS[name]
        O = oracle.Oracle(m)
        P = _P(m)
        assert (P.hierarchy() == O.hierarchy()).all()
        a, b = P.bath_coefficients(), O.coefficients()
        for k in ("gamma", "r", "c"):
            assert np.allclose(a[k], b[k], rtol=1e-14, atol=0)
        assert a["cdelta"] == pytest.approx(b["cdelta"], rel=1e-12, abs=1e-15)


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-12), ("mixed", 2e-5), ("bf16x3", 2e-4)])
def test_full_size_rhs(precision, tol):
    """The benchmark's workload (96 x 128 grid, depth 8, three modes, 165 elements, two states): one
    full right-hand side in the benchmark's launch configuration against the oracle (for the tensor-core
    form: 495 row tiles, several per persistent CTA)."""
    m = qi.photoisomerization_two_state()
    O = oracle.Oracle(m)
    P = _P(m, precision)
    W = qi.random_state(m, seed=40)
    P.set_state(W)
    Win = P.get_state(0)
    if precision != "fp64":
        Win[1:] = Win[1:].astype(np.complex64).astype(np.complex128)
    ref = O.rhs(Win)
    got = P.apply_rhs(0)
    assert rel(got, ref) < tol


def test_isolated_system_decouples_the_hierarchy():
    """eta = 0 (no bath): the couplings to lower tiers vanish (c_k = r_k = 0 in Eq. (heom)), so higher
    tiers that start at zero are never sourced and the zeroth tier evolves as the depth-0 hierarchy,
    i.e. the isolated system's Wigner-space equation of motion; against each other and the oracle."""
    m = qi.harmonic_two_state(nq=20, n_p=32, depth=2, eta=0.0, closure=0)
    W = qi.random_state(m, seed=41, hermitian=True)
    W[1:] = 0
    out = []
    for mm, WW in ((m, W), (dict(m, depth=0), W[:1])):
        P = _P(mm, "fp64")
        P.set_state(WW)
        P.step(20)
        out.append(P.get_state(0))
        P.close()
    assert np.abs(out[0][1:]).max() == 0.0
    assert rel(out[0][0], out[1][0]) < 1e-13
    ref, _ = oracle.Oracle(m).step(W, 20)
    assert rel(out[0], ref) < 1e-11


def test_set_state_rejects_non_finite():
    from paper_1706_09590_gb300 import QhfpeError
    m = MODELS["harmonic"]
    P = _P(m)
    W = qi.random_state(m, seed=50)
    W[1, 0, 1, 3, 4] = np.nan
    with pytest.raises(QhfpeError) as ei:
        P.set_state(W)
    assert ei.value.status == 4
    P.set_state(qi.random_state(m, seed=51))  # the handle stays usable
    P.step(1)


def test_device_wait_gives_up_and_context_survives():
    """A device wait on a flag that nothing sets returns ETIMEOUT after its limit; the handle and the
    context keep working afterwards."""
    m = MODELS["harmonic"]
    P = _P(m)
    assert P.wait_selftest(release=1, limit_ms=200) == 0
    assert P.wait_selftest(release=0, limit_ms=200) == 5
    W = qi.random_state(m, seed=80)
    P.set_state(W)
    P.step(3)
    O = oracle.Oracle(m)
    assert rel(P.get_state(0), O.step(W, 3)[0]) < 1e-11


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_resume_is_bitwise_identical(precision):
    """Checkpoint/resume: 7 + 9 steps through get_state/set_state on a second handle equal 16 steps."""
    m = MODELS["photoiso"]
    W = qi.random_state(m, seed=81)
    A = _P(m, precision)
    A.set_state(W)
    trA = A.step(16, record_trace=True)[0]
    B = _P(m, precision)
    B.set_state(W)
    trB1 = B.step(7, record_trace=True)[0]
    ck = B.get_state(0)
    C = _P(m, precision)
    C.set_state(ck)
    trC = C.step(9, record_trace=True)[0]
    assert np.array_equal(A.get_state(0), C.get_state(0))
    assert np.array_equal(trA[:8], trB1) and np.array_equal(trA[7:], trC)
