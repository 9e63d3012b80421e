"""The paper's own photoisomerization workload (Sec. III): displaced Morse diabats with a Gaussian
diabatic coupling on the 512 x 128 mesh (q in [-20, 80), p in [-25, 25)), beta = 0.48, in the
underdamped case (Drude zeta = 0.4, gamma = 5, depth 5) and the overdamped case (zeta = 4, the
depth-0 quantum Fokker-Planck limit).

* one right-hand side at full size against the oracle at sampled rows;
* RK4 steps on a coarser mesh of the same model against the oracle;
* the linear absorption spectrum: mixed form against the FP64 form (1e-4 on R1), and the broadened
  absorption peak that the paper reports near 20,000 cm^-1 (200 omega_0 with omega_0 = 100 cm^-1).
"""
import numpy as np
import pytest

import oracle
import qhfpe_inputs as qi

pytestmark = pytest.mark.gpu

BATHS = ["underdamped", "overdamped"]


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


@pytest.mark.parametrize("bath", BATHS)
@pytest.mark.parametrize("precision,tol", [("fp64", 1e-12), ("mixed", 2e-5)])
def test_full_size_rhs_at_sampled_rows(bath, precision, tol):
    m = qi.morse_photoisomerization(bath=bath)
    P = _P(m, precision)
    assert P.n_elem == (6 if bath == "underdamped" else 1)
    P.set_state(qi.random_state(m, seed=61))
    Win = P.get_state(0)
    if precision != "fp64":
        Win[1:] = Win[1:].astype(np.complex64).astype(np.complex128)
    got = P.apply_rhs(0)
    P.close()
    nq, n_elem = m["nq"], Win.shape[0]
    rng = np.random.default_rng(6)
    rows = [(e, j, k, i) for e in sorted({0, n_elem - 1}) for j in range(2) for k in range(2)
            for i in (0, 2, nq // 2, nq - 1)]
    rows += [(int(rng.integers(n_elem)), int(rng.integers(2)), int(rng.integers(2)), int(rng.integers(nq)))
             for _ in range(12)]
    ref = oracle.Oracle(m).rhs_rows(Win, rows)
    sel = np.stack([got[e, j, k, i] for e, j, k, i in rows])
    assert np.all(np.isfinite(got))
    assert rel(sel, ref) < tol


@pytest.mark.parametrize("bath", BATHS)
def test_steps_on_a_coarser_mesh(bath):
    m = qi.morse_photoisomerization(nq=64, n_p=32, bath=bath)
    O = oracle.Oracle(m)
    W = qi.random_state(m, seed=62, hermitian=True)
    ref_W, ref_tr = O.step(W, 20)
    P = _P(m, "fp64")
    P.set_state(W)
    tr = P.step(20, record_trace=True)[0]
    assert rel(P.get_state(0), ref_W) < 1e-11
    assert rel(tr, ref_tr) < 1e-11
    Q = _P(m, "mixed")
    Q.set_state(W)
    trm = Q.step(20, record_trace=True)[0]
    assert rel(Q.get_state(0)[0], ref_W[0]) < 1e-5
    assert rel(trm, ref_tr) < 1e-5


@pytest.mark.parametrize("bath", BATHS)
def test_linear_absorption_peak_near_20000_wavenumbers(bath):
    m = qi.morse_photoisomerization(bath=bath)
    T = qi.u_table(m)
    from paper_1706_09590_gb300 import Propagator
    E = Propagator(m, T, precision="fp64")
    E.equilibrate(1500)
    Weq = E.get_state(0)
    E.close()
    omega = np.linspace(100.0, 300.0, 401)
    R, I = {}, {}
    for precision in ("fp64", "mixed"):
        P = Propagator(m, T, precision=precision)
        P.set_equilibrium(Weq)
        R[precision] = P.linear_response(1500)
        I[precision] = P.spectrum_absorption(R[precision], m["dt"], omega)
        P.close()
    assert np.all(np.isfinite(R["fp64"]))
    err = rel(R["mixed"], R["fp64"])
    print(bath, "R1 mixed vs FP64 relative L2", err)
    assert err < 1e-4
    peak = omega[np.argmax(I["fp64"])]
    print(bath, "absorption peak (omega_0 = 100 cm^-1):", peak)
    assert 190.0 <= peak <= 215.0
    assert omega[np.argmax(I["mixed"])] == peak
    # a broadened band: the half maximum spans tens of omega_0 around the peak
    band = omega[I["fp64"] >= 0.5 * I["fp64"].max()]
    assert band.min() < peak - 20 and band.max() > peak + 20
