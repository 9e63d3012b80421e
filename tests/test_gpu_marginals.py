"""Adiabatic-basis wavepacket marginals (Sec. III, "Wavepacket dynamics") through the C ABI.

* parity with the numpy oracle on random states (two and three states, FP64 and mixed forms, a
  non-zero replica index, the paper's 512 x 128 Morse mesh);
* the paper's use of them: the two-pulse state W(t2) = G(t2) mu^-> mu^<- W_eq of the underdamped
  Morse model.  The pump puts the ground-state distribution on the excited diabat near q = 0, the
  packet slides down that surface towards its minimum (q = 18.98) and crosses the coupling region
  (q* = 10.28) fast, so past the crossing much of it lives on the lower adiabatic surface (the
  breakdown of the adiabatic picture that the paper reports for the underdamped case).  Mixed and FP64
  forms agree.
"""
import numpy as np
import pytest

import qhfpe_inputs as qi
from oracle import marginals as om

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


MODELS = {
    "harmonic": qi.harmonic_two_state(),
    "three_state": qi.three_state(nq=16, n_p=16, depth=2, n_matsubara=1),
    "morse_full": qi.morse_photoisomerization(),
}


@pytest.mark.parametrize("name", list(MODELS))
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_marginals_match_the_oracle(name, precision):
    m = MODELS[name]
    P = _P(m, precision, n_replicas=2)
    dp = (m["p_max"] - m["p_min"]) / m["np"]
    for r, seed in ((0, 91), (1, 92)):
        W = qi.random_state(m, seed=seed, hermitian=True)
        P.set_state(W, r)
        ref = om.adiabatic_marginals(W, qi.u_table(m), dp)
        got = P.adiabatic_marginals(r)
        assert got.shape == (m["S"], m["S"], m["nq"])
        # the zeroth tier is held in FP64 in both forms
        assert rel(got, ref) < 1e-12, (name, precision, r)
    P.close()


def test_pumped_morse_packet_crosses_to_the_lower_adiabatic_surface():
    m = qi.morse_photoisomerization()
    T = qi.u_table(m)
    from paper_1706_09590_gb300 import Propagator, LEFT, RIGHT
    E = Propagator(m, T, precision="fp64")
    E.equilibrate(1500)
    Weq = E.get_state(0)
    E.close()
    q = qi.axis(m["nq"], m["q_min"], m["q_max"])
    dq = (m["q_max"] - m["q_min"]) / m["nq"]
    marg = {}
    for precision in ("fp64", "mixed"):
        P = Propagator(m, T, precision=precision)
        P.set_state(Weq)
        P.apply_dipole(RIGHT)
        P.apply_dipole(LEFT)  # mu^-> mu^<- W_eq: the ground distribution moved to the excited diabat
        out = []
        done = 0
        for t2 in (0, 400, 940, 1500):
            if t2 > done:
                P.step(t2 - done)
            done = t2
            out.append(P.adiabatic_marginals(0))
        marg[precision] = np.stack(out)
        P.close()
    a, b = marg["mixed"], marg["fp64"]
    assert rel(a, b) < 1e-5
    pop_up = b[:, 1, 1].real.sum(axis=-1) * dq
    pop_lo = b[:, 0, 0].real.sum(axis=-1) * dq
    total = pop_up + pop_lo
    assert np.allclose(total, total[0], rtol=1e-3)  # populations conserved (open q edges: far away)
    # at t2 = 0 everything sits on the upper adiabatic surface near q = 0
    assert pop_lo[0] < 1e-3 * total[0]
    mean_q = (b[:, 1, 1].real * q).sum(axis=-1) * dq / np.maximum(pop_up, 1e-300)
    print("upper-surface populations", pop_up / total, "mean q", mean_q)
    assert np.all(np.diff(mean_q) > 1.0)  # sliding down the excited surface
    # as the packet passes q* = 10.28 population appears on the lower adiabatic surface beyond the
    # crossing: a few per cent at t2 = 0.94 / omega_0, a large part by t2 = 1.5 / omega_0
    beyond = q > 10.28
    lo_beyond = b[2:, 0, 0].real[:, beyond].sum(axis=-1) * dq
    print("lower-surface population beyond the crossing", lo_beyond / total[2:])
    assert 0.0 < lo_beyond[0] < lo_beyond[1]
    assert lo_beyond[1] > 0.1 * total[3]
