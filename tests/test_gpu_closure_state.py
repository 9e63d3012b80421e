"""The state-input learned closure (QHFPE_LEARNED_STATE: the network reads 3 x 3 patches of tiers N and
N-1 and predicts the part of W^(N+1) that the Eq. (GMFP) terminator misses) on the GPU: its training gradient and samples against the oracle, the
classic-RK4 propagation with the network inside every right-hand side against an oracle composition,
and the measurement that decides between it and the coefficient form: the pathway-additivity defect of
the third-order response (ket + bra - full) and the error against the deep hierarchy."""
import numpy as np
import pytest

import oracle
import qhfpe_inputs as qi
from oracle import closure as ocl

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    t = pytest.importorskip("torch")
    if not t.cuda.is_available():
        pytest.skip("no CUDA device")
    return t


def rel(a, b):
    return np.linalg.norm(np.ravel(a - b)) / max(np.linalg.norm(np.ravel(b)), 1e-300)


def _P(m, precision="fp64", **kw):
    from paper_1706_09590_gb300 import Propagator
    return Propagator(m, qi.u_table(m), precision=precision, **kw)


def _random_state_weights(S, seed, out_scale=0.02, scales=(1.0, 1.0, 1.0)):
    from paper_1706_09590_gb300.closure import initial_state_weights
    w = initial_state_weights(S, seed).astype(np.float64)
    n_in, n_out = ocl.state_sizes(S)
    rng = np.random.default_rng(seed + 1)
    o = len(w) - 3 - n_out * (ocl.N_HID + 1)
    w[o:len(w) - 3] = rng.normal(size=n_out * (ocl.N_HID + 1)) * out_scale
    w[-3:] = scales
    return w.astype(np.float32)


def test_state_gradient_matches_oracle(torch):
    from paper_1706_09590_gb300.qhfpe import closure_state_loss_grad
    S = 2
    n_in, n_out = ocl.state_sizes(S)
    rng = np.random.default_rng(71)
    w = _random_state_weights(S, 72, out_scale=0.05)
    X = rng.normal(size=(96, n_in)).astype(np.float32)
    Y = rng.normal(size=(96, n_out)).astype(np.float32)
    L_ref, g_ref = ocl.state_loss_and_grad(w.astype(np.float64), X.astype(np.float64), Y.astype(np.float64), S)
    L, g = closure_state_loss_grad(S, w, X, Y)
    assert L == pytest.approx(L_ref, rel=1e-5)
    assert rel(g.astype(np.float64), g_ref) < 1e-4


def test_state_samples_match_oracle(torch):
    m = qi.harmonic_two_state(nq=12, n_p=32, depth=4)
    P = _P(m, n_replicas=2)
    W0, W1 = qi.random_state(m, seed=73), qi.random_state(m, seed=74)
    P.set_state(W0, 0)
    P.set_state(W1, 1)
    n_in, n_out = ocl.state_sizes(2)
    cap = 2 * 12 * 32 + 5
    X = torch.zeros((cap, n_in), dtype=torch.float32, device="cuda")
    Y = torch.zeros((cap, n_out), dtype=torch.float32, device="cuda")
    n = P.closure_state_collect(3, X, Y, 5, cap)
    assert n == 2 * 12 * 32
    got_X, got_Y = X[5:].cpu().numpy(), Y[5:].cpu().numpy()
    ref_X = np.concatenate([ocl.state_inputs(W, 3, m).reshape(-1, n_in) for W in (W0, W1)])
    ref_Y = np.concatenate([ocl.state_targets(W, 3, m).reshape(-1, n_out) for W in (W0, W1)])
    assert rel(got_X, ref_X) < 1e-6 and rel(got_Y, ref_Y) < 1e-6
    P.close()


def _oracle_state_rk4(m, w, W, n_steps):
    """Classic RK4 of the oracle's right-hand side with the Eq. (GMFP) terminator plus the closure term
    d/dp D at the deepest tier, D from the oracle's forward of the network with bf16 inputs, weights and
    activations (the library's inference precision)."""
    O = oracle.Oracle(dict(m, closure=1))
    S, N = m["S"], m["depth"]
    dp = (m["p_max"] - m["p_min"]) / m["np"]

    def f(X):
        d = O.rhs(X)
        out = ocl.state_forward(w.astype(np.float64), ocl.state_inputs(X, N + 1, m), S, quantize=ocl.bf16)
        Wn1 = np.zeros((S, S, m["nq"], m["np"]), complex)
        for j in range(S):
            for k in range(S):
                Wn1[j, k] = out[..., 2 * (j * S + k)] + 1j * out[..., 2 * (j * S + k) + 1]
        dWp = (np.roll(Wn1, 2, -1) - 8 * np.roll(Wn1, 1, -1) + 8 * np.roll(Wn1, -1, -1) - np.roll(Wn1, -2, -1)) / (12 * dp)
        d[N] += dWp
        return d

    dt = m["dt"]
    for _ in range(n_steps):
        k1 = f(W)
        k2 = f(W + 0.5 * dt * k1)
        k3 = f(W + 0.5 * dt * k2)
        k4 = f(W + dt * k3)
        W = W + dt / 6 * (k1 + 2 * k2 + 2 * k3 + k4)
    return W


def test_state_closure_steps_match_oracle(torch):
    m = qi.harmonic_two_state(nq=12, n_p=32, depth=3, closure=3)
    w = _random_state_weights(2, 75, out_scale=0.05, scales=(0.7, 0.4, 0.3))
    W = qi.random_state(m, seed=76)
    P = _P(m)
    P.closure_state_load(w)
    P.set_state(W)
    tr = P.step(4, record_trace=True)[0]
    ref = _oracle_state_rk4(m, w, W, 4)
    got = P.get_state(0)
    assert np.all(np.isfinite(got)) and np.all(np.isfinite(tr))
    # bf16 inference: a pre-activation at a rounding boundary may land one bf16 step apart
    assert rel(got, ref) < 1e-5
    # without weights the network's element is zero: the terminator alone, classic RK4
    Q = _P(m)
    Q.set_state(W)
    Q.step(4)
    ref0, _ = oracle.Oracle(dict(m, closure=1)).step(W, 4)
    assert rel(Q.get_state(0), ref0) < 1e-11
    Q.close()
    P.close()


def test_state_closure_additivity_defect_and_error(torch):
    """Trained on depth-10 runs of the two-state harmonic model (32 x 32) at eta in {0.2, 0.5, 1}, deployed at depth
    4, judged at eta = 0.3 against depth 10: the additivity defect of the third-order response (ket +
    bra against the full commutator) of the state-input closure, against the coefficient form, where
    it is rounding only; and the R1 errors of both learned forms, the truncation and the terminator."""
    from paper_1706_09590_gb300 import closure as pcl
    base = qi.harmonic_two_state(depth=10)
    T = qi.u_table(base)
    dt = base["dt"]
    etas = (0.2, 0.5, 1.0)
    X, Y = pcl.state_training_set(base, T, etas, deep_depth=10, target_tier=5, n_eq=1500, n_prop=1000, every=20)
    ws, hist = pcl.train_state(2, X, Y, n_iters=1500, batch=2048, lr=1e-3)
    assert np.isfinite(hist).all() and hist[-50:].mean() < hist[:50].mean()
    Xc, Sc = pcl.training_set(base, T, etas, deep_depth=10, target_tier=5, n_eq=1500, n_prop=1000, every=20)
    wc, _ = pcl.train(Xc, Sc, n_iters=1500, batch=1024, lr=1e-3)
    eta = 0.3
    res = {}
    for name, depth, closure in (("truth", 10, 1), ("truncate", 4, 0), ("terminator", 4, 1), ("learned_coef", 4, 2),
                                 ("learned_state", 4, 3)):
        m = dict(base, eta=eta, depth=depth, closure=closure)
        P = _P(m)
        if closure == 2:
            P.closure_load(wc)
        if closure == 3:
            P.closure_state_load(ws)
        P.equilibrate(1500)
        P.set_equilibrium(P.get_state(0))
        r1 = P.linear_response(1000)
        full = P.third_order_response(3, 20, [0, 100], 200)
        split = P.third_order_response(3, 20, [0, 100], 200, split_pathways=True)
        res[name] = (r1, rel(split[0] + split[1], full))
        P.close()
    err = {k: rel(v[0], res["truth"][0]) for k, v in res.items() if k != "truth"}
    defect = {k: v[1] for k, v in res.items()}
    print("R1 errors vs depth 10 at eta 0.3:", err)
    print("pathway-additivity defect |ket + bra - full| / |full|:", defect)
    assert all(np.isfinite(list(err.values()))) and all(np.isfinite(list(defect.values())))
    assert defect["learned_coef"] < 1e-12 and defect["truncate"] < 1e-12
    assert defect["learned_state"] > 1e-12  # nonlinear in the state: additivity is lost
