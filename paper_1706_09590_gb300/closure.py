"""Learned-closure pipeline on the device: regression statistics from deep hierarchies, training, and
deployment (every numerical step runs in the library's kernels; this module only sequences calls).

Training data: for each bath coupling eta, a deep hierarchy (chain, one Drude mode) is equilibrated,
excited by one and by two dipole commutators (the first and second interactions of Eqs. (R1), (R3)),
and propagated; along the way the statistics of the target tier (the element that a shallow hierarchy
of depth target-1 truncates) against its two lower tiers are accumulated per grid point.
"""
import numpy as np

from .qhfpe import (CLOSURE_N_STATS, CLOSURE_N_WEIGHTS, COMMUTATOR, TERMINATOR, Propagator, closure_inputs,
                    closure_train)

N_IN, N_HID, N_OUT = 3, 256, 10


def network_inputs(model, eta):
    """(q/8, p/8, ln eta) for every grid point, [nq*np][3], from the library."""
    return closure_inputs(model, eta)


def initial_weights(seed=1706):
    """Glorot-uniform hidden layers, zero output layer (the untrained closure is the terminator)."""
    rng = np.random.default_rng(seed)
    parts = []
    for fan_out, fan_in in ((N_HID, N_IN), (N_HID, N_HID), (N_HID, N_HID)):
        lim = np.sqrt(6.0 / (fan_in + fan_out))
        parts += [rng.uniform(-lim, lim, fan_out * fan_in), np.zeros(fan_out)]
    parts += [np.zeros(N_OUT * N_HID), np.zeros(N_OUT)]
    w = np.concatenate(parts).astype(np.float32)
    assert w.size == CLOSURE_N_WEIGHTS
    return w


def deep_statistics(model, U_table, eta, deep_depth, target_tier, n_eq, n_prop, every, stream=None):
    """Statistics [nq*np][67] of tier `target_tier` from a depth-`deep_depth` run at this eta."""
    import torch
    m = dict(model, eta=eta, depth=deep_depth, closure=TERMINATOR)
    P = Propagator(m, U_table, precision="fp64", n_replicas=2, stream=stream)
    stats = torch.zeros(m["nq"] * m["np"] * CLOSURE_N_STATS, dtype=torch.float64, device="cuda")
    P.equilibrate(n_eq)
    P.closure_collect(target_tier, stats)
    P.apply_dipole(COMMUTATOR, [0, 1])
    P.apply_dipole(COMMUTATOR, [1])
    for _ in range(n_prop // every):
        P.step(every)
        P.closure_collect(target_tier, stats)
    P.close()
    return stats.cpu().numpy().reshape(-1, CLOSURE_N_STATS)


def training_set(model, U_table, etas, deep_depth, target_tier, n_eq=1500, n_prop=2000, every=20, stream=None):
    X, S = [], []
    for eta in etas:
        S.append(deep_statistics(model, U_table, eta, deep_depth, target_tier, n_eq, n_prop, every, stream))
        X.append(network_inputs(model, eta))
    return np.concatenate(X), np.concatenate(S)


def train(X, stats, n_iters=3000, batch=4096, lr=1e-3, ridge=0.01, seed=1706, weights=None):
    w0 = initial_weights(seed) if weights is None else weights
    return closure_train(w0, X, stats, n_iters, batch=batch, lr=lr, ridge=ridge, seed=seed)


# ---- state-input network (QHFPE_LEARNED_STATE): the network reads the deepest tiers' local values ------
def initial_state_weights(S, seed=1706):
    """Glorot-uniform hidden layers, zero output layer (the untrained network predicts a zero correction:
    the Eq. (GMFP) terminator alone),
    unit scales."""
    from .qhfpe import closure_state_n_weights
    n_in, n_out = 36 * S * S + 3, 2 * S * S
    rng = np.random.default_rng(seed)
    parts = []
    for fan_out, fan_in in ((N_HID, n_in), (N_HID, N_HID), (N_HID, N_HID)):
        lim = np.sqrt(6.0 / (fan_in + fan_out))
        parts += [rng.uniform(-lim, lim, fan_out * fan_in), np.zeros(fan_out)]
    parts += [np.zeros(n_out * N_HID), np.zeros(n_out), np.ones(3)]
    w = np.concatenate(parts).astype(np.float32)
    assert w.size == closure_state_n_weights(S)
    return w


def state_training_set(model, U_table, etas, deep_depth, target_tier, n_eq, n_prop, every, stream=None,
                       max_samples=400000, seed=1706):
    """Samples (X, Y) of the target tier from depth-`deep_depth` FP64 runs (Eq. (GMFP) terminator) at each
    eta, excited like the statistics of the coefficient form: every grid point of both replicas every
    `every` steps, then at most max_samples of them drawn at random (seeded).  Y is the target tier less
    the element that the terminator of the tier below stands for (qhfpe_closure_state_collect).  Returns
    host float32 arrays."""
    import torch
    S = model["S"]
    n_in, n_out = 36 * S * S + 3, 2 * S * S
    Xs, Ys = [], []
    for eta in etas:
        m = dict(model, eta=eta, depth=deep_depth, closure=TERMINATOR)
        P = Propagator(m, U_table, precision="fp64", n_replicas=2, stream=stream)
        n_snap = n_prop // every + 1
        cap = n_snap * 2 * m["nq"] * m["np"]
        X = torch.zeros((cap, n_in), dtype=torch.float32, device="cuda")
        Y = torch.zeros((cap, n_out), dtype=torch.float32, device="cuda")
        P.equilibrate(n_eq)
        off = P.closure_state_collect(target_tier, X, Y, 0, cap)
        P.apply_dipole(COMMUTATOR, [0, 1])
        P.apply_dipole(COMMUTATOR, [1])
        for _ in range(n_prop // every):
            P.step(every)
            off += P.closure_state_collect(target_tier, X, Y, off, cap)
        P.close()
        Xs.append(X[:off].cpu().numpy())
        Ys.append(Y[:off].cpu().numpy())
    X, Y = np.concatenate(Xs), np.concatenate(Ys)
    if X.shape[0] > max_samples:
        keep = np.sort(np.random.default_rng(seed).choice(X.shape[0], max_samples, replace=False))
        X, Y = X[keep], Y[keep]
    return X, Y


def train_state(S, X, Y, n_iters=3000, batch=4096, lr=1e-3, seed=1706, weights=None):
    from .qhfpe import closure_state_train
    w0 = initial_state_weights(S, seed) if weights is None else weights
    return closure_state_train(S, w0, X, Y, n_iters, batch=batch, lr=lr, seed=seed)
