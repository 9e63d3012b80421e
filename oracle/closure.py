"""Learned hierarchy closure, FP64 reference -- TEST INFRASTRUCTURE ONLY (part of the CPU oracle).

The closure corrects the terminator of Eq. (GMFP) at the deepest tier (one Drude mode, K = 0, so the
hierarchy is a chain): the terminator reads the missing element as W^(N+1) ~ (r_0 p + c_0 d/dp) W^N,
and the network adds a local linear combination of the two tiers below,

    dW^(N+1)(q_i, p_l) = sum_{b=-2..2} c_b(x) W^N(q_i, p_{l+b}) + c_{5+b}(x) W^(N-1)(q_i, p_{l+b}),

with the ten coefficients c(x) produced by a multilayer perceptron of x = (q/8, p/8, ln eta):
three tanh hidden layers of width 256 and a linear output of width 10.  The combination is linear in
the state, so the closed hierarchy keeps the linearity that the response functions of Eqs. (R1), (R3)
presuppose (the Green's function G(t) is a linear map); the network only sets its coefficients.  A zero
network is the terminator itself.

Training data are the deep hierarchy's own tiers: for every grid point x the samples (phi = the ten
patch values of tiers N and N-1, y = tier N+1 minus the terminator's estimate of it, with d/dp the
4th-order central difference) from many states are compressed to
    G_x = sum Re(conj(phi) phi^T)  (10 x 10),  h_x = sum Re(conj(phi) y),  yy_x = sum |y|^2,  n_x,
so that the mean squared error over all samples is  sum_x (c^T G_x c - 2 c^T h_x + yy_x) / sum_x n_x.
A ridge term  lam * sum_x (tr G_x / 10) |c_x|^2 / sum_x n_x  keeps the correction small where the data
do not determine it.

Flat weight layout (row-major): W1[256][3], b1[256], W2[256][256], b2[256], W3[256][256], b3[256],
W4[10][256], b4[10].  Statistics layout per point: G upper triangle (55, row-major), h (10), yy, n.
"""
import numpy as np

N_IN, N_HID, N_OUT = 3, 256, 10
SHAPES = [(N_HID, N_IN), (N_HID,), (N_HID, N_HID), (N_HID,), (N_HID, N_HID), (N_HID,), (N_OUT, N_HID), (N_OUT,)]
N_WEIGHTS = int(sum(np.prod(s) for s in SHAPES))
N_STATS = 55 + 10 + 2
TRIU = np.triu_indices(10)


def unpack(w):
    out, o = [], 0
    for s in SHAPES:
        n = int(np.prod(s))
        out.append(np.asarray(w[o:o + n], dtype=np.float64).reshape(s))
        o += n
    return out


def inputs(q, p, eta):
    """Network input for grid points (q, p) at bath coupling eta: (q/8, p/8, ln eta)."""
    q, p = np.broadcast_arrays(np.asarray(q, float), np.asarray(p, float))
    return np.stack([q / 8.0, p / 8.0, np.full(q.shape, np.log(eta))], axis=-1)


def init_weights(seed=1706):
    """Glorot-uniform hidden layers; the output layer starts at zero (closure = truncation)."""
    rng = np.random.default_rng(seed)
    parts = []
    for s in SHAPES:
        if len(s) == 2 and s[0] != N_OUT:
            lim = np.sqrt(6.0 / (s[0] + s[1]))
            parts.append(rng.uniform(-lim, lim, s).ravel())
        else:
            parts.append(np.zeros(int(np.prod(s))))
    return np.concatenate(parts)


def forward(w, X):
    W1, b1, W2, b2, W3, b3, W4, b4 = unpack(w)
    h1 = np.tanh(X @ W1.T + b1)
    h2 = np.tanh(h1 @ W2.T + b2)
    h3 = np.tanh(h2 @ W3.T + b3)
    c = h3 @ W4.T + b4
    return c, (X, h1, h2, h3)


def _full_G(stats):
    G = np.zeros(stats.shape[:-1] + (10, 10))
    G[..., TRIU[0], TRIU[1]] = stats[..., :55]
    G = G + np.swapaxes(G, -1, -2) - np.eye(10) * G
    return G


def _ridge_weight(G):
    return np.trace(G, axis1=-2, axis2=-1) / 10.0


def loss(w, X, stats, lam=0.0):
    c, _ = forward(w, X)
    G = _full_G(stats)
    h = stats[:, 55:65]
    q = np.einsum("ni,nij,nj->n", c, G, c) - 2 * np.einsum("ni,ni->n", c, h) + stats[:, 65]
    q = q + lam * _ridge_weight(G) * (c * c).sum(-1)
    return q.sum() / stats[:, 66].sum()


def loss_and_grad(w, X, stats, lam=0.0):
    """Mean squared closure error (+ ridge) and its gradient with respect to the flat weights."""
    W1, b1, W2, b2, W3, b3, W4, b4 = unpack(w)
    c, (X, h1, h2, h3) = forward(w, X)
    G = _full_G(stats)
    h = stats[:, 55:65]
    ntot = stats[:, 66].sum()
    rw = lam * _ridge_weight(G)
    q = np.einsum("ni,nij,nj->n", c, G, c) - 2 * np.einsum("ni,ni->n", c, h) + stats[:, 65]
    q = q + rw * (c * c).sum(-1)
    L = q.sum() / ntot
    dc = 2.0 * (np.einsum("nij,nj->ni", G, c) - h + rw[:, None] * c) / ntot
    dW4 = dc.T @ h3
    db4 = dc.sum(0)
    dz3 = (dc @ W4) * (1 - h3 ** 2)
    dW3 = dz3.T @ h2
    db3 = dz3.sum(0)
    dz2 = (dz3 @ W3) * (1 - h2 ** 2)
    dW2 = dz2.T @ h1
    db2 = dz2.sum(0)
    dz1 = (dz2 @ W2) * (1 - h1 ** 2)
    dW1 = dz1.T @ X
    db1 = dz1.sum(0)
    return L, np.concatenate([a.ravel() for a in (dW1, db1, dW2, db2, dW3, db3, dW4, db4)])


def coefficients(w, model):
    """[nq][np][10] closure coefficients on the model's grid at its eta."""
    from qhfpe_inputs import axis
    q = axis(model["nq"], model["q_min"], model["q_max"])
    p = axis(model["np"], model["p_min"], model["p_max"])
    Q, Pm = np.meshgrid(q, p, indexing="ij")
    c, _ = forward(w, inputs(Q, Pm, model["eta"]))
    return c


def patch_samples(W, tier, r0=0.0, c0=0.0, p=None, dp=1.0):
    """Samples of the closure regression from a K = 0 hierarchy state W ([n_elem][S][S][nq][np],
    element e = tier e): phi [nq][np][S*S][10] and y [nq][np][S*S] for the target tier `tier`, minus
    the terminator's estimate r0 p W^(tier-1) + c0 dW^(tier-1)/dp (p: the p grid)."""
    n_elem, S, _, nq, n_p = W.shape
    A = W[tier - 1].reshape(S * S, nq, n_p)
    B = W[tier - 2].reshape(S * S, nq, n_p) if tier >= 2 else np.zeros_like(A)
    phi = np.zeros((nq, n_p, S * S, 10), complex)
    for b in range(-2, 3):
        phi[..., 2 + b] = np.moveaxis(np.roll(A, -b, axis=-1), 0, -1)
        phi[..., 7 + b] = np.moveaxis(np.roll(B, -b, axis=-1), 0, -1)
    y = np.moveaxis(W[tier].reshape(S * S, nq, n_p), 0, -1)
    if r0 != 0.0 or c0 != 0.0:
        d1 = np.array([1.0, -8.0, 0.0, 8.0, -1.0]) / (12.0 * dp)
        term = r0 * np.asarray(p)[None, :, None] * phi[..., 2] + c0 * np.einsum("xysf,f->xys", phi[..., :5], d1)
        y = y - term
    return phi, y


def statistics(W, tier, r0=0.0, c0=0.0, p=None, dp=1.0):
    """Per-point statistics [nq*np][67] of one state (sum over the electronic pairs); with r0, c0 the
    target is the terminator's residual."""
    phi, y = patch_samples(W, tier, r0, c0, p, dp)
    nq, n_p = phi.shape[:2]
    G = np.einsum("xysa,xysb->xyab", np.conj(phi), phi).real
    h = np.einsum("xysa,xys->xya", np.conj(phi), y).real
    yy = (np.abs(y) ** 2).sum(-1)
    out = np.zeros((nq, n_p, N_STATS))
    out[..., :55] = G[..., TRIU[0], TRIU[1]]
    out[..., 55:65] = h
    out[..., 65] = yy
    out[..., 66] = phi.shape[2]
    return out.reshape(nq * n_p, N_STATS)


# ------------------------------------------------------------------------------------------------
# State-input closure (the literal network): W^(N+1) at (q_i, p_l), all pairs, from the 3 x 3 patches
# of tiers N and N-1 of the state itself and (q/8, p/8, ln eta).  Input layout: the three features,
# then tier N then tier N-1, each pair by pair (j, k row-major), patch row-major over (a, b) in
# {-1, 0, 1}^2 (q offset a: zero outside the grid unless periodic; p offset b: periodic), (re, im)
# innermost -- 36 S^2 + 3 values.  Output: (re, im) of W^(N+1)_jk pair by pair -- 2 S^2 values.  Weights:
# W1[256][n_in], b1, W2[256][256], b2, W3[256][256], b3, W4[n_out][256], b4, then three scales (tier-N
# inputs, tier-(N-1) inputs, outputs).
# ------------------------------------------------------------------------------------------------
def state_sizes(S):
    return 36 * S * S + 3, 2 * S * S


def state_shapes(S):
    n_in, n_out = state_sizes(S)
    return [(N_HID, n_in), (N_HID,), (N_HID, N_HID), (N_HID,), (N_HID, N_HID), (N_HID,), (n_out, N_HID), (n_out,)]


def state_n_weights(S):
    return int(sum(np.prod(s) for s in state_shapes(S))) + 3


def state_unpack(w, S):
    out, o = [], 0
    for s in state_shapes(S):
        n = int(np.prod(s))
        out.append(np.asarray(w[o:o + n], dtype=np.float64).reshape(s))
        o += n
    return out, np.asarray(w[o:o + 3], dtype=np.float64)


def state_inputs(W, tier, model):
    """Unscaled network inputs [nq][np][36 S^2 + 3] of the target tier `tier` from a K = 0 state W
    ([n_elem][S][S][nq][np], element e = tier e): tiers tier-1 and tier-2 (zeros below tier 0)."""
    from qhfpe_inputs import axis
    n_elem, S, _, nq, n_p = W.shape
    periodic = model.get("periodic_q", 0)
    q = axis(nq, model["q_min"], model["q_max"])
    p = axis(n_p, model["p_min"], model["p_max"])
    out = np.zeros((nq, n_p, 36 * S * S + 3))
    out[..., 0] = q[:, None] / 8.0
    out[..., 1] = p[None, :] / 8.0
    out[..., 2] = np.log(model["eta"])
    c = 3
    for t in (tier - 1, tier - 2):
        X = W[t] if t >= 0 else np.zeros_like(W[0])
        for j in range(S):
            for k in range(S):
                blk = X[j, k]
                for a in (-1, 0, 1):
                    sh = np.roll(blk, -a, axis=0)
                    if not periodic:
                        if a == 1:
                            sh[-1] = 0
                        elif a == -1:
                            sh[0] = 0
                    for b in (-1, 0, 1):
                        v = np.roll(sh, -b, axis=1)
                        out[..., c] = v.real
                        out[..., c + 1] = v.imag
                        c += 2
    return out


def terminator_element(W_low, model, r0, c0):
    """The element that the Eq. (GMFP) terminator stands for, r_0 p W + c_0 dW/dp, of one tier W_low
    [S][S][nq][np]: its d/dp is the terminator's d/dp (r_0 p W) + c_0 d2W/dp2 up to the composition of
    two first differences (the right-hand side's 4th-order central difference along the periodic p
    axis, written out here as a sum over the four neighbours)."""
    from qhfpe_inputs import axis
    n_p = W_low.shape[-1]
    p = axis(n_p, model["p_min"], model["p_max"])
    dp = (model["p_max"] - model["p_min"]) / n_p
    dW = (np.roll(W_low, 2, -1) - 8 * np.roll(W_low, 1, -1) + 8 * np.roll(W_low, -1, -1) - np.roll(W_low, -2, -1)) / (12 * dp)
    return r0 * p * W_low + c0 * dW


def state_targets(W, tier, model):
    """[nq][np][2 S^2] targets: (re, im) pair by pair of D = W^(tier) less the terminator's element of
    W^(tier-1) (the closure term of a depth tier-1 hierarchy is then the terminator plus d/dp D), with
    the bath's r_0 and c_0 (one Drude mode)."""
    import oracle
    co = oracle.Oracle(dict(model, closure=0)).coefficients()
    n_elem, S, _, nq, n_p = W.shape
    D = W[tier] - terminator_element(W[tier - 1], model, co["r"][0], co["c"][0])
    Y = np.zeros((nq, n_p, 2 * S * S))
    for j in range(S):
        for k in range(S):
            Y[..., 2 * (j * S + k)] = D[j, k].real
            Y[..., 2 * (j * S + k) + 1] = D[j, k].imag
    return Y


def state_forward(w, X, S, quantize=None, scaled=True):
    """Network output for inputs X [..][n_in].  scaled: divide the tier inputs by their scales and
    multiply the outputs by the output scale (the deployed network); quantize (optional) rounds the
    inputs, weights and activations (e.g. to bf16)."""
    (W1, b1, W2, b2, W3, b3, W4, b4), sc = state_unpack(w, S)
    qz = quantize or (lambda a: a)
    n_in, _ = state_sizes(S)
    half = (n_in - 3) // 2
    X = np.array(X, dtype=np.float64)
    if scaled:
        X[..., 3:3 + half] /= sc[0]
        X[..., 3 + half:] /= sc[1]
    h = qz(X)
    for Wl, bl in ((W1, b1), (W2, b2), (W3, b3)):
        h = qz(np.tanh(h @ qz(Wl).T + bl))
    out = h @ qz(W4).T + b4
    return out * sc[2] if scaled else out


def state_loss_and_grad(w, X, Y, S):
    """Mean squared error over all samples and outputs (unscaled X, Y) and its gradient with respect to
    the flat weights (without the three scales)."""
    (W1, b1, W2, b2, W3, b3, W4, b4), _ = state_unpack(w, S)
    h1 = np.tanh(X @ W1.T + b1)
    h2 = np.tanh(h1 @ W2.T + b2)
    h3 = np.tanh(h2 @ W3.T + b3)
    o = h3 @ W4.T + b4
    d = o - Y
    L = (d * d).mean()
    do = 2.0 * d / d.size
    dW4 = do.T @ h3
    db4 = do.sum(0)
    dz3 = (do @ W4) * (1 - h3 ** 2)
    dW3 = dz3.T @ h2
    db3 = dz3.sum(0)
    dz2 = (dz3 @ W3) * (1 - h2 ** 2)
    dW2 = dz2.T @ h1
    db2 = dz2.sum(0)
    dz1 = (dz2 @ W2) * (1 - h1 ** 2)
    dW1 = dz1.T @ X
    db1 = dz1.sum(0)
    return L, np.concatenate([a.ravel() for a in (dW1, db1, dW2, db2, dW3, db3, dW4, db4)])


def bf16(a):
    """Round to the nearest bf16 (ties to even), returned as float64."""
    x = np.asarray(a, dtype=np.float32)
    u = x.view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)
