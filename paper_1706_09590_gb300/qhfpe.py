"""Thin Python binding of the C ABI in include/qhfpe.h (argument marshalling only).

Every numerical step runs in libqhfpe.so; this module converts arguments (numpy / torch buffers,
scalars) into the ABI's plain pointers and sizes and raises on error statuses.  There is no fallback:
if the library is missing the import fails.
"""
import ctypes
import os

import numpy as np

from . import build as _build

LIB_PATH = _build.LIB

FP64, MIXED, MIXED_BF16X3, MIXED_TF32X3 = 0, 1, 2, 3  # TF32X3: declared, not built
TRUNCATE, TERMINATOR, LEARNED = 0, 1, 2
LEFT, RIGHT, COMMUTATOR = 1, 2, 3
TERM_KINETIC, TERM_POTENTIAL, TERM_DAMPING, TERM_TIER_UP, TERM_TIER_DOWN, TERM_ALL = 1, 2, 4, 8, 16, 31
LINEAR, THIRD_ORDER = 0, 1
PRECISIONS = {"fp64": FP64, "mixed": MIXED, "bf16x3": MIXED_BF16X3, "tf32x3": MIXED_TF32X3}

STATUS = {0: "OK", 1: "EINVAL", 2: "ENOMEM", 3: "ECUDA", 4: "ENUMERIC", 5: "ETIMEOUT", 6: "EUNSUPPORTED",
          7: "ESTATE"}

EXPORTED = [
    "qhfpe_create", "qhfpe_destroy", "qhfpe_last_error", "qhfpe_sizes", "qhfpe_hierarchy",
    "qhfpe_bath_coefficients", "qhfpe_max_stable_dt", "qhfpe_set_state", "qhfpe_get_state", "qhfpe_fork",
    "qhfpe_step", "qhfpe_apply_dipole", "qhfpe_apply_rhs", "qhfpe_trace", "qhfpe_equilibrate",
    "qhfpe_equilibrate_tol", "qhfpe_fp64_fma_rate", "qhfpe_stage_form", "qhfpe_set_persistent",
    "qhfpe_barrier_selftest", "qhfpe_closure_inputs", "qhfpe_closure_state_n_weights", "qhfpe_closure_state_load",
    "qhfpe_closure_state_collect", "qhfpe_closure_state_loss_grad", "qhfpe_closure_state_train",
    "qhfpe_set_equilibrium", "qhfpe_response", "qhfpe_spectrum_absorption", "qhfpe_spectrum_2d",
    "qhfpe_kernel_timing", "qhfpe_kernel_timing_read", "qhfpe_potential_term_static",
    "qhfpe_closure_collect", "qhfpe_closure_load", "qhfpe_closure_coefficients", "qhfpe_closure_loss_grad",
    "qhfpe_closure_train", "qhfpe_tile_rows", "qhfpe_wait_selftest", "qhfpe_adiabatic_marginals",
    "qhfpe_first_order_distribution", "qhfpe_set_dipole_table", "qhfpe_batch_create", "qhfpe_batch_step",
    "qhfpe_batch_tile_rows", "qhfpe_batch_destroy", "qhfpe_set_state32", "qhfpe_get_state32",
]

CLOSURE_N_WEIGHTS = 135178
LEARNED_STATE = 3
CLOSURE_N_STATS = 67


class QhfpeError(RuntimeError):
    def __init__(self, status, message):
        super().__init__(f"{STATUS.get(status, status)}: {message}")
        self.status = status


class Params(ctypes.Structure):
    _fields_ = [
        ("n_states", ctypes.c_int), ("nq", ctypes.c_int), ("np", ctypes.c_int),
        ("q_min", ctypes.c_double), ("q_max", ctypes.c_double), ("p_min", ctypes.c_double),
        ("p_max", ctypes.c_double),
        ("U_table", ctypes.POINTER(ctypes.c_double)), ("mu", ctypes.POINTER(ctypes.c_double)),
        ("eta", ctypes.c_double), ("gamma", ctypes.c_double), ("beta", ctypes.c_double),
        ("n_matsubara", ctypes.c_int), ("high_temperature", ctypes.c_int), ("use_cdelta", ctypes.c_int),
        ("depth", ctypes.c_int), ("closure", ctypes.c_int), ("periodic_q", ctypes.c_int),
        ("precision", ctypes.c_int), ("dt", ctypes.c_double), ("n_replicas", ctypes.c_int),
        ("v_c2", ctypes.c_double),
    ]


class Schedule(ctypes.Structure):
    _fields_ = [
        ("kind", ctypes.c_int), ("n_t1", ctypes.c_int), ("t1_stride", ctypes.c_int), ("n_t2", ctypes.c_int),
        ("t2_steps", ctypes.POINTER(ctypes.c_int)), ("n_t3", ctypes.c_int), ("split_pathways", ctypes.c_int),
    ]


_lib = None


def lib():
    """Load libqhfpe.so (building it first if the sources are newer).  Raises if it cannot."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH) or _build._stale():
        _build.build()
    L = ctypes.CDLL(LIB_PATH)
    vp, dp, ip, st = ctypes.c_void_p, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int), ctypes.c_int
    L.qhfpe_create.argtypes = [ctypes.POINTER(Params), vp, ctypes.POINTER(vp)]
    L.qhfpe_destroy.argtypes = [vp]
    L.qhfpe_last_error.argtypes = [vp]
    L.qhfpe_last_error.restype = ctypes.c_char_p
    L.qhfpe_sizes.argtypes = [vp, ip, ip, ctypes.POINTER(ctypes.c_size_t)]
    L.qhfpe_hierarchy.argtypes = [vp, ip]
    L.qhfpe_bath_coefficients.argtypes = [vp, dp, dp, dp, dp]
    L.qhfpe_max_stable_dt.argtypes = [vp, dp]
    L.qhfpe_set_state.argtypes = [vp, ctypes.c_int, vp, ctypes.c_int]
    L.qhfpe_get_state.argtypes = [vp, ctypes.c_int, vp, ctypes.c_int]
    L.qhfpe_set_state32.argtypes = [vp, ctypes.c_int, vp, ctypes.c_int]
    L.qhfpe_get_state32.argtypes = [vp, ctypes.c_int, vp, ctypes.c_int]
    L.qhfpe_fork.argtypes = [vp, ctypes.c_int, ip, ctypes.c_int]
    L.qhfpe_step.argtypes = [vp, ctypes.c_long, vp]
    L.qhfpe_apply_dipole.argtypes = [vp, ctypes.c_int, ip, ctypes.c_int]
    L.qhfpe_apply_rhs.argtypes = [vp, ctypes.c_int, ctypes.c_int, vp]
    L.qhfpe_trace.argtypes = [vp, vp]
    L.qhfpe_adiabatic_marginals.argtypes = [vp, ctypes.c_int, vp]
    L.qhfpe_set_dipole_table.argtypes = [vp, vp]
    L.qhfpe_first_order_distribution.argtypes = [vp, ctypes.c_int, ctypes.c_int, vp, ctypes.c_int, vp]
    L.qhfpe_equilibrate.argtypes = [vp, ctypes.c_long, dp]
    L.qhfpe_equilibrate_tol.argtypes = [vp, ctypes.c_double, ctypes.c_double, ctypes.c_long,
                                        ctypes.POINTER(ctypes.c_long), dp]
    L.qhfpe_set_equilibrium.argtypes = [vp, vp, ctypes.c_int]
    L.qhfpe_response.argtypes = [vp, ctypes.POINTER(Schedule), vp]
    L.qhfpe_spectrum_absorption.argtypes = [vp, vp, ctypes.c_long, ctypes.c_double, vp, ctypes.c_int, vp]
    L.qhfpe_spectrum_2d.argtypes = [vp, vp, ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_double, vp,
                                    ctypes.c_int, vp, ctypes.c_int, vp, vp]
    L.qhfpe_kernel_timing.argtypes = [vp, ctypes.c_int]
    L.qhfpe_kernel_timing_read.argtypes = [vp, ctypes.POINTER(ctypes.c_long), dp, ctypes.c_int]
    L.qhfpe_potential_term_static.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_double,
                                              ctypes.c_double, vp, ctypes.c_int, vp, vp, vp]
    L.qhfpe_tile_rows.argtypes = [vp, ip]
    L.qhfpe_stage_form.argtypes = [vp, ip]
    L.qhfpe_set_persistent.argtypes = [vp, ctypes.c_int]
    L.qhfpe_closure_inputs.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                       ctypes.c_double, ctypes.c_double, vp]
    L.qhfpe_closure_state_n_weights.argtypes = [ctypes.c_int]
    L.qhfpe_closure_state_n_weights.restype = ctypes.c_size_t
    L.qhfpe_closure_state_load.argtypes = [vp, vp, ctypes.c_size_t]
    L.qhfpe_closure_state_collect.argtypes = [vp, ctypes.c_int, vp, vp, ctypes.c_long, ctypes.c_long,
                                              ctypes.POINTER(ctypes.c_long)]
    L.qhfpe_closure_state_loss_grad.argtypes = [ctypes.c_int, vp, vp, vp, ctypes.c_int, dp, vp]
    L.qhfpe_closure_state_train.argtypes = [ctypes.c_int, vp, vp, vp, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                            ctypes.c_double, ctypes.c_uint, vp]
    L.qhfpe_barrier_selftest.argtypes = [vp, ctypes.c_int, ctypes.c_int]
    L.qhfpe_fp64_fma_rate.argtypes = [vp, ctypes.c_int, dp]
    L.qhfpe_batch_create.argtypes = [ctypes.POINTER(vp), st, ctypes.POINTER(vp)]
    L.qhfpe_batch_step.argtypes = [vp, ctypes.c_long, ctypes.POINTER(vp)]
    L.qhfpe_batch_tile_rows.argtypes = [vp, ip]
    L.qhfpe_batch_destroy.argtypes = [vp]
    L.qhfpe_wait_selftest.argtypes = [vp, ctypes.c_int, ctypes.c_int]
    L.qhfpe_closure_collect.argtypes = [vp, ctypes.c_int, vp]
    L.qhfpe_closure_load.argtypes = [vp, vp, ctypes.c_size_t]
    L.qhfpe_closure_coefficients.argtypes = [vp, vp]
    L.qhfpe_closure_loss_grad.argtypes = [vp, vp, vp, ctypes.c_int, ctypes.c_double, dp, vp]
    L.qhfpe_closure_train.argtypes = [vp, vp, vp, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_double,
                                      ctypes.c_double, ctypes.c_uint, vp]
    for name in EXPORTED:
        if name != "qhfpe_last_error":
            getattr(L, name).restype = st
    _lib = L
    return L


def _ptr(a):
    return ctypes.c_void_p(a.ctypes.data)


def _is_c64(t):
    return str(getattr(t, "dtype", "")) in ("torch.complex64", "torch.float32")


def _c128(a):
    return np.ascontiguousarray(a, dtype=np.complex128)


def _dev_ptr(t):
    """(pointer, is_device) for a numpy array or a torch tensor (CUDA tensors stay on the device)."""
    if hasattr(t, "data_ptr") and hasattr(t, "is_cuda"):
        if t.is_cuda:
            assert t.is_contiguous()
            return ctypes.c_void_p(t.data_ptr()), 1
        t = t.numpy()
    return _ptr(t), 0


def potential_term_static(U_table_dev, W_dev, out_dev, n_states, nq, np_, p_min, p_max, n_elem, stream=None):
    """-i[U, W] for n_elem hierarchy elements, all arguments device buffers (torch CUDA tensors or raw
    pointers), computed without any device allocation (static scratch; see include/qhfpe.h)."""
    L = lib()
    ptr = lambda t: ctypes.c_void_p(t.data_ptr() if hasattr(t, "data_ptr") else int(t))
    sptr = None if stream is None else ctypes.c_void_p(stream.cuda_stream if hasattr(stream, "cuda_stream")
                                                       else int(stream))
    s = L.qhfpe_potential_term_static(n_states, nq, np_, p_min, p_max, ptr(U_table_dev), n_elem, ptr(W_dev),
                                      ptr(out_dev), sptr)
    if s != 0:
        raise QhfpeError(s, L.qhfpe_last_error(None).decode())


def closure_loss_grad(w, X, stats, ridge=0.0):
    """Mean squared closure error and its gradient (FP32 kernels) for weights w on points X [n][3]
    with statistics [n][67]."""
    L = lib()
    w = np.ascontiguousarray(w, dtype=np.float32)
    X = np.ascontiguousarray(X, dtype=np.float64)
    stats = np.ascontiguousarray(stats, dtype=np.float64)
    assert w.size == CLOSURE_N_WEIGHTS and X.shape[1] == 3 and stats.shape == (X.shape[0], CLOSURE_N_STATS)
    loss = ctypes.c_double()
    grad = np.zeros(CLOSURE_N_WEIGHTS, dtype=np.float32)
    s = L.qhfpe_closure_loss_grad(_ptr(w), _ptr(X), _ptr(stats), X.shape[0], ridge, ctypes.byref(loss), _ptr(grad))
    if s != 0:
        raise QhfpeError(s, L.qhfpe_last_error(None).decode())
    return loss.value, grad


def closure_inputs(model, eta):
    """The closure network's inputs (q/8, p/8, ln eta) at every grid point, [nq*np][3], computed by the library."""
    L = lib()
    X = np.zeros((model["nq"] * model["np"], 3))
    s = L.qhfpe_closure_inputs(model["nq"], model["np"], model["q_min"], model["q_max"], model["p_min"],
                               model["p_max"], float(eta), _ptr(X))
    if s != 0:
        raise QhfpeError(s, L.qhfpe_last_error(None).decode())
    return X


def closure_state_n_weights(n_states):
    return int(lib().qhfpe_closure_state_n_weights(int(n_states)))


def closure_state_loss_grad(n_states, w, X, Y):
    """Mean squared error of the state-input network on (X, Y) and its gradient (FP32 kernels)."""
    L = lib()
    w = np.ascontiguousarray(w, dtype=np.float32)
    X = np.ascontiguousarray(X, dtype=np.float32)
    Y = np.ascontiguousarray(Y, dtype=np.float32)
    loss = ctypes.c_double()
    grad = np.zeros(closure_state_n_weights(n_states) - 3, dtype=np.float32)
    s = L.qhfpe_closure_state_loss_grad(int(n_states), _ptr(w), _ptr(X), _ptr(Y), X.shape[0], ctypes.byref(loss),
                                        _ptr(grad))
    if s != 0:
        raise QhfpeError(s, L.qhfpe_last_error(None).decode())
    return loss.value, grad


def closure_state_train(n_states, w, X, Y, n_iters, batch=4096, lr=1e-3, seed=1706):
    """Adam training of the state-input network on the device; returns (weights with scales, loss history)."""
    L = lib()
    w = np.ascontiguousarray(w, dtype=np.float32).copy()
    X = np.ascontiguousarray(X, dtype=np.float32)
    Y = np.ascontiguousarray(Y, dtype=np.float32)
    hist = np.zeros(max(n_iters, 1))
    s = L.qhfpe_closure_state_train(int(n_states), _ptr(w), _ptr(X), _ptr(Y), X.shape[0], n_iters, batch, lr, seed,
                                    _ptr(hist))
    if s != 0:
        raise QhfpeError(s, L.qhfpe_last_error(None).decode())
    return w, hist[:n_iters]


def closure_train(w, X, stats, n_iters, batch=4096, lr=1e-3, ridge=0.0, seed=1706):
    """Adam training of the closure network on the device; returns (weights, per-iteration loss)."""
    L = lib()
    w = np.ascontiguousarray(w, dtype=np.float32).copy()
    X = np.ascontiguousarray(X, dtype=np.float64)
    stats = np.ascontiguousarray(stats, dtype=np.float64)
    hist = np.zeros(max(n_iters, 1))
    s = L.qhfpe_closure_train(_ptr(w), _ptr(X), _ptr(stats), X.shape[0], n_iters, batch, lr, ridge, seed, _ptr(hist))
    if s != 0:
        raise QhfpeError(s, L.qhfpe_last_error(None).decode())
    return w, hist[:n_iters]


class Propagator:
    """One handle of the library: a model on a grid with `n_replicas` independent propagations."""

    def __init__(self, model, U_table, precision="fp64", n_replicas=1, stream=None, dt=None, closure=None):
        L = lib()
        self._L = L
        S = model["S"]
        self.T = np.ascontiguousarray(U_table, dtype=np.float64)
        assert self.T.shape == (S, S, model["nq"], model["np"] + 1), self.T.shape
        self.mu = np.ascontiguousarray(np.asarray(model["mu"], dtype=np.float64))
        prec = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
        dpp = ctypes.POINTER(ctypes.c_double)
        self.params = Params(S, model["nq"], model["np"], model["q_min"], model["q_max"], model["p_min"],
                             model["p_max"], self.T.ctypes.data_as(dpp), self.mu.ctypes.data_as(dpp),
                             model["eta"], model["gamma"], model["beta"], model["n_matsubara"],
                             model["high_temperature"], model["use_cdelta"], model["depth"],
                             model["closure"] if closure is None else closure, model.get("periodic_q", 0),
                             prec, model["dt"] if dt is None else dt, n_replicas, float(model.get("v_c2", 0.0)))
        self.model = model
        self.n_replicas = n_replicas
        self.dt = self.params.dt
        self._stream_obj = stream
        sptr = None
        if stream is not None:
            sptr = ctypes.c_void_p(stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))
        h = ctypes.c_void_p()
        s = L.qhfpe_create(ctypes.byref(self.params), sptr, ctypes.byref(h))
        if s != 0:
            raise QhfpeError(s, L.qhfpe_last_error(None).decode())
        self._h = h
        ne, nm, se = ctypes.c_int(), ctypes.c_int(), ctypes.c_size_t()
        L.qhfpe_sizes(h, ctypes.byref(ne), ctypes.byref(nm), ctypes.byref(se))
        self.n_elem, self.n_modes, self.state_elems = ne.value, nm.value, se.value
        self.shape = (self.n_elem, S, S, model["nq"], model["np"])

    def _check(self, s):
        if s != 0:
            raise QhfpeError(s, self._L.qhfpe_last_error(self._h).decode())

    def close(self):
        if getattr(self, "_h", None):
            self._L.qhfpe_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ---- introspection ---------------------------------------------------------------------------
    def hierarchy(self):
        out = np.zeros((self.n_elem, self.n_modes), dtype=np.int32)
        self._check(self._L.qhfpe_hierarchy(self._h, out.ctypes.data_as(ctypes.POINTER(ctypes.c_int))))
        return out

    def bath_coefficients(self):
        g, r, c, cd = (np.zeros(self.n_modes), np.zeros(self.n_modes), np.zeros(self.n_modes), np.zeros(1))
        dpp = ctypes.POINTER(ctypes.c_double)
        self._check(self._L.qhfpe_bath_coefficients(self._h, g.ctypes.data_as(dpp), r.ctypes.data_as(dpp),
                                                     c.ctypes.data_as(dpp), cd.ctypes.data_as(dpp)))
        return dict(gamma=g, r=r, c=c, cdelta=float(cd[0]))

    def max_stable_dt(self):
        v = ctypes.c_double()
        self._check(self._L.qhfpe_max_stable_dt(self._h, ctypes.byref(v)))
        return v.value

    # ---- state -----------------------------------------------------------------------------------
    def set_state(self, W, replica=-1):
        """Canonical state into one replica (or all, replica = -1): complex128, or complex64 (half the
        bytes; numpy array or CUDA tensor of that dtype)."""
        if hasattr(W, "is_cuda"):
            ptr, dev = _dev_ptr(W)
            f = self._L.qhfpe_set_state32 if _is_c64(W) else self._L.qhfpe_set_state
            self._check(f(self._h, replica, ptr, dev))
            return
        if isinstance(W, np.ndarray) and W.dtype == np.complex64:
            W = np.ascontiguousarray(W)
            assert W.shape == self.shape, (W.shape, self.shape)
            self._check(self._L.qhfpe_set_state32(self._h, replica, _ptr(W), 0))
            return
        W = _c128(W)
        assert W.shape == self.shape, (W.shape, self.shape)
        self._check(self._L.qhfpe_set_state(self._h, replica, _ptr(W), 0))

    def get_state(self, replica=0, out=None):
        """Canonical complex128 state of one replica.  out: optional destination (numpy array, e.g. a
        view of pinned memory, or a contiguous CUDA tensor of matching size); a complex64 destination
        receives the state rounded to FP32."""
        if out is not None and hasattr(out, "is_cuda"):
            ptr, dev = _dev_ptr(out)
            f = self._L.qhfpe_get_state32 if _is_c64(out) else self._L.qhfpe_get_state
            self._check(f(self._h, replica, ptr, dev))
            return out
        if out is not None:
            assert out.dtype in (np.complex128, np.complex64) and out.flags.c_contiguous
            assert out.size == int(np.prod(self.shape))
            f = self._L.qhfpe_get_state32 if out.dtype == np.complex64 else self._L.qhfpe_get_state
            self._check(f(self._h, replica, _ptr(out), 0))
            return out
        out = np.empty(self.shape, dtype=np.complex128)
        self._check(self._L.qhfpe_get_state(self._h, replica, _ptr(out), 0))
        return out

    def fork(self, src, dst):
        d = np.ascontiguousarray(dst, dtype=np.int32)
        self._check(self._L.qhfpe_fork(self._h, src, d.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), len(d)))

    # ---- propagation -----------------------------------------------------------------------------
    def step(self, n_steps, record_trace=False):
        if record_trace:
            tr = np.zeros((self.n_replicas, n_steps + 1), dtype=np.complex128)
            self._check(self._L.qhfpe_step(self._h, n_steps, _ptr(tr)))
            return tr
        self._check(self._L.qhfpe_step(self._h, n_steps, None))
        return None

    def apply_dipole(self, side=COMMUTATOR, replicas=None):
        if replicas is None:
            self._check(self._L.qhfpe_apply_dipole(self._h, side, None, 0))
        else:
            r = np.ascontiguousarray(replicas, dtype=np.int32)
            self._check(self._L.qhfpe_apply_dipole(self._h, side, r.ctypes.data_as(ctypes.POINTER(ctypes.c_int)),
                                                   len(r)))

    def apply_rhs(self, replica=0, terms=TERM_ALL):
        out = np.empty(self.shape, dtype=np.complex128)
        self._check(self._L.qhfpe_apply_rhs(self._h, replica, terms, _ptr(out)))
        return out

    def trace(self):
        out = np.zeros(self.n_replicas, dtype=np.complex128)
        self._check(self._L.qhfpe_trace(self._h, _ptr(out)))
        return out

    def set_dipole_table(self, mu_table):
        """Coordinate-dependent dipole mu_jk(q_i + s_t), [S][S][nq][np+1] (None: the Condon dipole)."""
        if mu_table is None:
            self._check(self._L.qhfpe_set_dipole_table(self._h, None))
            return
        T = np.ascontiguousarray(mu_table, dtype=np.float64)
        S = self.shape[1]
        assert T.shape == (S, S, self.shape[3], self.shape[4] + 1)
        self._check(self._L.qhfpe_set_dipole_table(self._h, _ptr(T)))

    def adiabatic_marginals(self, replica=0):
        """P^(ad)_ab(q_i) of the zeroth tier, complex [S][S][nq] (the adiabatic-basis coordinate
        marginals of Sec. III)."""
        S = self.shape[1]
        out = np.zeros((S, S, self.shape[3]), dtype=np.complex128)
        self._check(self._L.qhfpe_adiabatic_marginals(self._h, replica, _ptr(out)))
        return out

    def first_order_distribution(self, n_t1, t1_stride, omega):
        """W'(omega_1) of Sec. III for each frequency: complex [n_omega][n_elem][S][S][nq][np]."""
        om = np.ascontiguousarray(omega, dtype=np.float64)
        out = np.zeros((len(om),) + self.shape, dtype=np.complex128)
        self._check(self._L.qhfpe_first_order_distribution(self._h, int(n_t1), int(t1_stride), _ptr(om), len(om),
                                                           _ptr(out)))
        return out

    def equilibrate(self, n_steps):
        res = ctypes.c_double()
        self._check(self._L.qhfpe_equilibrate(self._h, n_steps, ctypes.byref(res)))
        return res.value

    def equilibrate_to(self, tol, t_max, check_every=100):
        """Equilibrate until ||L W|| / ||W|| < tol (checked every check_every steps) or t_max; returns
        (steps taken, residual)."""
        n, res = ctypes.c_long(), ctypes.c_double()
        self._check(self._L.qhfpe_equilibrate_tol(self._h, float(t_max), float(tol), int(check_every),
                                                  ctypes.byref(n), ctypes.byref(res)))
        return n.value, res.value

    def set_equilibrium(self, W):
        W = _c128(W)
        assert W.shape == self.shape
        self._check(self._L.qhfpe_set_equilibrium(self._h, _ptr(W), 0))

    # ---- response functions and spectra ----------------------------------------------------------
    def linear_response(self, n_t3):
        out = np.zeros(n_t3 + 1, dtype=np.complex128)
        sch = Schedule(LINEAR, 0, 0, 0, None, n_t3, 0)
        self._check(self._L.qhfpe_response(self._h, ctypes.byref(sch), _ptr(out)))
        return out

    def third_order_response(self, n_t1, t1_stride, t2_steps, n_t3, split_pathways=False):
        t2 = np.ascontiguousarray(t2_steps, dtype=np.int32)
        paths = 2 if split_pathways else 1
        out = np.zeros((paths, len(t2), n_t1, n_t3 + 1), dtype=np.complex128)
        sch = Schedule(THIRD_ORDER, n_t1, t1_stride, len(t2), t2.ctypes.data_as(ctypes.POINTER(ctypes.c_int)),
                       n_t3, int(bool(split_pathways)))
        self._check(self._L.qhfpe_response(self._h, ctypes.byref(sch), _ptr(out)))
        return out if split_pathways else out[0]

    def spectrum_absorption(self, R1, dt, omega):
        R1 = _c128(R1)
        om = np.ascontiguousarray(omega, dtype=np.float64)
        out = np.zeros(len(om))
        self._check(self._L.qhfpe_spectrum_absorption(self._h, _ptr(R1), len(R1), dt, _ptr(om), len(om), _ptr(out)))
        return out

    def spectrum_2d(self, R3, dt1, dt3, omega1, omega3):
        R3 = _c128(R3)
        w1 = np.ascontiguousarray(omega1, dtype=np.float64)
        w3 = np.ascontiguousarray(omega3, dtype=np.float64)
        nr = np.zeros((len(w3), len(w1)))
        re = np.zeros((len(w3), len(w1)))
        self._check(self._L.qhfpe_spectrum_2d(self._h, _ptr(R3), R3.shape[0], R3.shape[1] - 1, dt1, dt3, _ptr(w1),
                                              len(w1), _ptr(w3), len(w3), _ptr(nr), _ptr(re)))
        return nr, re, nr + re

    # ---- learned closure --------------------------------------------------------------------------
    def closure_collect(self, target_tier, stats_dev):
        """Accumulate regression statistics of `target_tier` into stats_dev (CUDA float64 tensor of
        nq*np*67 values)."""
        ptr, dev = _dev_ptr(stats_dev)
        assert dev == 1
        self._check(self._L.qhfpe_closure_collect(self._h, int(target_tier), ptr))

    def closure_load(self, weights):
        w = np.ascontiguousarray(weights, dtype=np.float32)
        self._check(self._L.qhfpe_closure_load(self._h, _ptr(w), w.size))

    def closure_state_load(self, weights):
        w = np.ascontiguousarray(weights, dtype=np.float32)
        self._check(self._L.qhfpe_closure_state_load(self._h, _ptr(w), w.size))

    def closure_state_collect(self, target_tier, X_dev, Y_dev, offset, capacity):
        """Samples of the target tier into device tensors X_dev [capacity][36 S^2 + 3], Y_dev [capacity][2 S^2]
        from sample `offset`; returns the number written."""
        n = ctypes.c_long()
        self._check(self._L.qhfpe_closure_state_collect(self._h, int(target_tier), ctypes.c_void_p(X_dev.data_ptr()),
                                                        ctypes.c_void_p(Y_dev.data_ptr()), int(offset), int(capacity),
                                                        ctypes.byref(n)))
        return n.value

    def closure_coefficients(self):
        out = np.zeros((self.model["nq"], self.model["np"], 10))
        self._check(self._L.qhfpe_closure_coefficients(self._h, _ptr(out)))
        return out

    # ---- measurement -----------------------------------------------------------------------------
    def wait_selftest(self, release, limit_ms=200):
        """Status of the bounded device wait self-test (0 = OK, 5 = ETIMEOUT)."""
        return self._L.qhfpe_wait_selftest(self._h, int(release), int(limit_ms))

    def set_persistent(self, on=True):
        """Whole runs of steps (and the response schedule's phases) in one cooperative, resident launch."""
        self._check(self._L.qhfpe_set_persistent(self._h, int(bool(on))))

    def barrier_selftest(self, withhold, limit_ms=200):
        return self._L.qhfpe_barrier_selftest(self._h, int(withhold), int(limit_ms))

    def stage_form(self):
        """1: q-window stage kernel, 0: general, -1: not yet chosen."""
        f = ctypes.c_int()
        self._check(self._L.qhfpe_stage_form(self._h, ctypes.byref(f)))
        return f.value

    def tile_rows(self):
        v = ctypes.c_int()
        self._check(self._L.qhfpe_tile_rows(self._h, ctypes.byref(v)))
        return v.value

    def kernel_timing(self, enable):
        self._check(self._L.qhfpe_kernel_timing(self._h, int(bool(enable))))

    def kernel_timing_read(self):
        n = (ctypes.c_long * 3)()
        ms = (ctypes.c_double * 3)()
        self._check(self._L.qhfpe_kernel_timing_read(self._h, n, ms, 3))
        names = ("stage", "potential", "aux")
        return {names[k]: (n[k], ms[k]) for k in range(3)}


class Batch:
    """Several Propagators advanced together (a heterogeneous batch: each Horner stage of all members is
    one fused kernel launch).  Members share np, the number of states and the precision; they may
    differ in grid, bath, depth, closure, dt and replica count.  The Propagators must outlive it."""

    def __init__(self, members):
        self.members = list(members)
        L = lib()
        self._L = L
        arr = (ctypes.c_void_p * len(self.members))(*[m._h.value for m in self.members])
        b = ctypes.c_void_p()
        s = L.qhfpe_batch_create(arr, len(self.members), ctypes.byref(b))
        if s != 0:
            raise QhfpeError(s, L.qhfpe_last_error(self.members[0]._h).decode())
        self._b = b

    def _check(self, s):
        if s != 0:
            raise QhfpeError(s, self._L.qhfpe_last_error(self.members[0]._h).decode())

    def step(self, n_steps, record_trace=False):
        """Advance every member n_steps RK4 steps; with record_trace, one [n_replicas][n_steps + 1]
        complex trace per member (as Propagator.step)."""
        if not record_trace:
            self._check(self._L.qhfpe_batch_step(self._b, n_steps, None))
            return None
        outs = [np.zeros((m.n_replicas, n_steps + 1), dtype=np.complex128) for m in self.members]
        ptrs = (ctypes.c_void_p * len(outs))(*[o.ctypes.data for o in outs])
        self._check(self._L.qhfpe_batch_step(self._b, n_steps, ptrs))
        return outs

    def tile_rows(self):
        v = ctypes.c_int()
        self._check(self._L.qhfpe_batch_tile_rows(self._b, ctypes.byref(v)))
        return v.value

    def close(self):
        if getattr(self, "_b", None):
            self._L.qhfpe_batch_destroy(self._b)
            self._b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def fp64_fma_rate(stream=None, repeats=5):
    """FP64 FMA throughput of the current device in flop/s (2 per DFMA), timed with CUDA events."""
    L = lib()
    out = ctypes.c_double()
    st = None if stream is None else ctypes.c_void_p(stream.cuda_stream)
    s = L.qhfpe_fp64_fma_rate(st, int(repeats), ctypes.byref(out))
    if s != 0:
        raise QhfpeError(s, L.qhfpe_last_error(None).decode())
    return out.value
