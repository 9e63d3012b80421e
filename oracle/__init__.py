"""CPU oracle for the multi-state QHFPE hot path -- TEST INFRASTRUCTURE ONLY.

Plain FP64 restatement of Ikeda & Tanimura (2017), Sec. II-III: the right-hand side of Eq. (heom) with
the linear-coupling operators and the terminator of Eq. (GMFP), classic RK4, the dipole
super-operators, the response functions of Eqs. (R1), (R3) and the spectra of Eqs. (I1), (nonreph),
(reph), (I3), (transient-absorption).  Only the tests, the smoke check and the benchmark's CPU
baseline use it; the CUDA product never imports it.

Parity pins (tests/test_oracle_pins.py): stencil moments, potential-kernel identities, trace and
Hermiticity invariants, R1(0) and dR1/dt(0) closed forms, the identical-surface closed form, the
harmonic equilibrium variances, an independent density-matrix HEOM in a vibrational basis, the
N = 0 Fokker-Planck special case, pathway additivity and the transient-absorption identity.
"""
import ctypes
import os

import numpy as np

from . import build as _build
from .spectra import absorption, two_d, transient_absorption, transient_absorption_from_corr  # noqa: F401

KINETIC, POTENTIAL, DAMPING, TIER_UP, TIER_DOWN, ALL = 1, 2, 4, 8, 16, 31
LEFT, RIGHT, COMMUTATOR = 1, 2, 3

_lib = None


class _Params(ctypes.Structure):
    _fields_ = [
        ("S", ctypes.c_int), ("nq", ctypes.c_int), ("np", ctypes.c_int),
        ("q_min", ctypes.c_double), ("q_max", ctypes.c_double),
        ("p_min", ctypes.c_double), ("p_max", ctypes.c_double),
        ("U_table", ctypes.POINTER(ctypes.c_double)), ("mu", ctypes.POINTER(ctypes.c_double)),
        ("eta", ctypes.c_double), ("gamma", ctypes.c_double), ("beta", ctypes.c_double),
        ("n_matsubara", ctypes.c_int), ("high_temperature", ctypes.c_int), ("use_cdelta", ctypes.c_int),
        ("depth", ctypes.c_int), ("closure", ctypes.c_int), ("periodic_q", ctypes.c_int),
        ("dt", ctypes.c_double), ("closure_coef", ctypes.POINTER(ctypes.c_double)),
        ("v_c2", ctypes.c_double),
    ]


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        L = ctypes.CDLL(path)
        dp = ctypes.POINTER(ctypes.c_double)
        L.oq_create.restype = ctypes.c_void_p
        L.oq_create.argtypes = [ctypes.POINTER(_Params)]
        L.oq_destroy.argtypes = [ctypes.c_void_p]
        L.oq_n_elements.argtypes = [ctypes.c_void_p]
        L.oq_n_modes.argtypes = [ctypes.c_void_p]
        L.oq_get_hierarchy.argtypes = [ctypes.c_void_p, ctypes.POINTER(ctypes.c_int)]
        L.oq_get_coefficients.argtypes = [ctypes.c_void_p, dp, dp, dp, dp]
        L.oq_rhs.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int]
        L.oq_rhs_rows.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p,
                                  ctypes.c_int]
        L.oq_step.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_long, ctypes.c_void_p]
        L.oq_trace.argtypes = [ctypes.c_void_p, ctypes.c_void_p, dp]
        L.oq_apply_dipole.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int]
        L.oq_equilibrate.argtypes = [ctypes.c_void_p, ctypes.c_long, ctypes.c_void_p, dp]
        L.oq_bath_coefficients.argtypes = [ctypes.c_double, ctypes.c_double, ctypes.c_double, ctypes.c_int,
                                           ctypes.c_int, ctypes.c_int, dp, dp, dp, dp]
        L.oq_hierarchy.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_int)]
        _lib = L
    return _lib


def num_threads():
    return lib().oq_num_threads()


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p)


class Oracle:
    """One model (grid, surfaces, bath, hierarchy) on the CPU.  States are complex128 arrays of shape
    [n_elem][S][S][nq][np] (hierarchy element, ket state, bra state, q, p)."""

    def __init__(self, model, U_table=None, periodic_q=None, closure_coef=None):
        """closure_coef: [nq][np][10] coefficients of the learned closure (closure 2), e.g. from
        oracle.closure.coefficients."""
        from qhfpe_inputs import u_table
        self.model = model
        self.T = np.ascontiguousarray(U_table if U_table is not None else u_table(model), dtype=np.float64)
        self.mu = np.ascontiguousarray(np.asarray(model["mu"], dtype=np.float64))
        per = model.get("periodic_q", 0) if periodic_q is None else periodic_q
        dp = ctypes.POINTER(ctypes.c_double)
        self._p = _Params(model["S"], model["nq"], model["np"], model["q_min"], model["q_max"],
                          model["p_min"], model["p_max"], self.T.ctypes.data_as(dp), self.mu.ctypes.data_as(dp),
                          model["eta"], model["gamma"], model["beta"], model["n_matsubara"],
                          model["high_temperature"], model["use_cdelta"], model["depth"], model["closure"],
                          int(per), model["dt"], None, float(model.get("v_c2", 0.0)))
        if closure_coef is not None:
            self._coef = np.ascontiguousarray(closure_coef, dtype=np.float64)
            assert self._coef.shape == (model["nq"], model["np"], 10)
            self._p.closure_coef = self._coef.ctypes.data_as(dp)
        self._h = lib().oq_create(ctypes.byref(self._p))
        if not self._h:
            raise ValueError("oracle rejected the model parameters")
        self.n_elem = lib().oq_n_elements(self._h)
        self.n_modes = lib().oq_n_modes(self._h)
        self.shape = (self.n_elem, model["S"], model["S"], model["nq"], model["np"])
        self.dq = (model["q_max"] - model["q_min"]) / model["nq"]
        self.dp = (model["p_max"] - model["p_min"]) / model["np"]
        self.dt = model["dt"]

    def __del__(self):
        if getattr(self, "_h", None):
            lib().oq_destroy(self._h)
            self._h = None

    def hierarchy(self):
        out = np.zeros((self.n_elem, self.n_modes), dtype=np.int32)
        lib().oq_get_hierarchy(self._h, out.ctypes.data_as(ctypes.POINTER(ctypes.c_int)))
        return out

    def coefficients(self):
        g = np.zeros(self.n_modes); r = np.zeros(self.n_modes); c = np.zeros(self.n_modes)
        cd = np.zeros(1)
        dp = ctypes.POINTER(ctypes.c_double)
        lib().oq_get_coefficients(self._h, g.ctypes.data_as(dp), r.ctypes.data_as(dp), c.ctypes.data_as(dp),
                                  cd.ctypes.data_as(dp))
        return dict(gamma=g, r=r, c=c, cdelta=float(cd[0]))

    def _check(self, W):
        W = np.ascontiguousarray(W, dtype=np.complex128)
        assert W.shape == self.shape, (W.shape, self.shape)
        return W

    def rhs(self, W, terms=ALL):
        W = self._check(W)
        out = np.empty_like(W)
        lib().oq_rhs(self._h, _ptr(W), _ptr(out), int(terms))
        return out

    def rhs_rows(self, W, rows, terms=ALL):
        """The right-hand side at selected rows only: rows = [(element, j, k, q index), ...] -> [n][np]."""
        W = self._check(W)
        R = np.ascontiguousarray(rows, dtype=np.int32).reshape(-1, 4)
        out = np.empty((len(R), self.shape[-1]), dtype=np.complex128)
        if lib().oq_rhs_rows(self._h, _ptr(W), _ptr(R), len(R), _ptr(out), int(terms)) != 0:
            raise ValueError("row index out of range")
        return out

    def step(self, W, n_steps):
        """Classic RK4; returns (W after n_steps, Tr{mu W^(0)} at steps 0..n_steps)."""
        W = self._check(W).copy()
        tr = np.zeros(2 * (n_steps + 1))
        lib().oq_step(self._h, _ptr(W), int(n_steps), _ptr(tr))
        return W, tr[0::2] + 1j * tr[1::2]

    def trace(self, W):
        W = self._check(W)
        out = np.zeros(2)
        lib().oq_trace(self._h, _ptr(W), out.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
        return complex(out[0], out[1])

    def apply_dipole(self, W, side=COMMUTATOR):
        W = self._check(W).copy()
        lib().oq_apply_dipole(self._h, _ptr(W), int(side))
        return W

    def equilibrate(self, n_steps):
        W = np.zeros(self.shape, dtype=np.complex128)
        res = np.zeros(1)
        lib().oq_equilibrate(self._h, int(n_steps), _ptr(W), res.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
        return W, float(res[0])

    # ---- response functions (Sec. III protocol) --------------------------------------------------
    def linear_response(self, W_eq, n_t):
        """R1(t_n) = (i/hbar) Tr{mu G(t_n) mu^x W_eq}, n = 0..n_t (Eq. (R1))."""
        W = self.apply_dipole(W_eq, COMMUTATOR)
        _, tr = self.step(W, n_t)
        return 1j * tr

    def first_order_distribution(self, W_eq, n_t1, t1_stride, omega):
        """W'(omega) = (i/hbar) [mu^-> F(omega) - mu^<- F(-omega)] with F(omega) = int dt1 e^{i omega t1}
        G(t1) mu^x W_eq (Sec. III, "One-dimensional spectrum"), the t1 integral by the trapezoid rule on
        t1 = a*t1_stride*dt, a < n_t1 (n_t1 >= 2).  Returns [len(omega)][n_elem][S][S][nq][np]."""
        assert n_t1 >= 2
        dt1 = t1_stride * self.dt
        wts = np.full(n_t1, dt1)
        wts[0] *= 0.5
        wts[-1] *= 0.5
        omega = np.asarray(omega, dtype=np.float64)
        Fp = np.zeros((len(omega),) + self.shape, dtype=np.complex128)
        Fm = np.zeros_like(Fp)
        X = self.apply_dipole(W_eq, COMMUTATOR)
        for a in range(n_t1):
            if a > 0:
                X, _ = self.step(X, t1_stride)
            for k, om in enumerate(omega):
                Fp[k] += wts[a] * np.exp(1j * om * a * dt1) * X
                Fm[k] += wts[a] * np.exp(-1j * om * a * dt1) * X
        return np.stack([1j * (self.apply_dipole(Fp[k], LEFT) - self.apply_dipole(Fm[k], RIGHT))
                         for k in range(len(omega))])

    def third_order_response(self, W_eq, n_t1, t1_stride, t2_steps, n_t3, first=COMMUTATOR):
        """R3(t3, t2, t1) = (i/hbar)^3 Tr{mu G(t3) mu^x G(t2) mu^x G(t1) mu^x W_eq} (Eq. (R3)) on the
        grid t1 = a*t1_stride*dt (a < n_t1), t2 in t2_steps*dt, t3 = c*dt (c <= n_t3).  `first`
        selects the first interaction: COMMUTATOR (mu^x), LEFT (mu^->, ket side) or RIGHT (-mu^<-,
        bra side); the LEFT and RIGHT results add up to the COMMUTATOR one.
        Returns complex array [len(t2_steps)][n_t1][n_t3 + 1]."""
        W = self.apply_dipole(W_eq, first)
        if first == RIGHT:
            W = -W
        out = np.zeros((len(t2_steps), n_t1, n_t3 + 1), dtype=np.complex128)
        for a in range(n_t1):
            if a > 0:
                W, _ = self.step(W, t1_stride)
            X = self.apply_dipole(W, COMMUTATOR)
            done = 0
            for b, t2 in enumerate(t2_steps):
                if t2 > done:
                    X, _ = self.step(X, t2 - done)
                    done = t2
                Y = self.apply_dipole(X, COMMUTATOR)
                _, tr = self.step(Y, n_t3)
                out[b, a] = (1j) ** 3 * tr
        return out
