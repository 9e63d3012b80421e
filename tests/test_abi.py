"""Host-side checks of the C ABI that need no GPU: the library loads, exports every symbol the header
declares, and rejects invalid parameters before touching the device."""
import ctypes
import os
import re

import numpy as np
import pytest

import qhfpe_inputs as qi

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_functions():
    src = open(os.path.join(ROOT, "include", "qhfpe.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(qhfpe_[a-z0-9_]+)\s*\(", src)))


def test_library_exports_every_declared_symbol():
    import paper_1706_09590_gb300.qhfpe as q
    L = q.lib()
    declared = _declared_functions()
    assert "qhfpe_create" in declared and "qhfpe_step" in declared
    for name in declared:
        assert hasattr(L, name), name
    assert set(declared) == set(q.EXPORTED)


def _params(**over):
    import paper_1706_09590_gb300.qhfpe as q
    m = qi.harmonic_two_state(nq=8, n_p=8)
    T = qi.u_table(m)
    mu = np.ascontiguousarray(m["mu"], dtype=np.float64)
    dp = ctypes.POINTER(ctypes.c_double)
    vals = dict(n_states=2, nq=8, np=8, q_min=-8.0, q_max=8.0, p_min=-8.0, p_max=8.0,
                U_table=T.ctypes.data_as(dp), mu=mu.ctypes.data_as(dp), eta=0.5, gamma=1.0, beta=0.48,
                n_matsubara=0, high_temperature=1, use_cdelta=0, depth=2, closure=1, periodic_q=0,
                precision=0, dt=0.01, n_replicas=1)
    vals.update(over)
    p = q.Params(**{k: v for k, v in vals.items()})
    return p, (T, mu)


@pytest.mark.parametrize("over,msg", [
    (dict(n_states=0), "n_states"),
    (dict(n_states=5), "n_states"),
    (dict(np=12), "power of two"),
    (dict(np=4), "power of two"),
    (dict(np=1024), "power of two"),
    (dict(nq=0), "nq"),
    (dict(dt=0.0), "dt"),
    (dict(dt=float("nan")), "dt"),
    (dict(depth=-1), "depth"),
    (dict(n_matsubara=8, high_temperature=0), "n_matsubara"),
    (dict(n_matsubara=1), "high_temperature"),
    (dict(n_matsubara=1, high_temperature=0, closure=1), "terminator"),
    (dict(q_max=-8.0), "range"),
    (dict(n_replicas=0), "n_replicas"),
    (dict(closure=7), "closure"),
    (dict(precision=9), "precision"),
    (dict(beta=-1.0), "bath"),
])
def test_create_rejects_invalid_parameters(over, msg):
    import paper_1706_09590_gb300.qhfpe as q
    L = q.lib()
    p, keep = _params(**over)
    h = ctypes.c_void_p()
    s = L.qhfpe_create(ctypes.byref(p), None, ctypes.byref(h))
    assert s == 1, s  # EINVAL
    assert not h.value
    assert msg in L.qhfpe_last_error(None).decode()


def test_split_tf32_precision_is_reserved():
    """QHFPE_MIXED_TF32X3 is declared but not built: creation answers QHFPE_EUNSUPPORTED with a reason."""
    import paper_1706_09590_gb300.qhfpe as q
    L = q.lib()
    p, keep = _params(precision=3)
    h = ctypes.c_void_p()
    assert L.qhfpe_create(ctypes.byref(p), None, ctypes.byref(h)) == 6  # EUNSUPPORTED
    assert not h.value
    assert "TF32X3" in L.qhfpe_last_error(None).decode()


def test_create_rejects_non_finite_tables():
    import paper_1706_09590_gb300.qhfpe as q
    L = q.lib()
    p, (T, mu) = _params()
    T[0, 0, 3, 2] = np.nan
    h = ctypes.c_void_p()
    assert L.qhfpe_create(ctypes.byref(p), None, ctypes.byref(h)) == 4  # ENUMERIC


def test_create_rejects_asymmetric_dipole():
    import paper_1706_09590_gb300.qhfpe as q
    L = q.lib()
    p, (T, mu) = _params()
    mu[0, 1] = 0.3
    h = ctypes.c_void_p()
    assert L.qhfpe_create(ctypes.byref(p), None, ctypes.byref(h)) == 1


def test_null_handle_calls_fail_cleanly():
    import paper_1706_09590_gb300.qhfpe as q
    L = q.lib()
    assert L.qhfpe_step(None, 1, None) == 1
    assert L.qhfpe_destroy(None) == 1
    assert L.qhfpe_trace(None, None) == 1
    n = ctypes.c_long(-1)
    assert L.qhfpe_equilibrate_tol(None, 1.0, 1e-6, 10, ctypes.byref(n), None) == 1


def test_null_batch_and_state32_calls_fail_cleanly():
    import paper_1706_09590_gb300.qhfpe as q
    L = q.lib()
    out = ctypes.c_void_p()
    assert L.qhfpe_batch_create(None, 0, ctypes.byref(out)) == 1
    assert out.value is None
    arr = (ctypes.c_void_p * 1)(None)
    assert L.qhfpe_batch_create(arr, 1, ctypes.byref(out)) == 1  # a NULL member
    assert L.qhfpe_batch_create(arr, 0, None) == 1
    assert L.qhfpe_batch_step(None, 1, None) == 1
    rows = ctypes.c_int(-1)
    assert L.qhfpe_batch_tile_rows(None, ctypes.byref(rows)) == 1
    assert L.qhfpe_batch_destroy(None) == 1
    buf = np.zeros(4, dtype=np.complex64)
    assert L.qhfpe_set_state32(None, 0, buf.ctypes.data, 0) == 1
    assert L.qhfpe_get_state32(None, 0, buf.ctypes.data, 0) == 1
