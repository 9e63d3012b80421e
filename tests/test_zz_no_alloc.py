"""The allocation-free potential-term entry point against the handle-based one (GPU).

qhfpe_potential_term_static serves callers that cannot allocate device memory: code whose device
memory is a fixed budget owned by another allocator, or code that must not synchronise the device,
which cudaMalloc/cudaFree can do.  It keeps its scratch in a static device array.  Here it must give
the same -i[U, W] as qhfpe_apply_rhs(..., QHFPE_TERM_POTENTIAL) on a handle, within the FP64
right-hand-side tolerance of the other parity tests (1e-12 relative L2), on two calls in a row with
different states (the array keeps the previous call's contents; the second call must not see them),
and the CPU oracle's potential term directly.  One grid needs several chunks of hierarchy elements,
so the chunk loop and the reuse of the scratch between chunks run too.

This file is collected last on purpose.
"""
import ctypes

import numpy as np
import pytest

import qhfpe_inputs as qi

pytestmark = pytest.mark.gpu


def rel(a, b):
    return np.linalg.norm(np.ravel(a - b)) / max(np.linalg.norm(np.ravel(b)), 1e-300)


@pytest.fixture(scope="module")
def torch():
    t = pytest.importorskip("torch")
    if not t.cuda.is_available():
        pytest.skip("no CUDA device")
    return t


@pytest.mark.parametrize("kind", ["two_state", "three_state", "chunked"])
def test_static_potential_term_matches_handle(torch, kind):
    import paper_1706_09590_gb300.qhfpe as q
    if kind == "two_state":
        m = qi.photoisomerization_two_state(nq=24, n_p=32, depth=3, n_matsubara=2)
    elif kind == "three_state":
        m = qi.three_state(nq=16, n_p=64, depth=2, n_matsubara=1)
    else:
        # 256 x 256, two states: 3 elements per chunk of the 32 MiB array, 6 elements -> two chunks
        m = qi.photoisomerization_two_state(nq=256, n_p=256, depth=2, n_matsubara=1)
    T = qi.u_table(m)
    P = q.Propagator(m, T, precision="fp64")
    L = q.lib()
    stream = torch.cuda.current_stream()
    U_dev = torch.from_numpy(T).cuda()
    for seed in (101, 202):  # two calls in a row
        W = qi.random_state(m, seed=seed)
        P.set_state(W)
        ref = P.apply_rhs(0, q.TERM_POTENTIAL)
        W_dev = torch.from_numpy(W.view(np.float64)).cuda()
        out_dev = torch.full_like(W_dev, float("nan"))
        s = L.qhfpe_potential_term_static(m["S"], m["nq"], m["np"], m["p_min"], m["p_max"],
                                          ctypes.c_void_p(U_dev.data_ptr()), P.n_elem,
                                          ctypes.c_void_p(W_dev.data_ptr()), ctypes.c_void_p(out_dev.data_ptr()),
                                          ctypes.c_void_p(stream.cuda_stream))
        assert s == 0, L.qhfpe_last_error(None).decode()
        torch.cuda.synchronize()
        got = out_dev.cpu().numpy().view(np.complex128).reshape(P.shape)
        assert np.isfinite(got).all()
        assert rel(got, ref) < 1e-12
        if kind != "chunked":
            import oracle
            assert rel(got, oracle.Oracle(m).rhs(W, oracle.POTENTIAL)) < 1e-12
    P.close()


def test_static_potential_term_rejects_oversized_grids(torch):
    import paper_1706_09590_gb300.qhfpe as q
    L = q.lib()
    dummy = torch.zeros(2, dtype=torch.float64, device="cuda")
    p = ctypes.c_void_p(dummy.data_ptr())
    # 4 states on a 512 x 128 grid need 7*16*512*128 doubles > 32 MiB: rejected before any launch
    s = L.qhfpe_potential_term_static(4, 512, 128, -8.0, 8.0, p, 1, p, p, None)
    assert s == 1
    assert "32 MiB" in L.qhfpe_last_error(None).decode()
    s = L.qhfpe_potential_term_static(2, 8, 12, -8.0, 8.0, p, 1, p, p, None)
    assert s == 1
