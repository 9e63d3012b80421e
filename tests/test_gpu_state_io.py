"""Canonical state I/O through the C ABI in complex64 (qhfpe_set_state32 / qhfpe_get_state32) and
complex128, host and device buffers: widening and rounding are exact element by element, and non-finite
input is rejected."""
import numpy as np
import pytest

import qhfpe_inputs as qi

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_complex64_state_io(precision):
    import torch
    from paper_1706_09590_gb300 import Propagator, QhfpeError
    m = qi.harmonic_two_state(nq=16, n_p=32, depth=2)
    P = Propagator(m, qi.u_table(m), precision=precision, n_replicas=2)
    W = qi.random_state(m, seed=7)
    W32 = W.astype(np.complex64)
    # complex64 in: every value widened exactly
    P.set_state(W32, 1)
    assert np.array_equal(P.get_state(1), W32.astype(np.complex128))
    out32 = np.empty(P.shape, dtype=np.complex64)
    P.get_state(1, out=out32)
    assert np.array_equal(out32, W32)
    # complex64 out after steps: each value (the FP64 zeroth tier of the mixed form too) rounded once
    P.set_state(W, 0)
    P.step(3)
    ref = P.get_state(0)
    P.get_state(0, out=out32)
    assert np.array_equal(out32, ref.astype(np.complex64))
    # device buffers
    d_in = torch.from_numpy(W32).cuda()
    P.set_state(d_in, 1)
    d_out = torch.empty(P.shape, dtype=torch.complex64, device="cuda")
    P.get_state(1, out=d_out)
    assert np.array_equal(d_out.cpu().numpy(), W32)
    # device buffers 8 bytes off a 16-byte boundary take the element-wise conversion (the four-cell
    # conversion needs 16-byte aligned canonical arrays)
    big_in = torch.zeros(W32.size + 1, dtype=torch.complex64, device="cuda")
    off_in = big_in[1:].view(P.shape)
    off_in.copy_(d_in)
    assert off_in.data_ptr() % 16 == 8
    P.set_state(off_in, 1)
    big_out = torch.zeros(W32.size + 1, dtype=torch.complex64, device="cuda")
    off_out = big_out[1:].view(P.shape)
    P.get_state(1, out=off_out)
    assert np.array_equal(off_out.cpu().numpy(), W32)
    # non-finite input, at the first and the last cell too
    for idx in ((0, 0, 0, 0, 0), tuple(d - 1 for d in W32.shape)):
        bad = W32.copy()
        bad[idx] = np.inf
        with pytest.raises(QhfpeError):
            P.set_state(bad, 0)
    bad = W32.copy()
    bad[1, 0, 1, 3, 5] = np.nan
    with pytest.raises(QhfpeError):
        P.set_state(bad, 0)
    P.close()
