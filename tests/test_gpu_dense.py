"""The tensor-core dense stage on its own (tusq_dense_check): y_t = U x_t for
256 vectors of 32 complex64 amplitudes through the tcgen05 path (Sec. II,
Eq. 1: a fused block of gates is one 2^k x 2^k matrix acting on groups of
2^k amplitudes), against numpy's complex128 product.

Bounds, relative to max |y|: the split modes drop the lo.lo product and the
roundings of the splits -- TF32X3 keeps about 21 significant bits per
operand (measured bound 2e-5 over a K = 64 real sum), BF16X3 about 16
(5e-4), one TF32 product about 11 (5e-3).  A signed permutation matrix is
exact in every mode up to the split of x, so it pins the operand layout
independently of the precision."""
import numpy as np
import pytest

import paper_2508_04880_b300 as T

pytestmark = pytest.mark.gpu

BOUND = {T.TC_TF32X3: 2e-5, T.TC_BF16X3: 5e-4, T.TC_TF32: 5e-3}


def _haar(rng, d=32):
    z = rng.normal(size=(d, d)) + 1j * rng.normal(size=(d, d))
    q, r = np.linalg.qr(z)
    return q * (np.diag(r) / np.abs(np.diag(r)))


def _run(mode, u, x):
    import torch
    xd = torch.from_numpy(np.ascontiguousarray(x.astype(np.complex64))).cuda()
    yd = torch.empty_like(xd)
    T.tusq_dense_check(mode, u, xd.data_ptr(), yd.data_ptr(), torch.cuda.current_stream().cuda_stream)
    return yd.cpu().numpy().astype(np.complex128)


@pytest.mark.parametrize("mode", [T.TC_TF32X3, T.TC_BF16X3, T.TC_TF32])
def test_dense_haar_matrix(mode):
    rng = np.random.default_rng(10 + mode)
    u = _haar(rng)
    x = (rng.normal(size=(256, 32)) + 1j * rng.normal(size=(256, 32))) / 8
    x = x.astype(np.complex64).astype(np.complex128)
    ref = x @ u.T
    got = _run(mode, u, x)
    err = np.abs(got - ref).max() / np.abs(ref).max()
    assert err <= BOUND[mode], (mode, err)


@pytest.mark.parametrize("mode", [T.TC_TF32X3, T.TC_BF16X3, T.TC_TF32])
def test_dense_signed_permutation(mode):
    rng = np.random.default_rng(20 + mode)
    perm = rng.permutation(32)
    u = np.zeros((32, 32), dtype=np.complex128)
    phases = np.array([1, -1, 1j, -1j])[rng.integers(0, 4, 32)]
    u[np.arange(32), perm] = phases
    x = (rng.normal(size=(256, 32)) + 1j * rng.normal(size=(256, 32))) / 8
    x = x.astype(np.complex64).astype(np.complex128)
    ref = x @ u.T
    got = _run(mode, u, x)
    err = np.abs(got - ref).max() / np.abs(ref).max()
    assert err <= BOUND[mode], (mode, err)
    # every output lands on the row the permutation sends it to
    assert np.all(np.abs(got - ref) <= 0.05 * np.abs(ref).max())
