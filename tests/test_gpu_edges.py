"""Degenerate sizes through the public binding: empty batches, zero orders and dimensions,
k = 0 and alpha = 0 updates, single problems.  Every call must return success and leave its
outputs exactly as BLAS/LAPACK specify (untouched, scaled, or zeroed), without launching on
empty work where nothing is defined."""
import numpy as np
import pytest
import torch

import bfsynth
from bfhelp import gpu, host

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def bf():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from bfhelp import build_lib
    m = build_lib()
    m.reset_table()
    return m


def test_empty_batches(bf):
    z = torch.empty(0, 4, 4, dtype=torch.float64, device="cuda")
    bf.dgemm("N", "N", 1.0, z, z, 1.0, z, m=4, n=4, k=4)
    bf.dtrsm("R", "L", "T", "N", 1.0, z, z, m=4, n=4)
    assert host(bf.dpotrf(z)).shape == (0,)
    bf.dsyrk("L", "N", 1.0, z, 1.0, z, n=4, k=4)
    bf.dtrmm("L", "U", "N", "N", 1.0, z, z, m=4, n=4)
    assert host(bf.dsyrk_dpotrf(z, z, n=4, k=4)).shape == (0,)
    piv, info = bf.dgetrf(z)
    assert host(info).shape == (0,)


def test_zero_dimensions_leave_outputs(bf):
    C = bfsynth.randn_batch(5, 4, 4, 4, 1, device="cuda")
    C0 = host(C).copy()
    A = bfsynth.randn_batch(5, 4, 4, 4, 2, device="cuda")
    bf.dgemm("N", "N", 1.0, A, A, 1.0, C, m=0, n=4, k=4)   # m = 0: nothing
    bf.dgemm("N", "N", 1.0, A, A, 1.0, C, m=4, n=0, k=4)   # n = 0: nothing
    bf.dgemm("N", "N", 1.0, A, A, 1.0, C, m=4, n=4, k=0)   # k = 0, beta = 1: nothing
    np.testing.assert_array_equal(host(C), C0)
    bf.dgemm("N", "N", 1.0, A, A, 2.0, C, m=4, n=4, k=0)   # k = 0: C <= beta C
    np.testing.assert_array_equal(host(C), 2.0 * C0)
    bf.dgemm("N", "N", 0.0, gpu(np.full((5, 4, 4), np.nan)), A, 0.0, C, m=4, n=4, k=4)  # alpha = beta = 0
    np.testing.assert_array_equal(host(C), np.zeros_like(C0))
    S = bfsynth.spd_batch(3, 5, 5, 3, device="cuda")
    S0 = host(S).copy()
    info = bf.dpotrf(S, n=0)                                # n = 0: info cleared, nothing else
    assert (host(info) == 0).all()
    np.testing.assert_array_equal(host(S), S0)
    B = bfsynth.randn_batch(3, 5, 2, 5, 4, device="cuda")
    B0 = host(B).copy()
    bf.dtrsm("L", "L", "N", "N", 1.0, S, B, m=5, n=0)
    bf.dtrmm("L", "L", "N", "N", 1.0, S, B, m=0, n=2)
    np.testing.assert_array_equal(host(B), B0)
    bf.dtrmm("L", "L", "N", "N", 0.0, gpu(np.full((3, 5, 5), np.nan)), B, m=5, n=2)  # alpha = 0: B <= 0
    np.testing.assert_array_equal(host(B), np.zeros_like(B0))


def test_dsyrk_k_zero_and_alpha_zero(bf):
    C = bfsynth.randn_batch(4, 6, 6, 6, 5, device="cuda")
    C0 = host(C).copy()
    low = np.tril(np.ones((6, 6), bool)).T
    bf.dsyrk("L", "N", 1.0, gpu(np.zeros((4, 1, 6))), 0.5, C, n=6, k=0)
    out = host(C)
    np.testing.assert_array_equal(out[:, low], 0.5 * C0[:, low])
    np.testing.assert_array_equal(out[:, ~low], C0[:, ~low])


def test_order_one_everywhere(bf, oracle):
    S = gpu(np.full((7, 1, 1), 4.0))
    assert (host(bf.dpotrf(S)) == 0).all()
    np.testing.assert_array_equal(host(S), np.full((7, 1, 1), 2.0))
    U = gpu(np.full((7, 1, 1), 9.0))
    bf.dpotrf(U, uplo="U")
    np.testing.assert_array_equal(host(U), np.full((7, 1, 1), 3.0))
    A = gpu(np.full((7, 1, 1), -2.0))
    piv, info = bf.dgetrf(A)
    np.testing.assert_array_equal(host(piv), np.ones((7, 1), np.int32))
    assert (host(info) == 0).all()
    Z = gpu(np.zeros((3, 1, 1)))
    piv, info = bf.dgetrf(Z)
    assert (host(info) == 1).all()  # exactly zero pivot
    X = gpu(np.full((7, 1, 1), 6.0))
    bf.dtrsm("L", "L", "N", "N", 1.0, S, X, m=1, n=1)
    np.testing.assert_array_equal(host(X), np.full((7, 1, 1), 3.0))
