"""GPU parity of the mixed-precision SPD solve (binary32 factor + binary64 refinement).

For every problem the oracle recomputes, in binary64 from the GPU's solution,
the normwise backward error eta = ||b - A x|| / (||A|| ||x|| + ||b||), which
must be <= 1e-12 (the refinement target), and compares x with its own
binary64 dpotrf + dpotrs solution (forward error bounded by cond(A) * 1e-12).
Refinement counts are compared with the oracle's own binary32/binary64 run of
the same algorithm; the binary64 fallback and LAPACK info on non-SPD input are
exercised with matrices built to trigger them.
"""
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
    return build_lib()


def colmajor_batch(A_rowmajor):
    """(b, n, n) row-major symmetric/any -> column-major (b, ncols, ld) layout."""
    return np.ascontiguousarray(np.transpose(A_rowmajor, (0, 2, 1)))


@pytest.mark.parametrize("n", [128, 96, 33, 5, 256, 1, 2, 127, 129, 200])
def test_dsposv_conditioned(bf, oracle, n):
    batch = 30
    A, b, kap = bfsynth.precision_batch(batch, n, (1e2, 1e4, 1e6), seed=77 + n)
    A = colmajor_batch(A.numpy())  # symmetric: same bytes, kept explicit
    b = b.numpy()
    Bc = b[:, None, :].copy()  # (batch, 1, n): one right-hand side
    Xg, it, info = bf.dsposv(gpu(A), gpu(Bc), tol=1e-12, itmax=30)
    x = host(Xg)[:, 0, :]
    it, info = host(it), host(info)
    assert (info == 0).all()
    eta = oracle.backward_error(A, x, b)
    assert eta.max() <= 1e-12, eta.max()
    # forward error against the oracle's binary64 solve
    L, _ = oracle.dpotrf_l(A)
    x64 = oracle.dpotrs_l(L, Bc.copy(), n, 1)[:, 0, :]
    fwd = np.abs(x - x64).max(1) / np.abs(x64).max(1)
    assert (fwd <= kap.numpy() * 1e-12 * 4).all()
    # refinement counts: the oracle runs the same binary32 / binary64 algorithm
    _, it_o, info_o = oracle.dsposv(A, b, tol=1e-12, itmax=30)
    assert (it >= 0).all()
    assert np.abs(it - it_o).max() <= 2, (it, it_o)
    # condition numbers 1e2 / 1e4 / 1e6: steps do not decrease with kappa
    k = kap.numpy()
    assert it[k == 1e2].mean() <= it[k == 1e6].mean()


def test_dsposv_multiple_rhs_and_padding(bf, oracle):
    n, batch, nrhs = 40, 9, 3
    A = bfsynth.spd_batch(batch, n, n + 3, 5).numpy()
    Bm = bfsynth.randn_batch(batch, n, nrhs, n + 1, 6).numpy()
    Xg = gpu(np.full((batch, nrhs, n + 2), np.nan))
    _, it, info = bf.dsposv(gpu(A), gpu(Bm), X=Xg, n=n, nrhs=nrhs)
    X = host(Xg)
    assert (host(info) == 0).all() and (host(it) >= 0).all()
    assert np.isnan(X[:, :, n:]).all()
    for c in range(nrhs):
        eta = oracle.backward_error(A, X[:, c, :n].copy(), Bm[:, c, :n].copy())
        assert eta.max() <= 1e-12


def test_dsposv_fallback_and_failure(bf, oracle):
    n = 6
    good = np.eye(n) * 3 + 0.1
    # SPD in binary64, singular once rounded to binary32 -> binary64 fallback
    near = np.eye(n)
    near[0, 1] = near[1, 0] = 1.0 - 2e-9
    near[0, 0] = near[1, 1] = 1.0
    # indefinite -> binary64 fallback fails at column 2
    bad = np.eye(n)
    bad[1, 1] = -1.0
    A = np.stack([good, near, bad, good])
    Ac = colmajor_batch(A)
    b = np.arange(1.0, n + 1)[None].repeat(4, 0)
    Xg, it, info = bf.dsposv(gpu(Ac), gpu(b[:, None, :].copy()))
    it, info, X = host(it), host(info), host(Xg)[:, 0, :]
    assert it[0] >= 0 and it[3] >= 0
    assert it[1] == -1 and info[1] == 0
    assert it[2] == -1 and info[2] == 2
    for q in (0, 1, 3):
        assert oracle.backward_error(Ac[q:q + 1], X[q], b[q])[0] <= 1e-12


