"""GPU parity of the three forms at their full sizes, in the launch configuration the
benchmark times (same generators, seeds, sizes and call paths), on sampled problems that
the oracle recomputes one by one, plus properties every problem must satisfy:

* ragged: 200,000 problems, n log-uniform in [2, 200], 4 right-hand sides, one
  graph-captured persistent launch with the tuned plan settings: every info is 0; sampled
  factors and solutions match the oracle's dpotrf + dpotrs within 1e-13;
* differentiation: 65,536 problems of order 32 through the autograd Functions: sampled
  gradients match the oracle's closed form within 1e-8, the solutions within 1e-12;
* precision: 16,384 systems of order 128, cond(A) in {1e2, 1e4, 1e6}: every problem's
  backward error (computed by the oracle in binary64) is <= 1e-12; sampled solutions are
  within cond(A) * 4e-12 of the oracle's binary64 solve, and their refinement counts within 2
  of the oracle's own binary32 / binary64 run.

The helpers take the device and the library objects as arguments (the tests pass "cuda").
"""
import numpy as np
import pytest
import torch

import bfsynth
from bfhelp import host

pytestmark = pytest.mark.gpu

TOL = 1e-13


@pytest.fixture(scope="module")
def bf():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from bfhelp import build_lib
    m = build_lib()
    m.reset_table()
    return m


def rel(a, b):
    a, b = np.asarray(a).ravel(), np.asarray(b).ravel()
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def sample(count, extra=(), k=14, seed=0):
    """Sorted distinct problem indices: the first, the last, `extra`, and k drawn at random."""
    rng = np.random.default_rng(seed)
    idx = {0, count - 1, *(int(e) for e in extra), *(int(i) for i in rng.integers(0, count, k))}
    return np.array(sorted(idx), dtype=np.int64)


def ragged_full(bf, oracle, device, count=200000, nrhs=4):
    ns_t = bfsynth.ragged_orders(count, 2, 200, bfsynth.BASE_SEED + 3)
    Sg, offS_t, Bg, offB_t = bfsynth.ragged_spd(ns_t, nrhs, bfsynth.BASE_SEED + 4, device=device)
    ns, offS, offB = ns_t.numpy(), offS_t.numpy(), offB_t.numpy()
    idx = sample(count, extra=(int(np.argmax(ns)), int(np.argmin(ns))))
    sizes_s = [int(ns[q]) ** 2 for q in idx]
    sizes_b = [int(ns[q]) * nrhs for q in idx]
    # the sampled problems' inputs, read before the launch overwrites them
    S_in = np.concatenate([host(Sg[int(offS[q]):int(offS[q]) + s]) for q, s in zip(idx, sizes_s)])
    B_in = np.concatenate([host(Bg[int(offB[q]):int(offB[q]) + s]) for q, s in zip(idx, sizes_b)])
    plan = bf.RaggedPlan(ns, Sg, offS, Bg, offB, nrhs, **bf.ragged_config())
    plan.launch()
    info = host(plan.info)
    assert (info == 0).all(), np.nonzero(info)[0][:10]
    # the sampled problems as a small ragged batch of their own for the oracle
    ns_s = ns[idx].astype(np.int32)
    offS_s = np.concatenate([[0], np.cumsum(sizes_s)[:-1]]).astype(np.int64)
    offB_s = np.concatenate([[0], np.cumsum(sizes_b)[:-1]]).astype(np.int64)
    So, Xo, info_o = oracle.ragged_potrf_potrs(ns_s, S_in, offS_s, B_in, offB_s, nrhs)
    assert (info_o == 0).all()
    for t, q in enumerate(idx):
        n = int(ns[q])
        Lg = np.tril(host(Sg[int(offS[q]):int(offS[q]) + n * n]).reshape(n, n).T)
        Lr = np.tril(So[offS_s[t]:offS_s[t] + n * n].reshape(n, n).T)
        assert rel(Lg, Lr) <= TOL, (q, n)
        xg = host(Bg[int(offB[q]):int(offB[q]) + n * nrhs])
        xr = Xo[offB_s[t]:offB_s[t] + n * nrhs]
        assert rel(xg, xr) <= TOL, (q, n)


def diff_full(ag, oracle, device, batch=65536, n=32, q=16, r=8):
    Qd, J, B, W = bfsynth.diff_batch(batch, n, q, r, seed=bfsynth.BASE_SEED + 5, device=device)
    ts = [x.clone().requires_grad_(True) for x in (Qd, J, B, W)]
    loss, X, _ = ag.spd_solve_loss(*ts)
    loss.backward()
    idx = sample(batch)
    sel = torch.as_tensor(idx, device=Qd.device)
    ref = oracle.spd_solve_loss_grad(*(host(x[sel]) for x in (Qd, J, B, W)))
    assert (ref["info"] == 0).all()
    assert rel(host(X.detach()[sel]), ref["X"]) <= 1e-12
    for t, key in zip(ts, ("Qbar", "Jbar", "Bbar", "Wbar")):
        assert rel(host(t.grad[sel]), ref[key]) <= 1e-8, key


def precision_full(bf, oracle, device, batch=16384, n=128):
    A, b, kap = bfsynth.precision_batch(batch, n, (1e2, 1e4, 1e6), seed=bfsynth.BASE_SEED + 6, device=device)
    Bm = b.unsqueeze(1).contiguous()
    X = torch.empty_like(Bm)
    it = torch.empty(batch, dtype=torch.int32, device=A.device)
    info = torch.empty(batch, dtype=torch.int32, device=A.device)
    bf.dsposv(A, Bm, X=X, iter=it, info=info)
    assert (host(info) == 0).all()
    An, xn, bn, itn, kn = host(A), host(X)[:, 0, :], host(b), host(it), kap.numpy()
    eta = oracle.backward_error(An, xn, bn)  # every problem
    assert eta.max() <= 1e-12, eta.max()
    idx = sample(batch, extra=(batch // 2, batch - 2))
    L, _ = oracle.dpotrf_l(An[idx])
    x64 = oracle.dpotrs_l(L, bn[idx][:, None, :].copy(), n, 1)[:, 0, :]
    fwd = np.abs(xn[idx] - x64).max(1) / np.abs(x64).max(1)
    assert (fwd <= kn[idx] * 4e-12).all(), (fwd, kn[idx])
    _, it_o, _ = oracle.dsposv(An[idx], bn[idx], tol=1e-12, itmax=30)
    assert np.abs(itn[idx] - it_o).max() <= 2, (itn[idx], it_o)


def test_ragged_full_size_sampled(bf, oracle):
    ragged_full(bf, oracle, "cuda")


def test_spd_solve_gradient_full_size_sampled(bf, oracle):
    from paper_1902_08115_gb300 import autograd
    diff_full(autograd, oracle, "cuda")


def test_dsposv_full_size(bf, oracle):
    precision_full(bf, oracle, "cuda")
