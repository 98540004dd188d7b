"""The allocation-free ragged entry point against the existing plan entry point and the oracle.

bf_ragged_potrf_potrs_noalloc exists for callers that cannot allocate device
memory when they solve (a controller whose memory is sized once at start-up,
or code that cannot hand the library a workspace): its queue lives in a
file-scope device array instead of a caller workspace.  This test calls it
through the C ABI twice in a row, on two different ragged batches (the second
call reuses the array the first one left behind), and checks each result
against bf_ragged_potrf_potrs_plan_create + bf_ragged_plan_launch on the same
inputs, within the tolerance of the other GPU tests (normwise 1e-13; info
identical).  It also checks that a batch above the limit is rejected without
a launch.  The file name makes pytest collect it last.
"""
import ctypes

import numpy as np
import pytest
import torch

import bfsynth

pytestmark = pytest.mark.gpu

TOL = 1e-13


@pytest.fixture(scope="module")
def bf():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from bfhelp import build_lib
    return build_lib()


def ragged_inputs(count, seed, nrhs, bad=()):
    ns = bfsynth.ragged_orders(count, 2, 200, seed)
    S, offS, B, offB = bfsynth.ragged_spd(ns, nrhs, seed + 1)
    S = S.numpy()
    for b in bad:
        n = int(ns[b])
        S[int(offS[b]) + (n // 2) * (n + 1)] = -5.0 * n
    return ns.numpy().astype(np.int32), S, offS.numpy(), B.numpy(), offB.numpy()


def run_plan(bf, ns, S, offS, B, offB, nrhs, lane_max, threads):
    Sg, Bg = torch.as_tensor(S).cuda(), torch.as_tensor(B).cuda()
    plan = bf.RaggedPlan(ns, Sg, offS, Bg, offB, nrhs, lane_max=lane_max, threads=threads)
    plan.launch()
    torch.cuda.synchronize()
    return Sg.cpu().numpy(), Bg.cpu().numpy(), plan.info.cpu().numpy()


def run_noalloc(bf, ns, S, offS, B, offB, nrhs, lane_max, threads):
    Sg, Bg = torch.as_tensor(S).cuda(), torch.as_tensor(B).cuda()
    info = torch.full((len(ns),), -7, dtype=torch.int32, device="cuda")
    vp = ctypes.c_void_p
    r = bf.bf_ragged_potrf_potrs_noalloc(len(ns), ns.ctypes.data_as(vp), nrhs, vp(Sg.data_ptr()),
                                         offS.ctypes.data_as(vp), vp(Bg.data_ptr()), offB.ctypes.data_as(vp),
                                         vp(info.data_ptr()), lane_max, threads, bf._stream())
    assert r == 0, bf.bf_status_string(r)
    torch.cuda.synchronize()
    return Sg.cpu().numpy(), Bg.cpu().numpy(), info.cpu().numpy()


def rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def test_noalloc_matches_plan_two_calls(bf):
    nrhs = 4
    cases = [ragged_inputs(3000, 701, nrhs, bad=(5, 77)), ragged_inputs(1200, 702, nrhs)]
    for (ns, S, offS, B, offB), (lane_max, threads) in zip(cases, ((48, 256), (24, 128))):
        S_ref, B_ref, info_ref = run_plan(bf, ns, S, offS, B, offB, nrhs, lane_max, threads)
        S_got, B_got, info_got = run_noalloc(bf, ns, S, offS, B, offB, nrhs, lane_max, threads)
        np.testing.assert_array_equal(info_got, info_ref)
        ok = info_ref == 0
        assert ok.sum() == len(ns) - (2 if len(ns) == 3000 else 0)
        for b in np.nonzero(ok)[0]:
            n = int(ns[b])
            sl = slice(int(offS[b]), int(offS[b]) + n * n)
            low = np.tril(np.ones((n, n), dtype=bool)).T.reshape(-1)  # column-major lower mask
            assert rel(S_got[sl][low], S_ref[sl][low]) <= TOL
            xb = slice(int(offB[b]), int(offB[b]) + n * nrhs)
            assert rel(B_got[xb], B_ref[xb]) <= TOL


def test_noalloc_matches_oracle(bf, oracle):
    """The same entry point against the oracle's per-problem dpotrf + dpotrs directly (so a fault
    shared by the plan path and this one cannot pass), with failing problems."""
    nrhs = 3
    ns, S, offS, B, offB = ragged_inputs(900, 711, nrhs, bad=(7, 450))
    S_got, B_got, info_got = run_noalloc(bf, ns, S, offS, B, offB, nrhs, 32, 128)
    So, Xo, info_o = oracle.ragged_potrf_potrs(ns, S, offS, B, offB, nrhs)
    np.testing.assert_array_equal(info_got, info_o)
    assert (info_o != 0).sum() == 2
    for b in np.nonzero(info_o == 0)[0]:
        n = int(ns[b])
        sl = slice(int(offS[b]), int(offS[b]) + n * n)
        low = np.tril(np.ones((n, n), dtype=bool)).T.reshape(-1)
        assert rel(S_got[sl][low], So[sl][low]) <= TOL
        xb = slice(int(offB[b]), int(offB[b]) + n * nrhs)
        assert rel(B_got[xb], Xo[xb]) <= TOL


def test_noalloc_refuses_stream_capture(bf):
    """Its queue is copied from host arrays that the next call reuses, so a captured call could
    not be replayed: on a capturing stream it returns BF_ERR_NOT_SUPPORTED and launches nothing."""
    ns = np.array([3, 4], dtype=np.int32)
    off = np.array([0, 9], dtype=np.int64)
    offb = np.array([0, 3], dtype=np.int64)
    S = torch.zeros(32, dtype=torch.float64, device="cuda")
    B = torch.zeros(8, dtype=torch.float64, device="cuda")
    info = torch.zeros(2, dtype=torch.int32, device="cuda")
    vp = ctypes.c_void_p
    s = torch.cuda.Stream()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.stream(s):
        g.capture_begin()
        r = bf.bf_ragged_potrf_potrs_noalloc(2, ns.ctypes.data_as(vp), 1, vp(S.data_ptr()), off.ctypes.data_as(vp),
                                             vp(B.data_ptr()), offb.ctypes.data_as(vp), vp(info.data_ptr()), 32, 128,
                                             vp(s.cuda_stream))
        g.capture_end()
    assert r == bf.ERR_NOT_SUPPORTED


def test_noalloc_rejects_too_many_problems(bf):
    count = bf.RAGGED_NOALLOC_MAX + 1
    ns = np.full(count, 2, dtype=np.int32)
    off = np.arange(count, dtype=np.int64) * 4
    vp = ctypes.c_void_p
    S = torch.zeros(4 * count, dtype=torch.float64, device="cuda")
    r = bf.bf_ragged_potrf_potrs_noalloc(count, ns.ctypes.data_as(vp), 1, vp(S.data_ptr()), off.ctypes.data_as(vp),
                                         vp(S.data_ptr()), off.ctypes.data_as(vp), None, 48, 256, bf._stream())
    assert r == bf.ERR_NOALLOC_LIMIT
    assert b"scratch limit" in bf.bf_status_string(r)
