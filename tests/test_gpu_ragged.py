"""GPU parity of the ragged persistent form (one graph-captured launch factors and
solves problems of different orders) against the oracle's per-problem
dpotrf + dpotrs on the same bytes.  Thresholds between the per-thread and
per-CTA forms and CTA sizes are varied; non-SPD problems must report LAPACK
info while every other problem matches; a plan relaunched on restored
inputs must reproduce its result bit for bit.
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
    return build_lib()


def make(count, seed, lo=2, hi=200, nrhs=4, bad=()):
    ns = bfsynth.ragged_orders(count, lo, hi, seed)
    S, offS, B, offB = bfsynth.ragged_spd(ns, nrhs, seed + 1)
    S = S.numpy()
    for b in bad:  # a negative pivot in the middle of problem b
        n = int(ns[b])
        j = n // 2
        S[int(offS[b]) + j + j * n] = -10.0 * n
    return ns.numpy(), S, offS.numpy(), B.numpy(), offB.numpy()


def check(ns, S, offS, B, offB, nrhs, Sg, Bg, info_g, oracle, bad=()):
    So, Xo, info_o = oracle.ragged_potrf_potrs(ns, S, offS, B, offB, nrhs)
    np.testing.assert_array_equal(info_g, info_o)
    for b in bad:
        assert info_o[b] == int(ns[b]) // 2 + 1
    worst_l = worst_x = 0.0
    for b, n in enumerate(ns):
        if info_o[b]:
            continue
        n = int(n)
        Lg = np.tril(Sg[offS[b]:offS[b] + n * n].reshape(n, n).T)
        Lr = np.tril(So[offS[b]:offS[b] + n * n].reshape(n, n).T)
        worst_l = max(worst_l, np.linalg.norm(Lg - Lr) / np.linalg.norm(Lr))
        xg = Bg[offB[b]:offB[b] + n * nrhs]
        xr = Xo[offB[b]:offB[b] + n * nrhs]
        worst_x = max(worst_x, np.linalg.norm(xg - xr) / np.linalg.norm(xr))
    assert worst_l <= TOL and worst_x <= TOL, (worst_l, worst_x)


@pytest.mark.parametrize("lane_max,threads", [(48, 256), (0, 256), (200, 128), (24, 512), (64, 128), (32, 64)])
def test_ragged_matches_oracle(bf, oracle, lane_max, threads):
    nrhs = 4
    bad = (3, 17, 1000)
    ns, S, offS, B, offB = make(1500, 11 + lane_max, bad=bad)
    Sg = torch.as_tensor(S).cuda()
    Bg = torch.as_tensor(B).cuda()
    plan = bf.RaggedPlan(ns, Sg, offS, Bg, offB, nrhs, lane_max=lane_max, threads=threads)
    d = plan.describe()
    assert d["big"] == int((ns > lane_max).sum())
    plan.launch()
    check(ns, S, offS, B, offB, nrhs, host(Sg), host(Bg), host(plan.info), oracle, bad)
    # relaunch the same graph on restored inputs: bit-identical result
    first_S, first_B = host(Sg).copy(), host(Bg).copy()
    Sg.copy_(torch.as_tensor(S))
    Bg.copy_(torch.as_tensor(B))
    plan.launch()
    np.testing.assert_array_equal(host(Sg), first_S)
    np.testing.assert_array_equal(host(Bg), first_B)


def test_ragged_edge_cases(bf, oracle):
    # orders 1..3, a large problem, and the largest order of the per-CTA form (256); nrhs = 1
    ns = np.array([1, 2, 3, 1, 150, 256], dtype=np.int32)
    S, offS, B, offB = bfsynth.ragged_spd(torch.as_tensor(ns), 1, 5)
    S, offS, B, offB = S.numpy(), offS.numpy(), B.numpy(), offB.numpy()
    Sg, Bg = torch.as_tensor(S).cuda(), torch.as_tensor(B).cuda()
    plan = bf.RaggedPlan(ns, Sg, offS, Bg, offB, 1, lane_max=2, threads=128)
    plan.launch()
    check(ns, S, offS, B, offB, 1, host(Sg), host(Bg), host(plan.info), oracle)


def test_ragged_arguments(bf):
    import ctypes
    out = ctypes.c_void_p()
    ns = np.array([4, 5], dtype=np.int32)
    offs = np.array([0, 16], dtype=np.int64)
    f = bf.bf_ragged_potrf_potrs_plan_create
    nsp = ns.ctypes.data_as(ctypes.c_void_p)
    op = offs.ctypes.data_as(ctypes.c_void_p)
    assert f(-1, nsp, 1, 1, op, 1, op, None, 1, 10 ** 6, 8, 256, None, ctypes.byref(out)) == -1
    assert f(2, nsp, 1, 1, op, 1, op, None, 1, 8, 8, 256, None, ctypes.byref(out)) == -10
    assert f(2, nsp, 1, 1, op, 1, op, None, 1, 10 ** 6, 8, 100, None, ctypes.byref(out)) == -12
    for nbig in (257, 400):  # above the per-CTA form's largest order and above lane_max
        big = np.array([nbig], dtype=np.int32)
        assert f(1, big.ctypes.data_as(ctypes.c_void_p), 1, 1, op, 1, op, None, 1, 10 ** 6, 8, 256, None,
                 ctypes.byref(out)) == bf.ERR_NOT_SUPPORTED


@pytest.mark.parametrize("lane_max", [0, 32, 200])
def test_ragged_odd_offsets(bf, oracle, lane_max):
    """Problems that start 8 bytes past a 16-byte boundary: the offsets are rebuilt here with a
    one-element gap before every other problem, so half of the matrices (and right-hand sides)
    start on an odd element offset.  Both per-thread and per-CTA forms, against the oracle."""
    nrhs = 4
    ns, S0, offS0, B0, offB0 = make(700, 91, bad=(5, 400))
    offS = np.zeros_like(offS0)
    offB = np.zeros_like(offB0)
    pos_s = pos_b = 1  # the first problem already starts at an odd element
    for b, n in enumerate(ns):
        n = int(n)
        offS[b], offB[b] = pos_s, pos_b
        pos_s += n * n + (b & 1)
        pos_b += n * nrhs + (b & 1)
    S = np.full(pos_s + 1, np.nan)
    B = np.full(pos_b + 1, np.nan)
    for b, n in enumerate(ns):
        n = int(n)
        S[offS[b]:offS[b] + n * n] = S0[offS0[b]:offS0[b] + n * n]
        B[offB[b]:offB[b] + n * nrhs] = B0[offB0[b]:offB0[b] + n * nrhs]
    assert (offS % 2 == 1).sum() > len(ns) // 4 and (offS % 2 == 0).sum() > len(ns) // 4
    Sg, Bg = torch.as_tensor(S).cuda(), torch.as_tensor(B).cuda()
    plan = bf.RaggedPlan(ns, Sg, offS, Bg, offB, nrhs, lane_max=lane_max, threads=128)
    plan.launch()
    Sh, Bh = host(Sg), host(Bg)
    check(ns, S, offS, B, offB, nrhs, Sh, Bh, host(plan.info), oracle, bad=(5, 400))
    # the gaps between problems are never written
    used = np.zeros(len(S), dtype=bool)
    for b, n in enumerate(ns):
        used[offS[b]:offS[b] + int(n) ** 2] = True
    assert np.isnan(Sh[~used]).all()
